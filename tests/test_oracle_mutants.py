"""The pins are strong enough: plant one plausible mistake at a time in a copy
of the oracle's source (a flipped sign, a swapped operand, a wrong index or
exponent, a dropped term), build it, and check that at least one pin rejects
it.  The mistakes are planted in the CPU oracle only; nothing runs on a GPU.
"""
from __future__ import annotations

import os

import pytest

from tests import test_oracle_ablations as abl
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "swe_oracle.c")

MUTANTS = {
    "y divergence sign": ("eta_n[G(i, j)] - dt * (divx + divy)", "eta_n[G(i, j)] - dt * (divx - divy)"),
    "predictor face side": ("f = (sx > 0) ? qx[G(i + 1, j)] : qx[G(i, j)];",
                            "f = (sx > 0) ? qx[G(i, j)] : qx[G(i + 1, j)];"),
    "friction exponent": ("pow(h[c], 4.0 / 3.0)", "pow(h[c], 2.0 / 3.0)"),
    "Manning n not squared": ("p->g * w->n2[c] * sqrt", "p->g * sqrt(w->n2[c]) * sqrt"),
    "pressure term over dy": ("p->g * dex / p->dx", "p->g * dex / p->dy"),
    "advection operands swapped": ("double Au = u[c] * dux / p->dx + v[c] * duy / p->dy",
                                   "double Au = v[c] * dux / p->dx + u[c] * duy / p->dy"),
    "corrector from predicted velocity": ("w->u, w->v, w->uss, w->vss", "w->us, w->vs, w->uss, w->vss"),
    "corrector friction of level n": ("w->Cs,\n             w->u, w->v, w->uss", "w->C,\n             w->u, w->v, w->uss"),
    "predictor y direction": ("momentum(p, w, dt, sx, sy,", "momentum(p, w, dt, sx, -sy,"),
    "average drops corrector": ("w->u1[c] = 0.5 * (w->us[c] + w->uss[c]);", "w->u1[c] = 0.5 * (w->us[c] + w->us[c]);"),
    "wall reflects tangential": ("case BC_WALL:   u[b] = -u[a]; v[b] = v[a]; break;",
                                 "case BC_WALL:   u[b] = u[a]; v[b] = -v[a]; break;"),
    "inflow ghost sign": ("case BC_INFLOW: u[b] = sgn * p->q_in[side]", "case BC_INFLOW: u[b] = -sgn * p->q_in[side]"),
    "outflow face closed": ("else f = qx[G(inner, j)];", "else f = 0.0;"),
    "wet/dry wall rule inverted": ("(!wet_nb && z_nb > eta_self)", "(!wet_nb && z_nb < eta_self)"),
    "dry cells keep velocity": ("if (d <= p->h_dry) { u[c] = 0.0; v[c] = 0.0; }", "if (d < 0.0) { u[c] = 0.0; v[c] = 0.0; }"),
    "dissipation sign": ("out[f][c] + p->kappa * (tx + ty)", "out[f][c] - p->kappa * (tx + ty)"),
    "dissipation across dry faces": ("if (i + 1 < nx && w->wet[c] && w->wet[G(i + 1, j)])", "if (i + 1 < nx)"),
    "switch second difference": ("fabs((hl + hr) - 2.0 * hc)", "fabs((hl + hr) - hc)"),
    "CFL y term over dx": ("(fabs(w->v[c]) + cel) / p->dy", "(fabs(w->v[c]) + cel) / p->dx"),
    "dt cap ignored": ("return dt < p->dt_max ? dt : p->dt_max;", "return dt;"),
    "clamp tally weight": ("acc[0] += 0.5 * clamp_pred + clamp_final;", "acc[0] += clamp_pred + clamp_final;"),
    "east boundary tally sign": ("acc[2] -= dt * p->dy * be;", "acc[2] += dt * p->dy * be;"),
    # face lengths of the side tallies and the cell area of the volume: only
    # cells with dx != dy (and != 1) tell these apart
    "west tally weighted by dx": ("acc[1] += dt * p->dy * bw;", "acc[1] += dt * p->dx * bw;"),
    "east tally weighted by dx": ("acc[2] -= dt * p->dy * be;", "acc[2] -= dt * p->dx * be;"),
    "south tally weighted by dy": ("acc[3] += dt * p->dx * bs;", "acc[3] += dt * p->dy * bs;"),
    "north tally weighted by dy": ("acc[4] -= dt * p->dx * bn;", "acc[4] -= dt * p->dy * bn;"),
    "volume without cell area": ("return s * p->dx * p->dy;", "return s;"),
    "volume times dx only": ("return s * p->dx * p->dy;", "return s * p->dx;"),
    "clamp tally without cell area": ("const double cell_area = p->dx * p->dy;", "const double cell_area = 1.0;"),
    # the ablation forms
    "explicit friction sign": ("(u_n[c] - dt * Au) - dt * C[c] * u[c];", "(u_n[c] - dt * Au) + dt * C[c] * u[c];"),
    "explicit friction on level-n velocity": ("(u_n[c] - dt * Au) - dt * C[c] * u[c];",
                                              "(u_n[c] - dt * Au) - dt * C[c] * u_n[c];"),
    "TVD face term difference of coefficients": ("return (ga + gb) * d;", "return (ga - gb) * d;"),
    "TVD limiter ratio of the wrong cell": ("double rmb = tvd_ratio(d * dp, d * d);", "double rmb = tvd_ratio(d * dp, dp * dp);"),
}

PIN_CALLS = [
    (pins.test_mass_conservation_closed_basin, dict(kappa=0.25)),
    (pins.test_volume_budget_open_boundaries, {}),
    (pins.test_volume_budget_with_drying, {}),
    (pins.test_flat_lake_volume_closed_form, {}),
    (pins.test_volume_budget_anisotropic_cells_all_sides_open, {}),
    (pins.test_volume_budget_anisotropic_cells_with_drying, {}),
    (pins.test_lake_at_rest, dict(islands=True, kappa=0.25)),
    (pins.test_lake_at_rest, dict(islands=False, kappa=0.0)),
    (pins.test_reduces_to_separate_1d_code, dict(case="dambreak")),
    (pins.test_reduces_to_separate_1d_code, dict(case="river")),
    (pins.test_linear_limit_is_lax_wendroff, {}),
    (pins.test_mirror_and_transpose_symmetry, {}),
    (pins.test_cfl_dt_brute_force, {}),
    (pins.test_prepare_state_normalises_and_rejects, {}),
    (pins.test_stoker_wet_dam_break, {}),
    (pins.test_ritter_dry_dam_break, {}),
    (pins.test_seiche_period_matches_sqrt_gh, {}),
    (pins.test_uniform_flow_friction_recursion_and_manning, {}),
    (pins.test_degenerate_grids_run, {}),
    (abl.test_friction_treatments_converge_to_the_decay_closed_form, {}),
    (abl.test_tvd_term_keeps_the_dam_break_total_variation, {}),
    (abl.test_tvd_term_mirror_and_transpose_symmetry, {}),
    (abl.test_ablations_conserve_mass_and_keep_a_lake_at_rest, dict(friction=1, dissipation=1)),
]


def _first_failing_pin(lib):
    for fn, kw in PIN_CALLS:
        try:
            fn(lib, **kw)
        except (AssertionError, ValueError, FloatingPointError):
            return fn.__name__
    return None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(oracle, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    # the forward step comes first in the file; the adjoint's recompute of it
    # repeats a few lines, which stay correct
    assert src.count(old) >= 1, f"mutation site missing: {old!r}"
    mutated = tmp_path / "swe_oracle_mutant.c"
    mutated.write_text(src.replace(old, new, 1))
    so = oracle.compile_source(str(mutated), str(tmp_path / "libmutant.so"))
    lib = oracle.OracleLib(so)
    assert _first_failing_pin(lib) is not None, f"no pin rejects the mistake '{name}'"


def test_unmodified_oracle_passes_every_pin(oracle):
    assert _first_failing_pin(oracle._default()) is None
