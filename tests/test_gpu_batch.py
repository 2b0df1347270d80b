"""GPU batched form: each scenario of a batch of uneven grids must equal, bit
for bit, the same scenario run alone by the single-grid fused FP32 step (the
per-cell arithmetic is shared and the CFL step is per scenario), with and
without skipping dry items; and a few scenarios are checked against the FP64
oracle at the FP32 tolerance (1e-4 relative in depth)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import assert_fp32_close, gpu_solver, oracle_params

pytestmark = pytest.mark.gpu


def _ensemble(count, seed, side=(20, 230)):
    return I.ensemble(count, seed=seed, side=side)


def _run_batch(cases, steps, **kw):
    from paper_1309_1230_gb300 import swe
    b = swe.Batch([(c["nx"], c["ny"]) for c in cases], [c["manning_n"] for c in cases], kappa=cases[0]["kappa"],
                  bc=cases[0]["bc"], q_in=cases[0]["q_in"], **kw)
    for i, c in enumerate(cases):
        b.set_bed(i, c["z"])
        b.set_state(i, c["eta"], c["u"], c["v"])
    infos = b.step(steps)
    out = [b.get_state(i) for i in range(len(cases))]
    b.close()
    return infos, out


@pytest.mark.parametrize("dry_skip", [1, 0])
def test_batch_equals_single_grid_runs(dry_skip):
    from paper_1309_1230_gb300 import swe
    cases = _ensemble(12, 99)
    steps = 60
    infos, out = _run_batch(cases, steps, dry_skip=dry_skip)
    for i, c in enumerate(cases):
        s = gpu_solver(c, swe.SWE_FP32, swe.SWE_KERNEL_FUSED)
        info = s.step(steps)
        ref = s.get_state()
        s.close()
        for a, b in zip(out[i], ref):
            assert np.array_equal(a, b), (i, c["nx"], c["ny"])
        assert infos[i].t == info.t and infos[i].dt_last == info.dt_last


def test_batch_two_calls_equal_one_call():
    cases = _ensemble(6, 5)
    _, a = _run_batch(cases, 40)
    from paper_1309_1230_gb300 import swe
    b = swe.Batch([(c["nx"], c["ny"]) for c in cases], [c["manning_n"] for c in cases], kappa=cases[0]["kappa"])
    for i, c in enumerate(cases):
        b.set_bed(i, c["z"])
        b.set_state(i, c["eta"], c["u"], c["v"])
    b.step(15)
    b.step(25)
    for i in range(len(cases)):
        for x, y in zip(b.get_state(i), a[i]):
            assert np.array_equal(x, y)
    b.close()


def test_batch_matches_oracle(oracle):
    cases = _ensemble(4, 7, side=(30, 120))
    steps = 80
    infos, out = _run_batch(cases, steps)
    for i, c in enumerate(cases):
        p = oracle_params(oracle, c)
        e0, u0, v0 = oracle.prepare_state(p, c["z"], c["eta"], c["u"], c["v"])
        ref = oracle.run(p, c["z"], e0, u0, v0, steps)
        assert_fp32_close(*out[i], ref.eta, ref.u, ref.v, c["z"])
        v0_ = oracle.volume(p, c["z"], e0)
        assert abs(infos[i].volume - v0_ - infos[i].clamp_volume) <= 1e-5 * v0_


def test_batch_on_anisotropic_cells(oracle):
    """Cells of 0.7 m by 1.9 m shared by the whole batch: every scenario
    bitwise equal to its single-grid run on the same cells, two of them
    against the FP64 oracle, and the volume budget."""
    from paper_1309_1230_gb300 import swe
    cases = [I.with_cell_size(c, 0.7, 1.9) for c in _ensemble(5, 77, side=(30, 140))]
    steps = 80
    infos, out = _run_batch(cases, steps, dx=0.7, dy=1.9)
    for i, c in enumerate(cases):
        s = gpu_solver(c, swe.SWE_FP32, swe.SWE_KERNEL_FUSED)
        info = s.step(steps)
        ref = s.get_state()
        s.close()
        for a, b in zip(out[i], ref):
            assert np.array_equal(a, b), (i, c["nx"], c["ny"])
        assert infos[i].t == info.t
    for i in (0, 3):
        c = cases[i]
        p = oracle_params(oracle, c)
        e0, u0, v0 = oracle.prepare_state(p, c["z"], c["eta"], c["u"], c["v"])
        ref = oracle.run(p, c["z"], e0, u0, v0, steps)
        assert_fp32_close(*out[i], ref.eta, ref.u, ref.v, c["z"])
        v0_ = oracle.volume(p, c["z"], e0)
        assert abs(infos[i].volume - v0_ - infos[i].clamp_volume) <= 1e-5 * v0_
        assert infos[i].clamp_volume == pytest.approx(ref.clamp_volume, rel=1e-4)


def _ritter(xi, t, h0, g=9.81):
    # Ritter's dry-bed dam break: still water ahead of the rarefaction, the
    # parabolic fan h = (2 c0 - x/t)^2 / (9 g) behind it, dry beyond the front
    c0 = np.sqrt(g * h0)
    h = np.where(xi <= -c0 * t, h0, (2.0 * c0 - xi / t) ** 2 / (9.0 * g))
    return np.where(xi >= 2.0 * c0 * t, 0.0, h)


def test_batch_dam_breaks_follow_ritter():
    """Frictionless members of a batch (flat bed, dam at Nx/2, dry ground
    ahead) against Ritter's solution along x, each at its own simulated time,
    before either wave reaches a wall: rows stay identical and the L1 depth
    error is below 5 % (the oracle's pin at a similar resolution gives 1.6 %)."""
    rng = np.random.Generator(np.random.PCG64(2024))
    cases = []
    for k in range(6):
        c = I.ensemble(1, seed=3000 + k, side=(600, 1000))[0]
        ny = int(rng.integers(4, 17))
        c.update(ny=ny, z=c["z"][:ny], eta=c["eta"][:ny], u=c["u"][:ny], v=c["v"][:ny], manning_n=0.0)
        cases.append(c)
    infos, out = _run_batch(cases, 400)
    for i, c in enumerate(cases):
        e = out[i][0]
        assert all(np.array_equal(e[0], e[j]) for j in range(1, c["ny"])), i
        t, h0, x0 = infos[i].t, c["dam_height"], c["nx"] // 2
        c0 = np.sqrt(9.81 * h0)
        assert c0 * t < x0 - 8 and 2.0 * c0 * t < c["nx"] - x0 - 8, (i, t)  # no reflection yet
        xi = (np.arange(c["nx"]) + 0.5) - x0
        he = _ritter(xi, t, h0)
        err = np.sum(np.abs(e[0] - he)) / np.sum(he)
        assert err <= 0.05, (i, c["nx"], h0, t, err)


def test_batch_autotune_keeps_states_and_results():
    """The batched autotuner rebuilds the items for each candidate height on
    the live states and restores them; later steps are bitwise those of an
    untuned batch."""
    from paper_1309_1230_gb300 import swe
    cases = _ensemble(6, 41)

    def make():
        b = swe.Batch([(c["nx"], c["ny"]) for c in cases], [c["manning_n"] for c in cases],
                      kappa=cases[0]["kappa"])
        for i, c in enumerate(cases):
            b.set_bed(i, c["z"])
            b.set_state(i, c["eta"], c["u"], c["v"])
        return b

    tuned, ref = make(), make()
    tuned.step(10, want_info=False)
    chosen, table = tuned.autotune(probe_steps=3, rows=[16, 32, 64])
    assert chosen in (16, 32, 64) and all(ms > 0 for ms in table.values())
    infos = tuned.step(30)
    rinfos = ref.step(40)
    for i in range(len(cases)):
        for a, b in zip(tuned.get_state(i), ref.get_state(i)):
            assert np.array_equal(a, b), i
        assert infos[i].t == rinfos[i].t
    tuned.close()
    ref.close()
