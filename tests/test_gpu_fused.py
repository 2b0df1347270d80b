"""GPU parity of the fused one-sweep step against the FP64 oracle, and the
determinism the paper relies on (Sec. 1: cells may be solved in any order
and the result stays deterministic): the fused result does not change with
the work decomposition, and equals the plain one-thread-per-cell kernel.

Tolerances as in test_gpu_plain.py: FP64 1e-10 of the field scale; FP32
1e-4 (max) and 1e-5 (L2) relative in depth and 5e-4 / 1e-4 in u and v
(tests/gpu_util.py says why); decomposition changes are bitwise.  The
"aniso" cases use cells of 0.7 m by 1.9 m (and 1.9 by 0.7), so that a swap of
dx and dy anywhere in a kernel (the step constants, the CFL speed, the side
tallies) shows.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import assert_fp32_close, gpu_solver, oracle_params, rel_depth_err, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "basin": (lambda: I.basin_hump(64, 64, manning_n=0.03, kappa=0.0), 200),
    "basin_k": (lambda: I.basin_hump(64, 64, manning_n=0.03, kappa=0.25), 200),
    "river": (lambda: I.river(300, 70, seed=7), 300),
    "dambreak": (lambda: I.dam_break(260, 90, seed=3), 300),
    "ragged": (lambda: I.dam_break(37, 23, seed=11), 150),
    "tall": (lambda: I.dam_break(9, 140, seed=12), 100),
    # widths 62 k + 1: the last column's dissipation switch sits one column
    # beyond a strip of 62 output columns (wet up to the east boundary)
    "river125": (lambda: I.river(125, 60, seed=7), 200),
    "basin63_k": (lambda: I.basin_hump(63, 50, manning_n=0.03, kappa=0.25), 200),
    # cells of 0.7 m x 1.9 m, water through all four sides; and 1.9 m x 0.7 m with drying
    "aniso_river": (lambda: I.with_cell_size(I.open_river(150, 70, seed=7), 0.7, 1.9), 250),
    "aniso_dam": (lambda: I.with_cell_size(I.dam_break(130, 60, seed=3), 1.9, 0.7), 250),
}


def _run(case, precision, kernel, steps, dt_fixed=None, **kw):
    s = gpu_solver(case, precision, kernel, **kw)
    info, dts = s.step(steps, dt_fixed=dt_fixed, want_dt=True)
    e, u, v = s.get_state()
    s.close()
    return info, dts, e, u, v


def _oracle(oracle, case, steps):
    p = oracle_params(oracle, case)
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    ref = oracle.run(p, case["z"], e0, u0, v0, steps, nthreads=4)
    assert ref.status == 0
    return ref


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_fp64_matches_oracle(oracle, name):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    ref = _oracle(oracle, case, steps)
    info, dts, e, u, v = _run(case, swe.SWE_FP64, swe.SWE_KERNEL_FUSED, steps)
    z = case["z"]
    assert rel_err(dts, ref.dt) <= 1e-10
    assert rel_err(e - z, ref.eta - z) <= 1e-10
    assert rel_err(u, ref.u, 1e-3) <= 1e-9 and rel_err(v, ref.v, 1e-3) <= 1e-9
    assert info.clamp_volume == pytest.approx(ref.clamp_volume, rel=1e-8, abs=1e-9)
    assert np.allclose(info.bflux, ref.bflux, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_fp32_matches_oracle(oracle, name):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    ref = _oracle(oracle, case, steps)
    info, dts, e, u, v = _run(case, swe.SWE_FP32, swe.SWE_KERNEL_FUSED, steps)
    assert_fp32_close(e, u, v, ref.eta, ref.u, ref.v, case["z"])
    assert rel_err(dts, ref.dt) <= 1e-4
    # FP32 tallies: within 1e-4 of the largest side flux, and the clamp
    # within 1e-7 of the water volume (it collects depths rounded near zero)
    assert abs(info.clamp_volume - ref.clamp_volume) <= 1e-4 * ref.clamp_volume + 1e-7 * info.volume
    assert np.max(np.abs(np.asarray(info.bflux) - ref.bflux)) <= 1e-4 * max(np.max(np.abs(ref.bflux)), 1e-9)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["dambreak", "river", "ragged", "tall", "river125", "basin63_k", "aniso_river",
                                  "aniso_dam"])
def test_fused_independent_of_decomposition(name, precision):
    """Bitwise identical state for different rows-per-item, and equal to the
    plain kernel."""
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    steps = min(steps, 120)
    runs = [_run(case, precision, swe.SWE_KERNEL_FUSED, steps, seg_rows=L) for L in (0, 16, 37, 24)]
    plain = _run(case, precision, swe.SWE_KERNEL_PLAIN, steps)
    for r in runs[1:] + [plain]:
        assert np.array_equal(r[1], runs[0][1])
        for a, b in zip(r[2:], runs[0][2:]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_all_wet_pass_falls_back_where_cells_dry(precision):
    """The FP32 fused step first runs an item on the assumption that every
    cell of it is wet, and recomputes it in the general form where a check
    fails.  A channel wet everywhere at the start, whose shoals then dry,
    makes items fail the check in mid-run; the state stays bitwise equal to
    the plain kernel, with and without the per-item flags that steer the
    pass (the dry-item skip on and off), over one call and several."""
    from paper_1309_1230_gb300 import swe
    case = I.drying_shoals(300, 90)
    steps = 300
    assert np.min(case["eta"] - case["z"]) > 2e-3
    plain = _run(case, precision, swe.SWE_KERNEL_PLAIN, steps)
    h = plain[2] - case["z"]
    assert 0 < int(np.sum(h <= 1e-3)) < h.size // 10  # the shoals dried
    for L, skip in ((16, 1), (16, 0), (0, 1)):
        one = _run(case, precision, swe.SWE_KERNEL_FUSED, steps, seg_rows=L, dry_skip=skip)
        assert np.array_equal(one[1], plain[1])
        for a, b in zip(one[2:], plain[2:]):
            assert np.array_equal(a, b)
    s = gpu_solver(case, precision, swe.SWE_KERNEL_FUSED, seg_rows=16)
    d = [s.step(q, want_dt=True)[1] for q in (1, 99, 200)]
    split = s.get_state()
    s.close()
    assert np.array_equal(np.concatenate(d), plain[1])
    for a, b in zip(split, plain[2:]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_dry_skip_bitwise(precision):
    """Skipping all-dry work items (their 3x3 item neighbourhood held no wet
    cell and their other copy already agrees) leaves the state bitwise equal
    to computing every item, in one call or several, with short items so that
    most of the dry half is skipped until the front arrives."""
    from paper_1309_1230_gb300 import swe
    case = I.dam_break(400, 120, seed=21)
    steps = 160
    ref = _run(case, precision, swe.SWE_KERNEL_FUSED, steps, seg_rows=16, dry_skip=0)
    one = _run(case, precision, swe.SWE_KERNEL_FUSED, steps, seg_rows=16, dry_skip=1)
    s = gpu_solver(case, precision, swe.SWE_KERNEL_FUSED, seg_rows=16, dry_skip=1)
    d1 = s.step(40, want_dt=True)[1]
    d2 = s.step(steps - 40, want_dt=True)[1]
    split = s.get_state()
    s.close()
    assert np.array_equal(one[1], ref[1]) and np.array_equal(np.concatenate([d1, d2]), ref[1])
    for a, b, c in zip(one[2:], ref[2:], split):
        assert np.array_equal(a, b) and np.array_equal(c, b)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (3, 3), (130, 5), (5, 130), (125, 4), (124, 3)])
def test_fused_small_and_degenerate_grids(oracle, shape):
    from paper_1309_1230_gb300 import swe
    nx, ny = shape
    case = I.dam_break(nx, ny, seed=nx * 1000 + ny, n_bumps=4)
    steps = 30
    ref = _oracle(oracle, case, steps)
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        info, dts, e, u, v = _run(case, prec, swe.SWE_KERNEL_FUSED, steps)
        if prec == swe.SWE_FP32:
            assert_fp32_close(e, u, v, ref.eta, ref.u, ref.v, case["z"])
        else:
            emax, _ = rel_depth_err(e - case["z"], ref.eta - case["z"])
            assert emax <= 1e-10 and rel_err(u, ref.u, 1e-3) <= 1e-9 and rel_err(v, ref.v, 1e-3) <= 1e-9


def test_fused_lake_at_rest_bitwise():
    from paper_1309_1230_gb300 import swe
    rng = np.random.Generator(np.random.PCG64(11))
    z = I.gaussian_sum_bed(300, 90, rng, 20, (0.0, 2.0), (3.0, 10.0))
    eta = np.maximum(1.0, z)
    zero = np.zeros_like(z)
    case = dict(nx=300, ny=90, z=z, eta=eta, u=zero, v=zero, manning_n=0.03, kappa=0.25)
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        s = gpu_solver(case, prec, swe.SWE_KERNEL_FUSED)
        e0, _, _ = s.get_state()
        s.step(50)
        e, u, v = s.get_state()
        s.close()
        assert np.array_equal(e, e0) and not u.any() and not v.any()


def test_fused_per_cell_manning_field(oracle):
    from paper_1309_1230_gb300 import swe
    case = I.dam_break(200, 60, seed=21)
    rng = np.random.Generator(np.random.PCG64(5))
    case["nfield"] = 0.02 + 0.03 * rng.uniform(size=(60, 200))
    steps = 100
    p = oracle_params(oracle, case)
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    ref = oracle.run(p, case["z"], e0, u0, v0, steps, nfield=case["nfield"])
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        info, dts, e, u, v = _run(case, prec, swe.SWE_KERNEL_FUSED, steps)
        if prec == swe.SWE_FP32:
            assert_fp32_close(e, u, v, ref.eta, ref.u, ref.v, case["z"])
        else:
            emax, _ = rel_depth_err(e - case["z"], ref.eta - case["z"])
            assert emax <= 1e-10 and rel_err(u, ref.u, 1e-3) <= 1e-9 and rel_err(v, ref.v, 1e-3) <= 1e-9


def test_fused_volume_and_resume():
    """Closed basin volume is conserved; stepping 2 x 60 equals 120 steps
    bitwise; get_state/set_state/set_clock resume bitwise."""
    from paper_1309_1230_gb300 import swe
    case = I.dam_break(180, 70, seed=9)
    s = gpu_solver(case, swe.SWE_FP64, swe.SWE_KERNEL_FUSED)
    v0 = s.info().volume
    s.step(60)
    mid = s.get_state()
    mid_info = s.info()
    s.step(60)
    a = s.get_state()
    info = s.info()
    assert abs(info.volume - v0 - info.clamp_volume) <= 1e-11 * v0
    s.close()
    s2 = gpu_solver(case, swe.SWE_FP64, swe.SWE_KERNEL_FUSED)
    s2.step(120)
    b = s2.get_state()
    s2.close()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    s3 = gpu_solver(case, swe.SWE_FP64, swe.SWE_KERNEL_FUSED)
    s3.set_state(*mid)
    s3.set_clock(mid_info.step, mid_info.t)
    s3.step(60)
    c = s3.get_state()
    s3.close()
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


def test_fused_dt_replay(oracle):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES["dambreak"]
    case = build()
    ref = _oracle(oracle, case, steps)
    info, dts, e, u, v = _run(case, swe.SWE_FP32, swe.SWE_KERNEL_FUSED, steps, dt_fixed=ref.dt)
    assert np.array_equal(dts, ref.dt)
    emax, _ = rel_depth_err(e - case["z"], ref.eta - case["z"])
    assert emax <= 1e-4


def test_autotune_keeps_the_state_and_the_results():
    """The work-item autotuner times candidate heights on the live state and
    restores it: the clock does not move and later steps are bitwise those
    of a context that was never tuned."""
    from paper_1309_1230_gb300 import swe
    case = CASES["dambreak"][0]()
    tuned = gpu_solver(case, swe.SWE_FP32, swe.SWE_KERNEL_FUSED)
    tuned.step(5)
    before = tuned.info()
    chosen, table = tuned.autotune(probe_steps=3)
    after = tuned.info()
    assert chosen in table and all(ms > 0 for ms in table.values()), table
    assert (after.t, after.step, after.clamp_volume) == (before.t, before.step, before.clamp_volume)
    chosen2, table2 = tuned.autotune(probe_steps=2, rows=[16, 40])
    assert chosen2 in (16, 40) and set(table2) == {16, 40}
    tuned.step(60)
    plain = gpu_solver(case, swe.SWE_FP32, swe.SWE_KERNEL_FUSED)
    plain.step(65)
    for a, b in zip(tuned.get_state(), plain.get_state()):
        assert np.array_equal(a, b)
    assert tuned.info().t == plain.info().t
    tuned.close()
    plain.close()
    p = gpu_solver(case, swe.SWE_FP32, swe.SWE_KERNEL_PLAIN)
    with pytest.raises(swe.SweError) as ei:
        p.autotune()
    assert ei.value.status == swe.SWE_ERR_UNSUPPORTED
    p.close()
