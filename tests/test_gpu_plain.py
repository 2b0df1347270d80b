"""GPU parity of the plain step (one thread per cell, two kernels per step)
against the FP64 CPU oracle on the same seeded inputs, through the C ABI.

Tolerances.  FP64: the GPU rounds differently from the oracle (fused
multiply-adds, dt/dx pre-multiplied, rcbrt instead of pow), about 1e-16
relative per operation and a few tens of operations per cell and step, so
after a few hundred steps of a smooth flow the state agrees to ~1e-13; the
tests allow 1e-10 of the field's scale.  FP32: the target is 1e-4 relative
in depth (max |h32 - h64| / max h64) and 1e-5 in L2; u and v within 5e-4
(max) and 1e-4 (L2) of their scale (tests/gpu_util.py says why).  The "aniso"
cases use cells of 0.7 m by 1.9 m and 1.9 m by 0.7 m.
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
    "river": (lambda: I.river(256, 64, seed=7), 300),
    "dambreak": (lambda: I.dam_break(96, 64, seed=3), 300),
    "ragged": (lambda: I.dam_break(37, 23, seed=11), 150),
    "aniso_river": (lambda: I.with_cell_size(I.open_river(150, 70, seed=7), 0.7, 1.9), 250),
    "aniso_dam": (lambda: I.with_cell_size(I.dam_break(130, 60, seed=3), 1.9, 0.7), 250),
}


def _run_both(oracle, name, precision, kernel, dt_replay=False):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    p = oracle_params(oracle, case)
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    ref = oracle.run(p, case["z"], e0, u0, v0, steps, nthreads=4)
    assert ref.status == 0
    s = gpu_solver(case, precision, kernel)
    info, dts = s.step(steps, dt_fixed=ref.dt if dt_replay else None, want_dt=True)
    e, u, v = s.get_state()
    s.close()
    return case, ref, info, dts, (e, u, v)


@pytest.mark.parametrize("name", sorted(CASES))
def test_plain_fp64_matches_oracle(oracle, name):
    from paper_1309_1230_gb300 import swe
    case, ref, info, dts, (e, u, v) = _run_both(oracle, name, swe.SWE_FP64, swe.SWE_KERNEL_PLAIN)
    z = case["z"]
    assert rel_err(dts, ref.dt) <= 1e-10
    assert rel_err(e - z, ref.eta - z) <= 1e-10
    assert rel_err(u, ref.u, 1e-3) <= 1e-9 and rel_err(v, ref.v, 1e-3) <= 1e-9
    assert info.step == len(ref.dt)
    assert info.clamp_volume == pytest.approx(ref.clamp_volume, rel=1e-8, abs=1e-9)
    assert np.allclose(info.bflux, ref.bflux, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("name", sorted(CASES))
def test_plain_fp32_matches_oracle(oracle, name):
    from paper_1309_1230_gb300 import swe
    case, ref, info, dts, (e, u, v) = _run_both(oracle, name, swe.SWE_FP32, swe.SWE_KERNEL_PLAIN)
    assert_fp32_close(e, u, v, ref.eta, ref.u, ref.v, case["z"])
    assert rel_err(dts, ref.dt) <= 1e-4
    # FP32 tallies: within 1e-4 of the largest side flux, and the clamp
    # within 1e-7 of the water volume (it collects depths rounded near zero)
    assert abs(info.clamp_volume - ref.clamp_volume) <= 1e-4 * ref.clamp_volume + 1e-7 * info.volume
    assert np.max(np.abs(np.asarray(info.bflux) - ref.bflux)) <= 1e-4 * max(np.max(np.abs(ref.bflux)), 1e-9)


def test_plain_fp64_volume_conserved(oracle):
    from paper_1309_1230_gb300 import swe
    case = I.basin_hump(64, 64, manning_n=0.03, kappa=0.25)
    s = gpu_solver(case, swe.SWE_FP64, swe.SWE_KERNEL_PLAIN)
    v0 = s.info().volume
    info = s.step(200)
    assert abs(info.volume - v0) <= 1e-12 * v0
    assert info.clamp_volume == 0.0


def test_plain_lake_at_rest_bitwise():
    from paper_1309_1230_gb300 import swe
    rng = np.random.Generator(np.random.PCG64(11))
    z = I.gaussian_sum_bed(48, 40, rng, 12, (0.0, 2.0), (3.0, 10.0))
    eta = np.maximum(1.0, z)
    zero = np.zeros_like(z)
    case = dict(nx=48, ny=40, z=z, eta=eta, u=zero, v=zero, manning_n=0.03, kappa=0.25)
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        s = gpu_solver(case, prec, swe.SWE_KERNEL_PLAIN)
        e0, _, _ = s.get_state()
        s.step(50)
        e, u, v = s.get_state()
        assert np.array_equal(e, e0) and not u.any() and not v.any()
