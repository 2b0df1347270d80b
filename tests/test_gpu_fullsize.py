"""Parity at the full workload sizes, in the launch configuration bench.py
times (fused kernel, automatic work plan).

* Dam break 2048^2, 1000 steps: the FP32 and FP64 GPU steps against the FP64
  oracle over the whole grid (the oracle runs on all host cores), with the
  CFL step and with the oracle's step sizes replayed.  FP64 agrees to 1e-9
  (measured ~2e-15).  FP32: at the moving wet/dry fronts the max-norm error
  is 2.8e-3 of max depth at ~40 of 4.2 M cells after 1000 steps.  Storing the
  state in binary32 is enough to cause it: the FP64 oracle with its state
  rounded to binary32 after every step moves 39 cells by up to 7.1e-4
  (oracle/perturbation.py; tests/test_fp32_storage_reading.py shows the same
  at 384^2 on the CPU), while a one-time rounding of its input moves nothing
  beyond 1e-7.  So the FP32 run is bounded by the relative L2 error
  (measured 2e-6 to 4e-6), the share of cells beyond 1e-4 (measured
  < 0.02 %) and a max of 1e-2.
* River 8192^2 (the benchmark grid), its full 500 steps: the FP32 GPU step
  against the FP64 GPU step (the fused sweep in FP64, which the tests above
  and the other parity files hold to 1e-10 of the oracle) over the whole
  grid, with the CFL step of each: step sizes within 1e-5, depth within 1e-4
  (max) and 1e-5 (L2), u and v within 5e-4 / 1e-4 of their scale.
* River 8192^2: the FP32 GPU step against the oracle on
  crops around sample points, interior, boundaries and corners, with a fixed
  step size.  A cell after K steps depends on cells at most 2 K away, so a
  crop margin of 2 K + 2 cells on its cut sides makes the crop's answer exact
  in its middle.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import assert_fp32_close, fp32_errors, gpu_solver, oracle_params, rel_depth_err

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def dambreak_ref(oracle):
    case = I.dam_break(2048, 2048)
    p = oracle_params(oracle, case)
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    ref = oracle.run(p, case["z"], e0, u0, v0, 1000, nthreads=THREADS)
    assert ref.status == 0
    return case, ref


@pytest.mark.parametrize("precision,replay", [(1, False), (1, True), (0, False)])
def test_dambreak_2048_1000_steps(dambreak_ref, precision, replay, record_property):
    from paper_1309_1230_gb300 import swe
    case, ref = dambreak_ref
    s = gpu_solver(case, precision, swe.SWE_KERNEL_FUSED)
    info, dts = s.step(1000, dt_fixed=ref.dt if replay else None, want_dt=True)
    e, u, v = s.get_state()
    s.close()
    emax, el2 = rel_depth_err(e - case["z"], ref.eta - case["z"])
    record_property("depth_rel_max", emax)
    record_property("depth_rel_l2", el2)
    print(f"dam break 2048^2 x 1000, precision {precision}, replay {replay}: max {emax:.3e} L2 {el2:.3e}")
    assert np.isfinite(e).all()
    if precision == swe.SWE_FP64:
        assert emax <= 1e-9, (emax, el2)
        return
    href = ref.eta - case["z"]
    share = float(np.mean(np.abs((e - case["z"]) - href) > 1e-4 * href.max()))
    record_property("share_above_1e-4", share)
    err = fp32_errors(e, u, v, ref.eta, ref.u, ref.v, case["z"])
    print("  FP32 errors (max, L2) of h, u, v:", err)
    assert el2 <= 1e-5, el2
    assert share <= 1e-3, share
    assert emax <= 1e-2, emax


def test_river_8192_sampled_crops(oracle):
    from paper_1309_1230_gb300 import swe
    case = I.river(8192, 8192)
    K, dt = 8, 0.04
    s = gpu_solver(case, swe.SWE_FP32, swe.SWE_KERNEL_FUSED)
    s.step(K, dt_fixed=np.full(K, dt))
    e, u, v = s.get_state()
    s.close()
    M = 2 * K + 2
    W = 64
    n = 8192
    # (x0, y0) of the W x W checked window; crops extend M beyond it where the grid goes on
    samples = [(4064, 4064), (0, 3000), (n - W, 5000), (0, 0), (n - W, n - W), (2500, n - W)]
    for x0, y0 in samples:
        cx0, cy0 = max(0, x0 - M), max(0, y0 - M)
        cx1, cy1 = min(n, x0 + W + M), min(n, y0 + W + M)
        sl = (slice(cy0, cy1), slice(cx0, cx1))
        # the crop keeps the true boundary condition on sides that are domain sides
        bc = (case["bc"][0] if cx0 == 0 else 2, case["bc"][1] if cx1 == n else 2,
              case["bc"][2] if cy0 == 0 else 2, case["bc"][3] if cy1 == n else 2)
        q = (case["q_in"][0] if cx0 == 0 else 0.0, 0.0, 0.0, 0.0)
        p = oracle.Params(nx=cx1 - cx0, ny=cy1 - cy0, manning_n=case["manning_n"], kappa=case["kappa"], bc=bc, q_in=q)
        z = case["z"][sl]
        e0, u0, v0 = oracle.prepare_state(p, z, case["eta"][sl], case["u"][sl], case["v"][sl])
        r = oracle.run(p, z, e0, u0, v0, K, dt_fixed=np.full(K, dt), nthreads=THREADS)
        assert r.status == 0
        w = (slice(y0 - cy0, y0 - cy0 + W), slice(x0 - cx0, x0 - cx0 + W))
        hg = e[y0:y0 + W, x0:x0 + W] - case["z"][y0:y0 + W, x0:x0 + W]
        hr = r.eta[w] - z[w]
        emax, _ = rel_depth_err(hg, hr)
        assert emax <= 1e-4, ((x0, y0), emax)
        assert np.max(np.abs(u[y0:y0 + W, x0:x0 + W] - r.u[w])) <= 1e-4 * max(1.0, np.max(np.abs(r.u[w])))


def test_river_8192_500_steps_fp32_against_fp64(record_property):
    from paper_1309_1230_gb300 import swe
    case = I.river(8192, 8192)
    res = {}
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        s = gpu_solver(case, prec, swe.SWE_KERNEL_FUSED)
        info, dts = s.step(500, want_dt=True)
        res[prec] = (dts, s.get_state(), info)
        s.close()
    d64, (e64, u64, v64), i64 = res[swe.SWE_FP64]
    d32, (e32, u32, v32), i32 = res[swe.SWE_FP32]
    del res
    assert np.isfinite(e32).all() and np.isfinite(u32).all() and np.isfinite(v32).all()
    assert float(np.max(np.abs(d32 - d64) / d64)) <= 1e-5
    err = fp32_errors(e32, u32, v32, e64, u64, v64, case["z"])
    for f in "huv":
        record_property(f"{f}_rel_max", err[f][0])
        record_property(f"{f}_rel_l2", err[f][1])
    print("river 8192^2 x 500, FP32 against FP64:", err)
    assert_fp32_close(e32, u32, v32, e64, u64, v64, case["z"])
    assert np.max(np.abs(np.asarray(i32.bflux) - i64.bflux)) <= 1e-4 * np.max(np.abs(i64.bflux))
