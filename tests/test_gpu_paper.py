"""The paper's own GPU layout of the step (Sec. 3.1: one kernel per sub-step,
intermediates in global memory, the step size computed on the host from a
device-to-host copy of the state every step), kept beside the fused sweep for
measurement.  Its per-cell arithmetic is shared with the other kernels, so:

* with the step sizes replayed, its state equals the plain step's bit for bit;
* with the step size reduced on the GPU (SWE_KERNEL_PAPER_DEVDT) it equals the
  plain step bit for bit without replay (a maximum does not depend on order);
* with the host step size, the step sizes agree with the GPU's to rounding
  (FP64 on the host from the stored state; FP32 or FP64 on the GPU) and the
  states within the FP32 tolerance of the other tests.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import gpu_solver, rel_depth_err

pytestmark = pytest.mark.gpu

CASES = {
    "dambreak": (lambda: I.dam_break(260, 90, seed=3), 80),
    # sizes that are not multiples of the 16 x 16 blocks, and thin grids
    "ragged": (lambda: I.dam_break(37, 23, seed=11), 60),
    "thin": (lambda: I.river(5, 70, seed=2), 60),
    "river": (lambda: I.river(300, 70, seed=7), 80),
    "basin_k": (lambda: I.basin_hump(64, 64, manning_n=0.03, kappa=0.25), 60),
    "aniso_river": (lambda: I.with_cell_size(I.open_river(150, 70, seed=7), 0.7, 1.9), 60),
}


def _run(case, precision, kernel, steps, dt_fixed=None, calls=1):
    s = gpu_solver(case, precision, kernel)
    dts = []
    per = steps // calls
    for q in range(calls):
        n = per if q < calls - 1 else steps - per * (calls - 1)
        fixed = None if dt_fixed is None else dt_fixed[q * per:q * per + n]
        info, d = s.step(n, dt_fixed=fixed, want_dt=True)
        dts.append(d)
    e, u, v = s.get_state()
    info = s.info()
    s.close()
    return np.concatenate(dts), (e, u, v), info


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_paper_layout_bitwise_with_the_same_step_sizes(name, precision):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    dts, plain, pinfo = _run(case, precision, swe.SWE_KERNEL_PLAIN, steps)
    _, replay, _ = _run(case, precision, swe.SWE_KERNEL_PAPER, steps, dt_fixed=dts)
    ddts, devdt, dinfo = _run(case, precision, swe.SWE_KERNEL_PAPER_DEVDT, steps, calls=2)
    # the 16 x 16 shared-memory design (Sec. 3.2), with replayed and GPU step sizes
    _, sreplay, _ = _run(case, precision, swe.SWE_KERNEL_PAPER_SHARED, steps, dt_fixed=dts)
    sdts, sdevdt, _ = _run(case, precision, swe.SWE_KERNEL_PAPER_SHARED_DEVDT, steps, calls=3)
    assert np.array_equal(ddts, dts) and np.array_equal(sdts, dts)
    for a, b, c, d, f in zip(replay, devdt, plain, sreplay, sdevdt):
        assert np.array_equal(a, c) and np.array_equal(b, c)
        assert np.array_equal(d, c) and np.array_equal(f, c)
    assert dinfo.t == pinfo.t
    # tallies are FP64 sums whose order differs between the layouts
    assert dinfo.clamp_volume == pytest.approx(pinfo.clamp_volume, rel=1e-9, abs=1e-9)
    assert np.allclose(dinfo.bflux, pinfo.bflux, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shared", [False, True])
def test_paper_layout_host_step_size(precision, shared):
    from paper_1309_1230_gb300 import swe
    case = I.dam_break(260, 90, seed=3)
    steps = 60
    dts, plain, _ = _run(case, precision, swe.SWE_KERNEL_PLAIN, steps)
    kern = swe.SWE_KERNEL_PAPER_SHARED if shared else swe.SWE_KERNEL_PAPER
    hdts, host, info = _run(case, precision, kern, steps, calls=3)
    assert np.max(np.abs(hdts - dts) / dts) <= (1e-12 if precision == swe.SWE_FP64 else 1e-6)
    emax, _ = rel_depth_err(host[0] - case["z"], plain[0] - case["z"])
    assert emax <= (1e-10 if precision == swe.SWE_FP64 else 1e-4), emax
    assert info.t == pytest.approx(float(np.sum(hdts)), rel=1e-12)
    assert np.isfinite(host[0]).all()
