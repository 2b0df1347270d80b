"""Every predictor direction schedule (dir_cycle, Sec. 1's MacCormack with
one-sided differences: the predictor differences in one direction per axis,
the corrector in the other).  Bit 0 alternates the directions every step,
bits 1 and 2 start x and y backward, so the schedules 2 to 5 run the fused
kernels whose x and y predictors point in opposite directions.

* the fused step equals the plain one-thread-per-cell step bit for bit, step
  sizes included, in FP32 and FP64, with open boundaries and with drying;
* the FP64 fused step matches the FP64 oracle run with the same schedule.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import gpu_solver, oracle_params, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "river": lambda: I.river(150, 70, seed=7),
    "dambreak": lambda: I.dam_break(130, 60, seed=3),
}
STEPS = 60


def _run(case, precision, kernel, dir_cycle):
    s = gpu_solver(case, precision, kernel, dir_cycle=dir_cycle)
    _, dts = s.step(STEPS, want_dt=True)
    state = s.get_state()
    s.close()
    return dts, state


@pytest.mark.parametrize("dir_cycle", [0, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_equals_plain_for_every_schedule(name, precision, dir_cycle):
    from paper_1309_1230_gb300 import swe
    case = CASES[name]()
    fd, fs = _run(case, precision, swe.SWE_KERNEL_FUSED, dir_cycle)
    pd, ps = _run(case, precision, swe.SWE_KERNEL_PLAIN, dir_cycle)
    assert np.array_equal(fd, pd)
    for a, b in zip(fs, ps):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dir_cycle", [2, 3, 5, 6])
def test_fused_fp64_matches_oracle_for_mixed_schedules(oracle, dir_cycle):
    from paper_1309_1230_gb300 import swe
    case = CASES["river"]()
    p = oracle_params(oracle, case, dir_cycle=dir_cycle)
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    ref = oracle.run(p, case["z"], e0, u0, v0, STEPS, nthreads=4)
    assert ref.status == 0
    dts, (e, u, v) = _run(case, swe.SWE_FP64, swe.SWE_KERNEL_FUSED, dir_cycle)
    z = case["z"]
    # the tolerances of the other FP64 parity tests (tests/test_gpu_fused.py)
    assert rel_err(dts, ref.dt) <= 1e-10
    assert rel_err(e - z, ref.eta - z) <= 1e-10
    assert rel_err(u, ref.u, 1e-3) <= 1e-9 and rel_err(v, ref.v, 1e-3) <= 1e-9
