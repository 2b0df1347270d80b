"""Failure statuses of the C ABI, each made on the host or with a short bounded
wait, never by faulting, trapping or hanging the GPU:

* SWE_ERR_NONFINITE: a valid state stepped with a step size so large that the
  arithmetic overflows (the paper reports NaNs in one of its Fortran runs,
  Sec. 4);
* SWE_ERR_NEGDEPTH: an initial elevation below the bed by more than 1e-12 m
  (the drying the paper's code lacked, Sec. 6.2), through the host and the
  device set-state calls; swe_step then answers SWE_ERR_STATE;
* SWE_ERR_TIMEOUT: the batched kernel's grid barrier with a 20 ms limit and
  one CTA that withholds its arrival (the test hook of swe_params.reserved);
  the other CTAs' waits run out and the kernel returns.

After each status the context (or batch) keeps accepting calls: a state set
again steps bit for bit like a new context's.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import gpu_solver

pytestmark = pytest.mark.gpu


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kernel", [0, 1, 3])  # fused, plain, paper layout with the GPU step size
def test_overflowing_step_reports_non_finite_and_the_context_recovers(precision, kernel):
    from paper_1309_1230_gb300 import swe
    case = I.basin_hump(70, 50, manning_n=0.03, kappa=0.25)
    s = gpu_solver(case, precision, kernel)
    with pytest.raises(swe.SweError) as ei:
        s.step(2, dt_fixed=[1e300, 1e300])
    assert ei.value.status == swe.SWE_ERR_NONFINITE
    info = s.info()
    assert info.flags & swe.SWE_FLAG_NONFINITE and info.step == 2
    e, _, _ = s.get_state()
    assert not np.isfinite(e).all()
    s.set_state(case["eta"], case["u"], case["v"])
    s.set_clock(0, 0.0)
    s.step(30)
    fresh = gpu_solver(case, precision, kernel)
    fresh.step(30)
    assert _same(s.get_state(), fresh.get_state())
    assert s.info().flags == 0
    s.close()
    fresh.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_negative_depth_is_rejected_through_host_and_device_calls(precision):
    import torch

    from paper_1309_1230_gb300 import swe
    case = I.dam_break(90, 40, seed=5)
    z = case["z"]
    s = gpu_solver(case, precision, swe.SWE_KERNEL_FUSED)
    bad = case["eta"].copy()
    bad[10, 70] = z[10, 70] - 1e-6
    with pytest.raises(swe.SweError) as ei:
        s.set_state(bad, case["u"], case["v"])
    assert ei.value.status == swe.SWE_ERR_NEGDEPTH
    with pytest.raises(swe.SweError) as ei:
        s.step(1)
    assert ei.value.status == swe.SWE_ERR_STATE
    # the device call, in the context's real type
    dt = torch.float64 if precision == swe.SWE_FP64 else torch.float32
    dev = torch.device("cuda", 0)
    zt = torch.tensor(z, dtype=dt, device=dev)
    et = torch.tensor(case["eta"], dtype=dt, device=dev)
    et[10, 70] = zt[10, 70] - 1e-3
    zero = torch.zeros_like(et)
    with pytest.raises(swe.SweError) as ei:
        s.set_state_device(et, zero, zero)
    assert ei.value.status == swe.SWE_ERR_NEGDEPTH
    with pytest.raises(swe.SweError) as ei:
        s.step(1)
    assert ei.value.status == swe.SWE_ERR_STATE
    # a negative depth within 1e-12 m is clamped to a dry cell, not rejected
    tiny = case["eta"].copy()
    tiny[10, 70] = z[10, 70] - 1e-13
    s.set_state(tiny, case["u"], case["v"])
    e, _, _ = s.get_state()
    assert e[10, 70] == (z[10, 70] if precision == swe.SWE_FP64 else np.float32(z[10, 70]))
    # a valid state steps like a new context
    s.set_state(case["eta"], case["u"], case["v"])
    s.step(25)
    fresh = gpu_solver(case, precision, swe.SWE_KERNEL_FUSED)
    fresh.step(25)
    assert _same(s.get_state(), fresh.get_state())
    s.close()
    fresh.close()


def _batch(cases, **kw):
    from paper_1309_1230_gb300 import swe
    b = swe.Batch([(c["nx"], c["ny"]) for c in cases], [c["manning_n"] for c in cases], kappa=cases[0]["kappa"], **kw)
    for i, c in enumerate(cases):
        b.set_bed(i, c["z"])
        b.set_state(i, c["eta"], c["u"], c["v"])
    return b


def test_batch_barrier_timeout_is_reported_and_the_batch_recovers():
    from paper_1309_1230_gb300 import swe
    cases = I.ensemble(6, seed=5, side=(40, 120))
    b = _batch(cases, reserved=(20000, 1, 0, 0))  # 20 ms limit; CTA 0 withholds its first arrival
    with pytest.raises(swe.SweError) as ei:
        b.step(10)
    assert ei.value.status == swe.SWE_ERR_TIMEOUT
    # the hook acted on that call only: set the states again and step (an
    # even step count keeps the direction parity of a new batch)
    for i, c in enumerate(cases):
        b.set_state(i, c["eta"], c["u"], c["v"])
    infos = b.step(10)
    assert all(i.flags == 0 for i in infos)
    fresh = _batch(cases)
    fresh.step(10)
    for i in range(len(cases)):
        assert _same(b.get_state(i), fresh.get_state(i)), i
    b.close()
    fresh.close()


def test_batch_rejects_bad_test_hook_values():
    from paper_1309_1230_gb300 import swe
    cases = I.ensemble(2, seed=5, side=(40, 60))
    for res in ((-1, 0, 0, 0), (10000001, 0, 0, 0), (0, -2, 0, 0)):
        with pytest.raises(swe.SweError) as ei:
            _batch(cases, reserved=res)
        assert ei.value.status == swe.SWE_ERR_ARG
