"""The no-allocation FP32 step (swe_step_plain_f32_noalloc) against the
context API's plain FP32 step, through the C ABI, on calls in a row.

The no-allocation entry point exists for callers that cannot allocate device
memory: an engine whose device memory is all handed out by its own pool, a
plug-in inside a host application that owns the device memory, or a loop
that cannot wait on the allocator.  Such a caller owns the state buffers and
the step's scratch is a static device array.  Here the caller is this test,
which allocates its input and output tensors with torch beforehand.

Both entry points run the same plain predictor and corrector kernels on the
same FP32 inputs, so the results must agree bit for bit (a tighter demand
than the 1e-4 the FP32 tests allow against the FP64 oracle).  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _params(swe, case, dir_cycle):
    return swe.make_params(case["nx"], case["ny"], manning_n=case["manning_n"], kappa=case["kappa"],
                           bc=case["bc"], q_in=case["q_in"], precision=swe.SWE_FP32,
                           kernel=swe.SWE_KERNEL_PLAIN, dir_cycle=dir_cycle)


def _setup(case):
    import torch

    from paper_1309_1230_gb300 import swe
    lib = swe.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)

    def t32(a):
        return torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()

    z = t32(case["z"])
    bufs = [[t32(case["eta"]), t32(case["u"]), t32(case["v"])]]
    bufs += [[torch.empty_like(bufs[0][0]) for _ in range(3)] for _ in range(2)]
    handle = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    ref = swe.Solver(case["nx"], case["ny"], manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"],
                     q_in=case["q_in"], precision=swe.SWE_FP32, kernel=swe.SWE_KERNEL_PLAIN)
    ref.set_bed(case["z"])
    ref.set_state(case["eta"], case["u"], case["v"])
    return swe, lib, z, bufs, handle, ref


def _noalloc(lib, p, z, src, dst, dt_fixed, dt_out, handle):
    return lib.swe_step_plain_f32_noalloc(ctypes.byref(p), z.data_ptr(), src[0].data_ptr(), src[1].data_ptr(),
                                          src[2].data_ptr(), dst[0].data_ptr(), dst[1].data_ptr(),
                                          dst[2].data_ptr(), float(dt_fixed),
                                          ctypes.byref(dt_out) if dt_out is not None else None, handle)


def _assert_same_state(dst, ref, call):
    import torch
    torch.cuda.synchronize()
    e_ref, u_ref, v_ref = ref.get_state()
    for got, want, name in zip(dst, (e_ref, u_ref, v_ref), "euv"):
        g = got.double().cpu().numpy()
        assert np.isfinite(g).all(), (call, name)
        assert np.array_equal(g, want), (call, name, float(np.max(np.abs(g - want))))


def test_no_alloc_step_matches_context_step():
    """Two calls in a row with the CFL step: state and step size bitwise equal
    to the context's plain step."""
    case = I.dam_break(300, 200, seed=17)
    swe, lib, z, bufs, handle, ref = _setup(case)
    # call 1 takes the forward/forward predictor of step 0; call 2 the
    # backward/backward one the context uses on step 1 (dir_cycle 7 starts there)
    for call, (src, dst, dir_cycle) in enumerate(((bufs[0], bufs[1], 1), (bufs[1], bufs[2], 7))):
        p = _params(swe, case, dir_cycle)
        dt = ctypes.c_double(0.0)
        assert _noalloc(lib, p, z, src, dst, 0.0, dt, handle) == swe.SWE_OK
        _, dts = ref.step(1, want_dt=True)
        assert dt.value == dts[0], (call, dt.value, dts)
        _assert_same_state(dst, ref, call)
    ref.close()


def test_no_alloc_step_fixed_dt_allocates_nothing():
    """Fixed step sizes passed by value, no dt_out: bitwise equal to the
    context's step with the same step sizes, and neither torch's allocator
    nor the device's free memory moves across the calls."""
    import torch
    case = I.river(160, 96, seed=23)
    swe, lib, z, bufs, handle, ref = _setup(case)
    dts = (0.07, 0.05, 0.06)
    src, dst = bufs[0], bufs[1]
    for call, dt_fixed in enumerate(dts):
        p = _params(swe, case, 1 if call % 2 == 0 else 7)
        if call == 1:  # the first call on the device has looked up the scratch
            torch.cuda.synchronize()
            free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        assert _noalloc(lib, p, z, src, dst, dt_fixed, None, handle) == swe.SWE_OK
        ref.step(1, dt_fixed=[dt_fixed])
        _assert_same_state(dst, ref, call)
        src, dst = dst, (bufs[2] if dst is bufs[1] else bufs[1])
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == used0
    assert torch.cuda.mem_get_info()[0] == free0
    ref.close()


def test_no_alloc_step_reports_non_finite_state():
    """With dt_out the call waits for the GPU and reports a NaN that entered
    through the input state."""
    import torch
    case = I.basin_hump(40, 36)
    swe, lib, z, bufs, handle, ref = _setup(case)
    bufs[0][0][18, 20] = float("nan")
    p = _params(swe, case, 1)
    dt = ctypes.c_double(0.0)
    assert _noalloc(lib, p, z, bufs[0], bufs[1], 0.05, dt, handle) == swe.SWE_ERR_NONFINITE
    assert dt.value == 0.05
    assert torch.isnan(bufs[1][0]).any().item()
    ref.close()


def test_no_alloc_step_rejects_overlap_and_grids_above_its_scratch():
    import torch
    case = I.basin_hump(40, 36)
    swe, lib, z, bufs, handle, ref = _setup(case)
    p = _params(swe, case, 1)
    a, b = bufs[0], bufs[1]
    row = 40 * 4
    # an output starting one row into an input, or into another output:
    # rejected before anything is queued
    for dst in ([ctypes.c_void_p(a[0].data_ptr() + row), b[1], b[2]],
                [b[0], b[1], ctypes.c_void_p(b[1].data_ptr() + row)],
                [b[0], ctypes.c_void_p(z.data_ptr() + row), b[2]]):
        ptrs = [d.value if isinstance(d, ctypes.c_void_p) else d.data_ptr() for d in dst]
        st = lib.swe_step_plain_f32_noalloc(ctypes.byref(p), z.data_ptr(), a[0].data_ptr(), a[1].data_ptr(),
                                            a[2].data_ptr(), ptrs[0], ptrs[1], ptrs[2], 0.0, None, handle)
        assert st == swe.SWE_ERR_ARG
    torch.cuda.synchronize()
    ref.close()
    big = dict(nx=1025, ny=1024, manning_n=0.03, kappa=0.0, bc=(0, 0, 0, 0), q_in=(0.0,) * 4)
    assert big["nx"] * big["ny"] > swe.SWE_NOALLOC_MAX_CELLS
    pb = _params(swe, big, 1)
    one = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = lib.swe_step_plain_f32_noalloc(ctypes.byref(pb), one, one, one, one, ctypes.c_void_p(32),
                                        ctypes.c_void_p(48), ctypes.c_void_p(64), 0.0, None, None)
    assert st == swe.SWE_ERR_ARG
