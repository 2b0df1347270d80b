"""The no-allocation FP32 step (swe_step_plain_f32_noalloc) against the
context API's plain FP32 step, through the C ABI, on two calls in a row.

The no-allocation entry point exists for callers that may not allocate
device memory (for example code running under CUDA-graph stream capture, or
an engine whose device memory is all in its own pool): the caller owns the
state buffers, the step's scratch is a static device array.  Here the caller
is this test, which allocates its own input and output tensors with torch.

It must agree with the existing entry point within the tolerance the other
FP32 tests use (1e-4 relative in depth and in the step size).  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import rel_depth_err, rel_err

pytestmark = pytest.mark.gpu


def _params(swe, case, dir_cycle):
    return swe.make_params(case["nx"], case["ny"], manning_n=case["manning_n"], kappa=case["kappa"],
                           bc=case["bc"], q_in=case["q_in"], precision=swe.SWE_FP32,
                           kernel=swe.SWE_KERNEL_PLAIN, dir_cycle=dir_cycle)


def test_no_alloc_step_matches_context_step():
    import torch

    from paper_1309_1230_gb300 import swe

    lib = swe.load()
    torch.cuda.set_device(0)
    case = I.dam_break(300, 200, seed=17)
    nx, ny = case["nx"], case["ny"]
    dev = torch.device("cuda", 0)

    def t32(a):
        return torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()

    z = t32(case["z"])
    a = [t32(case["eta"]), t32(case["u"]), t32(case["v"])]
    b = [torch.empty_like(a[0]) for _ in range(3)]
    c = [torch.empty_like(a[0]) for _ in range(3)]
    stream = torch.cuda.current_stream(dev)
    handle = ctypes.c_void_p(stream.cuda_stream)

    # existing entry point: the context API, plain FP32 kernels, default schedule
    ref = swe.Solver(nx, ny, manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"],
                     q_in=case["q_in"], precision=swe.SWE_FP32, kernel=swe.SWE_KERNEL_PLAIN)
    ref.set_bed(case["z"])
    ref.set_state(case["eta"], case["u"], case["v"])

    # call 1 takes the forward/forward predictor of step 0; call 2 the
    # backward/backward one the context uses on step 1 (dir_cycle 7 starts there)
    for call, (src, dst, dir_cycle) in enumerate(((a, b, 1), (b, c, 7))):
        p = _params(swe, case, dir_cycle)
        dt = ctypes.c_double(0.0)
        st = lib.swe_step_plain_f32_noalloc(ctypes.byref(p), z.data_ptr(), src[0].data_ptr(), src[1].data_ptr(),
                                            src[2].data_ptr(), dst[0].data_ptr(), dst[1].data_ptr(),
                                            dst[2].data_ptr(), 0.0, ctypes.byref(dt), handle)
        assert st == swe.SWE_OK
        torch.cuda.synchronize()
        info, dts = ref.step(1, want_dt=True)
        e_ref, u_ref, v_ref = ref.get_state()
        e, u, v = (x.double().cpu().numpy() for x in dst)
        assert rel_err(np.array([dt.value]), dts) <= 1e-4, (call, dt.value, dts)
        zz = np.asarray(case["z"], dtype=np.float32).astype(np.float64)
        emax, _ = rel_depth_err(e - zz, e_ref - zz)
        assert emax <= 1e-4, (call, emax)
        assert rel_err(u, u_ref, 1e-3) <= 1e-4 and rel_err(v, v_ref, 1e-3) <= 1e-4
        assert np.isfinite(e).all()
    ref.close()


def test_no_alloc_step_rejects_grids_above_its_scratch():
    from paper_1309_1230_gb300 import swe
    lib = swe.load()
    big = dict(nx=1025, ny=1024, manning_n=0.03, kappa=0.0, bc=(0, 0, 0, 0), q_in=(0.0,) * 4)
    assert big["nx"] * big["ny"] > swe.SWE_NOALLOC_MAX_CELLS
    p = _params(swe, big, 1)
    one = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = lib.swe_step_plain_f32_noalloc(ctypes.byref(p), one, one, one, one, ctypes.c_void_p(32),
                                        ctypes.c_void_p(48), ctypes.c_void_p(64), 0.0, None, None)
    assert st == swe.SWE_ERR_ARG
