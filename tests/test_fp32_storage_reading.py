"""The reading behind the FP32 form's tolerance at moving wet/dry fronts.

The FP32 form stores eta, u, v and z in binary32.  This test runs the FP64
oracle twice on a dam break over a bumpy dry bed (384^2 cells, 500 steps):
once in FP64 throughout, once with the state rounded to binary32 after every
step (FP64 arithmetic inside each step, so nothing but the storage format
differs).  The storage rounding alone moves the depth by more than 1e-4 of
its maximum at a handful of front cells, while the L2 difference stays near
1e-6 and the share of cells beyond 1e-4 below 1e-3.  So a max-norm bound of
1e-4 on depth is not met by any scheme that keeps its state in binary32 at a
moving front, and the FP32 form is held there to the L2 and share bounds
(its own max-norm error is bounded separately, by 1e-2).  Away from fronts
(the smooth parity cases, the 8192^2 river) the FP32 form meets 1e-4 in the
max norm.  At 2048^2 x 1000 steps (oracle/perturbation.py) the same storage
rounding moves 39 cells by up to 7.1e-4; the GPU FP32 step differs from the
oracle by 2.8e-3 at about 40 cells there.
"""
from __future__ import annotations

import numpy as np

from oracle.perturbation import depth_diff, round32
from paper_1309_1230_gb300 import inputs as I


def test_binary32_storage_alone_moves_front_cells_beyond_1e4(oracle):
    n, steps = 384, 500
    case = I.dam_break(n, n, seed=1310)
    p = oracle.Params(nx=n, ny=n, manning_n=case["manning_n"], kappa=case["kappa"])
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    base = oracle.run(p, case["z"], e0, u0, v0, steps, nthreads=4)
    assert base.status == 0
    z = round32(case["z"])
    e, u, v = oracle.prepare_state(p, z, round32(case["eta"]), case["u"], case["v"])
    for k in range(steps):
        r = oracle.run(p, z, e, u, v, 1, step0=k, nthreads=4)
        assert r.status == 0
        e, u, v = round32(r.eta), round32(r.u), round32(r.v)
    d = depth_diff(e - z, base.eta - case["z"])
    assert d["max"] > 1e-4, d          # the max norm is not a binary32 property at fronts
    assert 0 < d["cells_above_1e4"] and d["share_above_1e4"] <= 1e-3, d
    assert d["l2"] <= 1e-5, d
    # with the state rounded only once, at the start, the oracle stays within 1e-6
    e1, u1, v1 = oracle.prepare_state(p, z, round32(case["eta"]), case["u"], case["v"])
    once = oracle.run(p, z, e1, u1, v1, steps, nthreads=4)
    assert depth_diff(once.eta - z, base.eta - case["z"])["max"] <= 1e-6
