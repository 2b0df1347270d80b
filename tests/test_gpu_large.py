"""A grid above 2^31 cells (46341 x 46341, FP32, about 110 GB on the device):
the fused step's addressing, work plan, tensor maps and reductions beyond
32-bit cell counts.  The state is built on the host in FP32 and set through
the device-pointer calls; after three steps with a fixed step size, windows
at the corners, an edge and the interior are checked against the FP64 oracle
run on crops around them (a cell after K steps depends on cells at most 2K
away, so a margin of 2K + 2 makes a crop's answer exact in its middle).
Skipped where the device or the host lacks the memory."""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import rel_depth_err

pytestmark = pytest.mark.gpu

N = 46341  # N * N > 2^31


def _host_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def test_grid_above_two_to_the_31_cells(oracle):
    import torch

    from paper_1309_1230_gb300 import swe
    assert N * N > 2 ** 31
    if torch.cuda.get_device_properties(0).total_memory < 150e9 or _host_gb() < 80:
        pytest.skip("needs ~110 GB of device memory and ~40 GB of host memory")
    case = I.large_river(N, N)
    dev = torch.device("cuda", 0)
    K, dt = 3, 0.04
    s = swe.Solver(N, N, manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"], q_in=case["q_in"],
                   precision=swe.SWE_FP32)
    t = {k: torch.from_numpy(case[k]).to(dev) for k in ("z", "eta", "u", "v")}
    s.set_bed_device(t["z"])
    s.set_state_device(t["eta"], t["u"], t["v"])
    info, dts = s.step(K, dt_fixed=np.full(K, dt), want_dt=True)
    s.get_state_device(t["eta"], t["u"], t["v"])
    assert bool(torch.isfinite(t["eta"]).all()) and bool(torch.isfinite(t["u"]).all())
    assert info.step == K and np.all(dts == dt)
    s.close()
    M, W = 2 * K + 2, 48
    samples = [(0, 0), (N - W, N - W), (0, N // 2), (N - W, 7), (N // 2 + 11, N // 3), (30001, N - W)]
    for x0, y0 in samples:
        cx0, cy0 = max(0, x0 - M), max(0, y0 - M)
        cx1, cy1 = min(N, x0 + W + M), min(N, y0 + W + M)
        sl = (slice(cy0, cy1), slice(cx0, cx1))
        bc = (case["bc"][0] if cx0 == 0 else 2, case["bc"][1] if cx1 == N else 2,
              case["bc"][2] if cy0 == 0 else 2, case["bc"][3] if cy1 == N else 2)
        q = (case["q_in"][0] if cx0 == 0 else 0.0, 0.0, 0.0, 0.0)
        p = oracle.Params(nx=cx1 - cx0, ny=cy1 - cy0, manning_n=case["manning_n"], kappa=case["kappa"], bc=bc, q_in=q)
        z = case["z"][sl].astype(np.float64)
        e0, u0, v0 = oracle.prepare_state(p, z, case["eta"][sl].astype(np.float64), case["u"][sl].astype(np.float64),
                                          case["v"][sl].astype(np.float64))
        r = oracle.run(p, z, e0, u0, v0, K, dt_fixed=np.full(K, dt))
        assert r.status == 0
        w = (slice(y0 - cy0, y0 - cy0 + W), slice(x0 - cx0, x0 - cx0 + W))
        win = (slice(y0, y0 + W), slice(x0, x0 + W))
        hg = t["eta"][win].double().cpu().numpy() - case["z"][win].astype(np.float64)
        emax, _ = rel_depth_err(hg, r.eta[w] - z[w])
        assert emax <= 1e-4, ((x0, y0), emax)
        ug = t["u"][win].double().cpu().numpy()
        assert np.max(np.abs(ug - r.u[w])) <= 1e-4 * max(1.0, np.max(np.abs(r.u[w]))), (x0, y0)
