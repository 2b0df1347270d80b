"""Helpers shared by the GPU parity tests (running a case on the GPU through
the C ABI binding and on the oracle with the same seeded inputs)."""
from __future__ import annotations

import numpy as np


def oracle_params(O, case, **kw):
    d = dict(nx=case["nx"], ny=case["ny"], dx=case.get("dx", 1.0), dy=case.get("dy", 1.0),
             manning_n=case.get("manning_n", 0.0), kappa=case.get("kappa", 0.0),
             bc=case.get("bc", (0, 0, 0, 0)), q_in=case.get("q_in", (0.0,) * 4))
    d.update(kw)
    return O.Params(**d)


def gpu_solver(case, precision, kernel, **kw):
    from paper_1309_1230_gb300 import swe
    d = dict(dx=case.get("dx", 1.0), dy=case.get("dy", 1.0), manning_n=case.get("manning_n", 0.0),
             kappa=case.get("kappa", 0.0), bc=case.get("bc", (0, 0, 0, 0)), q_in=case.get("q_in", (0.0,) * 4),
             precision=precision, kernel=kernel)
    d.update(kw)
    s = swe.Solver(case["nx"], case["ny"], **d)
    s.set_bed(case["z"], case.get("nfield"))
    s.set_state(case["eta"], case["u"], case["v"])
    return s


def rel_depth_err(h_gpu, h_ref):
    """max |h - h_ref| / max h_ref and the L2 analogue."""
    scale = max(float(np.max(np.abs(h_ref))), 1e-3)  # floor: the wet/dry threshold
    d = h_gpu - h_ref
    return float(np.max(np.abs(d))) / scale, float(np.sqrt(np.mean(d * d))) / scale


def rel_err(a, b, floor=1e-300):
    scale = max(float(np.max(np.abs(b))), floor)
    return float(np.max(np.abs(a - b))) / scale
