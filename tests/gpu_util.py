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


# FP32 form against the FP64 oracle, relative to each field's scale (depth:
# its maximum; velocities: the largest velocity component of the flow, at
# least 1e-3 m/s, so that a component that is nearly zero everywhere, such
# as v in a narrow channel, is measured against the flow and not against its
# own rounding).  Depth: 1e-4 of the maximum depth in the max norm and 1e-5 in
# L2.  Velocities: the pressure term differences elevations of ~1-10 m stored
# with ~5e-7 m of rounding, so every step adds ~g dt/dx * 1e-6 m/s of noise
# (~5e-7 m/s); over a few hundred steps that is ~1e-5 m/s against velocities
# of 0.05 to a few m/s.  The measured worst case on the parity cases is 8e-5
# (max) and 1.5e-5 (L2); the bounds are 5e-4 and 1e-4.
FP32_TOL = dict(h_max=1e-4, h_l2=1e-5, uv_max=5e-4, uv_l2=1e-4)


def fp32_errors(e, u, v, ref_eta, ref_u, ref_v, z):
    """Max and L2 errors of depth, u and v against the FP64 reference, each
    relative to its scale (above)."""
    def rel(a, b, s):
        d = a - b
        return float(np.max(np.abs(d))) / s, float(np.sqrt(np.mean(d * d))) / s
    href = ref_eta - z
    sv = max(float(np.max(np.abs(ref_u))), float(np.max(np.abs(ref_v))), 1e-3)
    return dict(h=rel(e - z, href, max(float(np.max(np.abs(href))), 1e-3)), u=rel(u, ref_u, sv), v=rel(v, ref_v, sv))


def assert_fp32_close(e, u, v, ref_eta, ref_u, ref_v, z, tol=FP32_TOL):
    err = fp32_errors(e, u, v, ref_eta, ref_u, ref_v, z)
    assert err["h"][0] <= tol["h_max"] and err["h"][1] <= tol["h_l2"], err
    for f in "uv":
        assert err[f][0] <= tol["uv_max"] and err[f][1] <= tol["uv_l2"], err
    return err
