"""Recovery of a per-cell Manning field, or of the bed, from gauge records:
the inverse problems the discrete adjoint serves.

``calibrate_manning`` minimises the gauge misfit of ``autograd.gauge_misfit``
(plus an optional smoothness penalty on log n) over log n with L-BFGS;
``calibrate_bed`` does the same over the bed elevation z with the initial
surface held (a bed change is a depth change), with the adjoint's dL/dz.
Every loss and gradient is one forward run and one reverse sweep of the
library on the GPU; the optimiser's own vector arithmetic on the n field is
plain torch on the device the caller chooses.
"""
from __future__ import annotations

import numpy as np
import torch

from . import swe
from .autograd import gauge_misfit


def gauge_series(case: dict, n_field, nsteps: int, gauges, precision: int = swe.SWE_FP64, bed=None) -> np.ndarray:
    """Elevation at the gauge cells after each of nsteps steps (nsteps x ngauges),
    from a forward run of the library with the per-cell Manning field n_field
    over the bed `bed` (case["z"] when None)."""
    s = swe.Solver(case["nx"], case["ny"], dx=case.get("dx", 1.0), dy=case.get("dy", 1.0),
                   manning_n=float(case.get("manning_n", 0.03)), kappa=0.0, bc=case.get("bc", (0, 0, 0, 0)),
                   q_in=case.get("q_in", (0.0,) * 4), cfl=float(case.get("cfl", 0.5)),
                   dt_max=float(case.get("dt_max", 10.0)), precision=precision)
    g = np.asarray(gauges, dtype=np.int64)
    out = np.empty((int(nsteps), g.shape[0]))
    try:
        s.set_bed(case["z"] if bed is None else np.asarray(bed, dtype=np.float64),
                  np.asarray(n_field, dtype=np.float64))
        s.set_state(case["eta"], case["u"], case["v"])
        for k in range(int(nsteps)):
            s.step(1, want_info=False)
            out[k] = s.get_state()[0].ravel()[g]
    finally:
        s.close()
    return out


def calibrate_manning(case: dict, gauges, obs, nsteps: int, n_init, iters: int = 20, smooth: float = 0.0,
                      precision: int = swe.SWE_FP64, device: str = "cpu"):
    """Returns (n_field, history of the objective at each evaluation).  The
    optimiser sees the objective divided by its starting value, so that its
    stopping tolerances do not depend on the scale of the records."""
    theta = torch.tensor(np.log(np.asarray(n_init, dtype=np.float64)), device=device, requires_grad=True)
    eta0 = torch.tensor(np.asarray(case["eta"], dtype=np.float64), device=device)
    opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=int(iters), history_size=10,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-10, tolerance_change=1e-14)
    history = []
    scale = []

    def objective():
        n = torch.exp(theta)
        loss = gauge_misfit(n, eta0, case, nsteps, gauges, obs, precision)
        if smooth > 0.0:
            loss = loss + smooth * (torch.sum(torch.diff(theta, dim=0) ** 2) + torch.sum(torch.diff(theta, dim=1) ** 2))
        return loss

    def closure():
        opt.zero_grad()
        loss = objective()
        history.append(float(loss.detach()))
        if not scale:
            scale.append(1.0 / history[0] if history[0] > 0 else 1.0)
        (loss * scale[0]).backward()
        return loss * scale[0]

    opt.step(closure)
    return torch.exp(theta).detach().cpu().numpy(), history


def calibrate_bed(case: dict, gauges, obs, nsteps: int, z_init, n_field, iters: int = 20, smooth: float = 0.0,
                  precision: int = swe.SWE_FP64, device: str = "cpu"):
    """Returns (bed, history of the objective at each evaluation): L-BFGS over
    the bed elevation with the initial surface case["eta"] and the Manning
    field n_field held, from z_init.  The adjoint covers the fully wet
    regime, so the bed must stay below the surface by more than h_dry."""
    z = torch.tensor(np.asarray(z_init, dtype=np.float64), device=device, requires_grad=True)
    eta0 = torch.tensor(np.asarray(case["eta"], dtype=np.float64), device=device)
    n = torch.tensor(np.asarray(n_field, dtype=np.float64), device=device)
    opt = torch.optim.LBFGS([z], lr=1.0, max_iter=int(iters), history_size=10,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-12, tolerance_change=1e-14)
    history = []
    scale = []

    def closure():
        opt.zero_grad()
        loss = gauge_misfit(n, eta0, case, nsteps, gauges, obs, precision, bed=z)
        if smooth > 0.0:
            loss = loss + smooth * (torch.sum(torch.diff(z, dim=0) ** 2) + torch.sum(torch.diff(z, dim=1) ** 2))
        history.append(float(loss.detach()))
        if not scale:
            scale.append(1.0 / history[0] if history[0] > 0 else 1.0)
        (loss * scale[0]).backward()
        return loss * scale[0]

    opt.step(closure)
    return z.detach().cpu().numpy(), history
