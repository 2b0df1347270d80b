"""torch.autograd.Function over the library's discrete adjoint.

``gauge_misfit(n_field, eta0, ..., bed=None)`` returns the loss
L = 1/2 sum_k sum_g (eta_g^k - obs[k-1, g])^2 of a run of ``nsteps`` steps
that starts from (eta0, u0, v0) with the per-cell Manning field n_field over
the bed ``bed`` (case["z"] when None); ``backward`` returns dL/dn, dL/deta0
and dL/dz from ``swe_adjoint`` (one forward run and one reverse sweep with
checkpointing, all on the GPU).  Arguments are marshalled to the C ABI;
nothing is computed here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import swe


class GaugeMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, n_field, eta0, bed, case: dict, nsteps: int, gauges, obs, precision: int, checkpoint_every: int):
        s = swe.Solver(case["nx"], case["ny"], dx=case.get("dx", 1.0), dy=case.get("dy", 1.0),
                       manning_n=float(case.get("manning_n", 0.03)), kappa=0.0, bc=case.get("bc", (0, 0, 0, 0)),
                       q_in=case.get("q_in", (0.0,) * 4), cfl=float(case.get("cfl", 0.5)),
                       dt_max=float(case.get("dt_max", 10.0)), precision=precision)
        try:
            s.set_bed(bed.detach().double().cpu().numpy(), n_field.detach().double().cpu().numpy())
            s.set_state(eta0.detach().double().cpu().numpy(), case["u"], case["v"])
            loss, gn, ge, gz = s.adjoint(nsteps, gauges, obs, checkpoint_every, with_bed=True)
        finally:
            s.close()
        ctx.save_for_backward(torch.from_numpy(gn).to(n_field), torch.from_numpy(ge).to(eta0),
                              torch.from_numpy(gz).to(bed))
        return torch.tensor(loss, dtype=torch.float64, device=n_field.device)

    @staticmethod
    def backward(ctx, grad_out):
        gn, ge, gz = ctx.saved_tensors
        return grad_out * gn, grad_out * ge, grad_out * gz, None, None, None, None, None, None


def gauge_misfit(n_field, eta0, case: dict, nsteps: int, gauges, obs, precision: int = swe.SWE_FP64,
                 checkpoint_every: int = 0, bed=None):
    if bed is None:
        bed = torch.as_tensor(np.asarray(case["z"], dtype=np.float64), device=n_field.device)
    return GaugeMisfit.apply(n_field, eta0, bed, case, int(nsteps), np.asarray(gauges, dtype=np.int64),
                             np.asarray(obs, dtype=np.float64), int(precision), int(checkpoint_every))
