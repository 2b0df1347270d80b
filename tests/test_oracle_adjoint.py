"""Pins of the oracle's discrete adjoint: central finite differences of the
oracle's own forward map (the gradient is the directional derivative), in
random directions of the Manning field, the bed and the initial state, plus
its scope checks.  FP64, frozen step sizes, kappa = 0, fully wet."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I


def _case(nx=24, ny=20, T=30, seed=4, bc=(0, 0, 0, 0), q_in=(0.0,) * 4):
    c = I.adjoint_case(nx, ny, seed=seed, n_gauges=5)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    c["u"] = 0.05 * rng.standard_normal((ny, nx))
    c["v"] = 0.05 * rng.standard_normal((ny, nx))
    nfield = 0.03 * (1.0 + 0.2 * rng.uniform(-1, 1, (ny, nx)))
    return c, nfield, T, bc, q_in


def _loss(O, p, c, nfield, eta, u, v, dt, gauges, obs, z=None):
    z = c["z"] if z is None else z
    r = O.run(p, z, eta, u, v, len(dt), nfield=nfield, dt_fixed=dt)
    assert r.status == 0
    # re-run step by step to collect the gauge series (oracle forward only)
    L = 0.0
    e, uu, vv = eta, u, v
    for k in range(len(dt)):
        r = O.run(p, z, e, uu, vv, 1, nfield=nfield, dt_fixed=dt[k:k + 1], step0=k)
        e, uu, vv = r.eta, r.u, r.v
        res = e.ravel()[gauges] - obs[k]
        L += 0.5 * float(res @ res)
    return L


@pytest.mark.parametrize("bcs", ["walls", "open"])
def test_adjoint_matches_central_differences(oracle, bcs):
    bc, q = ((0, 0, 0, 0), (0.0,) * 4) if bcs == "walls" else ((1, 2, 0, 2), (0.4, 0.0, 0.0, 0.0))
    c, nfield, T, bc, q = _case(bc=bc, q_in=q)
    p = oracle.Params(nx=c["nx"], ny=c["ny"], manning_n=0.03, kappa=0.0, bc=bc, q_in=q)
    fwd = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], T, nfield=nfield)
    dt = fwd.dt
    gauges = c["gauges"]
    rng = np.random.Generator(np.random.PCG64(9))
    obs = np.stack([c["eta"].ravel()[gauges] + 0.01 * rng.standard_normal(len(gauges)) for _ in range(T)])
    adj = oracle.adjoint(p, c["z"], nfield, c["eta"], c["u"], c["v"], dt, gauges, obs)
    assert adj.status == 0
    L0 = _loss(oracle, p, c, nfield, c["eta"], c["u"], c["v"], dt, gauges, obs)
    assert adj.loss == pytest.approx(L0, rel=1e-12)
    for trial in range(4):
        dn = rng.standard_normal(nfield.shape) * 0.003
        de = rng.standard_normal(nfield.shape) * 0.01
        du = rng.standard_normal(nfield.shape) * 0.01
        eps = 1e-5
        Lp = _loss(oracle, p, c, nfield + eps * dn, c["eta"] + eps * de, c["u"] + eps * du, c["v"], dt, gauges, obs)
        Lm = _loss(oracle, p, c, nfield - eps * dn, c["eta"] - eps * de, c["u"] - eps * du, c["v"], dt, gauges, obs)
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(adj.grad_n * dn) + np.sum(adj.grad_eta0 * de) + np.sum(adj.grad_u0 * du))
        assert abs(fd - ad) <= 1e-5 * max(abs(fd), 1e-12), (trial, fd, ad)
    # the bed alone, with the initial elevation held (so the depth changes)
    for trial in range(3):
        dz = rng.standard_normal(nfield.shape) * 0.01
        eps = 1e-5
        Lp = _loss(oracle, p, c, nfield, c["eta"], c["u"], c["v"], dt, gauges, obs, z=c["z"] + eps * dz)
        Lm = _loss(oracle, p, c, nfield, c["eta"], c["u"], c["v"], dt, gauges, obs, z=c["z"] - eps * dz)
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(adj.grad_z * dz))
        assert abs(fd) > 0.0
        assert abs(fd - ad) <= 1e-5 * abs(fd), ("bed", trial, fd, ad)


def test_bed_gradient_of_a_lake_at_rest_is_zero(oracle):
    """A lake at rest (flat surface, zero velocity) stays at rest over any
    fully submerged bed, so the loss does not depend on the bed to first
    order: with gauge records 1 cm off the surface (nonzero residuals) the
    bed and Manning gradients are exactly zero while the gradient with
    respect to the initial surface is not."""
    c, nfield, T, bc, q = _case(T=12)
    eta = np.full_like(c["eta"], float(c["z"].max()) + 1.0)
    zero = np.zeros_like(eta)
    p = oracle.Params(nx=c["nx"], ny=c["ny"], manning_n=0.03, kappa=0.0)
    obs = np.full((T, len(c["gauges"])), eta[0, 0] + 0.01)
    adj = oracle.adjoint(p, c["z"], nfield, eta, zero, zero, np.full(T, 0.05), c["gauges"], obs)
    assert adj.status == 0 and adj.loss > 0.0
    assert np.abs(adj.grad_eta0).max() > 0.0
    assert not adj.grad_z.any() and not adj.grad_n.any()


def test_adjoint_scope_is_enforced(oracle):
    c, nfield, T, bc, q = _case(T=5)
    p = oracle.Params(nx=c["nx"], ny=c["ny"], manning_n=0.03, kappa=0.25)
    r = oracle.adjoint(p, c["z"], nfield, c["eta"], c["u"], c["v"], np.full(5, 0.05), c["gauges"],
                       np.zeros((5, len(c["gauges"]))))
    assert r.status == 5
    p0 = oracle.Params(nx=c["nx"], ny=c["ny"], manning_n=0.03, kappa=0.0)
    dry = c["eta"].copy()
    dry[0, 0] = c["z"][0, 0]
    r = oracle.adjoint(p0, c["z"], nfield, dry, c["u"] * 0, c["v"] * 0, np.full(5, 0.05), c["gauges"],
                       np.zeros((5, len(c["gauges"]))))
    assert r.status == 5
