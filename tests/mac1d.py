"""A separate one-dimensional MacCormack shallow-water step, vectorised numpy.

Written independently of the 2D oracle, from the textbook 1D form of the same
scheme: predictor with a one-sided difference, corrector with the opposite
one, average of the two (the explicit predictor/corrector MacCormack method
the paper names in Sec. 1), with the readings the oracle adopts for the parts
the paper leaves to Ransom's thesis (Manning friction taken point-implicitly,
wet/dry rule, Jameson-type dissipation switch, wall/inflow/outflow ends).

A y-invariant strip of the 2D oracle with walls on its long sides must
reproduce this code: the 2D step restricted to such data is exactly this 1D
step (every y difference and y flux is zero).  It is test infrastructure.
"""
from __future__ import annotations

import numpy as np

WALL, INFLOW, OUTFLOW = 0, 1, 2
TINY = 1e-12


def _ghost_velocity(bc, side_sign, q_in, u_in, h_in, h_dry):
    # side_sign +1 at the left end (flow into the domain is +x), -1 at the right end
    if bc == WALL:
        return -u_in
    if bc == INFLOW:
        return side_sign * q_in / max(h_in, h_dry)
    return u_in


def _extend(eta, u, z, h, wet, bcl, bcr, ql, qr, h_dry):
    E = np.concatenate([eta[:1], eta, eta[-1:]])
    Z = np.concatenate([z[:1], z, z[-1:]])
    H = np.concatenate([h[:1], h, h[-1:]])
    Wt = np.concatenate([wet[:1], wet, wet[-1:]])
    U = np.concatenate([[_ghost_velocity(bcl, +1.0, ql, u[0], h[0], h_dry)], u,
                        [_ghost_velocity(bcr, -1.0, qr, u[-1], h[-1], h_dry)]])
    return E, U, Z, H, Wt


def _faces(q, d, bcl, bcr, ql, qr):
    """Face fluxes, face k between cells k-1 and k (k = 0..N); q has ghosts."""
    N = len(q) - 2
    f = np.empty(N + 1)
    inner = q[1:-1]
    if d > 0:
        f[1:N] = inner[1:]      # face k carries cell k (forward difference)
    else:
        f[1:N] = inner[:-1]     # face k carries cell k-1 (backward difference)
    f[0] = 0.0 if bcl == WALL else (ql if bcl == INFLOW else inner[0])
    f[N] = 0.0 if bcr == WALL else (-qr if bcr == INFLOW else inner[-1])
    return f


def _seen(E_nb, Z_nb, W_nb, E_self):
    return np.where((~W_nb) & (Z_nb > E_self), E_self, E_nb)


def _momentum(E, U, Z, Wt, C, u_n, dt, d, dx, g):
    """(u_n - dt * (u u_x + g eta_x)) / (1 + dt C), one-sided in direction d."""
    e, uu = E[1:-1], U[1:-1]
    if d > 0:
        en = _seen(E[2:], Z[2:], Wt[2:], e)
        du = U[2:] - uu
        de = en - e
    else:
        en = _seen(E[:-2], Z[:-2], Wt[:-2], e)
        du = uu - U[:-2]
        de = e - en
    A = uu * du / dx + g * de / dx
    return (u_n - dt * A) / (1.0 + dt * C)


def _fix(eta, u, z, h_dry, area):
    d = eta - z
    neg = d < 0.0
    clamp = float(np.sum(np.where(neg, -d * area, 0.0)))
    eta = np.where(neg, z, eta)
    d = np.where(neg, 0.0, d)
    u = np.where(d <= h_dry, 0.0, u)
    return eta, u, d, clamp


def step(eta, u, z, n2, dt, d, *, dx, g, h_dry, kappa, bcl=WALL, bcr=WALL,
         ql=0.0, qr=0.0, dy=1.0):
    """One step; d = +1 forward predictor, -1 backward.  Returns eta, u."""
    h = eta - z
    wet = h > h_dry
    E, U, Z, H, Wt = _extend(eta, u, z, h, wet, bcl, bcr, ql, qr, h_dry)
    f = _faces(H * U, d, bcl, bcr, ql, qr)
    es = eta - dt * ((f[1:] - f[:-1]) / dx)
    C = np.where(wet, g * n2 * np.sqrt(u * u) / np.power(np.where(wet, h, 1.0), 4.0 / 3.0), 0.0)
    us = _momentum(E, U, Z, Wt, C, u, dt, d, dx, g)
    es, us, hs, _ = _fix(es, us, z, h_dry, dx * dy)
    wets = hs > h_dry
    Es, Us, _, Hs, Ws = _extend(es, us, z, hs, wets, bcl, bcr, ql, qr, h_dry)
    fs = _faces(Hs * Us, -d, bcl, bcr, ql, qr)
    ess = eta - dt * ((fs[1:] - fs[:-1]) / dx)
    Cs = np.where(wets, g * n2 * np.sqrt(us * us) / np.power(np.where(wets, hs, 1.0), 4.0 / 3.0), 0.0)
    uss = _momentum(Es, Us, Z, Ws, Cs, u, dt, -d, dx, g)
    e1 = 0.5 * (es + ess)
    u1 = 0.5 * (us + uss)
    if kappa != 0.0:
        hl, hr = H[:-2], H[2:]
        nu = np.abs((hl + hr) - 2.0 * h) / ((np.abs(hl) + np.abs(hr)) + 2.0 * np.abs(h) + TINY)
        N = len(eta)
        eps = np.zeros(N + 1)  # face k between cells k-1 and k; end faces stay 0
        if N > 1:
            both = wet[:-1] & wet[1:]
            eps[1:N] = np.where(both, np.maximum(nu[:-1], nu[1:]), 0.0)
        ee, ew = eps[1:], eps[:-1]
        for q, out in ((E, 0), (U, 1)):
            qc, qr_, ql_ = q[1:-1], q[2:], q[:-2]
            tx = (np.where(ee != 0.0, ee * (qr_ - qc), 0.0)
                  - np.where(ew != 0.0, ew * (qc - ql_), 0.0))
            if out == 0:
                e1 = e1 + kappa * tx
            else:
                u1 = u1 + kappa * tx
    e1, u1, _, _ = _fix(e1, u1, z, h_dry, dx * dy)
    return e1, u1


def cfl_dt(eta, u, z, *, dx, dy, g, cfl, h_dry, dt_max):
    """The 2D rule on a y-invariant state (v = 0): s = (|u|+c)/dx + (0+c)/dy."""
    h = eta - z
    wet = h > h_dry
    if not np.any(wet):
        return dt_max
    c = np.sqrt(g * h[wet])
    s = (np.abs(u[wet]) + c) / dx + (0.0 + c) / dy
    dt = cfl / np.max(s)
    return min(dt, dt_max)
