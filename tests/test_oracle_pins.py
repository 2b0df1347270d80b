"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test fixes the oracle to something independent of its own code: an
exact conservation law, an exact steady state, a textbook identity, a closed-
form solution, a symmetry of the equations, a brute-force recomputation, or a
separate 1D implementation.  Together they are chosen so that a dropped term,
a wrong sign or index, or a swapped operand in any of the 16 sub-steps fails
at least one of them (see test_oracle_mutants.py, which plants such mistakes).
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_1309_1230_gb300 import inputs as I
from tests import mac1d

G = 9.81


def params_of(O, case, **kw):
    d = dict(nx=case["nx"], ny=case["ny"], dx=case.get("dx", 1.0), dy=case.get("dy", 1.0),
             manning_n=case.get("manning_n", 0.0), kappa=case.get("kappa", 0.0),
             bc=case.get("bc", (0, 0, 0, 0)), q_in=case.get("q_in", (0.0,) * 4))
    d.update(kw)
    return O.Params(**d)


# ---------------------------------------------------------------- conservation
@pytest.mark.parametrize("kappa", [0.0, 0.25])
def test_mass_conservation_closed_basin(oracle, kappa):
    """Flux-form continuity telescopes and walls carry no flux: the volume of
    a closed basin is constant to round-off (64^2 hump, n = 0.03, 200 steps)."""
    c = I.basin_hump(64, 64)
    p = params_of(oracle, c, manning_n=0.03, kappa=kappa)
    r = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], 200)
    assert r.status == 0
    V0 = oracle.volume(p, c["z"], c["eta"])
    V1 = oracle.volume(p, c["z"], r.eta)
    assert r.clamp_volume == 0.0
    assert np.all(r.bflux == 0.0)
    assert abs(V1 - V0) <= 1e-12 * V0
    # the hump must actually have moved (the test is not vacuous)
    assert np.max(np.abs(r.eta - c["eta"])) > 1e-3


def test_volume_budget_open_boundaries(oracle):
    """Open boundaries: the volume change equals the tallied boundary inflow
    plus the tallied clamp volume (river reach 256 x 64, 300 steps)."""
    c = I.river(256, 64, seed=7)
    p = params_of(oracle, c)
    r = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], 300, nthreads=4)
    assert r.status == 0
    V0 = oracle.volume(p, c["z"], c["eta"])
    V1 = oracle.volume(p, c["z"], r.eta)
    assert r.bflux[0] > 0.0 and r.bflux[1] != 0.0
    assert r.bflux[2] == 0.0 and r.bflux[3] == 0.0
    budget = r.bflux.sum() + r.clamp_volume
    assert abs((V1 - V0) - budget) <= 1e-11 * V0


def test_volume_budget_with_drying(oracle):
    """Dam break onto dry ground: volume changes only by the clamp tally."""
    c = I.dam_break(96, 64, seed=3)
    p = params_of(oracle, c)
    r = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], 300)
    assert r.status == 0
    V0 = oracle.volume(p, c["z"], c["eta"])
    V1 = oracle.volume(p, c["z"], r.eta)
    assert r.clamp_volume > 0.0
    assert abs((V1 - V0) - r.clamp_volume) <= 1e-12 * V0
    assert np.min(r.eta - c["z"]) >= 0.0


# Cells of 0.7 m by 1.9 m: a west/east face is dy long, a south/north face dx
# long, and a cell holds h dx dy of water.  With dx = dy = 1 a swapped weight
# would not show.
DX_A, DY_A = 0.7, 1.9


def test_flat_lake_volume_closed_form(oracle):
    """A flat lake of depth H over a flat bed holds H times the domain area
    nx dx by ny dy."""
    nx, ny, H = 23, 17, 1.25
    z = np.full((ny, nx), -0.5)
    p = oracle.Params(nx=nx, ny=ny, dx=DX_A, dy=DY_A)
    V = oracle.volume(p, z, z + H)
    assert abs(V - H * (nx * DX_A) * (ny * DY_A)) <= 1e-13 * V


def test_volume_budget_anisotropic_cells_all_sides_open(oracle):
    """Inflow through the west and south sides, outflow east and north, on
    0.7 m by 1.9 m cells: the volume change equals the sum of the four
    tallied side inflows (each weighted by its own face length) plus the
    clamp tally, and every side carries water."""
    c = I.with_cell_size(I.open_river(96, 80, seed=17), DX_A, DY_A)
    p = params_of(oracle, c)
    r = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], 250, nthreads=4)
    assert r.status == 0
    V0 = oracle.volume(p, c["z"], c["eta"])
    V1 = oracle.volume(p, c["z"], r.eta)
    assert r.bflux[0] > 0.0 and r.bflux[2] > 0.0
    # none of the four terms is negligible next to the tolerance (the open
    # sides let water out or, where the surface tilts back, in)
    assert np.min(np.abs(r.bflux)) > 1e-3 * V0
    budget = r.bflux.sum() + r.clamp_volume
    assert abs((V1 - V0) - budget) <= 1e-11 * V0


def test_volume_budget_anisotropic_cells_with_drying(oracle):
    """Dam break onto dry ground on 0.7 m by 1.9 m cells: the volume changes
    only by the clamp tally, which counts the added depth times dx dy."""
    c = I.with_cell_size(I.dam_break(96, 64, seed=3), DX_A, DY_A)
    p = params_of(oracle, c)
    r = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], 300)
    assert r.status == 0
    V0 = oracle.volume(p, c["z"], c["eta"])
    V1 = oracle.volume(p, c["z"], r.eta)
    assert r.clamp_volume > 1e-9 * V0
    assert abs((V1 - V0) - r.clamp_volume) <= 1e-12 * V0


# ---------------------------------------------------------------- lake at rest
def _lake(nx, ny, seed, level, islands):
    rng = np.random.Generator(np.random.PCG64(seed))
    z = I.gaussian_sum_bed(nx, ny, rng, 12, (0.0, 2.0), (3.0, 10.0))
    if not islands:
        level = float(z.max()) + 0.25
    eta = np.maximum(level, z)
    return z, eta, level


@pytest.mark.parametrize("islands", [False, True])
@pytest.mark.parametrize("kappa", [0.0, 0.25])
def test_lake_at_rest(oracle, islands, kappa):
    """A flat free surface at rest over an uneven bed stays exactly at rest,
    whether the bed is fully submerged or pierces the surface (dry islands)."""
    z, eta, level = _lake(48, 40, 11, 1.0, islands)
    if islands:
        assert np.any(z > level) and np.any(z < level - 0.5)
    else:
        assert np.all(z < level)
    zeros = np.zeros_like(z)
    p = oracle.Params(nx=48, ny=40, manning_n=0.03, kappa=kappa)
    r = oracle.run(p, z, eta, zeros, zeros, 100)
    assert np.array_equal(r.eta, eta)
    assert np.array_equal(r.u, zeros) and np.array_equal(r.v, zeros)


# ---------------------------------------------------------------- 1D reduction
@pytest.mark.parametrize("case", ["dambreak", "river"])
def test_reduces_to_separate_1d_code(oracle, case):
    """A y-invariant strip with walls on its long sides keeps v = 0 and equal
    rows exactly, and matches an independent 1D MacCormack code."""
    N, ny, steps = 120, 3, 150
    x = (np.arange(N) + 0.5)
    if case == "dambreak":
        z1 = 0.6 * np.exp(-((x - 80.0) / 9.0) ** 2) + 0.3 * np.exp(-((x - 30.0) / 6.0) ** 2)
        e1 = np.where(x < 50.0, np.maximum(2.0, z1), z1)
        u1 = np.zeros(N)
        bc, q = (0, 0), (0.0, 0.0)
        nman, kappa = 0.035, 0.25
    else:
        z1 = -2e-3 * x + 0.05 * np.sin(x / 7.0)
        e1 = z1 + 1.0
        u1 = np.full(N, 0.3)
        bc, q = (1, 2), (1.5, 0.0)
        nman, kappa = 0.03, 0.25
    z = np.tile(z1, (ny, 1))
    eta = np.tile(e1, (ny, 1))
    u = np.tile(u1, (ny, 1))
    v = np.zeros_like(z)
    p = oracle.Params(nx=N, ny=ny, manning_n=nman, kappa=kappa, bc=(bc[0], bc[1], 0, 0),
                      q_in=(q[0], q[1], 0.0, 0.0))
    eta, u, v = oracle.prepare_state(p, z, eta, u, v)
    r = oracle.run(p, z, eta, u, v, steps)
    assert r.status == 0
    assert np.all(r.v == 0.0)
    for j in range(1, ny):
        assert np.array_equal(r.eta[j], r.eta[0]) and np.array_equal(r.u[j], r.u[0])
    e, uu = eta[0].copy(), u[0].copy()
    n2 = nman * nman
    for k in range(steps):
        dt = mac1d.cfl_dt(e, uu, z1, dx=1.0, dy=1.0, g=G, cfl=0.5, h_dry=1e-3, dt_max=10.0)
        assert dt == r.dt[k]
        d = +1 if k % 2 == 0 else -1
        e, uu = mac1d.step(e, uu, z1, n2, dt, d, dx=1.0, g=G, h_dry=1e-3, kappa=kappa,
                           bcl=bc[0], bcr=bc[1], ql=q[0], qr=q[1])
    assert np.max(np.abs(r.eta[0] - e)) <= 1e-14 * np.max(np.abs(e))
    assert np.max(np.abs(r.u[0] - uu)) <= 1e-14 * max(1.0, np.max(np.abs(uu)))
    # the run must exercise what it claims to
    if case == "dambreak":
        assert r.clamp_volume >= 0.0 and np.any(r.eta[0] - z1 <= 1e-3)
    assert np.max(np.abs(uu)) > 0.1


# ---------------------------------------------------------------- linear limit
def test_linear_limit_is_lax_wendroff(oracle):
    """For a small perturbation of still water (n = 0, kappa = 0, flat bed),
    one MacCormack step equals the 2D Lax-Wendroff-type update of the
    linearised system q_t + A q_x + B q_y = 0:
        q1 = q - dt/2 (L+ + L-) q + dt^2/2 L- L+ q,  L+- = A d_x^+- + B d_y^+-
    (predictor forward, corrector backward).  Nonlinear terms are O(a^2)."""
    nx, ny, H, a, dt = 40, 36, 1.0, 1e-6, 0.05
    rng = np.random.Generator(np.random.PCG64(42))
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    f = lambda: (np.sin(2 * np.pi * (x * rng.uniform(0.5, 3) / nx + rng.uniform()))
                 * np.cos(2 * np.pi * (y * rng.uniform(0.5, 3) / ny + rng.uniform())))
    ep, up, vp = a * f(), a * f(), a * f()
    z = np.zeros((ny, nx))
    dx, dy = 1.0, 1.3
    p = oracle.Params(nx=nx, ny=ny, dx=dx, dy=dy, manning_n=0.0, kappa=0.0)
    r = oracle.run(p, z, H + ep, up, vp, 1, dt_fixed=[dt])
    Q = np.stack([ep, up, vp])  # (3, ny, nx)
    A = np.array([[0, H, 0], [G, 0, 0], [0, 0, 0]], float)
    B = np.array([[0, 0, H], [0, 0, 0], [G, 0, 0]], float)
    dxp = lambda q: (np.roll(q, -1, axis=2) - q) / dx
    dxm = lambda q: (q - np.roll(q, 1, axis=2)) / dx
    dyp = lambda q: (np.roll(q, -1, axis=1) - q) / dy
    dym = lambda q: (q - np.roll(q, 1, axis=1)) / dy
    M = lambda m, q: np.einsum("ab,bij->aij", m, q)
    Lp = lambda q: M(A, dxp(q)) + M(B, dyp(q))
    Lm = lambda q: M(A, dxm(q)) + M(B, dym(q))
    Q1 = Q - 0.5 * dt * (Lp(Q) + Lm(Q)) + 0.5 * dt * dt * Lm(Lp(Q))
    got = np.stack([r.eta - H, r.u, r.v])
    sl = (slice(None), slice(3, ny - 3), slice(3, nx - 3))  # away from the walls
    err = np.max(np.abs(got[sl] - Q1[sl])) / np.max(np.abs(Q1[sl]))
    assert err <= 1e-5
    # the second-order (dt^2) term is visible at this tolerance
    Q1_first = Q - 0.5 * dt * (Lp(Q) + Lm(Q))
    assert np.max(np.abs(got[sl] - Q1_first[sl])) / np.max(np.abs(Q1[sl])) > 1e-4


# ---------------------------------------------------------------- wave speed
def _seiche_period(O, L, H=1.0, a=1e-3):
    """Period of the gravest closed-basin mode from zero crossings of the
    elevation in the first cell, fixed dt."""
    nx = L
    x = (np.arange(nx) + 0.5)
    eta1 = H + a * np.cos(np.pi * x / L)
    z = np.zeros((1, nx))
    eta = eta1[None, :]
    zeros = np.zeros_like(z)
    c = math.sqrt(G * H)
    T = 2.0 * L / c
    dt = 0.2 / c
    nsteps = int(2.6 * T / dt)
    p = O.Params(nx=nx, ny=1, dx=1.0, dy=1.0, manning_n=0.0, kappa=0.0)
    chunk = 8
    series = [eta[0, 0] - H]
    state = (eta, zeros, zeros)
    k = 0
    while k < nsteps:
        r = O.run(p, z, *state, chunk, step0=k, dt_fixed=[dt] * chunk)
        state = (r.eta, r.u, r.v)
        k += chunk
        series.append(r.eta[0, 0] - H)
    s = np.array(series)
    t = np.arange(len(s)) * dt * chunk
    idx = np.nonzero(np.sign(s[:-1]) != np.sign(s[1:]))[0]
    tz = t[idx] - s[idx] * (t[idx + 1] - t[idx]) / (s[idx + 1] - s[idx])
    assert len(tz) >= 4
    return 2.0 * np.mean(np.diff(tz[:4])), T


def test_seiche_period_matches_sqrt_gh(oracle):
    """Linear long waves travel at sqrt(g H): the gravest seiche of a closed
    basin of length L has period 2L / sqrt(g H), within 1% at L = 64 cells,
    with the error shrinking at second order under refinement."""
    errs = {}
    for L in (32, 64, 128):
        Tm, T = _seiche_period(oracle, L)
        errs[L] = abs(Tm / T - 1.0)
    assert errs[64] <= 0.01
    assert errs[32] / errs[64] >= 3.0 and errs[64] / errs[128] >= 3.0


# ---------------------------------------------------------------- dam breaks
def _dambreak_1d(O, N, h0, h1, T, length=2000.0, kappa=0.25, dissipation=0):
    dx = length / N
    x = (np.arange(N) + 0.5) * dx
    x0 = length / 2.0
    z = np.zeros((1, N))
    eta = np.where(x < x0, h0, h1)[None, :]
    zeros = np.zeros_like(z)
    c0 = math.sqrt(G * h0)
    dt = 0.3 * dx / (2.0 * c0)
    nsteps = int(round(T / dt))
    dt = T / nsteps
    p = O.Params(nx=N, ny=1, dx=dx, dy=dx, manning_n=0.0, kappa=kappa, dissipation=dissipation)
    r = O.run(p, z, eta, zeros, zeros, nsteps, dt_fixed=np.full(nsteps, dt))
    assert r.status == 0
    return x - x0, r.eta[0], r.u[0], dx


def _ritter(xi, t, h0):
    c0 = math.sqrt(G * h0)
    h = np.where(xi <= -c0 * t, h0, (2.0 * c0 - xi / t) ** 2 / (9.0 * G))
    return np.where(xi >= 2.0 * c0 * t, 0.0, h)


def _stoker(xi, t, h0, h1):
    c0, c1 = math.sqrt(G * h0), math.sqrt(G * h1)
    f = lambda cm: -8.0 * c1 ** 2 * cm ** 2 * (c0 - cm) ** 2 + (cm ** 2 - c1 ** 2) ** 2 * (cm ** 2 + c1 ** 2)
    cm = brentq(f, c1 * (1 + 1e-12), c0 * (1 - 1e-12))
    hm = cm * cm / G
    S = 2.0 * cm ** 2 * (c0 - cm) / (cm ** 2 - c1 ** 2)
    fan = (2.0 * c0 - xi / t) ** 2 / (9.0 * G)
    h = np.where(xi <= -c0 * t, h0, fan)
    h = np.where(xi >= (2.0 * c0 - 3.0 * cm) * t, hm, h)
    h = np.where(xi >= S * t, h1, h)
    return h, hm, S


def _l1(h, he, dx):
    return np.sum(np.abs(h - he)) * dx / (np.sum(np.abs(he)) * dx)


def test_stoker_wet_dam_break(oracle):
    """Wet-bed dam break (h0 = 1, h1 = 0.1 m): L1 depth error against the
    Stoker solution below 3% at 1000 cells and falling under refinement."""
    T = 60.0
    errs = []
    for N in (500, 1000, 2000):
        xi, eta, u, dx = _dambreak_1d(oracle, N, 1.0, 0.1, T)
        he, hm, S = _stoker(xi, T, 1.0, 0.1)
        errs.append(_l1(eta, he, dx))
    assert errs[1] <= 0.03
    assert errs[0] > errs[1] > errs[2]


def test_stoker_middle_state_closed_form():
    """The closed form itself: for h0 = 1, h1 = 0.1 the middle state and the
    shock satisfy the Rankine-Hugoniot mass balance across the shock."""
    h, hm, S = _stoker(np.array([0.0]), 1.0, 1.0, 0.1)
    um = 2.0 * (math.sqrt(G) - math.sqrt(G * hm))
    assert S * (hm - 0.1) == pytest.approx(hm * um, rel=1e-10)


def test_ritter_dry_dam_break(oracle):
    """Dry-bed dam break (h0 = 1 m, wet threshold 1e-3 m): L1 depth error
    against the Ritter solution below 5% at 1000 cells and falling under
    refinement; no depth is negative."""
    T = 40.0
    errs = []
    for N in (500, 1000, 2000):
        xi, eta, u, dx = _dambreak_1d(oracle, N, 1.0, 0.0, T)
        assert np.min(eta) >= 0.0
        errs.append(_l1(eta, _ritter(xi, T, 1.0), dx))
    assert errs[1] <= 0.05
    assert errs[0] > errs[1] > errs[2]


# ---------------------------------------------------------------- symmetry
def _random_state(nx, ny, seed, dry=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    z = I.gaussian_sum_bed(nx, ny, rng, 6, (0.0, 1.5), (3.0, 8.0))
    eta = np.maximum(1.0 + 0.2 * rng.standard_normal((ny, nx)) * 0.1, z if dry else z + 0.2)
    u = 0.3 * rng.standard_normal((ny, nx))
    v = 0.3 * rng.standard_normal((ny, nx))
    return z, eta, u, v


def test_mirror_and_transpose_symmetry(oracle):
    """The equations are invariant under x -> -x (u -> -u), y -> -y (v -> -v)
    and, on a square grid, x <-> y (u <-> v).  With the predictor directions
    mirrored accordingly the oracle's results map onto each other exactly."""
    n = 40
    z, eta, u, v = _random_state(n, n, 5)
    kw = dict(nx=n, ny=n, manning_n=0.03, kappa=0.25, bc=(1, 2, 0, 1), q_in=(0.7, 0.0, 0.0, 0.4))
    p = oracle.Params(**kw)
    eta, u, v = oracle.prepare_state(p, z, eta, u, v)
    base = oracle.run(p, z, eta, u, v, 40)
    assert base.status == 0
    # mirror x: swap W/E, start x backward (dir_cycle 1 -> 3)
    px = oracle.Params(**{**kw, "bc": (2, 1, 0, 1), "q_in": (0.0, 0.7, 0.0, 0.4), "dir_cycle": 3})
    rx = oracle.run(px, z[:, ::-1], eta[:, ::-1], -u[:, ::-1], v[:, ::-1], 40)
    assert np.array_equal(rx.eta[:, ::-1], base.eta)
    assert np.array_equal(-rx.u[:, ::-1], base.u) and np.array_equal(rx.v[:, ::-1], base.v)
    # mirror y: swap S/N, start y backward (dir_cycle 1 -> 5)
    py = oracle.Params(**{**kw, "bc": (1, 2, 1, 0), "q_in": (0.7, 0.0, 0.4, 0.0), "dir_cycle": 5})
    ry = oracle.run(py, z[::-1], eta[::-1], u[::-1], -v[::-1], 40)
    assert np.array_equal(ry.eta[::-1], base.eta)
    assert np.array_equal(ry.u[::-1], base.u) and np.array_equal(-ry.v[::-1], base.v)
    # transpose: W<->S, E<->N
    pt = oracle.Params(**{**kw, "bc": (0, 1, 1, 2), "q_in": (0.0, 0.4, 0.7, 0.0)})
    rt = oracle.run(pt, z.T, eta.T, v.T, u.T, 40)
    assert np.array_equal(rt.eta.T, base.eta)
    assert np.array_equal(rt.v.T, base.u) and np.array_equal(rt.u.T, base.v)


# ---------------------------------------------------------------- friction
def test_uniform_flow_friction_recursion_and_manning(oracle):
    """Away from the ends of a long sloping channel the flow stays uniform and
    every step reduces to the scalar point-implicit Manning recursion; its
    fixed point is Manning's normal flow q = h^(5/3) sqrt(S) / n."""
    N, S, n, h, dt = 6000, 0.01, 0.03, 1.0, 0.1
    x = (np.arange(N) + 0.5)
    z = (-S * x)[None, :]
    eta = z + h
    u0 = 0.5
    U = np.full((1, N), u0)
    V = np.zeros((1, N))
    p = oracle.Params(nx=N, ny=1, manning_n=n, kappa=0.0, bc=(1, 2, 0, 0), q_in=(h * u0, 0, 0, 0))
    steps = 3000  # 300 s: about 18 friction relaxation times; the ends stay far away
    r = oracle.run(p, z, eta, U, V, steps, dt_fixed=np.full(steps, dt), nthreads=4)
    mid = slice(N // 2 - 20, N // 2 + 20)
    # scalar recursion, written from the point-implicit Manning update
    C = lambda w: G * n * n * abs(w) / h ** (4.0 / 3.0)
    w = u0
    for _ in range(steps):
        ws = (w + dt * G * S) / (1.0 + dt * C(w))
        wss = (w + dt * G * S) / (1.0 + dt * C(ws))
        w = 0.5 * (ws + wss)
    assert np.max(np.abs(r.u[0, mid] - w)) <= 1e-10 * w
    assert np.max(np.abs(r.eta[0, mid] - z[0, mid] - h)) <= 1e-10
    q_manning = h ** (5.0 / 3.0) * math.sqrt(S) / n
    assert abs(h * w - q_manning) <= 1e-6 * q_manning


# ---------------------------------------------------------------- time step
def test_cfl_dt_brute_force(oracle):
    """S2 recomputed cell by cell in plain Python equals the oracle's dt."""
    z, eta, u, v = _random_state(17, 13, 9)
    p = oracle.Params(nx=17, ny=13, dx=0.8, dy=1.7, cfl=0.45, dt_max=10.0)
    eta, u, v = oracle.prepare_state(p, z, eta, u, v)
    smax = 0.0
    for j in range(13):
        for i in range(17):
            h = eta[j, i] - z[j, i]
            if h > 1e-3:
                c = math.sqrt(9.81 * h)
                s = (abs(u[j, i]) + c) / 0.8 + (abs(v[j, i]) + c) / 1.7
                smax = max(smax, s)
    assert oracle.cfl_dt(p, z, eta, u, v) == min(0.45 / smax, 10.0)
    r = oracle.run(p, z, eta, u, v, 1)
    assert r.dt[0] == min(0.45 / smax, 10.0)
    # the cap binds when the CFL step would be longer than dt_max
    pc = oracle.Params(nx=17, ny=13, dx=0.8, dy=1.7, cfl=0.45, dt_max=0.01)
    assert 0.45 / smax > 0.01 and oracle.cfl_dt(pc, z, eta, u, v) == 0.01
    # all dry: dt_max
    zz = np.zeros((13, 17))
    assert oracle.cfl_dt(p, zz, zz, zz, zz) == 10.0


def test_prepare_state_normalises_and_rejects(oracle):
    p = oracle.Params(nx=4, ny=2)
    z = np.zeros((2, 4))
    eta = np.array([[1.0, 5e-4, -1e-13, 2.0], [0.0, 1.0, 1.0, 1.0]])
    u = np.ones((2, 4))
    e, uu, vv = oracle.prepare_state(p, z, eta, u, u)
    assert e[0, 2] == 0.0
    assert uu[0, 1] == 0.0 and uu[0, 2] == 0.0 and uu[1, 0] == 0.0 and uu[0, 0] == 1.0
    with pytest.raises(ValueError):
        oracle.prepare_state(p, z, np.where(z == 0, -1e-9, 0.0), u, u)


def test_degenerate_grids_run(oracle):
    """1x1, 1xN and Nx1 grids step without error and conserve volume."""
    for nx, ny in ((1, 1), (1, 7), (9, 1)):
        z = np.zeros((ny, nx))
        eta = 1.0 + 0.1 * np.arange(nx * ny).reshape(ny, nx) / max(1, nx * ny)
        p = oracle.Params(nx=nx, ny=ny, manning_n=0.03, kappa=0.25)
        r = oracle.run(p, z, eta, z, z, 20)
        assert r.status == 0
        V0, V1 = oracle.volume(p, z, eta), oracle.volume(p, z, r.eta)
        assert abs(V1 - V0) <= 1e-13 * V0
