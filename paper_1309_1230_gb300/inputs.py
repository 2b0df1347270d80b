"""Seeded synthetic workloads.

This module only draws inputs (bed, initial state, friction field, gauge
positions) and holds none of the scheme's arithmetic, so both the CPU oracle
and the CUDA path are fed from it.  Seeds follow ``Generator(PCG64(seed))``.

The paper's five datasets (Five Drops, Inlet Flood, Five Drops Big, Channel
Flood, Vortex; Sec. 4, Table 1) are not available; these generators stand in
for them: closed-basin humps for "Five Drops", an inflow river reach for
"Inlet/Channel Flood", and a dam break over dry ground for the wet/dry path
the paper's code lacked (Sec. 6.2).

Every generator returns a dict with float64 arrays of shape (ny, nx)
(``z``, ``eta``, ``u``, ``v`` and optionally ``nfield``) and the scalar
settings (``nx``, ``ny``, ``dx``, ``dy``, ``manning_n``, ``kappa``, ``bc``,
``q_in``) in the W, E, S, N side order with 0 = wall, 1 = inflow,
2 = outflow.
"""
from __future__ import annotations

import numpy as np

WALL, INFLOW, OUTFLOW = 0, 1, 2


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _cell_centres(nx: int, ny: int, dx: float = 1.0, dy: float = 1.0):
    x = (np.arange(nx, dtype=np.float64) + 0.5) * dx
    y = (np.arange(ny, dtype=np.float64) + 0.5) * dy
    return x, y


def gaussian_sum_bed(nx: int, ny: int, rng: np.random.Generator, count: int,
                     amp: tuple, width_cells: tuple) -> np.ndarray:
    """Sum of `count` isotropic Gaussians: heights U(amp), widths U(width)
    cells, centres uniform over the domain."""
    a = rng.uniform(amp[0], amp[1], count)
    w = rng.uniform(width_cells[0], width_cells[1], count)
    cx = rng.uniform(0.0, nx, count)
    cy = rng.uniform(0.0, ny, count)
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    z = np.zeros((ny, nx), dtype=np.float64)
    for k in range(count):
        gx = np.exp(-((x - cx[k]) ** 2) / (2.0 * w[k] ** 2))
        gy = np.exp(-((y - cy[k]) ** 2) / (2.0 * w[k] ** 2))
        z += a[k] * np.outer(gy, gx)
    return z


def smooth_noise(nx: int, ny: int, rng: np.random.Generator, sigma_cells: float,
                 dtype=np.float64) -> np.ndarray:
    """White noise, separable Gaussian filter (sigma in cells, reflecting
    edges), rescaled so that max |N| = 1."""
    from scipy.ndimage import gaussian_filter1d
    n = rng.standard_normal((ny, nx)).astype(dtype, copy=False)
    n = gaussian_filter1d(n, sigma_cells, axis=1, mode="reflect")
    n = gaussian_filter1d(n, sigma_cells, axis=0, mode="reflect")
    m = float(np.max(np.abs(n)))
    if m > 0:
        n /= m
    return n


def basin_hump(nx: int = 64, ny: int = 64, amp: float = 0.1, sigma_cells: float = 5.0,
               depth: float = 1.0, manning_n: float = 0.03, kappa: float = 0.0) -> dict:
    """Closed square basin, flat bed, still depth plus a Gaussian hump centred
    at the domain centre (so the hump is mirror-symmetric in x and y)."""
    x, y = _cell_centres(nx, ny)
    r2 = (x[None, :] - nx / 2.0) ** 2 + (y[:, None] - ny / 2.0) ** 2
    eta = depth + amp * np.exp(-r2 / (2.0 * sigma_cells ** 2))
    z = np.zeros((ny, nx))
    return dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=np.zeros_like(z),
                v=np.zeros_like(z), manning_n=manning_n, kappa=kappa,
                bc=(WALL, WALL, WALL, WALL), q_in=(0.0, 0.0, 0.0, 0.0))


def dam_break(nx: int = 2048, ny: int = 2048, seed: int = 1310, level: float = 10.0,
              manning_n: float = 0.035, kappa: float = 0.25, n_bumps: int = 32) -> dict:
    """Dam break over a bumpy bed: bed = sum of Gaussians (heights U(0,2) m,
    widths U(20,200) cells at 2048^2, scaled with the grid); water level
    `level` on the left half (eta = max(level, z)), dry right half (eta = z);
    walls on every side."""
    rng = _rng(seed)
    s = min(nx, ny) / 2048.0
    z = gaussian_sum_bed(nx, ny, rng, n_bumps, (0.0, 2.0), (20.0 * s, 200.0 * s))
    eta = z.copy()
    left = np.arange(nx) < nx // 2
    eta[:, left] = np.maximum(level, z[:, left])
    return dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=np.zeros_like(z),
                v=np.zeros_like(z), manning_n=manning_n, kappa=kappa,
                bc=(WALL, WALL, WALL, WALL), q_in=(0.0, 0.0, 0.0, 0.0))


def river(nx: int = 8192, ny: int = 8192, seed: int = 1311, slope: float = 1e-3,
          noise_amp: float = 0.5, noise_sigma: float = 16.0, depth: float = 1.0,
          q_in: float = 2.0, manning_n: float = 0.03, kappa: float = 0.25) -> dict:
    """River reach: bed sloping `slope` along x plus smooth seeded noise of
    amplitude `noise_amp`; uniform initial depth; inflow discharge q_in on the
    west side, free outflow east, walls south and north."""
    rng = _rng(seed)
    x, _ = _cell_centres(nx, ny)
    z = smooth_noise(nx, ny, rng, noise_sigma)
    z *= noise_amp
    z += (-slope * x)[None, :]
    eta = z + depth
    return dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=np.zeros_like(z),
                v=np.zeros_like(z), manning_n=manning_n, kappa=kappa,
                bc=(INFLOW, OUTFLOW, WALL, WALL), q_in=(q_in, 0.0, 0.0, 0.0))


def ensemble(count: int = 256, seed: int = 1312, side=(128, 1024), kappa: float = 0.25) -> list:
    """Batch of dam-break scenarios of uneven size: Nx, Ny ~ U{side}, flat
    bed, dam at Nx/2 with level H ~ U(2,10) m on the left and dry ground on
    the right, Manning n ~ U(0.01, 0.05), walls."""
    rng = _rng(seed)
    nxs = rng.integers(side[0], side[1] + 1, count)
    nys = rng.integers(side[0], side[1] + 1, count)
    ns = rng.uniform(0.01, 0.05, count)
    hs = rng.uniform(2.0, 10.0, count)
    out = []
    for k in range(count):
        nx, ny = int(nxs[k]), int(nys[k])
        z = np.zeros((ny, nx))
        eta = np.zeros((ny, nx))
        eta[:, : nx // 2] = hs[k]
        out.append(dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=np.zeros_like(z),
                        v=np.zeros_like(z), manning_n=float(ns[k]), kappa=kappa,
                        bc=(WALL, WALL, WALL, WALL), q_in=(0.0, 0.0, 0.0, 0.0),
                        dam_height=float(hs[k])))
    return out


def adjoint_case(nx: int = 512, ny: int = 512, seed: int = 1313, n_gauges: int = 16,
                 n0: float = 0.03) -> dict:
    """Gaussian-hump basin on a bumpy bed, fully wet: bed = sum of 32
    Gaussians (U(0,0.5) m, widths U(10,50) cells at 512^2, scaled), still
    level max(z) + 1 m plus a 0.1 m hump of sigma 16 cells (scaled) at the
    centre; true Manning field n0 (1 + 0.2 N) with N smooth noise; gauges
    uniform at least 2 cells from the walls."""
    rng = _rng(seed)
    s = min(nx, ny) / 512.0
    z = gaussian_sum_bed(nx, ny, rng, 32, (0.0, 0.5), (10.0 * s, 50.0 * s))
    x, y = _cell_centres(nx, ny)
    r2 = (x[None, :] - nx / 2.0) ** 2 + (y[:, None] - ny / 2.0) ** 2
    sig = 16.0 * s
    eta = float(z.max()) + 1.0 + 0.1 * np.exp(-r2 / (2.0 * sig ** 2))
    noise = smooth_noise(nx, ny, rng, max(2.0, 16.0 * s))
    n_true = n0 * (1.0 + 0.2 * noise)
    gi = rng.integers(2, nx - 2, n_gauges)
    gj = rng.integers(2, ny - 2, n_gauges)
    gauges = (gj * nx + gi).astype(np.int64)
    return dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=np.zeros_like(z),
                v=np.zeros_like(z), manning_n=n0, kappa=0.0, n_true=n_true,
                bc=(WALL, WALL, WALL, WALL), q_in=(0.0, 0.0, 0.0, 0.0), gauges=gauges)


def large_river(nx: int, ny: int, seed: int = 1314, chunk_rows: int = 2048) -> dict:
    """A river reach too large for the filtered-noise generator: bed sloping
    1e-3 along x plus three seeded sinusoidal undulations (0.3, 0.1 and
    0.05 m), depth 1 m plus a 0.05 m long wave, u = 0.1 sin(.), v = 0; inflow
    2 m^2/s west, outflow east, walls south/north, n = 0.03, kappa = 0.25.
    Arrays are FP32 (ny x nx), built row block by row block to bound the
    host memory; the same seed gives the same arrays."""
    rng = _rng(seed)
    ph = rng.uniform(0.0, 2.0 * np.pi, 6)
    shape = (ny, nx)
    z = np.empty(shape, np.float32)
    eta = np.empty(shape, np.float32)
    u = np.empty(shape, np.float32)
    v = np.zeros(shape, np.float32)
    x = (np.arange(nx) + 0.5)[None, :]
    for j0 in range(0, ny, chunk_rows):
        j1 = min(ny, j0 + chunk_rows)
        y = (np.arange(j0, j1) + 0.5)[:, None]
        zz = (-1e-3 * x + 0.3 * np.sin(2 * np.pi * x / 1500.0 + ph[0]) * np.sin(2 * np.pi * y / 900.0 + ph[1])
              + 0.1 * np.sin(2 * np.pi * (x + y) / 377.0 + ph[2]) + 0.05 * np.sin(2 * np.pi * (x - y) / 131.0 + ph[3]))
        z[j0:j1] = zz
        eta[j0:j1] = zz + 1.0 + 0.05 * np.sin(2 * np.pi * x / 2000.0 + ph[4])
        u[j0:j1] = 0.1 * np.sin(2 * np.pi * y / 700.0 + ph[5]) + 0.0 * x
    return dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=u, v=v, manning_n=0.03, kappa=0.25,
                bc=(INFLOW, OUTFLOW, WALL, WALL), q_in=(2.0, 0.0, 0.0, 0.0))


def with_cell_size(case: dict, dx: float, dy: float) -> dict:
    """The same arrays and settings on cells of dx by dy metres (the arrays
    are given per cell, so only the two sizes change)."""
    out = dict(case)
    out["dx"], out["dy"] = float(dx), float(dy)
    return out


def open_river(nx: int, ny: int, seed: int = 1315, q_w: float = 2.0, q_s: float = 1.0) -> dict:
    """River reach open on all four sides: inflow q_w through the west side
    and q_s through the south side, free outflow east and north (every side
    carries water), otherwise as `river`."""
    c = river(nx, ny, seed=seed)
    c["bc"] = (INFLOW, OUTFLOW, INFLOW, OUTFLOW)
    c["q_in"] = (q_w, 0.0, q_s, 0.0)
    return c


def drying_shoals(nx: int = 300, ny: int = 90, depth: float = 0.5, freeboard: float = 0.004,
                  u0: float = 0.3, q_in: float = 0.15, manning_n: float = 0.03, kappa: float = 0.25) -> dict:
    """A channel wet everywhere at the start whose shoals dry out as the
    water flows over them: flat bed with four Gaussian shoals (the highest
    point `freeboard` below the still surface), uniform depth `depth`, current
    u0 eastwards, inflow q_in on the west side, free outflow east, walls south
    and north.  Positions and widths are fixed fractions of the grid."""
    x, y = _cell_centres(nx, ny)
    z = np.zeros((ny, nx))
    for fx, fy, fs in ((0.27, 0.33, 0.13), (0.5, 0.67, 0.11), (0.73, 0.39, 0.16), (0.4, 0.78, 0.09)):
        cx, cy, s = fx * nx, fy * ny, fs * ny
        g = np.exp(-((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2) / (2.0 * s * s))
        z = np.maximum(z, (depth - freeboard) * g)
    eta = np.full((ny, nx), depth)
    return dict(nx=nx, ny=ny, dx=1.0, dy=1.0, z=z, eta=eta, u=np.full((ny, nx), u0),
                v=np.zeros((ny, nx)), manning_n=manning_n, kappa=kappa,
                bc=(INFLOW, OUTFLOW, WALL, WALL), q_in=(q_in, 0.0, 0.0, 0.0))

