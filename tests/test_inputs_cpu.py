"""The seeded input generators: the same seed gives the same arrays, and each
workload has the shape, sizes, value ranges and structure its docstring
states (the recipe the parity tests and the benchmark rely on).  No GPU and
no scheme arithmetic: these check the inputs only."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I

FIELDS = ("z", "eta", "u", "v")


def _same(a: dict, b: dict) -> bool:
    return all(np.array_equal(a[f], b[f]) for f in FIELDS)


@pytest.mark.parametrize("make", [
    lambda s: I.dam_break(96, 64, seed=s),
    lambda s: I.river(128, 48, seed=s),
    lambda s: I.adjoint_case(64, 64, seed=s),
    lambda s: I.large_river(200, 70, seed=s, chunk_rows=16),
])
def test_seeded_and_repeatable(make):
    a, b, c = make(5), make(5), make(6)
    assert _same(a, b)
    assert not _same(a, c)
    for f in FIELDS:
        assert a[f].shape == (a["ny"], a["nx"])
        assert np.isfinite(a[f]).all()


def test_river_recipe():
    c = I.river(256, 96, seed=3)
    x = np.arange(c["nx"]) + 0.5
    noise = c["z"] + 1e-3 * x[None, :]
    assert np.max(np.abs(noise)) == pytest.approx(0.5, rel=1e-12)   # amplitude 0.5 m, max |N| = 1
    assert np.allclose(c["eta"] - c["z"], 1.0, rtol=0, atol=1e-12)  # uniform depth 1 m
    assert not c["u"].any() and not c["v"].any()
    assert c["bc"] == (I.INFLOW, I.OUTFLOW, I.WALL, I.WALL) and c["q_in"][0] == 2.0
    assert c["kappa"] == 0.25 and c["manning_n"] == 0.03
    # smooth: the filtered noise changes little from cell to cell
    assert np.max(np.abs(np.diff(noise, axis=1))) < 0.1


def test_large_river_rows_do_not_depend_on_the_chunking():
    a = I.large_river(150, 77, seed=9, chunk_rows=8)
    b = I.large_river(150, 77, seed=9, chunk_rows=77)
    assert _same(a, b)
    assert a["z"].dtype == np.float32
    assert np.all(a["eta"] - a["z"] > 0.9)


def test_dam_break_recipe():
    c = I.dam_break(200, 120, seed=4)
    nx = c["nx"]
    left = np.arange(nx) < nx // 2
    assert np.array_equal(c["eta"][:, ~left], c["z"][:, ~left])            # dry right half
    assert np.array_equal(c["eta"][:, left], np.maximum(10.0, c["z"][:, left]))
    assert c["z"].min() >= 0.0 and c["z"].max() <= 2.0 * 32
    assert c["bc"] == (I.WALL,) * 4


def test_basin_hump_is_mirror_symmetric():
    c = I.basin_hump(64, 64)
    e = c["eta"]
    assert np.array_equal(e, e[:, ::-1]) and np.array_equal(e, e[::-1, :]) and np.array_equal(e, e.T)
    assert e.max() == pytest.approx(1.0 + 0.1, abs=2e-3) and e.min() >= 1.0


def test_ensemble_recipe():
    cases = I.ensemble(256)
    assert len(cases) == 256
    for c in cases:
        nx, ny = c["nx"], c["ny"]
        assert 128 <= nx <= 1024 and 128 <= ny <= 1024
        assert 0.01 <= c["manning_n"] <= 0.05
        h = c["dam_height"]
        assert 2.0 <= h <= 10.0
        assert np.all(c["eta"][:, : nx // 2] == h) and not c["eta"][:, nx // 2:].any()
        assert not c["z"].any()
    sizes = {(c["nx"], c["ny"]) for c in cases}
    assert len(sizes) > 200  # uneven sizes


def test_adjoint_case_recipe():
    c = I.adjoint_case(128, 96, seed=2)
    nx, ny = c["nx"], c["ny"]
    g = c["gauges"]
    gi, gj = g % nx, g // nx
    assert np.all((gi >= 2) & (gi < nx - 2) & (gj >= 2) & (gj < ny - 2))
    assert np.all(c["eta"] - c["z"] >= 1.0 - 1e-12)                        # fully wet
    rel = c["n_true"] / c["manning_n"] - 1.0
    assert np.max(np.abs(rel)) == pytest.approx(0.2, rel=1e-12)            # n0 (1 + 0.2 N), max |N| = 1
    assert c["kappa"] == 0.0
