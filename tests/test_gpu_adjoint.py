"""GPU discrete adjoint: against the FP64 oracle's adjoint (1e-10 relative),
against central differences of the GPU's own forward runs with the same
frozen step sizes (1e-5 relative, FP64), FP32 against FP64, checkpoint
spacing not changing the result, and the torch.autograd.Function."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(nx=32, ny=28, seed=4, bc=(0, 0, 0, 0), q_in=(0.0,) * 4):
    c = I.adjoint_case(nx, ny, seed=seed, n_gauges=6)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    c["u"] = 0.05 * rng.standard_normal((ny, nx))
    c["v"] = 0.05 * rng.standard_normal((ny, nx))
    c["bc"], c["q_in"] = bc, q_in
    nfield = 0.03 * (1.0 + 0.2 * rng.uniform(-1, 1, (ny, nx)))
    return c, nfield


def _solver(c, nfield, precision):
    from paper_1309_1230_gb300 import swe
    s = swe.Solver(c["nx"], c["ny"], dx=c["dx"], dy=c["dy"], manning_n=0.03, kappa=0.0, bc=c["bc"], q_in=c["q_in"],
                   precision=precision)
    s.set_bed(c["z"], nfield)
    s.set_state(c["eta"], c["u"], c["v"])
    return s


def _obs(c, T, seed=9):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([c["eta"].ravel()[c["gauges"]] + 0.01 * rng.standard_normal(len(c["gauges"])) for _ in range(T)])


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("bcs", ["walls", "open", "open_aniso"])
def test_gpu_adjoint_matches_oracle_adjoint(oracle, bcs):
    """32 x 28 cells, 40 steps; "open_aniso" on cells of 0.7 m by 1.9 m."""
    from paper_1309_1230_gb300 import swe
    bc, q = ((0, 0, 0, 0), (0.0,) * 4) if bcs == "walls" else ((1, 2, 0, 2), (0.4, 0.0, 0.0, 0.0))
    c, nfield = _case(bc=bc, q_in=q)
    if bcs == "open_aniso":
        c = I.with_cell_size(c, 0.7, 1.9)
    T = 40
    obs = _obs(c, T)
    s = _solver(c, nfield, swe.SWE_FP64)
    loss, gn, ge, gz = s.adjoint(T, c["gauges"], obs, with_bed=True)
    s.close()
    p = oracle.Params(nx=c["nx"], ny=c["ny"], dx=c["dx"], dy=c["dy"], manning_n=0.03, kappa=0.0, bc=bc, q_in=q)
    fwd = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], T, nfield=nfield)
    ref = oracle.adjoint(p, c["z"], nfield, c["eta"], c["u"], c["v"], fwd.dt, c["gauges"], obs)
    assert ref.status == 0
    assert loss == pytest.approx(ref.loss, rel=1e-10)
    assert _rel(gn, ref.grad_n) <= 1e-10
    assert _rel(ge, ref.grad_eta0) <= 1e-10
    assert np.abs(ref.grad_z).max() > 0.0
    assert _rel(gz, ref.grad_z) <= 1e-10


def test_gpu_adjoint_on_the_512_grid_matches_oracle_adjoint(oracle):
    """The adjoint workload's own grid: 512 x 512 cells, Gaussian-sum bed,
    fully wet, kappa 0, gradient at the uniform n = 0.03, over 120 steps (the
    oracle keeps every forward state, 0.95 GB at this size) with the default
    sqrt(T) checkpoints (11).  In 120 steps the hump's wave travels about 30
    cells, so 8 gauges within 24 cells of the centre join the 16 uniform ones
    (otherwise no gauge sees moving water and the Manning gradient is zero).
    FP64 against the oracle's adjoint at 1e-10; FP32 against FP64 within
    2e-4 of each gradient's scale."""
    from paper_1309_1230_gb300 import swe
    c = I.adjoint_case(512, 512)
    T = 120
    rng = np.random.Generator(np.random.PCG64(512))
    gi, gj = rng.integers(256 - 24, 256 + 24, 8), rng.integers(256 - 24, 256 + 24, 8)
    c["gauges"] = np.concatenate([c["gauges"], gj * 512 + gi]).astype(np.int64)
    nfield = np.full((512, 512), 0.03)
    obs = _obs(c, T, seed=21)
    res = {}
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        s = _solver(c, nfield, prec)
        res[prec] = s.adjoint(T, c["gauges"], obs, with_bed=True)
        s.close()
    loss, gn, ge, gz = res[swe.SWE_FP64]
    p = oracle.Params(nx=512, ny=512, manning_n=0.03, kappa=0.0)
    fwd = oracle.run(p, c["z"], c["eta"], c["u"], c["v"], T, nfield=nfield, nthreads=8)
    ref = oracle.adjoint(p, c["z"], nfield, c["eta"], c["u"], c["v"], fwd.dt, c["gauges"], obs)
    assert ref.status == 0
    assert loss == pytest.approx(ref.loss, rel=1e-10)
    assert _rel(gn, ref.grad_n) <= 1e-10
    assert _rel(ge, ref.grad_eta0) <= 1e-10
    assert _rel(gz, ref.grad_z) <= 1e-10
    for g in (gn, ge, gz):  # no gradient is trivial: each spreads over thousands of cells
        assert np.count_nonzero(np.abs(g) > 1e-6 * np.max(np.abs(g))) > 1000
    l32, gn32, ge32, gz32 = res[swe.SWE_FP32]
    assert l32 == pytest.approx(loss, rel=1e-5)
    errs = (_rel(gn32, gn), _rel(ge32, ge), _rel(gz32, gz))
    assert max(errs) <= 2e-4, errs


def test_gpu_adjoint_matches_central_differences():
    from paper_1309_1230_gb300 import swe
    c, nfield = _case()
    T = 40
    obs = _obs(c, T)
    s = _solver(c, nfield, swe.SWE_FP64)
    _, dts = s.step(T, want_dt=True)
    s.close()
    s = _solver(c, nfield, swe.SWE_FP64)
    loss, gn, ge, gz = s.adjoint(T, c["gauges"], obs, with_bed=True)
    s.close()

    def L(nf, eta, z=None):
        q = swe.Solver(c["nx"], c["ny"], manning_n=0.03, kappa=0.0, precision=swe.SWE_FP64)
        q.set_bed(c["z"] if z is None else z, nf)
        q.set_state(eta, c["u"], c["v"])
        tot = 0.0
        for k in range(T):
            q.step(1, dt_fixed=dts[k:k + 1], want_info=False)
            e, _, _ = q.get_state()
            r = e.ravel()[c["gauges"]] - obs[k]
            tot += 0.5 * float(r @ r)
        q.close()
        return tot

    assert loss == pytest.approx(L(nfield, c["eta"]), rel=1e-12)
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(3):
        dn = rng.standard_normal(nfield.shape) * 0.003
        de = rng.standard_normal(nfield.shape) * 0.01
        eps = 1e-5
        fd = (L(nfield + eps * dn, c["eta"] + eps * de) - L(nfield - eps * dn, c["eta"] - eps * de)) / (2 * eps)
        ad = float(np.sum(gn * dn) + np.sum(ge * de))
        assert abs(fd - ad) <= 1e-5 * abs(fd), (fd, ad)
    for _ in range(2):  # the bed, with the initial elevation held
        dz = rng.standard_normal(nfield.shape) * 0.01
        eps = 1e-5
        fd = (L(nfield, c["eta"], c["z"] + eps * dz) - L(nfield, c["eta"], c["z"] - eps * dz)) / (2 * eps)
        ad = float(np.sum(gz * dz))
        assert abs(fd - ad) <= 1e-5 * abs(fd), ("bed", fd, ad)


def test_gpu_adjoint_fp32_and_checkpoint_spacing():
    from paper_1309_1230_gb300 import swe
    c, nfield = _case()
    T = 40
    obs = _obs(c, T)
    res = {}
    for prec, every in ((swe.SWE_FP64, 0), (swe.SWE_FP64, 1), (swe.SWE_FP64, 7), (swe.SWE_FP32, 0)):
        s = _solver(c, nfield, prec)
        res[(prec, every)] = s.adjoint(T, c["gauges"], obs, checkpoint_every=every)
        s.close()
    a = res[(swe.SWE_FP64, 0)]
    for every in (1, 7):  # same arithmetic, other checkpoints: bitwise
        b = res[(swe.SWE_FP64, every)]
        assert b[0] == a[0] and np.array_equal(b[1], a[1]) and np.array_equal(b[2], a[2])
    # FP32 against FP64: measured 1.1e-6 (loss), 3.8e-6 (grad n) and 1.8e-5
    # (grad eta0) here, at most 2.1e-5 up to 512^2 x 400 steps; bounds 10x that
    f = res[(swe.SWE_FP32, 0)]
    assert f[0] == pytest.approx(a[0], rel=1e-5)
    assert _rel(f[1], a[1]) <= 2e-4 and _rel(f[2], a[2]) <= 2e-4


def test_autograd_function():
    import torch
    from paper_1309_1230_gb300 import autograd as A
    c, nfield = _case()
    T = 20
    obs = _obs(c, T)
    n_t = torch.tensor(nfield, dtype=torch.float64, requires_grad=True)
    e_t = torch.tensor(c["eta"], dtype=torch.float64, requires_grad=True)
    z_t = torch.tensor(c["z"], dtype=torch.float64, requires_grad=True)
    loss = A.gauge_misfit(n_t, e_t, c, T, c["gauges"], obs, bed=z_t)
    loss.backward()
    from paper_1309_1230_gb300 import swe
    s = _solver(c, nfield, swe.SWE_FP64)
    l2, gn, ge, gz = s.adjoint(T, c["gauges"], obs, with_bed=True)
    s.close()
    assert float(loss.detach()) == l2
    assert np.array_equal(n_t.grad.numpy(), gn) and np.array_equal(e_t.grad.numpy(), ge)
    assert np.array_equal(z_t.grad.numpy(), gz)
    # without a bed tensor the case's bed is used and no bed gradient is asked for
    n2 = torch.tensor(nfield, dtype=torch.float64, requires_grad=True)
    l3 = A.gauge_misfit(n2, torch.tensor(c["eta"], dtype=torch.float64), c, T, c["gauges"], obs)
    l3.backward()
    assert float(l3.detach()) == l2 and np.array_equal(n2.grad.numpy(), gn)


def test_gpu_bed_gradient_of_a_lake_at_rest_is_zero():
    """A lake at rest stays at rest over any submerged bed: with gauge records
    1 cm off the surface the loss is positive, yet the bed and Manning
    gradients are exactly zero (FP64 and FP32)."""
    from paper_1309_1230_gb300 import swe
    c, nfield = _case()
    c["eta"] = np.full_like(c["eta"], float(c["z"].max()) + 1.0)
    c["u"] = np.zeros_like(c["eta"])
    c["v"] = np.zeros_like(c["eta"])
    T = 15
    obs = np.full((T, len(c["gauges"])), c["eta"][0, 0] + 0.01)
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        s = _solver(c, nfield, prec)
        loss, gn, ge, gz = s.adjoint(T, c["gauges"], obs, with_bed=True)
        s.close()
        assert loss > 0.0 and np.abs(ge).max() > 0.0
        assert not gz.any() and not gn.any()


def test_gpu_adjoint_rejects_runs_outside_its_regime():
    """The adjoint differentiates the fully wet, kappa = 0 step: a dry cell
    anywhere in the run, or dissipation, is refused (SWE_ERR_UNSUPPORTED)."""
    from paper_1309_1230_gb300 import swe
    c, nfield = _case()
    T = 10
    obs = _obs(c, T)
    c_dry = dict(c)
    c_dry["eta"] = c["eta"].copy()
    c_dry["eta"][5, 7] = c["z"][5, 7]
    for prec in (swe.SWE_FP64, swe.SWE_FP32):
        s = _solver(c_dry, nfield, prec)
        with pytest.raises(swe.SweError) as ei:
            s.adjoint(T, c["gauges"], obs)
        assert ei.value.status == swe.SWE_ERR_UNSUPPORTED
        s.close()
    s = swe.Solver(c["nx"], c["ny"], manning_n=0.03, kappa=0.25, precision=swe.SWE_FP64)
    s.set_bed(c["z"], nfield)
    s.set_state(c["eta"], c["u"], c["v"])
    with pytest.raises(swe.SweError) as ei:
        s.adjoint(T, c["gauges"], obs)
    assert ei.value.status == swe.SWE_ERR_UNSUPPORTED
    s.close()


def test_calibration_recovers_the_gauge_records():
    """L-BFGS over log n with the adjoint's gradient (the calibration loop):
    starting from a uniform field, the misfit against records made with a
    spatially varying field falls at least tenfold."""
    from paper_1309_1230_gb300 import calibrate as C
    c = I.adjoint_case(48, 40, seed=8, n_gauges=12)
    c["dt_max"] = 0.25  # below the CFL step: the same step sizes in every run
    T = 120
    obs = C.gauge_series(c, c["n_true"], T, c["gauges"])
    n0 = np.full_like(c["n_true"], 0.03)
    loss0 = float(np.sum((C.gauge_series(c, n0, T, c["gauges"]) - obs) ** 2) / 2)
    n_fit, hist = C.calibrate_manning(c, c["gauges"], obs, T, n0, iters=20)
    assert hist[0] == pytest.approx(loss0, rel=1e-9)
    assert min(hist) <= 0.1 * hist[0], hist[:3] + hist[-3:]
    assert np.all(n_fit > 0)


def test_bed_calibration_recovers_the_gauge_records():
    """L-BFGS over the bed with the adjoint's dL/dz: records made over a bed
    with an added smooth 10 cm mound; starting from the bed without it, the
    misfit falls at least tenfold."""
    from paper_1309_1230_gb300 import calibrate as C
    c = I.adjoint_case(48, 40, seed=8, n_gauges=12)
    c["dt_max"] = 0.25  # below the CFL step: the same step sizes in every run
    T = 120
    x, y = np.meshgrid(np.arange(48) + 0.5, np.arange(40) + 0.5)
    z_true = c["z"] + 0.1 * np.exp(-((x - 20.0) ** 2 + (y - 22.0) ** 2) / (2 * 6.0 ** 2))
    n = np.full_like(c["z"], 0.03)
    obs = C.gauge_series(c, n, T, c["gauges"], bed=z_true)
    z_fit, hist = C.calibrate_bed(c, c["gauges"], obs, T, c["z"], n, iters=20)
    assert min(hist) <= 0.1 * hist[0], hist[:3] + hist[-3:]
    assert np.all(z_fit < c["eta"] - 1e-3)
