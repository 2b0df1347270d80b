"""The ablation forms on the GPU (explicit friction; the TVD-MacCormack term in
place of S15's switch): the plain kernel against the FP64 oracle running the
same forms (FP64 1e-10, FP32 at the FP32 bounds), bitwise equality of the
paper-layout kernels (row blocks and 16 x 16 shared-memory blocks) with the
plain kernel, and SWE_ERR_UNSUPPORTED from the paths that do not run them."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import assert_fp32_close, gpu_solver, oracle_params, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "dambreak": (lambda: I.dam_break(160, 70, seed=3), 200),
    "river": (lambda: I.river(150, 60, seed=7), 200),
    "aniso": (lambda: I.with_cell_size(I.open_river(90, 50, seed=17), 0.7, 1.9), 150),
}
FORMS = [(1, 0), (0, 1), (1, 1)]


def _oracle(oracle, case, steps, friction, dissipation):
    p = oracle_params(oracle, case, friction=friction, dissipation=dissipation)
    e0, u0, v0 = oracle.prepare_state(p, case["z"], case["eta"], case["u"], case["v"])
    ref = oracle.run(p, case["z"], e0, u0, v0, steps, nthreads=4)
    assert ref.status == 0
    return ref


def _gpu(case, precision, kernel, steps, friction, dissipation, dt_fixed=None):
    s = gpu_solver(case, precision, kernel, friction=friction, dissipation=dissipation)
    info, dts = s.step(steps, dt_fixed=dt_fixed, want_dt=True)
    e, u, v = s.get_state()
    s.close()
    return info, dts, e, u, v


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_plain_ablation_forms_match_the_oracle(oracle, name, form):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    ref = _oracle(oracle, case, steps, *form)
    info, dts, e, u, v = _gpu(case, swe.SWE_FP64, swe.SWE_KERNEL_PLAIN, steps, *form)
    z = case["z"]
    assert rel_err(dts, ref.dt) <= 1e-10
    assert rel_err(e - z, ref.eta - z) <= 1e-10
    assert rel_err(u, ref.u, 1e-3) <= 1e-9 and rel_err(v, ref.v, 1e-3) <= 1e-9
    assert info.clamp_volume == pytest.approx(ref.clamp_volume, rel=1e-8, abs=1e-9)
    assert np.allclose(info.bflux, ref.bflux, rtol=1e-9, atol=1e-9)
    info, dts, e, u, v = _gpu(case, swe.SWE_FP32, swe.SWE_KERNEL_PLAIN, steps, *form)
    assert_fp32_close(e, u, v, ref.eta, ref.u, ref.v, z)
    assert rel_err(dts, ref.dt) <= 1e-4


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("form", FORMS)
def test_paper_layouts_run_the_ablation_forms_bitwise(precision, form):
    from paper_1309_1230_gb300 import swe
    case = CASES["dambreak"][0]()
    steps = 80
    _, dts, *plain = _gpu(case, precision, swe.SWE_KERNEL_PLAIN, steps, *form)
    for kern in (swe.SWE_KERNEL_PAPER_DEVDT, swe.SWE_KERNEL_PAPER_SHARED_DEVDT, swe.SWE_KERNEL_PAPER_SHARED):
        fixed = dts if kern == swe.SWE_KERNEL_PAPER_SHARED else None
        _, d2, *other = _gpu(case, precision, kern, steps, *form, dt_fixed=fixed)
        assert np.array_equal(d2, dts), kern
        for a, b in zip(other, plain):
            assert np.array_equal(a, b), kern


def test_ablation_forms_are_refused_where_not_run():
    from paper_1309_1230_gb300 import swe
    case = CASES["dambreak"][0]()
    for form in FORMS:
        with pytest.raises(swe.SweError) as ei:
            swe.Solver(case["nx"], case["ny"], kernel=swe.SWE_KERNEL_FUSED, friction=form[0], dissipation=form[1])
        assert ei.value.status == swe.SWE_ERR_UNSUPPORTED
        with pytest.raises(swe.SweError) as ei:
            swe.Batch([(40, 30)], [0.03], friction=form[0], dissipation=form[1])
        assert ei.value.status == swe.SWE_ERR_UNSUPPORTED
    c = I.adjoint_case(24, 20, n_gauges=3)
    s = swe.Solver(24, 20, manning_n=0.03, kernel=swe.SWE_KERNEL_PLAIN, friction=1)
    s.set_bed(c["z"])
    s.set_state(c["eta"], c["u"], c["v"])
    with pytest.raises(swe.SweError) as ei:
        s.adjoint(3, c["gauges"], np.zeros((3, 3)))
    assert ei.value.status == swe.SWE_ERR_UNSUPPORTED
    s.close()
    with pytest.raises(swe.SweError) as ei:
        swe.Solver(8, 8, friction=2, kernel=swe.SWE_KERNEL_PLAIN)
    assert ei.value.status == swe.SWE_ERR_ARG
