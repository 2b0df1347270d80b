"""Row-strip decomposition of one domain over several contexts (the paper's
Sec. 6.1 proposal for several GPUs, here on one): every strip steps its own
rows plus two halo rows per cut side; between steps the halos are refreshed
from the neighbours and the CFL maxima are combined.  The own rows and the
step sizes must equal the undecomposed domain's bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import gpu_solver

pytestmark = pytest.mark.gpu

H = 2  # halo rows per cut side: the step's dependency radius in rows


def _strip_case(case, r0, r1, south_cut, north_cut):
    sub = dict(case)
    sub["ny"] = r1 - r0
    for f in ("z", "eta", "u", "v"):
        sub[f] = np.ascontiguousarray(case[f][r0:r1])
    bc = list(case["bc"])
    if south_cut:
        bc[2] = 2  # any condition: it only reaches halo rows
    if north_cut:
        bc[3] = 0
    sub["bc"] = tuple(bc)
    return sub


@pytest.mark.parametrize("nstrips", [2, 3])
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["dambreak", "river"])
def test_strips_equal_one_domain(name, precision, kernel, nstrips):
    from paper_1309_1230_gb300 import swe
    case = I.dam_break(150, 97, seed=5) if name == "dambreak" else I.river(140, 89, seed=6)
    steps = 60
    one = gpu_solver(case, precision, kernel)
    info1, dts1 = one.step(steps, want_dt=True)
    ref = one.get_state()
    one.close()

    ny = case["ny"]
    cuts = [round(ny * q / nstrips) + (q % 2) for q in range(nstrips + 1)]
    cuts[0], cuts[-1] = 0, ny
    strips, own = [], []
    for q in range(nstrips):
        lo, hi = cuts[q], cuts[q + 1]
        r0, r1 = max(0, lo - H), min(ny, hi + H)
        s = gpu_solver(_strip_case(case, r0, r1, q > 0, q < nstrips - 1), precision, kernel)
        s.set_own_rows(lo - r0, hi - r0)
        strips.append((s, r0, r1))
        own.append((lo, hi))
    swe.cfl_combine([s for s, _, _ in strips])
    dts = []
    for k in range(steps):
        d = None
        for s, _, _ in strips:
            _, dd = s.step(1, want_dt=True)
            d = dd if d is None else d
            assert dd[0] == d[0]
        dts.append(d[0])
        for q in range(nstrips - 1):
            (a, a0, a1), (b, b0, b1) = strips[q], strips[q + 1]
            cut = cuts[q + 1]
            b.copy_rows_from(a, cut - H - a0, cut - H - b0, H)  # b's south halo
            a.copy_rows_from(b, cut - b0, cut - a0, H)          # a's north halo
        swe.cfl_combine([s for s, _, _ in strips])
    assert np.array_equal(np.array(dts), dts1)
    vol = 0.0
    for (s, r0, _), (lo, hi) in zip(strips, own):
        st = s.get_state()
        for a, b in zip(st, ref):
            assert np.array_equal(a[lo - r0:hi - r0], b[lo:hi]), (name, lo, hi)
        vol += s.info().volume
        s.close()
    assert vol == pytest.approx(info1.volume, rel=1e-12)
