"""The checked build (compiled with SWE_CHECKED): the fused and batched row
steps check every shared-memory row and column they read in the ring, every
global store, every per-cell Manning load and every TMA coordinate's 16-byte
alignment; a failed check sets SWE_FLAG_CHECK (SWE_ERR_CHECK from the step)
and the access is made safe instead, so nothing traps.  The planes are NaN in
every byte until set, so that a read of a plane's padding or of a cell never
written shows as a non-finite state.  compute-sanitizer being closed on this
pool, these runs are the memory-safety check of the hot path: on grids of
ragged, degenerate and anisotropic shapes, every sweep direction, the all-wet
pass with its fallback, several rows per item and the batched form, the
checked build must report no failed check and give the normal build's state
bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1309_1230_gb300 import inputs as I
from tests.gpu_util import gpu_solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked_lib():
    from paper_1309_1230_gb300 import swe
    return swe.load_checked()


CASES = {
    "ragged": (lambda: I.dam_break(37, 23, seed=11), 120),
    "tall": (lambda: I.dam_break(9, 140, seed=12), 80),
    "one_cell": (lambda: I.dam_break(1, 1, seed=1, n_bumps=4), 20),
    "row": (lambda: I.dam_break(130, 5, seed=2, n_bumps=4), 40),
    "col": (lambda: I.dam_break(3, 3, seed=3, n_bumps=4), 30),
    "river125": (lambda: I.river(125, 60, seed=7), 120),
    "aniso_river": (lambda: I.with_cell_size(I.open_river(150, 70, seed=7), 0.7, 1.9), 120),
    "shoals": (lambda: I.drying_shoals(300, 90), 300),
}


def _run(case, precision, steps, lib=None, **kw):
    from paper_1309_1230_gb300 import swe
    s = gpu_solver(case, precision, swe.SWE_KERNEL_FUSED, lib=lib, **kw)
    info, dts = s.step(steps, want_dt=True)
    out = s.get_state()
    s.close()
    return info, dts, out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_checked_fused_matches_and_passes_checks(checked_lib, name, precision):
    from paper_1309_1230_gb300 import swe
    build, steps = CASES[name]
    case = build()
    for kw in ({}, {"seg_rows": 16}, {"dir_cycle": 3}):  # dir_cycle 3: the other two sweep directions
        ref = _run(case, precision, steps, **kw)
        chk = _run(case, precision, steps, lib=checked_lib, **kw)  # raises SweError on SWE_ERR_CHECK
        assert not (chk[0].flags & swe.SWE_FLAG_CHECK)
        assert np.array_equal(chk[1], ref[1])
        for a, b in zip(chk[2], ref[2]):
            assert np.array_equal(a, b)


def test_checked_batch_matches_and_passes_checks(checked_lib):
    from paper_1309_1230_gb300 import swe
    cases = I.ensemble(6, seed=31, side=(37, 131))
    sizes = [(c["nx"], c["ny"]) for c in cases]
    n = [c["manning_n"] for c in cases]

    def run(lib):
        b = swe.Batch(sizes, n, lib=lib, kappa=0.25, seg_rows=32)
        for i, c in enumerate(cases):
            b.set_bed(i, c["z"])
            b.set_state(i, c["eta"], c["u"], c["v"])
        infos = b.step(60)
        states = [b.get_state(i) for i in range(len(cases))]
        b.close()
        return infos, states

    ref_i, ref_s = run(None)
    chk_i, chk_s = run(checked_lib)
    for a, b in zip(chk_i, ref_i):
        assert not (a.flags & swe.SWE_FLAG_CHECK)
        assert a.t == b.t
    for sa, sb in zip(chk_s, ref_s):
        for a, b in zip(sa, sb):
            assert np.array_equal(a, b)
