"""Thin ctypes binding of the C ABI in ``include/swe.h``.

Argument marshalling only: every step of the scheme runs in the CUDA library
``libswe.so``.  There is no other implementation behind these names; if the
library is missing or cannot load, every call raises.

The functions keep the C names (``swe_create``, ``swe_set_bed``,
``swe_set_state``, ``swe_step``, ``swe_get_state``, ``swe_destroy``, ...).
``Solver`` is a small convenience wrapper over them for numpy and torch
arrays.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

SWE_OK, SWE_ERR_ARG, SWE_ERR_CUDA, SWE_ERR_NONFINITE = 0, 1, 2, 3
SWE_ERR_NEGDEPTH, SWE_ERR_TIMEOUT, SWE_ERR_STATE, SWE_ERR_UNSUPPORTED, SWE_ERR_CHECK = 4, 5, 6, 7, 8
SWE_BC_WALL, SWE_BC_INFLOW, SWE_BC_OUTFLOW = 0, 1, 2
SWE_FP64, SWE_FP32 = 0, 1
SWE_KERNEL_FUSED, SWE_KERNEL_PLAIN, SWE_KERNEL_PAPER, SWE_KERNEL_PAPER_DEVDT = 0, 1, 2, 3
SWE_KERNEL_PAPER_SHARED, SWE_KERNEL_PAPER_SHARED_DEVDT = 4, 5
SWE_FLAG_NONFINITE, SWE_FLAG_TIMEOUT, SWE_FLAG_CLAMPED, SWE_FLAG_CHECK = 1, 2, 4, 8
SWE_NOALLOC_MAX_CELLS = 1 << 20


class swe_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("g", ctypes.c_double), ("cfl", ctypes.c_double),
        ("h_dry", ctypes.c_double), ("dt_max", ctypes.c_double),
        ("kappa", ctypes.c_double), ("manning_n", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("q_in", ctypes.c_double * 4),
        ("precision", ctypes.c_int32), ("dir_cycle", ctypes.c_int32),
        ("device", ctypes.c_int32), ("kernel", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("seg_rows", ctypes.c_int32), ("cta_warps", ctypes.c_int32),
        ("use_graph", ctypes.c_int32), ("dry_skip", ctypes.c_int32),
        ("friction", ctypes.c_int32), ("dissipation", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


class swe_step_info(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("dt_last", ctypes.c_double),
        ("dt_min", ctypes.c_double), ("dt_max_seen", ctypes.c_double),
        ("volume", ctypes.c_double), ("clamp_volume", ctypes.c_double),
        ("bflux", ctypes.c_double * 4),
        ("step", ctypes.c_int64), ("n_wet", ctypes.c_int64),
        ("flags", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_ctxp = ctypes.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "swe_params_default": (None, [ctypes.POINTER(swe_params)]),
    "swe_create": (ctypes.c_int, [ctypes.POINTER(swe_params), ctypes.POINTER(ctypes.c_void_p)]),
    "swe_set_bed": (ctypes.c_int, [_ctxp, _dp, _dp]),
    "swe_set_state": (ctypes.c_int, [_ctxp, _dp, _dp, _dp]),
    "swe_set_clock": (ctypes.c_int, [_ctxp, ctypes.c_int64, ctypes.c_double]),
    "swe_step": (ctypes.c_int, [_ctxp, ctypes.c_int32, _dp, _dp, ctypes.POINTER(swe_step_info)]),
    "swe_get_state": (ctypes.c_int, [_ctxp, _dp, _dp, _dp]),
    "swe_get_info": (ctypes.c_int, [_ctxp, ctypes.POINTER(swe_step_info)]),
    "swe_set_state_device": (ctypes.c_int, [_ctxp, _vp, _vp, _vp]),
    "swe_get_state_device": (ctypes.c_int, [_ctxp, _vp, _vp, _vp]),
    "swe_set_bed_device": (ctypes.c_int, [_ctxp, _vp, _vp]),
    "swe_stream": (ctypes.c_void_p, [_ctxp]),
    "swe_destroy": (None, [_ctxp]),
    "swe_last_error": (ctypes.c_char_p, [_ctxp]),
    "swe_step_plain_f32_noalloc": (ctypes.c_int, [ctypes.POINTER(swe_params), _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                                  ctypes.c_double, _dp, _vp]),
    "swe_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "swe_batch_create": (ctypes.c_int, [ctypes.POINTER(swe_params), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), _dp, ctypes.POINTER(ctypes.c_void_p)]),
    "swe_batch_set_bed": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
    "swe_batch_set_state": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp, _dp]),
    "swe_batch_step": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(swe_step_info)]),
    "swe_batch_get_state": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp, _dp]),
    "swe_batch_destroy": (None, [_vp]),
    "swe_batch_last_error": (ctypes.c_char_p, [_vp]),
    "swe_adjoint": (ctypes.c_int, [_ctxp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, _dp,
                                   ctypes.c_int32, _dp, _dp, _dp, _dp]),
    "swe_set_own_rows": (ctypes.c_int, [_ctxp, ctypes.c_int32, ctypes.c_int32]),
    "swe_copy_rows": (ctypes.c_int, [_ctxp, ctypes.c_int32, _ctxp, ctypes.c_int32, ctypes.c_int32]),
    "swe_cfl_combine": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32]),
    "swe_autotune_candidates": (ctypes.c_int32, [_ctxp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "swe_autotune": (ctypes.c_int, [_ctxp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _dp,
                                    ctypes.POINTER(ctypes.c_int32)]),
    "swe_batch_autotune_candidates": (ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "swe_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _dp,
                                          ctypes.POINTER(ctypes.c_int32)]),
}


def library_path() -> str:
    return _build.LIB


def _open(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libswe.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run the build first")
            _lib = _open(path)
    return _lib


_lib_checked = None


def load_checked() -> ctypes.CDLL:
    """Loads the checked build (device-side index and alignment checks,
    NaN-poisoned padding), building it first if needed; pass it to Solver or
    Batch as `lib=` (tests)."""
    global _lib_checked
    with _lock:
        if _lib_checked is None:
            if not _build.up_to_date(checked=True):
                _build.build(checked=True)
            _lib_checked = _open(_build.LIB_CHECKED)
    return _lib_checked


class SweError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(st: int, ctx=None):
    if st != SWE_OK:
        lib = load()
        text = lib.swe_last_error(ctx).decode() if ctx else lib.swe_status_string(st).decode()
        raise SweError(st, text or lib.swe_status_string(st).decode())


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def make_params(nx, ny, *, dx=1.0, dy=1.0, g=9.81, cfl=0.5, h_dry=1e-3, dt_max=10.0, kappa=0.0,
                manning_n=0.0, bc=(0, 0, 0, 0), q_in=(0.0, 0.0, 0.0, 0.0), precision=SWE_FP64,
                dir_cycle=1, device=0, kernel=SWE_KERNEL_FUSED, stream=None, seg_rows=0, cta_warps=0,
                use_graph=1, dry_skip=1, friction=0, dissipation=0, reserved=(0, 0)) -> swe_params:
    p = swe_params()
    load().swe_params_default(ctypes.byref(p))
    p.nx, p.ny, p.dx, p.dy, p.g, p.cfl = int(nx), int(ny), dx, dy, g, cfl
    p.h_dry, p.dt_max, p.kappa, p.manning_n = h_dry, dt_max, kappa, manning_n
    for s in range(4):
        p.bc[s] = int(bc[s])
        p.q_in[s] = float(q_in[s])
    p.precision, p.dir_cycle, p.device, p.kernel = int(precision), int(dir_cycle), int(device), int(kernel)
    p.stream = stream
    p.seg_rows, p.cta_warps, p.use_graph, p.dry_skip = int(seg_rows), int(cta_warps), int(use_graph), int(dry_skip)
    p.friction, p.dissipation = int(friction), int(dissipation)
    for q in range(2):
        p.reserved[q] = int(reserved[q])
    return p


@dataclass
class StepInfo:
    t: float
    dt_last: float
    dt_min: float
    dt_max_seen: float
    volume: float
    clamp_volume: float
    bflux: tuple
    step: int
    n_wet: int
    flags: int


def _info(i: swe_step_info) -> StepInfo:
    return StepInfo(i.t, i.dt_last, i.dt_min, i.dt_max_seen, i.volume, i.clamp_volume, tuple(i.bflux),
                    int(i.step), int(i.n_wet), int(i.flags))


class Solver:
    """One grid on one GPU: owns a swe_ctx."""

    def __init__(self, nx, ny, lib=None, **kw):
        self.lib = lib if lib is not None else load()
        self.params = make_params(nx, ny, **kw)
        self.nx, self.ny = int(nx), int(ny)
        ctx = ctypes.c_void_p()
        st = self.lib.swe_create(ctypes.byref(self.params), ctypes.byref(ctx))
        if st != SWE_OK:
            raise SweError(st, "swe_create failed: " + self.lib.swe_status_string(st).decode())
        self.ctx = ctx

    @property
    def shape(self):
        return (self.ny, self.nx)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.swe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_bed(self, z, n_field=None):
        z = _f64(z, self.shape)
        nf = None if n_field is None else _f64(n_field, self.shape)
        _check(self.lib.swe_set_bed(self.ctx, _p(z), _p(nf)), self.ctx)

    def set_state(self, eta, u, v):
        e, uu, vv = (_f64(a, self.shape) for a in (eta, u, v))
        _check(self.lib.swe_set_state(self.ctx, _p(e), _p(uu), _p(vv)), self.ctx)

    def set_clock(self, step: int, t: float):
        _check(self.lib.swe_set_clock(self.ctx, int(step), float(t)), self.ctx)

    def step(self, nsteps: int, dt_fixed=None, want_dt: bool = False, want_info: bool = True):
        dtf = None
        if dt_fixed is not None:
            dtf = np.ascontiguousarray(dt_fixed, dtype=np.float64)
            if dtf.shape != (nsteps,):
                raise ValueError("dt_fixed must hold nsteps values")
        dto = np.zeros(max(1, nsteps), dtype=np.float64) if want_dt else None
        info = swe_step_info()
        st = self.lib.swe_step(self.ctx, int(nsteps), _p(dtf), _p(dto),
                               ctypes.byref(info) if want_info else None)
        _check(st, self.ctx)
        out = _info(info) if want_info else None
        if want_dt:
            return out, dto[:nsteps]
        return out

    def get_state(self):
        e = np.empty(self.shape)
        u = np.empty(self.shape)
        v = np.empty(self.shape)
        _check(self.lib.swe_get_state(self.ctx, _p(e), _p(u), _p(v)), self.ctx)
        return e, u, v

    def info(self) -> StepInfo:
        i = swe_step_info()
        _check(self.lib.swe_get_info(self.ctx, ctypes.byref(i)), self.ctx)
        return _info(i)

    def adjoint(self, nsteps: int, gauges, obs, checkpoint_every: int = 0, with_bed: bool = False):
        """Loss and its gradient w.r.t. the Manning field and the initial
        elevation (and, with_bed, the bed elevation) over nsteps steps from
        the current state (advances it).  Returns (loss, dL/dn, dL/deta0) or
        (loss, dL/dn, dL/deta0, dL/dz)."""
        g = np.ascontiguousarray(gauges, dtype=np.int64)
        ob = np.ascontiguousarray(obs, dtype=np.float64).reshape(int(nsteps), g.shape[0])
        loss = np.zeros(1)
        gn, ge = np.zeros(self.shape), np.zeros(self.shape)
        gz = np.zeros(self.shape) if with_bed else None
        st = self.lib.swe_adjoint(self.ctx, int(nsteps), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  int(g.shape[0]), _p(ob), int(checkpoint_every), _p(loss), _p(gn), _p(ge), _p(gz))
        _check(st, self.ctx)
        if with_bed:
            return float(loss[0]), gn, ge, gz
        return float(loss[0]), gn, ge

    def set_own_rows(self, lo: int, hi: int):
        """Rows [lo, hi) are this strip's own; the rest are halo rows."""
        _check(self.lib.swe_set_own_rows(self.ctx, int(lo), int(hi)), self.ctx)

    def copy_rows_from(self, src: "Solver", src_row: int, dst_row: int, nrows: int):
        """Copies nrows rows of src's current level into this context."""
        _check(self.lib.swe_copy_rows(self.ctx, int(dst_row), src.ctx, int(src_row), int(nrows)), self.ctx)

    def autotune(self, probe_steps: int = 10, rows=None):
        """Times each candidate rows-per-item of the fused step on the current
        state (which is restored) and keeps the fastest; returns (chosen,
        {rows: ms per step})."""
        if rows is None:
            buf = (ctypes.c_int32 * 16)()
            n = self.lib.swe_autotune_candidates(self.ctx, buf, 16)
            if n < 0:
                _check(-n, self.ctx)
            rows = list(buf[:n])
        cand = (ctypes.c_int32 * len(rows))(*[int(r) for r in rows])
        ms = np.zeros(len(rows))
        chosen = ctypes.c_int32(0)
        _check(self.lib.swe_autotune(self.ctx, int(probe_steps), cand, len(rows), _p(ms), ctypes.byref(chosen)),
               self.ctx)
        return int(chosen.value), dict(zip([int(r) for r in rows], ms.tolist()))

    # torch tensors on the context's device, of the context's real type
    def set_bed_device(self, z, n_field=None):
        for a in (z,) + ((n_field,) if n_field is not None else ()):
            _torch_check(a, self)
        _check(self.lib.swe_set_bed_device(self.ctx, z.data_ptr(), n_field.data_ptr() if n_field is not None else None),
               self.ctx)

    def set_state_device(self, eta, u, v):
        for a in (eta, u, v):
            _torch_check(a, self)
        _check(self.lib.swe_set_state_device(self.ctx, eta.data_ptr(), u.data_ptr(), v.data_ptr()), self.ctx)

    def get_state_device(self, eta, u, v):
        for a in (eta, u, v):
            _torch_check(a, self)
        _check(self.lib.swe_get_state_device(self.ctx, eta.data_ptr(), u.data_ptr(), v.data_ptr()), self.ctx)

    def stream_handle(self) -> int:
        return int(self.lib.swe_stream(self.ctx) or 0)


def cfl_combine(solvers):
    """Gives every strip the CFL maximum over all of them (swe_cfl_combine)."""
    arr = (ctypes.c_void_p * len(solvers))(*[x.ctx.value for x in solvers])
    st = load().swe_cfl_combine(arr, len(solvers))
    _check(st, solvers[0].ctx)


def _torch_check(a, s: Solver):
    import torch
    want = torch.float64 if s.params.precision == SWE_FP64 else torch.float32
    if not (a.is_cuda and a.dtype == want and a.is_contiguous() and tuple(a.shape) == s.shape):
        raise ValueError(f"expected a contiguous CUDA {want} tensor of shape {s.shape}")


class Batch:
    """Many scenarios advanced together (FP32): owns a swe_batch."""

    def __init__(self, sizes, manning_n, lib=None, **kw):
        self.lib = lib if lib is not None else load()
        kw.setdefault("precision", SWE_FP32)
        self.params = make_params(1, 1, **kw)
        self.sizes = [(int(nx), int(ny)) for nx, ny in sizes]
        n = len(self.sizes)
        nx = (ctypes.c_int32 * n)(*[a for a, _ in self.sizes])
        ny = (ctypes.c_int32 * n)(*[b for _, b in self.sizes])
        mn = np.ascontiguousarray(manning_n, dtype=np.float64)
        b = ctypes.c_void_p()
        st = self.lib.swe_batch_create(ctypes.byref(self.params), n, nx, ny, _p(mn), ctypes.byref(b))
        if st != SWE_OK:
            raise SweError(st, "swe_batch_create failed: " + self.lib.swe_status_string(st).decode())
        self.b = b
        self.count = n

    def _chk(self, st):
        if st != SWE_OK:
            raise SweError(st, self.lib.swe_batch_last_error(self.b).decode())

    def close(self):
        if getattr(self, "b", None):
            self.lib.swe_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, i):
        nx, ny = self.sizes[i]
        return (ny, nx)

    def set_bed(self, i, z):
        self._chk(self.lib.swe_batch_set_bed(self.b, int(i), _p(_f64(z, self._shape(i)))))

    def set_state(self, i, eta, u, v):
        e, uu, vv = (_f64(a, self._shape(i)) for a in (eta, u, v))
        self._chk(self.lib.swe_batch_set_state(self.b, int(i), _p(e), _p(uu), _p(vv)))

    def step(self, nsteps, want_info=True):
        infos = (swe_step_info * self.count)() if want_info else None
        self._chk(self.lib.swe_batch_step(self.b, int(nsteps), infos))
        return [_info(x) for x in infos] if want_info else None

    def autotune(self, probe_steps: int = 10, rows=None):
        """Times each candidate rows-per-item on the current states (which are
        restored) and keeps the fastest; returns (chosen, {rows: ms per step})."""
        if rows is None:
            buf = (ctypes.c_int32 * 16)()
            n = self.lib.swe_batch_autotune_candidates(self.b, buf, 16)
            if n < 0:
                self._chk(-n)
            rows = list(buf[:n])
        cand = (ctypes.c_int32 * len(rows))(*[int(r) for r in rows])
        ms = np.zeros(len(rows))
        chosen = ctypes.c_int32(0)
        self._chk(self.lib.swe_batch_autotune(self.b, int(probe_steps), cand, len(rows), _p(ms), ctypes.byref(chosen)))
        return int(chosen.value), dict(zip([int(r) for r in rows], ms.tolist()))

    def get_state(self, i):
        sh = self._shape(i)
        e, u, v = np.empty(sh), np.empty(sh), np.empty(sh)
        self._chk(self.lib.swe_batch_get_state(self.b, int(i), _p(e), _p(u), _p(v)))
        return e, u, v
