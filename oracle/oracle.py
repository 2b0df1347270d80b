"""ctypes shim over the FP64 CPU oracle (``swe_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  Nothing here is imported by, or
imports, the CUDA package; the two sides share no code.

The oracle computes one explicit 2D MacCormack predictor-corrector step of the
shallow-water equations as 16 full-grid sub-steps (Seitz et al., Sec. 1; the
variable time step of Sec. 3.1; drying of Sec. 6.2 read as described in
``swe_oracle.c``).  Arrays are float64, shape (ny, nx), row-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libswe_oracle.so")
_lock = threading.Lock()
_lib = None

WALL, INFLOW, OUTFLOW = 0, 1, 2


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("g", ctypes.c_double), ("cfl", ctypes.c_double),
        ("h_dry", ctypes.c_double), ("dt_max", ctypes.c_double),
        ("kappa", ctypes.c_double), ("manning_n", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("q_in", ctypes.c_double * 4),
        ("dir_cycle", ctypes.c_int32),
        ("friction", ctypes.c_int32), ("dissipation", ctypes.c_int32),
    ]


@dataclass
class Params:
    """Scheme parameters (m, s).  bc/q_in order: W, E, S, N.

    q_in is the discharge per unit width entering the domain (m^2/s).
    dir_cycle: bit 0 alternates the predictor directions every step,
    bit 1 starts x backward, bit 2 starts y backward.  friction and
    dissipation select the ablation forms (explicit friction; the
    TVD-MacCormack term in place of S15's switch).
    """
    nx: int
    ny: int
    dx: float = 1.0
    dy: float = 1.0
    g: float = 9.81
    cfl: float = 0.5
    h_dry: float = 1e-3
    dt_max: float = 10.0
    kappa: float = 0.0
    manning_n: float = 0.0
    bc: tuple = (WALL, WALL, WALL, WALL)
    q_in: tuple = (0.0, 0.0, 0.0, 0.0)
    dir_cycle: int = 1
    friction: int = 0       # 0: point-implicit Manning; 1: explicit (ablation)
    dissipation: int = 0    # 0: the switch form of S15 (kappa); 1: the TVD-MacCormack term

    def _c(self) -> _Params:
        p = _Params()
        p.nx, p.ny = int(self.nx), int(self.ny)
        p.dx, p.dy, p.g, p.cfl = self.dx, self.dy, self.g, self.cfl
        p.h_dry, p.dt_max, p.kappa, p.manning_n = self.h_dry, self.dt_max, self.kappa, self.manning_n
        for s in range(4):
            p.bc[s] = int(self.bc[s])
            p.q_in[s] = float(self.q_in[s])
        p.dir_cycle = int(self.dir_cycle)
        p.friction, p.dissipation = int(self.friction), int(self.dissipation)
        return p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def compile_source(src_path: str, out_path: str) -> str:
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src_path, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


@dataclass
class RunResult:
    eta: np.ndarray
    u: np.ndarray
    v: np.ndarray
    dt: np.ndarray
    clamp_volume: float
    bflux: np.ndarray = field(default_factory=lambda: np.zeros(4))
    status: int = 0


class OracleLib:
    """One loaded build of the oracle.  The module-level functions use the
    build of ``swe_oracle.c``; a test may load another build of a modified
    copy of the source to check that the pins reject it."""
    Params = Params

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_run.argtypes = [P, dp, dp, dp, dp, dp, ctypes.c_int64, ctypes.c_int32,
                                dp, dp, dp, ctypes.c_int32]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_dt.argtypes = [P, dp, dp, dp, dp]
        lib.orc_dt.restype = ctypes.c_double
        lib.orc_volume.argtypes = [P, dp, dp]
        lib.orc_volume.restype = ctypes.c_double
        lib.orc_prepare_state.argtypes = [P, dp, dp, dp, dp]
        lib.orc_prepare_state.restype = ctypes.c_int
        if hasattr(lib, "orc_adjoint"):
            lp = ctypes.POINTER(ctypes.c_int64)
            lib.orc_adjoint.argtypes = [P, dp, dp, dp, dp, dp, ctypes.c_int64, ctypes.c_int32, dp, lp,
                                        ctypes.c_int32, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_adjoint.restype = ctypes.c_int
        self.lib = lib

    def run(self, p: Params, z, eta, u, v, nsteps: int, *, nfield=None, step0: int = 0,
            dt_fixed=None, nthreads: int = 1) -> RunResult:
        """Advance (eta, u, v) by nsteps steps; inputs are not modified."""
        shape = (p.ny, p.nx)
        z = _arr(z, shape)
        e, uu, vv = _arr(eta, shape).copy(), _arr(u, shape).copy(), _arr(v, shape).copy()
        nf = None if nfield is None else _arr(nfield, shape)
        dtf = None
        if dt_fixed is not None:
            dtf = np.ascontiguousarray(dt_fixed, dtype=np.float64)
            if dtf.shape != (nsteps,):
                raise ValueError("dt_fixed must hold nsteps values")
        dt_out = np.zeros(max(nsteps, 1), dtype=np.float64)
        acc = np.zeros(5, dtype=np.float64)
        pc = p._c()
        st = self.lib.orc_run(ctypes.byref(pc), _ptr(z), _ptr(nf), _ptr(e), _ptr(uu), _ptr(vv),
                              int(step0), int(nsteps), _ptr(dtf), _ptr(dt_out), _ptr(acc),
                              int(nthreads))
        if st == 1:
            raise ValueError("oracle rejected the arguments")
        return RunResult(e, uu, vv, dt_out[:nsteps].copy(), float(acc[0]), acc[1:5].copy(), st)

    def cfl_dt(self, p: Params, z, eta, u, v) -> float:
        shape = (p.ny, p.nx)
        pc = p._c()
        return float(self.lib.orc_dt(ctypes.byref(pc), _ptr(_arr(z, shape)), _ptr(_arr(eta, shape)),
                                     _ptr(_arr(u, shape)), _ptr(_arr(v, shape))))

    def volume(self, p: Params, z, eta) -> float:
        shape = (p.ny, p.nx)
        pc = p._c()
        return float(self.lib.orc_volume(ctypes.byref(pc), _ptr(_arr(z, shape)),
                                         _ptr(_arr(eta, shape))))

    def prepare_state(self, p: Params, z, eta, u, v):
        """Set-state normalisation (see ``orc_prepare_state``); returns copies."""
        shape = (p.ny, p.nx)
        z = _arr(z, shape)
        e, uu, vv = _arr(eta, shape).copy(), _arr(u, shape).copy(), _arr(v, shape).copy()
        pc = p._c()
        if self.lib.orc_prepare_state(ctypes.byref(pc), _ptr(z), _ptr(e), _ptr(uu), _ptr(vv)) != 0:
            raise ValueError("state rejected (negative depth below -1e-12 m or non-finite value)")
        return e, uu, vv


class AdjointResult:
    def __init__(self, loss, grad_n, grad_eta0, grad_u0, grad_v0, status, grad_z=None):
        self.loss, self.grad_n, self.grad_eta0 = loss, grad_n, grad_eta0
        self.grad_u0, self.grad_v0, self.status = grad_u0, grad_v0, status
        self.grad_z = grad_z


def _adjoint(lib, p, z, nfield, eta, u, v, dt, gauges, obs, step0=0):
    shape = (p.ny, p.nx)
    z, nf = _arr(z, shape), _arr(nfield, shape)
    e, uu, vv = _arr(eta, shape), _arr(u, shape), _arr(v, shape)
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    T = dt.shape[0]
    g = np.ascontiguousarray(gauges, dtype=np.int64)
    ob = np.ascontiguousarray(obs, dtype=np.float64).reshape(T, g.shape[0])
    loss = np.zeros(1)
    gn, ge, gu, gv, gz = (np.zeros(shape) for _ in range(5))
    pc = p._c()
    st = lib.orc_adjoint(ctypes.byref(pc), _ptr(z), _ptr(nf), _ptr(e), _ptr(uu), _ptr(vv), int(step0), int(T),
                         _ptr(dt), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(g.shape[0]), _ptr(ob),
                         _ptr(loss), _ptr(gn), _ptr(ge), _ptr(gu), _ptr(gv), _ptr(gz))
    if st == 1:
        raise ValueError("oracle rejected the adjoint arguments")
    return AdjointResult(float(loss[0]), gn, ge, gu, gv, st, gz)


OracleLib.adjoint = lambda self, *a, **k: _adjoint(self.lib, *a, **k)


def _default() -> OracleLib:
    global _lib
    with _lock:
        if _lib is None:
            _lib = OracleLib(build())
    return _lib


def run(p: Params, z, eta, u, v, nsteps: int, **kw) -> RunResult:
    """Advance (eta, u, v) by nsteps steps; inputs are not modified."""
    return _default().run(p, z, eta, u, v, nsteps, **kw)


def cfl_dt(p: Params, z, eta, u, v) -> float:
    return _default().cfl_dt(p, z, eta, u, v)


def volume(p: Params, z, eta) -> float:
    return _default().volume(p, z, eta)


def prepare_state(p: Params, z, eta, u, v):
    """Set-state normalisation (see ``orc_prepare_state``); returns copies."""
    return _default().prepare_state(p, z, eta, u, v)


def adjoint(p: Params, z, nfield, eta, u, v, dt, gauges, obs, step0: int = 0) -> AdjointResult:
    """Discrete adjoint of nsteps = len(dt) steps with frozen step sizes:
    gradient of L = 1/2 sum_k sum_g (eta_g^k - obs[k-1, g])^2 with respect to
    the per-cell Manning n, the bed z and the initial eta, u, v (kappa 0,
    fully wet)."""
    return _default().adjoint(p, z, nfield, eta, u, v, dt, gauges, obs, step0)
