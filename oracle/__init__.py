"""Plain FP64 CPU oracle of the LES stage residual and Runge-Kutta update.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports, links or calls it, and it shares no code with the library.

The arithmetic lives in ``les_oracle.c`` (plain C loops, FP64, written from
the paper's sections in their order; see that file's header for the list of
readings of garbled equations).  This module only builds it with gcc and
marshals numpy arrays through ctypes.  ``oracle.fwh`` (plain numpy, FP64) is
the far-field FW-H integral of the probe surface's data.

Parameter vector layout (``Params.as_array``):
  [gamma, Pr, Pr_sgs, Cs, k2, k4, Re, mach_j, TR, T_inf_dim, S1_dim, theta,
   noise_amp, cfl]
Boundary-condition codes: 0 periodic, 1 far field, 2 jet inflow, 3 exit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "les_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

BC_PERIODIC, BC_FARFIELD, BC_INFLOW_JET, BC_EXIT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def _declare(L):
    grid = [_ip, _ip, _dp, _ip, _dp, _dp, _dp]
    L.ora_metrics.argtypes = grid + [_dp]
    L.ora_metrics.restype = None
    L.ora_qhat_from.argtypes = grid + [_dp, _dp, _dp, ctypes.c_int, _dp]
    L.ora_qhat_from.restype = None
    L.ora_state_out.argtypes = grid + [_dp, _dp, _dp, ctypes.c_int, _dp]
    L.ora_state_out.restype = None
    L.ora_apply_bc.argtypes = grid + [_dp, ctypes.c_uint64, _dp, _dp, ctypes.c_long]
    L.ora_apply_bc.restype = None
    L.ora_rhs.argtypes = grid + [_dp, _dp, _dp, _dp]
    L.ora_rhs.restype = ctypes.c_int
    L.ora_rhs_sampled.argtypes = grid + [_dp, _dp, _dp, ctypes.c_long, _lp, _dp]
    L.ora_rhs_sampled.restype = ctypes.c_int
    L.ora_field.argtypes = grid + [_dp, _dp, _dp, ctypes.c_int, _dp]
    L.ora_field.restype = ctypes.c_int
    L.ora_dt.argtypes = grid + [_dp, _dp, _dp]
    L.ora_dt.restype = ctypes.c_double
    L.ora_step.argtypes = grid + [_dp, ctypes.c_uint64, _dp, _dp, ctypes.c_long,
                                  ctypes.c_long, ctypes.c_double]
    L.ora_step.restype = ctypes.c_int
    L.ora_diag.argtypes = grid + [_dp, _dp, _dp, _dp]
    L.ora_diag.restype = ctypes.c_int
    L.ora_probe.argtypes = grid + [_dp, _dp, _dp, ctypes.c_long, _dp, _dp]
    L.ora_probe.restype = ctypes.c_int
    L.ora_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.ora_splitmix64.restype = ctypes.c_uint64
    L.ora_inflow_profile.argtypes = [_dp, ctypes.c_double]
    L.ora_inflow_profile.restype = ctypes.c_double
    L.ora_sutherland.argtypes = [_dp, ctypes.c_double]
    L.ora_sutherland.restype = ctypes.c_double
    L.ora_face_state.argtypes = [_dp, ctypes.c_int, _dp, _dp, _dp]
    L.ora_face_state.restype = None


def _d(a):
    return a.ctypes.data_as(_dp)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Flow and scheme parameters in jet units (rho_j = a_j = T_j = D = 1)."""
    gamma: float = 1.4
    Pr: float = 0.72
    Pr_sgs: float = 0.6
    Cs: float = 0.17
    k2: float = 0.25
    k4: float = 0.016
    Re: float = 1.0e5
    mach_j: float = 1.4
    TR: float = 1.0
    T_inf_dim: float = 288.15
    S1_dim: float = 110.4
    theta: float = 0.05
    noise_amp: float = 1.0e-3
    cfl: float = 0.5
    seed: int = 1

    def as_array(self) -> np.ndarray:
        return np.array([self.gamma, self.Pr, self.Pr_sgs, self.Cs, self.k2, self.k4,
                         self.Re, self.mach_j, self.TR, self.T_inf_dim, self.S1_dim,
                         self.theta, self.noise_amp, self.cfl], dtype=np.float64)


@dataclass
class Grid:
    """Structured grid: coordinates (ni*nj*nk each, i fastest), periodicity,
    per-axis period shift (3x3: [axis][x,y,z]) and face BC codes
    (i-, i+, j-, j+, k-, k+)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    dims: tuple
    periodic: tuple = (0, 0, 0)
    shift: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    bc: tuple = (1, 1, 1, 1, 1, 1)

    def __post_init__(self):
        self.x = _c64(self.x).reshape(-1)
        self.y = _c64(self.y).reshape(-1)
        self.z = _c64(self.z).reshape(-1)
        self.shift = _c64(self.shift).reshape(3, 3)
        self._dims = np.array(self.dims, dtype=np.int32)
        self._per = np.array(self.periodic, dtype=np.int32)
        self._bc = np.array(self.bc, dtype=np.int32)
        self._shift = np.ascontiguousarray(self.shift.reshape(-1))

    @property
    def N(self) -> int:
        return int(np.prod(self.dims))

    def args(self):
        return (self._dims.ctypes.data_as(_ip), self._per.ctypes.data_as(_ip),
                _d(self._shift), self._bc.ctypes.data_as(_ip),
                _d(self.x), _d(self.y), _d(self.z))


def metrics(g: Grid) -> np.ndarray:
    """10 x N: the nine J^-1 metric cofactors (xi row, eta row, zeta row) and J^-1."""
    m = np.empty((10, g.N))
    lib().ora_metrics(*g.args(), _d(m))
    return m


def qhat_from(g: Grid, P: Params, m: np.ndarray, state: np.ndarray, primitive: bool) -> np.ndarray:
    """Qhat = J^-1 Q (5 x N) from primitive (rho,u,v,w,p) or conserved input."""
    st = _c64(state).reshape(5, -1)
    q = np.empty((5, g.N))
    lib().ora_qhat_from(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(st), int(primitive), _d(q))
    return q


def state_out(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray, primitive: bool) -> np.ndarray:
    out = np.empty((5, g.N))
    lib().ora_state_out(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat)),
                        int(primitive), _d(out))
    return out


def apply_bc(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray, level: int) -> np.ndarray:
    q = _c64(qhat).copy()
    lib().ora_apply_bc(*g.args(), _d(P.as_array()), P.seed, _d(_c64(m)), _d(q), int(level))
    return q


def rhs(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray) -> np.ndarray:
    out = np.empty((5, g.N))
    rc = lib().ora_rhs(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat)), _d(out))
    if rc:
        raise MemoryError("oracle rhs allocation failed")
    return out


def rhs_sampled(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray, pts: np.ndarray) -> np.ndarray:
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    out = np.empty((5, len(pts)))
    rc = lib().ora_rhs_sampled(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat)),
                               len(pts), pts.ctypes.data_as(_lp), _d(out))
    if rc:
        raise MemoryError("oracle rhs allocation failed")
    return out


FIELD_MU_SGS, FIELD_MU, FIELD_P, FIELD_T = 0, 1, 2, 3
FIELD_LAMBDA_BAR = (4, 5, 6)
FIELD_SENSOR = (7, 8, 9)


def point_field(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray, which: int) -> np.ndarray:
    out = np.empty(g.N)
    rc = lib().ora_field(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat)), int(which),
                         _d(out))
    if rc:
        raise MemoryError("oracle field allocation failed")
    return out


def dt_cfl(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray) -> float:
    return float(lib().ora_dt(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat))))


def step(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray, nsteps: int, level0: int,
         dt: float) -> np.ndarray:
    q = _c64(qhat).copy()
    rc = lib().ora_step(*g.args(), _d(P.as_array()), P.seed, _d(_c64(m)), _d(q), int(nsteps),
                        int(level0), float(dt))
    if rc:
        raise MemoryError("oracle step allocation failed")
    return q


def diag(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray) -> dict:
    out = np.empty(11)
    rc = lib().ora_diag(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat)), _d(out))
    if rc:
        raise MemoryError("oracle diag allocation failed")
    return {"max_abs_rhs_rho": out[0], "l2_rhs": out[1:6].copy(), "sum_qhat": out[6:11].copy()}


def probe(g: Grid, P: Params, m: np.ndarray, qhat: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    xyz = _c64(xyz).reshape(3, -1)
    out = np.empty((5, xyz.shape[1]))
    rc = lib().ora_probe(*g.args(), _d(P.as_array()), _d(_c64(m)), _d(_c64(qhat)),
                         xyz.shape[1], _d(xyz), _d(out))
    if rc:
        raise ValueError("probe: not a Cartesian-product grid or point outside the grid")
    return out


def splitmix64(seed: int, n: int) -> int:
    return int(lib().ora_splitmix64(seed, n))


def inflow_profile(P: Params, r: float) -> float:
    return float(lib().ora_inflow_profile(_d(P.as_array()), float(r)))


def sutherland(P: Params, T: float) -> float:
    return float(lib().ora_sutherland(_d(P.as_array()), float(T)))


def face_state(P: Params, kind: str, Qe, n) -> np.ndarray:
    """Single-point far-field ('farfield') or exit ('exit') boundary state."""
    Qe = _c64(Qe)
    n = _c64(n)
    Qf = np.empty(5)
    lib().ora_face_state(_d(P.as_array()), 0 if kind == "farfield" else 1, _d(Qe), _d(n), _d(Qf))
    return Qf
