"""Python binding of libles.so (ctypes): the C ABI of include/les.h with the same
names, plus a small ``Solver`` convenience wrapper.  Argument marshalling only:
every step of the method runs in the library's CUDA kernels.  There is no CPU
fallback: if the library or a GPU is missing, calls raise.

PyTorch is used only to obtain the current CUDA stream (and, optionally, a
device workspace tensor).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from .inputs import FlowParams, GridSpec

_HERE = os.path.dirname(os.path.abspath(__file__))
# LES_LIBRARY selects another in-tree build of the same library (the
# bounds-checked debug build, _build_bounds/libles.so)
LIB_PATH = os.environ.get("LES_LIBRARY") or os.path.join(_HERE, "_build", "libles.so")

LES_OK, LES_ERR_ARG, LES_ERR_OOM, LES_ERR_CUDA, LES_ERR_NONFINITE, LES_ERR_TIMEOUT, LES_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
LES_BC_PERIODIC, LES_BC_FARFIELD, LES_BC_INFLOW_JET, LES_BC_EXIT, LES_BC_CENTERLINE = 0, 1, 2, 3, 4
LES_FP64, LES_FP32, LES_FP32_SEPARABLE = 0, 1, 2
LES_STATE_CONSERVED, LES_STATE_PRIMITIVE, LES_STATE_RAW = 0, 1, 2
(LES_FIELD_MU_SGS, LES_FIELD_MU, LES_FIELD_P, LES_FIELD_T, LES_FIELD_LAMBDA_XI,
 LES_FIELD_LAMBDA_ETA, LES_FIELD_LAMBDA_ZETA, LES_FIELD_METRICS) = range(8)

EXPORTED = [
    "les_workspace_bytes", "les_create_grid", "les_create_batch", "les_set_state",
    "les_set_state_jet", "les_step", "les_get_state", "les_get_state_jet", "les_set_time",
    "les_get_time", "les_probe_surface", "les_probe_frames", "les_get_diagnostics",
    "les_get_diagnostics_jet", "les_debug_rhs", "les_debug_field", "les_profile_step",
    "les_set_fused_tiling", "les_debug_stage_wait", "les_last_launch_count", "les_bounds_checking", "les_bounds_violation",
    "les_diag_sums_noalloc", "les_measure_peak", "les_fwh", "les_describe",
    "les_last_error", "les_destroy",
]

_dp = ctypes.POINTER(ctypes.c_double)


class les_grid_desc(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("nk", ctypes.c_int),
                ("x", _dp), ("y", _dp), ("z", _dp),
                ("periodic", ctypes.c_int * 3),
                ("period_shift", (ctypes.c_double * 3) * 3),
                ("face_bc", ctypes.c_int * 6),
                ("precision", ctypes.c_int),
                ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


class les_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("gamma", "Pr", "Pr_sgs", "Cs", "k2", "k4", "Re", "mach_j", "TR", "T_inf_dim",
                 "S1_dim", "theta", "noise_amp", "cfl", "dt")] + [("seed", ctypes.c_uint64)]


class les_diag(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("step", ctypes.c_int64),
                ("max_abs_rhs_rho", ctypes.c_double), ("l2_rhs", ctypes.c_double * 5),
                ("sum_qhat", ctypes.c_double * 5), ("nonfinite", ctypes.c_int64)]


_lib = None


def lib():
    """Load libles.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libles.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.les_workspace_bytes.argtypes = [ctypes.POINTER(les_grid_desc)]
        L.les_workspace_bytes.restype = ctypes.c_size_t
        L.les_create_grid.argtypes = [ctypes.POINTER(les_grid_desc), ctypes.POINTER(les_params), vp,
                                      ctypes.POINTER(vp)]
        L.les_create_batch.argtypes = [ctypes.POINTER(les_grid_desc), ctypes.POINTER(les_params),
                                       ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.les_set_state.argtypes = [vp, _dp, ctypes.c_int]
        L.les_set_state_jet.argtypes = [vp, ctypes.c_int, _dp, ctypes.c_int]
        L.les_step.argtypes = [vp, ctypes.c_int]
        L.les_get_state.argtypes = [vp, _dp, ctypes.c_int]
        L.les_get_state_jet.argtypes = [vp, ctypes.c_int, _dp, ctypes.c_int]
        L.les_set_time.argtypes = [vp, ctypes.c_int64, ctypes.c_double]
        L.les_get_time.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), _dp]
        L.les_probe_surface.argtypes = [vp, _dp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
        L.les_probe_frames.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.les_get_diagnostics.argtypes = [vp, ctypes.POINTER(les_diag)]
        L.les_get_diagnostics_jet.argtypes = [vp, ctypes.c_int, ctypes.POINTER(les_diag)]
        L.les_debug_rhs.argtypes = [vp, ctypes.c_int, _dp]
        L.les_debug_field.argtypes = [vp, ctypes.c_int, ctypes.c_int, _dp]
        L.les_profile_step.argtypes = [vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64)]
        L.les_set_fused_tiling.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.les_debug_stage_wait.argtypes = [vp, ctypes.c_int]
        L.les_last_launch_count.argtypes = [vp]
        L.les_last_launch_count.restype = ctypes.c_int64
        L.les_bounds_checking.argtypes = []
        L.les_bounds_violation.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.les_diag_sums_noalloc.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        L.les_measure_peak.argtypes = [ctypes.c_int, _dp]
        L.les_fwh.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                              ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, vp, _dp]
        L.les_describe.argtypes = [vp]
        L.les_describe.restype = ctypes.c_char_p
        L.les_last_error.argtypes = [vp]
        L.les_last_error.restype = ctypes.c_char_p
        L.les_destroy.argtypes = [vp]
        _lib = L
    return _lib


class LesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libles error {code}: {msg}")
        self.code = code


def _check(h, rc):
    if rc != LES_OK:
        msg = lib().les_last_error(h)
        raise LesError(rc, (msg or b"").decode(errors="replace"))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def current_stream():
    """torch's current CUDA stream handle (0 if torch CUDA is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def make_desc(spec: GridSpec, precision: int, keep: list, workspace=None) -> les_grid_desc:
    d = les_grid_desc()
    d.ni, d.nj, d.nk = (int(n) for n in spec.dims)
    for name in ("x", "y", "z"):
        a = np.ascontiguousarray(getattr(spec, name), dtype=np.float64).reshape(-1)
        keep.append(a)
        setattr(d, name, _dptr(a))
    for a in range(3):
        d.periodic[a] = int(spec.periodic[a])
        for c in range(3):
            d.period_shift[a][c] = float(np.asarray(spec.shift)[a, c])
    for f in range(6):
        d.face_bc[f] = int(spec.bc[f])
    d.precision = precision
    if workspace is not None:
        d.workspace = ctypes.c_void_p(int(workspace.data_ptr()))
        d.workspace_bytes = int(workspace.numel() * workspace.element_size())
    return d


def make_params(fp: FlowParams) -> les_params:
    p = les_params()
    for n, _ in les_params._fields_:
        setattr(p, n, getattr(fp, n) if n != "seed" else int(fp.seed))
    return p


# --- C-ABI names -------------------------------------------------------------

def les_workspace_bytes(spec: GridSpec, precision: int = LES_FP64) -> int:
    keep = []
    d = make_desc(spec, precision, keep)
    return int(lib().les_workspace_bytes(ctypes.byref(d)))


def les_create_grid(spec: GridSpec, fp: FlowParams, precision: int = LES_FP64, stream=None,
                    workspace=None):
    keep = []
    d = make_desc(spec, precision, keep, workspace)
    p = make_params(fp)
    h = ctypes.c_void_p()
    _check(None, lib().les_create_grid(ctypes.byref(d), ctypes.byref(p),
                                       stream if stream is not None else current_stream(),
                                       ctypes.byref(h)))
    return h


def les_create_batch(specs, fps, precision: int = LES_FP32, stream=None):
    keep = []
    n = len(specs)
    D = (les_grid_desc * n)(*[make_desc(s, precision, keep) for s in specs])
    P = (les_params * n)(*[make_params(f) for f in fps])
    h = ctypes.c_void_p()
    _check(None, lib().les_create_batch(D, P, n, stream if stream is not None else current_stream(),
                                        ctypes.byref(h)))
    return h


def les_set_state(h, q: np.ndarray, kind: int, jet: int = 0):
    q = np.ascontiguousarray(q, dtype=np.float64)
    _check(h, lib().les_set_state_jet(h, jet, _dptr(q), kind))


def les_get_state(h, n_points: int, kind: int, jet: int = 0) -> np.ndarray:
    out = np.empty((5, n_points))
    _check(h, lib().les_get_state_jet(h, jet, _dptr(out), kind))
    return out


def les_step(h, nsteps: int):
    _check(h, lib().les_step(h, int(nsteps)))


def les_set_time(h, step: int, dt: float):
    _check(h, lib().les_set_time(h, int(step), float(dt)))


def les_get_time(h):
    s = ctypes.c_int64()
    dt = ctypes.c_double()
    _check(h, lib().les_get_time(h, ctypes.byref(s), ctypes.byref(dt)))
    return s.value, dt.value


def les_get_diagnostics(h, jet: int = 0, check: bool = True) -> dict:
    d = les_diag()
    rc = lib().les_get_diagnostics_jet(h, jet, ctypes.byref(d))
    if check or rc not in (LES_OK, LES_ERR_NONFINITE, LES_ERR_TIMEOUT):
        _check(h, rc)
    return {"dt": d.dt, "step": d.step, "max_abs_rhs_rho": d.max_abs_rhs_rho,
            "l2_rhs": np.array(d.l2_rhs[:]), "sum_qhat": np.array(d.sum_qhat[:]),
            "nonfinite": d.nonfinite, "rc": rc}


def les_debug_rhs(h, n_points: int, jet: int = 0) -> np.ndarray:
    out = np.empty((5, n_points))
    _check(h, lib().les_debug_rhs(h, jet, _dptr(out)))
    return out


def les_debug_field(h, field: int, n_points: int, jet: int = 0) -> np.ndarray:
    out = np.empty((10, n_points) if field == LES_FIELD_METRICS else n_points)
    _check(h, lib().les_debug_field(h, jet, field, _dptr(out)))
    return out


def les_probe_surface(h, xyz: np.ndarray, every_n: int, dev_out_ptr: int, capacity: int):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(3, -1)
    _check(h, lib().les_probe_surface(h, _dptr(xyz), xyz.shape[1], int(every_n),
                                      ctypes.c_void_p(int(dev_out_ptr)), int(capacity)))


def les_probe_frames(h) -> int:
    f = ctypes.c_int64()
    _check(h, lib().les_probe_frames(h, ctypes.byref(f)))
    return f.value


KERNEL_KINDS = ("point", "grads", "iface", "update", "bc", "other")


def les_profile_step(h, nsteps: int):
    """Per-kernel-kind device time (ms, summed) and launch counts of nsteps
    eagerly launched, event-timed steps."""
    ms = np.zeros(len(KERNEL_KINDS))
    cnt = (ctypes.c_int64 * len(KERNEL_KINDS))()
    _check(h, lib().les_profile_step(h, int(nsteps), _dptr(ms), cnt))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}


def les_describe(h) -> str:
    return (lib().les_describe(h) or b"").decode()


def les_set_fused_tiling(h, ty: int, kc: int):
    """Fix the fused FP32 stage's tile height (8 or 16) and k-chunk (0 = balanced, -1 = lockstep)."""
    _check(h, lib().les_set_fused_tiling(h, int(ty), int(kc)))


def les_debug_stage_wait(h, max_polls: int):
    """Bound the fused FP32 stage's staging waits to max_polls polls (-1: default)."""
    _check(h, lib().les_debug_stage_wait(h, int(max_polls)))


def les_get_state_rc(h, n_points: int, kind: int, jet: int = 0):
    """The state and the return code of les_get_state_jet, without raising."""
    out = np.empty((5, n_points))
    rc = lib().les_get_state_jet(h, jet, _dptr(out), kind)
    return out, rc


def les_last_launch_count(h) -> int:
    return int(lib().les_last_launch_count(h))


def les_bounds_checking() -> bool:
    """True for a library built with -DLES_BOUNDS_CHECK."""
    return bool(lib().les_bounds_checking())


def les_bounds_violation(h) -> int:
    """First out-of-range index met by the handle's kernels ((site << 48) |
    value), 0 if none; site 8 (any build) is a staging wait of the fused
    FP32 stage that gave up."""
    v = ctypes.c_uint64(0)
    _check(h, lib().les_bounds_violation(h, ctypes.byref(v)))
    return int(v.value)


NOALLOC_MAX_POINTS = 268435456


def les_diag_sums_noalloc(qhat_ptr: int, rhs_ptr: int, npoints: int, out_ptr: int, stream=None) -> int:
    """Device-pointer form; returns the library's status code."""
    return int(lib().les_diag_sums_noalloc(ctypes.c_void_p(qhat_ptr), ctypes.c_void_p(rhs_ptr),
                                           int(npoints), ctypes.c_void_p(out_ptr),
                                           stream if stream is not None else current_stream()))


LES_PEAK_FP64_FMA, LES_PEAK_FP32_FMA, LES_PEAK_FP32X2_FMA = 0, 1, 2


def les_measure_peak(kind: int) -> float:
    """Measured multiply-add throughput of the current device in TFLOP/s
    (kind: LES_PEAK_FP64_FMA, LES_PEAK_FP32_FMA or LES_PEAK_FP32X2_FMA)."""
    v = ctypes.c_double(0.0)
    _check(None, lib().les_measure_peak(int(kind), ctypes.byref(v)))
    return float(v.value)


def les_fwh(ring_ptr: int, precision: int, capacity: int, frames_written: int, xyz, nrm, area, dtau: float,
            p0: float, c0: float, obs, t0: float, dt_obs: float, nt: int, stream=None, timings: bool = False):
    """Far-field pressure p' [nobs][nt] by the FW-H integral over the probe
    surface's frames (see include/les.h); with timings=True also the device
    times (ms) of the source and observer passes."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    nrm = np.ascontiguousarray(nrm, dtype=np.float64)
    area = np.ascontiguousarray(area, dtype=np.float64)
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    npts = area.shape[0]
    nobs = obs.shape[1]
    assert xyz.shape == (3, npts) and nrm.shape == (3, npts) and obs.shape == (3, nobs)
    out = np.empty((nobs, nt), dtype=np.float64)
    ms = np.zeros(2, dtype=np.float64)
    st = stream if stream is not None else current_stream()
    _check(None, lib().les_fwh(ctypes.c_void_p(ring_ptr), int(precision), int(capacity), int(frames_written),
                               int(npts), _dptr(xyz), _dptr(nrm), _dptr(area), float(dtau), float(p0), float(c0),
                               int(nobs), _dptr(obs), float(t0), float(dt_obs), int(nt), _dptr(out), st,
                               _dptr(ms) if timings else None))
    return (out, ms) if timings else out


def les_destroy(h):
    if h:
        lib().les_destroy(h)


# --- convenience wrapper -----------------------------------------------------

class Solver:
    """One jet (or a batch) on the current CUDA device and stream."""

    def __init__(self, spec, fp, precision: int = LES_FP64, stream=None, workspace=None):
        self.batch = isinstance(spec, (list, tuple))
        self.specs = list(spec) if self.batch else [spec]
        if self.batch:
            self.h = les_create_batch(self.specs, fp, precision, stream)
        else:
            self.h = les_create_grid(spec, fp, precision, stream, workspace)
        self.precision = precision
        self.workspace = workspace

    def npts(self, jet=0):
        return self.specs[jet].N

    def set_state(self, q, kind=LES_STATE_PRIMITIVE, jet=0):
        les_set_state(self.h, q, kind, jet)

    def get_state(self, kind=LES_STATE_CONSERVED, jet=0):
        return les_get_state(self.h, self.npts(jet), kind, jet)

    def step(self, n=1):
        les_step(self.h, n)

    def diagnostics(self, jet=0, check=True):
        return les_get_diagnostics(self.h, jet, check)

    def rhs(self, jet=0):
        return les_debug_rhs(self.h, self.npts(jet), jet)

    def field(self, f, jet=0):
        return les_debug_field(self.h, f, self.npts(jet), jet)

    def time(self):
        return les_get_time(self.h)

    def set_time(self, step, dt):
        les_set_time(self.h, step, dt)

    def close(self):
        if self.h:
            les_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
