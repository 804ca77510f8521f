"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the method's arithmetic: it only builds grids
(coordinates), initial primitive states and parameter draws with the shapes
of the paper's jet runs (Sec. "Numerical Results": Mach 1.4 perfectly
expanded jet, TR = PR = 1, tanh-refined structured mesh; Table "Mesh
information" for sizes) and the batched/probe workloads.  Both the CUDA
library and the oracle consume what it returns.

Jet units: lengths in jet diameters D, velocities in jet sound speeds a_j,
density in rho_j; the ambient state at rest has rho = TR, p = 1/gamma.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

BC_PERIODIC, BC_FARFIELD, BC_INFLOW_JET, BC_EXIT, BC_CENTERLINE = 0, 1, 2, 3, 4


@dataclass
class FlowParams:
    """Flow and scheme parameters (jet units)."""
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
    dt: float = 0.0
    seed: int = 1


@dataclass
class GridSpec:
    """Coordinates (flattened, i fastest), dims, periodicity, period shifts
    ([axis][x,y,z]) and face BC codes (i-, i+, j-, j+, k-, k+)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    dims: tuple
    periodic: tuple = (0, 0, 0)
    shift: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    bc: tuple = (BC_INFLOW_JET, BC_EXIT, BC_FARFIELD, BC_FARFIELD, BC_FARFIELD, BC_FARFIELD)

    @property
    def N(self) -> int:
        return int(np.prod(self.dims))


def tanh_stretched(n: int, L: float, h_center: float) -> np.ndarray:
    """n symmetric points on [-L/2, L/2], clustered at 0 by
    y(s) = sign(s) L/2 [1 - tanh(beta (1-|s|)) / tanh(beta)], s uniform in [-1, 1],
    with beta chosen by bisection so that the spacing at the centre is h_center."""
    s = np.linspace(-1.0, 1.0, n)
    uniform = L / (n - 1)
    if h_center >= uniform:
        return 0.5 * L * s

    def center_spacing(beta):
        # dy/ds at s = 0 is L beta / sinh(2 beta); ds = 2/(n-1)
        return L * beta / math.sinh(2.0 * beta) * 2.0 / (n - 1)

    lo, hi = 1e-8, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if center_spacing(mid) > h_center:
            lo = mid
        else:
            hi = mid
    beta = 0.5 * (lo + hi)
    y = np.sign(s) * 0.5 * L * (1.0 - np.tanh(beta * (1.0 - np.abs(s))) / math.tanh(beta))
    return y


def product_grid(x1: np.ndarray, y1: np.ndarray, z1: np.ndarray, **kw) -> GridSpec:
    ni, nj, nk = len(x1), len(y1), len(z1)
    Z, Y, X = np.meshgrid(z1, y1, x1, indexing="ij")
    return GridSpec(X.reshape(-1).copy(), Y.reshape(-1).copy(), Z.reshape(-1).copy(),
                    (ni, nj, nk), **kw)


def jet_grid(ni: int, nj: int, nk: int, Lx: float, Ly: float, Lz: float,
             hy: float, hz: float) -> GridSpec:
    """Cartesian jet box: x uniform on [0, Lx] (jet inflow at x = 0), y and z
    tanh-stretched around the jet axis y = z = 0 with centre spacings hy, hz."""
    x1 = np.linspace(0.0, Lx, ni)
    return product_grid(x1, tanh_stretched(nj, Ly, hy), tanh_stretched(nk, Lz, hz))


# ---------------------------------------------------------------------------
# Named workloads: synthetic stand-ins for the paper's jet run (Sec. "Numerical
# Results": Mach 1.4, temperature ratio 1, about 14 M points on a tanh-refined
# mesh), at the sizes of the measured configurations
# ---------------------------------------------------------------------------

def jet_small() -> tuple[GridSpec, FlowParams]:
    """48x32x32 jet, 20D x 10D x 10D, 8 points across D, M 1.4, TR 1, Re_D 1e5."""
    return (jet_grid(48, 32, 32, 20.0, 10.0, 10.0, 1.0 / 8.0, 1.0 / 8.0),
            FlowParams(mach_j=1.4, TR=1.0, Re=1.0e5, Cs=0.17, cfl=0.5, seed=1))


def jet_paper_scale() -> tuple[GridSpec, FlowParams]:
    """384x256x144 jet (~14.2M points), 30D x 12D x 12D; centre spacing 0.4x the
    uniform spacing in y and z."""
    hy = 0.4 * 12.0 / 255
    hz = 0.4 * 12.0 / 143
    return (jet_grid(384, 256, 144, 30.0, 12.0, 12.0, hy, hz),
            FlowParams(mach_j=1.4, TR=1.0, Re=1.0e5, Cs=0.17, cfl=0.5, seed=2))


def jet_medium() -> tuple[GridSpec, FlowParams]:
    """192x128x72 jet (~1.77M points): the paper-scale jet at half resolution
    per axis, for profiling captures (state + metrics still far above L2)."""
    hy = 0.4 * 12.0 / 127
    hz = 0.4 * 12.0 / 71
    return (jet_grid(192, 128, 72, 30.0, 12.0, 12.0, hy, hz),
            FlowParams(mach_j=1.4, TR=1.0, Re=1.0e5, Cs=0.17, cfl=0.5, seed=3))


def jet_large() -> tuple[GridSpec, FlowParams]:
    """768x384x192 jet (~56.6M points), 30D x 12D x 12D, TR 2."""
    hy = 0.4 * 12.0 / 383
    hz = 0.4 * 12.0 / 191
    return (jet_grid(768, 384, 192, 30.0, 12.0, 12.0, hy, hz),
            FlowParams(mach_j=1.4, TR=2.0, Re=1.0e5, Cs=0.17, cfl=0.5, seed=5))


def polar_jet_paper_scale() -> tuple[GridSpec, FlowParams]:
    """The paper's mesh topology at its size (~14 M points): 384 axial x 192
    radial x 192 azimuthal, 30D long, radius 12D, centerline at j = 0."""
    return (polar_jet_grid(384, 192, 192, 30.0, 12.0),
            FlowParams(mach_j=1.4, TR=1.0, Re=1.0e5, Cs=0.17, cfl=0.5, seed=6))


def jet_slab(spec: GridSpec, k0: int, k1: int) -> GridSpec:
    """Planes k0..k1-1 of a grid (a bounded sample of a larger workload)."""
    ni, nj, nk = spec.dims
    sl = slice(k0 * ni * nj, k1 * ni * nj)
    return replace(spec, x=spec.x[sl].copy(), y=spec.y[sl].copy(), z=spec.z[sl].copy(),
                   dims=(ni, nj, k1 - k0))


def batch_jets(njets: int = 64, seed: int = 4) -> list[tuple[GridSpec, FlowParams]]:
    """Independent jets: dims uniform in [32,128]x[32,96]x[32,96], Mach U[1.2, 2],
    TR U[1, 3], Re_D U[5e4, 5e5], domain 20D x 10D x 10D, per-jet seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(njets):
        ni = int(rng.integers(32, 129))
        nj = int(rng.integers(32, 97))
        nk = int(rng.integers(32, 97))
        M = float(rng.uniform(1.2, 2.0))
        TR = float(rng.uniform(1.0, 3.0))
        Re = float(rng.uniform(5e4, 5e5))
        hy = 0.4 * 10.0 / (nj - 1)
        hz = 0.4 * 10.0 / (nk - 1)
        g = jet_grid(ni, nj, nk, 20.0, 10.0, 10.0, hy, hz)
        p = FlowParams(mach_j=M, TR=TR, Re=Re, Cs=0.17, cfl=0.5,
                       seed=int(rng.integers(1, 2**62)))
        out.append((g, p))
    return out


# ---------------------------------------------------------------------------
# Test grids
# ---------------------------------------------------------------------------

def wavy_periodic_grid(n: tuple, h: float = 1.0, amp: float = 0.2) -> GridSpec:
    """Fully periodic curvilinear grid: each coordinate is h*index plus a
    sinusoidal displacement in the other two indices (periodic extension with
    shifts n_a h along the own axis)."""
    ni, nj, nk = n
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    si, sj, sk = (np.sin(2 * np.pi * i / ni), np.sin(2 * np.pi * j / nj),
                  np.sin(2 * np.pi * k / nk))
    ci, cj = np.cos(2 * np.pi * i / ni), np.cos(2 * np.pi * j / nj)
    x = h * i + amp * h * sj * sk + 0.5 * amp * h * cj
    y = h * j + amp * h * si * sk + 0.5 * amp * h * ci
    z = h * k + amp * h * si * sj + 0.5 * amp * h * ci * cj
    shift = np.diag([ni * h, nj * h, nk * h]).astype(np.float64)
    return GridSpec(x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64),
                    z.reshape(-1).astype(np.float64), (ni, nj, nk), periodic=(1, 1, 1),
                    shift=shift, bc=(0, 0, 0, 0, 0, 0))


def wavy_box_grid(n: tuple, L: tuple = (4.0, 3.0, 3.0), amp: float = 0.05,
                  bc: tuple = (BC_FARFIELD,) * 6, periodic=(0, 0, 0)) -> GridSpec:
    """Non-periodic curvilinear box [0,Lx]x[-Ly/2,Ly/2]x[-Lz/2,Lz/2] with smooth
    interior waviness (boundary faces stay planar)."""
    ni, nj, nk = n
    s = [np.linspace(0, 1, m) for m in n]
    K, J, I = np.meshgrid(s[2], s[1], s[0], indexing="ij")
    bump = np.sin(np.pi * I) * np.sin(np.pi * J) * np.sin(np.pi * K)
    x = L[0] * I + amp * L[0] * bump * np.sin(2 * np.pi * J)
    y = L[1] * (J - 0.5) + amp * L[1] * bump * np.sin(2 * np.pi * K)
    z = L[2] * (K - 0.5) + amp * L[2] * bump * np.sin(2 * np.pi * I)
    shift = np.zeros((3, 3))
    for a in range(3):
        if periodic[a]:
            raise ValueError("wavy_box_grid is non-periodic")
    return GridSpec(x.reshape(-1), y.reshape(-1), z.reshape(-1), (ni, nj, nk),
                    periodic=periodic, shift=shift, bc=bc)


def periodic_box_grid(n: tuple, h: tuple = (1.0, 1.0, 1.0)) -> GridSpec:
    """Uniform fully periodic Cartesian box."""
    x1, y1, z1 = (np.arange(n[a]) * h[a] for a in range(3))
    g = product_grid(x1, y1, z1)
    g.periodic = (1, 1, 1)
    g.shift = np.diag([n[0] * h[0], n[1] * h[1], n[2] * h[2]]).astype(np.float64)
    g.bc = (0, 0, 0, 0, 0, 0)
    return g


# ---------------------------------------------------------------------------
# Initial primitive states (rho, u, v, w, p), 5 x N
# ---------------------------------------------------------------------------

def ambient_primitives(N: int, TR: float = 1.0, gamma: float = 1.4) -> np.ndarray:
    """Quiescent ambient: rho = TR (T_inf = 1/TR in jet units), u = 0, p = 1/gamma."""
    s = np.zeros((5, N))
    s[0] = TR
    s[4] = 1.0 / gamma
    return s


def smooth_random_primitives(spec: GridSpec, seed: int, amp: float = 0.05,
                             modes: int = 3, gamma: float = 1.4,
                             base_u=(0.3, -0.2, 0.1)) -> np.ndarray:
    """Smooth seeded perturbation of a uniform state, periodic in the grid
    indices (a sum of a few low Fourier modes per primitive variable)."""
    rng = np.random.default_rng(seed)
    ni, nj, nk = spec.dims
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    base = np.array([1.0, base_u[0], base_u[1], base_u[2], 1.0 / gamma])
    out = np.empty((5, spec.N))
    for f in range(5):
        acc = np.zeros_like(i, dtype=np.float64)
        for _ in range(modes):
            a, b, c = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            acc += rng.uniform(-1, 1) * np.cos(2 * np.pi * (a * i / ni + b * j / nj + c * k / nk) + ph)
        scale = base[f] if f in (0, 4) else 1.0
        out[f] = (base[f] + amp * scale * acc).reshape(-1)
    return out


def random_field_primitives(N: int, seed: int, gamma: float = 1.4) -> np.ndarray:
    """Unstructured seeded random state (positive rho and p) for stencil tests."""
    rng = np.random.default_rng(seed)
    s = np.empty((5, N))
    s[0] = rng.uniform(0.7, 1.3, N)
    s[1] = rng.uniform(-0.5, 1.5, N)
    s[2] = rng.uniform(-0.3, 0.3, N)
    s[3] = rng.uniform(-0.3, 0.3, N)
    s[4] = rng.uniform(0.6, 0.85, N)
    return s


def cylinder_points(r: float, n_theta: int, n_x: int, x0: float, x1: float) -> np.ndarray:
    """Probe surface: a cylinder of radius r around the jet axis, 3 x (n_x*n_theta)."""
    th = np.arange(n_theta) * 2 * np.pi / n_theta
    xs = np.linspace(x0, x1, n_x)
    X, TH = np.meshgrid(xs, th, indexing="ij")
    return np.stack([X.reshape(-1), (r * np.cos(TH)).reshape(-1), (r * np.sin(TH)).reshape(-1)])


def cylinder_panels(r: float, n_theta: int, n_x: int, x0: float, x1: float):
    """The probe cylinder of cylinder_points as FW-H panels: centres (the same
    points, same order), unit outward (radial) normals and areas
    r dtheta dx, halved at the two axial ends (trapezoid weights; the end
    caps are left open)."""
    xyz = cylinder_points(r, n_theta, n_x, x0, x1)
    th = np.arange(n_theta) * 2 * np.pi / n_theta
    TH = np.broadcast_to(th[None, :], (n_x, n_theta)).reshape(-1)
    nrm = np.stack([np.zeros_like(TH), np.cos(TH), np.sin(TH)])
    wx = np.full(n_x, (x1 - x0) / (n_x - 1))
    wx[0] *= 0.5
    wx[-1] *= 0.5
    area = np.repeat(wx * r * 2 * np.pi / n_theta, n_theta)
    return xyz, nrm, area


def observer_arc(radius: float, n: int, x_centre: float, deg0: float = 20.0, deg1: float = 120.0) -> np.ndarray:
    """Far-field microphones on an arc in the x-y plane about (x_centre, 0, 0),
    angles from the jet axis deg0..deg1: 3 x n."""
    a = np.radians(np.linspace(deg0, deg1, n))
    return np.stack([x_centre + radius * np.cos(a), radius * np.sin(a), np.zeros(n)])


def polar_jet_grid(ni: int, nj: int, nk: int, Lx: float, R: float, spacing_ratio: float = 6.0,
                   width: float = 0.5, spreading: float = 0.094, x_developed: float = 20.0) -> GridSpec:
    """The paper's jet mesh (Sec. "Mesh Generation"): a 2-D (x, r) mesh
    refined with hyperbolic tangents, rotated about the x axis.
    - i, axial: x = Lx (1 - tanh(1.2 (1 - s)) / tanh(1.2)), s uniform on
      [0, 1]: finest at the jet entrance x = 0, coarsening downstream.
    - j, radial, from the centerline r = 0 (a degenerate line, J^-1 = 0) to
      R: at every station the spacing is h (1 + (q - 1) tanh(|r - r_s| / w)),
      q = spacing_ratio, w = width, finest on the slip line r_s(x) = 1/2,
      which moves outward at the shear-layer growth rate `spreading` beyond
      x = x_developed (the self-similar region), and h is scaled so that the
      last point is r = R; the radial lines therefore bend with x.
    - k, azimuthal: nk unique angles 2 pi k / nk (periodic, no duplicated
      point).
    Faces: jet inflow at x = 0, exit at x = Lx, centerline at j = 0, far field
    at r = R.  (The paper gives the ingredients, not the functions: these are
    this package's choice.)"""
    s = np.linspace(0.0, 1.0, ni)
    x1 = Lx * (1.0 - np.tanh(1.2 * (1.0 - s)) / np.tanh(1.2))
    rs = 0.5 + spreading * np.maximum(0.0, x1 - x_developed)

    def march(c):
        # radial coordinates of all stations for spacing scale c (midpoint rule)
        r = np.zeros((nj, ni))
        h = lambda rr: c * (1.0 + (spacing_ratio - 1.0) * np.tanh(np.abs(rr - rs) / width))
        for jj in range(nj - 1):
            r[jj + 1] = r[jj] + h(r[jj] + 0.5 * h(r[jj]))
        return r

    lo = np.zeros(ni)
    hi = np.full(ni, R)
    for _ in range(80):  # bisection on the scale of every station at once
        mid = 0.5 * (lo + hi)
        over = march(mid)[-1] > R
        hi = np.where(over, mid, hi)
        lo = np.where(over, lo, mid)
    r2 = march(0.5 * (lo + hi))
    r2 *= R / r2[-1]  # the last point exactly on r = R
    r2[0] = 0.0
    th = 2.0 * np.pi * np.arange(nk) / nk
    K, J, Iax = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    x = x1[Iax].reshape(-1)
    rr = r2[J, Iax]
    y = (rr * np.cos(th[K])).reshape(-1)
    z = (rr * np.sin(th[K])).reshape(-1)
    return GridSpec(x=x, y=y, z=z, dims=(ni, nj, nk), periodic=(0, 0, 1),
                    shift=np.zeros((3, 3)),
                    bc=(BC_INFLOW_JET, BC_EXIT, BC_CENTERLINE, BC_FARFIELD, BC_PERIODIC, BC_PERIODIC))


def unique_periodic_planes(spec: GridSpec, tol: float = 1e-12) -> GridSpec:
    """Convert a grid in the paper's overlapping periodic form (Sec. "Periodic
    Boundary Condition": the last plane of a periodic axis repeats the first,
    shifted by the period) to the form the library takes, the unique planes:
    the repeated last plane of every such axis is dropped."""
    ni, nj, nk = spec.dims
    X = [c.reshape(nk, nj, ni) for c in (spec.x, spec.y, spec.z)]
    dims = [ni, nj, nk]
    for a in range(3):
        if not spec.periodic[a]:
            continue
        ax = 2 - a  # array axis of grid axis a ([k][j][i] layout)
        first = [np.take(c, 0, axis=ax) for c in X]
        last = [np.take(c, dims[a] - 1, axis=ax) for c in X]
        scale = max(1.0, max(np.abs(f).max() for f in first))
        if max(np.abs(l - (f + spec.shift[a][c])).max() for c, (f, l) in enumerate(zip(first, last))) <= tol * scale:
            X = [np.delete(c, dims[a] - 1, axis=ax) for c in X]
            dims[a] -= 1
    return GridSpec(x=X[0].reshape(-1).copy(), y=X[1].reshape(-1).copy(), z=X[2].reshape(-1).copy(),
                    dims=tuple(dims), periodic=spec.periodic, shift=spec.shift, bc=spec.bc)


def curved_periodic_grid(n: tuple, L: float = 1.0, A: float = 0.04) -> GridSpec:
    """Fully periodic curvilinear grid with a FIXED physical displacement of
    amplitude A (independent of the resolution, for refinement studies):
    x = L s_i + A sin(2 pi s_j) sin(2 pi s_k), etc., s_a = index_a / n_a."""
    ni, nj, nk = n
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    si, sj, sk = i / ni, j / nj, k / nk
    tp = 2 * np.pi
    x = L * si + A * np.sin(tp * sj) * np.sin(tp * sk)
    y = L * sj + A * np.sin(tp * si) * np.cos(tp * sk)
    z = L * sk + A * np.cos(tp * si) * np.sin(tp * sj)
    shift = np.diag([L, L, L]).astype(np.float64)
    return GridSpec(x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64),
                    z.reshape(-1).astype(np.float64), (ni, nj, nk), periodic=(1, 1, 1),
                    shift=shift, bc=(0, 0, 0, 0, 0, 0))
