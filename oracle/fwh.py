"""Far-field pressure from a permeable surface by the Ffowcs Williams-Hawkings
equation: the acoustic post-processing the paper's probe surface feeds (its
Sec. "Introduction" and "Concluding Remarks" name FW-H as the far-field
method but give no formulation).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the CUDA library
shares no code with it.  Plain numpy, FP64.

Formulation adopted (published, cited): Farassat's Formulation 1A
(F. Farassat, "Derivation of Formulations 1 and 1A of Farassat", NASA
TM-2007-214853, 2007) with the permeable-surface source terms of
P. di Francescantonio, J. Sound Vib. 202 (1997) 491-509, for a surface at
rest in a medium at rest (ambient rho0, p0, sound speed c0).  With the
surface unit outward normal n, the fluid density rho, velocity u and pressure
p on the surface,

    Q   = rho (u . n)                         (mass flux; rho0 U_n)
    L_i = (p - p0) n_i + rho u_i (u . n)      (momentum flux; viscous stress neglected)

and, at an observer x outside the surface, time t,

    4 pi p'(x, t) = int_S [ dQ/dtau / r  +  (dL_r/dtau) / (c0 r)  +  L_r / r^2 ]_ret dS

with r = |x - y|, L_r = L . (x - y) / r, each bracket evaluated at the
retarded (emission) time tau = t - r / c0 (the surface Mach number is zero,
so the Doppler factors of Formulation 1A are 1 and its surface-velocity
terms vanish).

Discretisation (none in the paper; this is the library's, and the oracle
follows it): the surface is a set of panels (centre y_j, unit outward normal
n_j, area A_j) and the integral their sum; the surface data come as frames
at tau_m = m dtau, m = 0..N-1; d/dtau is the second-order central difference
(F_{m+1} - F_{m-1}) / (2 dtau), one-sided second order (-3F_0 + 4F_1 - F_2)
/ (2 dtau) at the first frame and its mirror at the last; the retarded value
is the linear interpolation between the two frames around tau (s = tau/dtau,
m = floor(s) limited to [0, N-2], weight s - m).
"""
from __future__ import annotations

import numpy as np


def sources(frames: np.ndarray, nrm: np.ndarray, p0: float):
    """Q and L_i per frame and panel from frames [N][5][P] = (rho, u, v, w, p)
    and unit normals nrm [3][P]: returns Q [N][P] and L [3][N][P]."""
    rho, u, v, w, p = (frames[:, f, :] for f in range(5))
    un = u * nrm[0] + v * nrm[1] + w * nrm[2]
    Q = rho * un
    vel = (u, v, w)
    L = np.stack([(p - p0) * nrm[i] + rho * vel[i] * un for i in range(3)])
    return Q, L


def ddtau(F: np.ndarray, dtau: float, axis: int = 0) -> np.ndarray:
    """Second-order derivative along the frame axis: central inside,
    one-sided three-point at the two ends."""
    F = np.moveaxis(F, axis, 0)
    D = np.empty_like(F)
    D[1:-1] = (F[2:] - F[:-2]) / (2.0 * dtau)
    D[0] = (-3.0 * F[0] + 4.0 * F[1] - F[2]) / (2.0 * dtau)
    D[-1] = (3.0 * F[-1] - 4.0 * F[-2] + F[-3]) / (2.0 * dtau)
    return np.moveaxis(D, 0, axis)


def retarded(F: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Linear interpolation of F [N][P] at fractional frame positions
    s [..., P] (per panel)."""
    N = F.shape[0]
    m = np.clip(np.floor(s).astype(np.int64), 0, N - 2)
    wgt = s - m
    cols = np.arange(F.shape[1])
    return (1.0 - wgt) * F[m, cols] + wgt * F[m + 1, cols]


def pressure(frames: np.ndarray, xyz: np.ndarray, nrm: np.ndarray, area: np.ndarray, dtau: float,
             rho0: float, p0: float, c0: float, obs: np.ndarray, t0: float, dt_obs: float, nt: int) -> np.ndarray:
    """Acoustic pressure p' [M][nt] at observers obs [3][M] and times
    t_k = t0 + k dt_obs (frame m at tau = m dtau), from the surface frames
    [N][5][P] at panels xyz [3][P] with normals nrm [3][P] and areas area [P].
    (rho0 enters through the data: Q is rho u.n with the full density.)"""
    del rho0  # Q = rho0 U_n = rho u.n: the ambient density is in the data
    frames = np.asarray(frames, dtype=np.float64)
    Q, L = sources(frames, nrm, p0)
    Qd = ddtau(Q, dtau)
    Ld = ddtau(L, dtau, axis=1)
    M = obs.shape[1]
    out = np.zeros((M, nt))
    for o in range(M):
        d = obs[:, o, None] - xyz
        r = np.sqrt((d * d).sum(axis=0))
        rh = d / r
        for k in range(nt):
            s = (t0 + k * dt_obs - r / c0) / dtau
            qd = retarded(Qd, s)
            lr = sum(retarded(L[i], s) * rh[i] for i in range(3))
            lrd = sum(retarded(Ld[i], s) * rh[i] for i in range(3))
            out[o, k] = (area * (qd / r + lrd / (c0 * r) + lr / (r * r))).sum() / (4.0 * np.pi)
    return out
