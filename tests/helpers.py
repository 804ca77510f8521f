"""Test helpers: input conversion and textbook reference solutions.

Nothing here implements the LES scheme; the reference solutions are
independent textbook results (exact Riemann problem, Runge-Kutta
amplification polynomial of a given coefficient set).
"""
import math

import numpy as np


def to_oracle(spec, fp):
    """Seeded GridSpec/FlowParams -> oracle Grid/Params."""
    import oracle
    g = oracle.Grid(x=spec.x, y=spec.y, z=spec.z, dims=tuple(spec.dims),
                    periodic=tuple(spec.periodic), shift=np.asarray(spec.shift),
                    bc=tuple(spec.bc))
    p = oracle.Params(**{k: getattr(fp, k) for k in oracle.Params.__dataclass_fields__})
    return g, p


def rk_amplification(z, alphas):
    """One-step amplification of the low-storage multistage scheme
    Q(l) = Q(0) + alpha_l z Q(l-1) applied to dQ/dt = lambda Q, z = lambda dt."""
    g = 1.0 + 0j
    for a in alphas:
        g = 1.0 + a * z * g
    return g


def exact_riemann(WL, WR, gamma, S):
    """Exact solution of the 1-D Euler Riemann problem (Toro, Riemann Solvers
    and Numerical Methods for Fluid Dynamics, Ch. 4) sampled at S = x/t.
    WL, WR = (rho, u, p).  Returns arrays rho, u, p."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    al, ar = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1) / (2 * gamma)
    g2 = (gamma + 1) / (2 * gamma)

    def fk(p, rk, pk, ak):
        if p > pk:
            A = 2.0 / ((gamma + 1) * rk)
            B = (gamma - 1) / (gamma + 1) * pk
            f = (p - pk) * math.sqrt(A / (p + B))
            df = math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        else:
            f = 2 * ak / (gamma - 1) * ((p / pk) ** g1 - 1)
            df = 1.0 / (rk * ak) * (p / pk) ** (-g2)
        return f, df

    p = 0.5 * (pl + pr)
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, al)
        f2, d2 = fk(p, rr, pr, ar)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-14 * p:
            break
    f1, _ = fk(p, rl, pl, al)
    f2, _ = fk(p, rr, pr, ar)
    us = 0.5 * (ul + ur) + 0.5 * (f2 - f1)
    ps = p
    S = np.atleast_1d(np.asarray(S, dtype=np.float64))
    rho = np.empty_like(S)
    u = np.empty_like(S)
    pp = np.empty_like(S)
    gm1, gp1 = gamma - 1, gamma + 1
    for n, s in enumerate(S):
        if s <= us:
            if ps > pl:
                SL = ul - al * math.sqrt(g2 * ps / pl + g1)
                if s <= SL:
                    rho[n], u[n], pp[n] = rl, ul, pl
                else:
                    rho[n] = rl * (ps / pl + gm1 / gp1) / (gm1 / gp1 * ps / pl + 1)
                    u[n], pp[n] = us, ps
            else:
                SHL = ul - al
                aSL = al * (ps / pl) ** g1
                STL = us - aSL
                if s <= SHL:
                    rho[n], u[n], pp[n] = rl, ul, pl
                elif s >= STL:
                    rho[n] = rl * (ps / pl) ** (1 / gamma)
                    u[n], pp[n] = us, ps
                else:
                    uu = 2 / gp1 * (al + gm1 / 2 * ul + s)
                    aa = 2 / gp1 * (al + gm1 / 2 * (ul - s))
                    rho[n] = rl * (aa / al) ** (2 / gm1)
                    u[n] = uu
                    pp[n] = pl * (aa / al) ** (2 * gamma / gm1)
        else:
            if ps > pr:
                SR = ur + ar * math.sqrt(g2 * ps / pr + g1)
                if s >= SR:
                    rho[n], u[n], pp[n] = rr, ur, pr
                else:
                    rho[n] = rr * (ps / pr + gm1 / gp1) / (gm1 / gp1 * ps / pr + 1)
                    u[n], pp[n] = us, ps
            else:
                SHR = ur + ar
                aSR = ar * (ps / pr) ** g1
                STR = us + aSR
                if s >= SHR:
                    rho[n], u[n], pp[n] = rr, ur, pr
                elif s <= STR:
                    rho[n] = rr * (ps / pr) ** (1 / gamma)
                    u[n], pp[n] = us, ps
                else:
                    uu = 2 / gp1 * (-ar + gm1 / 2 * ur + s)
                    aa = 2 / gp1 * (ar - gm1 / 2 * (ur - s))
                    rho[n] = rr * (aa / ar) ** (2 / gm1)
                    u[n] = uu
                    pp[n] = pr * (aa / ar) ** (2 * gamma / gm1)
    return rho, u, pp


def rel_l2(a, b):
    """Relative L2 error per field (rows)."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    num = np.sqrt(((a - b) ** 2).sum(axis=1))
    den = np.sqrt((b ** 2).sum(axis=1))
    return num / np.where(den > 0, den, 1.0)


def error_split(a, b, dims, margin=1):
    """FP32-against-FP64 error decomposition on a grid of dims (ni, nj, nk):
    relative L2 per field over the whole grid, over the interior (points at
    least `margin` from every face) and the share of each field's squared
    error that lies on the inflow plane i = 0."""
    ni, nj, nk = dims
    a = np.asarray(a).reshape(5, nk, nj, ni)
    b = np.asarray(b).reshape(5, nk, nj, ni)
    d2 = (a - b) ** 2
    den = np.sqrt((b.reshape(5, -1) ** 2).sum(axis=1))
    whole = np.sqrt(d2.reshape(5, -1).sum(axis=1)) / den
    m = margin
    inner = np.sqrt(d2[:, m:nk - m, m:nj - m, m:ni - m].reshape(5, -1).sum(axis=1)) / den
    tot = np.maximum(d2.reshape(5, -1).sum(axis=1), 1e-300)
    share_i0 = d2[:, :, :, 0].reshape(5, -1).sum(axis=1) / tot
    return whole, inner, share_i0
