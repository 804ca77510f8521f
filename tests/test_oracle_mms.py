"""Manufactured-solution order pins for the full spatial operator.

For a smooth analytic state, RHS / J^-1 must converge at second order to the
exact divergence of the continuous filtered Navier-Stokes fluxes (System I
with the Smagorinsky/Eidson closures, Secs. "Large Eddy Simulation
Formulation" and "Subgrid Scale Modeling", in the jet-unit scaling of Sec.
"Dimensionless Formulation").  The artificial dissipation is third order and
must not spoil this.  The exact divergence is computed independently of the
oracle: sympy gives the exact first derivatives of the primitives, and the
divergence of the flux vectors is taken by complex-step differentiation.
A dropped term, a wrong sign or a transposed metric gives an O(1) error.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import to_oracle
from paper_2212_12365_gb300 import inputs as I

sp = pytest.importorskip("sympy")

GAMMA = 1.4


def _analytic():
    x, y, z = sp.symbols("x y z")
    tp = 2 * sp.pi
    rho = 1 + sp.Rational(1, 10) * sp.sin(tp * x) * sp.cos(tp * y) + sp.Rational(1, 20) * sp.cos(tp * z)
    # velocity with a rotating shear (u, w) ~ (sin, cos)(2 pi y), whose strain
    # magnitude is constant, plus smaller 3-D modes: |S| stays well away from
    # zero (|S| is not smooth where S = 0, which the SGS check must avoid)
    u = (sp.Rational(2, 5) + sp.Rational(1, 10) * sp.sin(tp * y)
         + sp.Rational(1, 50) * sp.cos(tp * (z - x)))
    v = -sp.Rational(1, 5) + sp.Rational(1, 50) * sp.cos(tp * (2 * x - y + z))
    w = (sp.Rational(1, 10) + sp.Rational(1, 10) * sp.cos(tp * y)
         + sp.Rational(1, 50) * sp.sin(tp * (x + 2 * z + sp.Rational(7, 10))))
    p = 1 / sp.Float(GAMMA) + sp.Rational(1, 20) * sp.cos(tp * y) * sp.sin(tp * x + 1)
    T = GAMMA * p / rho
    prims = [rho, u, v, w, p]
    grads = [[sp.diff(f, s) for s in (x, y, z)] for f in (u, v, w, T)]
    fp = sp.lambdify((x, y, z), prims, "numpy")
    fg = sp.lambdify((x, y, z), grads, "numpy")
    return fp, fg


def test_manufactured_strain_nonvanishing():
    """Precondition of the Smagorinsky check: |S| is bounded away from zero.
    The rotating shear alone gives |S| = 2 pi 0.1; the other modes change the
    strain components by at most 3 * 2 pi 0.02 * 2 in magnitude."""
    fp, fg = _analytic()
    g = np.linspace(0, 1, 48, endpoint=False)
    X = np.stack([a.reshape(-1) for a in np.meshgrid(g, g, g, indexing="ij")])
    G = [[np.asarray(a) * np.ones_like(X[0]) for a in row] for row in fg(*X)]
    SS = sum((0.5 * (G[i][j] + G[j][i])) ** 2 for i in range(3) for j in range(3))
    assert np.sqrt(2 * SS).min() > 0.2


def _fluxes(X, fp, fg, P, CsDelta):
    """Continuous flux vectors F^c - F_v^c (c = x, y, z) at points X (3 x M,
    may be complex).  Returns array (3, 5, M)."""
    rho, u, v, w, p = [np.asarray(a) * np.ones_like(X[0]) for a in fp(*X)]
    G = [[np.asarray(a) * np.ones_like(X[0]) for a in row] for row in fg(*X)]
    vel = [u, v, w]
    T = GAMMA * p / rho
    S1 = P.S1_dim / (P.TR * P.T_inf_dim)
    mu = T**1.5 * (1 + S1) / (T + S1)
    Sij = [[0.5 * (G[i][j] + G[j][i]) for j in range(3)] for i in range(3)]
    SS = sum(Sij[i][j] * Sij[i][j] for i in range(3) for j in range(3))
    musgs = rho * CsDelta**2 * np.sqrt(2 * SS)
    div = Sij[0][0] + Sij[1][1] + Sij[2][2]
    tau = [[2 * (mu / P.Re + musgs) * (Sij[i][j] - (div / 3 if i == j else 0)) for j in range(3)]
           for i in range(3)]
    kap = (mu / P.Re) / ((GAMMA - 1) * P.Pr) + musgs / ((GAMMA - 1) * P.Pr_sgs)
    e = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)
    out = []
    for c in range(3):
        uc = vel[c]
        inv = [rho * uc, rho * u * uc + (p if c == 0 else 0), rho * v * uc + (p if c == 1 else 0),
               rho * w * uc + (p if c == 2 else 0), (e + p) * uc]
        beta_c = tau[c][0] * u + tau[c][1] * v + tau[c][2] * w + kap * G[3][c]
        visc = [0 * rho, tau[0][c], tau[1][c], tau[2][c], beta_c]
        out.append([inv[f] - visc[f] for f in range(5)])
    return np.array(out)


def _exact_divergence(X, fp, fg, P, CsDelta):
    h = 1e-30
    div = np.zeros((5, X.shape[1]))
    for c in range(3):
        Xc = X.astype(np.complex128)
        Xc[c] += 1j * h
        F = _fluxes(Xc, fp, fg, P, CsDelta)
        div += F[c].imag / h
    return div


def _mms_error(spec, fp, CsDelta, P_over=None):
    g, P = to_oracle(spec, fp)
    m = oracle.metrics(g)
    fpr, fgr = _analytic()
    X = np.stack([spec.x, spec.y, spec.z])
    prim = np.array([np.asarray(a) * np.ones_like(X[0]) for a in fpr(*X)])
    q = oracle.qhat_from(g, P, m, prim, True)
    r = oracle.rhs(g, P, m, q)
    ex = _exact_divergence(X, fpr, fgr, P, CsDelta)
    return np.abs(r / m[9] - ex).max(axis=1), np.abs(ex).max(axis=1)


def test_mms_second_order_curved_grid():
    """Curved periodic grid (fixed physical waviness), molecular viscosity at
    Re = 50, Sutherland mu(T), heat flux, artificial dissipation on, no SGS."""
    errs = []
    for n in (16, 32):
        spec = I.curved_periodic_grid((n, n, n), L=1.0, A=0.04)
        fp = I.FlowParams(Re=50.0, Cs=0.0, k2=0.25, k4=0.016)
        e, scale = _mms_error(spec, fp, 0.0)
        errs.append(e / scale)
    order = np.log2(errs[0] / errs[1])
    assert np.all(order > 1.8), (errs, order)
    assert np.all(errs[1] < 0.05), errs


def test_mms_second_order_smagorinsky():
    """Uniform periodic grid with Cs = C0/h so that Cs*Delta = C0 is fixed under
    refinement: the discrete mu_sgs = rho (Cs Delta)^2 |S| and the Eidson
    k_sgs = mu_sgs Cp / Pr_sgs enter the fluxes at second order."""
    C0 = 0.08
    errs = []
    for n in (16, 32):
        h = 1.0 / n
        spec = I.periodic_box_grid((n, n, n), (h, h, h))
        fp = I.FlowParams(Re=1.0e4, Cs=C0 / h, k2=0.25, k4=0.016)
        e, scale = _mms_error(spec, fp, C0)
        errs.append(e / scale)
    order = np.log2(errs[0] / errs[1])
    assert np.all(order > 1.8), (errs, order)
