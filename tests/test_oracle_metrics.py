"""Oracle pins for the metric terms and Jacobian (Sec. "Transformation of
Coordinates"): exactness on affine grids, second-order convergence to the
analytic cofactors, and the discrete geometric conservation law that makes a
uniform flow an exact discrete steady state on curved grids."""
import numpy as np
import pytest

import oracle
from helpers import to_oracle
from paper_2212_12365_gb300 import inputs as I


def _affine_spec(A, b, n, periodic=(0, 0, 0)):
    ni, nj, nk = n
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    idx = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)]).astype(np.float64)
    X = A @ idx + np.asarray(b)[:, None]
    shift = np.zeros((3, 3))
    for a in range(3):
        if periodic[a]:
            shift[a] = A[:, a] * n[a]
    return I.GridSpec(X[0].copy(), X[1].copy(), X[2].copy(), n, periodic=periodic, shift=shift,
                      bc=tuple(0 if periodic[f // 2] else 1 for f in range(6)))


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 0, 1), (1, 1, 1)])
def test_affine_grid_metrics_exact(periodic):
    """x = A xi + b: J^-1 = det A and J^-1 d xi^a/d x_c = det(A) (A^-1)[a, c]
    at every point, including one-sided end points and periodic seams."""
    A = np.array([[1.3, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.15, 1.1]])
    spec = _affine_spec(A, [0.3, -1.0, 2.0], (6, 5, 7), periodic)
    g, _ = to_oracle(spec, I.FlowParams())
    m = oracle.metrics(g)
    C = np.linalg.det(A) * np.linalg.inv(A)
    for a in range(3):
        for c in range(3):
            np.testing.assert_allclose(m[3 * a + c], C[a, c], rtol=0, atol=1e-12)
    np.testing.assert_allclose(m[9], np.linalg.det(A), rtol=1e-13)


def _smooth_map(n):
    """Non-periodic smooth mapping of the unit cube with index spacing h."""
    ni = nj = nk = n
    h = 1.0 / (n - 1)
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    s, t, u = i * h, j * h, k * h
    e = 0.1
    x = s + e * np.sin(np.pi * t) * np.sin(np.pi * u)
    y = t + e * np.sin(np.pi * s) * np.cos(np.pi * u)
    z = u + e * np.sin(np.pi * s + 0.3) * np.sin(np.pi * t)
    pi = np.pi
    # analytic derivatives d(x,y,z)/d(s,t,u)
    J = np.empty((3, 3) + s.shape)
    J[0, 0] = 1.0
    J[0, 1] = e * pi * np.cos(pi * t) * np.sin(pi * u)
    J[0, 2] = e * pi * np.sin(pi * t) * np.cos(pi * u)
    J[1, 0] = e * pi * np.cos(pi * s) * np.cos(pi * u)
    J[1, 1] = 1.0
    J[1, 2] = -e * pi * np.sin(pi * s) * np.sin(pi * u)
    J[2, 0] = e * pi * np.cos(pi * s + 0.3) * np.sin(pi * t)
    J[2, 1] = e * pi * np.sin(pi * s + 0.3) * np.cos(pi * t)
    J[2, 2] = 1.0
    spec = I.GridSpec(x.reshape(-1), y.reshape(-1), z.reshape(-1), (ni, nj, nk),
                      bc=(1,) * 6)
    return spec, J.reshape(3, 3, -1), h


def test_metrics_second_order_convergence():
    """Cofactors/h^2 and J^-1/h^3 converge at second order to the analytic
    adjugate and determinant of d(x,y,z)/d(s,t,u) (all points, ends included)."""
    errs = []
    for n in (17, 33):
        spec, J, h = _smooth_map(n)
        g, _ = to_oracle(spec, I.FlowParams())
        m = oracle.metrics(g)
        Jm = np.moveaxis(J, -1, 0)  # (N, 3, 3): [x_c][xi^a]
        det = np.linalg.det(Jm)
        adj = np.linalg.inv(Jm) * det[:, None, None]  # [a][c] = det * d xi^a / d x_c
        e_cof = max(np.abs(m[3 * a + c] / h**2 - adj[:, a, c]).max()
                    for a in range(3) for c in range(3))
        e_det = np.abs(m[9] / h**3 - det).max()
        errs.append((e_cof, e_det))
    for q in range(2):
        order = np.log2(errs[0][q] / errs[1][q])
        assert order > 1.8, (errs, order)


@pytest.mark.parametrize("amp", [0.1, 0.25])
def test_gcl_freestream_wavy_periodic(amp):
    """Uniform flow on a curved periodic grid is an exact discrete steady state
    (all terms on): max |RHS| at round-off relative to the flux scale."""
    spec = I.wavy_periodic_grid((12, 10, 8), amp=amp)
    fp = I.FlowParams(Re=100.0, Cs=0.17)
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    prim = np.zeros((5, g.N))
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1.2, 0.7, -0.3, 0.2, 1 / 1.4
    q = oracle.qhat_from(g, p, m, prim, True)
    r = oracle.rhs(g, p, m, q)
    assert np.abs(r).max() < 1e-13


def test_gcl_freestream_wavy_box_interior():
    """Same on a non-periodic curved box (one-sided metrics at the ends): the
    interior residual of a uniform flow vanishes to round-off."""
    spec = I.wavy_box_grid((14, 11, 9), amp=0.08)
    g, p = to_oracle(spec, I.FlowParams(Re=1000.0))
    m = oracle.metrics(g)
    prim = np.zeros((5, g.N))
    prim[0], prim[1], prim[2], prim[3], prim[4] = 0.9, 1.1, 0.2, -0.4, 0.8
    q = oracle.qhat_from(g, p, m, prim, True)
    r = oracle.rhs(g, p, m, q)
    assert np.abs(r).max() < 2e-13
