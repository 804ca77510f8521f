"""Oracle pins for the parts of the artificial dissipation that act at the ends
of a non-periodic axis and for the exact value of the pressure sensor.

- Boundary fourth difference (Sec. "Centerline Boundary Condition"): the paper
  prints the dissipation of the first interface next to a boundary point as
  d = (dw)_{j+3/2} - 3 (dw)_{j+1/2}, the result of the extrapolation
  (dw)_outside = -(dw)_adjacent.  On a line of points with a density-only
  perturbation, zero velocity, uniform pressure, k2 = 0 and no viscosity,
  every term of the residual but that fourth difference cancels, so the
  residual at the first and last interior points is the printed boundary
  stencil weighted by the interface spectral radius; the test evaluates it by
  hand, in the printed form, and the oracle must agree.  The same residual with
  the extrapolation's sign flipped, (dw)_outside = +(dw)_adjacent, is shown
  to differ.
- Pressure sensor (Eq. p_grad_sensor, reading R5): exact rational values on a
  pressure profile chosen by hand, including the end-point rule (an end point
  of a non-periodic axis takes its interior neighbour's value).
- Far-field branch at a normal velocity of zero (Sec. "Far Field Boundary",
  reading R14): a perturbation of a fluid at rest at the level of rounding
  must not change the boundary state, while a weak but physical inflow or
  outflow must take the paper's entrance or exit side.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import to_oracle
from paper_2212_12365_gb300 import inputs as I

GAMMA = 1.4


def _line_grid(ni, hx, hy, hz, nj=4, nk=4):
    """Uniform Cartesian line: i non-periodic (far-field faces, which the
    residual does not touch), j and k periodic with a uniform state along
    them."""
    spec = I.product_grid(np.arange(ni) * hx, np.arange(nj) * hy, np.arange(nk) * hz)
    spec.periodic = (0, 1, 1)
    spec.shift = np.diag([0.0, nj * hy, nk * hz])
    spec.bc = (I.BC_FARFIELD, I.BC_FARFIELD, 0, 0, 0, 0)
    return spec


def _line_state(spec, rho_i, p0):
    ni, nj, nk = spec.dims
    prim = np.zeros((5, spec.N))
    prim[0] = np.tile(rho_i, nj * nk)
    prim[4] = p0
    return prim


def _hand_residual_rho(rho, p0, k4, hx, hy, hz, flipped=False):
    """Continuity residual at the interior points of the line from the
    paper's interior stencil, Eq. dissip_term with eps2 = 0, and its printed
    boundary stencil at the two interfaces next to the end points."""
    n = len(rho)
    c = np.sqrt(GAMMA * p0 / rho)
    # spectral radii of a fluid at rest on a uniform grid: c |grad xi^a|
    lx, ly, lz = c / hx, c / hy, c / hz
    lbar = lx + np.sqrt(lx * ly) + np.sqrt(lx * lz)
    jinv = hx * hy * hz
    dW = np.diff(rho)  # (dw)_{i+1/2}, i = 0 .. n-2
    D3 = np.empty(n - 1)
    for i in range(n - 1):
        if i == 0:
            # printed: d_{j+1/2} = (dw)_{j+3/2} - 3 (dw)_{j+1/2}
            D3[i] = dW[1] - 3.0 * dW[0] if not flipped else dW[1] - dW[0]
        elif i == n - 2:
            # the same extrapolation at the other end, mirrored
            D3[i] = -3.0 * dW[i] + dW[i - 1] if not flipped else -dW[i] + dW[i - 1]
        else:
            D3[i] = dW[i + 1] - 2.0 * dW[i] + dW[i - 1]
    lam_face = 0.5 * (lbar[:-1] + lbar[1:])
    # numerical flux H = average - J^-1 d, d = lambda (eps2 dW - eps4 D3)
    H = jinv * lam_face * k4 * D3
    return H[1:] - H[:-1]  # residual at points 1 .. n-2


@pytest.mark.parametrize("ni", [6, 9])
def test_boundary_fourth_difference_matches_printed_stencil(ni):
    hx, hy, hz = 0.3, 0.7, 1.1
    rng = np.random.default_rng(5)
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, ni)
    p0 = 1.0 / GAMMA
    k4 = 0.016
    spec = _line_grid(ni, hx, hy, hz)
    fp = I.FlowParams(Re=math.inf, Cs=0.0, k2=0.0, k4=k4)
    g, P = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.qhat_from(g, P, m, _line_state(spec, rho, p0), True)
    r = oracle.rhs(g, P, m, q).reshape(5, -1, ni)  # [field][j,k][i]
    want = _hand_residual_rho(rho, p0, k4, hx, hy, hz)
    scale = np.abs(want).max()
    for jk in range(r.shape[1]):
        np.testing.assert_allclose(r[0, jk, 1:-1], want, rtol=0, atol=1e-12 * scale)
        # momentum and energy: uniform pressure flux and uniform total enthalpy
        assert np.abs(r[1:, jk]).max() <= 1e-12 * scale
    # the extrapolation with the opposite sign gives another residual at the
    # two boundary-adjacent points (and only there)
    flipped = _hand_residual_rho(rho, p0, k4, hx, hy, hz, flipped=True)
    diff = np.abs(flipped - want)
    assert diff[0] > 1e-3 * scale and diff[-1] > 1e-3 * scale
    assert np.all(diff[2:-2] == 0.0)


def test_pressure_sensor_exact_values_and_end_rule():
    """p = p_s (1, 1, 1.5, 3, 3, 2, 2, 5) along a non-periodic line: interior
    values |p+ - 2p + p-| / (p+ + 2p + p-) are 1/9, 1/7, 1/7, 1/11, 1/9, 3/11
    (by hand), and the end points repeat their neighbours' values."""
    prof = np.array([1.0, 1.0, 1.5, 3.0, 3.0, 2.0, 2.0, 5.0])
    want_interior = np.array([1 / 9, 1 / 7, 1 / 7, 1 / 11, 1 / 9, 3 / 11])
    want = np.concatenate([[want_interior[0]], want_interior, [want_interior[-1]]])
    ni = len(prof)
    spec = _line_grid(ni, 0.25, 0.5, 0.5)
    g, P = to_oracle(spec, I.FlowParams())
    m = oracle.metrics(g)
    prim = _line_state(spec, np.full(ni, 1.3), 0.0)
    prim[4] = np.tile(prof / GAMMA, 16)
    q = oracle.qhat_from(g, P, m, prim, True)
    nu = oracle.point_field(g, P, m, q, oracle.FIELD_SENSOR[0]).reshape(-1, ni)
    for row in nu:
        np.testing.assert_allclose(row, want, rtol=1e-14, atol=0)
    # along the periodic axes the pressure is uniform: no sensor there
    for a in (1, 2):
        assert np.abs(oracle.point_field(g, P, m, q, oracle.FIELD_SENSOR[a])).max() == 0.0


def _farfield(P, rho, u, p, n):
    u = np.asarray(u, dtype=np.float64)
    Qe = np.array([rho, *(rho * u), p / (GAMMA - 1) + 0.5 * rho * (u @ u)])
    Qf = oracle.face_state(P, "farfield", Qe, n)
    rf = Qf[0]
    uf = Qf[1:4] / rf
    pf = (GAMMA - 1) * (Qf[4] - 0.5 * rf * (uf @ uf))
    return rf, uf, pf


def test_farfield_branch_insensitive_to_rounding_at_rest():
    """A fluid at rest next to a far-field face, its normal velocity
    perturbed at the level of rounding (|q_n| / c of 1e-16 .. 1e-13, either
    sign, as two evaluation orders of the same state give), yields the same
    face state to within that level; a weak physical inflow (q_n / c = -1e-5)
    takes the freestream's tangential velocity and entropy, a weak outflow
    (+1e-5) the interior's."""
    P = to_oracle(I.periodic_box_grid((4, 4, 4)), I.FlowParams(TR=1.0))[1]
    n = np.array([0.0, -1.0, 0.0])  # outward normal of a j- face
    c = 1.0  # sound speed of the ambient state (TR = 1)
    rho, p = 1.02, 1.0 / GAMMA * 0.99  # slightly off-ambient interior entropy
    tang = np.array([0.01, 0.0, -0.02])  # tangential velocity of the interior point
    ref = _farfield(P, rho, tang, p, n)
    for eps in (1e-16, -1e-16, 3e-14, -3e-14, 1e-13, -1e-13):
        got = _farfield(P, rho, tang - eps * c * n, p, n)
        assert abs(got[0] - ref[0]) <= 1e-12 * ref[0]
        np.testing.assert_allclose(got[1] - (got[1] @ n) * n, tang, atol=1e-12)
        assert abs(got[2] - ref[2]) <= 1e-12 * ref[2]
    # physical weak waves follow the paper's sign rule
    r_in, u_in, p_in = _farfield(P, rho, tang - 1e-5 * c * n, p, n)
    np.testing.assert_allclose(u_in - (u_in @ n) * n, 0.0, atol=1e-15)  # freestream at rest
    assert p_in / r_in**GAMMA == pytest.approx((1 / GAMMA) / 1.0**GAMMA, rel=1e-12)
    r_out, u_out, p_out = _farfield(P, rho, tang + 1e-5 * c * n, p, n)
    np.testing.assert_allclose(u_out - (u_out @ n) * n, tang, atol=1e-15)
    assert p_out / r_out**GAMMA == pytest.approx(p / rho**GAMMA, rel=1e-12)
