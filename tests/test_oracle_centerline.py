"""Oracle pins for the paper's polar jet mesh and its centerline condition
(Secs. "Mesh Generation", "Centerline Boundary Condition").

The mesh is a 2-D (x, r) mesh rotated about the x axis, so the j = 0 line is
the degenerate axis with J^-1 = 0.  Pinned here, independently of the
oracle's own arithmetic:
- the axis is exactly degenerate and every other point has a positive J^-1;
- a uniform (also oblique) stream is preserved to round-off, including at
  the first ring whose stencils reach the axis (the conservative metric form
  keeps the discrete metric identities there);
- the centerline state is the azimuthal mean of the first ring's unscaled
  conserved variables (numpy mean), the same at every azimuth, invariant
  under a rotation of the ring data, and a purely radial velocity field
  gives no transverse momentum on the axis.
"""
import numpy as np
import pytest

import oracle
from helpers import to_oracle
from paper_2212_12365_gb300 import inputs as I


def _setup(dims=(12, 9, 16), Re=1e3, Lx=6.0):
    spec = I.polar_jet_grid(*dims, Lx, 3.0)
    fp = I.FlowParams(Re=Re)
    g, p = to_oracle(spec, fp)
    return spec, fp, g, p, oracle.metrics(g)


def test_polar_axis_degenerate():
    spec, _, _, _, m = _setup()
    ni, nj, nk = spec.dims
    J = m[9].reshape(nk, nj, ni)
    assert np.all(J[:, 0, :] == 0.0)
    assert J[:, 1:, :].min() > 0.0


@pytest.mark.parametrize("Lx", [6.0, 30.0])  # 30: radial lines bend past x = 20
@pytest.mark.parametrize("vel", [(1.4, 0.0, 0.0), (1.2, 0.3, -0.2)])
def test_polar_freestream_preserved(vel, Lx):
    spec, fp, g, p, m = _setup(Lx=Lx)
    prim = np.zeros((5, spec.N))
    prim[0] = 1.0
    prim[1:4] = np.array(vel)[:, None]
    prim[4] = 1.0 / fp.gamma
    q = oracle.qhat_from(g, p, m, prim, True)
    r = oracle.rhs(g, p, m, q)
    # flux scale: rho u^2 + p times the largest cofactor
    scale = (1.0 + np.sum(np.square(vel))) * np.abs(m[:9]).max()
    assert np.abs(r).max() <= 1e-13 * scale, np.abs(r).max(axis=1)


def _ring_state(spec, fp, seed):
    prim = I.smooth_random_primitives(spec, seed, amp=0.08)
    return prim


def test_centerline_is_azimuthal_mean_of_first_ring():
    spec, fp, g, p, m = _setup()
    ni, nj, nk = spec.dims
    prim = _ring_state(spec, fp, 3)
    q = oracle.qhat_from(g, p, m, prim, True)
    qb = oracle.apply_bc(g, p, m, q, 0)
    Q = oracle.state_out(g, p, m, qb, False).reshape(5, nk, nj, ni)
    # the first ring is interior (not touched by the boundary pass) except at
    # the x faces, which the x pass (applied after y) overwrites afterwards
    Qin = oracle.state_out(g, p, m, q, False).reshape(5, nk, nj, ni)
    mean = Qin[:, :, 1, :].mean(axis=1)  # numpy mean over k of the unscaled ring
    for i in range(1, ni - 1):
        for k in range(nk):
            np.testing.assert_allclose(Q[:, k, 0, i], mean[:, i], rtol=1e-14, atol=1e-15)


def test_centerline_rotation_invariant_and_radial_flow_cancels():
    spec, fp, g, p, m = _setup()
    ni, nj, nk = spec.dims
    x = spec.x.reshape(nk, nj, ni)
    y = spec.y.reshape(nk, nj, ni)
    z = spec.z.reshape(nk, nj, ni)
    r = np.sqrt(y ** 2 + z ** 2)
    prim = np.zeros((5, nk, nj, ni))
    prim[0] = 1.0 + 0.1 * np.sin(x)
    prim[1] = 1.0
    # purely radial velocity U_r(r) e_r, no swirl
    ur = 0.2 * r
    with np.errstate(invalid="ignore", divide="ignore"):
        prim[2] = np.where(r > 0, ur * y / np.where(r > 0, r, 1), 0.0)
        prim[3] = np.where(r > 0, ur * z / np.where(r > 0, r, 1), 0.0)
    prim[4] = 1.0 / fp.gamma
    q = oracle.qhat_from(g, p, m, prim.reshape(5, -1), True)
    Q = oracle.state_out(g, p, m, oracle.apply_bc(g, p, m, q, 0), False).reshape(5, nk, nj, ni)
    assert np.abs(Q[2:4, :, 0, 1:-1]).max() <= 1e-15
    # rotate the data by one azimuthal index: the axis state is unchanged
    qr = np.roll(prim.reshape(5, nk, nj, ni), 1, axis=1).reshape(5, -1)
    qr[2:4] = prim.reshape(5, -1)[2:4]  # keep the Cartesian velocity field of the unrotated data
    Q1 = oracle.state_out(g, p, m, oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, qr, True), 0),
                          False).reshape(5, nk, nj, ni)
    np.testing.assert_allclose(Q1[[0, 1, 4], :, 0, 1:-1], Q[[0, 1, 4], :, 0, 1:-1], rtol=1e-15, atol=1e-15)


def test_polar_jet_steps_stay_finite_and_axis_consistent():
    spec, fp, g, p, m = _setup((16, 10, 12), Re=1e4)
    prim = I.ambient_primitives(spec.N, fp.TR)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    dt = oracle.dt_cfl(g, p, m, q)
    q5 = oracle.step(g, p, m, q, 5, 0, dt)
    ni, nj, nk = spec.dims
    Q = oracle.state_out(g, p, m, q5, False).reshape(5, nk, nj, ni)
    assert np.all(np.isfinite(Q))
    # the axis carries one state per x station (the x faces, applied last,
    # own their edge points)
    assert np.abs(Q[:, :, 0, 1:-1] - Q[:, :1, 0, 1:-1]).max() == 0.0
    # the jet has entered: axis velocity at the inflow equals the jet Mach number
    assert Q[1, 0, 0, 0] / Q[0, 0, 0, 0] == pytest.approx(fp.mach_j, rel=1e-2)
