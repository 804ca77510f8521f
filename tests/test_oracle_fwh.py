"""Pins of the FW-H oracle (oracle/fwh.py) against closed forms of linear
acoustics: a point monopole and a point dipole inside a closed sphere of
panels must give, at an outside observer, the pressure their exact fields
radiate there; the result must not depend on the surface; the ambient at
rest is silent; the discrete derivative and the retarded interpolation are
exact on the polynomials of their order; and the quadratic momentum-flux
term, which the linear fields leave out, against the closed form of a steady
uniform stream through the sphere.  The sound speed is not 1 and the source
sits off the sphere's centre, so that a dropped 1/c0, a wrong sign of the
retarded time or of r, or a missing term does not cancel."""
import numpy as np
import pytest

from oracle import fwh

RHO0, P0, C0 = 1.3, 1.0 / 1.4, 0.8
SRC = np.array([0.1, -0.05, 0.07])
SIG, TC, AMP = 0.6, 2.0, 1e-4
DTAU, NFR = 0.02, 800


def q(t):
    return AMP * np.exp(-((t - TC) / SIG) ** 2)


def qd(t):
    return -2.0 * (t - TC) / SIG ** 2 * q(t)


def qdd(t):
    return (4.0 * (t - TC) ** 2 / SIG ** 4 - 2.0 / SIG ** 2) * q(t)


def sphere(a, nth, nph):
    """UV sphere of radius a about the origin: panel centres, unit outward
    normals and exact band areas."""
    th_e = np.linspace(0.0, np.pi, nth + 1)
    th = 0.5 * (th_e[1:] + th_e[:-1])
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    n = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)]).reshape(3, -1)
    dA = (a * a * (np.cos(th_e[:-1]) - np.cos(th_e[1:])) * 2 * np.pi / nph)
    area = np.repeat(dA, nph)
    return a * n, n, area


def monopole(x, t, need_u=True):
    """Exact field of a point monopole, velocity potential -q(t - R/c)/(4 pi R)."""
    d = x - SRC[:, None]
    R = np.sqrt((d * d).sum(axis=0))
    tr = t - R / C0
    ur = qd(tr) / (4 * np.pi * C0 * R) + q(tr) / (4 * np.pi * R * R)
    p = RHO0 * qd(tr) / (4 * np.pi * R)
    return p, ur * d / R


def dipole_phi(x, t, e):
    d = x - SRC[:, None]
    R = np.sqrt((d * d).sum(axis=0))
    tr = t - R / C0
    return (e @ d / R) * (qd(tr) / (4 * np.pi * C0 * R) + q(tr) / (4 * np.pi * R * R))


def dipole(x, t, need_u=True, e=np.array([0.0, 0.6, 0.8])):
    """Exact field of a point dipole along e, velocity potential
    e . grad(monopole potential); the velocity by a 4th-order difference."""
    d = x - SRC[:, None]
    R = np.sqrt((d * d).sum(axis=0))
    tr = t - R / C0
    p = -RHO0 * (e @ d / R) * (qdd(tr) / (4 * np.pi * C0 * R) + qd(tr) / (4 * np.pi * R * R))
    if not need_u:
        return p, None
    h = 1e-4
    u = np.empty_like(x)
    for i in range(3):
        dx = np.zeros((3, 1))
        dx[i] = h
        u[i] = (-dipole_phi(x + 2 * dx, t, e) + 8 * dipole_phi(x + dx, t, e)
                - 8 * dipole_phi(x - dx, t, e) + dipole_phi(x - 2 * dx, t, e)) / (12 * h)
    return p, u


def frames_of(field, xyz, dtau=DTAU):
    nfr = int(round(NFR * DTAU / dtau))
    fr = np.empty((nfr, 5, xyz.shape[1]))
    for m in range(nfr):
        p, u = field(xyz, m * dtau)
        fr[m, 0] = RHO0 + p / C0 ** 2
        fr[m, 1:4] = u
        fr[m, 4] = P0 + p
    return fr


def observe(field, obs, a=1.0, nth=24, nph=48, t0=None, nt=120, dt=0.02, dtau=DTAU):
    xyz, nrm, area = sphere(a, nth, nph)
    D = np.sqrt((obs ** 2).sum(axis=0))
    if t0 is None:
        t0 = TC + D.min() / C0 - 1.2
    got = fwh.pressure(frames_of(field, xyz, dtau), xyz, nrm, area, dtau, RHO0, P0, C0, obs, t0, dt, nt)
    t = t0 + dt * np.arange(nt)
    ref = np.stack([field(obs[:, o:o + 1], t, need_u=False)[0] for o in range(obs.shape[1])])
    return got, ref


def rel_err(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


def test_monopole_radiates_its_exact_field():
    obs = np.array([[8.0, 0.0, 0.0], [0.0, -4.0, 6.0]]).T / 1.0
    e1 = rel_err(*observe(monopole, obs))
    e2 = rel_err(*observe(monopole, obs, nth=48, nph=96, dtau=DTAU / 2))
    assert e2 < 1e-3, (e1, e2)
    # second order in the panel size and the frame interval
    assert e2 < 0.35 * e1, (e1, e2)


@pytest.mark.parametrize("dist", [2.2, 8.0])
def test_dipole_radiates_its_exact_field_near_and_far(dist):
    # near the sphere the 1/r^2 loading term carries much of the signal
    obs = (dist * np.array([[0.0, 0.6, 0.8], [0.8, 0.0, -0.6]])).T
    got, ref = observe(dipole, obs, nth=48, nph=96, dtau=DTAU / 2)
    assert rel_err(got, ref) < 2e-3


def test_result_does_not_depend_on_the_surface():
    obs = np.array([[2.0, 3.0, 6.0]]).T
    g1, _ = observe(dipole, obs, a=1.0, nth=48, nph=96)
    g2, _ = observe(dipole, obs, a=1.5, nth=64, nph=128)
    assert np.abs(g1 - g2).max() < 2e-3 * np.abs(g1).max()


def test_ambient_at_rest_is_silent():
    xyz, nrm, area = sphere(1.0, 8, 16)
    fr = np.zeros((20, 5, xyz.shape[1]))
    fr[:, 0] = RHO0
    fr[:, 4] = P0
    out = fwh.pressure(fr, xyz, nrm, area, DTAU, RHO0, P0, C0, np.array([[5.0, 1.0, 0.0]]).T, 7.0, 0.01, 10)
    assert np.all(out == 0.0)


def test_derivative_and_retarded_interpolation_orders():
    tau = np.arange(12) * 0.3
    F = np.stack([1.0 + 2.0 * tau - 0.7 * tau ** 2, -3.0 * tau ** 2]).T   # [N][2]
    D = fwh.ddtau(F, 0.3)
    np.testing.assert_allclose(D[:, 0], 2.0 - 1.4 * tau, atol=1e-12)
    np.testing.assert_allclose(D[:, 1], -6.0 * tau, atol=1e-12)
    G = np.stack([4.0 - 2.5 * tau, tau]).T
    s = np.array([[0.0, 10.999], [3.25, 7.5]])
    np.testing.assert_allclose(fwh.retarded(G, s), np.stack([4.0 - 2.5 * 0.3 * s[:, 0], 0.3 * s[:, 1]]).T,
                               atol=1e-12)


@pytest.mark.parametrize("U", [np.array([0.3, 0.0, 0.0]), np.array([0.1, -0.2, 0.25])])
def test_quadratic_momentum_flux_of_a_steady_uniform_stream(U):
    """The quadratic source term rho u_i (u . n), which linear acoustics leaves
    out: a steady uniform stream U through a sphere of radius a (p = p0) has
    dQ/dtau = dL/dtau = 0, so 4 pi p' = sum A L_r / r^2 with L = rho U (U . n).
    By the divergence theorem and the mean-value property of the harmonic
    function (U . grad_y)^2 (1/|x - y|), the surface integral equals the
    sphere's volume times that function at the centre:
        p' = rho a^3 / 3 * (3 (U . d)^2 - |d|^2 |U|^2) / |d|^5,  d = x - centre.
    Swapping u_i for n_i in the term, dropping u . n, or a wrong power of r
    fails it; second order in the panel size."""
    a = 1.0
    obs = np.array([[2.5, 1.0, -0.7], [0.4, -2.2, 1.9]]).T
    d = obs
    R = np.sqrt((d * d).sum(axis=0))
    exact = RHO0 * a ** 3 / 3.0 * (3.0 * (U @ d) ** 2 - R ** 2 * (U @ U)) / R ** 5
    errs = []
    for nth, nph in ((24, 48), (48, 96)):
        xyz, nrm, area = sphere(a, nth, nph)
        fr = np.empty((12, 5, xyz.shape[1]))
        fr[:, 0] = RHO0
        fr[:, 1:4] = U[None, :, None]
        fr[:, 4] = P0
        got = fwh.pressure(fr, xyz, nrm, area, DTAU, RHO0, P0, C0, obs, 0.1 + R.max() / C0, DTAU, 3)
        # steady: every observer time gives the same value
        np.testing.assert_allclose(got, got[:, :1].repeat(3, axis=1), rtol=1e-13, atol=0.0)
        errs.append(np.abs(got[:, 0] - exact).max() / np.abs(exact).max())
    assert errs[1] < 2e-4, errs
    assert errs[1] < 0.35 * errs[0], errs
