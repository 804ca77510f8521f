"""Oracle pins for the boundary conditions (Sec. "Boundary Conditions") and
the inflow noise generator.  Far field: the Riemann invariants carried along
the incoming/outgoing characteristics, entropy and tangential velocity are
the properties the condition is built to impose; exit: pressure from outside,
temperature/velocity from inside; inflow: tanh profile of momentum thickness
theta, linear total enthalpy (Crocco-Busemann), bounded uniform noise."""
import math
import os

import numpy as np
import pytest

import oracle
from helpers import to_oracle
from paper_2212_12365_gb300 import inputs as I

GAMMA = 1.4


def _prim(Q):
    rho = Q[0]
    u = Q[1:4] / rho
    p = (GAMMA - 1) * (Q[4] - 0.5 * rho * (u @ u))
    return rho, u, p


def _cons(rho, u, p):
    u = np.asarray(u, dtype=np.float64)
    return np.array([rho, *(rho * u), p / (GAMMA - 1) + 0.5 * rho * (u @ u)])


def _params(TR=1.0):
    return to_oracle(I.periodic_box_grid((4, 4, 4)), I.FlowParams(TR=TR))[1]


@pytest.mark.parametrize("TR", [1.0, 2.3])
def test_farfield_characteristic_properties(TR):
    """Random interior states and outward normals: subsonic exit keeps R+ of
    the interior, R- of the freestream, interior entropy and tangential
    velocity; subsonic entrance takes entropy and tangential velocity from the
    freestream; supersonic exit copies the interior; supersonic entrance
    imposes the freestream."""
    P = _params(TR)
    rng = np.random.default_rng(11)
    rho_inf, p_inf = TR, 1 / GAMMA
    c_inf = math.sqrt(GAMMA * p_inf / rho_inf)
    seen = set()
    for _ in range(400):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        rho = rng.uniform(0.5, 2.0)
        p = rng.uniform(0.4, 1.2)
        c = math.sqrt(GAMMA * p / rho)
        Mn = rng.uniform(-1.8, 1.8)
        t = rng.normal(size=3)
        t -= (t @ n) * n
        u = Mn * c * n + 0.3 * t
        Qe = _cons(rho, u, p)
        Qf = oracle.face_state(P, "farfield", Qe, n)
        rf, uf, pf = _prim(Qf)
        cf = math.sqrt(GAMMA * pf / rf)
        qne, qnf = u @ n, uf @ n
        Rp_e, Rp_f = qne + 2 * c / (GAMMA - 1), qnf + 2 * cf / (GAMMA - 1)
        Rm_inf, Rm_f = 0.0 - 2 * c_inf / (GAMMA - 1), qnf - 2 * cf / (GAMMA - 1)
        if Mn >= 1:
            seen.add("sup-exit")
            np.testing.assert_array_equal(Qf, Qe)
        elif Mn <= -1:
            seen.add("sup-entry")
            np.testing.assert_allclose(Qf, _cons(rho_inf, [0, 0, 0], p_inf), rtol=1e-15)
        else:
            assert Rp_f == pytest.approx(Rp_e, rel=1e-12, abs=1e-12)
            assert Rm_f == pytest.approx(Rm_inf, rel=1e-12, abs=1e-12)
            tang_f = uf - qnf * n
            if Mn >= 0:
                seen.add("sub-exit")
                assert pf / rf**GAMMA == pytest.approx(p / rho**GAMMA, rel=1e-12)
                np.testing.assert_allclose(tang_f, u - qne * n, atol=1e-12)
            else:
                seen.add("sub-entry")
                assert pf / rf**GAMMA == pytest.approx(p_inf / rho_inf**GAMMA, rel=1e-12)
                np.testing.assert_allclose(tang_f, 0.0, atol=1e-12)
    assert seen == {"sup-exit", "sup-entry", "sub-exit", "sub-entry"}


def test_farfield_preserves_ambient():
    P = _params(1.7)
    Qa = _cons(1.7, [0, 0, 0], 1 / GAMMA)
    for n in (np.array([1.0, 0, 0]), np.array([0, -0.6, 0.8])):
        np.testing.assert_allclose(oracle.face_state(P, "farfield", Qa, n), Qa, rtol=1e-14,
                                   atol=1e-15)


def test_exit_condition_properties():
    """Subsonic exit: p = p_inf, internal energy (temperature) and velocity of
    the interior point; supersonic exit copies the interior."""
    P = _params(1.0)
    rng = np.random.default_rng(5)
    n = np.array([1.0, 0.0, 0.0])
    for _ in range(100):
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.4, 1.2)
        c = math.sqrt(GAMMA * p / rho)
        u = np.array([rng.uniform(-0.5, 2.0) * c, rng.normal() * 0.2, rng.normal() * 0.2])
        Qe = _cons(rho, u, p)
        Qf = oracle.face_state(P, "exit", Qe, n)
        rf, uf, pf = _prim(Qf)
        if u[0] / c >= 1:
            np.testing.assert_array_equal(Qf, Qe)
        else:
            assert pf == pytest.approx(1 / GAMMA, rel=1e-12)
            assert pf / rf == pytest.approx(p / rho, rel=1e-12)  # same T
            np.testing.assert_allclose(uf, u, rtol=1e-12, atol=1e-15)


def test_inflow_profile_momentum_thickness():
    """u~(r) = [1 + tanh((0.5 - r)/(2 theta))]/2: half velocity at r = D/2 and
    momentum thickness int u~(1 - u~) dr = theta."""
    fp = I.FlowParams(theta=0.05)
    _, P = to_oracle(I.periodic_box_grid((4, 4, 4)), fp)
    assert oracle.inflow_profile(P, 0.5) == pytest.approx(0.5, abs=1e-15)
    r = np.linspace(0.0, 3.0, 30001)
    u = np.array([oracle.inflow_profile(P, x) for x in r])
    f = u * (1 - u)
    mt = ((f[1:] + f[:-1]) * 0.5 * np.diff(r)).sum()
    assert mt == pytest.approx(0.05, rel=1e-3)


def _jet_face():
    spec, fp = I.jet_small()
    g, P = to_oracle(spec, fp)
    m = oracle.metrics(g)
    prim = I.ambient_primitives(g.N, fp.TR)
    q = oracle.qhat_from(g, P, m, prim, True)
    return spec, fp, g, P, m, q


def test_inflow_face_jet_state_and_noise():
    """Time level 0: the profile without noise, linear total enthalpy in u~
    (Crocco-Busemann), uniform pressure 1/gamma; outside u~ >= 0.01 the
    ambient is kept by the far-field condition.  Level n >= 1: velocity noise
    uniform in +-A M_j, zero-mean, different for each level, reproducible."""
    spec, fp, g, P, m, q = _jet_face()
    ni, nj, nk = spec.dims
    face = np.arange(g.N) % ni == 0
    q0 = oracle.apply_bc(g, P, m, q, 0)
    out = oracle.state_out(g, P, m, q0, True)
    rho, u, v, w, p = (o[face] for o in out)
    r = np.hypot(spec.y[face], spec.z[face])
    ut = np.array([oracle.inflow_profile(P, x) for x in r])
    jet = ut >= 0.01
    assert jet.sum() > 20 and (~jet).sum() > 20
    M = fp.mach_j
    np.testing.assert_allclose(u[jet], M * ut[jet], rtol=1e-14)
    np.testing.assert_allclose(p[jet], 1 / GAMMA, rtol=1e-14)
    T = GAMMA * p / rho
    h0 = T / (GAMMA - 1) + 0.5 * u**2
    h0_inf = (1 / fp.TR) / (GAMMA - 1)
    h0_jet = 1 / (GAMMA - 1) + 0.5 * M**2
    np.testing.assert_allclose(h0[jet], h0_inf + (h0_jet - h0_inf) * ut[jet], rtol=1e-13)
    amb = I.ambient_primitives(1, fp.TR)[:, 0]
    for f, o in enumerate((rho, u, v, w, p)):
        np.testing.assert_allclose(o[~jet], amb[f], atol=1e-14)
    # noise at levels 1, 2
    q1 = oracle.apply_bc(g, P, m, q, 1)
    q2 = oracle.apply_bc(g, P, m, q, 2)
    o1 = oracle.state_out(g, P, m, q1, True)
    o2 = oracle.state_out(g, P, m, q2, True)
    A = fp.noise_amp * M
    d1 = np.stack([o1[1][face][jet] - M * ut[jet], o1[2][face][jet], o1[3][face][jet]])
    d2 = np.stack([o2[1][face][jet] - M * ut[jet], o2[2][face][jet], o2[3][face][jet]])
    assert np.abs(d1).max() <= A * (1 + 1e-9)
    assert abs(d1.mean()) < 0.2 * A
    assert d1.std() == pytest.approx(A / math.sqrt(3), rel=0.2)
    assert np.abs(d1 - d2).max() > 0.1 * A
    np.testing.assert_array_equal(q1, oracle.apply_bc(g, P, m, q, 1))


def test_subsonic_entrance_isentropic_jet_state():
    """Subsonic jet entrance (Sec. "Entrance Boundary", reading R18) on the
    inflow face of a Mach 0.8 jet whose interior carries a transverse flow:
    - u is the profile M_j u~ at level 0, and at level n its deviation from
      the profile, over A = noise_amp M_j, is the u noise of the supersonic
      rule at the same level (same seed and counter);
    - v, w are those of the adjacent interior point;
    - every jet point is on the jet's isentrope, p / rho^gamma = 1/gamma
      (total conditions of the jet, an isentropic expansion);
    - in the undisturbed core (v = w = 0, u~ = 1, no noise) the state is the
      jet design state rho = 1, T = 1, p = 1/gamma, u = M_j — the point where
      the subsonic and the supersonic rules must agree."""
    spec, _ = I.jet_small()
    ni = spec.dims[0]
    face = np.arange(spec.N) % ni == 0
    r = np.hypot(spec.y[face], spec.z[face])
    states = {}
    for M in (0.8, 1.4):
        fp = I.FlowParams(mach_j=M, seed=9)
        g, P = to_oracle(spec, fp)
        m = oracle.metrics(g)
        prim = I.ambient_primitives(g.N, fp.TR)
        # a transverse flow in the interior next to the face
        inner = np.arange(g.N) % ni == 1
        prim[2][inner] = 0.05 * np.sin(3.0 * spec.y[inner])
        prim[3][inner] = -0.03 * np.cos(2.0 * spec.z[inner])
        q = oracle.qhat_from(g, P, m, prim, True)
        states[M] = (fp, P, [oracle.state_out(g, P, m, oracle.apply_bc(g, P, m, q, lv), True) for lv in (0, 3)],
                     prim)
    fp, P, (o0, o3), prim = states[0.8]
    M = 0.8
    ut = np.array([oracle.inflow_profile(P, x) for x in r])
    jet = ut >= 0.01
    assert jet.sum() > 20 and (~jet).sum() > 20
    rho, u, v, w, p = (o[face] for o in o0)
    np.testing.assert_allclose(u[jet], M * ut[jet], rtol=1e-14)  # rho u / rho: a few ulp
    inner = np.roll(face, 1)  # the i = 1 point of each face point
    np.testing.assert_allclose(v[jet], prim[2][inner][jet], rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(w[jet], prim[3][inner][jet], rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(p[jet] / rho[jet] ** GAMMA, 1 / GAMMA, rtol=1e-13)
    core = jet & (ut > 1 - 1e-12) & (np.abs(v) < 1e-300) & (np.abs(w) < 1e-300)
    if core.any():
        np.testing.assert_allclose(rho[core], 1.0, rtol=1e-14)
        np.testing.assert_allclose(p[core], 1 / GAMMA, rtol=1e-14)
    # the u noise of level 3 is the supersonic rule's, scaled by M_j
    u3 = o3[1][face]
    _, Ps, (_, s3), _ = states[1.4]
    us3 = s3[1][face]
    noise_sub = (u3[jet] - M * ut[jet]) / (fp.noise_amp * M)
    noise_sup = (us3[jet] - 1.4 * ut[jet]) / (fp.noise_amp * 1.4)
    np.testing.assert_allclose(noise_sub, noise_sup, rtol=0, atol=1e-9)
    assert np.abs(noise_sub).max() > 0.5


def test_subsonic_entrance_core_matches_design_state():
    """A flat core (u~ = 1 to rounding) with no transverse flow: the subsonic
    rule gives exactly the jet state of the supersonic rule at TR = 1
    (rho = T = 1, p = 1/gamma, u = M_j) for any M_j < 1."""
    spec, _ = I.jet_small()
    ni = spec.dims[0]
    face = np.arange(spec.N) % ni == 0
    r = np.hypot(spec.y[face], spec.z[face])
    for M in (0.3, 0.9, 0.999):
        fp = I.FlowParams(mach_j=M, theta=0.01)
        g, P = to_oracle(spec, fp)
        m = oracle.metrics(g)
        q = oracle.qhat_from(g, P, m, I.ambient_primitives(g.N, fp.TR), True)
        out = oracle.state_out(g, P, m, oracle.apply_bc(g, P, m, q, 0), True)
        c = r < 0.2
        assert c.sum() >= 4
        np.testing.assert_allclose(out[0][face][c], 1.0, rtol=1e-13)
        np.testing.assert_allclose(out[1][face][c], M, rtol=1e-13)
        np.testing.assert_allclose(out[4][face][c], 1 / GAMMA, rtol=1e-13)


def test_splitmix64_reference_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_reference.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for seed, n, out in rows:
        assert oracle.splitmix64(int(seed), int(n)) == int(out)


def test_boundary_conditions_keep_ambient_box():
    """An ambient state at rest is a fixed point of every face condition
    (far field on all lateral faces, exit at x max, far-field part of the
    inflow plane away from the jet), with the faces applied y, z, x."""
    spec = I.wavy_box_grid((10, 9, 8), amp=0.06, bc=(I.BC_FARFIELD, I.BC_EXIT) + (I.BC_FARFIELD,) * 4)
    g, P = to_oracle(spec, I.FlowParams(TR=1.6))
    m = oracle.metrics(g)
    q = oracle.qhat_from(g, P, m, I.ambient_primitives(g.N, 1.6), True)
    q1 = oracle.apply_bc(g, P, m, q, 3)
    np.testing.assert_allclose(q1, q, rtol=1e-13, atol=1e-15)


def test_farfield_zero_normal_velocity_takes_the_exit_branch():
    """Reading R14: the paper's subsonic ranges leave q_n = 0 open; a normal
    Mach number within 1e-8 of zero takes the exit side (entropy and
    tangential velocity from inside), one beyond it the entrance side."""
    P = _params(1.0)
    n = np.array([-1.0, 0.0, 0.0])
    c = math.sqrt(GAMMA * (1 / GAMMA) / 1.0)
    for Mn, exit_side in ((0.0, True), (-5e-9, True), (5e-9, True), (-3e-8, False)):
        u = np.array([-Mn * c, 0.02, -0.01])  # q_n = u . n = Mn c
        rho, p = 1.1, 1 / GAMMA * 1.05
        Qf = oracle.face_state(P, "farfield", _cons(rho, u, p), n)
        rf, uf, pf = _prim(Qf)
        tang = uf - (uf @ n) * n
        if exit_side:
            np.testing.assert_allclose(tang, u - (u @ n) * n, atol=1e-15)
            assert pf / rf**GAMMA == pytest.approx(p / rho**GAMMA, rel=1e-12)
        else:
            np.testing.assert_allclose(tang, 0.0, atol=1e-15)
