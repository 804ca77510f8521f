"""GPU parity: libles.so (through its C ABI) against the FP64 oracle on the same
seeded inputs.  Tolerances: FP64 relative L2 <= 1e-12 per field after 10
steps (stage-level checks tighter); FP32 relative L2 <= 1e-5 after 100 steps.
Every case builds its oracle reference from the seeded primitives itself; no
oracle input comes from the GPU."""
import math

import numpy as np
import pytest

import oracle
from helpers import rel_l2, to_oracle
from paper_2212_12365_gb300 import inputs as I
from paper_2212_12365_gb300 import les

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()


def _oracle_state(spec, fp, prim, level=0):
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.qhat_from(g, p, m, prim, True)
    q = oracle.apply_bc(g, p, m, q, level)
    return g, p, m, q


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {
    "wavy_periodic": lambda: (I.wavy_periodic_grid((13, 11, 9), amp=0.2), I.FlowParams(Re=300.0)),
    "wavy_box_ff_exit": lambda: (I.wavy_box_grid((14, 11, 9), amp=0.06,
                                                  bc=(1, 3, 1, 1, 1, 1)), I.FlowParams(Re=500.0)),
    "jet_ragged": lambda: (I.jet_grid(37, 23, 19, 8.0, 6.0, 6.0, 0.15, 0.18), I.FlowParams(Re=1e4)),
    "mixed_periodic_z": lambda: (_mixed_periodic(), I.FlowParams(Re=2e3)),
    "tiny_4x4x4": lambda: (I.wavy_box_grid((4, 4, 4), amp=0.02), I.FlowParams(Re=100.0)),
}


def _mixed_periodic():
    g = I.jet_grid(21, 17, 12, 6.0, 5.0, 4.0, 0.2, 4.0 / 11)
    nk = 12
    z1 = np.arange(nk) * (4.0 / nk)
    ni, nj, _ = g.dims
    g.z = np.repeat(z1, ni * nj)
    g.periodic = (0, 0, 1)
    g.shift = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 4.0]], dtype=float)
    g.bc = (2, 3, 1, 1, 0, 0)
    return g


def _prims(spec, seed):
    s = I.smooth_random_primitives(spec, seed, amp=0.08)
    return s


@pytest.mark.parametrize("case", sorted(CASES))
def test_metrics_parity_fp64(case):
    spec, fp = CASES[case]()
    g, _ = to_oracle(spec, fp)
    m_or = oracle.metrics(g)
    s = les.Solver(spec, fp, les.LES_FP64)
    m_gpu = s.field(les.LES_FIELD_METRICS)
    for t in range(10):
        assert _rel_max(m_gpu[t], m_or[t]) < 1e-13 or np.abs(m_gpu[t] - m_or[t]).max() < 1e-14, t
    s.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_set_state_bc_and_rhs_parity_fp64(case):
    spec, fp = CASES[case]()
    prim = _prims(spec, 5)
    g, p, m, q = _oracle_state(spec, fp, prim)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim, les.LES_STATE_PRIMITIVE)
    raw = s.get_state(les.LES_STATE_RAW)
    assert _rel_max(raw, q) < 1e-14
    r_gpu = s.rhs()
    r_or = oracle.rhs(g, p, m, q)
    for f in range(5):
        scale = max(np.abs(r_or[f]).max(), 1e-3 * np.abs(r_or).max())
        assert np.abs(r_gpu[f] - r_or[f]).max() <= 1e-12 * scale, (f, np.abs(r_gpu[f] - r_or[f]).max(), scale)
    # time step
    _, dt = s.time()
    assert dt == pytest.approx(oracle.dt_cfl(g, p, m, q), rel=1e-13)
    # point fields
    mus = s.field(les.LES_FIELD_MU_SGS)
    mus_or = oracle.point_field(g, p, m, q, oracle.FIELD_MU_SGS)
    assert np.abs(mus - mus_or).max() <= 1e-12 * max(np.abs(mus_or).max(), 1e-30)
    for k, f_or in ((les.LES_FIELD_LAMBDA_XI, 4), (les.LES_FIELD_LAMBDA_ETA, 5), (les.LES_FIELD_LAMBDA_ZETA, 6)):
        a, b = s.field(k), oracle.point_field(g, p, m, q, f_or)
        assert _rel_max(a, b) < 1e-13
    s.close()


def test_jet_small_10_steps_fp64():
    """48x32x32 jet, M 1.4, TR 1, Re_D 1e5, 10 steps at CFL 0.5: relative L2
    per field <= 1e-12 against the oracle."""
    spec, fp = I.jet_small()
    prim = I.ambient_primitives(spec.N, fp.TR)
    g, p, m, q = _oracle_state(spec, fp, prim)
    dt = oracle.dt_cfl(g, p, m, q)
    q10 = oracle.step(g, p, m, q, 10, 0, dt)
    ref = oracle.state_out(g, p, m, q10, False)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim, les.LES_STATE_PRIMITIVE)
    assert s.time()[1] == pytest.approx(dt, rel=1e-14)
    s.step(10)
    out = s.get_state(les.LES_STATE_CONSERVED)
    err = rel_l2(out, ref)
    print("jet_small fp64 rel L2 per field:", err)
    assert np.all(err <= 1e-12), err
    # diagnostics of the final state
    d = s.diagnostics()
    dor = oracle.diag(g, p, m, q10)
    assert d["max_abs_rhs_rho"] == pytest.approx(dor["max_abs_rhs_rho"], rel=1e-10)
    np.testing.assert_allclose(d["l2_rhs"], dor["l2_rhs"], rtol=1e-10)
    # sums of mostly cancelling terms: compare against the sum of magnitudes
    mag = np.abs(q10).sum(axis=1)
    assert np.all(np.abs(d["sum_qhat"] - dor["sum_qhat"]) <= 1e-13 * mag)
    s.close()


def test_jet_small_100_steps_fp32():
    """FP32 storage and stencil arithmetic: relative L2 per field <= 1e-5 after
    100 steps against the FP64 oracle (error reported per field)."""
    spec, fp = I.jet_small()
    prim = I.ambient_primitives(spec.N, fp.TR)
    g, p, m, q = _oracle_state(spec, fp, prim)
    dt = oracle.dt_cfl(g, p, m, q)
    q100 = oracle.step(g, p, m, q, 100, 0, dt)
    ref = oracle.state_out(g, p, m, q100, False)
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(prim, les.LES_STATE_PRIMITIVE)
    s.step(100)
    out = s.get_state(les.LES_STATE_CONSERVED)
    err = rel_l2(out, ref)
    print("jet_small fp32 rel L2 per field after 100 steps:", err)
    assert np.all(err <= 1e-5), err
    s.close()


@pytest.mark.parametrize("prec,tol", [(les.LES_FP64, 1e-12), (les.LES_FP32, 2e-5)])
def test_multistep_ragged_cases(prec, tol):
    for name in ("wavy_box_ff_exit", "jet_ragged", "mixed_periodic_z"):
        spec, fp = CASES[name]()
        prim = _prims(spec, 9)
        g, p, m, q = _oracle_state(spec, fp, prim)
        dt = 0.5 * oracle.dt_cfl(g, p, m, q)
        fp.dt = dt
        p.cfl = fp.cfl
        q5 = oracle.step(g, p, m, q, 5, 0, dt)
        s = les.Solver(spec, fp, prec)
        s.set_state(prim, les.LES_STATE_PRIMITIVE)
        s.step(5)
        err = rel_l2(s.get_state(les.LES_STATE_CONSERVED), oracle.state_out(g, p, m, q5, False))
        assert np.all(err <= tol), (name, err)
        s.close()


def test_conservation_periodic_fp64():
    spec = I.wavy_periodic_grid((16, 12, 10), amp=0.2)
    fp = I.FlowParams(Re=200.0)
    prim = _prims(spec, 3)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim, les.LES_STATE_PRIMITIVE)
    q0 = s.get_state(les.LES_STATE_RAW)
    s.step(100)
    q1 = s.get_state(les.LES_STATE_RAW)
    scale = np.abs(q0).sum(axis=1)
    drift = np.abs(q1.sum(axis=1) - q0.sum(axis=1)) / scale
    assert np.all(drift <= 1e-13), drift
    assert np.abs(q1 - q0).max() > 1e-3
    s.close()


def test_bit_reproducible_and_resume():
    """Two runs are bit-identical; a RAW checkpoint at step 4 resumed in a new
    handle gives the same bits at step 9 (noise counter = time level)."""
    spec, fp = I.jet_small()
    prim = I.ambient_primitives(spec.N, fp.TR)
    outs = []
    for _ in range(2):
        s = les.Solver(spec, fp, les.LES_FP64)
        s.set_state(prim)
        s.step(9)
        outs.append(s.get_state(les.LES_STATE_RAW))
        s.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim)
    s.step(4)
    ck = s.get_state(les.LES_STATE_RAW)
    step, dt = s.time()
    s.close()
    s2 = les.Solver(spec, fp, les.LES_FP64)
    s2.set_time(step, dt)
    s2.set_state(ck, les.LES_STATE_RAW)
    s2.step(5)
    np.testing.assert_array_equal(s2.get_state(les.LES_STATE_RAW), outs[0])
    s2.close()


def test_workspace_mode_matches():
    import torch
    spec, fp = CASES["jet_ragged"]()
    prim = _prims(spec, 2)
    nb = les.les_workspace_bytes(spec, les.LES_FP64)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    a = les.Solver(spec, fp, les.LES_FP64, workspace=ws)
    b = les.Solver(spec, fp, les.LES_FP64)
    for s in (a, b):
        s.set_state(prim)
        s.step(3)
    np.testing.assert_array_equal(a.get_state(les.LES_STATE_RAW), b.get_state(les.LES_STATE_RAW))
    a.close()
    b.close()


def test_probe_parity():
    """Probe frames (levels 2 and 4) against the oracle's trilinear probe of its
    own state at level 4."""
    import torch
    spec, fp = I.jet_small()
    prim = _prims(spec, 4)
    g, p, m, q = _oracle_state(spec, fp, prim)
    dt = oracle.dt_cfl(g, p, m, q)
    q4 = oracle.step(g, p, m, q, 4, 0, dt)
    xyz = I.cylinder_points(3.0, 16, 12, 1.0, 18.0)
    ref = oracle.probe(g, p, m, q4, xyz)
    for prec, dtype, tol in ((les.LES_FP64, torch.float64, 1e-12), (les.LES_FP32, torch.float32, 2e-5)):
        s = les.Solver(spec, fp, prec)
        s.set_state(prim)
        cap = 3
        buf = torch.zeros((cap, 5, xyz.shape[1]), dtype=dtype, device="cuda")
        les.les_probe_surface(s.h, xyz, 2, buf.data_ptr(), cap)
        s.step(4)
        assert les.les_probe_frames(s.h) == 2
        torch.cuda.synchronize()
        got = buf[1].double().cpu().numpy()
        for f in range(5):
            assert np.abs(got[f] - ref[f]).max() <= tol * max(np.abs(ref[f]).max(), 1e-3), (prec, f)
        s.close()


def test_invalid_arguments_rejected():
    spec, fp = CASES["jet_ragged"]()
    bad = I.FlowParams(mach_j=0.0)  # an inflow face with no jet velocity
    with pytest.raises(les.LesError) as e:
        les.Solver(spec, bad, les.LES_FP64)
    assert e.value.code == les.LES_ERR_ARG
    s = les.Solver(spec, fp, les.LES_FP64)
    with pytest.raises(les.LesError) as e:
        s.step(1)  # no state yet
    assert e.value.code == les.LES_ERR_STATE
    s.close()


def test_nonfinite_detected():
    spec, fp = CASES["wavy_periodic"]()
    prim = _prims(spec, 1)
    prim[4, 17] = np.nan
    fp.dt = 0.01
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim)
    d = s.diagnostics(check=False)
    assert d["rc"] == les.LES_ERR_NONFINITE and d["nonfinite"] > 0
    s.close()
