"""The paper's polar jet mesh (Sec. "Mesh Generation") with the centerline
condition (Sec. "Centerline Boundary Condition") on the GPU, through the C
ABI, against the FP64 oracle: residual and multi-step parity in FP64 and FP32,
batched with a Cartesian jet (bit-identical to single-jet runs), and the
argument checks of the centerline face."""
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


def _polar(dims=(40, 18, 24)):
    return I.polar_jet_grid(*dims, 10.0, 4.0), I.FlowParams(mach_j=1.4, TR=1.2, Re=2e4, seed=7)


def _oracle_state(spec, fp, prim):
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    return g, p, m, q


@pytest.mark.parametrize("prec,tol", [(les.LES_FP64, 1e-12), (les.LES_FP32, 2e-5)])
def test_polar_residual_parity(prec, tol):
    spec, fp = _polar((37, 15, 20))
    prim = I.smooth_random_primitives(spec, 21, amp=0.06)
    g, p, m, q = _oracle_state(spec, fp, prim)
    r_or = oracle.rhs(g, p, m, q)
    s = les.Solver(spec, fp, prec)
    s.set_state(prim)
    s.step(0)
    r = s.rhs()
    s.close()
    scale = np.abs(r_or).max(axis=1, keepdims=True) + 1e-30
    err = np.abs(r - r_or) / scale
    print("polar residual error / scale:", err.max(axis=1))
    assert err.max() < tol, err.max(axis=1)


def test_polar_jet_10_steps_fp64():
    spec, fp = _polar()
    prim = I.ambient_primitives(spec.N, fp.TR)
    g, p, m, q = _oracle_state(spec, fp, prim)
    dt = oracle.dt_cfl(g, p, m, q)
    ref = oracle.state_out(g, p, m, oracle.step(g, p, m, q, 10, 0, dt), False)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim)
    assert s.time()[1] == pytest.approx(dt, rel=1e-14)
    s.step(10)
    out = s.get_state(les.LES_STATE_CONSERVED)
    s.close()
    err = rel_l2(out, ref)
    print("polar jet fp64 10 steps rel L2 per field:", err)
    assert np.all(err <= 1e-12), err
    ni, nj, nk = spec.dims
    axis = out.reshape(5, nk, nj, ni)[:, :, 0, 1:-1]
    assert np.abs(axis - axis[:, :1]).max() == 0.0  # one state per axial station


def test_polar_jet_100_steps_fp32():
    spec, fp = _polar()
    prim = I.ambient_primitives(spec.N, fp.TR)
    g, p, m, q = _oracle_state(spec, fp, prim)
    dt = oracle.dt_cfl(g, p, m, q)
    ref = oracle.state_out(g, p, m, oracle.step(g, p, m, q, 100, 0, dt), False)
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(prim)
    s.step(100)
    err = rel_l2(s.get_state(les.LES_STATE_CONSERVED), ref)
    s.close()
    print("polar jet fp32 100 steps rel L2 per field:", err)
    assert np.all(err <= 1e-5), err


@pytest.mark.parametrize("prec", [les.LES_FP64, les.LES_FP32])
def test_polar_and_cartesian_batch_bit_identical(prec):
    jets = [_polar((30, 14, 16)), (I.jet_grid(33, 21, 19, 8.0, 6.0, 6.0, 0.15, 0.18), I.FlowParams(seed=3))]
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    b = les.Solver(specs, fps, prec)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.ambient_primitives(g.N, f.TR), jet=j)
    b.step(3)
    for j, (g, f) in enumerate(jets):
        s = les.Solver(g, f, prec)
        s.set_state(I.ambient_primitives(g.N, f.TR))
        s.step(3)
        np.testing.assert_array_equal(b.get_state(les.LES_STATE_RAW, jet=j), s.get_state(les.LES_STATE_RAW))
        s.close()
    b.close()


def test_centerline_face_checks():
    spec, fp = _polar((12, 8, 8))
    bad = I.polar_jet_grid(12, 8, 8, 10.0, 4.0)
    bad.bc = (2, 3, 1, 4, 0, 0)  # centerline on the j+ face
    with pytest.raises(les.LesError) as e:
        les.Solver(bad, fp, les.LES_FP64)
    assert "j- face" in str(e.value)
    bad = I.polar_jet_grid(12, 8, 8, 10.0, 4.0)
    bad.bc = (2, 3, 1, 1, 0, 0)  # axis without the centerline condition: J^-1 = 0 rejected
    with pytest.raises(les.LesError) as e:
        les.Solver(bad, fp, les.LES_FP64)
    assert "volume" in str(e.value)
