"""Subsonic jet entrance (Sec. "Entrance Boundary", reading R18) on the GPU
against the oracle: the boundary state and residual at set-up, FP64 steps to
1e-12, FP32 steps to 1e-5, and a batch mixing subsonic and supersonic jets
bit-identical to single-jet runs."""
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


def _case(M=0.8):
    spec = I.jet_grid(37, 23, 19, 8.0, 6.0, 6.0, 0.15, 0.18)
    fp = I.FlowParams(mach_j=M, Re=1e4, seed=5)
    prim = I.smooth_random_primitives(spec, 29, amp=0.06)
    return spec, fp, prim


def test_subsonic_entrance_state_rhs_and_steps_fp64():
    spec, fp, prim = _case()
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim)
    raw = s.get_state(les.LES_STATE_RAW)
    assert np.abs(raw - q).max() <= 1e-14 * np.abs(q).max()
    r_or = oracle.rhs(g, p, m, q)
    r = s.rhs()
    scale = np.abs(r_or).max(axis=1, keepdims=True)
    assert (np.abs(r - r_or) / scale).max() <= 1e-12
    _, dt = s.time()
    assert dt == pytest.approx(oracle.dt_cfl(g, p, m, q), rel=1e-13)
    s.step(10)
    out = s.get_state(les.LES_STATE_CONSERVED)
    s.close()
    ref = oracle.state_out(g, p, m, oracle.step(g, p, m, q, 10, 0, dt), False)
    err = rel_l2(out, ref)
    print("subsonic jet fp64 10 steps rel L2 per field:", err)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("prec", [les.LES_FP32, les.LES_FP32_SEPARABLE])
def test_subsonic_jet_fp32_100_steps(prec):
    spec, fp = I.jet_small()
    fp.mach_j = 0.9
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    prim = I.ambient_primitives(spec.N, fp.TR)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    dt = oracle.dt_cfl(g, p, m, q)
    ref = oracle.state_out(g, p, m, oracle.step(g, p, m, q, 100, 0, dt), False)
    s = les.Solver(spec, fp, prec)
    s.set_state(prim)
    s.step(100)
    out = s.get_state(les.LES_STATE_CONSERVED)
    s.close()
    err = rel_l2(out, ref)
    print("subsonic jet fp32 (form", prec, ") 100 steps rel L2 per field:", err)
    assert np.all(err <= 1e-5), err


@pytest.mark.parametrize("prec", [les.LES_FP64, les.LES_FP32])
def test_batch_mixing_subsonic_and_supersonic_jets_bit_identical(prec):
    jets = I.batch_jets(4, seed=21)
    for (g, f), M in zip(jets, (0.6, 1.5, 0.95, 1.2)):
        f.mach_j = M
    b = les.Solver([g for g, _ in jets], [f for _, f in jets], prec)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.smooth_random_primitives(g, 50 + j, amp=0.05), jet=j)
    b.step(4)
    for j, (g, f) in enumerate(jets):
        s = les.Solver(g, f, prec)
        s.set_state(I.smooth_random_primitives(g, 50 + j, amp=0.05))
        s.step(4)
        np.testing.assert_array_equal(b.get_state(les.LES_STATE_RAW, jet=j), s.get_state(les.LES_STATE_RAW))
        s.close()
    b.close()
