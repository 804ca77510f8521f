"""Separable-metric FP32 stage (LES_FP32_SEPARABLE) on Cartesian-product grids.

On a grid x = x(i), y = y(j), z = z(k) the cofactor matrix is diagonal and
made of products of the three 1-D spacings; the separable kernel evaluates
the same method from those 1-D tables.  It is checked like the general FP32
form against the FP64 oracle (which uses the general metrics), against the
general FP32 form, in the batched form (bit-identical to single jets), and
it must reject a grid that is not a product.
"""
import numpy as np
import pytest

import oracle
from helpers import rel_l2, to_oracle
from paper_2212_12365_gb300 import inputs as I
from paper_2212_12365_gb300 import les

pytestmark = pytest.mark.gpu
SEP = les.LES_FP32_SEPARABLE


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()


def _mixed():
    g = I.jet_grid(45, 33, 12, 6.0, 5.0, 4.0, 0.2, 4.0 / 11)
    ni, nj, _ = g.dims
    g.z = np.repeat(np.arange(12) * (4.0 / 12), ni * nj)
    g.periodic = (0, 0, 1)
    g.shift = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 4.0]], dtype=float)
    g.bc = (2, 3, 1, 1, 0, 0)
    return g


def _stretched_periodic():
    x1 = np.cumsum(np.linspace(0.8, 1.2, 37)) * 0.1
    y1 = np.cumsum(np.linspace(1.1, 0.9, 19)) * 0.1
    z1 = np.arange(10) * 0.11
    g = I.product_grid(x1 - x1[0], y1 - y1[0], z1)
    g.periodic = (1, 1, 1)
    g.shift = np.diag([x1[-1] - x1[0] + 0.12, y1[-1] - y1[0] + 0.09, 1.1])
    g.bc = (0, 0, 0, 0, 0, 0)
    return g


CASES = {
    "jet_ragged_70x37x29": lambda: I.jet_grid(70, 37, 29, 8.0, 6.0, 6.0, 0.15, 0.18),
    "mixed_periodic_z": _mixed,
    "stretched_periodic_37x19x10": _stretched_periodic,
    "tiny_jet_4x4x4": lambda: I.jet_grid(4, 4, 4, 2.0, 2.0, 2.0, 0.5, 0.5),
    "tiny_periodic_4x5x4": lambda: I.periodic_box_grid((4, 5, 4), (0.3, 0.25, 0.3)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_separable_residual_parity(case):
    spec = CASES[case]()
    fp = I.FlowParams(Re=800.0)
    prim = I.smooth_random_primitives(spec, 17, amp=0.08)
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    r_or = oracle.rhs(g, p, m, q)
    s = les.Solver(spec, fp, SEP)
    s.set_state(prim)
    s.step(0)
    assert "separable" in les.les_describe(s.h)
    r = s.rhs()
    s.close()
    scale = np.abs(r_or).max(axis=1, keepdims=True) + 1e-30
    err = np.abs(r - r_or) / scale
    assert err.max() < 2e-5, (case, err.max(axis=1))


def test_separable_jet_small_100_steps():
    """Same bar as the general FP32 form: relative L2 per field <= 1e-5 after
    100 steps against the FP64 oracle."""
    spec, fp = I.jet_small()
    prim = I.ambient_primitives(spec.N, fp.TR)
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    dt = oracle.dt_cfl(g, p, m, q)
    ref = oracle.state_out(g, p, m, oracle.step(g, p, m, q, 100, 0, dt), False)
    s = les.Solver(spec, fp, SEP)
    s.set_state(prim)
    s.step(100)
    err = rel_l2(s.get_state(les.LES_STATE_CONSERVED), ref)
    s.close()
    print("jet_small separable fp32 rel L2 per field after 100 steps:", err)
    assert np.all(err <= 1e-5), err


def test_separable_matches_general_fp32():
    spec = I.jet_grid(70, 37, 29, 8.0, 6.0, 6.0, 0.15, 0.18)
    fp = I.FlowParams(Re=2e3)
    prim = I.smooth_random_primitives(spec, 5, amp=0.08)
    out = []
    for prec in (les.LES_FP32, SEP):
        s = les.Solver(spec, fp, prec)
        s.set_state(prim)
        s.step(10)
        out.append(s.get_state(les.LES_STATE_CONSERVED))
        s.close()
    err = rel_l2(out[1], out[0])
    print("separable vs general fp32 after 10 steps:", err)
    assert np.all(err <= 5e-6), err


def test_separable_batched_bit_identical_to_single():
    jets = I.batch_jets(5, seed=4)
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    b = les.Solver(specs, fps, SEP)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.ambient_primitives(g.N, f.TR), jet=j)
    b.step(4)
    for j, (g, f) in enumerate(jets):
        s = les.Solver(g, f, SEP)
        s.set_state(I.ambient_primitives(g.N, f.TR))
        s.step(4)
        np.testing.assert_array_equal(b.get_state(les.LES_STATE_RAW, jet=j), s.get_state(les.LES_STATE_RAW))
        s.close()
    b.close()


def test_separable_rejects_curvilinear_grid():
    spec = I.wavy_box_grid((12, 10, 9), amp=0.05)
    with pytest.raises(les.LesError) as e:
        les.Solver(spec, I.FlowParams(), SEP)
    assert e.value.code == -1 and "product" in str(e.value)


def test_separable_paper_scale_sampled_residual():
    """Paper-scale jet (384x256x144): the separable residual at sampled points
    (faces, edges, interior) against the oracle's sampled residual."""
    spec, fp = I.jet_paper_scale()
    prim = I.smooth_random_primitives(spec, seed=31, amp=0.05)
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    ni, nj, nk = spec.dims
    rng = np.random.default_rng(5)
    pts = [np.stack([rng.integers(1, ni - 1, 2000), rng.integers(1, nj - 1, 2000), rng.integers(1, nk - 1, 2000)], 1)]
    for i in (1, ni // 2, ni - 2):
        for j in (1, nj // 2, nj - 2):
            for k in (1, nk // 2, nk - 2):
                pts.append(np.array([[i, j, k]]))
    pq = np.concatenate(pts)
    lin = (pq[:, 2].astype(np.int64) * nj + pq[:, 1]) * ni + pq[:, 0]
    r_or = oracle.rhs_sampled(g, p, m, q, lin)
    del m, q
    s = les.Solver(spec, fp, SEP)
    s.set_state(prim)
    s.step(0)
    r = s.rhs()[:, lin]
    s.close()
    scale = np.abs(r_or).max(axis=1, keepdims=True) + 1e-30
    err = np.abs(r - r_or) / scale
    print("paper-scale separable sampled residual error / scale:", err.max(axis=1))
    assert err.max() < 2e-5, err.max(axis=1)
