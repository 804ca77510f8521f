"""Full-size checks in the configurations bench.py times.

The oracle cannot step a 14M- or 57M-point grid in test time, but it can
evaluate the residual at sampled points of the same state: the GPU residual
(the kernels of a stage, through les_debug_rhs) is compared there, on the
paper-scale FP64 jet (384x256x144) and the large FP32 jet (768x384x192).
The samples include points next to every face and edge of the grid.
"""
import numpy as np
import pytest

import oracle
from helpers import rel_l2, to_oracle
from paper_2212_12365_gb300 import inputs as I
from paper_2212_12365_gb300 import les

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()


def _samples(dims, n, seed):
    ni, nj, nk = dims
    rng = np.random.default_rng(seed)
    pts = [np.stack([rng.integers(1, ni - 1, n), rng.integers(1, nj - 1, n), rng.integers(1, nk - 1, n)], 1)]
    # points adjacent to faces, edges and corners of the interior
    for i in (1, ni // 2, ni - 2):
        for j in (1, nj // 2, nj - 2):
            for k in (1, nk // 2, nk - 2):
                pts.append(np.array([[i, j, k]]))
    p = np.concatenate(pts)
    return (p[:, 2].astype(np.int64) * nj + p[:, 1]) * ni + p[:, 0]


def _check(make, precision, tol, nsamp):
    spec, fp = make()
    prim = I.smooth_random_primitives(spec, seed=31, amp=0.05)
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    pts = _samples(spec.dims, nsamp, 5)
    r_or = oracle.rhs_sampled(g, p, m, q, pts)
    del m, q
    s = les.Solver(spec, fp, precision)
    s.set_state(prim)
    s.step(0)
    r = s.rhs()[:, pts]
    s.close()
    scale = np.abs(r_or).max(axis=1, keepdims=True) + 1e-30
    err = np.abs(r - r_or) / scale
    print(make.__name__, "max sampled residual error / field scale:", err.max(axis=1))
    assert err.max() < tol, err.max(axis=1)


def test_paper_scale_fp64_sampled_residual():
    _check(I.jet_paper_scale, les.LES_FP64, 1e-12, 3000)


def test_large_fp32_sampled_residual():
    _check(I.jet_large, les.LES_FP32, 2e-5, 3000)


def test_paper_scale_fp32_vs_fp64_100_steps():
    """Precision form on the paper-scale jet: FP32 against the GPU FP64 path
    after 100 steps from the ambient start (relative L2 per field)."""
    spec, fp = I.jet_paper_scale()
    prim = I.ambient_primitives(spec.N, fp.TR)
    out = {}
    for prec in (les.LES_FP64, les.LES_FP32):
        s = les.Solver(spec, fp, prec)
        s.set_state(prim)
        s.step(100)
        out[prec] = s.get_state(les.LES_STATE_CONSERVED)
        s.close()
    err = rel_l2(out[les.LES_FP32], out[les.LES_FP64])
    print("paper-scale fp32 vs fp64, 100 steps, rel L2 per field:", err)
    assert np.all(err <= 1e-5), err
