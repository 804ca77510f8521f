"""Binary reproducibility in the manner of the paper's partitioning check
(Sec. "Computational Performance Assessment": the continuity residual monitor
of runs on differently partitioned meshes must agree bit for bit).  Here the
partitions are the fused FP32 stage's work decompositions — tile heights,
k-chunks, and the balanced tile-plane ranges whose cuts fall mid-column — and
for FP64 a second run: over 1500 steps of a jet the max |RHS_rho| history
(every 100 steps) and the final state are identical bit for bit."""
import numpy as np
import pytest

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


def _history(prec, tiling=None, steps=1500, every=100):
    spec, fp = I.jet_small()
    s = les.Solver(spec, fp, prec)
    if tiling:
        les.les_set_fused_tiling(s.h, *tiling)
    s.set_state(I.ambient_primitives(spec.N, fp.TR))
    hist = []
    for _ in range(steps // every):
        s.step(every)
        hist.append(s.diagnostics()["max_abs_rhs_rho"])
    q = s.get_state(les.LES_STATE_RAW)
    s.close()
    return np.array(hist), q


def test_fp32_residual_monitor_identical_across_decompositions():
    runs = [_history(les.LES_FP32, t) for t in ((8, 100000), (16, 5), (8, 0), (16, 0))]
    h0, q0 = runs[0]
    assert np.all(np.isfinite(h0)) and h0[-1] > 0
    for h, q in runs[1:]:
        np.testing.assert_array_equal(h, h0)
        np.testing.assert_array_equal(q, q0)


def test_fp64_residual_monitor_identical_across_runs():
    h0, q0 = _history(les.LES_FP64)
    h1, q1 = _history(les.LES_FP64)
    assert np.all(np.isfinite(h0)) and h0[-1] > 0
    np.testing.assert_array_equal(h1, h0)
    np.testing.assert_array_equal(q1, q0)
