"""The allocation-free diagnostics entry point (les_diag_sums_noalloc) against
the handle-based les_get_diagnostics, through the C ABI.

Callers that cannot allocate device memory (a framework's caching allocator
owns the device, or a per-step monitoring hook must avoid cudaMalloc latency
and device-wide synchronisation) pass their own state/residual/output
buffers; the entry point's only scratch is a fixed file-scope device array.
This file is collected last on purpose.  It must pass alone in a fresh
process and after every other test."""
import numpy as np
import pytest

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


def _check(out, ref, q):
    assert out[0] == ref["max_abs_rhs_rho"]
    np.testing.assert_allclose(out[1:6], ref["l2_rhs"], rtol=1e-12)
    mag = np.abs(q).sum(axis=1)
    assert np.all(np.abs(out[6:11] - ref["sum_qhat"]) <= 1e-13 * mag)
    assert out[11] == 0


def test_noalloc_diagnostics_match_handle_twice():
    import torch
    spec = I.wavy_box_grid((37, 23, 19), amp=0.06, bc=(1, 3, 1, 1, 1, 1))
    fp = I.FlowParams(Re=500.0)
    prim = I.smooth_random_primitives(spec, seed=21, amp=0.08)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim)
    out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        if call == 1:
            s.step(2)  # the second call sees a different state
        ref = s.diagnostics()
        q = s.get_state(les.LES_STATE_RAW)
        r = s.rhs()
        dq = torch.from_numpy(q).cuda()
        dr = torch.from_numpy(r).cuda()
        out.fill_(float("nan"))
        rc = les.les_diag_sums_noalloc(dq.data_ptr(), dr.data_ptr(), spec.N, out.data_ptr())
        assert rc == les.LES_OK
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref, q)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = les.les_diag_sums_noalloc(buf.data_ptr(), buf.data_ptr(), les.NOALLOC_MAX_POINTS + 1,
                                   buf.data_ptr())
    assert rc == les.LES_ERR_ARG
    assert les.les_diag_sums_noalloc(buf.data_ptr(), buf.data_ptr(), 0, buf.data_ptr()) == les.LES_ERR_ARG
