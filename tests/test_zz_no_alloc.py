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


def test_noalloc_multi_block_sums_against_host():
    """3 x 65,536 + 17 points: three full reduction blocks and a partial one,
    so the cross-block combine (maximum, sums of squares, Neumaier merge of
    the per-block sums with their compensations, non-finite count) runs.
    Two calls in a row on different data, compared with sums formed on the
    host (math.fsum, exactly rounded); the second input plants two non-finite
    values in different blocks."""
    import math
    import torch
    n = 3 * 65536 + 17
    rng = np.random.default_rng(31)
    out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        q = rng.normal(1.0, 0.3, (5, n)) * (1.0 + 1e3 * (rng.uniform(size=(5, n)) < 1e-3))
        r = rng.normal(0.0, 1e-2, (5, n))
        r[:, -5:] = 0.0
        nbad = 0
        if call == 1:
            q[2, 70000] = np.inf
            r[4, 150000] = np.nan
            nbad = 2
        dq = torch.from_numpy(q).cuda()
        dr = torch.from_numpy(r).cuda()
        out.fill_(float("nan"))
        rc = les.les_diag_sums_noalloc(dq.data_ptr(), dr.data_ptr(), n, out.data_ptr())
        assert rc == les.LES_OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[11] == nbad
        if nbad:
            continue
        assert o[0] == np.abs(r[0]).max()
        np.testing.assert_allclose(o[1:6], np.sqrt((r ** 2).sum(axis=1)), rtol=1e-12)
        for f in range(5):
            exact = math.fsum(q[f])
            assert abs(o[6 + f] - exact) <= 4 * np.finfo(float).eps * abs(exact), f
