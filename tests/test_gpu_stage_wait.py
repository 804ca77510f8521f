"""Timeout path of the fused FP32 stage's bounded staging waits.

The next plane's state reaches the fused stage by a TMA copy that completes
an mbarrier, and every wait on it is bounded.  With the bound set to zero
polls (les_debug_stage_wait) the first wait of every CTA gives up while its
copy is still in flight, on a healthy device.  The library must then report
LES_ERR_TIMEOUT at the next synchronising call and record site 8 in the
handle's error word; and, since the stage falls back to direct global loads
for the rest of the launch and waits for the abandoned copy before the CTA
exits, the state must still be the bits of a normal step.  The failure is
made by the bound, not by a copy that never comes: nothing here can hang.
"""
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


def _stretched_periodic():
    # a Cartesian-product grid periodic in i and j: no TMA map, so the
    # separable form stages its planes with per-thread copies
    x1 = np.cumsum(np.linspace(0.8, 1.2, 37)) * 0.1
    y1 = np.cumsum(np.linspace(1.1, 0.9, 19)) * 0.1
    z1 = np.arange(10) * 0.11
    g = I.product_grid(x1 - x1[0], y1 - y1[0], z1)
    g.periodic = (1, 1, 1)
    g.shift = np.diag([x1[-1] - x1[0] + 0.12, y1[-1] - y1[0] + 0.09, 1.1])
    g.bc = (0, 0, 0, 0, 0, 0)
    return g


def _run(specs, fps, prec, tiling, polls, steps=3):
    s = les.Solver(specs, fps, prec)
    les.les_set_fused_tiling(s.h, *tiling)
    if polls is not None:
        les.les_debug_stage_wait(s.h, polls)
    for j, g in enumerate(specs):
        s.set_state(I.smooth_random_primitives(g, 70 + j, amp=0.05), jet=j)
    s.step(steps)
    out = [les.les_get_state_rc(s.h, g.N, les.LES_STATE_RAW, j) for j, g in enumerate(specs)]
    word = les.les_bounds_violation(s.h)
    d = les.les_get_diagnostics(s.h, 0, check=False)
    s.close()
    return out, word, d["rc"]


@pytest.mark.parametrize("prec", [les.LES_FP32, les.LES_FP32_SEPARABLE])
@pytest.mark.parametrize("tiling", [(8, 0), (16, 5)])
def test_wait_timeout_reported_and_state_unchanged(prec, tiling):
    """Single jet (TMA staging on every tile); tile height 16 with 5-plane
    chunks also walks several items per CTA after the fallback."""
    spec, fp = I.jet_small()
    ref, w0, rc0 = _run([spec], [fp], prec, tiling, None)
    got, w1, rc1 = _run([spec], [fp], prec, tiling, 0)
    assert ref[0][1] == les.LES_OK and w0 == 0 and rc0 == les.LES_OK
    assert got[0][1] == les.LES_ERR_TIMEOUT
    assert rc1 == les.LES_ERR_TIMEOUT
    assert w1 >> 48 == 8
    np.testing.assert_array_equal(got[0][0], ref[0][0])


@pytest.mark.parametrize("prec", [les.LES_FP32, les.LES_FP32_SEPARABLE])
def test_wait_timeout_in_a_batch_with_unstaged_jets(prec):
    """A batch whose jets take both staging paths (TMA box; per-thread copies
    or direct loads on the grid periodic in i and j): after a CTA's wait gives
    up, its later items of either kind use direct loads, with the same bits."""
    spec, fp = I.jet_small()
    per = _stretched_periodic()
    fper = I.FlowParams(Re=800.0)
    specs, fps = [spec, per, spec], [fp, fper, fp]
    ref, _, _ = _run(specs, fps, prec, (8, 3), None)
    got, w1, _ = _run(specs, fps, prec, (8, 3), 0)
    assert w1 >> 48 == 8
    for (a, rca), (b, rcb) in zip(ref, got):
        assert rca == les.LES_OK and rcb == les.LES_ERR_TIMEOUT
        np.testing.assert_array_equal(b, a)


def test_default_bound_restored_and_arguments_checked():
    spec, fp = I.jet_small()
    ref, _, _ = _run([spec], [fp], les.LES_FP32, (8, 0), None, steps=1)
    s = les.Solver(spec, fp, les.LES_FP32)
    les.les_set_fused_tiling(s.h, 8, 0)
    les.les_debug_stage_wait(s.h, 0)
    les.les_debug_stage_wait(s.h, -1)
    s.set_state(I.smooth_random_primitives(spec, 70, amp=0.05))
    s.step(1)
    q, rc = les.les_get_state_rc(s.h, spec.N, les.LES_STATE_RAW)
    assert rc == les.LES_OK and les.les_bounds_violation(s.h) == 0
    np.testing.assert_array_equal(q, ref[0][0])
    with pytest.raises(les.LesError):
        les.les_debug_stage_wait(s.h, -2)
    s.close()
    s = les.Solver(spec, fp, les.LES_FP64)
    with pytest.raises(les.LesError):
        les.les_debug_stage_wait(s.h, 0)
    s.close()


@pytest.mark.parametrize("ty", [8, 16])
def test_wait_timeout_in_lockstep_waves(ty):
    """The lockstep form (kc = -1) with more tiles than CTAs, so that the
    CTAs first march whole columns in waves and then take balanced shares of
    the rest: after the first wait of each CTA gives up, the cursor keeps
    walking both kinds of work with direct loads, and the bits are those of
    a normal step."""
    import torch
    spec, fp = I.jet_small()
    ni, nj, _ = spec.dims
    tiles = -(-(ni - 2) // 30) * -(-(nj - 2) // (ty - 2))
    n = torch.cuda.get_device_properties(0).multi_processor_count // tiles + 2
    specs, fps = [spec] * n, [fp] * n
    ref, _, _ = _run(specs, fps, les.LES_FP32, (ty, -1), None, steps=2)
    got, w1, rc = _run(specs, fps, les.LES_FP32, (ty, -1), 0, steps=2)
    assert w1 >> 48 == 8 and rc == les.LES_ERR_TIMEOUT
    for (a, rca), (b, rcb) in zip(ref, got):
        assert rca == les.LES_OK and rcb == les.LES_ERR_TIMEOUT
        np.testing.assert_array_equal(b, a)
