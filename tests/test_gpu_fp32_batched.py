"""FP32 fused stage and the batched form, through the C ABI.

- residual of the fused single-pass FP32 kernel against the FP64 oracle on
  ragged, periodic, mixed and minimum-size grids (relative to the residual
  scale, FP32 rounding of fluxes that are differences of O(1) terms);
- batched jets (uneven grids, per-jet Mach/TR/Re/seed, one persistent launch
  per stage) are bit-identical to single-jet runs of the same precision;
- the fused stage gives the same bits for every tile height and k-chunk,
  and for the balanced tile-plane ranges (les_set_fused_tiling).
"""
import numpy as np
import pytest

import oracle
from helpers import error_split, rel_l2, to_oracle
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


def _mixed():
    g = I.jet_grid(45, 33, 12, 6.0, 5.0, 4.0, 0.2, 4.0 / 11)
    ni, nj, _ = g.dims
    g.z = np.repeat(np.arange(12) * (4.0 / 12), ni * nj)
    g.periodic = (0, 0, 1)
    g.shift = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 4.0]], dtype=float)
    g.bc = (2, 3, 1, 1, 0, 0)
    return g


CASES = {
    "jet_ragged_70x37x29": lambda: I.jet_grid(70, 37, 29, 8.0, 6.0, 6.0, 0.15, 0.18),
    "wavy_box_33x18x21": lambda: I.wavy_box_grid((33, 18, 21), amp=0.06, bc=(1, 3, 1, 1, 1, 1)),
    "wavy_periodic_40x17x9": lambda: I.wavy_periodic_grid((40, 17, 9), amp=0.2),
    "mixed_periodic_z": _mixed,
    "tiny_4x4x4": lambda: I.wavy_box_grid((4, 4, 4), amp=0.02),
    "tiny_periodic_4x5x4": lambda: I.wavy_periodic_grid((4, 5, 4), amp=0.1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fused_fp32_residual_parity(case):
    spec = CASES[case]()
    fp = I.FlowParams(Re=800.0)
    prim = I.smooth_random_primitives(spec, 17, amp=0.08)
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
    r_or = oracle.rhs(g, p, m, q)
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(prim)
    s.step(0)  # runs the tuner for this shape
    r = s.rhs()
    s.close()
    scale = np.abs(r_or).max(axis=1, keepdims=True) + 1e-30
    err = np.abs(r - r_or) / scale
    assert err.max() < 2e-5, (case, err.max(axis=1))


def test_batched_bit_identical_to_single_fp32():
    jets = I.batch_jets(6, seed=4)
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    prims = [I.ambient_primitives(g.N, f.TR) for g, f in jets]
    b = les.Solver(specs, fps, les.LES_FP32)
    for j, pr in enumerate(prims):
        b.set_state(pr, jet=j)
    b.step(4)
    for j, (g, f) in enumerate(jets):
        s = les.Solver(g, f, les.LES_FP32)
        s.set_state(prims[j])
        s.step(4)
        np.testing.assert_array_equal(b.get_state(les.LES_STATE_RAW, jet=j), s.get_state(les.LES_STATE_RAW))
        s.close()
    b.close()


def test_batched_bit_identical_to_single_fp64():
    jets = I.batch_jets(3, seed=9)
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    b = les.Solver(specs, fps, les.LES_FP64)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.ambient_primitives(g.N, f.TR), jet=j)
    b.step(2)
    for j, (g, f) in enumerate(jets):
        s = les.Solver(g, f, les.LES_FP64)
        s.set_state(I.ambient_primitives(g.N, f.TR))
        s.step(2)
        np.testing.assert_array_equal(b.get_state(les.LES_STATE_RAW, jet=j), s.get_state(les.LES_STATE_RAW))
        s.close()
    b.close()


def test_batched_fp32_against_oracle():
    """One jet of the batch, 20 steps from the ambient start, against the FP64
    oracle: relative L2 <= 1e-5 for every field, over the whole grid and in
    the interior.  The transverse momenta (only the inflow noise and its
    start-up waves, ~1e-3 of rho u) are the sensitive fields: outside the jet
    the entrained ambient flow crosses the inflow plane with a normal velocity
    near zero, where the far-field condition switches the tangential velocity
    and entropy between the interior and the freestream (Sec. "Far Field
    Boundary"), so FP32 rounding of the face state could select the other
    branch at a few face points; the FP32 boundary arithmetic forms its small
    differences accurately (c_e - c_inf from T_e - T_inf in FP64), which keeps
    this jet's faces on the FP64 branches."""
    jets = I.batch_jets(3, seed=12)
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    b = les.Solver(specs, fps, les.LES_FP32)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.ambient_primitives(g.N, f.TR), jet=j)
    b.step(20)
    g, f = jets[1]
    go, po = to_oracle(g, f)
    m = oracle.metrics(go)
    q = oracle.apply_bc(go, po, m, oracle.qhat_from(go, po, m, I.ambient_primitives(g.N, f.TR), True), 0)
    dt = oracle.dt_cfl(go, po, m, q)
    ref = oracle.state_out(go, po, m, oracle.step(go, po, m, q, 20, 0, dt), False)
    got = b.get_state(les.LES_STATE_CONSERVED, jet=1)
    b.close()
    whole, inner, share = error_split(got, ref, g.dims)
    print("batched fp32 jet 1, 20 steps, rel L2 per field:", whole, " interior:", inner, " i=0 share:", share)
    assert np.all(inner <= 1e-5), inner
    assert np.all(whole <= 1e-5), (whole, share)


@pytest.mark.parametrize("prec", [les.LES_FP32, les.LES_FP32_SEPARABLE])
def test_fused_stage_independent_of_tiling(prec):
    """Every work decomposition of the fused stage (tile height 8 or 16; fixed
    k-chunks, including a chunk of one plane; the balanced tile-plane ranges
    whose cuts fall mid-column; the lockstep form's whole-column waves before
    them) gives the same bits, on a batch of uneven jets."""
    jets = I.batch_jets(4, seed=11)
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    out = []
    for ty, kc in ((8, 100000), (16, 100000), (8, 1), (16, 5), (8, 0), (16, 0), (8, -1), (16, -1)):
        b = les.Solver(specs, fps, prec)
        for j, (g, f) in enumerate(jets):
            b.set_state(I.smooth_random_primitives(g, 40 + j, amp=0.05), jet=j)
        les.les_set_fused_tiling(b.h, ty, kc)
        b.step(3)
        out.append([b.get_state(les.LES_STATE_RAW, jet=j) for j in range(len(jets))])
        assert f"ty={ty}" in les.les_describe(b.h)
        b.close()
    for other in out[1:]:
        for a, c in zip(out[0], other):
            np.testing.assert_array_equal(a, c)


def test_fused_tiling_arguments_checked():
    spec, fp = I.jet_small()
    s = les.Solver(spec, fp, les.LES_FP32)
    for ty, kc in ((4, 0), (8, -2)):
        with pytest.raises(les.LesError):
            les.les_set_fused_tiling(s.h, ty, kc)
    s.close()
    s = les.Solver(spec, fp, les.LES_FP64)
    with pytest.raises(les.LesError):
        les.les_set_fused_tiling(s.h, 8, 0)
    s.close()


@pytest.mark.slow
def test_config4_batch64_bit_identical_to_single_jets():
    """The 64-jet batch of the batched benchmark form (master seed 4), FP32,
    one persistent launch per stage in a captured step: every jet's state after
    3 steps has the same bits as the same jet run alone."""
    jets = I.batch_jets(64, seed=4)
    specs = [g for g, _ in jets]
    fps = [f for _, f in jets]
    b = les.Solver(specs, fps, les.LES_FP32)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.ambient_primitives(g.N, f.TR), jet=j)
    b.step(3)
    for j, (g, f) in enumerate(jets):
        s = les.Solver(g, f, les.LES_FP32)
        s.set_state(I.ambient_primitives(g.N, f.TR))
        s.step(3)
        np.testing.assert_array_equal(b.get_state(les.LES_STATE_RAW, jet=j), s.get_state(les.LES_STATE_RAW))
        s.close()
    b.close()


@pytest.mark.parametrize("prec", [les.LES_FP32, les.LES_FP32_SEPARABLE])
def test_fp32_unscaled_store_state_and_diagnostics(prec):
    """FP32 handles store the unscaled Q: a uniform ambient state is stored
    bit-identically at every point of a stretched grid and stays so over a
    step (the far-field faces see the ambient itself); the raw state is Q; the
    conservation sums are those of Qhat = J^-1 Q (FP64, against the oracle's
    sums of the same state)."""
    spec, fp = I.jet_small()
    ni, nj, nk = spec.dims
    s = les.Solver(spec, fp, prec)
    amb = I.ambient_primitives(spec.N, fp.TR)
    s.set_state(amb, les.LES_STATE_PRIMITIVE)
    raw = s.get_state(les.LES_STATE_RAW)
    q = s.get_state(les.LES_STATE_CONSERVED)
    np.testing.assert_array_equal(raw, q)
    # every interior point holds the same FP32 words
    body = raw.reshape(5, nk, nj, ni)[:, 1:-1, 1:-1, 1:-1]
    for f in range(5):
        assert np.unique(body[f]).size == 1, f
    ref = body[:, 0, 0, 0].copy()
    s.step(1)
    q1 = s.get_state(les.LES_STATE_CONSERVED).reshape(5, nk, nj, ni)
    # points no face reaches within one step (5 stages x 2 points) keep the
    # ambient to far below FP32 rounding (a J^-1-scaled FP32 store gives
    # differences of ~1e-8 here)
    far = q1[:, 11:nk - 11, 11:nj - 11, ni // 2:ni - 11]
    dev = np.abs(far - ref[:, None, None, None]).max(axis=(1, 2, 3))
    assert np.all(dev <= 1e-12), dev
    # conservation sums: Qhat of the (FP32-valued) state, summed in FP64
    s.set_state(I.smooth_random_primitives(spec, seed=31, amp=0.05), les.LES_STATE_PRIMITIVE)
    s.step(2)
    qc = s.get_state(les.LES_STATE_CONSERVED)
    d = s.diagnostics()
    s.close()
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    dor = oracle.diag(g, p, m, oracle.qhat_from(g, p, m, qc, False))
    qh = oracle.qhat_from(g, p, m, qc, False)
    mag = np.abs(qh).sum(axis=1)
    assert np.all(np.abs(d["sum_qhat"] - dor["sum_qhat"]) <= 1e-13 * mag), (d["sum_qhat"], dor["sum_qhat"])


def test_handles_stepped_from_two_host_threads():
    """Two FP32 handles of new grid shapes stepped at the same time from two
    host threads (both run the autotuner and share its cache): both finish
    with the state a single-threaded run gives."""
    import threading
    shapes = [I.jet_grid(29 + 2 * t, 21, 17, 8.0, 6.0, 6.0, 0.15, 0.18) for t in range(2)]
    fp = I.FlowParams(Re=1e4)

    def run(spec, out, idx):
        s = les.Solver(spec, fp, les.LES_FP32)
        s.set_state(I.smooth_random_primitives(spec, 60 + idx, amp=0.05))
        s.step(3)
        out[idx] = s.get_state(les.LES_STATE_RAW)
        s.close()

    res = [None, None]
    th = [threading.Thread(target=run, args=(shapes[i], res, i)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i in range(2):
        ref = [None, None]
        run(shapes[i], ref, i)
        np.testing.assert_array_equal(res[i], ref[i])


@pytest.mark.parametrize("prec", [les.LES_FP32, les.LES_FP32_SEPARABLE])
def test_lockstep_waves_bit_identical(prec):
    """A grid with more tiles than CTAs (400 x 160 x 12: 378 tiles of 32 x 8,
    168 of 32 x 16), so that the lockstep form runs a wave of whole columns
    before sharing out the rest: the same bits as whole columns, k-chunks and
    the balanced ranges."""
    spec = I.jet_grid(400, 160, 12, 20.0, 10.0, 10.0, 0.125, 0.1)
    fp = I.FlowParams(Re=1e4)
    prim = I.smooth_random_primitives(spec, 5, amp=0.05)
    out = []
    for ty, kc in ((8, 100000), (8, 0), (8, -1), (16, -1), (16, 3)):
        s = les.Solver(spec, fp, prec)
        s.set_state(prim)
        les.les_set_fused_tiling(s.h, ty, kc)
        s.step(2)
        out.append(s.get_state(les.LES_STATE_RAW))
        if kc == -1:
            assert "kc=lockstep" in les.les_describe(s.h)
        s.close()
    for o in out[1:]:
        np.testing.assert_array_equal(o, out[0])
