"""Long runs of the jet configurations (slow GPU tests).

- Paper-scale FP64 jet, 384x256x144, 1000 steps: the time-averaged
  centerline velocity over steps 991-1000 is compared with the oracle
  restarted from the GPU state at step 990 (the oracle cannot march 1000
  steps of 14M points in test time, but it can march the last 10).
- The same jet in FP32: per-field relative L2 against the FP64 GPU path
  after 100 and 1000 steps (reported; bounded), and after 1000 steps also
  over the interior away from the boundary planes.
- Large FP32 jet, 768x384x192, TR 2, 500 steps with the surface probe on a
  cylinder r = 3 every 5 steps: the state stays finite and the probe ring
  holds the expected frames, the last of which matches the oracle's
  trilinear probe of the final state.
"""
import numpy as np
import pytest

import oracle
from helpers import error_split, rel_l2, to_oracle
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


def _centerline_u(spec, q):
    """4-point average of u = (rho u)/rho around y = z = 0 (even nj, nk with a
    symmetric grid: the axis lies midway between rows nj/2-1, nj/2 and planes
    nk/2-1, nk/2).  q: conserved state [5][N]."""
    ni, nj, nk = spec.dims
    r = q[0].reshape(nk, nj, ni)
    ru = q[1].reshape(nk, nj, ni)
    js, ks = (nj // 2 - 1, nj // 2), (nk // 2 - 1, nk // 2)
    return sum(ru[k, j] / r[k, j] for j in js for k in ks) / 4.0


@pytest.fixture(scope="module")
def fp64_run():
    spec, fp = I.jet_paper_scale()
    prim = I.ambient_primitives(spec.N, fp.TR)
    s = les.Solver(spec, fp, les.LES_FP64)
    s.set_state(prim)
    out = {}
    s.step(100)
    out["q100"] = s.get_state(les.LES_STATE_CONSERVED)
    s.step(890)
    out["raw990"] = s.get_state(les.LES_STATE_RAW)
    out["time990"] = s.time()
    cl = []
    for _ in range(10):
        s.step(1)
        cl.append(_centerline_u(spec, s.get_state(les.LES_STATE_CONSERVED)))
    out["cl_mean"] = np.mean(cl, axis=0)
    out["q1000"] = s.get_state(les.LES_STATE_CONSERVED)
    out["diag"] = s.diagnostics()
    s.close()
    return spec, fp, out


def test_paper_scale_1000_steps_centerline_vs_oracle(fp64_run):
    spec, fp, out = fp64_run
    step, dt = out["time990"]
    assert step == 990
    assert np.all(np.isfinite(out["q1000"]))
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    q = out["raw990"]
    cl = []
    for l in range(10):
        q = oracle.step(g, p, m, q, 1, step + l, dt)
        cl.append(_centerline_u(spec, oracle.state_out(g, p, m, q, False)))
    ref = np.mean(cl, axis=0)
    err = np.abs(out["cl_mean"] - ref).max() / np.abs(ref).max()
    print("centerline u (steps 991-1000): max |gpu - oracle| / max|u| =", err,
          "; u on the axis at x = 0, L/4, L/2:", ref[0], ref[len(ref) // 4], ref[len(ref) // 2])
    assert err <= 1e-11
    # the jet has entered the domain: core velocity at the inflow plane is M_j
    assert ref[0] == pytest.approx(fp.mach_j, rel=1e-2)


def test_paper_scale_fp32_error_100_and_1000_steps(fp64_run):
    spec, fp, out = fp64_run
    prim = I.ambient_primitives(spec.N, fp.TR)
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(prim)
    s.step(100)
    e100 = rel_l2(s.get_state(les.LES_STATE_CONSERVED), out["q100"])
    s.step(900)
    q = s.get_state(les.LES_STATE_CONSERVED)
    s.close()
    e1000 = rel_l2(q, out["q1000"])
    # the interior (8-point margin) without the boundary planes, where the
    # far-field condition of the inflow face may take the other branch in
    # FP32 for a normal velocity near zero
    ni, nj, nk = spec.dims
    d = (q - out["q1000"]).reshape(5, nk, nj, ni)[:, 8:-8, 8:-8, 8:-8]
    den = np.sqrt((out["q1000"] ** 2).sum(axis=1))
    ein = np.sqrt((d.reshape(5, -1) ** 2).sum(axis=1)) / den
    share = error_split(q, out["q1000"], spec.dims)[2]
    print("fp32 vs fp64 rel L2 per field, 100 steps:", e100, " 1000 steps:", e1000, " interior:", ein,
          " i=0 share:", share)
    assert np.all(np.isfinite(q))
    assert np.all(e100 <= 1e-5), e100
    assert np.all(ein <= 1e-5), ein
    # over the whole grid: rho, rho u, e at the bar; the transverse momenta
    # may exceed it only by the inflow plane's far-field branch (see
    # test_batched_fp32_against_oracle), which must then hold the excess
    assert np.all(e1000[[0, 1, 4]] <= 1e-5), e1000
    for f in (2, 3):
        assert e1000[f] <= 1e-5 or (e1000[f] <= 2e-4 and share[f] >= 0.9), (f, e1000, share)


def test_large_fp32_500_steps_with_probe():
    import torch
    spec, fp = I.jet_large()
    xyz = I.cylinder_points(3.0, 256, 384, 0.5, spec.x.max() - 0.5)
    npts = xyz.shape[1]
    cap = 128
    dev = torch.zeros((cap, 5, npts), dtype=torch.float32, device="cuda")
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(I.ambient_primitives(spec.N, fp.TR))
    les.les_probe_surface(s.h, xyz, 5, dev.data_ptr(), cap)
    s.step(500)
    torch.cuda.synchronize()
    nfr = les.les_probe_frames(s.h)
    q = s.get_state(les.LES_STATE_CONSERVED)
    d = s.diagnostics()
    s.close()
    assert nfr == 100
    assert np.all(np.isfinite(q)) and np.isfinite(d["max_abs_rhs_rho"])
    frames = dev.double().cpu().numpy()
    assert np.all(np.isfinite(frames[:nfr]))
    # the last frame (step 500) against the oracle's probe of the final state
    g, p = to_oracle(spec, fp)
    m = oracle.metrics(g)
    ref = oracle.probe(g, p, m, oracle.qhat_from(g, p, m, q, False), xyz)
    last = frames[(nfr - 1) % cap]
    scale = np.abs(ref).max(axis=1, keepdims=True)
    err = np.abs(last - ref) / scale
    print("large fp32 probe frame 100 vs oracle probe: max rel", err.max(axis=1))
    assert err.max() <= 2e-5
