"""FW-H far-field pressure on the GPU (les_fwh) against the oracle
(oracle/fwh.py) element by element: on the exact field of a point monopole
(either ring precision, a wrapped ring; the staged observer pass and, for
observer times far apart, the direct one), on a steady uniform stream (the
quadratic momentum-flux term alone, against its closed form as well), on the
probe frames of an LES jet run (real flow through the surface), bit-identical
reruns, and the refused inputs."""
import numpy as np
import pytest

from oracle import fwh
from paper_2212_12365_gb300 import inputs as I
from paper_2212_12365_gb300 import les

pytestmark = pytest.mark.gpu

RHO0, P0, C0 = 1.3, 1.0 / 1.4, 0.8
SIG, TC, AMP = 0.5, 7.0, 1e-3
SRC = np.array([0.1, -0.05, 0.07])


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()


def _sphere(a, nth, nph):
    th_e = np.linspace(0.0, np.pi, nth + 1)
    th = 0.5 * (th_e[1:] + th_e[:-1])
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    n = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)]).reshape(3, -1)
    area = np.repeat(a * a * (np.cos(th_e[:-1]) - np.cos(th_e[1:])) * 2 * np.pi / nph, nph)
    return a * n, n, area


def _monopole(x, t):
    d = x - SRC[:, None]
    R = np.sqrt((d * d).sum(axis=0))
    tr = t - R / C0
    q = AMP * np.exp(-((tr - TC) / SIG) ** 2)
    qd = -2.0 * (tr - TC) / SIG ** 2 * q
    ur = qd / (4 * np.pi * C0 * R) + q / (4 * np.pi * R * R)
    p = RHO0 * qd / (4 * np.pi * R)
    return p, ur * d / R


def _frames(xyz, n, dtau):
    fr = np.empty((n, 5, xyz.shape[1]))
    for m in range(n):
        p, u = _monopole(xyz, m * dtau)
        fr[m, 0] = RHO0 + p / C0 ** 2
        fr[m, 1:4] = u
        fr[m, 4] = P0 + p
    return fr


def _ring(frames, cap, dtype):
    """A device ring as les_probe_surface leaves it after writing all frames."""
    import torch
    n = frames.shape[0]
    ring = np.zeros((cap,) + frames.shape[1:])
    for m in range(n):
        ring[m % cap] = frames[m]
    return torch.tensor(ring, dtype=dtype, device="cuda")


@pytest.mark.parametrize("prec", [les.LES_FP64, les.LES_FP32])
def test_monopole_against_the_oracle_and_the_exact_field(prec):
    import torch
    xyz, nrm, area = _sphere(1.0, 48, 96)
    dtau, nfr, cap = 0.01, 1400, 1000          # the ring holds the last 1000 of 1400 frames
    frames = _frames(xyz, nfr, dtau)
    ring = _ring(frames, cap, torch.float64 if prec == les.LES_FP64 else torch.float32)
    obs = np.array([[6.0, 0.0, 0.0], [0.0, 3.0, -5.0], [-2.0, -2.0, 4.0]]).T
    used = frames[nfr - cap:]                  # tau = 0 at frame nfr - cap
    if prec == les.LES_FP32:
        used = used.astype(np.float32).astype(np.float64)
    t0, dt_obs, nt = 8.8, 0.015, 400           # emission times within the ring's 1000 frames
    got = les.les_fwh(ring.data_ptr(), prec, cap, nfr, xyz, nrm, area, dtau, P0, C0, obs, t0, dt_obs, nt)
    ref = fwh.pressure(used, xyz, nrm, area, dtau, RHO0, P0, C0, obs, t0, dt_obs, nt)
    scale = np.abs(ref).max()
    # FP32 storage of the per-frame sources and FP32 products: ~1e-6 of the signal
    assert np.abs(got - ref).max() <= 2e-5 * scale, np.abs(got - ref).max() / scale
    # and the physics: the monopole's exact pressure at the observers
    t = t0 + dt_obs * np.arange(nt) + (nfr - cap) * dtau
    exact = np.stack([_monopole(obs[:, o:o + 1], t)[0] for o in range(obs.shape[1])])
    assert np.abs(got - exact).max() <= 5e-3 * np.abs(exact).max()


def test_sparse_observer_times_take_the_direct_pass():
    """Observer times far apart (a window of frames per panel too long to
    stage in shared memory): the direct observer pass, against the oracle."""
    import torch
    xyz, nrm, area = _sphere(1.0, 24, 48)
    dtau, nfr = 0.01, 1400
    frames = _frames(xyz, nfr, dtau)
    ring = _ring(frames, nfr, torch.float64)
    obs = np.array([[6.0, 0.0, 0.0]]).T
    t0, dt_obs, nt = 8.8, 0.9, 6                 # 90 frames between observer times
    got = les.les_fwh(ring.data_ptr(), les.LES_FP64, nfr, nfr, xyz, nrm, area, dtau, P0, C0, obs, t0, dt_obs, nt)
    ref = fwh.pressure(frames, xyz, nrm, area, dtau, RHO0, P0, C0, obs, t0, dt_obs, nt)
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


def test_reruns_are_bit_identical_and_bad_inputs_refused():
    import torch
    xyz, nrm, area = _sphere(1.0, 12, 24)
    dtau, nfr = 0.02, 400
    ring = _ring(_frames(xyz, nfr, dtau), nfr, torch.float64)
    obs = np.array([[5.0, 1.0, 0.0]]).T
    a = les.les_fwh(ring.data_ptr(), les.LES_FP64, nfr, nfr, xyz, nrm, area, dtau, P0, C0, obs, 7.7, 0.02, 100)
    b = les.les_fwh(ring.data_ptr(), les.LES_FP64, nfr, nfr, xyz, nrm, area, dtau, P0, C0, obs, 7.7, 0.02, 100)
    np.testing.assert_array_equal(a, b)
    bad = [
        dict(t0=6.0),                          # emission times before the first frame
        dict(t0=7.7, nt=100000),               # ... after the last frame
        dict(frames=2),                        # no derivative stencil
        dict(obs=xyz[:, :1].copy()),           # an observer on a panel
    ]
    for kw in bad:
        with pytest.raises(les.LesError) as e:
            les.les_fwh(ring.data_ptr(), les.LES_FP64, nfr, kw.get("frames", nfr), xyz, nrm, area, dtau, P0, C0,
                        kw.get("obs", obs), kw.get("t0", 7.7), 0.02, kw.get("nt", 100))
        assert e.value.code == les.LES_ERR_ARG
        assert les.lib().les_last_error(None)


def test_les_probe_frames_against_the_oracle():
    """The FP32 jet's probe surface (every step) through FW-H on the GPU and
    through the oracle on the same frames."""
    import torch
    spec, fp = I.jet_small()
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(I.ambient_primitives(spec.N, fp.TR))
    xyz, nrm, area = I.cylinder_panels(3.0, 24, 20, 2.0, 10.0)
    cap, steps = 600, 660
    ring = torch.zeros((cap, 5, xyz.shape[1]), dtype=torch.float32, device="cuda")
    les.les_probe_surface(s.h, xyz, 1, ring.data_ptr(), cap)
    s.step(steps)
    nfr = les.les_probe_frames(s.h)
    dtau = s.diagnostics()["dt"]
    s.close()
    c0 = np.sqrt(1.0 / fp.TR)
    obs = I.observer_arc(25.0, 3, 6.0)
    d = obs[:, :, None] - xyz[:, None, :]
    r = np.sqrt((d * d).sum(axis=0))
    t0 = r.max() / c0 + 0.01
    nt = int(((cap - 1) * dtau + r.min() / c0 - t0) / dtau) - 1
    assert nt > 20
    got = les.les_fwh(ring.data_ptr(), les.LES_FP32, cap, nfr, xyz, nrm, area, dtau, 1.0 / 1.4, c0, obs, t0, dtau, nt)
    host = ring.double().cpu().numpy()
    first = (nfr - cap) % cap
    used = np.stack([host[(first + m) % cap] for m in range(cap)])
    ref = fwh.pressure(used, xyz, nrm, area, dtau, fp.TR, 1.0 / 1.4, c0, obs, t0, dtau, nt)
    assert np.all(np.isfinite(got))
    assert np.abs(ref).max() > 0.0
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("prec", [les.LES_FP64, les.LES_FP32])
def test_steady_uniform_stream_quadratic_term(prec):
    """A steady uniform stream through a sphere: only the quadratic
    momentum-flux term radiates, 4 pi p' = sum A rho (U.n)(U.r)/r^2, whose
    closed form is rho a^3 (3 (U.d)^2 - |d|^2 |U|^2) / (3 |d|^5); the GPU
    against the oracle and against that value."""
    import torch
    U = np.array([0.1, -0.2, 0.25])
    xyz, nrm, area = _sphere(1.0, 48, 96)
    nfr, dtau = 80, 0.05
    frames = np.empty((nfr, 5, xyz.shape[1]))
    frames[:, 0] = RHO0
    frames[:, 1:4] = U[None, :, None]
    frames[:, 4] = P0
    ring = _ring(frames, nfr, torch.float64 if prec == les.LES_FP64 else torch.float32)
    obs = np.array([[2.5, 1.0, -0.7], [0.4, -2.2, 1.9]]).T
    R = np.sqrt((obs * obs).sum(axis=0))
    t0 = (R.max() + 1.0) / C0 + 0.1          # emission times of every panel inside the 80 frames
    got = les.les_fwh(ring.data_ptr(), prec, nfr, nfr, xyz, nrm, area, dtau, P0, C0, obs, t0, dtau, 8)
    used = frames if prec == les.LES_FP64 else frames.astype(np.float32).astype(np.float64)
    ref = fwh.pressure(used, xyz, nrm, area, dtau, RHO0, P0, C0, obs, t0, dtau, 8)
    exact = RHO0 / 3.0 * (3.0 * (U @ obs) ** 2 - R ** 2 * (U @ U)) / R ** 5
    scale = np.abs(exact).max()
    assert np.abs(got - ref).max() <= 2e-5 * scale, np.abs(got - ref).max() / scale
    assert np.abs(got - exact[:, None]).max() <= 2e-4 * scale
