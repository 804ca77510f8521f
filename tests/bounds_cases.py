"""Cases run through the index-bounds-checked debug build (and, for the
bit comparison, through the normal build): every kind of grid and every
kernel family — FP64 four-kernel stage, FP32 fused stage at several tilings
and in its separable form, periodic and mixed axes, the polar mesh with its
centerline, a batch, the surface probe, diagnostics, residual and point-field
exports.  Which library is used is decided by the binding (LES_LIBRARY).

Run as a script: python tests/bounds_cases.py OUT.npz — saves every case's
raw state and export plus the violation word of each handle."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2212_12365_gb300 import inputs as I  # noqa: E402
from paper_2212_12365_gb300 import les  # noqa: E402


def _mixed_periodic():
    g = I.jet_grid(21, 17, 12, 6.0, 5.0, 4.0, 0.2, 4.0 / 11)
    ni, nj, _ = g.dims
    g.z = np.repeat(np.arange(12) * (4.0 / 12), ni * nj)
    g.periodic = (0, 0, 1)
    g.shift = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 4.0]], dtype=float)
    g.bc = (2, 3, 1, 1, 0, 0)
    return g


GRIDS = {
    "wavy_periodic": lambda: (I.wavy_periodic_grid((13, 11, 9), amp=0.2), I.FlowParams(Re=300.0)),
    "wavy_box": lambda: (I.wavy_box_grid((14, 11, 9), amp=0.06, bc=(1, 3, 1, 1, 1, 1)), I.FlowParams(Re=500.0)),
    "jet_ragged": lambda: (I.jet_grid(37, 23, 19, 8.0, 6.0, 6.0, 0.15, 0.18), I.FlowParams(Re=1e4)),
    "mixed_periodic_z": lambda: (_mixed_periodic(), I.FlowParams(Re=2e3)),
    "tiny_4x4x4": lambda: (I.wavy_box_grid((4, 4, 4), amp=0.02), I.FlowParams(Re=100.0)),
    "polar": lambda: (I.polar_jet_grid(20, 10, 16, 6.0, 3.0), I.FlowParams(Re=1e4)),
    # more tiles than CTAs: the lockstep form runs whole-column waves first
    "wide": lambda: (I.jet_grid(400, 160, 12, 20.0, 10.0, 10.0, 0.125, 0.1), I.FlowParams(Re=1e4)),
}

# (grid, precision, tiling or None)
CASES = [
    ("wavy_periodic", les.LES_FP64, None), ("wavy_periodic", les.LES_FP32, (8, 4)),
    ("wavy_box", les.LES_FP64, None), ("wavy_box", les.LES_FP32, (16, 100000)),
    ("jet_ragged", les.LES_FP64, None), ("jet_ragged", les.LES_FP32, (8, 5)),
    ("jet_ragged", les.LES_FP32, (16, 0)), ("jet_ragged", les.LES_FP32_SEPARABLE, (8, 100000)),
    ("mixed_periodic_z", les.LES_FP32, (8, 0)), ("mixed_periodic_z", les.LES_FP64, None),
    ("tiny_4x4x4", les.LES_FP64, None), ("tiny_4x4x4", les.LES_FP32, (8, 1)),
    ("polar", les.LES_FP64, None), ("polar", les.LES_FP32, (8, 100000)),
    ("wide", les.LES_FP32, (8, -1)), ("wide", les.LES_FP32_SEPARABLE, (16, -1)),
]


def run_cases() -> dict:
    import torch
    out = {}
    for name, prec, tiling in CASES:
        spec, fp = GRIDS[name]()
        s = les.Solver(spec, fp, prec)
        if tiling:
            les.les_set_fused_tiling(s.h, *tiling)
        s.set_state(I.smooth_random_primitives(spec, 5, amp=0.06))
        s.step(2)
        key = f"{name}_{prec}_{tiling}"
        out[key + "_raw"] = s.get_state(les.LES_STATE_RAW)
        out[key + "_rhs"] = s.rhs()
        out[key + "_p"] = s.field(les.LES_FIELD_P)
        out[key + "_musgs"] = s.field(les.LES_FIELD_MU_SGS)
        d = s.diagnostics(check=False)
        out[key + "_diag"] = np.concatenate([[d["max_abs_rhs_rho"]], d["l2_rhs"], d["sum_qhat"]])
        out[key + "_oob"] = np.array([les.les_bounds_violation(s.h)], dtype=np.uint64)
        s.close()
    # a batch of uneven jets in one persistent launch, FP32
    jets = I.batch_jets(3, seed=12)
    b = les.Solver([g for g, _ in jets], [f for _, f in jets], les.LES_FP32)
    for j, (g, f) in enumerate(jets):
        b.set_state(I.ambient_primitives(g.N, f.TR), jet=j)
    b.step(3)
    for j in range(3):
        out[f"batch_{j}_raw"] = b.get_state(les.LES_STATE_RAW, jet=j)
    out["batch_oob"] = np.array([les.les_bounds_violation(b.h)], dtype=np.uint64)
    b.close()
    # the surface probe on a jet, every step
    spec, fp = I.jet_small()
    xyz = I.cylinder_points(1.5, 16, 24, 0.5, spec.x.max() - 0.5)
    dev = torch.zeros((4, 5, xyz.shape[1]), dtype=torch.float32, device="cuda")
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(I.ambient_primitives(spec.N, fp.TR))
    les.les_probe_surface(s.h, xyz, 1, dev.data_ptr(), 4)
    s.step(3)
    torch.cuda.synchronize()
    out["probe_frames"] = dev.double().cpu().numpy()
    out["probe_oob"] = np.array([les.les_bounds_violation(s.h)], dtype=np.uint64)
    s.close()
    return out


if __name__ == "__main__":
    res = run_cases()
    res["checking"] = np.array([int(les.les_bounds_checking())])
    np.savez(sys.argv[1], **res)
    print("cases", len(CASES), "checking", int(les.les_bounds_checking()))
