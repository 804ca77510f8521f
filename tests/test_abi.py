"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every entry point declared in include/les.h, and rejects invalid
descriptors before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2212_12365_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_12365_gb300 import build, les
    build.build()
    return les.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "les.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(les_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("les_create_grid", "les_set_state", "les_step", "les_get_state", "les_probe_surface",
              "les_get_diagnostics", "les_destroy", "les_create_batch", "les_debug_rhs"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2212_12365_gb300 import les
    syms = declared_symbols()
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(les.EXPORTED) == syms


def test_bounds_checked_build_loads_and_reports_itself(lib):
    """The debug build (-DLES_BOUNDS_CHECK) builds, exports the same entry
    points and says it checks; the normal build says it does not."""
    from paper_2212_12365_gb300 import build
    path = build.build(bounds=True)
    dbg = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(dbg, s), s
    assert dbg.les_bounds_checking() == 1
    assert lib.les_bounds_checking() == 0
    out = ctypes.c_uint64(7)
    assert lib.les_bounds_violation(None, ctypes.byref(out)) != 0  # NULL handle: LES_ERR_ARG


def test_stage_wait_bound_rejects_null_handle(lib):
    from paper_2212_12365_gb300 import les
    assert lib.les_debug_stage_wait(None, 0) == les.LES_ERR_ARG


def _desc(spec, **over):
    from paper_2212_12365_gb300 import les
    keep = []
    d = les.make_desc(spec, les.LES_FP64, keep)
    for k, v in over.items():
        if k == "face_bc":
            for f in range(6):
                d.face_bc[f] = v[f]
        elif k == "periodic":
            for a in range(3):
                d.periodic[a] = v[a]
        else:
            setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over,pover", [
    ({"ni": 3}, {}),
    ({"face_bc": (2, 3, 0, 1, 1, 1)}, {}),           # PERIODIC face on non-periodic axis
    ({"periodic": (0, 1, 0)}, {}),                    # periodic axis without PERIODIC faces
    ({"face_bc": (1, 2, 1, 1, 1, 1)}, {}),           # INFLOW_JET off the i- face
    ({}, {"mach_j": 0.0}),                            # no jet velocity at an inflow face
    ({"precision": 7}, {}),
    ({}, {"gamma": 1.0}),
    ({}, {"Re": -1.0}),
    # an FP32 grid whose five fields need offsets of 2^31 or more (checked
    # before any coordinate is read)
    ({"ni": 1024, "nj": 1024, "nk": 512, "precision": 1}, {}),
])
def test_invalid_descriptors_rejected_without_gpu(lib, over, pover):
    from paper_2212_12365_gb300 import les
    spec = I.jet_grid(8, 6, 6, 4.0, 3.0, 3.0, 0.3, 0.3)
    d, keep = _desc(spec, **over)
    fp = I.FlowParams(**pover)
    p = les.make_params(fp)
    h = ctypes.c_void_p()
    rc = lib.les_create_grid(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == les.LES_ERR_ARG
    assert not h.value


def test_workspace_size_query(lib):
    from paper_2212_12365_gb300 import les
    spec = I.jet_grid(48, 32, 32, 20.0, 10.0, 10.0, 0.125, 0.125)
    b64 = les.les_workspace_bytes(spec, les.LES_FP64)
    b32 = les.les_workspace_bytes(spec, les.LES_FP32)
    # state, metrics, scratch: at least 50 values per point
    assert b64 > 50 * 8 * spec.N and b32 > 50 * 4 * spec.N and b64 > b32


def _overlapping_polar(ni=12, nj=8, nk=16):
    """The paper's overlapping azimuthal form of the polar mesh: nk + 1 planes,
    the last at 2 pi (= the first)."""
    g = I.polar_jet_grid(ni, nj, nk, 6.0, 3.0)
    X = [c.reshape(nk, nj, ni) for c in (g.x, g.y, g.z)]
    X = [np.concatenate([c, c[:1]], axis=0) for c in X]
    return I.GridSpec(x=X[0].reshape(-1), y=X[1].reshape(-1), z=X[2].reshape(-1), dims=(ni, nj, nk + 1),
                      periodic=g.periodic, shift=g.shift, bc=g.bc), g


def test_overlapping_periodic_form_rejected_and_converted(lib):
    """A periodic axis given in the paper's overlapping form (last plane =
    first plane + period shift) is rejected before any device work, with a
    message saying so; inputs.unique_periodic_planes turns it into the mesh
    the library takes, which is the unique-plane polar mesh itself."""
    from paper_2212_12365_gb300 import les
    over, unique = _overlapping_polar()
    keep = []
    d = les.make_desc(over, les.LES_FP64, keep)
    h = ctypes.c_void_p()
    rc = lib.les_create_grid(ctypes.byref(d), ctypes.byref(les.make_params(I.FlowParams())), None, ctypes.byref(h))
    assert rc == les.LES_ERR_ARG
    assert b"overlapping" in lib.les_last_error(None)
    conv = I.unique_periodic_planes(over)
    assert conv.dims == unique.dims
    for a, b in ((conv.x, unique.x), (conv.y, unique.y), (conv.z, unique.z)):
        np.testing.assert_array_equal(a, b)
    # a translational period: the repeated plane carries the shift
    box = I.periodic_box_grid((6, 5, 4), h=(1.0, 1.0, 1.0))
    ni, nj, nk = box.dims
    X = [c.reshape(nk, nj, ni) for c in (box.x, box.y, box.z)]
    X = [np.concatenate([c, c[:, :, :1] + box.shift[0][q]], axis=2) for q, c in enumerate(X)]
    over_box = I.GridSpec(x=X[0].reshape(-1), y=X[1].reshape(-1), z=X[2].reshape(-1), dims=(ni + 1, nj, nk),
                          periodic=box.periodic, shift=box.shift, bc=box.bc)
    conv = I.unique_periodic_planes(over_box)
    assert conv.dims == box.dims
    np.testing.assert_array_equal(conv.x, box.x)
