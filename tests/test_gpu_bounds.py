"""The index-bounds-checked debug build (-DLES_BOUNDS_CHECK, the stand-in
for a memory checker): every kernel family on every kind of grid records no
out-of-range index, and the checks change no result — the FP64 states,
residuals, point fields and diagnostics are bit-identical to the normal
build's; in FP32 the extra code changes some of the compiler's
multiply-add fusions, so those agree to FP32 rounding."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()
    build.build(bounds=True)


def test_bounds_checked_build_clean_and_matches_normal_build(tmp_path):
    from paper_2212_12365_gb300 import build, les
    assert not les.les_bounds_checking()
    out = tmp_path / "checked.npz"
    env = dict(os.environ, LES_LIBRARY=build.BOUNDS_LIB)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    chk = np.load(out)
    assert int(chk["checking"][0]) == 1
    bad = {k: hex(int(chk[k][0])) for k in chk.files if k.endswith("_oob") and int(chk[k][0]) != 0}
    assert not bad, bad
    sys.path.insert(0, HERE)
    import bounds_cases
    ref = bounds_cases.run_cases()
    assert set(ref) == set(chk.files) - {"checking"}
    for k, v in ref.items():
        if k.endswith("_oob"):
            assert int(v[0]) == 0, k
            continue
        if "_0_None_" in k:  # the FP64 cases (precision code 0, no fused tiling)
            np.testing.assert_array_equal(chk[k], v, err_msg=k)
        else:
            scale = max(np.abs(v).max(), 1e-30)
            np.testing.assert_allclose(chk[k], v, rtol=1e-5, atol=1e-6 * scale, err_msg=k)
