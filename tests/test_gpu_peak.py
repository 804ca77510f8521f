"""The arithmetic-peak probe behind the FLOP rooflines (les_measure_peak):
positive, finite rates in the range GB300's units allow, FP32 far above FP64
(the FP64 units run at 1/64 of the FP32 rate), the paired FP32 FMA issuing two
results per instruction at about the scalar instruction rate, and an invalid
kind refused."""
import math

import pytest

from paper_2212_12365_gb300 import les

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()


def test_measured_peaks_are_plausible():
    import torch
    props = torch.cuda.get_device_properties(0)
    nsm = props.multi_processor_count
    # upper bounds from the unit counts at 2.2 GHz (above any boost clock):
    # 2 DFMA and 128 FFMA lanes per SM and clock, 2 FLOP each
    fp64_max = nsm * 2 * 2 * 2.2e9 / 1e12
    fp32_max = nsm * 128 * 2 * 2.2e9 / 1e12
    d = les.les_measure_peak(les.LES_PEAK_FP64_FMA)
    f = les.les_measure_peak(les.LES_PEAK_FP32_FMA)
    f2 = les.les_measure_peak(les.LES_PEAK_FP32X2_FMA)
    for v in (d, f, f2):
        assert math.isfinite(v) and v > 0.0
    assert d < fp64_max and f < fp32_max and f2 < 2 * fp32_max
    assert d > 0.3 * fp64_max and f > 0.3 * fp32_max
    assert f > 20.0 * d
    assert 0.5 * f < f2 < 2.2 * f


def test_invalid_kind_is_refused():
    with pytest.raises(les.LesError):
        les.les_measure_peak(3)
    with pytest.raises(les.LesError):
        les.les_measure_peak(-1)
