"""Host logic of bench.py on CPU: the DRAM-traffic figure of the bench line is
the one captured for the run's own workload, precision and fused-stage
decomposition (read from the handle's description), only while the kernel's
source file still has the hash recorded with the capture, and nothing
otherwise; the HBM denominator is labelled by where it came from."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

TUNED = " (tuned over ty {16,8} x kc {8,16,24,48,96,all,balanced,lockstep})"


def test_traffic_follows_the_decomposition_and_the_source_in_use():
    f = bench.traffic_bytes_per_point
    fused = bench.source_sha16("k_fused")
    stage = bench.source_sha16("k_iface")
    assert fused and stage and len(fused) == 16
    table = {("jet-384x256x144", "fp32", "k_fused", "ty=8 kc=lockstep"): (148.3, fused),
             ("jet-384x256x144", "fp32", "k_fused", "ty=8 kc=balanced"): (196.7, fused),
             ("jet-384x256x144", "fp32-sep", "k_fused", "ty=16 kc=lockstep"): (54.0, fused),
             ("jet-384x256x144", "fp32", "k_fused", "ty=16 kc=lockstep"): (128.1, "0" * 16),
             ("jet-384x256x144", "fp64", "k_iface", None): (938.0, stage)}

    def d32(ty, kc):
        return f"fp32 jets=1 device_bytes=1 stage=fused ty={ty} kc={kc}" + TUNED + " launches_per_step=21"

    def sep(ty, kc):
        return f"fp32 jets=1 device_bytes=1 stage=fused separable ty={ty} kc={kc} (set by the caller)"

    assert f("jet-384x256x144", "fp32", "k_fused", d32(8, "lockstep"), table) == 148.3
    assert f("jet-384x256x144", "fp32", "k_fused", d32(8, "balanced"), table) == 196.7
    assert f("jet-384x256x144", "fp32-sep", "k_fused", sep(16, "lockstep"), table) == 54.0
    # captured from another version of the kernel's source: no figure
    assert f("jet-384x256x144", "fp32", "k_fused", d32(16, "lockstep"), table) is None
    # a decomposition, workload or precision without a capture: no figure
    assert f("jet-384x256x144", "fp32", "k_fused", d32(8, 24), table) is None
    assert f("jet-768x384x192", "fp32", "k_fused", d32(8, "lockstep"), table) is None
    assert f("jet-384x256x144", "fp32", "k_fused", "fp32 stage=fused ty=8 (untuned)", table) is None
    # the FP64 stage has no decomposition
    fp64 = "fp64 jets=1 device_bytes=1 stage=point+grads+iface+update launches_per_step=36"
    assert f("jet-384x256x144", "fp64", "k_iface", fp64, table) == 938.0
    assert f("batch-64", "fp64", "k_iface", fp64, table) is None


def test_committed_traffic_figures_name_a_source_hash():
    for key, val in bench.TRAFFIC_BYTES_PER_POINT.items():
        assert len(val) == 2 and val[0] > 0 and len(val[1]) == 16, key


def test_hbm_denominator_is_labelled(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6672.2})
    v, src = bench.hbm_peak_gbs()
    assert v == 6672.2 and src.startswith("measured")
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    v, src = bench.hbm_peak_gbs()
    assert v == 6800.0 and src.startswith("fallback")


def test_flop_counts_of_the_two_forms():
    # the FP32 fused stage: the FP64 kernels' work less the 5 multiplications
    # of the J^-1 Q scaling, plus one J multiplication in the update and the
    # three 1/2 factors of the interface averages per interface (the FP64
    # kernels read them folded into the stored half interface J^-1)
    assert sum(bench.FLOPS_PER_PT_STAGE.values()) == 706
    assert bench.FLOPS_PER_PT_STAGE_FUSED == 706 - 5 + 1 + 3 * 3
    assert bench.FLOPS_PER_PT_STAGE["iface"] == 3 * 155
