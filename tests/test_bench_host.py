"""Host logic of bench.py on CPU: the DRAM-traffic figure of the bench line is
the one captured for the run's own workload, precision and fused-stage
decomposition (read from the handle's description), and nothing otherwise."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

TUNED = " (tuned over ty {16,8} x kc {8,16,24,48,96,all,balanced,lockstep})"


def test_traffic_follows_the_decomposition_in_use():
    f = bench.traffic_bytes_per_point
    def d32(ty, kc):
        return f"fp32 jets=1 device_bytes=1 stage=fused ty={ty} kc={kc}" + TUNED + " launches_per_step=21"

    def sep(ty, kc):
        return f"fp32 jets=1 device_bytes=1 stage=fused separable ty={ty} kc={kc} (set by the caller)"

    assert f("jet-384x256x144", "fp32", "k_fused", d32(8, "lockstep")) == 148.3
    assert f("jet-384x256x144", "fp32", "k_fused", d32(8, "balanced")) == 196.7
    assert f("jet-384x256x144", "fp32-sep", "k_fused", sep(16, "lockstep")) == 54.0
    # a decomposition, workload or precision without a capture: no figure
    assert f("jet-384x256x144", "fp32", "k_fused", d32(8, 24)) is None
    assert f("jet-768x384x192", "fp32", "k_fused", d32(8, "lockstep")) is None
    assert f("jet-384x256x144", "fp32", "k_fused", "fp32 stage=fused ty=8 (untuned)") is None
    # the FP64 stage has no decomposition
    fp64 = "fp64 jets=1 device_bytes=1 stage=point+grads+iface+update launches_per_step=36"
    assert f("jet-384x256x144", "fp64", "k_iface", fp64) == 938.0
    assert f("batch-64", "fp64", "k_iface", fp64) is None
