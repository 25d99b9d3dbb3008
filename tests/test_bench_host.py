"""Host-side arithmetic of bench.py: the ALU roofline of the kernel product and the
source gate of the recorded DRAM traffic (no GPU)."""
import pytest

import bench


def test_pair_roofline_from_unit_rates():
    # Matern-5/2 at d = 4: 1/16 + 1/32 MUFU clocks per pair (sqrt, ex2) -> 10.67 pairs/clk/SM,
    # below the FP32 bound (11 ops per pair); 152 SMs at 2070 MHz
    assert bench.pair_peak_gps("matern52", 4) == pytest.approx(152 * (32 / 3) * 2.07, rel=1e-3)
    assert bench.pair_peak_gps("matern52", 4) == pytest.approx(3356, abs=1)
    # RBF at d = 2: ex2 alone is 32 per clock and 4 FP32 ops per pair do not bind
    assert bench.pair_peak_gps("rbf", 2) == pytest.approx(152 * 32 * 2.07, rel=1e-3)
    # large d: the FP32 pipes bind (2 d + 3 ops per pair for Matern)
    assert bench.pair_peak_gps("matern52", 16) < bench.pair_peak_gps("matern52", 4)


def test_traffic_is_reported_only_for_the_sources_it_was_measured_on():
    import hashlib
    import os
    rel = "paper_2405_03474_gb300/csrc/kz_sym.cu"
    with open(os.path.join(bench.ROOT, rel), "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()[:16]
    assert bench.measured_traffic({"bytes": 1.5e9, "sources": {rel: digest}}) == 1.5e9
    assert bench.measured_traffic({"bytes": 1.5e9, "sources": {rel: "0" * 16}}) is None
    # the kernel, its device helpers, and the point order that decides which points share a tile
    assert set(bench.KZ_SYM_TRAFFIC["sources"]) == {rel, "paper_2405_03474_gb300/csrc/tc_common.cuh",
                                                    "paper_2405_03474_gb300/csrc/point_order.cu"}
