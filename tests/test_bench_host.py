"""Host logic of bench.py (no GPU): the roofline arithmetic on a recorded
kernel class, the bound of each class, the recorded-traffic lookup keyed by
the sources of the kernel's class, and the peak table."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6779.0, "bf16_tflops": 1864.0, "sm_max_mhz": 2070.0}


def test_peak_table():
    tab = bench.peak_table(PEAKS, "measured", sms=152)
    assert tab["hbm"][0] == 6779.0
    assert tab["alu"][0] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert tab["tensor"][0] == pytest.approx(1864.0 / 2 / 3)
    # the SM count is the device's (the nominal 152 without one)
    assert bench.peak_table(PEAKS, "measured", sms=76)["alu"][0] == pytest.approx(
        tab["alu"][0] / 2)
    assert bench.sm_count(default=152) > 0


def test_bounds_of_the_kernel_classes():
    k = {"ms": 1.0, "launches": 1, "bytes": 1e9, "flops": 1e10}
    assert bench.bound_of("col_conv", k, True) == "hbm"
    assert bench.bound_of("row_fwd_iter", dict(k, flops=0.0), True) == "hbm"
    assert bench.bound_of("contract_pixels", k, True) == "tensor"
    assert bench.bound_of("contract_pixels", k, False) == "alu"


def test_roofline_of_the_column_pass_uses_the_recorded_traffic(tmp_path, monkeypatch):
    # 24 launches, 0.588 ms each, the algorithmic bytes and flops of a
    # thyroid256 column pass (all 768 right-hand sides in each launch)
    k = {"ms": 24 * 0.588, "launches": 24, "bytes": 24 * 1150637397.33,
         "flops": 24 * 13656653824.0}
    rec = {"records": [{"kernel": "col_conv", "workload": "thyroid256",
                        "dram_bytes": 475181568, "algorithmic_bytes": 539000832,
                        "src": bench.kernel_source_hash("col_conv")},
                       {"kernel": "col_conv", "workload": "large512",
                        "dram_bytes": 1.0, "algorithmic_bytes": 1.0, "src": "stale"}]}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(path))
    r = bench.roofline("col_conv", k, PEAKS, "measured", "thyroid256", True)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1150637397.33 / 0.588e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6779.0)
    assert r["fft_tflops_nominal"] == pytest.approx(13656653824.0 / 0.588e-3 / 1e12)
    dram, alg = bench.recorded_traffic("col_conv", "thyroid256")
    assert (dram, alg) == (475181568, 539000832)
    assert r["traffic"] == pytest.approx(dram * 1150637397.33 / alg)
    assert r["traffic_over_algorithmic"] == pytest.approx(dram / alg)
    # a record of changed sources, another workload or class: none
    assert bench.recorded_traffic("col_conv", "large512") is None
    assert bench.recorded_traffic("col_conv", "volume3d") is None
    assert bench.roofline("row_inv_t", dict(k, flops=0.0), PEAKS, "measured", "thyroid256",
                          True)["traffic"] is None


def test_committed_traffic_records_are_well_formed():
    if not os.path.exists(bench.TRAFFIC_PATH):
        pytest.skip("no traffic record")
    with open(bench.TRAFFIC_PATH) as f:
        recs = json.load(f)["records"]
    for r in recs:
        assert {"kernel", "workload", "dram_bytes", "algorithmic_bytes", "src"} <= set(r)
        assert r["dram_bytes"] > 0 and r["algorithmic_bytes"] > 0


def test_source_hash_is_per_kernel_class():
    assert bench.kernel_source_hash("col_conv") == bench.kernel_source_hash("row_fwd_s")
    assert bench.kernel_source_hash("col_conv") != bench.kernel_source_hash("contract_pixels")
