"""The bench line's roofline arithmetic (no GPU): fed the live stage times
of a 1280x720, D = 128, 8-path run on 152 SMs at 2070 MHz, it names the
path kernel, divides its algorithmic ops by its per-launch time, and puts the
result against the derived INT32 peak, the measured add and minimum rates
and, with the recorded ncu traffic, the HBM copy peak."""
import pytest

import bench
from paper_2201_11924_gb300 import configs

PEAKS = {"hbm_gbs": 6657.6, "sm_max_mhz": 2070.0}


def test_roofline_of_the_1280x720_workload():
    wl = configs.HD_720
    steps = 1000
    per_step = {"census": 0.0155, "cost": 0.0525, "paths": 0.2613, "select": 0.1771}     # ms
    r = bench.roofline_object(wl, {k: v * steps for k, v in per_step.items()}, steps, 152, PEAKS, "measured")
    assert r["kernel"] == "paths" and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    want = bench.algorithmic_ops(wl)["paths"] / 0.2613e-3 / 1e12
    assert r["achieved"] == pytest.approx(want)
    assert r["frac"] == pytest.approx(want / r["peak"])
    assert 0.55 < r["frac"] < 0.7
    pm = r["peak_measured"]
    assert pm["add_tops"] == pytest.approx(152 * 124 * 2.07e9 / 1e12)
    assert pm["min_tops"] == pytest.approx(152 * 64 * 2.07e9 / 1e12)
    assert pm["frac_of_add"] == pytest.approx(want / pm["add_tops"])
    assert r["stage_ms_per_step"]["paths"] == pytest.approx(0.2613)
    # the recorded DRAM bytes of the path kernel count only while its source
    # is the one they were captured from (else the line reports null)
    if r["traffic"] is None:
        assert "traffic_gbs" not in r
    else:
        rd, wr = bench.MEASURED_DRAM[wl.name]["paths"][:2]
        assert r["traffic"] == rd + wr
        assert r["traffic_frac_of_hbm_peak"] == pytest.approx(r["traffic"] / 0.2613e-3 / 1e9 / 6657.6)
    # the whole frame's measured DRAM bytes: the sum over the four kernels
    # when every capture matches its source
    per = r["dram_bytes_per_kernel"]
    if r["dram_bytes_per_frame"] is not None:
        assert r["dram_bytes_per_frame"] == sum(per.values())
        assert r["dram_bound_frames_per_s"] == pytest.approx(6657.6e9 / r["dram_bytes_per_frame"])
    else:
        assert any(v is None for v in per.values())


def test_roofline_without_recorded_traffic():
    wl = configs.SMALL_320                     # no ncu capture recorded for this workload
    r = bench.roofline_object(wl, {"census": 1.0, "cost": 2.0, "paths": 9.0, "select": 5.0}, 10, 152, PEAKS,
                              "measured")
    assert r["kernel"] == "paths" and r["traffic"] is None
    assert "traffic_gbs" not in r
