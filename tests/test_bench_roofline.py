"""bench.py's roofline arithmetic for the raster kernels, on CPU with made-up
pipe rates: the SFU instruction costs follow from the measured mixed-stream
rates, the issue bound and the SFU-pipe bound are computed separately and
the larger one binds."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_sfu_slot_cost_from_mixed_streams():
    import bench
    # overlap: a stream of one ex2 per seven fma at the fma rate -> one slot;
    # one rcp per eight fma at 9/12 of the fma rate -> 9 * 4/3 - 8 = 4 slots
    w = bench.sfu_slot_cost({"ffma": 120.0, "ex2_in_ffma_stream": 120.0, "rcp_in_ffma_stream": 90.0})
    assert w["ex2"] == pytest.approx(1.0)
    assert w["rcp"] == pytest.approx(4.0)
    # a faster mixed stream than fma alone is clamped to one slot
    assert bench.sfu_slot_cost({"ffma": 100.0, "ex2_in_ffma_stream": 110.0, "rcp_in_ffma_stream": 100.0})["ex2"] == 1.0
    # no measurement: the SFU's lane count (16 of 128)
    assert bench.sfu_slot_cost(None) == {"ex2": 8.0, "rcp": 8.0}


def test_raster_roofline_bounds():
    import bench
    rates = {"ffma": 128.0, "ex2": 32.0, "rcp": 16.0, "ex2_in_ffma_stream": 128.0, "rcp_in_ffma_stream": 128.0}
    sms, mhz = 100, 1000.0
    pairs = (10 ** 10, 10 ** 10)
    # intensity pass: 10 fp32 + 1 ex2 (1 slot) = 11 slots per pair; at 100 % of
    # 100 x 128 x 1e9 slots/s the launch takes 10^10 x 11 / 1.28e13 s
    t_issue_ms = pairs[0] * 11 / (sms * 128 * mhz * 1e6) * 1e3
    out = bench.raster_roofline({"intensity_fwd": 2 * t_issue_ms}, pairs, sms, mhz, rates)
    k = out["k_intensity_fwd"]
    assert k["slots_per_pair"] == pytest.approx(11.0)
    assert k["frac_issue"] == pytest.approx(0.5, rel=1e-3)
    # SFU pipe: one ex2 per pair at 32 per SM cycle
    t_sfu_ms = pairs[0] / (sms * 32 * mhz * 1e6) * 1e3
    assert k["frac_sfu_pipe"] == pytest.approx(t_sfu_ms / (2 * t_issue_ms), rel=1e-3)
    assert k["binds"] == "issue" and k["frac"] == k["frac_issue"]
    # a kernel whose SFU pipe bound exceeds its issue bound reports that one
    slow_sfu = dict(rates, ex2=1.0)
    k2 = bench.raster_roofline({"splat_fwd": 1000.0}, pairs, sms, mhz, slow_sfu)["k_splat_fwd"]
    assert k2["binds"] == "sfu" and k2["frac"] == k2["frac_sfu_pipe"] > k2["frac_issue"]
    # kernels without a time are left out
    assert set(bench.raster_roofline({"intensity_bwd": 0.0}, pairs, sms, mhz, rates)) == set()
