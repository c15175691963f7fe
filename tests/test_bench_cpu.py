"""Host arithmetic of bench.py's roofline objects (no GPU): achieved bytes per second from the
library's counters and the launch time, the fraction of the peak, and the texel-writeback
figure beside it (32 B of texels per FP32 sample, 16 B per 16-bit sample)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(frames=4, samples=4_000_000_000, brick_bytes=40_000_000_000, fragments=50_000_000,
           ms_raycast=12.0):
    return {"timed_frames": frames, "samples": samples, "brick_bytes_sampled": brick_bytes,
            "fragments": fragments, "ms_raycast": ms_raycast}


def test_roofline_divides_algorithmic_bytes_by_the_launch_time():
    st = _stats()
    r = bench.roofline(st, 4, 6800.0, "measured", "k_raycast<test>")
    per_launch = (40e9 + 16 * 50e6) / 4                 # bricks' stored bytes + 16 B fragments
    launch_s = 12.0 / 4 * 1e-3
    assert r["algorithmic_bytes_per_launch"] == int(per_launch)
    assert r["launch_ms"] == pytest.approx(3.0)
    assert r["achieved"] == pytest.approx(per_launch / launch_s / 1e9, rel=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0, rel=1e-3)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0


def test_mip_fragments_count_four_bytes():
    st = _stats()
    r16 = bench.roofline(st, 4, 6800.0, "measured", "k", 32, 16)
    r4 = bench.roofline(st, 4, 6800.0, "measured", "k", 32, 4)
    assert r16["algorithmic_bytes_per_launch"] - r4["algorithmic_bytes_per_launch"] == 12 * 50_000_000 // 4


def test_texel_writeback_counts_the_texel_size():
    st = _stats()
    if bench.traffic_entry("l1tex_texel_writeback_peak_gbs") is None:
        pytest.skip("no texel-writeback peak recorded")
    f32 = bench.roofline(st, 4, 6800.0, "measured", "k", 32)["l1tex"]
    f16 = bench.roofline(st, 4, 6800.0, "measured", "k", 16)["l1tex"]
    assert f32["achieved"] == pytest.approx(32 * 1e9 / 3e-3 / 1e9, rel=1e-4)   # 1e9 samples per launch
    assert f16["achieved"] == pytest.approx(f32["achieved"] / 2, rel=1e-4)
    assert f16["frac"] == pytest.approx(f32["frac"] / 2, rel=1e-3)


def test_recorded_traffic_names_a_kernel_source():
    """Every traffic record names the ray-cast source it was captured on (the bench reports
    `traffic` only while that source is unchanged)."""
    for name in ("k_raycast<f32,DVR>", "k_raycast<f16,DVR>"):
        e = bench.traffic_entry(name)
        assert e is not None and len(e["source_sha"]) == 16 and e["dram_bytes_per_launch"] > 0
