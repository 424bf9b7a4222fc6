"""The benchmark's host logic on CPU: the ray-cast counters of the committed
ncu summary are used only while the hash of the ray-cast sources matches and
only for a warp tile they were taken for."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def profile_values():
    kv = {}
    for line in open(os.path.join(ROOT, "profiles", "k_trace_dram.txt")):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    return kv


def test_counters_gated_by_source_hash_and_tile(monkeypatch):
    kv = profile_values()
    sha = kv["ray_cast_sources_sha256_16"]
    monkeypatch.setattr(bench, "ray_cast_sources_sha", lambda: sha)
    got = bench.traffic_from_profile(4, 8)
    assert got == {"dram": float(kv["tb4_occ8_dram_bytes_per_frame"]), "l2": float(kv["tb4_occ8_l2_bytes_per_frame"])}
    # per frame = (read + write) / frames per launch, as recorded
    n = int(kv["frames_per_launch"])
    assert abs(got["dram"] - (int(kv["tb4_occ8_dram_bytes_read"]) + int(kv["tb4_occ8_dram_bytes_write"])) / n) <= 1
    assert bench.traffic_from_profile(1, 8) is None          # a tile the counters were not taken for
    assert bench.traffic_from_profile(4, 0) is None          # the other register variant
    monkeypatch.setattr(bench, "ray_cast_sources_sha", lambda: "0" * 16)
    assert bench.traffic_from_profile(4, 8) is None          # the kernel changed since


def test_source_hash_covers_the_ray_cast_sources():
    assert all(os.path.exists(os.path.join(ROOT, p)) for p in bench.RAY_CAST_SOURCES)
    assert any(p.endswith("trace.cu") for p in bench.RAY_CAST_SOURCES)
    assert len(bench.ray_cast_sources_sha()) == 16


def test_config_names_the_workload_and_the_cast_bound():
    full = bench.arm_config(64, 32768, 1)
    small = bench.arm_config(8, 32768, 1, small=True)
    assert full["workload"] == bench.WORKLOAD and "2,100,512 tris" in full["workload"]
    assert small["workload"] == bench.SMALL_WORKLOAD and "527,648 tris" in small["workload"]
    assert "r_max" in full["cast"] and full["frames_per_step"] == 64 and full["parallelism"] == "dp1"
