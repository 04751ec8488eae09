"""Host-side logic of bench.py (no GPU): the algorithmic byte model of the
five passes, the kernel each pass runs, and when ncu traffic is reported."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_byte_model_at_n512():
    """n = 512, L = 1024: T1 = n^2 L = 2N and T2 = n L^2 = 4N complex64 values.
    One B-form matvec: X fwd reads x, S and writes T1 (4N), Y fwd 6N, Z 8N plus
    the (L/2+1)^3 spectrum entries, Y inv 6N, X inv reads T1, x, S and writes y
    (5N): 29N + spectrum, 32.2 GB.  One COCG iteration: the X fwd prologue also
    reads r and writes p (6N), the X inv epilogue reads p (5N), the update moves
    6N: 37N + spectrum, 40.8 GB."""
    n, L, cb = 512, 1024, 8
    N, H3 = n ** 3, (L // 2 + 1) ** 3
    assert bench.matvec_alg_bytes(n, L, cb) == (29 * N + H3) * cb
    assert abs(bench.matvec_alg_bytes(n, L, cb) / 1e9 - 32.2) < 0.05
    it = sum(bench.alg_bytes(k, n, L, cb) for k in ("xfwd", "yfwd", "zconv", "yinv", "xinv", "update"))
    assert it == (37 * N + H3) * cb
    assert abs(it / 1e9 - 40.8) < 0.05
    assert abs(bench.alg_bytes("zconv", n, L, cb) / 1e9 - 9.67) < 0.01


def test_kernel_names_follow_length_and_schedule():
    pers = {"yfwd": 0, "zconv": 0, "yinv": 0}
    tiles = {"yfwd": 1, "zconv": 1, "yinv": 1}
    assert bench.fp32_kernel_name("zconv", 1024, pers) == "k_zconv_pipe<float, 1024, 16, 32>"
    assert bench.fp32_kernel_name("zconv", 1024, dict(pers, zconv_variant=1)) == "k_zconv_pipe<float, 1024, 8, 32>"
    assert bench.fp32_kernel_name("zconv", 1024, dict(pers, zconv_variant=2)) == "k_zconv_pipe<float, 1024, 16, 64>"
    assert bench.fp32_kernel_name("yfwd", 512, dict(pers, yfwd_variant=2)) == "k_yfwd_pipe<float, 512, 16, 64>"
    assert bench.fp32_kernel_name("yinv", 256, dict(pers, yinv_variant=1)) == "k_yinv_pipe<256, 8, 16>"
    assert bench.fp32_kernel_name("zconv", 128, dict(pers, zconv_variant=2)) == "k_zconv_pipe<float, 128, 16, 16>"
    assert bench.fp32_kernel_name("zconv", 1024, tiles) == "k_strided<float, 1024>(ZCONV)"
    assert bench.fp32_kernel_name("zconv", 2048, pers) == "k_zconv_pipe<float, 2048, 8, 64>"
    assert bench.fp32_kernel_name("zconv", 2048, tiles) == "k_zconv_smem<float, 2048, 8>"
    assert bench.fp32_kernel_name("yinv", 2048, pers) == "k_yinv_pipe<2048, 8, 64>"
    assert bench.fp32_kernel_name("yfwd", 2048, tiles) == "k_strided_smem<float, 2048, 4>(FWD)"
    # the X passes have one kernel per length whatever the schedule
    assert bench.fp32_kernel_name("xfwd", 2048, pers) == bench.fp32_kernel_name("xfwd", 2048, tiles)
    assert bench.fp32_kernel_name("xinv", 2048, pers) == "k_xinv_pipe<2048, 4>"
    assert bench.fp32_kernel_name("update", 1024, pers) == "k_cocg_update<float>"


def _write_traffic(tmp_path, monkeypatch, source_hash, n):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({
        "source_hash": source_hash,
        "kernels": {"zconv": {"0": {"n": n, "dram_bytes_per_launch": 1.0e10},
                              "2": {"n": n, "dram_bytes_per_launch": 1.1e10}}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))


def test_traffic_reported_only_for_current_sources_and_same_grid(tmp_path, monkeypatch):
    current = bench.source_hash()                    # of the real kernel sources
    monkeypatch.setattr(bench, "source_hash", lambda: current)
    _write_traffic(tmp_path, monkeypatch, current, 512)
    assert bench.traffic_from_profiles("zconv", 512) == 1.0e10
    assert bench.traffic_from_profiles("zconv", 512, 2) == 1.1e10  # another launch variant
    assert bench.traffic_from_profiles("zconv", 512, 1) is None    # not captured
    assert bench.traffic_from_profiles("zconv", 1000) is None     # another L, other kernels
    assert bench.traffic_from_profiles("xfwd", 512) is None       # not captured


def test_traffic_dropped_once_sources_change(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "source_hash", lambda: "0123456789abcdef")
    _write_traffic(tmp_path, monkeypatch, "fedcba9876543210", 512)
    assert bench.traffic_from_profiles("zconv", 512) is None


def test_committed_traffic_agrees_with_the_byte_model():
    """profiles/traffic.json, while it belongs to the kernel sources in the tree:
    every captured kernel moves between 0.9 and 1.3 times its algorithmic bytes
    (less would mean the model counts bytes the kernels never move, more that
    they re-read).  After a kernel change bench.py reports the traffic as null
    until the next capture; this check then has nothing to look at."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        pytest.skip("no committed traffic capture")
    with open(path) as f:
        d = json.load(f)
    if d["source_hash"] != bench.source_hash():
        pytest.skip("kernel sources changed since the committed capture (bench reports traffic null)")
    for kind in ("xfwd", "yfwd", "zconv", "yinv", "xinv", "update"):
        for variant, ent in d["kernels"][kind].items():
            ratio = ent["dram_bytes_per_launch"] / bench.alg_bytes(kind, ent["n"], 2 * ent["n"], 8)
            assert 0.9 < ratio < 1.3, (kind, variant, ratio)


def test_committed_bench_line_keeps_the_output_contract():
    """The committed n = 512 bench line carries every key of the output
    contract, and its derived figures agree with their inputs."""
    path = os.path.join(ROOT, "profiles", "bench_solve_n512_latest.json")
    with open(path) as f:
        d = json.loads(f.readline())
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["metric"] == bench.METRIC and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["warmup"] >= 3 and d["n_gpus"] == 1 and "workload" in d["config"]
    assert abs(d["ms_per_step"] / 1e3 - d["value"]) < 1e-9 * d["value"]
    roof = d["roofline"]
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-12
    assert abs(roof["achieved"] - roof["alg_bytes_per_launch"] / (roof["ms_per_launch"] * 1e-3) / 1e9) < 1e-6 * roof["achieved"]
    # the peak is the measured copy bandwidth of the box the line ran on; the
    # measurement is repeated on each fresh box, so it may differ by a few per cent
    assert roof["peak_source"].startswith("measured")
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        with open(peaks) as f:
            assert abs(roof["peak"] / float(json.load(f)["hbm_gbs"]) - 1.0) < 0.1
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["sample"]
    e2e = d["e2e"]
    assert e2e["unit"] == d["unit"] and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert e2e["value"] > d["value"]                   # the copies are inside its timed region
    assert d["gpu_launches"] > 0
    assert not set(d["clocks"]["reasons"]) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
