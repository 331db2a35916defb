"""Host logic of bench.py that needs no GPU: the parsing of the nvidia-smi
clock samples taken during the timed region (a run that saw a thermal or
hardware slowdown must say so) and the algorithmic-bytes table of the
roofline."""
import os
import tempfile

import bench


TS = "2026/12/04 06:00:00.{:03d}"


def _summary(lines, marks=()):
    clk = bench.ClockSampler(0, "test window")
    clk.marks = list(marks)
    clk.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    clk.file.write("\n".join(lines) + "\n")
    clk.proc = object()          # stands in for the finished nvidia-smi process
    out = clk.summary()
    assert not os.path.exists(clk.file.name)
    return out


def test_clock_summary_median_max_and_no_reasons():
    na = "Not Active"
    rows = [f"{TS.format(100 * k)}, 0, {mhz}, 2070, 950.0, 0x0000000000000000, {na}, {na}, {na}, {na}"
            for k, mhz in enumerate((2070, 2055, 1987, 2070, 2070))]
    out = _summary(rows)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5,
                   "window": "test window"}


def test_clock_summary_counts_the_samples_inside_the_timed_region():
    import datetime
    na = "Not Active"
    rows = [f"{TS.format(100 * k)}, 0, 2070, 2070, 950.0, 0x0, {na}, {na}, {na}, {na}" for k in range(6)]
    t = lambda ms: datetime.datetime.strptime(TS.format(ms), "%Y/%m/%d %H:%M:%S.%f").timestamp()
    out = _summary(rows, marks=(t(150), t(420)))
    assert out["samples"] == 6 and out["samples_in_timed_region"] == 3   # at 200, 300, 400 ms


def test_clock_summary_reports_every_active_reason():
    na, a = "Not Active", "Active"
    rows = [f"{TS.format(0)}, 0, 1800, 2070, 1400.0, 0x4, {na}, {na}, {na}, {a}",
            f"{TS.format(50)}, 0, 1500, 2070, 1400.0, 0x48, {a}, {na}, {a}, {na}",
            "garbage line",
            f"{TS.format(99)}, 0, [N/A], 2070, 1400.0, 0x0, {na}, {na}, {na}, {na}"]
    out = _summary(rows)
    assert out["samples"] == 2 and out["sm_mhz"] == 1650.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert _summary([])["reasons"] == ["no samples"]
    clk = bench.ClockSampler(0)
    assert clk.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_bytes_table():
    u = {"pairs": 1000, "visible": 100, "runs": 50, "evals": 0, "loaded": 10}
    hw = 1920 * 1080
    assert bench.kernel_bytes("preprocess", 200, u, hw) == 44 * 200 + 192 * 100 + 40 * 200 + 64 * 100
    assert bench.kernel_bytes("tile_scatter_rows", 200, u, hw) == 8 * 50 + 4 * 1000
    assert bench.kernel_bytes("render", 200, u, hw) == 52 * 10 + 12 * hw
    assert bench.kernel_bytes("slice", 200, u, hw) is None       # depends on the slices' sizes
    assert bench.kernel_bytes("no_such_kernel", 200, u, hw) is None


def test_oracle_frame_sample_scales_to_a_full_frame():
    # the CPU baseline / reference arm: a Gaussian sample and a tile sample of
    # one frame, each timed and scaled by its sampling factor
    from paper_2409_08669_gb300 import scenes as S
    scene = S.tiny_scene(0, n=4000)
    cam = S.look_at((0, 0, -3), width=128, height=96)
    of = bench.OracleFrame(scene, g_div=4, t_div=8, seed=1)
    assert of.sub.n == 1000
    secs = of.frame_seconds(cam, S.Settings(mode=S.MODE_AABB), key=0)
    assert 0.0 < secs < 60.0
    _, ranges, _, tile_scale = of.cache[0]
    assert tile_scale == (8 * 6) / (8 * 6 // 8)           # 48 tiles, 6 sampled
    base = bench.cpu_baseline(scene, [cam], S.Settings(mode=S.MODE_AABB), budget_s=0.0)
    assert base["kind"] == "oracle" and base["cores"] == 1 and base["value"] > 0
    ac = base["all_cores"]
    assert ac["cores"] == (os.cpu_count() or 1) and ac["value"] > 0


def test_all_cores_render_renders_every_sampled_tile_once():
    """The threads' tile subsets partition the sampled tiles: summing their
    images gives the single-threaded render of the sample."""
    import numpy as np
    import oracle
    from paper_2409_08669_gb300 import scenes as S
    scene = S.tiny_scene(2, n=3000)
    cam = S.look_at((0, 0, -3), width=96, height=80)
    st = S.Settings(mode=S.MODE_AABB)
    of = bench.OracleFrame(scene, g_div=4, t_div=2, seed=3)
    full, ranges, svals, _ = of._tile_lists(0, cam, st)
    one = oracle.render_tiled(full, ranges, svals, st)["img"]
    tiles = np.nonzero(ranges[:, 1] > ranges[:, 0])[0]
    acc = np.zeros_like(one)
    for p in np.array_split(tiles, 3):
        r = np.zeros_like(ranges)
        r[p] = ranges[p]
        acc += oracle.render_tiled(full, r, svals, st)["img"]
    np.testing.assert_array_equal(acc, one)
    assert bench.render_all_cores(of, cam, st, 0, 3) > 0.0


def test_sort_throughput_counts_what_the_kernels_move():
    kt = {"depth_pass": {"ms_per_frame": 0.1}, "tile_count_columns": {"ms_per_frame": 0.02},
          "tile_count_scan": {"ms_per_frame": 0.01}, "tile_scatter_columns": {"ms_per_frame": 0.02}}
    u = {"visible": 1_000_000, "runs_built": 500_000, "runs": 9_000_000}
    out = bench.sort_throughput(kt, u)
    assert out["depth_sort_gaussians_per_s"] == 1_000_000 / 1e-4
    assert abs(out["tile_pass1_runs_per_s"] - 500_000 / 5e-5) < 1e-3 * 1e10
    assert out["runs_built_per_frame"] == 500_000


def test_reference_arm_line_shares_the_config_and_times_its_steps(capsys, monkeypatch):
    """`--impl reference` on the tiny workload: one JSON line whose config is
    our arm's, whose ms_per_step is the wall time of a step as run (the
    bounded sample) and whose value is frames/s of full frames (each step's
    sample scaled up, so slower than the sample's own rate)."""
    import argparse
    import json
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    bench.select_workload("tiny-10k-256")
    try:
        bench.run_reference(argparse.Namespace(steps=2, warmup=3, gpus=1))
        d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
        assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["steps"] == 2
        assert d["config"] == bench.workload_config(1)
        assert abs(d["ms_per_step"] - d["sample_ms_per_step"]) < 0.5 * d["ms_per_step"] + 50.0
        assert d["scaled_ms_per_frame"] > d["sample_ms_per_step"]
        assert abs(d["value"] - 1e3 / d["scaled_ms_per_frame"]) < 1e-9 * max(1.0, d["value"])
        assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["value"] == d["value"]
    finally:
        bench.select_workload("heavy-3M-1080p")   # the module's default
