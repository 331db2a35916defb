"""Benchmark of the AdR-Gaussian rasterization path on GB300.

Workload (the headline metric: FPS at 1920x1080 with 3M Gaussians, AdR vs the
plain 3DGS-style path): the heavy-load synthetic scene (3M Gaussians, 30% in
one dense central cluster, the rest in 64 anisotropic clusters plus a uniform
background; SH degree 3, fp32), rendered from 50 cameras on a circle of
radius 4.  One step = one frame = Preprocess + scan + emission, the tile
sort + ranges, and Render (every stage of the forward path) for the next
camera in the cycle.  The scene (708 MB) and the per-frame working set are
larger than the 129 MB L2, so no explicit L2 flush is used.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 restatement of the
paper) on the host cores, on a bounded sample of the same workload.
Under torchrun (N > 1) every rank renders its own cameras (replicas: the
frames are independent), the timed region is bracketed by barriers and the
slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2409_08669_gb300 import scenes as S  # noqa: E402

METRIC = "FPS @1080p, 3M Gaussians, AdR vs plain 3DGS path on 1 GB300; serving p50/p99 ms"
# name -> (scene builder, gaussians, width, height, pair capacity)
WORKLOADS = {
    "tiny-10k-256": ("tiny", 10_000, 256, 256, 1 << 22),
    "heavy-3M-1080p": ("heavy", 3_000_000, 1920, 1080, 1 << 29),
    "heavy-3M-4k": ("heavy", 3_000_000, 3840, 2160, 1 << 30),
    "cluster-1M-1080p": ("cluster", 1_000_000, 1920, 1080, 1 << 27),
    "heavy-600k-1080p": ("heavy", 600_000, 1920, 1080, 1 << 26),
}
WORKLOAD = "heavy-3M-1080p"
N_GAUSS = 3_000_000
WIDTH, HEIGHT = 1920, 1080
N_CAMERAS = 50
PAIR_CAPACITY = 1 << 29


def select_workload(name):
    global WORKLOAD, N_GAUSS, WIDTH, HEIGHT, PAIR_CAPACITY
    kind, n, w, h, cap = WORKLOADS[name]
    WORKLOAD, N_GAUSS, WIDTH, HEIGHT, PAIR_CAPACITY = name, n, w, h, cap
    return kind
EVAL_FP32_OPS = 15        # FP32 lane operations per Gaussian-pixel evaluation in Render
# Kernels of one forward frame: frame parameters 1, preprocess 1, depth sort
# 4 x (count, count scan, scatter) 12, run scan + pair total 2, slice-0 setup 1,
# tile pass 1 (count, count scan, scatter) 3, render slice 0 1,
# unfinished-tile table (rows, columns) + compaction (count, scan, scatter) 5,
# tile pass 1 of slice 1 3, render slice 1 1 (each render derives its column ranges).
KERNELS_PER_FRAME = 30
# DRAM bytes (read + write) of one launch from one-pass ncu captures at the
# heavy 3M-Gaussian 1080p frame: Render (profiles/render_heavy-3M-1080p_traffic.md,
# its two launches of one frame, 54.8 MB) and the per-tile list pass
# (profiles/tile_scatter_rows_heavy-3M-1080p_traffic.md, 128.34 + 576.92 MB over
# P = 1.5958e8 pairs, scaled by the measured P).
TRAFFIC_BYTES_PER_FRAME = {"render": (10479616 + 8927232) + (35350528 + 17920)}
TRAFFIC_BYTES_PER_PAIR = {"tile_scatter_rows": (128.34e6 + 576.92e6) / 1.5958e8}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples, every ~50 ms (the first arrives ~10 ms
    after start).  The sampler starts before the warm-up frames and waits (up
    to 2 s) for its first sample; `mark()` brackets the timed region, whose own
    samples are counted separately (a 20-frame region lasts ~20 ms, so it holds
    one at most; the window around it runs the same frames)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0, window="warm-up and timed frames"):
        self.gpu = gpu_index
        self.proc = None
        self.file = None
        self.window = window
        self.marks = []

    def mark(self):
        self.marks.append(time.time())

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 2.0 and os.path.getsize(self.file.name) == 0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = parse_clock_rows(open(self.file.name).read().splitlines())
        os.unlink(self.file.name)
        return summarise_clocks(rows, self.marks, self.window)


def parse_clock_rows(lines):
    """(epoch seconds or None, sm MHz, max sm MHz, [hw, hw_thermal, sw_thermal,
    sw_power_cap] flags) per nvidia-smi line of ClockSampler.FIELDS."""
    import datetime
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        try:
            rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
        except ValueError:
            continue
    return rows


def summarise_clocks(rows, marks=(), window=""):
    """Median SM clock, max clock, active throttle reasons and sample counts
    (all samples of the window, and those inside the first two marks)."""
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for _, _, _, r in rows for i, v in enumerate(r) if v == "Active"})
    out = {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
           "reasons": reasons, "samples": len(rows), "window": window}
    if len(marks) >= 2:
        out["samples_in_timed_region"] = sum(1 for r in rows if r[0] is not None and
                                             marks[0] <= r[0] <= marks[1])
    return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, device_sync=True):
    import torch
    if device_sync and torch.cuda.is_available():
        torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value):
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def deal_cameras(cams, rank):
    """Replica `rank` starts its camera cycle at camera `rank` (replicas render
    different frames of the same orbit)."""
    k = rank % len(cams)
    return cams[k:] + cams[:k]


def aggregate_fps(pg, local_seconds, steps, world):
    """Whole-job frames/s: the frames of all replicas over the slowest
    replica's time (max over ranks)."""
    t = max_over_ranks(pg, local_seconds)
    return steps * world / t, t


def build_workload(rank=0):
    """The workload's scene and its 50 orbit cameras (radius 4; the tiny scene,
    10k Gaussians in [-1, 1]^3, is seen from distance 3)."""
    kind = WORKLOADS[WORKLOAD][0]
    if kind == "heavy":
        scene = S.heavy_scene(n=N_GAUSS, seed=2)
    elif kind == "tiny":
        scene = S.tiny_scene(0, n=N_GAUSS)
    else:
        scene = S.cluster_scene(n=N_GAUSS, seed=1)
    cams = S.orbit_cameras(N_CAMERAS, radius=3.0 if kind == "tiny" else 4.0, width=WIDTH, height=HEIGHT)
    return scene, deal_cameras(cams, rank)


# ---------------------------------------------------------------------------
# Our arm: the CUDA path through the C ABI
# ---------------------------------------------------------------------------

L2_BYTES = 129 * 1024 * 1024


def workload_config(world):
    """The `config` object of both arms' JSON lines."""
    return {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT,
            "cameras": N_CAMERAS, "mode": "adr_aabb", "sh_degree": 3,
            "parallelism": f"replicas x{world}",
            "l2": (f"inputs smaller than L2 ({N_GAUSS * 236 / 1e6:.1f} MB scene): a 256 MB "
                   "buffer is written before every timed frame, which is timed on its own"
                   if scene_fits_l2() else
                   f"inputs larger than L2 ({N_GAUSS * 236 / 1e6:.0f} MB scene, "
                   f"{N_GAUSS * 48 / 1e6:.0f} MB render records); no flush")}


def scene_fits_l2():
    """Whether the workload's inputs fit the 129 MB L2 (then every timed frame
    starts after an L2 flush)."""
    return N_GAUSS * 236 <= L2_BYTES


def time_mode(rast, params, cams, st, steps, warmup, stream, pg=None, with_stages=True,
              kernel_times=False, clock=None):
    """Returns (seconds for `steps` frames, per-stage ms lists, per-kernel times).

    With kernel_times the library records CUDA events around each of its kernel
    launches on `stream` during the timed frames (adr_profile_enable).  When
    the inputs fit in L2, a 256 MB buffer is written before every timed frame
    (an L2 flush) and the time is the sum of the frames' own event intervals."""
    import torch
    if scene_fits_l2():
        return time_mode_flushed(rast, params, cams, st, steps, warmup, stream, pg, with_stages,
                                 kernel_times, clock)
    for k in range(warmup):
        rast.forward(params, cams[k % len(cams)], st, stream=stream, want_aux=False)
    barrier(pg)
    if kernel_times:
        rast.profile(True)
        rast.profile_read()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device="cuda")
    if clock is not None:
        clock.mark()
    start.record(stream)
    for k in range(steps):
        cam = cams[(warmup + k) % len(cams)]
        if with_stages:
            ev[k][0].record(stream)
        rast.preprocess(params, cam, st, stream=stream)
        if with_stages:
            ev[k][1].record(stream)
        rast.sort(stream=stream)
        if with_stages:
            ev[k][2].record(stream)
        rast.render(img=img, stream=stream, want_aux=False)
        if with_stages:
            ev[k][3].record(stream)
    stop.record(stream)
    barrier(pg)
    if clock is not None:
        clock.mark()
    total = start.elapsed_time(stop) / 1e3
    stages = None
    if with_stages:
        stages = {"preprocess_scan_emit": [e[0].elapsed_time(e[1]) for e in ev],
                  "sort_ranges": [e[1].elapsed_time(e[2]) for e in ev],
                  "render": [e[2].elapsed_time(e[3]) for e in ev]}
    kernels = None
    if kernel_times:
        kernels = rast.profile_read()
        rast.profile(False)
    return total, stages, kernels


def time_mode_flushed(rast, params, cams, st, steps, warmup, stream, pg, with_stages, kernel_times,
                      clock):
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k in range(warmup):
        rast.forward(params, cams[k % len(cams)], st, stream=stream, want_aux=False)
    barrier(pg)
    if kernel_times:
        rast.profile(True)
        rast.profile_read()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device="cuda")
    if clock is not None:
        clock.mark()
    with torch.cuda.stream(stream):
        for k in range(steps):
            cam = cams[(warmup + k) % len(cams)]
            flush.fill_(k & 0xFF)                 # evict the scene and the workspace from L2
            ev[k][0].record(stream)
            rast.preprocess(params, cam, st, stream=stream)
            ev[k][1].record(stream)
            rast.sort(stream=stream)
            ev[k][2].record(stream)
            rast.render(img=img, stream=stream, want_aux=False)
            ev[k][3].record(stream)
    barrier(pg)
    if clock is not None:
        clock.mark()
    total = sum(e[0].elapsed_time(e[3]) for e in ev) / 1e3
    stages = None
    if with_stages:
        stages = {"preprocess_scan_emit": [e[0].elapsed_time(e[1]) for e in ev],
                  "sort_ranges": [e[1].elapsed_time(e[2]) for e in ev],
                  "render": [e[2].elapsed_time(e[3]) for e in ev]}
    kernels = None
    if kernel_times:
        kernels = rast.profile_read()
        rast.profile(False)
    return total, stages, kernels


def frame_units(rast, params, cams, st, stream, count):
    """Untimed, per frame: pairs P, Gaussians with tiles V, the sum over pixels
    of Gaussians evaluated, and the sum over tiles of the list prefix Render
    had to load (the longest pixel traversal in the tile, in whole batches of
    256, capped at the list length)."""
    out = []
    for k in range(count):
        rast.forward(params, cams[k], st, stream=stream, want_aux=False)
        p = rast.num_pairs()
        geom, rect, tiles = rast.read_gaussians(stream=stream)
        v = int(np.count_nonzero(tiles))
        _, trav = rast.read_pixel_stats(stream=stream)
        ranges = rast.read_ranges(stream=stream).astype(np.int64)
        h, w = trav.shape
        ty, tx = (h + 15) // 16, (w + 15) // 16
        pad = np.zeros((ty * 16, tx * 16), np.int64)
        pad[:h, :w] = trav
        tmax = pad.reshape(ty, 16, tx, 16).max(axis=(1, 3)).reshape(-1)
        length = ranges[:, 1] - ranges[:, 0]
        loaded = np.minimum(length, ((tmax + 255) // 256) * 256)
        runs = int((rect[:, 2].astype(np.int64) - rect[:, 0])[tiles > 0].sum())
        # the runs the tile sort built (both depth slices, or all), from the
        # forward frame itself: render it again without the inspection reads
        rast.forward(params, cams[k], st, stream=stream, want_aux=False)
        fc = rast.frame_counts()
        built = fc["runs_slice0"] + fc["runs_slice1"] if fc["sliced"] else fc["runs"]
        out.append(dict(pairs=p, visible=v, runs=runs, evals=int(trav.astype(np.int64).sum()),
                        loaded=int(loaded.sum()), runs_built=built, sliced=fc["sliced"],
                        visible_slice1=fc["visible_slice1"]))
    return out


def kernel_bytes(name, n, u, hw):
    """Algorithmic DRAM bytes per frame of each kernel (the data the stage has
    to move; see the design notes for the derivation), or None where the work
    depends on the depth slices' sizes, which the frame does not report."""
    P, V = u["pairs"], u["visible"]
    return {
        # params (+SH of kept) in; records of kept (64 B), radii/depth, key, box out
        "preprocess": 44 * n + 192 * V + 40 * n + 64 * V,
        # 4 passes: the first reads the n keys twice and writes the V kept keys +
        # values; the others count, read and write V keys + values; the last
        # also gathers and writes the V packed rectangles
        "depth_pass": 8 * n + 76 * V,
        "scan_tiles": 8 * V,                       # boxes in depth order in, run offsets out (slice 1 on top)
        "tile_count_columns": None,                # runs of the two depth slices
        "tile_count_scan": 0,                      # 2 x 256 x grid words, L2-resident
        "tile_scatter_columns": None,
        "tile_count_rows": 8 * u["runs"],          # column runs in (per-tile lists only)
        "tile_scatter_rows": 8 * u["runs"] + 4 * P,
        "tile_ranges": 12 * (hw // 256),           # column / tile ranges
        "slice": None,                             # unfinished-tile table, compaction of slice 1
        "render": 52 * u["loaded"] + 12 * hw,      # records + ids of loaded prefixes, image out
    }.get(name)


def sort_throughput(ktable, u):
    """Items per second of the depth sort (Gaussians with tiles over its four
    passes) and of tile pass 1 (column runs built over its count, count scan
    and scatter kernels), from the live kernel table."""
    ms = lambda names: sum(ktable[k]["ms_per_frame"] for k in names if k in ktable)
    depth_ms = ms(("depth_pass",))
    pass1_ms = ms(("tile_count_columns", "tile_count_scan", "tile_scatter_columns"))
    return {"depth_sort_gaussians_per_s": u["visible"] / (depth_ms / 1e3) if depth_ms else None,
            "depth_sort_ms_per_frame": depth_ms,
            "tile_pass1_runs_per_s": u["runs_built"] / (pass1_ms / 1e3) if pass1_ms else None,
            "tile_pass1_ms_per_frame": pass1_ms,
            "runs_built_per_frame": u["runs_built"], "runs_all_gaussians_per_frame": u["runs"],
            "visible_per_frame": u["visible"]}


def alpha_low_sweep(rast, params, cams, stream, pg, steps, warmup):
    """Raising the splatting-opacity threshold (the paper's remark that a
    higher alpha_low speeds rendering up): AdR-AABB frames/s at 1, 2 and 4 /
    255 (cull and skip both use it), the largest pixel change and the PSNR
    against the 1/255 render on three cameras."""
    import torch
    base = S.Settings(mode=S.MODE_AABB)
    ref = []
    for k in range(3):
        img, _, _ = rast.forward(params, cams[k], base, stream=stream, want_aux=False)
        torch.cuda.synchronize()
        ref.append(img.clone())
    out = []
    for num in (1, 2, 4):
        st = S.Settings(mode=S.MODE_AABB, alpha_low=float(np.float32(num / 255.0)))
        t, _, _ = time_mode(rast, params, cams, st, steps, warmup, stream, pg, with_stages=False)
        diff, mse = 0.0, 0.0
        for k in range(3):
            img, _, _ = rast.forward(params, cams[k], st, stream=stream, want_aux=False)
            torch.cuda.synchronize()
            diff = max(diff, float((img - ref[k]).abs().max()))
            mse += float(((img - ref[k]) ** 2).mean()) / 3
        out.append({"alpha_low": f"{num}/255", "fps": steps / max_over_ranks(pg, t),
                    "pairs": rast.num_pairs(), "max_abs_pixel_change_vs_1_255": diff,
                    "psnr_db_vs_1_255": None if mse == 0 else 10 * math.log10(1.0 / mse)})
    return out


def train_step_rate(local, steps=20, warmup=5):
    """Differentiable training step on 1M clustered Gaussians at 1280x720 with
    the paper's total loss (Sec. 4.4): forward, L1 + SSIM (adr_image_loss) and
    L_load (adr_load_loss) against the render of a perturbed copy, backward
    through adr_render_backward, and an Adam update of the raw parameters."""
    import torch
    from paper_2409_08669_gb300.finetune import FinetuneConfig, Finetuner, render_targets
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    base = S.cluster_scene(n=1_000_000, seed=1)
    target = S.perturbed_scene(base, seed=4)
    cams = S.orbit_cameras(50, width=1280, height=720)[:8]
    st = S.Settings(mode=S.MODE_AABB)
    rast = Rasterizer(max_gaussians=base.n, pair_capacity=1 << 27, max_width=1280,
                      max_height=720, device=local)
    targets = render_targets(rast, upload(target, f"cuda:{local}"), cams, st)
    ft = Finetuner(base, cams, targets, rast, st, FinetuneConfig())
    for _ in range(warmup):
        ft.step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        loss = ft.step()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    # Per-kernel device time of the library's launches over as many more steps
    # (CUDA events on the launching stream), then the work units of the
    # backward on the same cameras: the list positions each pixel walks back
    # (its last blend) and the blended pairs (l_i).
    rast.profile(True)
    rast.profile_read()
    for _ in range(steps):
        ft.step()
    kernels = rast.profile_read()
    rast.profile(False)
    walked, blended = [], []
    with torch.no_grad():
        p = ft.activated_copy()
        for cam in cams:
            _, _, load = rast.forward(p, cam, st)
            last, _ = rast.read_pixel_stats()
            walked.append(int(last.astype(np.int64).sum()))
            blended.append(int(load.to(torch.int64).sum().item()))
    n_vis = int(np.count_nonzero(rast.read_gaussians()[2]))
    rast.close()
    table = {name: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps,
                    "share": v[0] / sum(x[0] for x in kernels.values())}
             for name, v in kernels.items()}
    u = {"walked": statistics.mean(walked), "blended": statistics.mean(blended),
         "visible": n_vis, "gaussians": base.n}
    return {"workload": "cluster-1M-720p", "steps_per_s": 1e3 / ms, "ms_per_step": ms,
            "final_loss": float(loss.item()),
            "step": "forward + L1/SSIM + L_load (lambda 0.44/0.11/0.45) + adr_render_backward + "
                    "Adam on 1M Gaussians, 1280x720",
            "kernels": table, "units": u, "backward_roofline": backward_roofline(table, u)}


# FP32 lane operations of the Render backward: per list position a pixel walks
# back, the forward's evaluation (eigen-form quadratic with its k term, the
# exponential, clamp and skip test); per blended pair the transmittance
# recovery, the colour, opacity and conic terms and the colour behind.
BWD_OPS_PER_WALKED = 15
BWD_OPS_PER_BLENDED = 35
# Preprocess backward, bytes per Gaussian with tiles: parameters (236 B), the
# forward's conic record (32 B), the 2D gradients (36 B) and the tile box in,
# the parameter gradients (236 B) out; without tiles only the box in and zeros out.
BWD_PRE_BYTES_VISIBLE = 236 + 32 + 36 + 4 + 236
BWD_PRE_BYTES_CULLED = 4 + 236


def backward_roofline(table, u, sm_count=152, clk_mhz=2070.0):
    out = {}
    hbm_gbs, _, src = peaks()
    rb = table.get("render_backward")
    if rb:
        ops = BWD_OPS_PER_WALKED * u["walked"] + BWD_OPS_PER_BLENDED * u["blended"]
        ach = ops / (rb["ms_per_step"] / 1e3) / 1e12
        peak = sm_count * 128 * clk_mhz * 1e6 / 1e12
        out["render_backward"] = {"bound": "alu", "achieved": ach, "peak": peak,
                                  "unit": "T FP32 lane-ops/s", "frac": ach / peak,
                                  "work": f"{BWD_OPS_PER_WALKED} per walked position + "
                                          f"{BWD_OPS_PER_BLENDED} per blended pair"}
    pb = table.get("preprocess_backward")
    if pb:
        b = BWD_PRE_BYTES_VISIBLE * u["visible"] + BWD_PRE_BYTES_CULLED * (u["gaussians"] - u["visible"])
        ach = b / (pb["ms_per_step"] / 1e3) / 1e9
        out["preprocess_backward"] = {"bound": "hbm", "achieved": ach, "peak": hbm_gbs,
                                      "unit": "GB/s", "frac": ach / hbm_gbs,
                                      "algorithmic_bytes_per_step": b, "peak_source": src}
    return out


def finetune_measure(local, steps=500):
    """The load-balancing fine-tune (Sec. 4.4) on the 1M-Gaussian clustered
    scene at 1280x720: the scene is fitted to renders of its perturbed copy
    from 10 orbit cameras for `steps` iterations with the paper's weights
    (lambda_load = 0.45) under both readings of d l_i / d alpha
    (straight-through; through the early stop) and once without the load
    term (L1 0.8, SSIM 0.2); frames/s, load std, PSNR and SSIM are measured
    on the training cameras and on 10 other orbit cameras, before and after."""
    import torch
    from paper_2409_08669_gb300.finetune import (FinetuneConfig, Finetuner, evaluate,
                                                 render_targets)
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    base = S.cluster_scene(n=1_000_000, seed=1)
    target = S.perturbed_scene(base, seed=4)
    cams = S.orbit_cameras(50, width=1280, height=720)
    train_cams, eval_cams = cams[0::5], cams[2::5]
    st = S.Settings(mode=S.MODE_AABB)
    rast = Rasterizer(max_gaussians=base.n, pair_capacity=1 << 27, max_width=1280,
                      max_height=720, device=local)
    dev = f"cuda:{local}"
    tparams = upload(target, dev)
    train_tgt = render_targets(rast, tparams, train_cams, st)
    eval_tgt = render_targets(rast, tparams, eval_cams, st)
    b = upload(base, dev)
    out = {"workload": "cluster-1M-720p", "steps": steps, "train_cameras": len(train_cams),
           "eval_cameras": len(eval_cams),
           "before": {"train": evaluate(rast, b, train_cams, train_tgt, st),
                      "eval": evaluate(rast, b, eval_cams, eval_tgt, st)}}
    del b
    st_stop = S.Settings(mode=S.MODE_AABB, load_grad=S.LOAD_GRAD_TERMINATION)
    for name, cfg, s in (
            ("lambda_load_0.45_straight", FinetuneConfig(steps=steps), st),
            ("lambda_load_0.45_termination", FinetuneConfig(steps=steps), st_stop),
            ("lambda_load_0", FinetuneConfig(steps=steps, lambda_l1=0.8, lambda_ssim=0.2,
                                             lambda_load=0.0), st)):
        ft = Finetuner(base, train_cams, train_tgt, rast, s, cfg)
        for _ in range(steps):
            ft.step()
        torch.cuda.synchronize()
        p = ft.activated_copy()
        out[name] = {"train": evaluate(rast, p, train_cams, train_tgt, st),
                     "eval": evaluate(rast, p, eval_cams, eval_tgt, st)}
        del ft, p
    rast.close()
    return out


SERVE_SCENES = (6_000_000, 3_000_000, 1_000_000, 500_000)


def serve_measure(local, n_requests=2000, warmup_requests=200, rate=200.0, seed=21, max_batch=1,
                  slots=16, params=None):
    """Serving: 4 resident clustered scenes (0.5M, 1M, 3M, 6M Gaussians), a
    Poisson stream of `rate` requests/s, each a random camera on the radius-4
    sphere at a resolution drawn from {800x800, 1280x720, 1920x1080}, through
    the continuous-batching server (adr_serve_*) with `slots` frame slots in
    groups of `max_batch` (1: frames overlap, each request its own launches;
    4: up to four requests on one scene share one batched frame).  Latency is
    submit to completion; a closed-loop burst of the same request mix gives
    the saturation throughput."""
    import torch
    from paper_2409_08669_gb300.serve import Server
    sizes = SERVE_SCENES
    st = S.Settings(mode=S.MODE_AABB)
    srv = Server(max_slots=slots, mem_budget_bytes=24 << 30, slot_pair_capacity=1 << 27,
                 slot_max_gaussians=max(sizes), max_width=1920, max_height=1080, device=local,
                 max_batch=max_batch)
    ids = [srv.add_scene(p, st) for p in params]
    res = ((800, 800), (1280, 720), (1920, 1080))
    rng = np.random.default_rng(seed)
    nbuf = 64
    bufs = [torch.empty(3 * 1920 * 1080, dtype=torch.float32, device=f"cuda:{local}") for _ in range(nbuf)]
    torch.cuda.synchronize()
    owner = [None] * nbuf
    failed = []

    def finish(b):
        status = srv.poll(owner[b])
        if status != 0:
            failed.append(status)
        owner[b] = None

    def request(k):
        w, h = res[int(rng.integers(0, 3))]
        cam = S.sphere_camera(rng, radius=4.0, width=w, height=h)
        b = k % nbuf
        if owner[b] is not None:
            finish(b)
        owner[b] = srv.submit(ids[int(rng.integers(0, 4))], cam, bufs[b][: 3 * w * h].view(3, h, w))
        return owner[b]

    def drain():
        for b in range(nbuf):
            if owner[b] is not None:
                finish(b)

    def poisson(count, k0):
        gaps = rng.exponential(1.0 / rate, size=count)
        t = time.perf_counter()
        for k in range(count):
            t += gaps[k]
            while time.perf_counter() < t:
                pass
            request(k0 + k)
        drain()

    poisson(warmup_requests, 0)
    srv.reset_stats()
    t0 = time.perf_counter()
    poisson(n_requests, warmup_requests)
    wall = time.perf_counter() - t0
    open_loop = srv.stats()
    srv.reset_stats()
    burst = 400
    t0 = time.perf_counter()
    for k in range(burst):
        request(k)
    drain()
    closed = srv.stats()
    burst_wall = time.perf_counter() - t0
    srv.close()
    del bufs
    torch.cuda.empty_cache()
    return {"workload": "serve-4scenes-poisson200",
            "scenes": list(sizes), "resolutions": [f"{w}x{h}" for w, h in res],
            "arrival_rate_per_s": rate, "requests": n_requests,
            "p50_ms": open_loop["p50_ms"], "p99_ms": open_loop["p99_ms"],
            "mean_ms": open_loop["mean_ms"], "frames_per_s": n_requests / wall,
            "max_inflight": int(open_loop["max_inflight"]),
            "admitted_while_busy": int(open_loop["admitted_while_busy"]),
            "capacity_errors": int(open_loop["capacity_errors"]),
            "mean_batch": open_loop["mean_batch"],
            "saturation_frames_per_s": burst / burst_wall,
            "saturation_p50_ms": closed["p50_ms"], "saturation_p99_ms": closed["p99_ms"],
            "saturation_mean_batch": closed["mean_batch"],
            "failed_requests": len(failed), "slots": slots, "max_batch": max_batch, "graphs": True}


def serve_both(local):
    """The serving measurement without and with batched frames, on the same
    resident scenes and the same request streams (same seeds)."""
    from paper_2409_08669_gb300.raster import upload
    params = [upload(S.cluster_scene(n=n, seed=31 + k), device=f"cuda:{local}")
              for k, n in enumerate(SERVE_SCENES)]
    out = {"unbatched": serve_measure(local, max_batch=1, params=params),
           "batched": serve_measure(local, max_batch=4, params=params)}
    del params
    return out


def e2e_host(rast_ctx, scene, cams, st, steps, warmup, mode):
    """FPS through adr_render_host with pinned host buffers, every step from
    host to host: with `mode` = HOST_READ_MAPPED, Preprocess reads the scene
    in place over the host link and Render writes the image in place; with
    HOST_READ_COPY, the scene is copied in and the image copied back."""
    import ctypes
    import torch
    from paper_2409_08669_gb300 import _lib
    _lib.adr_set_host_reads(rast_ctx, mode)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in scene.arrays()]
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream().cuda_stream
    st_c = _lib.make_settings(st)
    ptrs = [p.data_ptr() for p in pinned]

    def one(cam):
        _lib.adr_render_host(rast_ctx, *ptrs, scene.n, _lib.make_camera(cam), st_c, img.data_ptr(),
                             0, 0, stream)

    for k in range(warmup):
        one(cams[k % len(cams)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        one(cams[(warmup + k) % len(cams)])
    dt = time.perf_counter() - t0
    d2h = img.numel() * 4
    _lib.adr_set_host_reads(rast_ctx, _lib.HOST_READ_MAPPED)
    del ctypes
    return steps / dt, d2h


def run_ours(args):
    import torch
    from paper_2409_08669_gb300.raster import Rasterizer, upload

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    scene, cams = build_workload(rank)
    params = upload(scene)
    rast = Rasterizer(max_gaussians=N_GAUSS, pair_capacity=PAIR_CAPACITY, max_width=WIDTH,
                      max_height=HEIGHT, device=local)
    stream = torch.cuda.Stream()
    st_adr = S.Settings(mode=S.MODE_AABB)
    st_plain = S.Settings(mode=S.MODE_PLAIN)
    st_circle = S.Settings(mode=S.MODE_CIRCLE)

    # Correctness gate before timing: device flags clear, pair capacity respected.
    rast.forward(params, cams[0], st_adr, stream=stream)
    torch.cuda.synchronize()
    rast.num_pairs()

    window = ("warm-up and timed AdR frames, the instrumented AdR pass" +
              ("" if args.quick else ", then the plain, circle and tile-split legs"))
    with ClockSampler(local, window) as clk:
        # The headline: the frames alone, with no event inside the timed region.
        t_adr, _, _ = time_mode(rast, params, cams, st_adr, args.steps, args.warmup, stream, pg,
                                with_stages=False, clock=clk)
        status = rast.sync_status()
        if status != 0:
            raise SystemExit(f"device status {status} after the timed region")
        # The same frames again with CUDA events around every stage and every
        # launch of the library: the per-stage and per-kernel times.  The events
        # cost ~8% of the frame rate, so they stay out of the headline.
        t_inst, stages, kernels = time_mode(rast, params, cams, st_adr, args.steps, args.warmup,
                                            stream, pg, kernel_times=True)
        status = rast.sync_status()
        if status != 0:
            raise SystemExit(f"device status {status} after the instrumented pass")
        # The PLAIN and circle legs: a leg whose frames hold more pairs than the
        # context's pair capacity (PLAIN at 4K exceeds the 2^30 maximum) renders
        # incomplete images, so it is reported as over capacity, not timed.
        leg_status = {}
        if not args.quick:
            t_plain, _, _ = time_mode(rast, params, cams, st_plain, args.steps, args.warmup,
                                      stream, pg, with_stages=False)
            _, stages_plain, _ = time_mode(rast, params, cams, st_plain, min(args.steps, 50),
                                           args.warmup, stream, pg)
            leg_status["plain"] = rast.sync_status()
            t_circle, _, _ = time_mode(rast, params, cams, st_circle, args.steps, args.warmup,
                                       stream, pg, with_stages=False)
            leg_status["circle"] = rast.sync_status()
            # f2: the last depth slice's tiles as pixel halves on two CTAs each
            from paper_2409_08669_gb300 import _lib as L
            rast.set_tile_split(L.TILE_SPLIT_LAST_SLICE)
            t_split, _, _ = time_mode(rast, params, cams, st_adr, args.steps, args.warmup, stream, pg,
                                      with_stages=False)
            rast.set_tile_split(L.TILE_SPLIT_OFF)
            leg_status["tile_split"] = rast.sync_status()
    clocks = clk.summary()
    for leg, code in leg_status.items():
        if code not in (0, 2):   # 2: ADR_ERR_CAPACITY
            raise SystemExit(f"device status {code} after the {leg} leg")
    plain_ok = leg_status.get("plain") == 0
    circle_ok = leg_status.get("circle") == 0
    if args.quick:
        rast.close()
        fps, _ = aggregate_fps(pg, t_adr, args.steps, world)
        if rank == 0:
            print(json.dumps({"workload": WORKLOAD, "fps": fps,
                              "stages_ms": {k: statistics.mean(v) for k, v in stages.items()}}))
        return
    fps, t_adr = aggregate_fps(pg, t_adr, args.steps, world)
    t_plain = max_over_ranks(pg, t_plain)
    t_circle = max_over_ranks(pg, t_circle)
    frames = args.steps * world

    # Units of work for the roofline (untimed, on the first cameras of the timed cycle).
    nu = min(args.steps, 5)
    ucams = [cams[(args.warmup + k) % len(cams)] for k in range(nu)]
    units_adr = frame_units(rast, params, ucams, st_adr, stream, nu)
    units_plain = frame_units(rast, params, ucams, st_plain, stream, nu) if plain_ok else None
    over_cap = f"over the pair capacity ({PAIR_CAPACITY} pairs) at this workload"
    u_mean = {k: statistics.mean(u[k] for u in units_adr) for k in units_adr[0]}
    hbm_gbs, sm_max_mhz, peak_src = peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = clocks.get("sm_mhz") or sm_max_mhz
    hw = WIDTH * HEIGHT
    # Per-kernel live timing from the library's events on the launch stream.
    ktable = {}
    for name, (ms, launches) in kernels.items():
        per = ms / launches
        per_frame = ms / args.steps
        b = kernel_bytes(name, N_GAUSS, u_mean, hw)
        ktable[name] = {"launches_per_frame": launches / args.steps, "ms_per_launch": per,
                        "ms_per_frame": per_frame,
                        "share": ms / sum(v[0] for v in kernels.values()),
                        "algorithmic_bytes_per_frame": b,
                        "gbs": None if b is None else b / (per_frame / 1e3) / 1e9}
    dominant = max(ktable, key=lambda k: ktable[k]["ms_per_frame"])
    dk = ktable[dominant]
    tpp = TRAFFIC_BYTES_PER_PAIR.get(dominant)
    traffic = tpp * u_mean["pairs"] if tpp else TRAFFIC_BYTES_PER_FRAME.get(dominant)
    if dominant == "render":
        alu_peak = sm_count * 128 * clk_mhz * 1e6 / 1e12
        achieved = u_mean["evals"] * EVAL_FP32_OPS / (dk["ms_per_frame"] / 1e3) / 1e12
        roofline = {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": alu_peak,
                    "unit": "T FP32 lane-ops/s", "frac": achieved / alu_peak, "traffic": traffic,
                    "peak_source": f"{sm_count} SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz"}
    else:
        roofline = {"kernel": dominant, "bound": "hbm", "achieved": dk["gbs"], "peak": hbm_gbs,
                    "unit": "GB/s", "frac": dk["gbs"] / hbm_gbs, "traffic": traffic,
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "algorithmic_bytes_per_frame": dk["algorithmic_bytes_per_frame"]}
    render = ktable.get("render")
    render_ms = render["ms_per_frame"] if render else float("nan")
    alu_peak = sm_count * 128 * clk_mhz * 1e6 / 1e12
    render_alu = u_mean["evals"] * EVAL_FP32_OPS / (render_ms / 1e3) / 1e12
    stage_ms = {k: statistics.mean(v) for k, v in stages.items()}
    stage_ms_plain = ({k: statistics.mean(v) for k, v in stages_plain.items()} if plain_ok
                      else over_cap)

    from paper_2409_08669_gb300 import _lib as L
    e2e_steps = max(3, min(args.steps, 10))
    e2e_fps, d2h = e2e_host(rast.ctx, scene, cams, st_adr, e2e_steps, 2, L.HOST_READ_MAPPED)
    e2e_copy_fps, _ = e2e_host(rast.ctx, scene, cams, st_adr, e2e_steps, 2, L.HOST_READ_COPY)
    # bytes that cross the host link each step: Preprocess reads at most 44 B
    # of every Gaussian (means, scales, rots, opacity) in place, and the colour
    # kernels 204 B (SH + mean) of each Gaussian a Render launch blends; the
    # copy path moves every array
    blended = (math.ceil(u_mean["visible"] / 16) + u_mean["visible_slice1"]
               if u_mean["sliced"] else u_mean["visible"])
    h2d = int(44 * N_GAUSS + 204 * blended)
    h2d_copy = sum(a.nbytes for a in scene.arrays())

    result = {
        "metric": METRIC,
        "value": fps,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_adr / args.steps,
        "instrumented_fps": args.steps / t_inst,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": f"synthetic (seeded {WORKLOADS[WORKLOAD][0]} scene; no dataset or trained model)",
        "config": workload_config(world),
        "plain_fps": frames / t_plain if plain_ok else over_cap,
        "circle_fps": frames / t_circle if circle_ok else over_cap,
        "tile_split_fps": frames / max_over_ranks(pg, t_split),
        "speedup_vs_plain": t_plain / t_adr if plain_ok else None,
        "stages_ms": stage_ms,
        "stages_ms_plain": stage_ms_plain,
        "pairs_per_frame": {"adr_aabb": u_mean["pairs"],
                            "plain": (statistics.mean(u["pairs"] for u in units_plain)
                                      if plain_ok else over_cap)},
        "evals_per_frame": {"adr_aabb": u_mean["evals"],
                            "plain": (statistics.mean(u["evals"] for u in units_plain)
                                      if plain_ok else None)},
        "culled_pair_fraction": (1.0 - u_mean["pairs"] / statistics.mean(u["pairs"] for u in units_plain)
                                 if plain_ok else None),
        # What the sorting kernels move: the depth sort orders the V Gaussians
        # with tiles (4 passes); tile pass 1 groups the column runs it builds
        # (both depth slices' runs when sliced) by tile column.  The pairs
        # themselves are never written on the forward path.
        "sort_throughput": sort_throughput(ktable, u_mean),
        "roofline": roofline,
        "kernels": ktable,
        "render_roofline": {"alu": {"achieved": render_alu, "peak": alu_peak,
                                    "unit": "T FP32 lane-ops/s", "frac": render_alu / alu_peak,
                                    "work": f"{EVAL_FP32_OPS} FP32 ops per Gaussian-pixel evaluation"},
                            "hbm": {"achieved_gbs": render["gbs"] if render else None,
                                    "peak_gbs": hbm_gbs,
                                    "frac": (render["gbs"] / hbm_gbs) if render else None}},
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": ("adr_render_host with pinned host buffers: Preprocess and the colour "
                        "kernels read the scene in place over the host link and Render writes "
                        "the image in place"),
                "copy_path": {"value": e2e_copy_fps, "unit": "frames/s",
                              "h2d_bytes_per_step": h2d_copy, "d2h_bytes_per_step": d2h}},
        "gpu_launches": KERNELS_PER_FRAME * args.steps,
        "clocks": clocks,
    }
    result["alpha_low_sweep"] = alpha_low_sweep(rast, params, cams, stream, pg, min(args.steps, 100),
                                                args.warmup)
    rast.close()
    del params
    if not args.no_train:
        result["train_step"] = train_step_rate(local)
        result["load_balance_finetune"] = finetune_measure(local)
    if not args.no_serve and world == 1:
        result["serve"] = serve_both(local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(scene, cams, st_adr, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(result))


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)
# ---------------------------------------------------------------------------

class OracleFrame:
    """Times the CPU oracle on a bounded sample of one frame and scales to a
    full frame: Preprocess on a 1/g_div sample of the Gaussians (scaled by
    g_div), emission + sort of that sample's pairs (scaled by g_div), and the
    tiled render of a 1/t_div sample of the tiles over their full sorted lists
    (scaled by t_div).  The full lists for the sampled tiles come from one
    untimed preprocess of the whole scene per camera."""

    def __init__(self, scene, g_div=16, t_div=64, seed=0):
        import oracle
        self.oracle = oracle
        self.scene = scene
        self.g_div = g_div
        self.t_div = t_div
        rng = np.random.default_rng(seed)
        self.sample = np.sort(rng.choice(scene.n, scene.n // g_div, replace=False))
        self.sub = scene.subset(self.sample)
        self.rng = rng
        self.cache = {}

    def _tile_lists(self, key, cam, st):
        """Untimed, once per camera: the full preprocess and the sorted lists of
        a random 1/t_div sample of the tiles."""
        if key not in self.cache:
            o = self.oracle
            full = o.preprocess(self.scene, cam, st)
            keys, vals = o.emit_pairs(full)
            tiles = (keys >> np.uint64(32)).astype(np.int64)
            nt = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
            chosen = np.sort(self.rng.choice(nt, max(1, nt // self.t_div), replace=False))
            m = np.isin(tiles, chosen)
            skeys, svals = o.sort_pairs(keys[m], vals[m])
            ranges = o.tile_ranges(skeys, cam.width, cam.height)
            self.cache[key] = (full, ranges, svals, nt / len(chosen))
        return self.cache[key]

    def frame_seconds(self, cam, st, key=None):
        o = self.oracle
        full, ranges, svals, tile_scale = self._tile_lists(key if key is not None else id(cam), cam, st)
        t0 = time.perf_counter()
        pre_s = o.preprocess(self.sub, cam, st)
        k, v = o.emit_pairs(pre_s)
        o.sort_pairs(k, v)
        t_pre = time.perf_counter() - t0
        t1 = time.perf_counter()
        o.render_tiled(full, ranges, svals, st)
        t_render = time.perf_counter() - t1
        self.last_split = (t_pre * self.g_div, t_render * tile_scale)
        self.last_raw = t_pre + t_render   # wall seconds of the sample itself
        return t_pre * self.g_div + t_render * tile_scale


def render_all_cores(of, cam, st, key, threads):
    """Seconds of the oracle's tiled render of the same tile sample on
    `threads` host threads, each rendering its share of the sampled tiles (the
    other tiles' ranges emptied) into its own buffers.  The C oracle holds no
    global state and ctypes releases the GIL during the call, so the threads
    run in parallel; the oracle itself is unchanged."""
    from concurrent.futures import ThreadPoolExecutor
    o = of.oracle
    full, ranges, svals, tile_scale = of._tile_lists(key, cam, st)
    tiles = np.nonzero(ranges[:, 1] > ranges[:, 0])[0]
    parts = [p for p in np.array_split(tiles, threads) if p.size]
    subs = []
    for p in parts:
        r = np.zeros_like(ranges)
        r[p] = ranges[p]
        subs.append(r)
    with ThreadPoolExecutor(max_workers=len(subs)) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda r: o.render_tiled(full, r, svals, st), subs))
        return (time.perf_counter() - t0) * tile_scale


def cpu_baseline(scene, cams, st, budget_s=30.0):
    of = OracleFrame(scene)
    t0 = time.perf_counter()
    secs, pre, ren = [], [], []
    for i, cam in enumerate(cams):
        secs.append(of.frame_seconds(cam, st, key=i))
        pre.append(of.last_split[0])
        ren.append(of.last_split[1])
        if time.perf_counter() - t0 > budget_s:
            break
    cores = os.cpu_count() or 1
    par = [render_all_cores(of, cams[i], st, i, cores) for i in range(len(secs))]
    t_par = statistics.mean(pre) + statistics.mean(par)
    return {"value": 1.0 / statistics.mean(secs), "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": (f"{len(secs)} frame(s): preprocess+emit+sort of a 1/{of.g_div} Gaussian "
                       f"sample and render of a 1/{of.t_div} tile sample, each scaled to the "
                       f"full frame; single-threaded FP64 C"),
            "render_s_per_frame_1_core": statistics.mean(ren),
            "all_cores": {"value": 1.0 / t_par, "unit": "frames/s", "cores": cores,
                          "render_s_per_frame": statistics.mean(par),
                          "preprocess_emit_sort_s_per_frame": statistics.mean(pre),
                          "how": f"the same tile sample rendered on {cores} host threads over "
                                 f"disjoint tile subsets; preprocess, emission and the pair sort "
                                 f"(qsort) stay single-threaded"}}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene, cams = build_workload(0)
    st = S.Settings(mode=S.MODE_AABB)
    of = OracleFrame(scene, g_div=64, t_div=256)
    ncam = 2   # the untimed full-scene lists are built once per distinct camera
    warmup = max(args.warmup, 3)
    for k in range(warmup):
        of.frame_seconds(cams[k % ncam], st, key=k % ncam)
    secs, raw = [], []
    t_wall = time.perf_counter()
    for k in range(args.steps):
        secs.append(of.frame_seconds(cams[(warmup + k) % ncam], st, key=(warmup + k) % ncam))
        raw.append(of.last_raw)
    t_wall = time.perf_counter() - t_wall
    total = sum(secs)
    fps = args.steps / total
    # A step is the bounded sample: ms_per_step is its wall time, and `value`
    # scales each step's sample to a full frame of the workload.
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(world),
        "step": ("a bounded sample of one frame: preprocess, emission and sort of 1/64 of the "
                 "Gaussians and the tiled render of 1/256 of the tiles, each scaled to the full "
                 "frame for `value`"),
        "sample_ms_per_step": 1e3 * sum(raw) / args.steps,
        "scaled_ms_per_frame": 1e3 * total / args.steps,
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": "per step: 1/64 Gaussian sample (preprocess, emit, sort) and "
                                   "1/256 tile sample (render), scaled to a full frame; "
                                   "2 distinct cameras"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def tile_trace_summary(cameras=(0, 12, 25)):
    """Per-tile Render trace (adr_trace_tiles) of single frames of the selected
    workload: for each depth slice, the span from the first tile's start to
    the last tile's end, the mean and peak number of tiles in flight, how long
    fewer than half of the peak were in flight at the end, per-tile duration
    quantiles and the longest tiles (tx, ty, us, start us, positions staged)."""
    import torch
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    scene, cams = build_workload(0)
    params = upload(scene)
    rast = Rasterizer(max_gaussians=N_GAUSS, pair_capacity=PAIR_CAPACITY, max_width=WIDTH,
                      max_height=HEIGHT)
    rast.trace_tiles(True)
    st = S.Settings(mode=S.MODE_AABB)
    for k in range(6):
        rast.forward(params, cams[k], st, want_aux=False)
    tx = (WIDTH + 15) // 16
    out = {"workload": WORKLOAD}
    for k in cameras:
        rast.forward(params, cams[k], st, want_aux=False)
        torch.cuda.synchronize()
        tr = rast.read_tile_trace().astype(np.int64)
        rec = {}
        for ph in (0, 1):
            t = tr[ph]
            used = (t[:, 0] != 0) | (t[:, 1] != 0)
            if not used.any():
                continue
            s0 = t[used, 0]
            base = s0.min()
            s = (s0 - base) % (1 << 32)
            e = (t[used, 1] - base) % (1 << 32)
            d = e - s
            bins = np.zeros(int(e.max()) // 1000 + 2)
            for a, b in zip(s // 1000, e // 1000):
                bins[a:b + 1] += 1
            half = np.nonzero(bins >= 0.5 * bins.max())[0]
            idx = np.nonzero(used)[0]
            top = np.argsort(-d)[:5]
            rec["slice0" if ph == 0 else "slice1"] = {
                "tiles": int(used.sum()), "span_us": float(e.max()) / 1e3,
                "mean_in_flight": float(bins.mean()), "peak_in_flight": int(bins.max()),
                "tail_below_half_us": int(len(bins) - 1 - half[-1]) if half.size else 0,
                "tile_us_p50": float(np.median(d)) / 1e3, "tile_us_p99": float(np.percentile(d, 99)) / 1e3,
                "longest": [[int(idx[i] % tx), int(idx[i] // tx), round(float(d[i]) / 1e3, 1),
                             round(float(s[i]) / 1e3, 1), int(t[idx[i], 3])] for i in top]}
        out[f"camera{k}"] = rec
    rast.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="heavy-3M-1080p")
    ap.add_argument("--quick", action="store_true",
                    help="time the AdR mode only (no plain/circle arms, e2e or baselines)")
    ap.add_argument("--serve-only", action="store_true",
                    help="only the serving measurement (unbatched and batched), one JSON line")
    ap.add_argument("--train-only", action="store_true",
                    help="only the training-step measurement, one JSON line")
    ap.add_argument("--tile-trace", action="store_true",
                    help="only the per-tile Render trace of three frames of the workload, one JSON line")
    args = ap.parse_args()
    select_workload(args.workload)
    args.warmup = max(args.warmup, 3)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.train_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"train_step": train_step_rate(0, steps=args.steps, warmup=args.warmup)}))
    elif args.tile_trace:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(tile_trace_summary()))
    elif args.serve_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"serve": serve_both(0)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
