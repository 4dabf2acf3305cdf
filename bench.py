#!/usr/bin/env python
"""Benchmark of the sliding-window optimisation step of GS-LIVO's Gaussian map
(Sec. II-B.2): one step renders every keyframe of the window (projection,
tile binning, compositing), takes the L1 photometric loss, back-propagates to
every Gaussian parameter and applies Adam.

Workload: a box-room window of 200,000 planar Gaussians (SH degree 1) seen by
8 keyframes at 640x512 on a 2 m arc, FP32, Adam lr 1e-3; seeded synthetic
data shaped like the paper's LiDAR-seeded windows (its datasets are not
available).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

--impl reference times the FP64 CPU oracle on a bounded pixel sample of the
same workload (the method has no other reference implementation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "fwd+bwd window-opt iters/s at 200k Gaussians×8 views 640×512; % of roofline"
UNIT = "it/s"
N_GAUSS = 200_000
N_VIEWS = 8
W_IMG, H_IMG = 640, 512
FOCAL = 600.0
LR = 1e-3
WORKLOAD = "box-room sliding window: 200k planar Gaussians (SH degree 1), 8 keyframes 640x512 on a 2 m arc"

# Algorithmic FP32 operations per fragment (FMA = 2; compares, min/max and
# selects not counted; ex2 and the divide count 1 each):
#   every visited fragment:  d = x - q (2), t_k = d . v_k (2 x 3), p = l - t1^2 - t2^2 (4)   = 12
#   forward, contributing:   ex2, w = alpha T, T (1 - alpha) = T - w, C += w c (6)           = 9
#   backward, contributing:  ex2, 1 - alpha, T / (1 - alpha), w, dL/dc += w g (6), g.c (5),
#                            g.c - g.R, dL/dalpha, g.R update (2), ga, ga t1, ga t2 (4),
#                            ga dx, ga dy, ga dx^2, ga dx dy, ga dy^2 (6), sum ga            = 34
FLOP_VISITED = 12.0
FLOP_CONTRIB = {"raster_fwd": 9.0, "raster_bwd": 34.0}
FP32_LANES = 128
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# compositing kernels from ncu captures of this workload, per launch shape
# (tile size, pixels per thread, batch, bin size: the autotuner's two fastest,
# within 0.1 % of each other), valid only for the kernel source they were taken
# on (sha256 prefix of gs_raster.cu up to the L1 kernels, which holds both
# compositing kernels); otherwise the roofline reports traffic null.
TRAFFIC = {"raster_fwd": [("b545d25b20f69256", (8, 2, 128, 32), 198.9e6),
                          ("b545d25b20f69256", (16, 4, 128, 32), 189.7e6)],
           "raster_bwd": [("b545d25b20f69256", (8, 2, 128, 32), 262.8e6),
                          ("b545d25b20f69256", (16, 4, 128, 32), 249.3e6)]}


def raster_source_hash():
    with open(os.path.join(HERE, "paper_2501_08672_b300", "csrc", "gs_raster.cu")) as f:
        src = f.read()
    return hashlib.sha256(src[:src.index("constexpr int kL1Threads")].encode()).hexdigest()[:16]


MAX_SM_MHZ = 2032


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="window",
                    choices=["window", "plain", "uneven", "mixed", "odometry", "maintenance"],
                    help="window: the headline window step; plain, uneven, mixed: the other window "
                         "configurations; odometry: Gauss-Newton pose iterations")
    ap.add_argument("--cpu-pixels", type=int, default=0,
                    help="oracle pixels sampled per view (0: 64 per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100,
                    help="steps of the end-to-end timing (including its pipeline fill and drain)")
    ap.add_argument("--tile-size", type=int, default=0, help="0: autotune tile size, pixels per thread, batch")
    ap.add_argument("--ppt", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--bin-tile-size", type=int, default=0,
                    help="binning tile size with --tile-size (0: the tile size; 2 or 4 times it: bins split per tile)")
    ap.add_argument("--maint-n", default="",
                    help="maintenance workload: comma-separated window sizes (default: the full sweep)")
    ap.add_argument("--compare-forms", dest="compare_forms", action="store_true", default=None,
                    help="also time the workload with FP32 storage and in the plain per-view form "
                         "(default for --workload mixed)")
    ap.add_argument("--no-compare-forms", dest="compare_forms", action="store_false")
    ap.add_argument("--odo-frames", type=int, default=0, help="odometry workload: frames (0: 200)")
    ap.add_argument("--deterministic", action="store_true",
                    help="bit-reproducible backward (fixed-order sums instead of float atomics)")
    ap.add_argument("--ssim-lambda", type=float, default=0.0,
                    help="weight of the D-SSIM term in the photometric loss (0: the L1 loss of the paper)")
    return ap.parse_args()


def max_over_ranks(values, world, device="cuda"):
    """Element-wise maximum of per-rank timings over all ranks (the job ends
    when its slowest replica does); the identity for one rank."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(world, steps, max_ms):
    """Units per second of the whole job: every rank ran `steps` units in at
    most `max_ms` milliseconds (replicas: weak scaling)."""
    return world * steps / (max_ms / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(seed=0, name="window"):
    """(params, views, storage dtypes, metric, description) of a window
    workload.  "window" is the headline; "plain", "uneven" and "mixed" are
    the single-view, batched-uneven and mixed-precision windows of the
    parity tests, timed the same way."""
    import torch
    from paper_2501_08672_b300 import scenes
    if name == "window":
        params = scenes.box_room_scene(N_GAUSS, seed=seed, sh_degree=1)
        views = scenes.arc_views(N_VIEWS, W_IMG, H_IMG, FOCAL, n_gaussians=N_GAUSS)
        return params, views, None, METRIC, WORKLOAD
    if name == "plain":
        n = 10_000
        params = scenes.frustum_scene(n, seed=seed)
        views = [scenes.identity_view(320, 256, 300.0, 0, n)]
        return (params, views, None, "fwd+bwd window-opt iters/s at 10k Gaussians x 1 view 320x256",
                "plain single view: 10k random Gaussians (SH degree 0) in front of an identity camera, 320x256")
    if name == "uneven":
        params, views = scenes.uneven_batch(16, 2_000_000, seed=seed)
        desc = ("batched uneven: 16 views of a 2M-Gaussian box room (SH degree 1), widths %s, "
                "contiguous Gaussian ranges of %d to %d" % (sorted({int(v["W"]) for v in views}),
                                                        min(v["g_end"] - v["g_begin"] for v in views),
                                                        max(v["g_end"] - v["g_begin"] for v in views)))
        return params, views, None, "fwd+bwd window-opt iters/s, 16 uneven views of a 2M-Gaussian window", desc
    if name == "mixed":
        params, views = scenes.mixed_precision_scene(2_000_000, seed=seed)
        storage = dict(log_scales=torch.bfloat16, quats=torch.bfloat16, opacity=torch.float16, sh=torch.float16)
        return (params, views, storage,
                "fwd+bwd window-opt iters/s at 2M Gaussians x 10 views 1280x1024, FP16/BF16 storage",
                "mixed precision: 2M-Gaussian box room (SH degree 1), 10 keyframes 1280x1024; colour/SH and "
                "opacity stored FP16, log-scale and quaternion BF16, means FP32; FP32 arithmetic")
    raise ValueError(name)


def peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_iteration(params, views, pixels_per_view, seed=1, n_threads=0):
    """Times the FP64 oracle on a pixel sample of one window iteration and
    scales the per-pixel parts to the full images.  n_threads 0: every host
    core, for the pixel loops and the projection passes alike (each pixel,
    each Gaussian is independent in the oracle).  Returns (seconds per
    iteration estimate, threads used, description)."""
    from oracle import oracle as O
    threads = n_threads if n_threads > 0 else host_cores()
    O.set_threads(threads)
    rng = np.random.default_rng(seed)
    t_fixed = 0.0
    t_pix = 0.0
    n_pix_total = 0
    try:
        for v in views:
            W, H = int(v["W"]), int(v["H"])
            px = rng.integers(0, W, pixels_per_view)
            py = rng.integers(0, H, pixels_per_view)
            t0 = time.perf_counter()
            pr = O.project(params, v)
            t1 = time.perf_counter()
            O.render_pixels(params, v, px, py, proj=pr, n_threads=threads)
            t2 = time.perf_counter()
            dl = [rng.standard_normal((pixels_per_view, 3)) * 1e-6]
            O.backward(params, [v], dl, pixels=[(px, py)], n_threads=threads)
            t3 = time.perf_counter()
            O.backward(params, [v], [np.zeros((0, 3))], pixels=[(px[:0], py[:0])], n_threads=threads)
            t4 = time.perf_counter()
            scale = (W * H) / float(pixels_per_view)
            t_fixed += (t1 - t0) + (t4 - t3)
            t_pix += ((t2 - t1) + max(0.0, (t3 - t2) - (t4 - t3))) * scale
            n_pix_total += pixels_per_view
        n = sum(int(params[k].size) for k in ("means", "log_scales", "quats", "opacity", "sh"))
        p = rng.standard_normal(n)
        g = rng.standard_normal(n)
        m = np.zeros(n)
        vv = np.zeros(n)
        t0 = time.perf_counter()
        O.adam(p, g, m, vv, LR, 0.9, 0.999, 1e-8, 1)
        t_adam = time.perf_counter() - t0
    finally:
        O.set_threads(0)
    desc = ("oracle FP64 on %d host threads: %d random pixels per view (%d of %d) rendered and back-propagated, "
            "projection and projection backward over all Gaussians, Adam over all %d parameters (one thread); "
            "per-pixel time scaled to the full images"
            % (threads, pixels_per_view, n_pix_total, sum(int(v["W"]) * int(v["H"]) for v in views), n))
    return t_fixed + t_pix + t_adam, threads, desc


def run_reference(args, world, rank):
    if rank != 0:
        return
    params, views = workload()[:2]
    # a bounded sample per step: 16 pixels per view per host core (about a
    # second per step on 16 cores)
    ppv = 16 * host_cores()
    for _ in range(args.warmup):
        cpu_oracle_iteration(params, views[:1], ppv)
    times = []
    threads = 1
    desc = ""
    for k in range(args.steps):
        t, threads, desc = cpu_oracle_iteration(params, views, ppv, seed=100 + k)
        times.append(t)
    sec = float(np.mean(times))
    val = 1.0 / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "views": N_VIEWS, "image": [W_IMG, H_IMG]},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_rooflines(kms, n_gauss, n_records, n_pairs, n_tiles, n_params, param_bytes, lowp_elems, visited,
                     contrib, ffma_tflops, hbm_gbs, n_bins=None, n_list=None):
    """Achieved fraction of its roofline for every kernel family of one
    iteration, from its CUDA-event time per iteration (kms, ms) and its
    algorithmic work: FP32 FLOP per the fragment model for the compositing
    kernels (bound by FP32 issue), bytes for the others (bound by HBM).
    Algorithmic bytes (the minimum a kernel must move, not its traffic):
      project      per record: the Gaussian's parameters (param_bytes) read,
                   the 48 B record, 16 B rectangle, 4 B tile count and 12 B
                   depth key and index written
      depth_sort   per record: the 12 B (64-bit key, index) read and written
                   once (one pass; more passes count as overhead)
      tile_scan    per record: tile count and sorted index read, 8 B offset
                   written
      emit         per pair: 8 B (tile key, record index) written
      tile_sort    per pair: 8 B read and 8 B written once
      ranges       per pair: 4 B key read; per bin 8 B range written
      refine       (bins of several tiles) per pair 8 B (key with its tile
                   mask, record index) read; per entry of the tiles' lists
                   (n_list) 4 B written; per tile 8 B range written
    A pair is a (bin, record) pair; without bins larger than the tiles a bin
    is a tile (n_bins = n_tiles, n_list = n_pairs, no refine).
      project_bwd  per record 36 B of 2D gradients read; per Gaussian its
                   parameters read and 4 B per parameter written
      adam         per parameter 28 B (p, g, m, v read; p, m, v written),
                   plus the low-precision copy written"""
    work = {
        "project": ("hbm", n_records * (param_bytes + 80.0)),
        "depth_sort": ("hbm", n_records * 24.0),
        "tile_scan": ("hbm", n_records * 16.0),
        "emit": ("hbm", n_pairs * 8.0),
        "tile_sort": ("hbm", n_pairs * 16.0),
        "ranges": ("hbm", n_pairs * 4.0 + (n_bins or n_tiles) * 8.0),
        "refine": ("hbm", n_pairs * 8.0 + (n_list or 0) * 4.0 + n_tiles * 8.0),
        "raster_fwd": ("alu", FLOP_VISITED * visited + FLOP_CONTRIB["raster_fwd"] * contrib),
        "raster_bwd": ("alu", FLOP_VISITED * visited + FLOP_CONTRIB["raster_bwd"] * contrib),
        "project_bwd": ("hbm", n_records * 36.0 + n_gauss * param_bytes + n_params * 4.0),
        "adam": ("hbm", n_params * 28.0 + lowp_elems * 2.0),
    }
    out = {}
    for k, (bound, amount) in work.items():
        ms = kms.get(k)
        if not ms:
            continue
        if bound == "alu":
            ach = amount / (ms / 1e3) / 1e12
            out[k] = {"bound": "alu", "ms": ms, "achieved": ach, "peak": ffma_tflops, "unit": "TFLOP/s",
                      "frac": ach / ffma_tflops, "work": amount}
        else:
            ach = amount / (ms / 1e3) / 1e9
            out[k] = {"bound": "hbm", "ms": ms, "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
                      "frac": ach / hbm_gbs, "work": amount}
    return out


def run_b300(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2501_08672_b300 import binding as B
    from paper_2501_08672_b300 import scenes
    from paper_2501_08672_b300.render import GaussianWindow, Renderer, WindowOptimizer, autotune

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    params, views, storage, metric, wdesc = workload(seed=rank, name=args.workload)
    n_gauss = int(params["means"].shape[0])
    n_px = sum(int(v["W"]) * int(v["H"]) for v in views)
    # target keyframes: render of a perturbed copy of the window
    q = scenes.perturbed_copy(params, seed=1000 + rank)
    rt = Renderer(views, local, 16)
    wq = GaussianWindow(q, local, storage)
    rt.forward(wq.struct())
    target = rt.rgb.clone()
    del rt, wq

    # launch shape: autotuned over the compiled variants unless given
    tune_table = None
    if args.tile_size:
        shape = (args.tile_size, args.ppt, args.batch, args.bin_tile_size)
    else:
        shape, tune_table = autotune(params, views, target, steps=3, device=local, storage=storage,
                                     deterministic=int(args.deterministic))
    opt = WindowOptimizer(params, views, target, lr=LR, device=local, tile_size=shape[0],
                          ssim_lambda=args.ssim_lambda,
                          pixels_per_thread=shape[1], batch=shape[2], bin_tile_size=shape[3], storage=storage,
                          deterministic=int(args.deterministic))
    ctx = opt.r.ctx
    opt.step(count=True)  # sizes the pair workspace
    cap0 = opt.r.cap
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K = args.steps
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x.strip() for x in vis.split(",") if x.strip()]
    sampler = ClockSampler(int(ids[local]) if local < len(ids) and ids[local].isdigit() else local)

    def timed(run_step):
        """K steps, each bracketed by CUDA events on the launching stream, with
        an L2 flush (256 MB write) between steps outside the events."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()
            ev[k][0].record()
            run_step()
            ev[k][1].record()
        torch.cuda.synchronize()
        barrier()
        return float(sum(a.elapsed_time(b) for a, b in ev))

    # warm-up of the host-issued form, every kernel family timed once to find
    # the dominant one
    ctx.profile(B.KERNEL_FAMILIES)
    n_warm = max(args.warmup, 3)
    for _ in range(n_warm):
        opt.step(count=False)
    prof_all = ctx.profile_collect()
    rc, need = opt.r.check_status()
    if rc != B.GS_OK:
        raise RuntimeError("pair capacity exceeded during warm-up (%d needed, %d reserved)" % (need, cap0))
    dominant = max(prof_all, key=lambda k: prof_all[k][1])

    # timed region 1: host-issued launches, dominant kernel timed by events
    ctx.profile([dominant])
    sampler.start()
    launches0 = ctx.launch_count()
    plain_ms = timed(lambda: opt.step(count=False))
    launches_per_step = (ctx.launch_count() - launches0) / K
    prof = ctx.profile_collect()
    ctx.profile([])

    # timed region 2 (headline): the same iteration captured once in a CUDA
    # graph and replayed
    opt.capture()
    for _ in range(n_warm):
        opt.step()
    total_ms = timed(opt.step)
    clocks = sampler.stop()
    # the graph holds the same launches plus the device step-counter kernel of Adam
    launches = int(round((launches_per_step + 1) * K))
    rc, need = opt.r.check_status()
    if rc != B.GS_OK:
        raise RuntimeError("pair capacity exceeded in the timed region (%d needed)" % need)
    max_ms, max_plain_ms = max_over_ranks([total_ms, plain_ms], world)
    value = whole_job_rate(world, K, max_ms)

    # roofline of the dominant kernel
    dom_launches, dom_ms = prof.get(dominant, (0, 0.0))
    avg_ms = dom_ms / max(dom_launches, 1)
    hbm, hbm_kind = peaks()
    # measured ALU peaks of this device (FFMA and ex2 microbenchmarks, outside timing)
    ffma_tflops, ex2_gops = ctx.calibrate_alu()
    # fragment counts of the last parameters (one extra forward, outside timing)
    n_used = torch.empty_like(opt.r.n_contrib)
    opt.r.forward(opt._g, count=False, n_used=n_used)
    torch.cuda.synchronize()
    visited = float(opt.r.n_contrib.double().sum().item())
    contrib = float(n_used.double().sum().item())
    # the same count over 16 x 16-tile lists (the 3D-GS tiling), for comparison:
    # finer lists visit fewer fragments for the same image, so the work of the
    # kernel's own lists understates what it does against that tiling
    visited16 = visited
    if shape[0] != 16 or (shape[3] or 16) != 16:
        r16 = Renderer(views, local, 16)
        r16.forward(opt._g, count=True)
        torch.cuda.synchronize()
        visited16 = float(r16.n_contrib.double().sum().item())
        del r16
    if dominant in FLOP_CONTRIB:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        nominal = sms * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
        peak = ffma_tflops
        flop = FLOP_VISITED * visited + FLOP_CONTRIB[dominant] * contrib
        achieved = flop / (avg_ms / 1e3) / 1e12
        traffic = None
        for sha, tshape, tbytes in TRAFFIC.get(dominant, []):
            if raster_source_hash() == sha and tuple(shape) == tshape and args.workload == "window":
                traffic = tbytes
        roof = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                "avg_launch_ms": avg_ms,
                "visited_fragments": visited, "contributing_fragments": contrib,
                "flop_per_launch": flop,
                "visited_fragments_16x16_lists": visited16,
                "frac_16x16_lists": (FLOP_VISITED * visited16 + FLOP_CONTRIB[dominant] * contrib)
                / (avg_ms / 1e3) / 1e12 / peak,
                "peak_basis": "measured: FP32 FMA microbenchmark (gs_calibrate_alu, best of 3)",
                "peak_nominal": nominal,
                "peak_nominal_basis": "%d SMs x 128 lanes x 2 FLOP x %d MHz (maximum SM clock)" % (sms, MAX_SM_MHZ),
                "frac_of_nominal": achieved / nominal,
                "ex2_measured_gops": ex2_gops}
    else:
        roof = {"bound": "hbm", "kernel": dominant, "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "traffic": None, "avg_launch_ms": avg_ms, "peak_kind": hbm_kind}
    # every kernel family against its own roofline
    L = opt.r.layout()
    K_sh = (int(params["sh_degree"]) + 1) ** 2
    st = storage or {}
    esz = lambda k: (2 if k in st else 4)  # noqa: E731
    param_bytes = 12 + 3 * esz("log_scales") + 4 * esz("quats") + esz("opacity") + 3 * K_sh * esz("sh")
    n_params = n_gauss * (11 + 3 * K_sh)
    lowp_elems = sum(n_gauss * w for k, w in (("log_scales", 3), ("quats", 4), ("opacity", 1), ("sh", 3 * K_sh))
                     if k in st)
    kms = {k: v[1] / n_warm for k, v in prof_all.items()}
    n_list = opt.r.list_entries()
    by_kernel = kernel_rooflines(kms, n_gauss, int(L.n_records), int(opt.r.last_pairs), int(L.n_tiles), n_params,
                                 param_bytes, lowp_elems, visited, contrib, ffma_tflops, hbm, n_bins=int(L.n_bins),
                                 n_list=n_list)

    # end to end through the public API with host buffers: per step the step's
    # input, the keyframe images (targets), goes host->device from pinned
    # memory and its result, the loss, comes back device->host; the window's
    # parameters stay resident on the device (the window of the method lives
    # in device memory across iterations).  The copies are pipelined against
    # the compute: the targets of the next steps are uploaded on one copy
    # stream into a ring of three target buffers while step k computes on its
    # own (the iteration is captured once per buffer, so no copy into a fixed
    # buffer is needed, and each upload may take two steps' time), and step
    # k's loss is read back on another copy stream while step k+1 computes;
    # every byte still crosses the link inside the timed region.
    host_target = target.cpu().pin_memory()
    back_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    E = args.e2e_steps
    comp = torch.cuda.current_stream()
    c_in, c_out = torch.cuda.Stream(), torch.cuda.Stream()
    NB = 3
    in_t = [torch.empty_like(target) for _ in range(NB)]
    out_l = [torch.empty(1, device=target.device) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(E)]
    ev_staged = [torch.cuda.Event() for _ in range(E)]
    ev_out = [torch.cuda.Event() for _ in range(E)]
    ev_drained = [torch.cuda.Event() for _ in range(E)]

    def upload(k):
        with torch.cuda.stream(c_in):
            if k >= NB:
                c_in.wait_event(ev_staged[k - NB])
            in_t[k % NB].copy_(host_target, non_blocking=True)
            ev_in[k].record(c_in)

    e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    opt.capture(targets=in_t)  # one graph per target buffer (outside the timed region)
    # this host link's rate for the step's upload, alone (outside the timed
    # region): the end-to-end rate cannot exceed it / the bytes per step
    h_s, h_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(c_in):
        in_t[0].copy_(host_target, non_blocking=True)
        h_s.record(c_in)
        for _ in range(5):
            in_t[0].copy_(host_target, non_blocking=True)
        h_e.record(c_in)
    torch.cuda.synchronize()
    h2d_gbs = 5 * host_target.numel() * 4 / (h_s.elapsed_time(h_e) / 1e3) / 1e9
    torch.cuda.synchronize()
    e_s.record(comp)
    for j in range(min(NB - 1, E)):
        upload(j)
    for k in range(E):
        if k + NB - 1 < E:
            upload(k + NB - 1)
        comp.wait_event(ev_in[k])
        loss = opt.step(slot=k % NB)
        ev_staged[k].record(comp)  # buffer k % NB read: step k + NB's upload may overwrite it
        if k >= 2:
            comp.wait_event(ev_drained[k - 2])
        out_l[k % 2].copy_(loss, non_blocking=True)
        ev_out[k].record(comp)
        with torch.cuda.stream(c_out):
            c_out.wait_event(ev_out[k])
            back_loss.copy_(out_l[k % 2], non_blocking=True)
            ev_drained[k].record(c_out)
    comp.wait_event(ev_drained[E - 1])
    e_e.record(comp)
    torch.cuda.synchronize()
    e2e_ms = e_s.elapsed_time(e_e) / E
    h2d = host_target.numel() * 4
    d2h = 4

    # the same workload in other forms, each graph-replayed and timed like the
    # headline: FP32 storage batched, and the plain per-view FP32 form (one
    # launch sequence per view, gradients accumulated, one Adam step)
    other_forms = {}
    if args.compare_forms or (args.compare_forms is None and args.workload == "mixed"):
        from paper_2501_08672_b300.render import PerViewOptimizer

        def form_rate(o):
            o.step(count=True)
            for _ in range(n_warm):
                o.step(count=False)
            o.capture()
            for _ in range(n_warm):
                o.step()
            ms = timed(o.step)
            st = o.check_status() if hasattr(o, "check_status") else o.r.check_status()
            if st[0] != B.GS_OK:
                raise RuntimeError("pair capacity exceeded in a compared form")
            return whole_job_rate(world, K, max_over_ranks([ms], world)[0])

        kw = dict(lr=LR, device=local, tile_size=shape[0], pixels_per_thread=shape[1], batch=shape[2],
                  bin_tile_size=shape[3])
        if storage:
            o = WindowOptimizer(params, views, target, **kw)
            other_forms["batched_fp32_storage_it_s"] = form_rate(o)
            del o
        o = PerViewOptimizer(params, views, target, **kw)
        other_forms["per_view_fp32_storage_it_s"] = form_rate(o)
        del o
        torch.cuda.empty_cache()

    cpu = None
    if (rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "window"
            and args.ssim_lambda == 0):
        ppv = args.cpu_pixels or 64 * host_cores()
        sec, threads, desc = cpu_oracle_iteration(params, views, ppv)
        cpu = {"value": 1.0 / sec, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
        # the same oracle on one host thread (a smaller pixel sample)
        sec1, _, desc1 = cpu_oracle_iteration(params, views, max(ppv // 16, 8), seed=2, n_threads=1)
        cpu["single_thread"] = {"value": 1.0 / sec1, "unit": UNIT, "cores": 1, "sample": desc1}
        cpu["speedup_over_one_thread"] = sec1 / sec

    if rank == 0:
        mpix = world * K * n_px / (max_ms / 1e3) / 1e6
        line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": max_ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wdesc, "n_gaussians": n_gauss, "views": len(views),
                           "image": ([int(views[0]["W"]), int(views[0]["H"])] if len({(v["W"], v["H"]) for v in views}) == 1
                                     else [[int(v["W"]), int(v["H"])] for v in views]),
                           "tile_size": shape[0], "pixels_per_thread": shape[1],
                           "batch": shape[2], "bin_tile_size": shape[3] or shape[0],
                           "sh_degree": int(params["sh_degree"]), "lr": LR,
                           "loss": ("L1" if args.ssim_lambda == 0 else
                                    "(1 - %g) L1 + %g (1 - SSIM), 11x11 window" % (args.ssim_lambda, args.ssim_lambda)),
                           "storage": ({k: str(v).replace("torch.", "") for k, v in storage.items()} if storage
                                       else "float32"),
                           "autotune_ms": ({"%d/%d/%d/%d" % k: round(v, 4) for k, v in tune_table.items()}
                                           if tune_table else None),
                           "l2": "flushed between steps (256 MB write outside the timed events)",
                           "pairs_per_step": int(opt.r.last_pairs), "parallelism": "replicas" if world > 1 else "1 GPU",
                           "deterministic": bool(args.deterministic),
                           "mpix_per_s": mpix},
                "roofline": roof,
                "kernel_ms_per_step": {k: v[1] / n_warm for k, v in prof_all.items()},
                "roofline_by_kernel": by_kernel,
                "forms": dict({"graph_replay_it_s": value,
                               "host_issued_it_s": whole_job_rate(world, K, max_plain_ms)}, **other_forms),
                "cpu_baseline": cpu,
                "e2e": {"value": 1e3 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "h2d_link_gbs": h2d_gbs,
                        "upload_only_it_s": h2d_gbs * 1e9 / max(h2d, 1)},
                "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


ODO_METRIC = ("odometry photometric pose iterations/s at 500k Gaussians, one 1280x1024 view "
              "(forward + L1 + pose-only backward), 200 frames x 5 iterations; % of roofline")
ODO_N, ODO_W, ODO_H, ODO_F, ODO_FRAMES, ODO_ITERS = 500_000, 1280, 1024, 1200.0, 200, 5
# host step of the pose-gradient form, T <- Exp(-eta g) T, per unit of dL/dxi
# (rotation, translation); the paper feeds the gradient to its IESKF, the
# step rule does not change the GPU work
ODO_ETA = (2e-2, 2e-2)
# algorithmic FP32 operations of the pose normal equations (FMA = 2):
#   per visited fragment 12 (the test, as above);
#   per contributing fragment 10 (forward) + 16 (m = M d, its products, the alpha
#   tangent scale) + 6 x 28 (dp, dalpha, dw, dC (3), dT per pose component) = 194;
#   per pixel 36 (H = dC + bg dT) + 126 (H H^T, 21 entries x 3 channels) + 36 (H r) + 6 (r^2) = 204
FLOP_PN_VISITED, FLOP_PN_CONTRIB, FLOP_PN_PIXEL = 12.0, 194.0, 204.0


def run_odometry(args, world, rank, local):
    """Configuration 5, the photometric pose update: 500k fixed Gaussians,
    one 1280x1024 view, 200 frames on an arc, each started from a pose
    perturbed by 2 degrees and 5 cm, 5 iterations per frame.  Two forms run
    over all frames, each timed per iteration by CUDA events (device time)
    and by the host clock (end to end, with the read-back and host step):
      pose gradient (the headline value): project, bin, composite with the
        L1 loss folded in, pose-only backward (gs_pose_grad), read back the 6
        floats, host step T <- Exp(-eta g) T;
      normal equations: project, bin, per-pixel pose Jacobian normal
        equations (gs_pose_normal), read back the 28 sums, host Gauss-Newton
        solve (the linearisation the paper's IESKF update uses)."""
    import torch
    from paper_2501_08672_b300 import binding as B
    from paper_2501_08672_b300 import scenes
    from paper_2501_08672_b300.render import GaussianWindow, Renderer, apply_left

    torch.cuda.set_device(local)
    n = ODO_N
    n_frames = args.odo_frames or ODO_FRAMES
    params = scenes.box_room_scene(n, seed=2 + rank, sh_degree=1)
    true_v, start_v = scenes.odometry_frames(n_frames, ODO_W, ODO_H, ODO_F, seed=rank)
    for v in true_v + start_v:
        v["g_begin"], v["g_end"] = 0, n
    win = GaussianWindow(params, local)
    g = win.struct()
    # launch shape of both forms: the window's default (8 x 8 tiles split from
    # 32 x 32 bins) unless given
    oshape = (args.tile_size, args.ppt, args.batch, args.bin_tile_size) if args.tile_size else (8, 2, 128, 32)
    r = Renderer([true_v[0]], local, oshape[0], pixels_per_thread=oshape[1], batch=oshape[2],
                 bin_tile_size=oshape[3])
    targets = []
    most = 0
    for v in true_v:                      # input generation: the camera frames
        r.set_views([v])
        r.forward(g, count=True)
        most = max(most, r.last_pairs)
        targets.append(r.rgb.clone())
    r.ensure_capacity(int(most * 1.5))
    torch.cuda.synchronize()

    def pose_err(a, b):
        D = np.eye(4); D[:3, :3] = np.asarray(a["R"], np.float64); D[:3, 3] = a["t"]
        E = np.eye(4); E[:3, :3] = np.asarray(b["R"], np.float64); E[:3, 3] = b["t"]
        X = D @ np.linalg.inv(E)
        return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(X[:3, :3]) - 1) / 2)))), float(np.linalg.norm(X[:3, 3]))

    def iterate_grad(view, target, ev=None):
        r.set_views([view])
        if ev is not None:
            ev[0].record()
        r.forward(g, count=False, target=target)
        r.pose_grad(g, r.dL_drgb)
        if ev is not None:
            ev[1].record()
        gp = r.dL_dpose.double().cpu().numpy()        # synchronises: D2H of 6 floats
        xi = np.concatenate([-ODO_ETA[0] * gp[:3], -ODO_ETA[1] * gp[3:]])
        return apply_left(view, xi)

    def iterate_normal(view, target, ev=None):
        r.set_views([view])
        if ev is not None:
            ev[0].record()
        r.ctx.project(g, r.views, r.ws_struct)
        r.ctx.bin(r.views, r.ws_struct)
        normal = r.pose_normal(g, target)
        if ev is not None:
            ev[1].record()
        A, b, rr = B.unpack_normal(normal)[0]          # synchronises: D2H of 28 doubles
        xi = np.linalg.solve(A + 1e-6 * np.trace(A) / 6.0 * np.eye(6), b)
        return apply_left(view, xi)

    def run_path(iterate, families):
        v = start_v[0]
        for _ in range(max(args.warmup, 3)):
            v = iterate(v, targets[0])
        K = n_frames * ODO_ITERS
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        r.ctx.profile(families)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        finals, start_err = [], []
        k = 0
        for fr in range(n_frames):
            v = start_v[fr]
            start_err.append(pose_err(v, true_v[fr]))
            for _ in range(ODO_ITERS):
                v = iterate(v, targets[fr], evs[k])
                k += 1
            finals.append(pose_err(v, true_v[fr]))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        prof = r.ctx.profile_collect()
        r.ctx.profile([])
        rc, need = r.check_status()
        if rc != B.GS_OK:
            raise RuntimeError("pair capacity exceeded in the timed region (%d needed)" % need)
        dev_ms = float(sum(a.elapsed_time(b) for a, b in evs))
        rot = [a for a, _ in finals]
        trn = [t for _, t in finals]
        conv = {"frames": len(finals), "median_start_rot_deg": float(np.median([a for a, _ in start_err])),
                "median_start_trans_m": float(np.median([t for _, t in start_err])),
                "median_final_rot_deg": float(np.median(rot)), "median_final_trans_m": float(np.median(trn)),
                "max_final_rot_deg": float(np.max(rot)), "max_final_trans_m": float(np.max(trn))}
        return K, dev_ms, wall, prof, conv, v

    sampler = ClockSampler(local)
    sampler.start()
    K, dev_ms, wall, prof, conv, v_last = run_path(iterate_grad, B.KERNEL_FAMILIES)
    Kn, dev_ms_n, wall_n, prof_n, conv_n, v_last_n = run_path(iterate_normal, B.KERNEL_FAMILIES)
    clocks = sampler.stop()
    value = K / (dev_ms / 1e3)
    ffma, ex2 = r.ctx.calibrate_alu()

    def fragments(view):
        n_used = torch.empty_like(r.n_contrib)
        r.set_views([view])
        r.forward(g, count=False, n_used=n_used)
        torch.cuda.synchronize()
        return float(r.n_contrib.double().sum().item()), float(n_used.double().sum().item())

    # roofline of the dominant kernel of the pose-gradient form (the
    # compositing backward) and of the normal-equation kernels, from
    # fragment counts at each form's last pose
    visited, contrib = fragments(v_last)
    dom = max(prof, key=lambda kk: prof[kk][1])
    d_l, d_ms = prof[dom]
    if dom in FLOP_CONTRIB:
        flop = FLOP_VISITED * visited + FLOP_CONTRIB[dom] * contrib
        ach = flop / (d_ms / max(d_l, 1) / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": ffma, "unit": "TFLOP/s", "frac": ach / ffma,
                "traffic": None, "avg_launch_ms": d_ms / max(d_l, 1), "visited_fragments": visited,
                "contributing_fragments": contrib, "flop_per_launch": flop,
                "peak_basis": "measured: FP32 FMA microbenchmark (gs_calibrate_alu, best of 3)"}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": peaks()[0], "unit": "GB/s", "frac": None,
                "traffic": None}
    visited_n, contrib_n = fragments(v_last_n)
    pn_launches, pn_ms = prof_n.get("pose_normal", (0, 0.0))
    flop_n = FLOP_PN_VISITED * visited_n + FLOP_PN_CONTRIB * contrib_n + FLOP_PN_PIXEL * ODO_W * ODO_H
    ach_n = flop_n / (pn_ms / Kn / 1e3) / 1e12
    line = {"metric": ODO_METRIC, "value": value, "unit": "it/s", "n_gpus": world, "steps": K,
            "warmup": max(args.warmup, 3), "ms_per_step": dev_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "odometry: 500k fixed planar Gaussians (SH degree 1), one 1280x1024 view, "
                                   "%d frames on an arc, start poses perturbed by 2 deg and 5 cm, %d iterations "
                                   "per frame" % (n_frames, ODO_ITERS),
                       "n_gaussians": n, "image": [ODO_W, ODO_H], "tile_size": oshape[0],
                       "pixels_per_thread": oshape[1], "batch": oshape[2], "bin_tile_size": oshape[3] or oshape[0],
                       "frames": n_frames,
                       "iterations_per_frame": ODO_ITERS,
                       "timed": "device time per iteration (CUDA events): project + bin + composite with the L1 "
                                "loss + pose-only backward",
                       "host_step": "T <- Exp(-eta g) T, eta = %g (rotation), %g (translation)" % ODO_ETA,
                       "l2": "inputs larger than L2 (500k x 48 B records, 1.3 Mpix images)"},
            "frames_per_s": value / ODO_ITERS,
            "roofline": roof,
            "kernel_ms_per_step": {kk: vv[1] / K for kk, vv in prof.items()},
            "e2e": {"value": K / wall, "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 6 * 4,
                    "note": "host clock per iteration including the read-back of the pose gradient and the host "
                            "step; the frames are resident"},
            "convergence": conv,
            "forms": {"normal_equations": {
                "value": Kn / (dev_ms_n / 1e3), "unit": "it/s", "frames_per_s": Kn / (dev_ms_n / 1e3) / ODO_ITERS,
                "ms_per_step": dev_ms_n / Kn,
                "timed": "device time per iteration: project + bin + pose normal equations (tangents, "
                         "forward-mode compositing, FP64 totals)",
                "e2e_it_s": Kn / wall_n, "e2e_note": "with the read-back of 28 doubles and the host 6x6 solve",
                "kernel_ms_per_step": {kk: vv[1] / Kn for kk, vv in prof_n.items()},
                "roofline": {"bound": "alu", "kernel": "pose_normal", "achieved": ach_n, "peak": ffma,
                             "unit": "TFLOP/s", "frac": ach_n / ffma, "flop_per_call": flop_n},
                "convergence": conv_n}},
            "gpu_launches": int(sum(vv[0] for vv in prof.values())), "clocks": clocks}
    print(json.dumps(line), flush=True)

MAINT_SIZES = (100_000, 500_000, 1_000_000, 2_000_000, 5_000_000)


def measure_append_overlap(local, n_append=500_000, iters=10):
    """Step 4 overlapped with the optimisation: the headline window (200k
    Gaussians, 8 keyframes 640x512, spare capacity for the new rows) runs
    `iters` graph-replayed iterations on the compute stream while n_append
    Gaussians are appended on a copy stream (host-to-device from pinned
    memory, moments cleared, SH0 from a keyframe image).  Adam touches the
    active rows only, so the two never touch the same rows.  Device times
    (CUDA events) of each alone and of both issued together."""
    import torch
    from paper_2501_08672_b300.render import GaussianWindow, Renderer, WindowOptimizer

    params, views = workload()[:2]
    n = int(params["means"].shape[0])
    q = scenes_perturbed(params)
    rt = Renderer(views, local, 16)
    wq = GaussianWindow(q, local)
    rt.forward(wq.struct())
    target = rt.rgb.clone()
    del rt, wq
    opt = WindowOptimizer(params, views, target, lr=LR, device=local, tile_size=16, pixels_per_thread=2, batch=128,
                          capacity=n + n_append)
    opt.step(count=True)
    opt.capture()
    from paper_2501_08672_b300 import scenes
    new = scenes.box_room_scene(n_append, seed=77, sh_degree=int(params["sh_degree"]))
    pinned = {k: torch.as_tensor(np.ascontiguousarray(new[k], np.float32)).pin_memory() for k in GaussianWindow.GROUPS}
    w = opt.win
    image = target[:3 * int(views[0]["W"]) * int(views[0]["H"])].view(3, int(views[0]["H"]), int(views[0]["W"]))
    side = torch.cuda.Stream()
    comp = torch.cuda.current_stream()

    def append_on(stream):
        with torch.cuda.stream(stream):
            for k in GaussianWindow.GROUPS:
                w.column(k)[n:n + n_append].view(n_append, -1).copy_(pinned[k].view(n_append, -1), non_blocking=True)
            w.ctx().window_clear([w.column(k, f) for k in GaussianWindow.GROUPS for f in (w.m, w.v)], n,
                                 n + n_append, stream=stream)
            w.n = n + n_append
            w.ctx().sh_init_bilinear(w.struct(), dict(views[0], g_begin=0, g_end=n + n_append), image, n,
                                     n + n_append, w.column("sh"), stream=stream)
            w.n = n

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(comp)
        fn()
        b.record(comp)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def iterate():
        for _ in range(iters):
            opt.step()

    def app():
        side.wait_stream(comp)
        append_on(side)
        comp.wait_stream(side)

    def both():
        side.wait_stream(comp)
        append_on(side)
        iterate()
        comp.wait_stream(side)

    for fn in (iterate, app, both):
        fn()
    res = {}
    for name, fn in (("iterations_ms", iterate), ("append_ms", app), ("together_ms", both)):
        res[name] = float(np.median([timed(fn) for _ in range(5)]))
    hidden = res["iterations_ms"] + res["append_ms"] - res["together_ms"]
    res.update({"iterations": iters, "appended": n_append, "h2d_bytes": n_append * 92,
                "hidden_fraction_of_append": hidden / res["append_ms"]})
    return res


def scenes_perturbed(params):
    from paper_2501_08672_b300 import scenes
    return scenes.perturbed_copy(params, seed=1000)


def run_maintenance(args, world, rank, local):
    """Sliding-window maintenance on the device (Sec. II-C) against the window
    size N: per step 10 % of the window leaves (gathered for the global map,
    Step 1, and compacted, Step 2) and as many new Gaussians enter (host to
    device from pinned memory, gradients and moments cleared, SH0 from a
    640x512 image, Step 4).  Each part is captured in a CUDA graph and timed
    by replay (device time, no host launch overhead): `value` is the whole
    step, the roofline covers the kernels alone (HBM bound; the host-to-device
    copy is bound by the host link and reported beside it).  Algorithmic bytes
    of the kernels: every compaction mover copies its parameters and both Adam
    moments (3 x 92 B read + written; gradients are dead between iterations,
    every backward overwrites them), every leaving row is gathered (92 B read
    + written), every new row gets 2 x 92 B cleared, its mean read and its SH
    written by the initialisation (12 + 48 B), and the keep flags are read
    (1 B per row).  `e2e`: the same step through
    GaussianWindow.maintain / append, which also copy the leaving Gaussians
    and the row map to the host."""
    import torch
    from paper_2501_08672_b300 import binding as B
    from paper_2501_08672_b300 import scenes
    from paper_2501_08672_b300.render import GaussianWindow

    torch.cuda.set_device(local)
    hbm, hbm_kind = peaks()
    rows = []
    v = scenes.lookat_view((4.0, -1.0, 2.2), (0.0, 0.0, 0.6), 640, 512, 600.0, 0, 1)
    image = torch.rand(3, 512, 640, device="cuda")
    K = max(args.steps // 5, 5)

    def replay_ms(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            fn()
        for _ in range(3):
            g.replay()
        ts = []
        for _ in range(K):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            g.replay()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    sizes = [int(x) for x in args.maint_n.split(",") if x.strip()] or list(MAINT_SIZES)
    for N in sizes:
        params = scenes.box_room_scene(N, seed=rank, sh_degree=1)
        turn = N // 10
        extra = scenes.box_room_scene(turn, seed=rank + 1, sh_degree=1)
        pinned = {k: torch.as_tensor(np.ascontiguousarray(extra[k], np.float32)).pin_memory()
                  for k in GaussianWindow.GROUPS}
        win = GaussianWindow(params, local, capacity=N + turn)
        ctx = win.ctx()
        rng = np.random.default_rng(rank)
        keep = torch.as_tensor((rng.uniform(size=N) >= 0.1).astype(np.uint8)).cuda()
        leave_idx = torch.nonzero(keep == 0).view(-1).to(torch.int32)
        n_leave = int(leave_idx.numel())
        n_keep_t = torch.zeros(1, dtype=torch.int64, device="cuda")
        moved = torch.empty(N, dtype=torch.int32, device="cuda")
        scratch = torch.empty(int(B.lib().gs_window_scratch_bytes(N)), dtype=torch.uint8, device="cuda")
        cols = win._columns(N)
        # the parameter column of each group receives the leaving rows (room for N rows)
        leave = [None] * len(cols)
        c = 0
        for k in GaussianWindow.GROUPS:
            leave[c] = torch.empty((N,) + tuple(win.widths[k]), device="cuda").reshape(N, -1)
            c += 3 + (1 if k in win.lowp else 0)
        zcols = [win.column(k, f) for k in GaussianWindow.GROUPS for f in (win.m, win.v)]
        nk = N - n_leave

        def kernels():
            ctx.window_remove(cols, leave, keep, n_keep_t, moved, scratch=scratch)
            ctx.window_clear(zcols, nk, nk + turn)
            win.n = nk + turn
            ctx.sh_init_bilinear(win.struct(), dict(v, g_begin=0, g_end=win.n), image, nk, nk + turn,
                                 win.column("sh"))
            win.n = N

        def h2d():
            for k in GaussianWindow.GROUPS:
                win.column(k)[nk:nk + turn].view(turn, -1).copy_(pinned[k].view(turn, -1), non_blocking=True)

        def step():
            kernels()
            h2d()

        ms_k = replay_ms(kernels)
        ms_h = replay_ms(h2d)
        ms = replay_ms(step)
        movers = int((moved[:nk].cpu().numpy() != np.arange(nk)).sum())
        # end to end through the window API (host syncs and read-backs
        # included); the entering Gaussians come from a pinned host map
        pinned_params = dict(pinned, sh_degree=1)
        # steady state: one window, each step maintain (10 % leave) then append
        # (10 % enter); the first step (allocations) is not counted
        win2 = GaussianWindow(params, local, capacity=N + 2 * turn)
        e2e = []
        for k in range(6):
            keep_h = rng.uniform(size=win2.n) >= 0.1
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            win2.maintain(keep_h)
            win2.append(pinned_params, image=image, view=dict(v, g_begin=0, g_end=win2.n + turn))
            torch.cuda.synchronize()
            if k > 0:
                e2e.append((time.perf_counter() - t0) * 1e3)
        del win2
        algo = movers * 3 * 92 * 2 + n_leave * 92 * 2 + turn * (2 * 92 + 12 + 48) + N
        rows.append({"n": N, "step_ms": ms, "kernels_ms": ms_k, "h2d_ms": ms_h, "e2e_ms": float(np.median(e2e)),
                     "movers": movers, "leaving": n_leave, "appended": turn, "kernel_bytes": algo,
                     "kernels_gbs": algo / (ms_k / 1e3) / 1e9, "h2d_gbs": turn * 92 / (ms_h / 1e3) / 1e9})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del win, cols, leave, zcols
    overlap = measure_append_overlap(local)
    print(json.dumps({"append_overlap": overlap}), file=sys.stderr, flush=True)
    big = rows[-1]
    line = {"metric": "window maintenance step (10 pct leave: gather + compact; 10 pct enter: copy in, clear, "
                      "SH0 init), device ms at N=%d" % big["n"],
            "value": big["step_ms"], "unit": "ms", "n_gpus": world, "steps": K, "warmup": 3,
            "ms_per_step": big["step_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sliding-window maintenance of a box-room window of N Gaussians (SH degree 1)",
                       "sizes": sizes, "per_size": rows, "append_overlap": overlap,
                       "l2": "window larger than L2 from N=1M (368 B per Gaussian with gradient and moments)"},
            "roofline": {"bound": "hbm", "achieved": big["kernels_gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": big["kernels_gbs"] / hbm, "traffic": None, "peak_kind": hbm_kind,
                         "kernel": "maintenance kernels (gather, compaction, clear, SH0 init) as one graph"},
            "e2e": {"value": big["e2e_ms"], "unit": "ms", "h2d_bytes_per_step": big["appended"] * 92,
                    "d2h_bytes_per_step": big["leaving"] * 92 + 8}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.workload != "window" and args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the headline window workload"}))
        return
    if args.workload == "odometry":
        run_odometry(args, world, rank, local)
    elif args.workload == "maintenance":
        run_maintenance(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_b300(args, world, rank, local)


if __name__ == "__main__":
    main()
