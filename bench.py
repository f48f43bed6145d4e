#!/usr/bin/env python
"""Training throughput of the GB300 tile rasterizer.

Workload (Kingsnake-scale stand-in): 4,000,000 Gaussians on the 0.5 level of
a seeded 200-blob field, SH degree 3, FP32 parameters and Adam state; 256
orbit cameras (16 azimuths x 16 elevations, radius 4, 60 degree FOV) at
2048x2048; targets are renders of the reference set, the trained set starts
from a seeded +-5% perturbation of it.  One step = projection, binning (scans,
depth sort of the visible Gaussians, emission of the tile instances, tile
sort, ranges), forward compositing, L1 loss, backward compositing,
projection backward and Adam, over a batch of B=16 views.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gs|reference]
                    [--workload blobs4M|gyroid500k|noise18M] [--serve-sweep]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (bounded sample of the same workload).  The other
workloads: gyroid500k = 500,000 Gaussians on the gyroid level set, 64 orbit
cameras (radius 15) at 1024x1024, B=8; noise18M = 18,000,000 Gaussians on the
zero level of 6-octave fractal noise, 4096x4096, B=4, with the device memory
the training state holds reported beside the throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "train views/s @4M Gauss 2048² batched vs 1-view; render p50/p99 ms"
HP = dict(lr_mean=1.6e-4 * 1.0, lr_scale=5e-3, lr_quat=1e-3, lr_opacity=0.05, lr_sh_dc=2.5e-3,
          lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"])
    ap.add_argument("--workload", default="blobs4M", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="override the workload's Gaussian count")
    ap.add_argument("--res", type=int, default=0, help="override the workload's resolution")
    ap.add_argument("--batch", type=int, default=0, help="override the workload's views per step")
    ap.add_argument("--plain-views", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--serve-rate", type=float, default=100.0, help="render requests/s (0: skip serving)")
    ap.add_argument("--serve-saturating-rate", type=float, default=1000.0,
                    help="second serving rate, above one-request-per-launch saturation")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="sweep the request rate over 50..2000 req/s instead of one rate")
    ap.add_argument("--fwd-variant", type=int, default=0, help="force the forward compositing variant")
    ap.add_argument("--bwd-variant", type=int, default=0, help="force the backward compositing variant")
    ap.add_argument("--bwd-direct", type=int, default=-1,
                    help="force the backward's direct-atomic lane limit (with forced variants)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-init-bench", action="store_true", help="skip the point-cloud initialisation timings")
    ap.add_argument("--cache", default=os.environ.get("GS_SCENE_CACHE", "/tmp/gs_scene_cache"))
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    args.n = args.n or w["n"]
    args.res = args.res or w["res"]
    args.batch = args.batch or w["batch"]
    return args


# ---------------------------------------------------------------- workload

# name -> scene builder, seed, sampling grid, Gaussians, resolution, views per
# step, orbit grid (azimuths x elevations) and radius
WORKLOADS = {
    "blobs4M": dict(scene="blobs_scene", seed=4, grid=128, n=4_000_000, res=2048, batch=16, orbit=(16, 16),
                    radius=4.0, title="blobs-isosurface-4M-2048sq-B16"),
    "gyroid500k": dict(scene="gyroid_scene", seed=3, grid=96, n=500_000, res=1024, batch=8, orbit=(8, 8),
                       radius=15.0, title="gyroid-isosurface-500k-1024sq-B8"),
    "noise18M": dict(scene="noise_scene", seed=5, grid=256, n=18_000_000, res=4096, batch=4, orbit=(16, 16),
                     radius=4.0, title="fractal-noise-isosurface-18M-4096sq-B4"),
}


def workload(args, device=None):
    from paper_2509_05216_gb300 import inputs
    w = WORKLOADS[args.workload]
    os.makedirs(args.cache, exist_ok=True)
    path = os.path.join(args.cache, "%s_n%d_s%d.npz" % (w["scene"], args.n, w["seed"]))
    if os.path.exists(path):
        z = np.load(path)
        scene = {"params": z["params"], "n": int(z["n"]), "deg": int(z["deg"])}
    else:
        scene = getattr(inputs, w["scene"])(args.n, seed=w["seed"], deg=3, res=w["grid"], device=device)
        tmp = path + ".%d.tmp.npz" % os.getpid()
        np.savez(tmp, params=scene["params"], n=scene["n"], deg=scene["deg"])
        os.replace(tmp, path)
    cams = inputs.orbit_cameras(w["orbit"][0], w["orbit"][1], w["radius"], args.res, args.res)
    trained = inputs.perturb(scene, 100 + w["seed"])
    return scene, trained, cams


def config_dict(args, n_gpus):
    w = WORKLOADS[args.workload]
    title = w["title"]
    if (args.n, args.res, args.batch) != (w["n"], w["res"], w["batch"]):
        title += " (resized: n=%d res=%d B=%d)" % (args.n, args.res, args.batch)
    P = 59
    state = 4 * args.n * P * 4 // 10**6          # parameters, gradients, Adam moments
    images = 3 * args.batch * 3 * args.res * args.res * 4 // 10**6  # targets, image, image gradient
    return {"workload": title, "gaussians": args.n, "sh_degree": 3,
            "resolution": [args.res, args.res], "batch_views": args.batch,
            "orbit_cameras": w["orbit"][0] * w["orbit"][1],
            "global_batch": args.batch * n_gpus, "parallelism": "replicas x%d" % n_gpus,
            "l2": "no flush: every step streams a working set larger than the 129 MB L2 (%d MB training "
                  "state, %d MB of images, plus records and sort buffers)" % (state, images)}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, interval_ms=50, first_wait_s=3.0):
        self.index = index
        self.interval_ms = interval_ms
        self.first_wait_s = first_wait_s
        self.rows = []
        self.start = 0
        self.proc = None

    def _launch(self, interval_ms):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a while to print its first line: wait for it
        # (bounded) so that the samples cover the region that follows
        t0 = time.time()
        while not self.rows and time.time() - t0 < self.first_wait_s:
            if self.proc.poll() is not None:
                self.t.join(timeout=1.0)
                break
            time.sleep(0.005)

    def __enter__(self):
        self._launch(self.interval_ms)
        if self.proc is not None and not self.rows and self.proc.poll() is not None and self.interval_ms < 200:
            self._launch(200)  # the short interval was refused: the tool's usual one
        # summarise only the samples taken from here on
        self.start = len(self.rows)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = self.rows[self.start:] or self.rows[-1:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm

class Trainer:
    """Training state on one GPU and the step through the C ABI."""

    def __init__(self, ctx, trained, device):
        import torch
        self.ctx = ctx
        self.n, self.deg = trained["n"], trained["deg"]
        self.p = torch.from_numpy(trained["params"]).to(device)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.loss = torch.zeros(1, device=device)
        self.t = 0

    def step(self, cams, target, img, dimg, hp=HP):
        c = self.ctx
        c.gs_project(self.p, self.n, self.deg, cams)
        c.gs_bin_sort()
        c.gs_raster_fwd_l1(img, target, self.loss, dimg)
        c.gs_raster_bwd(self.p, self.n, self.deg, dimg, self.g)
        self.t += 1
        c.gs_adam(self.p, self.g, self.m, self.v, self.n, self.deg, hp, self.t)


def replica_batches(rank, world, nbatch, count):
    """Camera batches of one replica: rank r takes batches r, r + world, ...
    (modulo the orbit), so the replicas train on disjoint views."""
    return [(rank + i * world) % nbatch for i in range(count)]


def max_over_ranks(x, world, device=None):
    """Largest value of x over all ranks (the job's time is its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def render_targets(ctx, scene, cams, B, batches, device):
    """Target images of the given camera batches (renders of the reference
    set) and the largest instance count seen."""
    import torch
    from paper_2509_05216_gb300 import gs
    p = torch.from_numpy(scene["params"]).to(device)
    _, total = gs.image_offsets(cams[:B])
    out, most = [], 0
    for b in batches:
        cb = cams[b * B:(b + 1) * B]
        t = torch.empty(total, device=device)
        ctx.gs_project(p, scene["n"], scene["deg"], cb)
        ctx.gs_bin_sort()
        ctx.gs_raster_fwd(t)
        most = max(most, ctx.gs_get_counts()[0])
        out.append(t)
    ctx.gs_sync()
    return out, most


# Algorithmic work per launch: bytes for the HBM-bound kernels, FP32
# operations (an FMA counts 2) for the compositing kernels: the operations the
# method needs at one (pixel, Gaussian) pair, not the issued instructions.
# Every list entry up to a pixel's last contributor needs the alpha test
# (offset, quadratic form, opacity times ex2: 10 operations); a contributing
# pair (power <= 0, alpha >= 1/255) also needs the compositing arithmetic
# (forward: transmittance update and colour, 9 more; backward: recovered
# transmittance, dL/dalpha and the nine gradient terms, 30 more).  ex2 and
# the reciprocal run on the special-function unit and are not counted.
RASTER_OPS_TEST = 10
RASTER_OPS_FWD = 19   # per contributing pair, forward
RASTER_OPS_BWD = 40   # per contributing pair, backward


def raster_work(kind, entries, contributing):
    """FP32 operations of one compositing launch: contributing pairs at the
    full per-pair count, the other entries up to each pixel's last
    contributor at the alpha-test count."""
    full = RASTER_OPS_FWD if kind == "fwd" else RASTER_OPS_BWD
    return full * contributing + RASTER_OPS_TEST * (entries - contributing)


def algorithmic_work(name, n, P, B, I, pairs, pixels, V=0):
    """(bound, work per launch scope): bytes for the HBM-bound kernels, FP32
    operations for the compositing kernels.  I = tile instances; V = visible
    (view, Gaussian) pairs; pairs = (entries up to each pixel's last
    contributor, contributing pairs)."""
    if name == "project_fwd":
        # parameters once; per (view, Gaussian) the 48-byte record, the
        # 16-byte (radius, tiles, rect) entry and the (tiles, depth) pair
        return "hbm", n * (4 * P + B * 72.0)
    if name == "project_bwd":
        return "hbm", n * (8 * P + B * 36.0)
    if name == "adam":
        return "hbm", 28.0 * P * n
    if name == "compact":
        # (tile count, depth bits) per (view, Gaussian) read; (depth bits,
        # Gaussian) per visible pair written
        return "hbm", n * B * 8.0 + 8.0 * V
    if name == "depth_histogram":
        return "hbm", 4.0 * V
    if name == "depth_pass":
        # 32-bit key and value read and written per visible pair
        return "hbm", 16.0 * V
    if name == "emit":
        # sorted Gaussian and its 16-byte (radius, tiles, rect) entry per
        # visible pair; 32-bit bin and Gaussian per instance written
        return "hbm", 20.0 * V + 8.0 * I
    if name == "tile_pass":
        return "hbm", 16.0 * I
    if name == "tile_ranges":
        return "hbm", 4.0 * I
    if name == "raster_fwd":
        return "alu", raster_work("fwd", *pairs)
    if name == "raster_bwd":
        return "alu", raster_work("bwd", *pairs)
    return None, None


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    from paper_2509_05216_gb300 import autotune, gs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.zeros(1, device=dev)
    free0, hbm_total = torch.cuda.mem_get_info(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    scene, trained, cams = workload(args, device=dev)
    torch.cuda.empty_cache()
    B = args.batch
    nbatch = len(cams) // B
    ctx = gs.Context(local)
    t0 = time.time()
    order = replica_batches(rank, world, nbatch, min(nbatch, args.warmup + args.steps))
    targets, most = render_targets(ctx, scene, cams, B, order, dev)
    _, total = gs.image_offsets(cams[:B])
    img = torch.empty(total, device=dev)
    dimg = torch.empty(total, device=dev)
    tr = Trainer(ctx, trained, dev)

    def batch(i):
        k = i % len(order)
        b = order[k]
        return cams[b * B:(b + 1) * B], targets[k]

    for i in range(args.warmup):
        tr.step(*batch(i), img, dimg)
    ctx.gs_sync()
    # launch options picked by the autotuner (timed on this workload, cached)
    key = autotune.workload_key(tr.n, cams[:B], B)
    if args.fwd_variant or args.bwd_variant:
        tuned = {gs.GS_OPT_RASTER_FWD: args.fwd_variant or 2, gs.GS_OPT_RASTER_BWD: args.bwd_variant or 2,
                 gs.GS_OPT_BWD_DIRECT: args.bwd_direct if args.bwd_direct >= 0 else 2}
        for opt, val in tuned.items():
            ctx.gs_set_option(opt, val)
    else:
        tuned = autotune.tune([ctx], lambda: tr.step(*batch(0), img, dimg), key,
                              use_cache=not args.retune)
    ctx.gs_sync()
    # the batched step captured once in a CUDA graph (fixed instance capacity)
    torch.cuda.synchronize(dev)
    free_g0, _ = torch.cuda.mem_get_info(dev)
    gctx = gs.Context(local, instance_capacity=int(most * 1.3) + (1 << 20))
    for opt, val in tuned.items():
        gctx.gs_set_option(opt, val)
    gctx.gs_train_graph_capture(tr.p, tr.g, tr.m, tr.v, tr.n, tr.deg, HP, batch(0)[0], batch(0)[1], img, dimg,
                                tr.loss)
    torch.cuda.synchronize(dev)
    free_g1, _ = torch.cuda.mem_get_info(dev)

    def graph_step(cb, tb):
        tr.t += 1
        gctx.gs_train_graph_launch(cb, tb, tr.t)

    for i in range(2):
        graph_step(*batch(i))
    gctx.gs_sync()
    gctx.profile_reset()
    # timed region: K batched steps, each one graph launch
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        ev0.record(stream)
        for i in range(args.steps):
            graph_step(*batch(args.warmup + i))
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    gctx.gs_sync()  # raises on capacity overflow
    free_t, _ = torch.cuda.mem_get_info(dev)
    state_bytes = 4 * tr.p.numel() * 4
    memory = {"device_used_gb": round((free0 - free_t) / 1e9, 2),
              "training_state_gb": round(state_bytes / 1e9, 2),
              "graph_context_workspace_gb": round((free_g0 - free_g1) / 1e9, 2),
              "one_step_gb": round((state_bytes + (free_g0 - free_g1) + 3 * img.numel() * 4) / 1e9, 2),
              "hbm_total_gb": round(hbm_total / 1e9, 1),
              "note": "one_step = parameters, gradients and Adam moments + the graph context's workspace "
                      "(records, keys, sort, per-pixel state) + image, image gradient and one target batch; "
                      "device_used also holds the cached targets and the call-by-call context"}
    gk = gctx.profile_read()
    launches = sum(k["launches"] for k in gk)
    t_max = max_over_ranks(ms, world, dev)
    views = args.steps * B * world
    value = views / (t_max / 1000.0)

    # per-kernel times: the same K steps launched call by call with CUDA
    # events around every kernel on the launching stream
    ctx.profile_reset()
    ctx.profile_enable(True)
    torch.cuda.synchronize(dev)
    ek0, ek1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ek0.record(stream)
    for i in range(args.steps):
        tr.step(*batch(args.warmup + i), img, dimg)
    ek1.record(stream)
    torch.cuda.synchronize(dev)
    ms_calls = ek0.elapsed_time(ek1)
    ctx.profile_enable(False)
    kstats = ctx.profile_read()
    ctx.gs_sync()

    # work counters of one batched step (for the roofline): list entries up
    # to each pixel's last contributor and the contributing pairs among them
    inst, bins, pixels = ctx.gs_get_counts()
    pairs = ctx.gs_pair_stats()
    P = tr.p.shape[0]
    dom = max(kstats, key=lambda k: k["total_ms"])
    per_kernel = {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3),
                              "share": round(k["total_ms"] / max(sum(x["total_ms"] for x in kstats), 1e-9), 4)}
                  for k in kstats}
    ctrl = ctx.gs_get_buffer(gs.GS_BUF_SORT_CTRL).cpu().numpy()
    dctrl = ctx.gs_get_buffer(gs.GS_BUF_DEPTH_CTRL).cpu().numpy()
    executed = {"tile_pass": int(sum((ctrl[p] & 2) == 0 for p in range(ctrl.size - 1))),
                "depth_pass": int(sum((dctrl[p] & 2) == 0 for p in range(dctrl.size - 1)))}
    vm = ctx.gs_get_buffer(gs.GS_BUF_VISMASK).cpu().numpy().view(np.uint64)
    vis_pairs = int(sum(int(((vm >> np.uint64(v)) & np.uint64(1)).sum()) for v in range(B)))
    peak_hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    for k in kstats:
        kk, w = algorithmic_work(k["name"], tr.n, P, B, inst, pairs, pixels, vis_pairs)
        if kk is None or k["total_ms"] <= 0:
            continue
        runs = executed.get(k["name"], 1) * args.steps  # one launch scope per step, sort passes as executed
        rate = w * runs / (k["total_ms"] / 1e3)
        e = per_kernel[k["name"]]
        if kk == "hbm":
            e["GB_s"] = round(rate / 1e9, 1)
            e["frac_hbm"] = round(rate / 1e9 / peak_hbm, 3)
        else:
            e["TFLOP_s"] = round(rate / 1e12, 2)
    kind, work = algorithmic_work(dom["name"], tr.n, P, B, inst, pairs, pixels, vis_pairs)
    avg_ms = dom["total_ms"] / max(dom["launches"], 1)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    if kind == "hbm":
        peak = float(peaks.get("hbm_gbs", 6800.0))
        achieved = work / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": dom["name"],
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    else:
        clk_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = sms * 128 * 2 * clk_max * 1e6 / 1e12  # FP32 TFLOP/s, FMA = 2
        achieved = work / (avg_ms / 1e3) / 1e12
        variant = tuned.get(gs.GS_OPT_RASTER_BWD if dom["name"] == "raster_bwd" else gs.GS_OPT_RASTER_FWD, 2)
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "%s<%d>" % (dom["name"], variant),
                "work": "%d FP32 ops per contributing pair x %d contributing + %d per other entry up to the "
                        "last contributor x %d" % (RASTER_OPS_BWD if dom["name"] == "raster_bwd" else RASTER_OPS_FWD,
                                                   pairs[1], RASTER_OPS_TEST, pairs[0] - pairs[1]),
                "peak_source": "%d SMs (device attribute) x 128 FP32 lanes x 2 x max SM clock "
                               "(MEASURED_PEAKS sm_max_mhz)" % sms}

    # the visible-only Adam variant (off by default: it changes the
    # optimisation): the same steps call by call, with the fraction of
    # Gaussians that touch a tile in some view of the batch
    ctx.profile_reset()
    ctx.profile_enable(True)
    vis_frac = []
    for i in range(args.steps):
        tr.step(*batch(args.warmup + i), img, dimg, hp=dict(HP, visible_only=True))
        vm = ctx.gs_get_buffer(gs.GS_BUF_VISMASK)
        vis_frac.append(float((vm != 0).float().mean().item()))
    ctx.profile_enable(False)
    vk = {k["name"]: k for k in ctx.profile_read()}
    ctx.gs_sync()
    visible_only = {"visible_fraction": round(statistics.mean(vis_frac), 4),
                    "adam_ms": round(vk["adam"]["total_ms"] / args.steps, 3),
                    "project_bwd_ms": round(vk["project_bwd"]["total_ms"] / args.steps, 3),
                    "dense_adam_ms": round(per_kernel["adam"]["ms"] / args.steps, 3),
                    "dense_project_bwd_ms": round(per_kernel["project_bwd"]["ms"] / args.steps, 3),
                    "note": "per B-view step; the projection backward reads only the views where a Gaussian "
                            "touches a tile in both modes"}

    # the D-SSIM loss term (optional; the default training loss is L1) and the
    # paper's quality metrics on the last batch of those steps
    _, last_t = batch(args.warmup + args.steps - 1)
    dl = torch.zeros(1, device=dev)
    ctx.gs_ssim_loss(img, last_t, 0.2, dl, dimg)
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(5):
        ctx.gs_ssim_loss(img, last_t, 0.2, dl, dimg)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ssim_v, psnr_v = ctx.gs_image_metrics(img, last_t, B)
    dssim = {"ms_per_step": round(s0.elapsed_time(s1) / 5, 3), "lambda": 0.2,
             "ssim_mean": round(statistics.mean(ssim_v), 5), "psnr_mean_db": round(statistics.mean(psnr_v), 3),
             "note": "D-SSIM loss and gradient over the B views (kernels ssim_fwd, finish, ssim_bwd); SSIM / PSNR "
                     "of the trained set's render against the targets after the timed steps"}

    init = init_bench(ctx, scene, dev) if not args.no_init_bench else None

    # one adaptive-density-control step after a batch's statistic
    ga = torch.zeros(tr.n, device=dev)
    gc = torch.zeros(tr.n, device=dev)
    ctx.gs_set_densify_stats(ga, gc)
    tr.step(*batch(args.warmup), img, dimg)
    ctx.gs_set_densify_stats(None, None)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    noise = torch.randn((tr.n, 2, 3), device=dev, generator=gen)
    cap = 3 * tr.p.shape[1]
    outs = [torch.empty((tr.p.shape[0], cap), device=dev) for _ in range(3)]
    dhp = dict(grad_threshold=2e-4, percent_dense=0.01, scene_extent=1.1 * 2.0, min_opacity=0.005, split_n=2)
    ctx.gs_densify(tr.p, tr.m, tr.v, tr.n, tr.deg, ga, gc, noise, dhp, *outs)  # warm-up
    torch.cuda.synchronize(dev)
    t_d = time.perf_counter()
    n_new = ctx.gs_densify(tr.p, tr.m, tr.v, tr.n, tr.deg, ga, gc, noise, dhp, *outs)
    torch.cuda.synchronize(dev)
    densify = {"gaussians_in": int(tr.n), "gaussians_out": int(n_new), "wall_ms": round(1e3 * (time.perf_counter() - t_d), 3),
               "hp": dhp, "note": "statistic from one B-view step; counting pass, scan, host read of the new size, "
                                  "emitting pass into a second set of parameters and moments"}
    del outs

    # plain path: one view per launch, Adam after each view
    ctx2 = gs.Context(local)
    tr2 = Trainer(ctx2, trained, dev)
    one_img = torch.empty(3 * args.res * args.res, device=dev)
    one_dimg = torch.empty_like(one_img)
    one_t = targets[0][:one_img.numel()]
    if args.fwd_variant or args.bwd_variant:
        for opt, val in tuned.items():
            ctx2.gs_set_option(opt, val)
    else:
        autotune.tune([ctx2], lambda: tr2.step([batch(0)[0][0]], one_t, one_img, one_dimg),
                      autotune.workload_key(tr2.n, cams[:1], 1), use_cache=not args.retune)
    for i in range(2):
        tr2.step([batch(0)[0][i]], targets[0][i * one_img.numel():(i + 1) * one_img.numel()], one_img, one_dimg)
    ctx2.gs_sync()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.plain_views):
        b = i % B
        tr2.step([batch(0)[0][b]], targets[0][b * one_img.numel():(b + 1) * one_img.numel()], one_img, one_dimg)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain = args.plain_views / (e0.elapsed_time(e1) / 1000.0)
    ctx2.close()

    # end to end through the host-buffer entry point: every step uploads its
    # targets from pinned host memory (overlapped with the previous step on
    # the library's copy stream) and reads its loss back to pinned memory
    # the same batches as the device-timed steps, each target batch pinned
    # once in host memory
    e2e_k = [(args.warmup + i) % len(order) for i in range(args.e2e_steps)]
    host_t = {k: targets[k].cpu().pin_memory() for k in sorted(set(e2e_k))}
    loss_h = [torch.empty(1, pin_memory=True) for _ in range(args.e2e_steps)]
    # untimed warm-up launches of this entry point (its copy stream, events
    # and device target buffers are created on first use), as for the
    # device-timed steps
    for i in range(max(2, args.warmup)):
        tr.t += 1
        k = e2e_k[i % len(e2e_k)]
        gctx.gs_train_graph_launch_host(cams[order[k] * B:(order[k] + 1) * B], host_t[k], tr.t, loss_h[0])
    gctx.gs_sync()
    torch.cuda.synchronize(dev)
    t_e0 = time.perf_counter()
    e0.record(stream)
    for i in range(args.e2e_steps):
        k = e2e_k[i]
        tr.t += 1
        gctx.gs_train_graph_launch_host(cams[order[k] * B:(order[k] + 1) * B], host_t[k], tr.t, loss_h[i])
    e1.record(stream)
    gctx.gs_sync()
    torch.cuda.synchronize(dev)
    e2e_wall = time.perf_counter() - t_e0
    e2e_dev = e0.elapsed_time(e1) / 1000.0
    e2e = args.e2e_steps * B * world / max(e2e_dev, e2e_wall)
    assert all(np.isfinite(float(x)) for x in loss_h)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "views/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded blob-isosurface scene, random-init perturbation of a reference set)",
        "config": config_dict(args, world),
        "plain_1view_views_per_s": round(plain, 3), "batched_over_plain": round(value / plain / world, 3),
        "e2e": {"value": round(e2e, 3), "unit": "views/s", "h2d_bytes_per_step": total * 4,
                "d2h_bytes_per_step": 4, "steps": args.e2e_steps,
                "device_ms_per_step": round(1e3 * e2e_dev / args.e2e_steps, 3),
                "host_wall_ms_per_step": round(1e3 * e2e_wall / args.e2e_steps, 3),
                "note": "the device-timed steps' batches; each step's targets uploaded from pinned host memory "
                        "on a copy stream and its loss read back; the slower of the two clocks counts"},
        "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": roof,
        "graph": "each timed step is one CUDA-graph launch of the whole step; per-kernel times and the roofline "
                 "come from the same steps launched call by call (%.3f ms/step)" % (ms_calls / args.steps),
        "instances_per_step": int(inst), "visible_pairs_per_step": vis_pairs,
        "pair_entries_per_step": int(pairs[0]),
        "contributing_pairs_per_step": int(pairs[1]), "sort_passes_executed": executed,
        "kernels": per_kernel, "visible_only_adam": visible_only, "dssim": dssim, "init": init, "densify": densify,
        "setup_s": round(time.time() - t0, 1), "tuned_options": {str(k): v for k, v in tuned.items()},
        "autotune_ms": autotune.report(key),
        "memory": memory,
    }
    if args.serve_sweep:
        tr.ctx.gs_sync()
        torch.cuda.synchronize(dev)
        sweep = []
        for rate in SERVE_RATES:
            b = serve_run(tr.p, tr.n, tr.deg, local, rate, args.serve_seconds, 2, 16)
            o = serve_run(tr.p, tr.n, tr.deg, local, rate, args.serve_seconds, 1, 1)
            b["one_request_per_launch"] = {k: o[k] for k in ("p50_ms", "p99_ms", "frames_per_s")}
            sweep.append(b)
        out["render_sweep"] = sweep
    elif args.serve_rate > 0:
        tr.ctx.gs_sync()
        torch.cuda.synchronize(dev)
        # the requested rate and one above what one request per launch sustains
        render = []
        for rate in sorted({args.serve_rate, args.serve_saturating_rate}):
            batched = serve_run(tr.p, tr.n, tr.deg, local, rate, args.serve_seconds, 2, 16)
            single = serve_run(tr.p, tr.n, tr.deg, local, rate, args.serve_seconds, 1, 1)
            render.append({"rate_req_per_s": rate, "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"],
                           "frames_per_s": batched["frames_per_s"], "batches": batched["batches"],
                           "retried_batches": batched["retried"], "overlapping_batch_pairs": batched["overlaps"],
                           "one_request_per_launch": {k: single[k] for k in ("p50_ms", "p99_ms", "frames_per_s")}})
        out["render"] = {"rates": render, "resolutions": ["%dx%d" % r for r in SERVE_RES],
                         "slots": 2, "max_batch_views": 16}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scene, trained, cams, args)
    gctx.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- initialisation

def init_bench(ctx, scene, dev):
    """Point-cloud initialisation on the GPU at the benchmark's scale: the
    initial Gaussians of the workload's 4M isosurface points (normals from
    the scene's rotations) against the scene builder's host k-d-tree scales,
    and the edge crossings of a 512^3 gyroid volume."""
    import torch
    from scipy.spatial import cKDTree
    p = scene["params"]
    n = scene["n"]
    pts = np.ascontiguousarray(p[0:3, :n].T)
    w, x, y, z = (p[6 + i, :n].astype(np.float64) for i in range(4))
    nrm = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], 1)  # R(q) e_z
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    tp, tn = torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)
    out = torch.zeros_like(torch.from_numpy(p)).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.gs_init_gaussians(tp, tn, out, n, scene["deg"])  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0.record()
    ctx.gs_init_gaussians(tp, tn, out, n, scene["deg"])
    e1.record()
    torch.cuda.synchronize(dev)
    gpu_s = time.perf_counter() - t0
    got = out[3, :n].cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    d, _ = cKDTree(pts.astype(np.float64)).query(pts.astype(np.float64), k=4, workers=-1)
    host_s = time.perf_counter() - t0
    ref = 0.5 * np.log(np.maximum(np.mean(d[:, 1:] ** 2, axis=1), 1e-14))
    err = np.abs(got - ref)
    # edge crossings of the gyroid sin x cos y + sin y cos z + sin z cos x = 0
    res = 512
    ax = torch.linspace(-2 * math.pi, 2 * math.pi, res, device=dev)
    zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
    vol = (torch.sin(xx) * torch.cos(yy) + torch.sin(yy) * torch.cos(zz) + torch.sin(zz) * torch.cos(xx)).contiguous()
    del zz, yy, xx
    h = float(ax[1] - ax[0])
    ctx.gs_iso_crossings(vol, 0.0, (-2 * math.pi,) * 3, (h,) * 3)  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    cp, _ = ctx.gs_iso_crossings(vol, 0.0, (-2 * math.pi,) * 3, (h,) * 3)
    torch.cuda.synchronize(dev)
    cross_s = time.perf_counter() - t0
    return {"gaussians": int(n), "gpu_init_ms": round(e0.elapsed_time(e1), 2), "gpu_init_wall_s": round(gpu_s, 3),
            "host_kdtree_knn_s": round(host_s, 2), "host_threads": os.cpu_count(),
            "log_scale_vs_host": {"median_abs": float(np.median(err)), "p999_abs": float(np.quantile(err, 0.999)),
                                  "max_abs": float(err.max())},
            "crossings_512cube": {"count": int(cp.shape[0]), "wall_s": round(cross_s, 3)},
            "note": "gs_init_gaussians: exact 3-NN scales on the GPU (grid + radix sort) and the parameter planes; "
                    "host: scipy cKDTree query of the same FP32 points (all cores); crossings: two passes "
                    "(count, emit) with a host read of the count in between"}


# ---------------------------------------------------------------- serving

SERVE_RES = [(512, 512), (1024, 1024), (2048, 2048), (3840, 2160)]
SERVE_RATES = [50.0, 100.0, 200.0, 500.0, 1000.0, 2000.0]


def serve_run(params, n, deg, device, rate, duration_s, slots, max_batch, seed=6):
    """Poisson arrivals at `rate` req/s for `duration_s`; each request a random
    orbit camera (radius 4) at a resolution drawn uniformly from SERVE_RES.
    Returns latency percentiles (submit -> poll-complete, host clock) and
    frames/s."""
    import torch
    from paper_2509_05216_gb300 import gs, inputs
    rng = np.random.default_rng(seed)
    srv = gs.Server(params, n, deg, device=device, slots=slots, max_batch_views=max_batch,
                    memory_budget_bytes=(24 << 30) * slots, output_pool_bytes=8 << 30,
                    max_view_pixels=max(w * h for w, h in SERVE_RES))
    k = max(1, int(rate * duration_s))
    gaps = rng.exponential(1.0 / rate, size=k)
    cams = []
    for i in range(k):
        w, h = SERVE_RES[rng.integers(0, len(SERVE_RES))]
        cams.append(inputs.random_orbit_camera(rng, 4.0, w, h))
    # warm-up: one request per resolution
    for w, h in SERVE_RES:
        t = srv.gs_serve_submit(inputs.random_orbit_camera(rng, 4.0, w, h))
        srv.gs_serve_poll(t)
        srv.gs_serve_release(t)
    sub = [0.0] * k
    done = [0.0] * k
    tickets = [None] * k
    ready = threading.Semaphore(0)

    def poller():
        for i in range(k):
            ready.acquire()
            st, _ = srv.gs_serve_poll(tickets[i])
            done[i] = time.perf_counter()
            srv.gs_serve_release(tickets[i])

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    nxt = t0
    for i in range(k):
        nxt += gaps[i]
        dt = nxt - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        while True:
            try:
                sub[i] = time.perf_counter()
                tickets[i] = srv.gs_serve_submit(cams[i])
                break
            except gs.GsError:
                time.sleep(0.0005)  # queue or pool full: back-pressure
        ready.release()
    th.join()
    t1 = max(done)
    lat = np.array(done) - np.array(sub)
    stats = srv.gs_serve_stats()
    spans, retried = srv.gs_serve_timeline()
    srv.close()
    # batch pairs in flight at the same time on the device timeline
    spans.sort()
    overlaps, ends = 0, []
    for a, b in spans:
        ends = [e for e in ends if e > a]
        overlaps += len(ends)
        ends.append(b)
    return {"rate": rate, "requests": k, "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
            "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
            "frames_per_s": round(k / (t1 - t0), 2), "batches": stats["batches"], "retried": retried,
            "overlaps": overlaps}


# ---------------------------------------------------------------- oracle (CPU) arm

def cpu_sample(trained, scene, cams, args, budget_s):
    """Time the FP64 oracle on a bounded sample of one training view: forward
    and gradient over a random subset of tiles (plus the projection of all
    Gaussians, which the oracle needs for any tile).  Returns views/s scaled
    by the tile fraction, the sample description and the thread count."""
    from oracle import oracle
    cam = cams[0]
    gw = (cam["width"] + 15) // 16
    ntiles = gw * ((cam["height"] + 15) // 16)
    rng = np.random.default_rng(0)
    order = rng.permutation(ntiles)

    def run(frac):
        want = np.zeros(ntiles, np.uint8)
        want[order[:max(1, int(round(ntiles * frac)))]] = 1
        t0 = time.time()
        img, _, _, _ = oracle.render(trained, cam, tile_want=want)
        ref, _, _, _ = oracle.render(scene, cam, tile_want=want)
        _, dimg = oracle.l1(img, ref)
        oracle.render_grad(trained, [cam], [dimg.reshape(img.shape)])
        return int(want.sum()), time.time() - t0

    # grow the sample until it takes about budget_s of CPU time (the
    # projection of every Gaussian is a fixed cost, so extrapolate twice)
    frac = 1.0 / 64.0
    used, dt = run(frac)
    for _ in range(2):
        if frac >= 1.0 or dt >= 0.6 * budget_s:
            break
        frac = min(1.0, frac * budget_s / max(dt, 1e-3))
        used, dt = run(frac)
    return {"value": round((used / ntiles) / dt, 6), "unit": "views/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "one %dx%d view of the training workload: forward of the trained and the reference set, L1 "
                      "gradient and backward over %d of %d tiles (%.1f s), scaled by the tile fraction; "
                      "projection of all %d Gaussians included"
                      % (cam["width"], cam["height"], used, ntiles, dt, trained["n"])}


def cpu_baseline(scene, trained, cams, args):
    return cpu_sample(trained, scene, cams, args, args.cpu_seconds)


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene, trained, cams = workload(args, device=None)
    samples = []
    for _ in range(args.warmup):
        pass
    for _ in range(max(1, min(args.steps, 2))):
        samples.append(cpu_sample(trained, scene, cams, args, args.cpu_seconds))
    v = statistics.median(s["value"] for s in samples)
    out = {"metric": METRIC, "value": v, "unit": "views/s", "n_gpus": world, "steps": len(samples),
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "config": config_dict(args, world), "impl": "reference",
           "cpu_baseline": {"value": v, "unit": "views/s", "cores": samples[0]["cores"], "kind": "oracle",
                            "sample": samples[0]["sample"]},
           "e2e": {"value": v, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
