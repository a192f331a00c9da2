"""Benchmark of the GB300 direct-volume-rendering path.

Workload: the BrainWeb-shaped 181x217x181 uint16 T1 phantom rendered at
1920x1080 (2D transfer function over intensity x gradient magnitude with
curvature-modulated opacity, 8^3-brick empty-space skipping, step 0.5 voxel).
A step is one frame: one vr_render call over the resident volume.

  value  dense-equivalent Gsamples/s of the forward raymarch, inputs resident in
         HBM, L2 flushed (256 MB write) between timed frames, CUDA events on
         the context's stream, max over ranks, summed over ranks (weak scaling:
         every rank renders its own orbit view of its own copy of the volume).
  e2e    the same metric through the C ABI with host buffers: per frame the
         tissue uniforms and transfer function are uploaded from host memory
         and the image is copied back to pinned host memory.
Also reported (not timed in the step): fps_wall (vr_render wall clock, launch
included), fwd+bwd on the same 1080p view, fwd+bwd over the 8 views of the
differentiable 128^3 workload, the batched persistent render (4 volumes x 64
cameras, CUDA graph), the vesselness precompute, time to first pixel, and the
roofline of the forward kernel against a measured FP32 FMA peak, the 1080p render
of the vessel volume through its (I, V) table, the 64^3 head at 128x128, and the
200-step transfer-function fit (--no-fit skips it). Run `python bench.py --impl reference` for the
FP64 CPU oracle on the same workload (a bounded sample of the frame).
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsamples/s & FPS at 1080p (fwd, fwd+bwd) vs plain fwd, % of HBM roofline"
UNIT = "Gsamples/s"
L2_FLUSH_BYTES = 256 << 20
# FP32 operations per sample of the raymarch.
# The survey's per-unit figure for the method (per-sample trilinear I, gradient and
# Hessian, curvature, Eq. 4, shading, Eqs. 5-6): ~400 FP32 FLOP per evaluated sample.
# This is what `roofline.achieved` counts.
FLOPS_PER_SAMPLE_SURVEY = 400
# The count of the arithmetic this implementation does, from the algorithm.
# Derived bricks (voxel-wise I, gradient, Hessian), in two stages:
#   every interpolated sample (evaluated, and not in a cell classified empty):
#   position (18), trilinear weights (19), 8 corners x
#   (I, g) FMA (64), |g| and the unit normal (11), 2D bilinear transfer function
#   (36) = 148;
#   samples with a non-zero transfer-function opacity ("shaded") also: 8 corners x
#   6 Hessian channels FMA (96), curvature (27), Eq. 4 (8), Phong (16), Eqs. 5-6 (8)
#   = 155 (303 in all).
# Per-sample stencils (stencil and staged kernels; every evaluated sample shaded):
# the 56-voxel separable contraction (368 incl. the 4-tap weights) + spacing scale
# (15) in place of the 179 of the derived interpolation: 124 + 383 = 507.
FLOPS_STAGE1 = {"gather": 148, "stencil": 0, "staged": 0}
FLOPS_SHADED = {"gather": 155, "stencil": 507, "staged": 507}
KERNEL_SOURCES = ("paper_2605_19737_gb300/csrc/vr_render.cu", "paper_2605_19737_gb300/csrc/vr_march.cuh",
                  "paper_2605_19737_gb300/csrc/vr_sample.cuh", "paper_2605_19737_gb300/csrc/vr_internal.cuh")


def kernel_source_hash():
    """sha256 over the code (comments and blank lines removed) of the forward
    raymarch kernel's sources."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            code = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = "\n".join(ln.split("//")[0].rstrip() for ln in code.splitlines())
        h.update("\n".join(ln for ln in code.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def measured_traffic():
    """DRAM bytes per launch of k_render_gather on the benchmark frame, from the ncu
    capture recorded in profiles/traffic_gather_brainweb_1080p.json -- only while the
    kernel sources still hash to what was profiled; None otherwise."""
    p = os.path.join(ROOT, "profiles", "traffic_gather_brainweb_1080p.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    return d.get("dram_bytes_per_launch") if d.get("kernel_source_hash") == kernel_source_hash() else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        busy = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        return {"sm_mhz": float(np.median(busy)) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _json_line(d):
    print(json.dumps(d), flush=True)


def cpu_baseline(case, stride, threads=None, min_seconds=0.0):
    """Time the FP64 oracle on every `stride`-th row/column of the frame, repeating
    the render until at least `min_seconds` have passed (one render at least)."""
    import oracle
    from tests.gpu_util import oracle_params
    if threads:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    In = oracle.normalize(case["volume"])
    t0 = time.perf_counter()
    dense, reps = 0, 0
    while True:
        res = oracle.render(In, case["spacing"], oracle_params(case["params"], case["tf"]), case["tf"], case["cams"],
                            case["W"], case["H"], pix_stride=stride, alternatives=False)
        dense += int(res.dense.sum())
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    rays = len(range(0, case["H"], stride)) * len(range(0, case["W"], stride))
    nth = {2: "2nd", 3: "3rd"}.get(stride, "%dth" % stride)
    part = ("every %s row and column of the %dx%d frame" % (nth, case["W"], case["H"]) if stride > 1
            else "the whole %dx%d frame" % (case["W"], case["H"]))
    return {"value": dense / dt / 1e9, "unit": UNIT, "cores": int(res.threads), "kind": "oracle",
            "sample": "%s (%d rays, %d dense samples per render) x %d renders, including the oracle's "
                      "voxel-derivative setup, %.1f s" % (part, rays, dense // reps, reps, dt),
            "seconds": dt, "dense_samples": dense}


def workload_config(args, ws):
    """The benchmark workload, as both arms report it (the same object in both)."""
    return {"workload": "brainweb_1080p", "volume": "181x217x181 u16 (BrainWeb-shaped phantom)",
            "image": "1920x1080", "tf": "2D 256x64 (I, |g|/gmax), Table 2 windows", "step_vox": 0.5,
            "l2": "flushed between frames (256 MB write)",
            "parallelism": "replicas" if ws > 1 else "single"}


def run_reference(args):
    from phantoms import workloads
    ws, rank, _ = _dist()
    if rank != 0:
        return
    case = workloads.brainweb_1080p()
    # each step renders every stride-th row and column of the frame (about 0.6 s on
    # 16 cores at stride 2), so that warm-up + timed steps end within a few minutes
    n = args.warmup + args.steps
    stride = 2 if n <= 300 else (4 if n <= 1200 else 8)
    vals, last = [], None
    for i in range(args.warmup + args.steps):
        last = cpu_baseline(case, stride)
        if i >= args.warmup:
            vals.append(last["value"])
    v = float(np.mean(vals))
    cb = dict(last, value=v)
    _json_line({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * last["seconds"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args, args.gpus),
                "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}})


def fwd_bwd_multiview(ctx, dev, flush, args):
    """Forward + backward over the 8 views of the differentiable workload (128^3 head,
    512x512): transfer-function, uniform and voxel gradients, as one fit step
    computes them (without the optimiser)."""
    import torch

    import paper_2605_19737_gb300 as pkg
    from phantoms import workloads as wl
    case = wl.diff_head128_8cam()
    W, H, cams = case["W"], case["H"], case["cams"]
    vid = ctx.load_volume(torch.from_numpy(case["volume"]).to(dev), case["spacing"])
    ctx.precompute_morphology(vid)
    ctx.set_tissue_params(vid, case["tf"], **case["params"])
    out = torch.empty((cams.shape[0], H, W, 4), device=dev)
    # the forward's brick size and launch shape tuned on the stateless render; the
    # backward runs on the same bricks
    shape, tuned = tune_case(ctx, vid, case, "diff_head128_8cam", out)
    ctr = pkg.new_counters(dev.index or 0)
    ctx.render(vid, cams, W, H, out=out, counters=ctr, **shape)
    torch.cuda.synchronize()
    dense = int(ctr.cpu().numpy()[1])
    dl = torch.randn(out.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(20260523))
    dtf = torch.empty(tuple(case["tf"].shape), device=dev)
    dpar = torch.empty(5, device=dev)
    dvol = torch.empty(case["volume"].shape, device=dev)
    state = torch.empty((cams.shape[0], H, W, 2), device=dev)
    ts = []
    for i in range(args.warmup + max(3, min(20, args.steps // 4))):
        flush.zero_()
        s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s0.record()
        ctx.render(vid, cams, W, H, out=out, ray_state=state, **shape)
        s1.record()
        ctx.render_backward(vid, cams, W, H, dl, dtf=dtf, dparams=dpar, dvol=dvol, ray_state=state)
        s2.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append((s0.elapsed_time(s1), s1.elapsed_time(s2)))
    ctx.free_volume(vid)
    f_ms, b_ms = (float(np.mean([x[q] for x in ts])) for q in (0, 1))
    return {"workload": "diff_head128_8cam: 128^3 float32 head, 8 cameras, 512x512, 1D TF 256",
            "dense_samples": dense, "fwd_ms": f_ms, "bwd_ms": b_ms, "tuned": tuned,
            "fwd_gsamples_per_s": dense / (f_ms * 1e-3) / 1e9,
            "fwd_bwd_gsamples_per_s": dense / ((f_ms + b_ms) * 1e-3) / 1e9}


def tune_case(ctx, vid, case, key, out):
    """Autotune one workload's single-call render (skip-brick edge x packet x CTA
    size) on this GPU, leaving the chosen brick size set on the volume. Returns the
    launch shape and the choice (without the per-candidate timings)."""
    from paper_2605_19737_gb300 import autotune
    n, H, W = case["cams"].shape[0], case["H"], case["W"]

    def prepare(cells):
        ctx.set_brick_size(vid, cells)
        ctx.precompute_morphology(vid, case.get("sigmas", ()))
        ctx.set_tissue_params(vid, case["tf"], **case["params"])
    t = autotune.tune_render(ctx, vid, case["cams"], W, H, key, prepare=prepare, force=True, out=out)
    return ({"packet_w": t["packet_w"], "warps_per_block": t["warps_per_block"]},
            {k: t[k] for k in ("brick", "packet_w", "warps_per_block")})


def timed_view(ctx, vid, case, flush, args, kernel, label, key):
    """Forward render of one named workload's views at its autotuned launch: CUDA-event
    time per frame (L2 flushed between frames), dense-equivalent Gsamples/s and FPS."""
    import torch

    import paper_2605_19737_gb300 as pkg
    dev = flush.device
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    out = torch.empty((n, H, W, 4), device=dev)
    shape, tuned = tune_case(ctx, vid, case, key, out)
    ctr = pkg.new_counters(dev.index or 0)
    ctx.render(vid, case["cams"], W, H, out=out, kernel=kernel, counters=ctr, **shape)
    torch.cuda.synchronize()
    c = [int(x) for x in ctr.cpu().numpy()[:6]]
    ts = []
    for i in range(args.warmup + max(5, min(20, args.steps))):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        ctx.render(vid, case["cams"], W, H, out=out, kernel=kernel, **shape)
        e.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(s.elapsed_time(e))
    ms = float(np.mean(ts))
    return {"workload": label, "ms_per_frame": ms, "fps": 1000.0 * n / ms, "dense_samples": c[1],
            "evaluated_samples": c[2], "gsamples_per_s": c[1] / (ms * 1e-3) / 1e9, "tuned": tuned}


def run_batched(args, ctx, dev, flush):
    """Four uneven volumes x 64 orbit cameras at 512x512 in one persistent launch,
    replayed from a CUDA graph with the autotuned packet shape, beside the same 256
    views rendered one vr_render call at a time."""
    import torch

    import paper_2605_19737_gb300 as pkg
    from paper_2605_19737_gb300 import autotune
    from phantoms import workloads

    cases = workloads.batched_4vol_64cam()
    vids, views = [], []
    for case in cases:
        vid = ctx.load_volume(torch.from_numpy(case["volume"]).to(dev), case["spacing"])
        ctx.precompute_morphology(vid)
        ctx.set_tissue_params(vid, case["tf"], **case["params"])
        vids.append(vid)
        for c in range(case["cams"].shape[0]):
            out = torch.empty((case["H"], case["W"], 4), device=dev)
            views.append((vid, case["cams"][c], out, case["W"], case["H"]))
    bid = ctx.batch_create(views)

    def prepare(cells):  # skip-brick edge of every volume of the batch
        for vid, case in zip(vids, cases):
            ctx.set_brick_size(vid, cells)
            ctx.precompute_morphology(vid)
            ctx.set_tissue_params(vid, case["tf"], **case["params"])
        ctx.batch_update(bid)
    tune = autotune.tune_batch(ctx, bid, "batched_4vol_64cam_512", reps=2, force=True, prepare=prepare,
                               candidates=[(4, 4), (4, 8), (8, 4), (16, 4)])
    pw, wpb = tune["packet_w"], tune["warps_per_block"]
    ctr = pkg.new_counters(dev.index)
    ctx.batch_render(bid, packet_w=pw, warps_per_block=wpb, counters=ctr)
    torch.cuda.synchronize()
    dense = int(ctr[1])
    for _ in range(args.warmup):
        ctx.batch_render(bid, packet_w=pw, warps_per_block=wpb, graph=True)
    ts = []
    for _ in range(max(3, min(10, args.steps // 2))):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        ctx.batch_render(bid, packet_w=pw, warps_per_block=wpb, graph=True)
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    batch_ms = float(np.mean(ts))
    single = []
    for _ in range(2):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for vid, cam, out, W, H in views:
            ctx.render(vid, cam, W, H, out=out.view(1, H, W, 4))
        e.record()
        torch.cuda.synchronize()
        single.append(s.elapsed_time(e))
    single_ms = float(np.min(single))
    ctx.batch_free(bid)
    for vid in vids:
        ctx.free_volume(vid)
    return {"workload": "batched_4vol_64cam: 96^3, 128x160x128, 181x217x181, 256x256x176 float32; "
                        "64 orbit cameras each; 512x512", "views": len(views), "dense_samples": dense,
            "gsamples_per_s": dense / (batch_ms * 1e-3) / 1e9, "ms_per_batch": batch_ms,
            "launch": "one persistent kernel from a CUDA graph",
            "autotuned": {"packet_w": pw, "warps_per_block": wpb, "brick": tune["brick"],
                          "timings_ms": tune["timings"]},
            "single_view_gsamples_per_s": dense / (single_ms * 1e-3) / 1e9, "single_view_ms": single_ms}


def run(args):
    import torch
    import torch.distributed as dist

    import paper_2605_19737_gb300 as pkg
    from phantoms import cameras, workloads

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = workloads.brainweb_1080p(az=30.0 + 45.0 * rank)
    W, H = case["W"], case["H"]
    vol_np = case["volume"]
    vol_host = torch.from_numpy(vol_np.view(np.int16)).pin_memory()
    ctx = pkg.Context(local)

    # Time-to-first-pixel analogue: host volume -> load -> morphology -> params -> first frame on the host.
    img_host = torch.empty((1, H, W, 4), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vid0 = ctx.load_volume(vol_host, case["spacing"])
    ctx.precompute_morphology(vid0)
    ctx.set_tissue_params(vid0, case["tf"], **case["params"])
    ctx.render(vid0, case["cams"], W, H, out=img_host)
    ctx.synchronize()
    ttfp_ms = 1000.0 * (time.perf_counter() - t0)
    ctx.free_volume(vid0)

    vid = ctx.load_volume(vol_host.to(dev), case["spacing"])
    ctx.precompute_morphology(vid)
    ctx.set_tissue_params(vid, case["tf"], **case["params"])
    out = torch.empty((1, H, W, 4), dtype=torch.float32, device=dev)
    ctr = pkg.new_counters(local)
    ctx.render(vid, case["cams"], W, H, out=out, counters=ctr)
    torch.cuda.synchronize()
    rays, dense, evald, _, shaded, interp = [int(x) for x in ctr.cpu().numpy()[:6]]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    kernel = {"gather": pkg.VR_KERNEL_GATHER, "staged": pkg.VR_KERNEL_STAGED,
              "stencil": pkg.VR_KERNEL_GATHER_STENCIL}[args.kernel]
    # launch shape and skip-brick edge of the forward, tuned on this frame (the image
    # does not depend on them)
    shape = {"packet_w": 4, "warps_per_block": 4}
    tuned = None
    if args.kernel == "gather":
        from paper_2605_19737_gb300 import autotune

        def prepare(cells):
            ctx.set_brick_size(vid, cells)
            ctx.precompute_morphology(vid)
            ctx.set_tissue_params(vid, case["tf"], **case["params"])
        tuned = autotune.tune_render(ctx, vid, case["cams"], W, H, "brainweb_1080p", prepare=prepare, force=True,
                                     out=out)
        shape = {"packet_w": tuned["packet_w"], "warps_per_block": tuned["warps_per_block"]}
        ctx.render(vid, case["cams"], W, H, out=out, counters=ctr.zero_(), **shape)
        torch.cuda.synchronize()
        rays, dense, evald, _, shaded, interp = [int(x) for x in ctr.cpu().numpy()[:6]]

    def frame():
        ctx.render(vid, case["cams"], W, H, out=out, kernel=kernel, **shape)

    for _ in range(args.warmup):
        flush.zero_()
        frame()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    time.sleep(0.3)  # let the sampler start before the timed region
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s, e in evs:
        flush.zero_()
        s.record()
        frame()
        e.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = float(np.mean([s.elapsed_time(e) for s, e in evs]))
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        tot = torch.tensor([float(dense)], device=dev, dtype=torch.float64)
        dist.all_reduce(tot)
        dense_all = float(tot.item())
    else:
        dense_all = float(dense)
    value = dense_all / (ms * 1e-3) / 1e9

    # Wall-clock frame rate of vr_render (launch included) on a warm context, device output.
    walls = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        frame()
        ctx.synchronize()
        if i >= args.warmup:
            walls.append(time.perf_counter() - t1)
    fps_wall = 1.0 / float(np.mean(walls))

    # End to end through the C ABI with host buffers: uniforms + TF from pinned host
    # memory, image back to pinned host memory.
    tf_host = torch.from_numpy(np.ascontiguousarray(case["tf"])).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.set_tissue_params(vid, tf_host, **case["params"])
        ctx.render(vid, case["cams"], W, H, out=img_host, kernel=kernel, **shape)
        ctx.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t1)
    e2e_s = float(np.mean(e2e_times))
    if ws > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = dense_all / e2e_s / 1e9

    # Forward + backward on the same view: dL/dRGBA is a fixed seeded upstream gradient;
    # the backward returns transfer-function, uniform and voxel gradients.
    fwd_bwd = None
    if not args.no_backward:
        g = torch.Generator(device=dev).manual_seed(20260519)
        dl = torch.randn((1, H, W, 4), device=dev, generator=g)
        dtf = torch.empty(tuple(case["tf"].shape), device=dev)
        dpar = torch.empty(5, device=dev)
        dvol = torch.empty(vol_np.shape, device=dev)
        state = torch.empty((1, H, W, 2), device=dev)
        fb = []
        for i in range(args.warmup + max(3, min(20, args.steps // 4))):
            flush.zero_()
            s0, s1, s2, s3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            s0.record()
            ctx.render(vid, case["cams"], W, H, out=out, kernel=kernel, ray_state=state, **shape)
            s1.record()
            ctx.render_backward(vid, case["cams"], W, H, dl, dtf=dtf, dparams=dpar, dvol=dvol, ray_state=state)
            s2.record()
            ctx.render_backward(vid, case["cams"], W, H, dl, dtf=dtf, dparams=dpar, dvol=dvol)
            s3.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                fb.append((s0.elapsed_time(s1), s1.elapsed_time(s2), s2.elapsed_time(s3)))
        f_ms, b_ms, r_ms = (float(np.mean([x[q] for x in fb])) for q in (0, 1, 2))
        fwd_bwd = {"gsamples_per_s": dense_all / ((f_ms + b_ms) * 1e-3) / 1e9, "ms_per_step": f_ms + b_ms,
                   "fwd_ms": f_ms, "bwd_ms": b_ms, "fps": 1000.0 / (f_ms + b_ms),
                   "bwd_ms_re_march": r_ms,
                   "grads": "transfer function 256x64x4, 5 uniforms, 181x217x181 voxels",
                   "note": "forward records per-ray state (last sample, transmittance), the backward starts "
                           "its reverse sweeps there; bwd_ms_re_march: the backward re-marching each ray instead",
                   "plain_fwd_gsamples_per_s": value}

    # Per-volume vesselness precompute (sigma 1, 2, 3) on the 256x256x176 vessel phantom,
    # then the 1080p render of that volume through its (I, V) transfer function.
    precompute = vessel = head64 = None
    if not args.no_batch:
        vcase = workloads.vessel_1080p()
        vvid = ctx.load_volume(torch.from_numpy(vcase["volume"]).to(dev), vcase["spacing"])
        pre = []
        for _ in range(4):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            ctx.precompute_morphology(vvid, vcase["sigmas"])
            s1.record()
            torch.cuda.synchronize()
            pre.append(s0.elapsed_time(s1))
        precompute = {"workload": "vessel 256x256x176 float32, Frangi sigma 1, 2, 3 + |grad I|max",
                      "ms": float(np.median(pre[1:]))}
        ctx.set_tissue_params(vvid, vcase["tf"], **vcase["params"])
        vessel = timed_view(ctx, vvid, vcase, flush, args, kernel,
                            "vessel_1080p: 256x256x176 float32 vessel tree, 2D TF over (I, V), Phong, 1920x1080",
                            "vessel_1080p")
        ctx.free_volume(vvid)
        hcase = workloads.head64_128px()
        hvid = ctx.load_volume(torch.from_numpy(hcase["volume"]).to(dev), hcase["spacing"])
        ctx.precompute_morphology(hvid)
        ctx.set_tissue_params(hvid, hcase["tf"], **hcase["params"])
        head64 = timed_view(ctx, hvid, hcase, flush, args, kernel,
                            "head64_128px: 64^3 float32 head, 1D TF, Phong, 128x128", "head64_128px")
        ctx.free_volume(hvid)

    batched = None if args.no_batch else run_batched(args, ctx, dev, flush)
    multiview = None if args.no_backward else fwd_bwd_multiview(ctx, dev, flush, args)
    fit = None
    if not args.no_fit and ws == 1:
        from paper_2605_19737_gb300 import fit as fitmod
        fit = fitmod.run(steps=200)
    hbm, smax, peak_kind = _peaks()
    kind = args.kernel
    nbricks, _, derived_bytes = ctx.get_layout(vid)
    if kind == "gather" and derived_bytes == 0:
        kind = "stencil"  # derived bricks are not built above the memory budget
    # algorithmic bytes of a frame: the voxels at their stored dtype (u16; every voxel
    # once, an upper bound of what a frame touches) plus the RGBA float32 image it writes
    vox_bytes = int(vol_np.size * vol_np.dtype.itemsize)
    frame_bytes = vox_bytes + W * H * 16
    traffic = measured_traffic()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or smax
    fp32_nominal = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    fma_ms, fma_flops = ctx.fma_peak()
    fp32_peak = fma_flops / 1e12
    # algorithmic: the survey's per-sample figure for the method times every evaluated
    # sample (the samples outside empty bricks); builder count: this implementation's
    # own per-sample arithmetic; executed: what the kernel ran after its exact skips
    # (empty cells, zero-opacity samples)
    frame_flops = evald * FLOPS_PER_SAMPLE_SURVEY
    builder_flops = evald * (FLOPS_STAGE1[kind] + FLOPS_SHADED[kind])
    executed_flops = interp * FLOPS_STAGE1[kind] + shaded * FLOPS_SHADED[kind]
    achieved_tflops = frame_flops / (ms * 1e-3) / 1e12
    if rank == 0:
        cb = None
        if ws == 1 and not args.no_cpu_baseline:
            cb = cpu_baseline(workloads.brainweb_1080p(), stride=1, min_seconds=10.0)
            cb.pop("seconds", None)
            # and the whole small head frame (64^3, 128x128, 1D TF), every pixel
            small = cpu_baseline(workloads.head64_128px(), stride=1)
            cb["head64_128px_full_frame"] = {"value": small["value"], "unit": UNIT,
                                             "seconds": small["seconds"], "dense_samples": small["dense_samples"]}
        _json_line({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, ws), "kernel": args.kernel,
            "tuned": None if tuned is None else {k: tuned[k] for k in ("packet_w", "warps_per_block", "brick",
                                                                       "timings")},
            "fps": 1000.0 / ms, "fps_wall": fps_wall,
            "samples": {"dense_per_frame": dense, "evaluated_per_frame": evald, "interpolated_per_frame": interp,
                        "shaded_per_frame": shaded, "rays": rays},
            "ttfp_ms": ttfp_ms,
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved_tflops / fp32_peak, "traffic": traffic,
                         "flops_per_evaluated_sample": FLOPS_PER_SAMPLE_SURVEY,
                         "algorithmic_flops_per_frame": frame_flops,
                         "builder_flops_per_evaluated_sample": FLOPS_STAGE1[kind] + FLOPS_SHADED[kind],
                         "frac_builder_count": builder_flops / (ms * 1e-3) / 1e12 / fp32_peak,
                         "executed_flops_per_frame": executed_flops,
                         "executed_tflops": executed_flops / (ms * 1e-3) / 1e12,
                         "frac_executed": executed_flops / (ms * 1e-3) / 1e12 / fp32_peak,
                         "peak_source": "measured: FP32 FMA probe vr_fma_peak (8 independent chains per thread, "
                                        "%.3f ms per launch); nominal %d SMs x 128 lanes x 2 x %.0f MHz = %.1f"
                                        % (fma_ms, props.multi_processor_count, sm_mhz, fp32_nominal)},
            "hbm_roofline": {"achieved": frame_bytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": frame_bytes / (ms * 1e-3) / 1e9 / hbm, "frac_vs_8tbs":
                             frame_bytes / (ms * 1e-3) / 1e9 / 8000.0, "bytes_per_frame": frame_bytes,
                             "bytes": "algorithmic: %d voxels x %d B (u16, each once) + %dx%d RGBA float32 image"
                                      % (vol_np.size, vol_np.dtype.itemsize, W, H),
                             "layout_bytes_derived_store": derived_bytes, "bricks": nbricks,
                             "measured_dram_bytes_per_launch": traffic,
                             "measured_over_algorithmic": (traffic / frame_bytes) if traffic else None,
                             "peak_source": peak_kind},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(tf_host.numel() * 4 + 48),
                    "d2h_bytes_per_step": int(W * H * 16), "ms_per_step": 1000.0 * e2e_s},
            "fwd_bwd": fwd_bwd,
            "vessel_1080p": vessel,
            "head64": head64,
            "batched": batched,
            "fwd_bwd_multiview": multiview,
            "precompute": precompute,
            "fit": fit,
            "gpu_launches": args.steps,  # one raymarch kernel per timed frame
            "clocks": clk,
            "cpu_baseline": cb,
        })
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default="gather", choices=["gather", "staged", "stencil"])
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-fit", action="store_true", help="skip the 200-step transfer-function fit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
