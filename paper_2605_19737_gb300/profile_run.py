"""Render a named workload a few times (for Nsight Compute captures and quick timing).

    python -m paper_2605_19737_gb300.profile_run --workload brainweb_1080p --kernel gather --frames 3

Workloads: brainweb_1080p (181x217x181 uint16, 1920x1080), brainweb_540p (same
volume, 960x540), head64 (64^3 float32, 128x128), diff_head128_8cam (128^3
float32, 8 cameras at 512x512). Prints the mean frame time
from CUDA events (a number taken under a profiler is not a benchmark value).
"""

import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import paper_2605_19737_gb300 as pkg
    from phantoms import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="brainweb_1080p",
                    choices=["brainweb_1080p", "brainweb_540p", "head64", "diff_head128_8cam", "vessel_1080p",
                             "batched"])
    ap.add_argument("--kernel", default="gather", choices=["gather", "staged", "stencil", "staged_derived"])
    ap.add_argument("--brick", type=int, default=8, help="skip-brick edge in cells (4, 8 or 16)")
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--packet-w", type=int, default=4)
    ap.add_argument("--warps", type=int, default=4)
    ap.add_argument("--backward", action="store_true", help="also run the adjoint raymarch after each frame")
    ap.add_argument("--cams-per-volume", type=int, default=8,
                    help="batched: orbit cameras per volume (the benchmark uses 64)")
    ap.add_argument("--precompute-reps", type=int, default=1,
                    help="run the morphology precompute this many times (timed with CUDA events)")
    args = ap.parse_args()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "head64":
        case = workloads.head64_128px()
    elif args.workload == "diff_head128_8cam":
        case = workloads.diff_head128_8cam()
    elif args.workload == "vessel_1080p":
        case = workloads.vessel_1080p()
    elif args.workload == "brainweb_540p":
        case = workloads.brainweb_1080p(width=960, height=540)
    else:
        case = workloads.brainweb_1080p()
    kernel = {"gather": pkg.VR_KERNEL_GATHER, "staged": pkg.VR_KERNEL_STAGED,
              "stencil": pkg.VR_KERNEL_GATHER_STENCIL, "staged_derived": pkg.VR_KERNEL_STAGED_DERIVED}[args.kernel]
    vol = case["volume"]
    data = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
    with pkg.Context(0) as ctx:
        vid = ctx.load_volume(data, case["spacing"])
        ctx.set_brick_size(vid, args.brick)
        tp = []
        for _ in range(args.precompute_reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            ctx.precompute_morphology(vid, case["sigmas"])
            e.record()
            ctx.synchronize()
            tp.append(s.elapsed_time(e))
        print("%s precompute (sigmas %s): %.3f ms (last of %d)" % (args.workload, case["sigmas"], tp[-1], len(tp)))
        ctx.set_tissue_params(vid, case["tf"], **case["params"])
        out = torch.empty((case["cams"].shape[0], case["H"], case["W"], 4), device="cuda")
        dl = torch.randn(out.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
        # with --backward the forward records the per-ray state the backward starts from
        state = torch.empty(out.shape[:3] + (2,), device="cuda") if args.backward else None
        ts, tb = [], []
        for _ in range(args.frames):
            s, e, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            s.record()
            ctx.render(vid, case["cams"], case["W"], case["H"], out=out, kernel=kernel, packet_w=args.packet_w,
                       warps_per_block=args.warps, ray_state=state)
            e.record()
            if args.backward:
                ctx.render_backward(vid, case["cams"], case["W"], case["H"], dl, kernel=kernel, ray_state=state)
            b.record()
            ctx.synchronize()
            ts.append(s.elapsed_time(e))
            tb.append(e.elapsed_time(b))
    print("%s %s: %.3f ms/frame (mean of %d)" % (args.workload, args.kernel, float(np.mean(ts)), len(ts)))
    if args.backward:
        print("%s %s backward: %.3f ms/frame" % (args.workload, args.kernel, float(np.mean(tb))))


def run_batched(args):
    """The benchmark's batched workload (4 uneven volumes, 512x512 views) with fewer
    cameras per volume, rendered by the persistent batch kernel (4x8 packets, 4 warps
    per CTA: the autotuned shape) --frames times."""
    import torch

    import paper_2605_19737_gb300 as pkg
    from phantoms import workloads

    cases = workloads.batched_4vol_64cam(n_cams=args.cams_per_volume)
    with pkg.Context(0) as ctx:
        vids, views = [], []
        for case in cases:
            vid = ctx.load_volume(torch.from_numpy(case["volume"]).cuda(), case["spacing"])
            ctx.precompute_morphology(vid)
            ctx.set_tissue_params(vid, case["tf"], **case["params"])
            vids.append(vid)
            for c in range(case["cams"].shape[0]):
                views.append((vid, case["cams"][c], torch.empty((case["H"], case["W"], 4), device="cuda"),
                              case["W"], case["H"]))
        bid = ctx.batch_create(views)
        ts = []
        for _ in range(args.frames):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            ctx.batch_render(bid, packet_w=4, warps_per_block=4)
            e.record()
            ctx.synchronize()
            ts.append(s.elapsed_time(e))
        ctx.batch_free(bid)
        for vid in vids:
            ctx.free_volume(vid)
    print("batched %d views: %.3f ms/batch (mean of %d)" % (len(views), float(np.mean(ts)), len(ts)))


if __name__ == "__main__":
    main()
