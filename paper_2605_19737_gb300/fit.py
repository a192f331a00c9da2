"""Fit transfer-function entries to target views through the differentiable renderer.

The paper tunes tissue parameters interactively (uniform buffers, Sec. 4);
with the adjoint raymarch the same parameters can be fitted to a target image:
MSE between renders of n cameras and targets, Adam on sigmoid-parameterised
transfer-function entries. Forward and backward both run in libvr.so.

    python -m paper_2605_19737_gb300.fit --steps 200
"""

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def fit_transfer_function(ctx, vol, cams, W, H, tf0, target, fixed, params, steps=200, lr=1e-2):
    """Returns (fitted tf, per-step losses, mean ms per step measured with CUDA events)."""
    import torch

    from . import autograd as ag

    logit = torch.logit(tf0.clamp(1e-4, 1.0 - 1e-4)).detach().requires_grad_(True)
    opt = torch.optim.Adam([logit], lr=lr)
    losses, times = [], []
    for _ in range(steps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        opt.zero_grad(set_to_none=True)
        img = ag.render(ctx, vol, torch.sigmoid(logit), params, cams, W, H, fixed)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
        e.record()
        losses.append(loss.detach())
        times.append((s, e))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in times[1:]) / max(1, len(times) - 1)
    return torch.sigmoid(logit).detach(), [float(x) for x in losses], ms


def run(steps=200, lr=1e-2):
    import numpy as np
    import torch

    import paper_2605_19737_gb300 as pkg
    from phantoms import workloads
    from . import autograd as ag

    case = workloads.diff_head128_8cam()
    W, H = case["W"], case["H"]
    with pkg.Context(0) as ctx:
        vid = ctx.load_volume(torch.from_numpy(case["volume"]).cuda(), case["spacing"])
        ctx.precompute_morphology(vid)
        fixed = {k: v for k, v in case["params"].items() if k not in ag.PARAM_NAMES}
        params = torch.tensor([case["params"][k] for k in ag.PARAM_NAMES], dtype=torch.float32)
        with torch.no_grad():
            target = ag.render(ctx, vid, torch.from_numpy(case["tf_target"]).cuda(), params, case["cams"], W, H, fixed)
        tf0 = torch.from_numpy(case["tf"]).cuda()
        # entries the 8 views constrain: those the first loss gradient reaches
        probe = tf0.clone().requires_grad_(True)
        ((ag.render(ctx, vid, probe, params, case["cams"], W, H, fixed) - target) ** 2).mean().backward()
        g = probe.grad.abs()
        informative = (g > 1e-3 * g.max()).cpu().numpy()
        t0 = time.perf_counter()
        tf, losses, ms = fit_transfer_function(ctx, vid, case["cams"], W, H, tf0, target, fixed, params, steps, lr)
        wall = time.perf_counter() - t0
        d0 = np.abs(case["tf"] - case["tf_target"])
        d1 = np.abs(tf.cpu().numpy() - case["tf_target"])
    return {"workload": "diff_head128_8cam: 128^3 float32 head, 8 cameras, 512x512, MSE to a perturbed-TF target",
            "steps": steps, "loss_first": losses[0], "loss_last": losses[-1], "ms_per_step": ms,
            "wall_s": wall, "tf_mean_abs_err_start": float(d0.mean()), "tf_mean_abs_err_end": float(d1.mean()),
            "informative_entries": float(informative.mean()),
            "tf_mean_abs_err_informative_start": float(d0[informative].mean()),
            "tf_mean_abs_err_informative_end": float(d1[informative].mean()),
            "loss_curve_every_20": losses[::20]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-2)
    a = ap.parse_args()
    print(json.dumps(run(a.steps, a.lr)))


if __name__ == "__main__":
    main()
