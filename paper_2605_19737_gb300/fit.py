"""Fit transfer-function entries to target views through the differentiable renderer.

The paper tunes tissue parameters interactively (uniform buffers, Sec. 4);
with the adjoint raymarch the same parameters can be fitted to a target image:
MSE between renders of n cameras and targets, Adam on sigmoid-parameterised
transfer-function entries. Forward and backward both run in libvr.so.

    python -m paper_2605_19737_gb300.fit --steps 200 [--checkpoint fit.pt --every 50]
"""

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def adam_fit(loss_fn, tf0, steps, lr=1e-2, checkpoint=None, every=50):
    """Adam on sigmoid-parameterised entries x = sigmoid(logit), starting from tf0.

    loss_fn(x) returns a scalar tensor. Returns (fitted x, per-step losses, mean ms per
    step: CUDA events for device tensors, the host clock otherwise). With
    ``checkpoint`` (a path) the logits, the optimiser state and the loss history are
    saved with torch.save every ``every`` steps and after the last one (written to a
    temporary file, then renamed); when the file exists, the fit resumes from it and
    continues to ``steps`` in total, reproducing the uninterrupted run."""
    import torch

    logit = torch.logit(tf0.clamp(1e-4, 1.0 - 1e-4)).detach().requires_grad_(True)
    opt = torch.optim.Adam([logit], lr=lr)
    losses, start = [], 0
    if checkpoint and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location=tf0.device, weights_only=False)
        with torch.no_grad():
            logit.copy_(st["logit"])
        opt.load_state_dict(st["adam"])
        losses, start = list(st["losses"]), int(st["step"])

    def save(step):
        tmp = checkpoint + ".tmp"
        torch.save({"step": step, "logit": logit.detach().clone(), "adam": opt.state_dict(),
                    "losses": [float(x) for x in losses]}, tmp)
        os.replace(tmp, checkpoint)

    on_device = tf0.is_cuda
    times = []
    for step in range(start, steps):
        if on_device:
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
        else:
            t0 = time.perf_counter()
        opt.zero_grad(set_to_none=True)
        loss = loss_fn(torch.sigmoid(logit))
        loss.backward()
        opt.step()
        if on_device:
            e.record()
            times.append((s, e))
        else:
            times.append(time.perf_counter() - t0)
        losses.append(loss.detach())
        if checkpoint and ((step + 1) % every == 0 or step + 1 == steps):
            save(step + 1)
    if on_device:
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in times[1:]]
    else:
        ms = [1e3 * t for t in times[1:]]
    return torch.sigmoid(logit).detach(), [float(x) for x in losses], sum(ms) / max(1, len(ms))


def fit_transfer_function(ctx, vol, cams, W, H, tf0, target, fixed, params, steps=200, lr=1e-2, checkpoint=None,
                          every=50):
    """MSE between renders of the cameras and the targets, minimised over the transfer
    function by adam_fit. Returns (fitted tf, per-step losses, mean ms per step)."""
    from . import autograd as ag

    def loss_fn(tf):
        return ((ag.render(ctx, vol, tf, params, cams, W, H, fixed) - target) ** 2).mean()

    return adam_fit(loss_fn, tf0, steps, lr, checkpoint, every)


def run(steps=200, lr=1e-2, checkpoint=None, every=50):
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
        tf, losses, ms = fit_transfer_function(ctx, vid, case["cams"], W, H, tf0, target, fixed, params, steps, lr,
                                               checkpoint, every)
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
    ap.add_argument("--checkpoint", default=None, help="save/resume the fit state at this path")
    ap.add_argument("--every", type=int, default=50, help="checkpoint interval (steps)")
    a = ap.parse_args()
    print(json.dumps(run(a.steps, a.lr, a.checkpoint, a.every)))


if __name__ == "__main__":
    main()
