"""Data-parallel helpers: rays are independent, so views shard across ranks with no
exchange for rendering; a data-parallel fit sums the parameter gradients once per
step (the only collective the path has).

``dp_fit`` fits transfer-function entries (the tissue parameters of the paper's
Sec. 2.4, fitted to target views instead of tuned by hand) with the views sharded
across the ranks of a process group: each rank renders and differentiates only its
views, the per-rank gradient sums are gathered and added in rank order on every
rank, and every rank applies the same Adam step, so the parameters stay identical
everywhere without a broadcast. ``library_shard_loss_grad`` is the per-rank step
through libvr.so (vr_render / vr_render_backward via the autograd binding).
"""


def shard_range(n, world, rank):
    """Contiguous [lo, hi) slice of n items for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_sum_(tensors, group=None):
    """In-place sum of each tensor over the process group (fixed order of tensors)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def ordered_sum(t, group=None):
    """Sum of `t` over the ranks of `group`, added in rank order on every rank (an
    all-gather, then a local sum): the result is bit-identical on every rank and does
    not depend on the collective's internal reduction order. Without an initialised
    process group, `t` itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return t
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t.contiguous(), group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        acc += p
    return acc


def dp_fit(shard_loss_grad, tf0, n_views, steps, lr=1e-2, group=None):
    """Adam on sigmoid-parameterised entries x = sigmoid(logit), starting from tf0, of
    the mean squared error over all n_views views, with the views sharded by
    shard_range over the ranks of `group` (one process: all views).

    shard_loss_grad(x, lo, hi) returns (sum of squared errors over the pixels of views
    [lo, hi), number of those pixel values, d(that sum)/dx) for the entries x (a
    detached tensor like tf0). Per step the three are summed over the ranks in rank
    order (ordered_sum), the mean's gradient is chained through the sigmoid, and every
    rank takes the same Adam step. Returns (fitted x, per-step MSE)."""
    import torch
    import torch.distributed as dist
    dist_on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    lo, hi = shard_range(n_views, world, rank)
    logit = torch.logit(tf0.detach().clamp(1e-4, 1.0 - 1e-4)).clone().requires_grad_(True)
    opt = torch.optim.Adam([logit], lr=lr)
    losses = []
    for _ in range(steps):
        x = torch.sigmoid(logit)
        loss_sum, count, g = shard_loss_grad(x.detach(), lo, hi)
        head = torch.tensor([float(loss_sum), float(count)], dtype=g.dtype, device=g.device)
        tot = ordered_sum(torch.cat([head, g.reshape(-1)]), group)
        n = float(tot[1])
        opt.zero_grad(set_to_none=True)
        x.backward(gradient=(tot[2:] / n).reshape(x.shape).to(x.dtype))
        opt.step()
        losses.append(float(tot[0]) / n)
    return torch.sigmoid(logit).detach(), losses


def library_shard_loss_grad(ctx, vol, cams, W, H, fixed, params, targets):
    """shard_loss_grad for dp_fit through the library: render views [lo, hi) of
    `cams` with the transfer function x (autograd binding), squared error against
    targets[lo:hi] summed, and its gradient from vr_render_backward."""
    import numpy as np
    import torch

    from . import autograd as ag
    cams = np.asarray(cams, np.float32).reshape(-1, 12)

    def f(x, lo, hi):
        if hi <= lo:
            return 0.0, 0, torch.zeros_like(x)
        tf = x.clone().requires_grad_(True)
        img = ag.render(ctx, vol, tf, params, cams[lo:hi], W, H, fixed)
        loss = ((img - targets[lo:hi]) ** 2).sum()
        loss.backward()
        return float(loss.detach()), img.numel(), tf.grad
    return f
