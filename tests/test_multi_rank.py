"""World-size-2 gloo tests of the data-parallel path on CPU: each rank computes the
oracle gradient of its shard of cameras and the all-reduced sum equals the gradient
of all cameras in one process; the view shards cover every view exactly once; and
the data-parallel transfer-function fit (dp_fit, with a stub renderer standing in for
the library) reproduces the one-process fit step for step, identically on both
ranks."""

import os
import socket

import numpy as np
import pytest

from paper_2605_19737_gb300.distributed import dp_fit, shard_range


def test_shard_range_covers_views():
    for n in (1, 7, 64, 256):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def _case():
    import oracle
    import phantoms as ph
    dims, sp = (10, 9, 8), (1.0, 1.0, 1.0)
    In = ph.random_volume(dims, 91, np.float64, smooth=2)
    In = (In - In.min()) / (In.max() - In.min())
    cams = ph.camera_array([ph.orbit_camera(dims, sp, 60.0 * k, 10.0, width=8, height=6) for k in range(5)])
    rng = np.random.default_rng(92)
    tf = rng.random((1, 16, 4)).astype(np.float32)
    tf[..., 3] *= 0.3
    P = oracle.make_params(tf_shape=(1, 16), grad_mod=1, shading=1, gamma=0.2, kappa_ref=1.0)
    dl = rng.normal(size=(5, 6, 8, 4))
    return In, sp, cams, tf, P, dl


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2605_19737_gb300.distributed import allreduce_sum_
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    In, sp, cams, tf, P, dl = _case()
    lo, hi = shard_range(cams.shape[0], world, rank)
    gmax = oracle.gmax(In, sp)
    dtf, dpar, dIn = oracle.render_grad(In, sp, P, tf, cams[lo:hi], 8, 6, dl[lo:hi], gmax_value=gmax)
    t = [torch.from_numpy(dtf.copy()), torch.from_numpy(dpar.copy()), torch.from_numpy(dIn.copy())]
    allreduce_sum_(t)
    if rank == 0:
        q.put([x.numpy() for x in t])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gradient_allreduce_equals_single_process():
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    In, sp, cams, tf, P, dl = _case()
    want = oracle.render_grad(In, sp, P, tf, cams, 8, 6, dl, gmax_value=oracle.gmax(In, sp))
    for a, b in zip(got, want):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def _stub():
    """A linear stand-in for the renderer: view k of the entries x is M_k x (float64),
    with targets made from a perturbed table."""
    import torch
    g = torch.Generator().manual_seed(93)
    n_views, n_px, shape = 5, 24, (1, 16, 4)
    M = torch.randn((n_views, n_px, 64), generator=g, dtype=torch.float64) / 8.0
    x_true = torch.rand(shape, generator=g, dtype=torch.float64)
    targets = torch.einsum("kpe,e->kp", M, x_true.reshape(-1))
    x0 = (x_true + 0.2 * torch.randn(shape, generator=g, dtype=torch.float64)).clamp(0.05, 0.95)

    def shard_loss_grad(x, lo, hi):
        xx = x.clone().requires_grad_(True)
        img = torch.einsum("kpe,e->kp", M[lo:hi], xx.reshape(-1))
        loss = ((img - targets[lo:hi]) ** 2).sum()
        loss.backward()
        return float(loss), img.numel(), xx.grad
    return n_views, x0, shard_loss_grad


def _fit_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_views, x0, f = _stub()
    x, losses = dp_fit(f, x0, n_views, steps=25, lr=2e-2)
    q.put((rank, x.numpy(), losses))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_fit_equals_single_process():
    mp = pytest.importorskip("torch.multiprocessing")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_fit_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (x, l)) for r, x, l in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    n_views, x0, f = _stub()
    x1, l1 = dp_fit(f, x0, n_views, steps=25, lr=2e-2)
    # identical on both ranks (the same ordered sum and the same Adam step)
    np.testing.assert_array_equal(got[0][0], got[1][0])
    assert got[0][1] == got[1][1]
    # and the same fit as one process over all views, up to the order of the sums
    np.testing.assert_allclose(got[0][0], x1.numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(got[0][1], l1, rtol=1e-9)
    assert l1[-1] < 0.5 * l1[0]
