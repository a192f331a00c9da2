"""Autotuner for the raymarch's launch shape and skip-brick size.

Times candidates on the caller's own workload with CUDA events (median of
`reps` launches after one warm-up), keeps the fastest, and caches the choice per
(GPU name, workload key) in a JSON file so later runs skip the search.

* tune_render: one vr_render call (a view or several cameras of one volume) over
  skip-brick edges of 4, 8 or 16 cells (vr_set_brick_size), warp packets of 4x8,
  8x4 or 16x2 rays and CTAs of 2, 4 or 8 warps (the CTA tile: 8x8 .. 16x16 pixels).
* tune_batch: the batched persistent renderer over packet shapes 4x8, 8x4, 16x2
  and 32x1, 2, 4 or 8 warps per CTA, and optionally the skip-brick edge of the
  batch's volumes; the grid always fills the SMs at the kernel's resident-CTA
  occupancy.

Changing the brick size rebuilds a volume's grid, cell grid and derived bricks;
the caller passes `prepare(cells)`, which sets the size on its volumes and
re-runs their precompute and tissue parameters (and vr_batch_update for a batch).
The images do not depend on any of these choices.
"""

import json
import os

DEFAULT_CANDIDATES = [(pw, w) for pw in (4, 8, 16, 32) for w in (2, 4, 8)]
RENDER_CANDIDATES = [(pw, w) for pw in (4, 8, 16) for w in (2, 4, 8)]
BRICK_SIZES = (4, 8, 16)


def default_cache_path():
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "vr_autotune.json")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, table):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(launch, reps):
    import torch
    launch()  # warm-up
    ts = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        launch()
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    ts.sort()
    return ts[len(ts) // 2]


def _search(ctx, key, cache_path, force, bricks, prepare, candidates, launch, reps):
    """Shared search: every brick size (prepared once) x every (packet_w, warps)."""
    import torch
    cache_path = cache_path or default_cache_path()
    ckey = "%s|%s" % (torch.cuda.get_device_name(ctx.device), key)
    table = _load(cache_path)
    if not force and ckey in table:
        entry = dict(table[ckey], cached=True)
        if prepare is not None and entry.get("brick"):
            prepare(entry["brick"])
        return entry
    timings = {}
    for b in bricks:
        if prepare is not None:
            prepare(b)
        for pw, w in candidates:
            timings["%dx%d/%s" % (pw, w, b)] = _time(lambda: launch(pw, w), reps)
    best = min(timings, key=timings.get)
    shape, b = best.split("/")
    pw, w = (int(x) for x in shape.split("x"))
    b = None if b == "None" else int(b)
    entry = {"packet_w": pw, "warps_per_block": w, "brick": b, "ms": timings[best], "timings": timings}
    if prepare is not None:
        prepare(b)
    table[ckey] = entry
    _store(cache_path, table)
    return dict(entry, cached=False)


def tune_render(ctx, vol, cams, W, H, key, prepare=None, bricks=BRICK_SIZES, candidates=None, reps=5,
                cache_path=None, force=False, out=None):
    """Return {"packet_w", "warps_per_block", "brick", "ms", "cached", "timings"} for
    vr_render of `cams` (W x H) on volume `vol`. Without `prepare` only the volume's
    current brick size is tried. The chosen brick size is left set (via prepare)."""
    import torch

    from . import VR_KERNEL_GATHER
    n = len(cams) if getattr(cams, "ndim", 1) > 1 else 1
    out = out if out is not None else torch.empty((n, H, W, 4), device="cuda:%d" % ctx.device)
    if prepare is None:
        bricks = (None,)

    def launch(pw, w):
        ctx.render(vol, cams, W, H, out=out, kernel=VR_KERNEL_GATHER, packet_w=pw, warps_per_block=w)
    return _search(ctx, key, cache_path, force, bricks, prepare, candidates or RENDER_CANDIDATES, launch, reps)


def tune_batch(ctx, batch, key, candidates=None, reps=5, cache_path=None, force=False, prepare=None,
               bricks=BRICK_SIZES):
    """Return {"packet_w", "warps_per_block", "brick", "ms", "cached", "timings"} for
    `batch`. Without `prepare` only the volumes' current brick size is tried."""
    if prepare is None:
        bricks = (None,)

    def launch(pw, w):
        ctx.batch_render(batch, packet_w=pw, warps_per_block=w)
    return _search(ctx, key, cache_path, force, bricks, prepare, candidates or DEFAULT_CANDIDATES, launch, reps)
