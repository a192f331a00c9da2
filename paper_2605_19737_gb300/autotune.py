"""Autotuner for the batched renderer's launch shape.

Times every (packet_w, warps_per_block) candidate on the caller's own batch
with CUDA events (median of `reps` launches after one warm-up), keeps the
fastest, and caches the choice per (GPU name, batch key) in a JSON file so
later runs skip the search. The candidates cover the packet shapes 4x8, 8x4,
16x2 and 32x1 pixels and 2, 4 or 8 warps per CTA; the grid always fills the
SMs at the kernel's resident-CTA occupancy.
"""

import json
import os

DEFAULT_CANDIDATES = [(pw, w) for pw in (4, 8, 16, 32) for w in (2, 4, 8)]


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


def tune_batch(ctx, batch, key, candidates=None, reps=5, cache_path=None, force=False):
    """Return {"packet_w", "warps_per_block", "ms", "cached", "timings"} for `batch`."""
    import torch

    cache_path = cache_path or default_cache_path()
    gpu = torch.cuda.get_device_name(ctx.device)
    ckey = "%s|%s" % (gpu, key)
    table = _load(cache_path)
    if not force and ckey in table:
        return dict(table[ckey], cached=True)
    timings = {}
    for pw, w in candidates or DEFAULT_CANDIDATES:
        ctx.batch_render(batch, packet_w=pw, warps_per_block=w)
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            ctx.batch_render(batch, packet_w=pw, warps_per_block=w)
            e.record()
            e.synchronize()
            ts.append(s.elapsed_time(e))
        ts.sort()
        timings["%dx%d" % (pw, w)] = ts[len(ts) // 2]
    best = min(timings, key=timings.get)
    pw, w = (int(x) for x in best.split("x"))
    entry = {"packet_w": pw, "warps_per_block": w, "ms": timings[best], "timings": timings}
    table[ckey] = entry
    _store(cache_path, table)
    return dict(entry, cached=False)
