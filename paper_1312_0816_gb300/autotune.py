"""Autotuner of the batched persistent launch.

The launch has three schedule knobs (geo_batch_opts): the order in which tiles
are claimed (largest estimated cost first, or basket order), the number of
resident blocks per SM, and the tile shape (tiles of 384 tracks with 12
producer + 4 consumer warps, or of 256 with 8 + 4: two instantiations of the
kernel).  tune_batch() builds one batch per candidate, times
each as a CUDA graph of the one launch (CUDA events, after warm-up), and keeps
the fastest.  Results are cached in paper_1312_0816_gb300/_build/autotune.json
keyed by GPU name, a hash of the kernel sources and a size class of the batch
(log2 of tracks, log2 of the mean daughter count), so a later call with a
similar batch reuses the choice without timing.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

from . import build_lib, geonav

# (tile_order, blocks_per_sm, tile_tracks)
CANDIDATES = [(o, b, t) for t in (384, 256) for o in (0, 1) for b in (2, 1)]
CACHE = os.path.join(build_lib.OUT, "autotune.json")


def _sources_sha() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(build_lib.CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(build_lib.CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def _key(volumes, baskets) -> str:
    import torch

    n = sum(int(c) for _, _, c in baskets)
    nd = sum(v.n_daughters for v in volumes) / max(len(volumes), 1)
    cls = f"t{int(math.log2(max(n, 1)))}-d{int(math.log2(max(nd, 1)))}"
    return f"{torch.cuda.get_device_name()}|{_sources_sha()}|{cls}"


def _load():
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _save(tab):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    json.dump(tab, open(tmp, "w"), indent=1)
    os.replace(tmp, CACHE)


def time_graph(batch, x, step, hit, reps: int = 20) -> float:
    """Mean milliseconds of one batched launch replayed as a CUDA graph."""
    import torch

    geonav.geo_dist_to_boundary_batched(batch, *x, step=step, hit=hit)   # first call outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            geonav.geo_dist_to_boundary_batched(batch, *x, step=step, hit=hit)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(volumes, baskets, x, step, hit, use_cache: bool = True, reps: int = 20):
    """Returns (tile_order, blocks_per_sm, tile_tracks, timings) for this
    batch; x = the six device SoA tensors, step/hit preallocated outputs."""
    key = _key(volumes, baskets)
    tab = _load() if use_cache else {}
    if key in tab and "tile_tracks" in tab[key]:
        c = tab[key]
        return c["tile_order"], c["blocks_per_sm"], c["tile_tracks"], c.get("timings_ms", {})
    timings = {}
    for order, bps, tile in CANDIDATES:
        b = geonav.geo_build_batch(volumes, baskets, tile_order=order, blocks_per_sm=bps, tile_tracks=tile)
        timings[f"{order},{bps},{tile}"] = time_graph(b, x, step, hit, reps)
        b.close()
    best = min(timings, key=timings.get)
    order, bps, tile = (int(v) for v in best.split(","))
    tab = _load()
    tab[key] = {"tile_order": order, "blocks_per_sm": bps, "tile_tracks": tile, "timings_ms": timings}
    _save(tab)
    return order, bps, tile, timings
