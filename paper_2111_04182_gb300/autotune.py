"""Autotuner for the batched forest: leaf size L and the thread mapping of
the search (one thread per query, or one warp per 32 Morton-consecutive
queries).

Each candidate (L, mapping) builds the forest and runs the all-points k-NN on
the caller's data; the step is timed with CUDA events on the current stream
(best of `reps` after one warm-up).  The answer does not depend on the
choice -- every candidate returns the same exact neighbours -- so the tuner
only picks the fastest.  Results are cached as JSON keyed by GPU name,
workload signature and k (default file: _tune/cache.json next to this module,
or $ZD_TUNE_CACHE).
"""
from __future__ import annotations

import json
import os

import torch

from . import zd

LEAF_SIZES = (8, 16, 32, 64)
MAPPINGS = {"thread": zd.ZD_KNN_THREAD_PER_QUERY, "warp_group": zd.ZD_KNN_WARP_GROUP}


def _cache_path() -> str:
    return os.environ.get("ZD_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "cache.json"))


def _load() -> dict:
    try:
        return json.load(open(_cache_path()))
    except Exception:
        return {}


def _store(cache: dict) -> None:
    path = _cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    json.dump(cache, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, path)


def signature(pts: torch.Tensor, offsets, k: int, coord_bits: int) -> str:
    off = torch.as_tensor(offsets, dtype=torch.int64)
    sizes = off[1:] - off[:-1]
    return "%s|n=%d|clouds=%d|max=%d|%s|d=%d|B=%d|k=%d" % (
        torch.cuda.get_device_name(pts.device), int(off[-1]), len(sizes), int(sizes.max()) if len(sizes) else 0,
        str(pts.dtype).replace("torch.", ""), pts.shape[1], coord_bits, k)


def time_step(pts, offsets, k, coord_bits, leaf_size, mapping, out, reps: int = 3) -> float:
    """Best-of-reps milliseconds of build + all-points k-NN + free."""
    s = torch.cuda.current_stream()

    def step():
        t = zd.zd_build_batched(pts, offsets, leaf_size, coord_bits)
        zd.zd_knn_batched(t, k, out=out, mapping=mapping)
        t.free()

    step()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        step()
        b.record(s)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    if zd.zd_check() != 0:
        raise RuntimeError("device status set while tuning")
    return best


def tune_batched(pts: torch.Tensor, offsets, k: int, coord_bits: int, out=None, leaf_sizes=LEAF_SIZES,
                 mappings=None, reps: int = 3, use_cache: bool = True) -> dict:
    """Pick (leaf_size, mapping) for the batched build + all-points k-NN.
    Returns {"leaf_size", "mapping", "mapping_name", "ms", "table", "cached"}."""
    mappings = mappings or MAPPINGS
    key = signature(pts, offsets, k, coord_bits)
    cache = _load() if use_cache else {}
    if key in cache:
        r = dict(cache[key])
        r["cached"] = True
        return r
    n = int(torch.as_tensor(offsets, dtype=torch.int64)[-1])
    if out is None:
        ddt = torch.float32 if pts.dtype == torch.float32 else torch.int64
        out = (torch.empty((n, k), dtype=torch.int32, device=pts.device),
               torch.empty((n, k), dtype=ddt, device=pts.device))
    table = []
    for L in leaf_sizes:
        for name, mp in mappings.items():
            ms = time_step(pts, offsets, k, coord_bits, L, mp, out, reps)
            table.append({"leaf_size": L, "mapping_name": name, "mapping": mp, "ms": ms})
    best = min(table, key=lambda r: r["ms"])
    r = {"leaf_size": best["leaf_size"], "mapping": best["mapping"], "mapping_name": best["mapping_name"],
         "ms": best["ms"], "table": table}
    if use_cache:
        cache[key] = r
        _store(cache)
    r = dict(r)
    r["cached"] = False
    return r
