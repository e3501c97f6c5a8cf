"""Autotuner for batched circuits: tile size and fusion depth per qudit dimension.

For each qudit dimension d present in a batch, a sample of its largest
circuits is built into small batches with every candidate (tile qudits,
gates per pass) and timed forward + backward through the captured graph on
the current GPU; the fastest candidate wins.  Results are cached in a JSON
file keyed by GPU name, d and dtype, so a later batch reuses them.  Every
measurement runs the library's own kernels through the C ABI.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, List, Optional, Tuple

from . import qf

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _default_tile_qudits(d: int, c128: bool) -> int:
    cap = 4096 if c128 else 8192
    nt, t = 0, 1
    while t * d <= cap:
        t *= d
        nt += 1
    return nt


def candidates(d: int, c128: bool) -> List[Tuple[int, int]]:
    top = _default_tile_qudits(d, c128)
    tiles = sorted({max(2, top - k) for k in (0, 1, 2)}, reverse=True)
    return [(t, ops) for t in tiles for ops in (16, 96)]


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


def _time_batch(circuits, progs, params, dtype: int, d: int, tile: int, max_ops: int, reps: int = 2) -> float:
    import torch
    b = qf.qf_batch_create(dtype)
    try:
        for c, p in zip(circuits, progs):
            qf.qf_batch_add(b, p, [1.0] + [0.0] * (c.n - 1))
        qf.qf_batch_tune(b, d, tile, max_ops)
        qf.qf_batch_build(b, len(params))
        qf.qf_batch_run(b, params, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            qf.qf_batch_run(b, params, True)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        qf.qf_batch_free(b)


def tune(circuits, params, dtype: int = qf.QF_C64, sample: int = 12, use_cache: bool = True,
         cache_path: Optional[str] = None) -> Dict[int, dict]:
    """Returns {d: {"tile_qudits", "max_ops", "ms", "tried"}} for every d in
    the batch (circuits: objects with d, n, ops)."""
    path = cache_path or CACHE
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    gpu = _gpu_name()
    c128 = dtype == qf.QF_C128
    out: Dict[int, dict] = {}
    for d in sorted({c.d for c in circuits}):
        key = "%s|d=%d|%s" % (gpu, d, "c128" if c128 else "c64")
        if use_cache and key in cache:
            out[d] = cache[key]
            continue
        pool = sorted((c for c in circuits if c.d == d), key=lambda c: -(c.d ** c.n))
        subset = pool[:sample]
        progs = [qf.program_from_ops(c.d, c.n, c.ops) for c in subset]
        tried = []
        try:
            for tile, ops in candidates(d, c128):
                ms = _time_batch(subset, progs, params, dtype, d, tile, ops)
                tried.append({"tile_qudits": tile, "max_ops": ops, "ms": ms})
        finally:
            for p in progs:
                qf.qf_program_free(p)
        best = min(tried, key=lambda r: r["ms"])
        out[d] = {"tile_qudits": best["tile_qudits"], "max_ops": best["max_ops"], "ms": best["ms"], "tried": tried}
        cache[key] = out[d]
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return out


def apply(batch: int, tuning: Dict[int, dict]) -> None:
    """Sets a (not yet built) batch's per-d tile size and fusion depth."""
    for d, t in tuning.items():
        qf.qf_batch_tune(batch, int(d), int(t["tile_qudits"]), int(t["max_ops"]))
