"""Autotuner for batched runs of many independent handles.

Two knobs decide how a batch of independent updates fills the GPU: the number
of concurrent streams of `svlcov_batch_run`, and the Jacobi tile width
(`jacobi_block`, columns per block: narrower blocks give each SVD more CTAs
and more rounds).  `tune` times every candidate pair on throwaway handles
built from the same start (each candidate gets fresh handles and one untimed
warm-up run) and caches the fastest in a JSON file keyed by GPU name and a
signature of the problem.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Iterable, List, Optional, Sequence, Tuple

import torch

from .svlcov import batch_run

DEFAULT_CANDIDATES: List[Tuple[int, int]] = [(c, b) for c in (8, 16, 32, 64) for b in (8, 16)]


def cache_key(signature: str) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|{signature}"


def load_cache(path: Optional[str]) -> dict:
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def tune(make_handles: Callable[[int], Sequence], make_items: Callable[[Sequence, int], list], signature: str,
         candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES, cache_path: Optional[str] = None,
         log: Optional[Callable[[str], None]] = None):
    """Return (concurrency, jacobi_block, timings_ms).

    make_handles(jacobi_block) -> fresh handles; make_items(handles, r) ->
    the items of batch r for those handles (r = 0 warm-up, r = 1 timed)."""
    key = cache_key(signature)
    cache = load_cache(cache_path)
    if key in cache:
        c = cache[key]
        return int(c["concurrency"]), int(c["jacobi_block"]), c.get("timings", {})
    timings = {}
    best = None
    for conc, blk in candidates:
        hs = make_handles(blk)
        batch_run(make_items(hs, 0), conc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch_run(make_items(hs, 1), conc)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        timings[f"{conc}x{blk}"] = ms
        if log:
            log(f"autotune concurrency={conc} jacobi_block={blk}: {ms:.2f} ms")
        if best is None or ms < best[2]:
            best = (conc, blk, ms)
        del hs
        torch.cuda.empty_cache()
    if cache_path:
        cache[key] = dict(concurrency=best[0], jacobi_block=best[1], timings=timings)
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best[0], best[1], timings
