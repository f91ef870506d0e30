"""Autotuner for batched runs of many independent handles.

Two knobs decide how a batch of independent updates fills the GPU: the number
of concurrent streams of `svlcov_batch_run`, and the Jacobi tile width
(`jacobi_block`, columns per block: narrower blocks give each SVD more CTAs
and more rounds).  `tune` times every candidate pair on throwaway handles
built from the same start (each candidate gets fresh handles and one untimed
warm-up run) and caches the fastest in a JSON file keyed by GPU name and a
signature of the problem.  A candidate is timed the way batched rounds are
meant to run: captured once in a CUDA graph and replayed (an eager enqueue
of ~50k launches is bound by the host and hides the difference between
concurrencies); where capture fails the eager enqueue is timed instead.
Within 2% of the fastest, the higher concurrency wins (more independent
branches for the graph).
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


def pick(timings: dict, candidates: Iterable[Tuple[int, int]], slack: float = 1.02) -> Tuple[int, int]:
    """The candidate to keep: among those within `slack` of the fastest time,
    the highest concurrency (then the fastest of those)."""
    cands = list(candidates)
    fastest = min(timings[f"{c}x{b}"] for c, b in cands)
    near = [(c, b) for c, b in cands if timings[f"{c}x{b}"] <= slack * fastest]
    return max(near, key=lambda cb: (cb[0], -timings[f"{cb[0]}x{cb[1]}"]))


def _time_graph(hs, make_items, conc) -> Optional[float]:
    """One replay of batch 1 captured in a CUDA graph (ms), or None."""
    s = torch.cuda.Stream()
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                batch_run(make_items(hs, 1), conc, stream=s)
    except Exception:   # capture is an optimisation; time the eager enqueue instead
        torch.cuda.synchronize()
        return None
    torch.cuda.synchronize()
    g.replay()          # warm replay
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    del g
    return e0.elapsed_time(e1)


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
    for conc, blk in candidates:
        hs = make_handles(blk)
        batch_run(make_items(hs, 0), conc)
        torch.cuda.synchronize()
        ms = _time_graph(hs, make_items, conc)
        if ms is None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch_run(make_items(hs, 1), conc)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        timings[f"{conc}x{blk}"] = ms
        if log:
            log(f"autotune concurrency={conc} jacobi_block={blk}: {ms:.2f} ms")
        del hs
        torch.cuda.empty_cache()
    conc, blk = pick(timings, candidates)
    best = (conc, blk, timings[f"{conc}x{blk}"])
    if cache_path:
        cache[key] = dict(concurrency=best[0], jacobi_block=best[1], timings=timings)
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best[0], best[1], timings
