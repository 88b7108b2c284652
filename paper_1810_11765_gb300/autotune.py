"""Launch-shape autotuner for graph-captured step loops.

Searches do-all threads per CTA, slots per thread (one block per 64 threads, or one
block per warp), the enumeration (two kernels or the single-pass look-back kernel)
(or a thread-block cluster per type) and the waves of the method do-all grid; the streamed enumeration and the fused
cooperative do-all are tried in a few shapes.
Each candidate runs a fresh world from the same seed, captures one step as a CUDA
graph and times replays with CUDA events (L2 flushed between replays, as in the
benchmark).  Results are cached per GPU name and workload in ``_tune/``.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

import torch

from . import dsoa as D
from .apps import WatorWorld

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_DIR = os.path.join(HERE, "_tune")

CANDIDATES = [dict(tpb=tpb, ctas_per_sm=8, slots_per_thread=spt, scan_tiles=scan, waves=waves, fused=0)
              for tpb, spt, scan, waves in itertools.product((128, 256, 512), (1, 2), (1, 3, 5), (1, 2, 4, 8))]
CANDIDATES += [dict(tpb=tpb, ctas_per_sm=8, slots_per_thread=1, scan_tiles=4, waves=4, fused=0) for tpb in (128, 256)]
CANDIDATES.append(dict(tpb=256, ctas_per_sm=8, slots_per_thread=1, scan_tiles=3, waves=1, fused=1))


def apply(heap: D.Heap, launch: dict):
    """Set a tuned launch shape on a heap (fused = cooperative enumeration + do-all)."""
    shape = {k: v for k, v in launch.items() if k != "fused"}
    heap.set_launch(**shape)
    heap.set_flags(D.FLAG_FUSED if launch.get("fused") else 0)


def _cache_path(key: str) -> str:
    gpu = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(CACHE_DIR, f"{key}-{gpu}.json")


def time_wator_step(seed: int, launch: dict, side: int = 1024, warmup: int = 5, reps: int = 15,
                    flush: torch.Tensor | None = None) -> float:
    """Median ms of one graph replay of a Wa-Tor step under `launch`."""
    heap = D.Heap(512 << 20)
    w = WatorWorld(heap)
    heap.freeze()
    apply(heap, launch)
    w.add(side, side, seed)
    heap.graph_begin()
    w.step()
    g = heap.graph_end()
    for _ in range(warmup):
        g.launch()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.launch()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    g.close()
    heap.close()
    return statistics.median(times)


def best_wator_launch(seed: int, use_cache: bool = True, verbose: bool = False) -> dict:
    path = _cache_path("wator1024-v6")
    if use_cache and os.path.exists(path):
        with open(path) as f:
            return json.load(f)["best"]
    results = []
    # stream capture needs a non-default stream
    stream = torch.cuda.current_stream()
    if stream.cuda_stream == 0:
        stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        for cand in CANDIDATES:
            ms = time_wator_step(seed, cand, flush=flush)
            results.append((ms, cand))
            if verbose:
                print(f"{ms:.4f} ms  {cand}")
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    os.makedirs(CACHE_DIR, exist_ok=True)
    with open(path, "w") as f:
        json.dump({"best": best, "ms": results[0][0],
                   "all": [{"ms": m, **c} for m, c in results]}, f, indent=1)
    return best
