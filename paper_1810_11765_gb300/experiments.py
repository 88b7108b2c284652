"""The paper's detailed Wa-Tor analyses (Sec. 6.4-6.6), re-run on this runtime.

  python -m paper_1810_11765_gb300.experiments frag      # F over time      (Fig. 10d)
  python -m paper_1810_11765_gb300.experiments lookups   # F vs r            (Fig. 11)
  python -m paper_1810_11765_gb300.experiments ablation  # NoCoal / NoShift  (Fig. 10c)
  python -m paper_1810_11765_gb300.experiments heapsize  # time vs heap size (Fig. 12b)
  python -m paper_1810_11765_gb300.experiments capacity  # uniform vs per-type block capacity (Sec. 3.2)
  python -m paper_1810_11765_gb300.experiments problemsize  # time vs problem size (Fig. 10b)

Each prints one JSON line.  Workload: Wa-Tor 1024 x 1024, 30 % fish / 5 % sharks,
seed 0x5EED0003.  Fragmentation F = unused slots / slots of allocated blocks
(Sec. 6.4), from the allocated-block bitmaps and live counts on the device.
"""
from __future__ import annotations

import argparse
import json
import statistics

import torch

from . import build, dsoa as D, inputs
from .apps import WatorWorld


def _world(heap_bytes=512 << 20, flags=0, lookups=None, capacity_mode=D.CAPACITY_UNIFORM):
    heap = D.Heap(heap_bytes)
    w = WatorWorld(heap)
    heap.set_capacity_mode(capacity_mode)
    heap.freeze()
    heap.set_flags(flags)
    if lookups is not None:
        heap.set_lookups(lookups)
    w.add(1024, 1024, inputs.WatorConfig().seed)
    return heap, w


def _frag(heap, w):
    f, s = heap.type_stats(w.fish_type), heap.type_stats(w.shark_type)
    blocks = f["blocks"] + s["blocks"]
    objs = f["objects"] + s["objects"]
    slots = f["slots"] + s["slots"]
    return {"fish": f["objects"], "sharks": s["objects"], "blocks": blocks,
            "F": 1.0 - objs / slots if slots else 0.0}


def frag_over_time(steps=500, every=25, variants=("dsoa",)):
    """F every `every` steps (Fig. 10d) for allocation policies of FRAG_VARIANTS,
    with the time of each stretch of `every` plain steps."""
    out = {"experiment": "fragmentation over time (Fig. 10d)", "variants": {}}
    for name in variants:
        heap, w = _world(flags=FRAG_VARIANTS[name])
        rows = [dict(step=0, **_frag(heap, w))]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k in range(1, steps + 1):
            w.step()
            if k % every == 0:
                b.record()
                b.synchronize()
                rows.append(dict(step=k, ms_per_step=a.elapsed_time(b) / every, **_frag(heap, w)))
                a.record()
        out["variants"][name] = {"rows": rows, "device_errors": heap.get_error()}
        heap.close()
    return out


FRAG_VARIANTS = {
    # this runtime: r counts an allocation's active-block attempts (lost
    # reservations included); a group of 16+ requests takes a fresh block after a
    # lost round; per-warp block hint
    "dsoa": 0,
    # the earlier policy: r bounds the failed try_find_set calls of one round and
    # small groups search again in every round
    "r_per_round": D.FLAG_R_PER_ROUND,
    "no_hint": D.FLAG_NO_HINT,
    "no_fresh_group": D.FLAG_NO_FRESH_GROUP,
    # Alg. 1's reading of r alone: every group (large ones too) searches until r
    # attempts failed, then takes a fresh block
    "paper_r": D.FLAG_PAPER_R,
    "paper_r_no_hint": D.FLAG_PAPER_R | D.FLAG_NO_HINT,
    # blocks that fell to an eighth of their capacity drain: searches pass over
    # them and a warp drops its hint to one
    "drain": D.FLAG_DRAIN,
}


def frag_vs_lookups(rs=(1, 2, 3, 5, 8), steps=300, variants=None):
    """Fragmentation F after `steps` plain steps against r, for the allocation
    policies of FRAG_VARIANTS, with the mean step time of the last 50 steps."""
    rows = []
    for name in (variants or FRAG_VARIANTS):
        fl = FRAG_VARIANTS[name]
        for r in rs:
            heap, w = _world(lookups=r, flags=fl)
            for _ in range(steps - 50):
                w.step()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(50):
                w.step()
            b.record()
            b.synchronize()
            rows.append(dict(variant=name, r=r, **_frag(heap, w), ms_per_step=a.elapsed_time(b) / 50,
                             device_errors=heap.get_error()))
            heap.close()
    return {"experiment": f"fragmentation after {steps} steps vs active-block lookups r (Fig. 11)", "rows": rows}


def _timed_steps(heap, w, steps, flush):
    times = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        w.step()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times


def ablation(steps=200):
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    variants = {"dsoa": 0, "no_coalesce": D.FLAG_NO_COALESCE, "no_rotate": D.FLAG_NO_ROTATE,
                "no_coalesce_no_rotate": D.FLAG_NO_COALESCE | D.FLAG_NO_ROTATE,
                "no_hint": D.FLAG_NO_HINT, "fused": D.FLAG_FUSED, "drain": D.FLAG_DRAIN}
    rows, ref = [], None
    for name, fl in variants.items():
        heap, w = _world(heap_bytes=2 << 30, flags=fl)
        t = _timed_steps(heap, w, steps, flush)
        pops, grid = w.counts(), w.read(0)
        if ref is None:
            ref = (pops, grid)
        rows.append(dict(variant=name, steps_per_s=steps / (sum(t) / 1e3), median_ms=statistics.median(t),
                         **_frag(heap, w), device_errors=heap.get_error(), fish_sharks=list(pops),
                         same_as_dsoa=bool(pops == ref[0] and (grid == ref[1]).all())))
        heap.close()
    base = rows[0]["steps_per_s"]
    for r in rows:
        r["slowdown_vs_dsoa"] = base / r["steps_per_s"]
    return {"experiment": f"ablations, {steps} plain steps (Fig. 10c)", "rows": rows}


def heap_size(sizes_gib=(0.5, 1, 2, 4, 8, 16), steps=100):
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    for g in sizes_gib:
        heap, w = _world(heap_bytes=int(g * (1 << 30)))
        t = _timed_steps(heap, w, steps, flush)
        rows.append(dict(heap_gib=g, blocks=heap.info()["num_blocks"], levels=heap.info()["num_levels"],
                         steps_per_s=steps / (sum(t) / 1e3), device_errors=heap.get_error()))
        heap.close()
        torch.cuda.empty_cache()
    return {"experiment": f"heap size vs step time, {steps} plain steps (Fig. 12b)", "rows": rows}


def problem_size(sides=(256, 512, 768, 1024, 1536, 2048, 2560), steps=100):
    """Wa-Tor in a fixed 1 GiB heap at growing torus sides (Fig. 10b): time per
    step and per cell (the paper finds the running time linear in problem size)."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    for side in sides:
        heap = D.Heap(1 << 30)
        w = WatorWorld(heap)
        heap.freeze()
        w.add(side, side, inputs.WatorConfig().seed)
        t = _timed_steps(heap, w, steps, flush)
        ms = sum(t) / steps
        rows.append(dict(side=side, cells=side * side, ms_per_step=ms, ns_per_cell=ms * 1e6 / (side * side),
                         **_frag(heap, w), device_errors=heap.get_error()))
        heap.close()
        torch.cuda.empty_cache()
    return {"experiment": f"problem size in a 1 GiB heap, {steps} plain steps (Fig. 10b)", "rows": rows}


def capacity(steps=300):
    """Uniform 64-slot blocks vs per-type block capacity N_T (Sec. 3.2): block
    bytes, capacities, step rate, fragmentation and the heap bytes held by
    allocated blocks after `steps` plain steps."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    for name, mode in (("uniform", D.CAPACITY_UNIFORM), ("per_type", D.CAPACITY_PER_TYPE)):
        heap, w = _world(heap_bytes=512 << 20, capacity_mode=mode)
        t = _timed_steps(heap, w, steps, flush)
        fr = _frag(heap, w)
        bb = heap.info()["block_bytes"]
        rows.append(dict(mode=name, block_bytes=bb, fish_capacity=heap.capacity(w.fish_type),
                         shark_capacity=heap.capacity(w.shark_type), steps_per_s=steps / (sum(t) / 1e3),
                         median_ms=statistics.median(t), bytes_in_blocks=fr["blocks"] * bb, **fr,
                         device_errors=heap.get_error()))
        heap.close()
    return {"experiment": f"block capacity per type, Wa-Tor 1024^2, {steps} plain steps (Sec. 3.2)", "rows": rows}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("which", choices=["frag", "lookups", "ablation", "heapsize", "capacity", "problemsize"])
    p.add_argument("--variants", default=None,
                   help="frag / lookups: comma-separated allocation policies (" + ", ".join(FRAG_VARIANTS) + ")")
    a = p.parse_args()
    build.build()
    kw = {}
    if a.variants and a.which in ("frag", "lookups"):
        kw["variants"] = tuple(a.variants.split(","))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        res = {"frag": frag_over_time, "lookups": frag_vs_lookups, "ablation": ablation,
               "heapsize": heap_size, "capacity": capacity, "problemsize": problem_size}[a.which](**kw)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
