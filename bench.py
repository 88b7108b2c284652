"""Benchmark of the GB300 SMMO runtime (allocator + do-all).

Headline: Wa-Tor 1024x1024 torus (30 % fish / 5 % sharks), app steps/s with each
step captured as a CUDA graph around the persistent do-all kernels, next to the same
steps launched plainly.  One step = 4 do-alls (each: hierarchical bitmap scan +
prefix-sum compaction + do-all kernel) with allocations (births) and frees (eaten
fish, starved sharks), i.e. every step of the hot path.  L2 is flushed (a 256 MiB
write) between timed steps, outside the timed region.

Secondary figures in the same JSON line: the do-all kernel's HBM GB/s on >L2 object
sets (2^26 objects, full and 50 % holes), alloc+free ops/s (allocation storm then
delete-all), heap utilisation (fill a fixed heap until OOM), per-kernel roofline of
the dominant step kernel, the end-to-end figure through host buffers, and the
oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dsoa|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "app steps/s (graph+persistent vs plain); alloc+free ops/s; do-all HBM GB/s"
WORKLOAD = "wa-tor 1024x1024 torus, 30% fish / 5% sharks, 500 steps"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=490)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="dsoa", choices=["dsoa", "reference"])
    p.add_argument("--skip-secondary", action="store_true", help="headline legs only")
    return p.parse_args()


def ncu_traffic(kernel: str, units: float, key: str = "dram_bytes_per_unit"):
    """DRAM bytes (read + write) per launch of `kernel` (or, with `key`, another
    per-unit counter) from an ncu capture recorded in profiles/ncu_traffic.json,
    scaled to `units` (objects) per launch; None when there is no capture or the
    kernels changed since (build fingerprint differs)."""
    try:
        from paper_1810_11765_gb300 import build
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)
        if rec.get("fingerprint") != build.fingerprint():
            return None
        k = rec["kernels"][kernel]
        return k[key] * units
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- legs
def ev():
    import torch
    return torch.cuda.Event(enable_timing=True)


def wator_world(seed, heap_bytes=512 << 20, launch=None):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import WatorWorld
    heap = D.Heap(heap_bytes)
    w = WatorWorld(heap)
    heap.freeze()
    if launch:
        from paper_1810_11765_gb300 import autotune
        autotune.apply(heap, launch)
    return heap, w


def run_wator(seed, warmup, steps, mode, flush, launch=None):
    """Returns (per-step ms list, final grid, launches per step)."""
    import torch
    heap, w = wator_world(seed, launch=launch)
    slot = w.add(1024, 1024, seed)
    g = None
    if mode == "graph":
        heap.graph_begin()
        w.step()
        g = heap.graph_end()
    step = (lambda: g.launch()) if g else w.step
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    l0 = heap.launches
    times = []
    for _ in range(steps):
        flush.zero_()
        a, b = ev(), ev()
        a.record()
        step()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    per_step_launches = (heap.launches - l0) / steps if mode == "plain" else None
    torch.cuda.synchronize()
    grid = w.read(slot)
    fish, sharks = w.counts()
    err = heap.get_error()
    fs, ss = heap.type_stats(w.fish_type), heap.type_stats(w.shark_type)
    blocks = fs["blocks"] + ss["blocks"]
    slots = fs["slots"] + ss["slots"]
    frag = {"blocks": blocks, "F": 1.0 - (fs["objects"] + ss["objects"]) / slots if slots else 0.0}
    if g:
        g.close()
    heap.close()
    return times, grid, per_step_launches, (fish, sharks), err, frag


WATOR_KERNELS = [  # (type attr, method, reuses the previous snapshot, algorithmic bytes per agent)
    ("fish_type", "M_WATOR_FISH_CHOOSE", False, 24),
    ("fish_type", "M_WATOR_FISH_MOVE", True, 20),
    ("shark_type", "M_WATOR_SHARK_CHOOSE", False, 28),
    ("shark_type", "M_WATOR_SHARK_MOVE_ADVANCE", True, 32),
]
WATOR_KERNELS_DEFERRED = [  # the same step with births created by the births kernel
    ("fish_type", "M_WATOR_FISH_CHOOSE", False, 24),
    ("fish_type", "M_WATOR_FISH_MOVE_DEFER", True, 20),
    ("fish_type", "K_WATOR_BIRTHS", None, 0),
    ("shark_type", "M_WATOR_SHARK_CHOOSE", False, 28),
    ("shark_type", "M_WATOR_SHARK_MOVE_ADVANCE", True, 32),
]


def wator_kernel_profile(seed, warmup, steps, flush, launch=None):
    """CUDA-event duration of each phase of a plain Wa-Tor step, launched exactly
    as the step launches it (choose methods: enumeration + do-all kernel; move
    methods: one do-all kernel on the choose snapshot)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    heap, w = wator_world(seed, launch=launch)
    w.add(1024, 1024, seed)
    for _ in range(warmup):
        w.step()
    M = heap.info()["num_blocks"]
    acc = {}
    a = w.args()
    for _ in range(steps):
        fish, sharks = w.counts()
        flush.zero_()
        for tattr, meth, reuse, bpa in (WATOR_KERNELS_DEFERRED if w.defer_births else WATOR_KERNELS):
            t = getattr(w, tattr)
            e0, e1 = ev(), ev()
            e0.record()
            if reuse is None:                             # plain kernel over the instances
                heap.run_kernel(getattr(D, meth), 1, a)
            elif reuse:
                heap.parallel_do_enumerated(t, getattr(D, meth), a)
            else:
                heap.parallel_do(t, getattr(D, meth), a)
            e1.record()
            e1.synchronize()
            n_agents = fish if tattr == "fish_type" else sharks
            blocks = n_agents / 64.0
            alg = n_agents * bpa + blocks * 12            # fields + R / snapshot read
            if reuse is None:                             # births: the occupancy grid scanned once
                alg = 1024 * 1024
            elif not reuse:                               # enumeration inside the kernel
                alg += M / 8.0 + blocks * (12 + 8)        # level-0 bitmap, R/snapshot write, slot words
            r = acc.setdefault(meth, {"ms": [], "bytes": [], "units": []})
            r["ms"].append(e0.elapsed_time(e1))
            r["bytes"].append(alg)
            r["units"].append(n_agents)
    torch.cuda.synchronize()
    heap.close()
    return acc


DOALL_KERNELS = {"vec128": ("M_MICRO_SCALE", "k_micro_scale_vec<4,2>"),
                 "bulk": ("M_MICRO_SCALE_TMA", "k_micro_scale_bulk<8,4>")}


def doall_sweep(log2n, holes, flush, iters=10, kernel="vec128"):
    """do-all HBM GB/s of an SOA do-all kernel (x = x*1.5f + id)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    n = 1 << log2n
    m = Micro(int(n * 16 * 1.3) + (64 << 20), 0x5EED0001, n)
    m.new(0)
    if holes:
        m.delete(0)
    live = m.heap.count(m.type)
    m.heap.enumerate(m.type)
    args = m.args()
    meth = getattr(D, DOALL_KERNELS[kernel][0])
    single = []
    for _ in range(3):                      # one launch, L2 flushed before it
        flush.zero_()
        a, b = ev(), ev()
        a.record()
        m.heap.parallel_do_enumerated(m.type, meth, args)
        b.record()
        b.synchronize()
        single.append(a.elapsed_time(b))
    # average launch duration over back-to-back launches (every launch streams the
    # whole >L2 object set, so no flush is needed between them)
    m.heap.parallel_do_enumerated(m.type, meth, args)
    a, b = ev(), ev()
    a.record()
    for _ in range(iters):
        m.heap.parallel_do_enumerated(m.type, meth, args)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / iters
    err = m.heap.get_error()
    m.heap.close()
    del m
    torch.cuda.empty_cache()
    return {"objects": live, "ms": ms, "alg_bytes": live * 12, "gbs": live * 12 / ms / 1e6,
            "single_launch_ms": statistics.median(single), "err": err}


def bitmap_legs(flush):
    """BitmapAlloc (Sec. 6), the flat AOS bitmap allocator, on the same microbench
    workloads as DynaSOAr: do-all HBM GB/s on 2^26 objects (full and 50 % holes),
    the alloc/free storm at 2^24 and the heap utilisation of a 1 GiB heap."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    out = {}
    for holes in (False, True):
        n = 1 << 26
        nbytes = int(n * 16 * 1.1) + (64 << 20)
        m = Micro(nbytes, 0x5EED0001, n, heap=D.BitmapHeap(nbytes))
        m.new(0)
        if holes:
            m.delete(0)
        live = m.heap.count(m.type)
        m.scale()
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            flush.zero_()
            a, b = ev(), ev()
            a.record()
            m.scale()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        out[f"doall_2^26{'_holes' if holes else ''}"] = {
            "objects": live, "ms": ms, "gbs": live * 12 / ms / 1e6, "err": m.heap.get_error(),
            "note": "snapshot copy + do-all over the allocation bitmap, L2 flushed before each launch"}
        m.heap.close()
        del m
        torch.cuda.empty_cache()
    n = 1 << 24
    nbytes = int(n * 16 * 1.2) + (64 << 20)
    m = Micro(nbytes, 0x5EED0001, n, heap=D.BitmapHeap(nbytes))
    res = []
    for _ in range(3):
        flush.zero_()
        a, b, c = ev(), ev(), ev()
        a.record()
        m.new(0)
        b.record()
        m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
        c.record()
        c.synchronize()
        res.append((a.elapsed_time(b), b.elapsed_time(c)))
    new_ms = statistics.median(r[0] for r in res)
    del_ms = statistics.median(r[1] for r in res)
    out["alloc_free_2^24"] = {"new_ms": new_ms, "delete_ms": del_ms, "ops_per_s": 2 * n / ((new_ms + del_ms) / 1e3),
                              "left": m.heap.count(m.type), "err": m.heap.get_error()}
    m.heap.close()
    del m
    torch.cuda.empty_cache()
    heap_bytes = 1 << 30
    m = Micro(heap_bytes, 0x5EED0001, 1 << 20, heap=D.BitmapHeap(heap_bytes))
    cap = m.heap.info()["num_slots"]
    rnd = 0
    while True:
        m.new(rnd)
        rnd += 1
        if m.heap.get_error() or rnd * (1 << 20) > cap + (1 << 20):
            break
    live = m.heap.count(m.type)
    out["heap_utilisation"] = {"heap_bytes": heap_bytes, "objects": live, "object_bytes": 16,
                               "utilisation": live * 16 / heap_bytes}
    m.heap.close()
    torch.cuda.empty_cache()
    return out


def alloc_free_storm(log2n, flush, iters=3):
    """parallel_new of 2^log2n objects into an empty heap, then delete-all."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    n = 1 << log2n
    m = Micro(int(n * 16 * 2.2) + (64 << 20), 0x5EED0001, n)
    res = []
    for _ in range(iters):
        flush.zero_()
        a, b, c = ev(), ev(), ev()
        a.record()
        m.new(0)
        b.record()
        m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
        c.record()
        c.synchronize()
        res.append((a.elapsed_time(b), b.elapsed_time(c)))
    left = m.heap.count(m.type)
    err = m.heap.get_error()
    m.heap.close()
    torch.cuda.empty_cache()
    new_ms = statistics.median(r[0] for r in res)
    del_ms = statistics.median(r[1] for r in res)
    return {"objects": n, "new_ms": new_ms, "delete_ms": del_ms,
            "ops_per_s": 2 * n / ((new_ms + del_ms) / 1e3), "left": left, "err": err}


def alloc_linux_scalability(threads, per_thread, flush, iters=3):
    """The Linux-scalability allocation pattern (Sec. 6.5): `threads` threads each
    create `per_thread` objects one after another (K_MICRO_NEW_EACH), then every
    object is deleted (delete-all do-all)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    n = threads * per_thread
    m = Micro(int(n * 16 * 2.2) + (64 << 20), 0x5EED0001, n)
    a = m.args(round=per_thread, n_ids=m.type)
    res = []
    for _ in range(iters):
        flush.zero_()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record()
        m.heap.run_kernel(D.K_MICRO_NEW_EACH, threads, a)
        e1.record()
        m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
        e2.record()
        e2.synchronize()
        res.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
    left = m.heap.count(m.type)
    err = m.heap.get_error()
    m.heap.close()
    torch.cuda.empty_cache()
    new_ms = statistics.median(r[0] for r in res)
    del_ms = statistics.median(r[1] for r in res)
    return {"threads": threads, "per_thread": per_thread, "objects": n, "new_ms": new_ms, "delete_ms": del_ms,
            "ops_per_s": 2 * n / ((new_ms + del_ms) / 1e3), "new_per_s": n / (new_ms / 1e3), "left": left,
            "err": err}


# Minimum bitmap atomics of the method for the storm's pattern (full warps of one
# type into an empty heap, then delete-all), per 64-object block:
#   new:    free-bitmap take, allocated set, active set, 1 warp reservation (the
#           other is folded into the block's initialisation), active clear
#           when full                                                     = 5
#   delete: 2 warp-combined releases, active set at the first free,
#           invalidate, active clear, allocated clear, free set           = 7
# (upper-level propagation, once per 64 blocks per bitmap, not counted).
ALG_ATOMICS_PER_OBJECT = {"new": 5 / 64, "delete": 7 / 64}


def l2_atomic_peak(iters=64, reps=5, words=1 << 22):
    """Ceiling of single-lane 64-bit bitmap atomics with return: every lane's op
    is its own L2 request, on a 32 MiB (L2-resident) word array, one resident
    grid of threads (the K_MICRO_ATOMIC_PEAK probe of the library).  With
    words=32 every op contends with ~10^4 others on 32 words."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(4 << 20, 0x5EED0001, 64)
    nw = words
    buf = torch.zeros(nw, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    n = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 2048
    if nw < 1024:
        iters = 4
    a = m.args(handles_out=buf.data_ptr(), n_ids=nw, round=iters, stats=sink.data_ptr(), seed=1)
    for _ in range(3):
        m.heap.run_kernel(D.K_MICRO_ATOMIC_PEAK, n, a)
    ts = []
    for _ in range(reps):
        e0, e1 = ev(), ev()
        e0.record()
        m.heap.run_kernel(D.K_MICRO_ATOMIC_PEAK, n, a)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    m.heap.close()
    ms = statistics.median(ts)
    return {"atomics_per_s": n * iters / (ms / 1e3), "ms": ms, "threads": n, "ops_per_thread": iters,
            "words": nw}


def alloc_roofline(storm, peak):
    n = storm["objects"]
    alg = {k: v * n for k, v in ALG_ATOMICS_PER_OBJECT.items()}
    rate = (alg["new"] + alg["delete"]) / ((storm["new_ms"] + storm["delete_ms"]) / 1e3)
    p = peak["atomics_per_s"]
    key = "atomic_instructions_per_unit"
    t_new = ncu_traffic("dsoa_new_kernel<MicroCtor>", n, key)
    t_del = ncu_traffic("dsoa_doall_kernel<MicroDeleteAll>", n, key)
    return {"kernel": "dsoa_new_kernel<MicroCtor> + do-all MicroDeleteAll", "bound": "l2_atomic",
            "achieved": rate / 1e9, "peak": p / 1e9, "unit": "Gatomic/s", "frac": rate / p,
            "traffic": None if t_new is None or t_del is None else t_new + t_del,
            "traffic_unit": "atomic operations issued per storm (ncu smsp__sass_inst_executed_op_global_atom; "
                            "every allocator atomic is single-lane)",
            "alg_atomics_per_storm": alg["new"] + alg["delete"],
            "new": {"achieved": alg["new"] / (storm["new_ms"] / 1e3) / 1e9,
                    "frac": alg["new"] / (storm["new_ms"] / 1e3) / p},
            "delete": {"achieved": alg["delete"] / (storm["delete_ms"] / 1e3) / 1e9,
                       "frac": alg["delete"] / (storm["delete_ms"] / 1e3) / p},
            "peak_kind": "measured live: K_MICRO_ATOMIC_PEAK probe"}


def heap_utilisation(heap_bytes=1 << 30, object_bytes=16, threads=1 << 20):
    """Fill a fixed heap with objects until allocation fails (Sec. 6.5), `threads`
    new() per round.  16-byte objects are the microbench type; 64-byte objects a
    subtype of it with six more 8-byte fields (the Linux-scalability shape of
    Sec. 6.5: 16,384 threads per round, 64-byte objects, 1 GiB heap)."""
    import torch
    from paper_1810_11765_gb300.apps import Micro
    extra = None if object_bytes == 16 else [8] * ((object_bytes - 16) // 8)
    m = Micro(heap_bytes, 0x5EED0001, threads, sub_fields=extra, sub_share=1.0)
    t = m.type if extra is None else m.sub_type
    cap = m.heap.info()["num_blocks"] * 64
    rnd = 0
    while True:
        m.new(rnd)
        rnd += 1
        if m.heap.get_error() or rnd * threads > cap + threads:
            break
    live = m.heap.count(t)
    m.heap.close()
    torch.cuda.empty_cache()
    return {"heap_bytes": heap_bytes, "objects": live, "object_bytes": object_bytes,
            "threads_per_round": threads, "utilisation": live * object_bytes / heap_bytes}


def largest_instance(kind, heap_bytes=64 << 20, steps=40, mode=0, lo=64, hi=4096):
    """Largest torus side (a multiple of 32) of a game-of-life or Wa-Tor instance
    whose objects fit in a heap of `heap_bytes` for `steps` steps without an
    allocation failure, by bisection (the grids live outside the heap)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D, inputs
    from paper_1810_11765_gb300.apps import GolWorld, WatorWorld

    def fits(side):
        heap = D.Heap(heap_bytes)
        w = GolWorld(heap) if kind == "gol" else WatorWorld(heap)
        heap.set_capacity_mode(mode)
        heap.freeze()
        seed = inputs.GolConfig().seed if kind == "gol" else inputs.WatorConfig().seed
        ok = True
        try:
            w.add(side, side, seed)
            for _ in range(steps):
                w.step()
            ok = heap.get_error() == 0
        finally:
            heap.close()
            del w
            torch.cuda.empty_cache()
        return ok

    lo_s, hi_s = lo // 32, hi // 32 + 1          # fits(lo) assumed, fits(hi + 32) not
    if not fits(lo):
        return 0
    while hi_s - lo_s > 1:
        mid = (lo_s + hi_s) // 2
        if fits(mid * 32):
            lo_s = mid
        else:
            hi_s = mid
    return lo_s * 32


def largest_instance_leg(heap_bytes=64 << 20, steps=40):
    from paper_1810_11765_gb300 import dsoa as D
    out = {"heap_bytes": heap_bytes, "steps": steps,
           "method": "bisection over the torus side (multiples of 32); fits = no allocation failure"}
    for kind in ("wator", "gol"):
        for name, mode in (("uniform", D.CAPACITY_UNIFORM), ("per_type", D.CAPACITY_PER_TYPE)):
            side = largest_instance(kind, heap_bytes, steps, mode)
            out[f"{kind}_{name}"] = {"side": side, "cells": side * side}
    return out


def e2e_wator(seed, warmup, steps, flush, launch=None):
    """Whole job through the public API with host buffers: initial grid uploaded
    from pinned host memory, K graph steps, each step's populations stored into
    pinned host memory by the step's count kernel, final grid read back."""
    import numpy as np
    import torch
    heap, w = wator_world(seed)
    s0 = w.add(1024, 1024, seed)
    host_grid = torch.from_numpy(w.read(s0).copy()).pin_memory()
    heap.close()
    heap, w = wator_world(seed, launch=launch)
    # the populations of every step are stored by the count kernel straight into
    # pinned host memory (mapped into the device's address space): no copy
    counts_host = torch.zeros(2, dtype=torch.int64).pin_memory()
    out_host = torch.zeros(1024 * 1024, dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    flush.zero_()
    a, b = ev(), ev()
    a.record()
    dev_grid = host_grid.to("cuda", non_blocking=True)
    slot = w.add(1024, 1024, seed, init=dev_grid.view(-1))
    heap.graph_begin()                   # one step and its populations, as one graph
    w.step()
    heap.count_many_async([w.fish_type, w.shark_type], counts_host)
    g = heap.graph_end()
    for _ in range(steps):
        g.launch()
    out_host.copy_(w.bufs[slot][1], non_blocking=True)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    g.close()
    heap.close()
    h2d = 1024 * 1024
    return {"value": steps / (ms / 1e3), "unit": "steps/s",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": 16 + 1024 * 1024 / steps,
            "ms": ms, "final_fish": int(counts_host[0]), "final_sharks": int(counts_host[1])}


def app_steps(kind, steps, flush, warmup=3, side=None, heap_bytes=1 << 30):
    """Steps/s of the other apps, graph-captured step vs plain launches (L2
    flushed between timed steps).  `side` overrides the game-of-life torus side."""
    import numpy as np
    import torch
    from paper_1810_11765_gb300 import dsoa as D, inputs
    from paper_1810_11765_gb300.apps import GolWorld, TrafficWorld
    res, finals = {}, {}
    for mode in ("plain", "graph"):
        heap = D.Heap(heap_bytes)
        if kind == "gol":
            cfg = inputs.GolConfig()
            w = GolWorld(heap)
            heap.freeze()
            w.add(side or cfg.width, side or cfg.height, cfg.seed)
        else:
            L, thr = inputs.traffic_instances()
            w = TrafficWorld(heap, L, thr, inputs.SEED_TRAFFIC)
            heap.freeze()
            w.init()
        g = None
        if mode == "graph":
            heap.graph_begin()
            w.step()
            g = heap.graph_end()
        step = (lambda: g.launch()) if g else w.step
        for _ in range(warmup):
            step()
        times = []
        for _ in range(steps):
            flush.zero_()
            a, b = ev(), ev()
            a.record()
            step()
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        res[f"{mode}_steps_per_s"] = steps / (sum(times) / 1e3)
        res["device_errors"] = heap.get_error()
        state = w.read(0) if kind == "gol" else np.concatenate(w.read())
        finals[mode] = hashlib.sha256(np.ascontiguousarray(state).tobytes()).hexdigest()
        if g:
            g.close()
        heap.close()
    res["graph_vs_plain"] = res["graph_steps_per_s"] / res["plain_steps_per_s"]
    res["graph_equals_plain"] = finals["graph"] == finals["plain"]
    gs = side or 512
    res["workload"] = (f"game of life {gs}x{gs} torus, density 1/4" if kind == "gol"
                       else "traffic: 64 Nagel-Schreckenberg rings, 2^12..2^20 cells")
    return res


# Algorithmic operations of one unordered pair of the n-body force (both bodies'
# terms) in the configured workload, where G S is a power of two and the masses
# are small integers, so (G S m_i) m_j = (G S m_j) m_i and j's term is the negated
# i term: dx, dy (2 sub), d2 (2 mul, 2 add), sqrt, reciprocal, d^-3 (2 mul), the
# coefficient k (2 mul), k dx and k dy (2 mul), two conversions to the fixed-point
# grid, four adds (i and j).  With unequal coefficients it is 26 (a second k and
# its two products and conversions).
NBODY_OPS_PER_UNORDERED_PAIR = 20


def fp32_lane_peak(clock_mhz):
    """FP32 lane operations per second: SMs x 128 lanes x SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * clock_mhz * 1e6


def issue_peak(clock_mhz):
    """Warp instructions issued per second: SMs x 4 schedulers x 1 per cycle x SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 4 * clock_mhz * 1e6


def nbody_leg(flush, steps=5, collide_steps=10):
    """n-body (65,536 bodies, the listing's size): FORCE by the pairwise tiled
    kernel over unordered pairs (the default) and over ordered pairs, and by the
    per-thread device_do walk; steps/s plain vs graph; particle collisions on the
    same bodies (six do-alls per step)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D, inputs
    from paper_1810_11765_gb300.apps import NBodyWorld
    cfg = inputs.NBodyConfig()
    n = cfg.n
    out = {"workload": f"n-body {n} bodies in [-1,1)^2, integer masses 1..{cfg.mass_max}, G=2^-30, dt=1/4",
           "pairs_per_force": n * (n - 1)}
    for key, tiled, all_pairs in (("tiled", True, False), ("tiled_ordered", True, True), ("device_do", False, False)):
        heap = D.Heap(256 << 20)
        w = NBodyWorld(heap, cfg, tiled=tiled, all_pairs=all_pairs)
        heap.freeze()
        w.create(n)
        w.step()
        torch.cuda.synchronize()
        k = steps if tiled else 1
        flush.zero_()
        a, b = ev(), ev()
        a.record()
        for _ in range(k):
            w.force()
        b.record()
        b.synchronize()
        force_ms = a.elapsed_time(b) / k
        w.step()          # apply (and clear) the forces accumulated above
        out[f"force_ms_{key}"] = force_ms
        out[f"pair_terms_per_s_{key}"] = n * (n - 1) / (force_ms / 1e3)
        if key == "tiled":
            for mode in ("plain", "graph"):
                g = None
                if mode == "graph":
                    heap.graph_begin()
                    w.step()
                    g = heap.graph_end()
                step = (lambda: g.launch()) if g else w.step
                step()
                torch.cuda.synchronize()
                a, b = ev(), ev()
                a.record()
                for _ in range(steps):
                    step()
                b.record()
                b.synchronize()
                out[f"{mode}_steps_per_s"] = steps / (a.elapsed_time(b) / 1e3)
                if g:
                    g.close()
        out[f"device_errors_{key}"] = heap.get_error()
        heap.close()
    # collisions: 10 steps from the initial draw, plain launches
    heap = D.Heap(256 << 20)
    w = NBodyWorld(heap, cfg, collide=True, tiled=True)
    heap.freeze()
    w.create(n)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    for _ in range(collide_steps):
        w.step()
    b.record()
    b.synchronize()
    out["collision"] = {"steps": collide_steps, "steps_per_s": collide_steps / (a.elapsed_time(b) / 1e3),
                        "bodies_after": w.count(), "device_errors": heap.get_error()}
    heap.close()
    return out


def serving_leg(n_req=24, multiples=(0.25, 0.5, 1.0, 2.0)):
    """Continuous batching of game-of-life / wa-tor instances as configured: sides
    round(2^U(8,12)), 100..1000 steps, one heap capped at 64 GiB.  The service rate
    is measured first with every request arriving at once (requests / wall time);
    Poisson arrival rates are then swept as multiples of it."""
    from paper_1810_11765_gb300 import inputs
    from paper_1810_11765_gb300.serving import Server

    def run(rate):
        reqs = inputs.serving_requests(n_req, rate_per_s=rate)
        srv = Server(64 << 30, capacity=32)
        _, summary = srv.run(reqs)
        srv.close()
        summary.pop("rejected", None)
        return summary

    burst = run(1e9)                               # all arrivals at t = 0
    service_rate = n_req / burst["wall_s"]
    out = [{"rate_per_s": None, "arrivals": "all at once", "service_rate_per_s": service_rate, **burst}]
    for m in multiples:
        out.append({"rate_per_s": m * service_rate, "rate_vs_service": m, **run(m * service_rate)})
    return out


def cpu_baselines_secondary():
    """The oracle on bounded samples of the secondary workloads (single-threaded):
    n-body pair terms/s and microbench objects/s (new + do-all + delete per round)."""
    import oracle
    from paper_1810_11765_gb300 import inputs
    c = inputs.NBodyConfig()
    n = 4096
    t0 = time.perf_counter()
    oracle.nbody_run(n, 1, c.seed, G=c.G, dt=c.dt, eps2=c.eps2, rc2=c.rc2, fscale=c.fscale,
                     vscale=c.vscale, mass_max=c.mass_max)
    dt_nb = time.perf_counter() - t0
    m = inputs.MicroConfig()
    t0 = time.perf_counter()
    oracle.micro_run(m.seed, m.n_per_round, m.rounds)
    dt_mi = time.perf_counter() - t0
    return {"nbody": {"value": n * (n - 1) / dt_nb, "unit": "pair terms/s", "cores": 1, "kind": "oracle",
                      "sample": f"one FORCE + MOVE step of {n} bodies of the n-body workload"},
            "microbench": {"value": m.n_per_round * m.rounds / dt_mi, "unit": "objects/s", "cores": 1,
                           "kind": "oracle",
                           "sample": f"the configured microbench: {m.rounds} rounds of {m.n_per_round} new, "
                                     "do-all, parity delete"}}


def cpu_baseline(seed, sample_steps=100):
    import oracle
    t0 = time.perf_counter()
    oracle.wator_run(1024, 1024, sample_steps, seed=seed)
    dt = time.perf_counter() - t0
    return {"value": sample_steps / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first {sample_steps} steps of the same 1024x1024 wa-tor run (seed {seed:#x}), "
                      "single-threaded sequential oracle incl. its initialisation"}


# ----------------------------------------------------------------------------- arms
def reference_arm(args):
    """The oracle as the reference arm, on the same workload and metric."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import oracle
    from paper_1810_11765_gb300 import inputs
    seed = inputs.WatorConfig().seed
    oracle.build()
    t0 = time.perf_counter()
    oracle.wator_run(1024, 1024, args.warmup, seed=seed)
    t1 = time.perf_counter()
    oracle.wator_run(1024, 1024, args.warmup + args.steps, seed=seed)
    t2 = time.perf_counter()
    dt = max((t2 - t1) - (t1 - t0), 1e-9)
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "seed": seed, "mode": "sequential CPU oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "steps/s",
                             "sample": f"{args.steps} steps after {args.warmup} warm-up steps of the "
                                       "1024x1024 wa-tor run (difference of two runs)"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def dsoa_arm(args):
    import numpy as np
    import torch
    from paper_1810_11765_gb300 import build, inputs
    from paper_1810_11765_gb300.replicas import Replicas, rank_seed
    dist = Replicas()
    dev = dist.local if dist.world > 1 else 0
    torch.cuda.set_device(dev)
    build.build()
    # every heap and torch op of the bench runs on one non-default stream, which
    # stream capture (CUDA graphs) requires; events are recorded on it too
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    cfg = inputs.WatorConfig()
    seed = rank_seed(cfg.seed, dist.rank)      # one independent replica per rank
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    hbm_peak, peak_kind = peaks()

    from paper_1810_11765_gb300 import autotune
    launch = autotune.best_wator_launch(seed)

    # --- headline: graph + persistent do-all, L2 flushed between timed steps
    clocks = ClockSampler(dev)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_graph, grid_g, _, pop_g, err_g, frag_g = run_wator(seed, args.warmup, args.steps, "graph", flush, launch)
    dist.barrier()
    ms_graph = dist.max(sum(t_graph))         # slowest rank decides
    t_plain, grid_p, launches_per_step, pop_p, err_p, _ = run_wator(seed, args.warmup, args.steps, "plain",
                                                                    flush, launch)
    clk = clocks.stop()                       # sampled over both timed headline runs
    ms_plain = dist.max(sum(t_plain))
    same = bool(np.array_equal(grid_g, grid_p)) and pop_g == pop_p and err_g == 0 and err_p == 0
    value = dist.world * args.steps / (ms_graph / 1e3)
    plain_value = dist.world * args.steps / (ms_plain / 1e3)

    out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": dist.world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "seed": cfg.seed, "mode": "graph+persistent do-all",
                      "l2": "flushed (256 MiB write) between timed steps, outside the timed region",
                      "parallelism": f"replicas x{dist.world}", "launch": launch},
           "plain_steps_per_s": plain_value, "graph_steps_per_s": value,
           "graph_vs_plain": ms_plain / ms_graph, "graph_equals_plain": same,
           "populations_after": {"fish": pop_g[0], "sharks": pop_g[1],
                                 "steps": args.warmup + args.steps},
           "fragmentation_after": frag_g,
           "gpu_launches": int(round(launches_per_step * args.steps)) if launches_per_step else None,
           "clocks": clk}

    if dist.rank == 0 and not args.skip_secondary:
        # --- dominant kernel of the step, with its roofline
        prof = wator_kernel_profile(seed, 20, 20, flush, launch)
        tot = {k: sum(v["ms"]) for k, v in prof.items()}
        dom = max(tot, key=tot.get)
        d = prof[dom]
        avg_ms = statistics.mean(d["ms"])
        alg = statistics.mean(d["bytes"])
        ach = alg / (avg_ms / 1e3) / 1e9
        units = statistics.mean(d["units"])
        # traffic inside a step (ncu without cache control on a run that flushes L2
        # between steps, as here); the cold-cache figure (caches flushed before the
        # kernel alone) beside it
        t_step = ncu_traffic(dom, units, "dram_bytes_in_step_per_unit")
        t_cold = ncu_traffic(dom, units)
        out["roofline"] = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                           "unit": "GB/s", "frac": ach / hbm_peak,
                           "traffic": t_step if t_step is not None else t_cold,
                           "traffic_kind": "in step" if t_step is not None else "cold caches",
                           "traffic_cold": t_cold,
                           "peak_kind": peak_kind, "avg_launch_ms": avg_ms, "alg_bytes_per_launch": alg,
                           "units_per_launch": units}
        out["step_kernels_ms"] = {k: statistics.mean(v["ms"]) for k, v in prof.items()}
        out["step_phases"] = {k: {"ms": statistics.mean(v["ms"]),
                                  "alg_gbs": statistics.mean(v["bytes"]) / statistics.mean(v["ms"]) / 1e6,
                                  "frac_hbm": statistics.mean(v["bytes"]) / statistics.mean(v["ms"]) / 1e6
                                  / hbm_peak,
                                  "agents": statistics.mean(v["units"])} for k, v in prof.items()}
        # --- do-all HBM sweep (spec kernel), > L2 working sets
        sweep = {}
        for kern in DOALL_KERNELS:
            for lg, holes in ((26, False), (26, True), (24, False), (28, False)):
                r = doall_sweep(lg, holes, flush, kernel=kern)
                sweep[f"{kern}:2^{lg}{'_holes' if holes else ''}"] = r
        kbest = max(DOALL_KERNELS, key=lambda k: sweep[f"{k}:2^26"]["gbs"])
        best = sweep[f"{kbest}:2^26"]
        out["doall_hbm_gbs"] = best["gbs"]
        out["doall_hbm_gbs_2^28"] = sweep[f"{kbest}:2^28"]["gbs"]
        out["doall_roofline"] = {"kernel": DOALL_KERNELS[kbest][1], "bound": "hbm", "achieved": best["gbs"],
                                 "peak": hbm_peak, "unit": "GB/s", "frac": best["gbs"] / hbm_peak,
                                 "traffic": ncu_traffic(DOALL_KERNELS[kbest][1], best["objects"]),
                                 "peak_kind": peak_kind,
                                 "alg_bytes_per_launch": best["alg_bytes"], "avg_launch_ms": best["ms"]}
        out["doall_sweep"] = sweep
        # --- alloc + free
        out["l2_atomic_peak"] = l2_atomic_peak()
        out["l2_atomic_contended"] = l2_atomic_peak(words=32)
        # each step phase's L2 atomic rate against the probe's (both as L2 atomic
        # requests, counted by ncu per agent and per probe op)
        probe_req = ncu_traffic("k_atomic_peak", 1.0, "l2_atomic_requests_per_unit")
        for k, ph in out.get("step_phases", {}).items():
            req = ncu_traffic(k, ph["agents"], "l2_atomic_requests_per_unit")
            if req is None or probe_req is None:
                ph["l2_atomic"] = None
                continue
            rate = req / (ph["ms"] / 1e3)
            peak = out["l2_atomic_peak"]["atomics_per_s"] * probe_req
            ph["l2_atomic"] = {"requests_per_agent": req / ph["agents"], "requests_per_s": rate,
                               "peak_requests_per_s": peak, "frac": rate / peak}
        for k, ph in out.get("step_phases", {}).items():
            ph["dram_bytes_per_agent"] = {"in_step": ncu_traffic(k, 1.0, "dram_bytes_in_step_per_unit"),
                                          "cold": ncu_traffic(k, 1.0)}
        sweep = {}
        for lg in (18, 20, 22, 24):      # 2^18 threads' worth x {1, 4, 16, 64} objects
            st = alloc_free_storm(lg, flush)
            st["alloc_roofline_frac"] = alloc_roofline(st, out["l2_atomic_peak"])["frac"]
            sweep[f"2^{lg}"] = st
        storm = sweep["2^24"]
        out["alloc_free_ops_per_s"] = storm["ops_per_s"]
        out["alloc_free"] = storm
        out["alloc_free_sweep"] = sweep
        out["alloc_roofline"] = alloc_roofline(storm, out["l2_atomic_peak"])
        lsc = {}
        for threads in (1 << 18, 1 << 14):
            for k in (1, 4, 16, 64):
                r = alloc_linux_scalability(threads, k, flush)
                r["alloc_roofline_frac"] = alloc_roofline(r, out["l2_atomic_peak"])["frac"]
                lsc[f"{threads}x{k}"] = r
        out["alloc_linux_scalability"] = lsc
        out["heap_utilisation"] = heap_utilisation()
        out["heap_utilisation_64b"] = heap_utilisation(object_bytes=64, threads=16384)
        out["bitmapalloc"] = bitmap_legs(flush)
        out["largest_instance"] = largest_instance_leg()
        # --- other apps (plain vs graph) and serving
        out["gol_512"] = app_steps("gol", 100, flush)
        out["gol_4096"] = app_steps("gol", 20, flush, side=4096)
        out["traffic_64_rings"] = app_steps("traffic", 50, flush)
        out["serving"] = serving_leg()
        nb = nbody_leg(flush)
        clk_mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak_ops = fp32_lane_peak(clk_mhz)
        ach = nb["pair_terms_per_s_tiled"] / 2 * NBODY_OPS_PER_UNORDERED_PAIR
        # the kernel is bound by instruction issue (ncu: 74 % of issue slots):
        # warp instructions per unordered pair from the ncu record, times the
        # unordered pairs per second, against the issue slots of the SMs
        pairs_16k = 16384 * 16383 / 2
        inst_per_pair = ncu_traffic("k_force_sym", 16384, "warp_instructions_per_unit")
        inst_per_pair = None if inst_per_pair is None else inst_per_pair / pairs_16k
        pairs_per_s = nb["pair_terms_per_s_tiled"] / 2
        ipk = issue_peak(clk_mhz)
        iss = None if inst_per_pair is None else pairs_per_s * inst_per_pair
        nb["roofline"] = {"kernel": "k_force_sym", "bound": "issue",
                          "achieved": None if iss is None else iss / 1e9, "peak": ipk / 1e9,
                          "unit": "G warp instructions/s", "frac": None if iss is None else iss / ipk,
                          "warp_instructions_per_unordered_pair": inst_per_pair,
                          "traffic": ncu_traffic("k_force_sym", 1 << 16),
                          "traffic_unit": "DRAM bytes per launch (ncu, scaled per body from a 16,384-body "
                                          "capture: the bodies stay in L2, DRAM traffic grows with n)",
                          "peak_kind": f"derived: SMs x 4 schedulers x 1 warp instruction per cycle x {clk_mhz:.0f} "
                                       "MHz (median SM clock of the headline run)",
                          "alu_lane": {"achieved": ach / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                                       "frac": ach / peak_ops,
                                       "ops_per_unordered_pair": NBODY_OPS_PER_UNORDERED_PAIR,
                                       "peak_kind": f"derived: SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz; optimistic: "
                                                    "the square root, reciprocal and conversions run on the "
                                                    "quarter-rate pipe"}}
        out["nbody_65536"] = nb
        # --- end to end through host buffers
        out["e2e"] = e2e_wator(seed, args.warmup, args.steps, flush, launch)
        # --- oracle on the host cores
        out["cpu_baseline"] = cpu_baseline(seed)
        out["cpu_baselines_secondary"] = cpu_baselines_secondary()
    dist.barrier()
    if dist.rank == 0:
        # the benchmark spec's figures last, so that a tail of the line shows them
        for k in ("alloc_linux_scalability", "step_phases", "e2e", "cpu_baseline", "roofline", "alloc_roofline",
                  "alloc_free_ops_per_s", "doall_roofline", "doall_hbm_gbs_2^28", "doall_hbm_gbs"):
            if k in out:
                out[k] = out.pop(k)
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return dsoa_arm(args)


if __name__ == "__main__":
    sys.exit(main())
