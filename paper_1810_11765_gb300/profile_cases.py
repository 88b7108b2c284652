"""Small, bounded workloads for kernel profiling (ncu) and quick timing.

  python -m paper_1810_11765_gb300.profile_cases doall --log2n 24 [--holes] [--iters 3]
  python -m paper_1810_11765_gb300.profile_cases wator --side 1024 --steps 3 [--defer] [--flush]
  python -m paper_1810_11765_gb300.profile_cases alloc --log2n 22
  python -m paper_1810_11765_gb300.profile_cases atomic --iters 64
  python -m paper_1810_11765_gb300.profile_cases nbody --n 16384 [--walk] [--iters 3]

Each case prints CUDA-event timings of its kernels (without a profiler attached
these are the numbers to trust) and keeps its device footprint to a few hundred MB
so that a multi-pass ncu capture stays small.
"""
from __future__ import annotations

import argparse
import statistics

import torch

from . import build, dsoa as D
from .apps import Micro, NBodyWorld, WatorWorld


def _ev():
    return torch.cuda.Event(enable_timing=True)


METHODS = {"vec": D.M_MICRO_SCALE, "bulk": D.M_MICRO_SCALE_TMA, "scalar": D.M_MICRO_SCALE_SCALAR}


def case_doall(log2n: int, holes: bool, iters: int, method: str = "vec"):
    n = 1 << log2n
    m = Micro(int(n * 16 * 1.3) + (64 << 20), 0x5EED0001, n)
    m.new(0)
    if holes:
        m.delete(0)
    live = m.heap.count(m.type)
    m.heap.enumerate(m.type)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    times = []
    for _ in range(iters):
        flush.zero_()
        a, b = _ev(), _ev()
        a.record()
        m.heap.parallel_do_enumerated(m.type, METHODS[method], m.args())
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    ms = statistics.median(times)
    print(f"doall[{method}] 2^{log2n}{' holes' if holes else ''}: {live} objects, {ms:.4f} ms, "
          f"{live * 12 / ms / 1e6:.1f} GB/s algorithmic, err={m.heap.get_error()}")
    m.heap.close()


def case_wator(side: int, steps: int, defer: bool = False, flush: bool = False):
    """`flush`: a 256 MiB write before every step, as between the benchmark's timed
    steps, so that a capture without cache control sees each kernel's DRAM traffic
    as it is inside a benchmarked step (the first kernel to touch a line reads it).
    A read of a second 256 MiB buffer follows the write, so that the write's dirty
    lines are written back before the step and not counted as the step kernels'
    DRAM writes."""
    heap = D.Heap(512 << 20)
    w = WatorWorld(heap)
    w.defer_births = defer
    heap.freeze()
    w.add(side, side, 0x5EED0003)
    buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if flush else None
    rd = torch.ones(64 << 20, dtype=torch.int32, device="cuda") if flush else None
    for _ in range(steps):
        if buf is not None:
            buf.zero_()
            rd.sum()
        a, b = _ev(), _ev()
        a.record()
        w.step()
        b.record()
        b.synchronize()
        fs, ss = heap.type_stats(w.fish_type), heap.type_stats(w.shark_type)
        print(f"wator {side}^2 step: {a.elapsed_time(b):.4f} ms  populations {w.counts()}  "
              f"blocks {fs['blocks']} / {ss['blocks']}")
    print("err", heap.get_error())
    heap.close()


def case_alloc(log2n: int):
    n = 1 << log2n
    m = Micro(int(n * 16 * 2.2) + (64 << 20), 0x5EED0001, n)
    for it in range(3):
        a, b, c = _ev(), _ev(), _ev()
        a.record()
        m.new(0)
        b.record()
        m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
        c.record()
        c.synchronize()
        print(f"alloc 2^{log2n}: new {a.elapsed_time(b):.3f} ms, delete-all {b.elapsed_time(c):.3f} ms")
    print("err", m.heap.get_error(), "left", m.heap.count(m.type))
    m.heap.close()


def case_atomic(iters: int):
    """The L2 atomic-throughput probe (K_MICRO_ATOMIC_PEAK) on a 32 MiB word array."""
    m = Micro(4 << 20, 0x5EED0001, 64)
    nw = 1 << 22
    words = torch.zeros(nw, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    n = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 2048
    args = m.args(handles_out=words.data_ptr(), n_ids=nw, round=iters, stats=sink.data_ptr(), seed=1)
    for _ in range(3):
        a, b = _ev(), _ev()
        a.record()
        m.heap.run_kernel(D.K_MICRO_ATOMIC_PEAK, n, args)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        print(f"atomic probe: {n} threads x {iters} ops, {ms:.4f} ms, {n * iters / ms / 1e6:.1f} G atomics/s")
    print("err", m.heap.get_error())
    m.heap.close()


def case_nbody(n: int, walk: bool, iters: int, all_pairs: bool = False):
    """FORCE over n bodies of the configured n-body workload: the pairwise tiled
    kernel (over unordered pairs, or ordered ones with ``all_pairs``), or (walk)
    the per-thread device_do walk."""
    from . import inputs
    cfg = inputs.NBodyConfig()
    heap = D.Heap(max(64 << 20, n * 256))
    w = NBodyWorld(heap, cfg, tiled=not walk, all_pairs=all_pairs)
    heap.freeze()
    w.create(n)
    for _ in range(iters):
        a, b = _ev(), _ev()
        a.record()
        w.force()
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        kind = "walk" if walk else ("tiled ordered" if all_pairs else "tiled")
        print(f"nbody[{kind}] n={n}: FORCE {ms:.4f} ms, "
              f"{n * (n - 1) / ms / 1e6:.2f} G pair terms/s")
    print("err", heap.get_error())
    heap.close()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["doall", "wator", "alloc", "atomic", "nbody"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--walk", action="store_true")
    p.add_argument("--all-pairs", action="store_true")
    p.add_argument("--log2n", type=int, default=24)
    p.add_argument("--holes", action="store_true")
    p.add_argument("--iters", type=int, default=3)
    p.add_argument("--method", default="vec", choices=sorted(METHODS))
    p.add_argument("--side", type=int, default=1024)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--defer", action="store_true", help="wator: births allocated by the births kernel")
    p.add_argument("--flush", action="store_true", help="wator: write 256 MiB before every step (L2 flush)")
    a = p.parse_args()
    build.build()
    if a.case == "doall":
        case_doall(a.log2n, a.holes, a.iters, a.method)
    elif a.case == "wator":
        case_wator(a.side, a.steps, a.defer, a.flush)
    elif a.case == "atomic":
        case_atomic(a.iters)
    elif a.case == "nbody":
        case_nbody(a.n, a.walk, a.iters, a.all_pairs)
    else:
        case_alloc(a.log2n)


if __name__ == "__main__":
    main()
