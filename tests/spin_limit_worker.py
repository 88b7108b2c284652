"""Runs workloads on a test build of the library whose bounded waits give up early.

Started as a subprocess by ``test_gpu_spin_limit.py`` with the path of a library
built with a tiny ``DSOA_SPIN_LIMIT``, so that look-back waits and blocking bitmap
updates run into their bound.  Prints one JSON line with what it observed; the
test asserts on it.  Every wait in the library is bounded, a look-back that gives
up publishes an empty snapshot, and every index a method reads from an object
field is checked before it addresses an application array, so the calls return
and report errors instead of hanging or touching memory out of bounds.
"""
import json
import sys

import numpy as np
import torch

from paper_1810_11765_gb300 import dsoa as D

SEED = 0x5EED0001
KNOWN = D.DEV_OOM | D.DEV_SPIN | D.DEV_DOUBLE_FREE | D.DEV_BAD_HANDLE | D.DEV_BAD_INDEX


class _DeviceArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def _dev(ptr, n, typestr):
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda").cpu().numpy()


def enumeration(heap_bytes, flags, repeats):
    """Enumerations of one type, each compared with the allocated-block bitmap."""
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(heap_bytes, SEED, 1 << 20)
    m.heap.set_flags(flags)
    m.new(0)
    torch.cuda.synchronize()
    st = m.heap.export_state()
    M = m.heap.info()["num_blocks"]
    words = (M + 63) // 64
    alloc = np.unpackbits(st["bitmaps"][1, :words].view(np.uint8), bitorder="little")[:M].astype(bool)
    want_R = np.nonzero(alloc)[0].astype(np.uint32)
    want_occ = ~st["slot"][want_R]
    out = {"M": M, "blocks": int(want_R.size), "runs": 0, "gave_up": 0, "exact": 0,
           "r_when_gave_up": [], "R_in_bounds": True, "other_bits": 0, "mismatch": 0}
    m.heap.get_error()
    for _ in range(repeats):
        R, occ, r = m.heap.enumerate(m.type)
        torch.cuda.synchronize()
        err = m.heap.get_error()
        n = int(_dev(r, 1, "<u4")[0])
        Rall = _dev(R, M, "<u4")
        out["runs"] += 1
        out["R_in_bounds"] &= bool((Rall < M).all())
        out["other_bits"] |= err & ~D.DEV_SPIN
        if err & D.DEV_SPIN:
            out["gave_up"] += 1
            out["r_when_gave_up"].append(n)
        elif n == want_R.size and np.array_equal(Rall[:n], want_R) and \
                np.array_equal(_dev(occ, max(n, 1), "<u8")[:n], want_occ):
            out["exact"] += 1
        else:
            out["mismatch"] += 1
        if out["gave_up"] >= 5 and out["exact"] >= 1:
            break
    m.heap.close()
    return out


def workloads():
    """Small runs of every workload; only what the calls report is recorded."""
    from paper_1810_11765_gb300 import apps
    res = {}

    def finish(name, heap):
        torch.cuda.synchronize()
        err = heap.get_error()
        chk = heap.check()
        res[name] = {"err": err, "unknown_bits": err & ~KNOWN, "check_ran": isinstance(chk, dict)}
        heap.close()

    m = apps.Micro(64 << 20, SEED, 1 << 18)
    for rnd in range(4):
        m.round(rnd)
    m.stats()
    finish("micro", m.heap)

    heap = D.Heap(64 << 20)
    w = apps.WatorWorld(heap, 1)
    heap.freeze()
    w.add(128, 128, 0x5EED0003)
    for _ in range(30):
        w.step()
    w.counts()
    w.read(0)
    finish("wator", heap)

    heap = D.Heap(64 << 20)
    g = apps.GolWorld(heap, 1)
    heap.freeze()
    g.add(128, 128, 0x5EED0002)
    for _ in range(30):
        g.step()
    g.read(0)
    finish("gol", heap)

    heap = D.Heap(64 << 20)
    L = np.array([4096, 5000, 6000, 8192], np.uint64)
    thr = np.full(4, 858993459, np.uint32)
    tw = apps.TrafficWorld(heap, L, thr, 0x5EED0004)
    heap.freeze()
    tw.init()
    for _ in range(50):
        tw.step()
    tw.read()
    finish("traffic", heap)
    return res


def main():
    D._lib = D.load(sys.argv[1])
    torch.cuda.init()
    out = {"enumeration": {
        "one_tile_per_cta": enumeration(1 << 30, 0, 200),
        "several_tiles_per_cta": enumeration(8 << 30, 0, 200),
        "tickets": enumeration(1 << 30, D.FLAG_ENUM_TICKETS, 200),
    }, "workloads": workloads()}
    # the context stays usable: a fresh heap on the same library works
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(16 << 20, SEED, 1000)
    m.new(0)
    out["after"] = {"count": m.heap.count(m.type)}
    m.heap.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
