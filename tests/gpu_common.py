"""Helpers of the GPU tests: library build/load and a host-side allocator checker.

The host checker re-derives the hierarchical-bitmap layout from M alone (level l has
ceil(n_l / 64) containers, n_0 = M, n_{l+1} = containers of level l, levels stored
contiguously from level 0) and checks the invariants of Sec. 3.4 / App. A.4 with
numpy, independently of the library's own device checker.
"""
import numpy as np


def gpu_ready():
    from paper_1810_11765_gb300 import build
    build.build()
    import torch
    torch.cuda.init()


def levels_of(M):
    words, out = (M + 63) // 64, []
    while True:
        out.append(words)
        if words == 1:
            return out
        words = (words + 63) // 64


def bits_of(words: np.ndarray, n: int) -> np.ndarray:
    b = np.unpackbits(words.view(np.uint8), bitorder="little")
    return b[:n].astype(bool)


def host_check(heap, ntypes: int) -> dict:
    st = heap.export_state()
    M = heap.info()["num_blocks"]
    lv = levels_of(M)
    offs = np.concatenate([[0], np.cumsum(lv)])
    slot, btype, bms = st["slot"], st["btype"], st["bitmaps"]
    assert bms.shape[0] == 1 + 2 * ntypes
    bad = {"hier": 0, "free_xor": 0, "active_subset": 0, "type": 0, "free_word": 0,
           "empty_alloc": 0, "active_exact": 0, "tail": 0}
    L0 = []
    for b in range(bms.shape[0]):
        prev_n = M
        for l, nw in enumerate(lv):
            words = bms[b, offs[l]:offs[l] + nw]
            bits = bits_of(words, nw * 64)
            if bits[prev_n:].any():
                bad["tail"] += 1
            if l == 0:
                L0.append(bits[:M])
            else:
                lower = bms[b, offs[l - 1]:offs[l - 1] + prev_n]
                bad["hier"] += int(np.sum(bits[:prev_n] != (lower != 0)))
            prev_n = nw
    free = L0[0]
    # usable slots of a block of each type (block capacity N_T, Sec. 3.2); the
    # slots above stay marked free in the slot word
    caps = [heap.capacity(t) for t in range(ntypes)]
    capmask = [np.uint64(2**64 - 1) if n >= 64 else np.uint64((1 << n) - 1) for n in caps]
    alloc = np.array([L0[1 + 2 * t] for t in range(ntypes)])
    active = np.array([L0[2 + 2 * t] for t in range(ntypes)])
    any_alloc = alloc.any(axis=0)
    bad["free_xor"] = int(np.sum(free == any_alloc)) + int(np.sum(alloc.sum(axis=0) > 1))
    bad["active_subset"] = int(np.sum(active & ~alloc))
    bad["free_word"] = int(np.sum(free & (slot != 0)))
    bad["cap_bits"] = 0
    live = {}
    free_slots, total_slots = 0, 0
    for t in range(ntypes):
        sel = alloc[t]
        bad["type"] += int(np.sum(btype[sel] != t))
        bad["empty_alloc"] += int(np.sum(slot[sel] == np.uint64(2**64 - 1)))
        bad["active_exact"] += int(np.sum(active[t][sel] != ((slot[sel] & capmask[t]) != 0)))
        bad["cap_bits"] += int(np.sum((~slot[sel] & ~capmask[t]) != 0))
        occ = ~slot[sel]
        live[t] = int(np.unpackbits(occ.view(np.uint8)).sum())
        free_slots += int(np.unpackbits((slot[sel] & capmask[t]).view(np.uint8)).sum())
        total_slots += caps[t] * int(sel.sum())
    return {"violations": bad, "live": live, "blocks_in_use": int(any_alloc.sum()),
            "fragmentation": free_slots / total_slots if total_slots else 0.0}
