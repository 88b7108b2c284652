"""Hierarchical bitmaps at their level boundaries (Sec. 4.1, nested bitmaps).

A bitmap over M blocks has ceil(M / 64) level-0 words, ceil(M / 4096) level-1
words and so on up to a single top word; the tail bits of the last word of each
level and the propagation between levels are where an off-by-one would hide.
These heaps are cut from one device buffer at byte sizes found by bisection so
that M is exactly 1, 63, 64, 65, 4095, 4096, 4097 and 262,145 (= 64^3 + 1, the
first M with four levels).  Each heap is filled until every slot is used, freed
completely and filled again; the device checker and the independent host
checker must stay clean, and the counts must be exact (64 M objects when full,
0 when empty, every block back in the free bitmap).
"""
import pytest

from gpu_common import gpu_ready, host_check, levels_of

pytestmark = pytest.mark.gpu

SEED = 0x5EED0001
FIELDS = [4, 4, 8]          # the microbench type


@pytest.fixture(scope="module")
def buf():
    gpu_ready()
    import torch
    return torch.empty(400 << 20, dtype=torch.uint8, device="cuda")


def _blocks(buf, nbytes):
    """Block count of a heap of `nbytes` bytes of `buf` (0 if it holds none)."""
    from paper_1810_11765_gb300 import dsoa as D
    h = D.Heap(buffer=buf[:nbytes])
    try:
        h.register_type(FIELDS)
        h.freeze()
        return h.info()["num_blocks"]
    except D.DsoaError:
        return 0
    finally:
        h.close()


def heap_with(buf, M):
    """An unfrozen heap over a prefix of `buf` whose layout has exactly M blocks."""
    from paper_1810_11765_gb300 import dsoa as D
    lo, hi = 256, buf.numel()
    assert _blocks(buf, hi) >= M
    # smallest size in 256-byte steps with at least M blocks; a block is larger
    # than 256 bytes, so one step adds at most one block and the size has M
    while hi - lo > 256:
        mid = (lo + hi) // 2 // 256 * 256
        if _blocks(buf, mid) >= M:
            hi = mid
        else:
            lo = mid
    assert _blocks(buf, hi) == M
    return D.Heap(buffer=buf[:hi])


def fill(m, cap, tag):
    """Request the missing objects until every slot is used (some requests of a
    round may fail once the free-block bitmap is empty; they are reported)."""
    filled, rnd = m.heap.count(m.type), 0
    while filled < cap and rnd < 64:
        m.new(tag * 64 + rnd, cap - filled)
        m.heap.get_error()
        filled = m.heap.count(m.type)
        rnd += 1
    return filled


def assert_clean(m):
    dev = m.heap.check()
    assert all(v == 0 for v in dev.values()), dev
    host = host_check(m.heap, 1)
    assert all(v == 0 for v in host["violations"].values()), host
    return host


@pytest.mark.parametrize("M", [1, 63, 64, 65, 4095, 4096, 4097, 64 ** 3 + 1])
def test_fill_free_refill_at_level_boundaries(buf, M):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    heap = heap_with(buf, M)
    cap = 64 * M
    m = Micro(0, SEED, cap, heap=heap)
    assert heap.info()["num_blocks"] == M
    assert heap.info()["num_levels"] == len(levels_of(M))
    for tag in (0, 1):
        assert fill(m, cap, tag) == cap
        host = assert_clean(m)
        assert host["blocks_in_use"] == M and host["live"][m.type] == cap
        m.new(99, 5)                          # a full heap: the request fails, reported
        assert heap.get_error() & D.DEV_OOM
        assert heap.count(m.type) == cap
        heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
        assert heap.count(m.type) == 0
        host = assert_clean(m)
        assert host["blocks_in_use"] == 0
        assert heap.get_error() == 0
    heap.close()
