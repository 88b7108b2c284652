"""The enumeration entry point that allocates nothing (dsoa_enumerate_noalloc).

It is meant for callers that cannot allocate device memory while they run (a host
program whose allocator owns the GPU under a fixed budget, a latency-critical loop
where cudaMalloc / cudaFree would synchronise the device).  Its scan keeps its
working memory in a fixed array inside the library; outputs go to caller buffers.
These tests call it through the C ABI and compare it with dsoa_enumerate, whose
results are integers and must match exactly, on two calls in a row.  This file is
collected last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu

SEED = 0x5EED0001


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def reference_enumeration(heap, t):
    """Block list and occupancy snapshot from dsoa_enumerate (library-owned)."""
    import torch
    R, occ, r = heap.enumerate(t)
    n = int(torch.as_tensor(_DeviceArray(r, 1, "<i4"), device="cuda").cpu().item())
    R_t = torch.as_tensor(_DeviceArray(R, max(n, 1), "<i4"), device="cuda")[:n]
    occ_t = torch.as_tensor(_DeviceArray(occ, max(n, 1), "<i8"), device="cuda")[:n]
    return R_t.cpu().numpy().view(np.uint32), occ_t.cpu().numpy().view(np.uint64)


def no_alloc_enumeration(heap, t, capacity=None):
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    M = heap.info()["num_blocks"]
    cap = M if capacity is None else capacity
    R = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    occ = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = D.load().dsoa_enumerate_noalloc(heap.handle, t, R.data_ptr(), occ.data_ptr(), r.data_ptr(), cap)
    if rc != 0:
        return rc
    n = int(r.cpu().item())
    return R[:n].cpu().numpy().view(np.uint32), occ[:n].cpu().numpy().view(np.uint64)


def test_matches_dsoa_enumerate_on_two_calls_in_a_row():
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(64 << 20, SEED, 1 << 18)
    m.round(0)                                     # sparse blocks after the parity delete
    ref_R, ref_occ = reference_enumeration(m.heap, m.type)
    got = no_alloc_enumeration(m.heap, m.type)
    assert not isinstance(got, int), got
    assert np.array_equal(got[0], ref_R) and np.array_equal(got[1], ref_occ)
    assert ref_R.size > 4096                       # spans several 4096-block tiles
    m.round(1)                                     # change the heap, call again
    ref_R2, ref_occ2 = reference_enumeration(m.heap, m.type)
    got2 = no_alloc_enumeration(m.heap, m.type)
    assert not isinstance(got2, int), got2
    assert np.array_equal(got2[0], ref_R2) and np.array_equal(got2[1], ref_occ2)
    assert not np.array_equal(ref_occ, ref_occ2[:ref_occ.size]) or ref_R.size != ref_R2.size
    # the snapshot counts every live object once
    live = int(np.unpackbits(got2[1].view(np.uint8)).sum())
    assert live == m.heap.count(m.type)
    m.heap.close()


def test_empty_type_and_small_heap():
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(1 << 20, SEED, 100)                  # about 1000 blocks: one scan tile
    got = no_alloc_enumeration(m.heap, m.type)
    assert got[0].size == 0
    m.new(0)
    got = no_alloc_enumeration(m.heap, m.type)
    ref = reference_enumeration(m.heap, m.type)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    m.heap.close()


def test_rejects_what_it_cannot_hold():
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(8 << 20, SEED, 100)
    M = m.heap.info()["num_blocks"]
    assert no_alloc_enumeration(m.heap, m.type, capacity=M - 1) == -1     # output too small
    m.heap.close()
    # a heap of more than DSOA_NOALLOC_MAX_TILES * 4096 blocks (128-byte blocks)
    big = D.Heap(((4096 * 4096) + 8192) * 168)
    t = big.register_type([1])
    big.freeze()
    assert big.info()["num_blocks"] > 4096 * 4096
    assert no_alloc_enumeration(big, t) == -9
    big.close()


def test_allocates_nothing_and_can_be_captured_in_global_mode():
    """The property the entry point exists for, shown two ways after one warm-up
    call: device free memory and torch's reserved memory are unchanged across
    calls, and a call captured in global capture mode (where a cudaMalloc or
    cudaFree from any thread would invalidate the capture) replays to the same
    result as dsoa_enumerate."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    s = torch.cuda.Stream()
    m = Micro(64 << 20, SEED, 1 << 18, stream=s)
    m.round(0)
    M = m.heap.info()["num_blocks"]
    R = torch.full((M,), -1, dtype=torch.int32, device="cuda")
    occ = torch.zeros(M, dtype=torch.int64, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = D.load()

    def call():
        return L.dsoa_enumerate_noalloc(m.heap.handle, m.type, R.data_ptr(), occ.data_ptr(), r.data_ptr(), M)

    torch.cuda.synchronize()
    assert call() == 0                               # warm-up: the array's address
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(3):
        assert call() == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0

    R.fill_(-1)
    occ.zero_()
    r.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
        rc = call()
    assert rc == 0
    assert int(r.cpu().item()) == 0                  # captured, not run
    g.replay()
    torch.cuda.synchronize()
    Rr, occr, rr = m.heap.enumerate(m.type)
    torch.cuda.synchronize()
    n = int(torch.as_tensor(_DeviceArray(rr, 1, "<i4"), device="cuda").cpu().item())
    ref_R = torch.as_tensor(_DeviceArray(Rr, n, "<i4"), device="cuda").cpu().numpy().view(np.uint32)
    ref_occ = torch.as_tensor(_DeviceArray(occr, n, "<i8"), device="cuda").cpu().numpy().view(np.uint64)
    assert n > 4096 and int(r.cpu().item()) == n
    assert np.array_equal(R[:n].cpu().numpy().view(np.uint32), ref_R)
    assert np.array_equal(occ[:n].cpu().numpy().view(np.uint64), ref_occ)
    del g
    m.heap.close()
