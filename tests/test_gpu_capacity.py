"""Per-type block capacity N_T (Sec. 3.2 "Block Capacity") on the GPU.

In this mode a block holds 64 objects of the smallest type and a type T gets
N_T = floor(64 size(T_s) / size(T)) slots (lowered until its columns fit); the
slots above N_T stay marked free in the slot word and are never reserved.  The
workloads must give the oracle's results bit for bit whatever the capacities,
and the allocator invariants (including "slots beyond N_T are free") must hold.
A tiny first type shrinks every other type's capacity to a few slots, which
drives the FULL / FIRST / EMPTY block transitions far more often.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready, host_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def per_type_heap(nbytes, tiny=False):
    from paper_1810_11765_gb300 import dsoa as D
    heap = D.Heap(nbytes)
    extra = 0
    if tiny:
        heap.register_type([1])          # smallest type: 64 x 1 byte -> 128-byte blocks
        extra = 1
    heap.set_capacity_mode(D.CAPACITY_PER_TYPE)
    return heap, extra


def assert_clean(heap, ntypes):
    assert heap.get_error() == 0
    dev = heap.check()
    assert all(v == 0 for v in dev.values()), dev
    host = host_check(heap, ntypes)
    assert all(v == 0 for v in host["violations"].values()), host


def test_capacities_follow_the_block_capacity_rule():
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import GolWorld, WatorWorld
    heap, _ = per_type_heap(16 << 20)
    g = GolWorld(heap)                   # Cell 13 B, Alive 8 B
    heap.freeze()
    assert heap.capacity(g.alive_type) == 64
    assert heap.capacity(g.cell_type) == 36          # floor(64*8/13) = 39, lowered to fit 512 B
    assert heap.info()["block_bytes"] == 512
    heap.close()
    heap, _ = per_type_heap(16 << 20)
    w = WatorWorld(heap)                 # Fish 16 B, Shark 24 B
    heap.freeze()
    assert heap.capacity(w.fish_type) == 64
    assert heap.capacity(w.shark_type) == 40         # floor(64*16/24) = 42, lowered to fit 1024 B
    assert heap.info()["block_bytes"] == 1024
    with pytest.raises(D.DsoaError):
        heap.set_capacity_mode(D.CAPACITY_UNIFORM)   # after the freeze
    heap.close()
    heap = D.Heap(16 << 20)
    w = WatorWorld(heap)
    heap.freeze()
    assert heap.capacity(w.shark_type) == 64 and heap.info()["block_bytes"] == 1536   # uniform default
    heap.close()
    heap, _ = per_type_heap(16 << 20, tiny=True)
    heap.register_type([16, 16, 16, 16, 16])         # 80 x the smallest type: no slot fits
    with pytest.raises(D.DsoaError):
        heap.freeze()
    heap.close()


@pytest.mark.parametrize("tiny", [False, True])
@pytest.mark.parametrize("W,H,steps,seed", [(64, 48, 60, 3), (200, 100, 80, 4)])
def test_wator_parity(W, H, steps, seed, tiny):
    from paper_1810_11765_gb300.apps import WatorWorld
    heap, extra = per_type_heap(64 << 20, tiny)
    types = None
    if tiny:
        types = (heap.register_type(WatorWorld.FISH_FIELDS), heap.register_type(WatorWorld.SHARK_FIELDS))
    w = WatorWorld(heap, types=types)
    heap.freeze()
    if tiny:
        assert (heap.capacity(w.fish_type), heap.capacity(w.shark_type)) == (4, 2)
    s = w.add(W, H, seed)
    _, st = oracle.wator_run(W, H, steps, seed=seed)
    for k in range(steps):
        w.step()
        assert w.counts() == (st[k]["fish"], st[k]["sharks"]), k
    ref, _ = oracle.wator_run(W, H, steps, seed=seed)
    assert np.array_equal(w.read(s), ref)
    assert_clean(heap, 2 + extra)
    heap.close()


@pytest.mark.parametrize("tiny", [False, True])
def test_gol_parity(tiny):
    from paper_1810_11765_gb300.apps import GolWorld
    W, H, gens, seed = 64, 48, 40, 11
    heap, extra = per_type_heap(64 << 20, tiny)
    types = None
    if tiny:
        types = (heap.register_type(GolWorld.CELL_FIELDS), heap.register_type(GolWorld.ALIVE_FIELDS))
    g = GolWorld(heap, types=types)
    heap.freeze()
    if tiny:
        assert (heap.capacity(g.cell_type), heap.capacity(g.alive_type)) == (4, 8)
    s = g.add(W, H, seed)
    for _ in range(gens):
        g.step()
    ref, alive, _ = oracle.gol_run(W, H, gens, seed=seed)
    assert np.array_equal(g.read(s), ref)
    assert g.alive_objects() == alive[-1]
    assert_clean(heap, 2 + extra)
    heap.close()


def test_microbench_with_four_slot_blocks():
    """The microbench type gets 4 slots per block behind a 1-byte type; the column
    kernels fall back to the per-object method, results stay bit-exact."""
    from paper_1810_11765_gb300.apps import Micro
    seed, n, rounds = 0x5EED0001, 3000, 4
    heap, _ = per_type_heap(32 << 20, tiny=True)
    m = Micro(0, seed, n, heap=heap)
    assert heap.capacity(m.type) == 4
    ref, x_ref, live_ref = oracle.micro_run(seed, n, rounds, per_object=True)
    for r in range(rounds):
        m.round(r)
        s = m.stats()
        assert (s["live"], s["xor_tag"]) == (ref[r]["live"], ref[r]["xor_tag"])
        assert heap.count(m.type) == ref[r]["live"]
        assert_clean(heap, 2)
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))
    heap.close()
