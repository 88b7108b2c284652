"""GPU parity of BitmapAlloc (the paper's flat bitmap allocator, Sec. 6) on the
allocator + do-all microbench: the same semantics as on the DynaSOAr heap, so the
same oracle and the same bar (live counts, integer sums and per-object x bit-exact,
fp64 sum of x within 1e-6 relative), plus its bitmap invariants at quiescence.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu

SEED = 0x5EED0001


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def make(heap_bytes=64 << 20, n=1 << 18):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    return Micro(heap_bytes, SEED, n, heap=D.BitmapHeap(heap_bytes))


def compare_round(g, o):
    assert g["live"] == o["live"]
    assert g["sum_id"] == o["sum_id"] % 2**64
    assert g["sum_tag"] == o["sum_tag"]
    assert g["xor_tag"] == o["xor_tag"]
    assert abs(g["sum_x"] - o["sum_x"]) <= 1e-6 * max(abs(o["sum_x"]), 1.0)


def assert_clean(m):
    assert m.heap.get_error() == 0
    chk = m.heap.check()
    assert all(v == 0 for v in chk.values()), chk


def test_layout_is_one_record_array():
    m = make(8 << 20, 64)
    info = m.heap.info()
    assert info["record_bytes"] == 16                     # {i32 id, f32 x, i64 tag}, AOS
    assert info["num_slots"] * 16 <= 8 << 20
    assert info["num_slots"] * 16 > 0.95 * (8 << 20)      # bitmaps take ~3 bits per slot
    m.heap.close()


@pytest.mark.parametrize("n,rounds", [(1, 3), (63, 4), (1000, 5), (1 << 18, 10)])
def test_microbench_parity(n, rounds):
    """The configured microbench (2^18 new per round, 10 rounds, 64 MiB heap) and
    ragged small cases, bit-exact per object."""
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    m = make(64 << 20, n)
    for r in range(rounds):
        m.round(r)
        compare_round(m.stats(), ref[r])
        assert m.heap.count(m.type) == ref[r]["live"]
        assert_clean(m)
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))
    m.heap.close()


def test_fill_until_oom_then_free_all():
    """Every slot can be allocated once (no slot handed out twice, no slot lost);
    the allocation beyond capacity reports OOM; delete-all returns every slot."""
    from paper_1810_11765_gb300 import dsoa as D
    m = make(4 << 20, 1 << 16)
    cap = m.heap.info()["num_slots"]
    m.new(0, cap)
    assert m.heap.count(m.type) == cap
    assert m.heap.get_error() == 0
    _, live = m.gather(cap)
    assert live.sum() == cap
    m.new(1, 100)                                          # heap full
    assert m.heap.get_error() & D.DEV_OOM
    assert m.heap.count(m.type) == cap
    m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
    assert m.heap.count(m.type) == 0
    assert_clean(m)
    m.new(2, cap)                                          # the freed slots are reusable
    assert m.heap.count(m.type) == cap
    assert_clean(m)
    m.heap.close()


def test_rejects_unknown_and_mismatched():
    from paper_1810_11765_gb300 import dsoa as D
    h = D.BitmapHeap(4 << 20)
    t = h.register_type([4, 4, 4])
    with pytest.raises(D.DsoaError):
        h.parallel_new(t, 10, D.C_MICRO, D.MicroArgs())   # not the microbench field layout
    h2 = D.BitmapHeap(4 << 20)
    t2 = h2.register_type([4, 4, 8])
    with pytest.raises(D.DsoaError):
        h2.parallel_do(t2, D.M_WATOR_FISH_MOVE, D.MicroArgs())
    h.close()
    h2.close()
