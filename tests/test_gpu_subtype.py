"""Subtypes (Sec. 1 "Subclassing/Inheritance", Sec. 3.1, Sec. 3.4) on the GPU.

A subtype's blocks start with its base's SOA columns, so the base's methods run
on subtype objects unchanged; each type keeps its own blocks and bitmaps; a
do-all on the base visits the objects of the base and of every subtype that
exist at entry.  The microbench with part of every round's objects created as
subtype objects must give the oracle's results bit for bit (the workload's
semantics do not depend on the split), in both capacity modes.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready, host_check

pytestmark = pytest.mark.gpu

SEED = 0x5EED0001


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def make(n, per_type=False, sub_fields=(8, 8), share=0.5, heap_bytes=64 << 20):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    heap = D.Heap(heap_bytes)
    if per_type:
        heap.set_capacity_mode(D.CAPACITY_PER_TYPE)
    return Micro(0, SEED, n, heap=heap, sub_fields=list(sub_fields), sub_share=share)


def assert_clean(m):
    assert m.heap.get_error() == 0
    dev = m.heap.check()
    assert all(v == 0 for v in dev.values()), dev
    host = host_check(m.heap, 2)
    assert all(v == 0 for v in host["violations"].values()), host


@pytest.mark.parametrize("per_type", [False, True])
@pytest.mark.parametrize("n,rounds,share", [(1, 3, 0.5), (1000, 5, 0.5), (3000, 4, 0.9), (1 << 18, 10, 0.5)])
def test_microbench_through_the_base_type(n, rounds, share, per_type):
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    m = make(n, per_type, share=share)
    assert m.heap.type_base(m.sub_type) == m.type and m.heap.type_base(m.type) == -1
    if per_type:
        assert m.heap.capacity(m.type) == 64 and m.heap.capacity(m.sub_type) == 32
    for r in range(rounds):
        m.round(r)
        s = m.stats()
        o = ref[r]
        assert (s["live"], s["sum_id"], s["sum_tag"], s["xor_tag"]) == \
            (o["live"], o["sum_id"] % 2**64, o["sum_tag"], o["xor_tag"])
        assert abs(s["sum_x"] - o["sum_x"]) <= 1e-6 * max(abs(o["sum_x"]), 1.0)
        assert m.heap.count(m.type) + m.heap.count(m.sub_type) == o["live"]
        assert_clean(m)
    if n > 1:
        assert m.heap.count(m.sub_type) > 0 and m.heap.count(m.type) > 0
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))
    m.heap.close()


def test_subtype_objects_live_in_their_own_blocks():
    """A do-all on the subtype visits its objects only; its blocks are not in the
    base type's bitmaps (live counts per exact type add up to the family's)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    n = 5000
    m = make(n, share=0.3)
    m.new(0)
    st = torch.zeros(64, dtype=torch.uint8, device="cuda")
    m.heap.parallel_do(m.sub_type, D.M_MICRO_STATS, m.args(stats=st.data_ptr()))
    sub = D.MicroStats.from_buffer_copy(bytes(st[:40].cpu().numpy()))
    assert sub.live == m.heap.count(m.sub_type) == int(n * 0.3)
    assert m.heap.count(m.type) == n - int(n * 0.3)
    ids = np.arange(n - int(n * 0.3), n)
    assert sub.sum_id == int(ids.sum())
    fam = m.stats()
    assert fam["live"] == n
    assert m.heap.type_stats(m.sub_type)["blocks"] > 0
    assert_clean(m)
    m.heap.close()


def test_base_do_all_is_graph_capturable():
    """The family do-all (one enumeration launch, one method launch per type)
    captured once and replayed each round gives the oracle's objects."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    n, rounds = 2000, 5
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m = make(n)
        m.heap.graph_begin()
        m.scale()
        g = m.heap.graph_end()
        for r in range(rounds):
            m.new(r)
            g.launch()
            m.delete(r)
        x, live = m.gather(n * rounds)
        assert m.heap.get_error() == 0
        g.close()
        m.heap.close()
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))


def test_register_subtype_rejects_bad_requests():
    from paper_1810_11765_gb300 import dsoa as D
    heap = D.Heap(4 << 20)
    t = heap.register_type([4, 4, 8])
    with pytest.raises(D.DsoaError):
        heap.register_subtype(7, [4])                       # no such base
    with pytest.raises(D.DsoaError):
        heap.register_subtype(t, [4] * 10)                   # 13 fields
    with pytest.raises(D.DsoaError):
        heap.register_subtype(t, [3])                        # bad field size
    s = heap.register_subtype(t, [])                         # no new field
    s2 = heap.register_subtype(s, [2])                       # subtype of a subtype
    assert heap.type_base(s2) == s and heap.type_base(s) == t
    heap.freeze()
    with pytest.raises(D.DsoaError):
        heap.register_subtype(t, [4])                        # after the freeze
    heap.close()
