"""Checkpoint / resume of a heap (dsoa_heap_save / dsoa_heap_load).

A Wa-Tor world is saved after 30 steps (heap image + its grids and step counter),
restored into a fresh heap at another address, and continued: the restored world
must match the uninterrupted one and the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready, host_check

pytestmark = pytest.mark.gpu

W, H, SEED = 128, 96, 5


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def world(nbytes=32 << 20):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import WatorWorld
    heap = D.Heap(nbytes)
    w = WatorWorld(heap)
    heap.freeze()
    return heap, w


def test_save_resume_matches_uninterrupted_run_and_oracle():
    heap_a, wa = world()
    sa = wa.add(W, H, SEED)
    for _ in range(30):
        wa.step()
    image = heap_a.save()
    saved = [b.clone() for b in wa.bufs[sa][:3]]          # cell map, occupancy, claims
    t = wa.table.read_t(sa)
    assert t == 30
    for _ in range(20):
        wa.step()
    grid_a = wa.read(sa)
    counts_a = wa.counts()

    heap_b, wb = world()
    sb = wb.add(W, H, SEED + 1)                           # buffers of the right size
    heap_b.load_image(image)                              # replaces every object
    for dst, src in zip(wb.bufs[sb][:3], saved):
        dst.copy_(src)
    wb.table.host[sb].t = t                               # the instance's step index and
    wb.table.host[sb].seed = SEED                         # key are state of the world too
    wb.table.put(sb)
    st30 = oracle.wator_run(W, H, 30, seed=SEED)[1][-1]
    assert wb.counts() == (st30["fish"], st30["sharks"])
    for _ in range(20):
        wb.step()
    ref, st = oracle.wator_run(W, H, 50, seed=SEED)
    assert np.array_equal(wb.read(sb), grid_a)
    assert np.array_equal(grid_a, ref)
    assert wb.counts() == counts_a == (st[-1]["fish"], st[-1]["sharks"])
    assert heap_b.get_error() == 0
    host = host_check(heap_b, 2)
    assert all(v == 0 for v in host["violations"].values()), host
    heap_a.close()
    heap_b.close()


def test_load_rejects_other_layouts():
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import GolWorld
    heap_a, wa = world()
    wa.add(32, 32, 1)
    image = heap_a.save()
    heap_small, _ = world(16 << 20)                        # other byte size
    with pytest.raises(D.DsoaError):
        heap_small.load_image(image)
    heap_gol = D.Heap(32 << 20)                            # other types
    GolWorld(heap_gol)
    heap_gol.freeze()
    with pytest.raises(D.DsoaError):
        heap_gol.load_image(image)
    heap_pt = D.Heap(32 << 20)                             # other capacity mode
    from paper_1810_11765_gb300.apps import WatorWorld
    WatorWorld(heap_pt)
    heap_pt.set_capacity_mode(D.CAPACITY_PER_TYPE)
    heap_pt.freeze()
    with pytest.raises(D.DsoaError):
        heap_pt.load_image(image)
    with pytest.raises(D.DsoaError):
        heap_a.load_image(image[:-1])                      # truncated
    for h in (heap_a, heap_small, heap_gol, heap_pt):
        h.close()
