"""GPU parity of Game of Life (Cell per site + Alive agents) against the oracle.

Bar: bit-exact grids and alive counts per generation; Alive objects == live cells.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready, host_check
from test_oracle_gol import PATTERNS, place

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def world(heap_bytes=64 << 20, capacity=1):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import GolWorld
    heap = D.Heap(heap_bytes)
    w = GolWorld(heap, capacity)
    heap.freeze()
    return heap, w


@pytest.mark.parametrize("name", ["blinker", "glider", "toad", "beehive"])
def test_patterns(name):
    pat, period, dx, dy = PATTERNS[name]
    g0 = place(pat, 20, 16, 3, 4)
    heap, w = world(8 << 20)
    s = w.add(20, 16, 1, init=g0)
    for gen in range(1, 2 * period + 1):
        w.step()
        ref, alive, _ = oracle.gol_run(20, 16, gen, init=g0)
        assert np.array_equal(w.read(s), ref)
        assert w.alive_objects() == alive[-1]
    assert heap.get_error() == 0


@pytest.mark.parametrize("W,H,gens,seed", [(64, 64, 40, 11), (100, 37, 30, 12), (257, 129, 25, 13)])
def test_random_grids(W, H, gens, seed):
    heap, w = world(32 << 20)
    s = w.add(W, H, seed)
    _, alive_ref, _ = oracle.gol_run(W, H, gens, seed=seed)
    assert w.alive_objects() == alive_ref[0]
    for g in range(1, gens + 1):
        w.step()
        assert w.alive_objects() == alive_ref[g], g
    ref, _, _ = oracle.gol_run(W, H, gens, seed=seed)
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    host = host_check(heap, 2)
    assert all(v == 0 for v in host["violations"].values()), host
    assert all(v == 0 for v in heap.check().values())


def test_full_config_512_200():
    """512 x 512 torus, density 1/4, 200 generations (the configured workload)."""
    from paper_1810_11765_gb300 import inputs
    cfg = inputs.GolConfig()
    ref, alive_ref, objs_ref = oracle.gol_run(cfg.width, cfg.height, cfg.gens, seed=cfg.seed)
    heap, w = world(64 << 20)
    s = w.add(cfg.width, cfg.height, cfg.seed)
    counts = [w.alive_objects()]
    for g in range(cfg.gens):
        w.step()
        counts.append(w.alive_objects())
    assert np.array_equal(np.array(counts), alive_ref)
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    assert all(v == 0 for v in heap.check().values())


def test_batched_instances_match_alone():
    """Three instances of different sizes step together in one heap; each matches
    an oracle run of that instance alone."""
    heap, w = world(64 << 20, capacity=4)
    specs = [(64, 48, 21), (130, 70, 22), (33, 200, 23)]
    slots = [w.add(a, b, sd) for a, b, sd in specs]
    for _ in range(30):
        w.step()
    for slot, (a, b, sd) in zip(slots, specs):
        ref, _, _ = oracle.gol_run(a, b, 30, seed=sd)
        assert np.array_equal(w.read(slot), ref)
    # removing one instance deletes its objects only
    w.remove(slots[1])
    alive = sum(int(oracle.gol_run(a, b, 30, seed=sd)[0].sum()) for a, b, sd in (specs[0], specs[2]))
    assert w.alive_objects() == alive
    assert heap.count(w.cell_type) == specs[0][0] * specs[0][1] + specs[2][0] * specs[2][1]
    assert heap.get_error() == 0
    assert all(v == 0 for v in heap.check().values())


@pytest.mark.parametrize("launch,flags", [(dict(), 16), (dict(scan_tiles=1, waves=8), 16), (dict(scan_tiles=4), 16),
                                          (dict(scan_tiles=5), 0), (dict(scan_tiles=5, waves=8), 16),
                                          (dict(), 256), (dict(tpb=512, waves=2), 128 | 16), (dict(), 1024)])
def test_launch_modes_graph_captured(launch, flags):
    """Programmatic dependent launch, the two-kernel and the streamed enumeration:
    a graph-captured generation replayed 30 times equals the oracle."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    W, H, gens, seed = 200, 150, 30, 21
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        heap, w = world(32 << 20)
        if launch:
            heap.set_launch(**launch)
        heap.set_flags(flags)
        slot = w.add(W, H, seed)
        heap.graph_begin()
        w.step()
        g = heap.graph_end()
        for _ in range(gens):
            g.launch()
        s.synchronize()
        grid = w.read(slot)
        alive = w.alive_objects()
    ref, alive_ref, _ = oracle.gol_run(W, H, gens, seed=seed)
    assert np.array_equal(grid, ref)
    assert alive == alive_ref[-1]
    assert heap.get_error() == 0
    g.close()


def test_separate_advance_launch_equals_folded():
    """The generation counter advanced by its own kernel (K_GOL_ADVANCE) or by CTA 0
    of Cell.decide (DECIDE_ADVANCE, the default): the same generations."""
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import GolWorld

    class Separate(GolWorld):
        def step(self):
            a = self.args()
            self.heap.parallel_do(self.alive_type, D.M_GOL_SPREAD, a)
            self.heap.parallel_do_enumerated(self.alive_type, D.M_GOL_REAP, a)
            self.heap.parallel_do(self.cell_type, D.M_GOL_DECIDE, a)
            self.heap.run_kernel(D.K_GOL_ADVANCE, self.table.capacity, a)

    W, H, gens, seed = 64, 48, 25, 19
    heap = D.Heap(32 << 20)
    g = Separate(heap)
    heap.freeze()
    s = g.add(W, H, seed)
    for _ in range(gens):
        g.step()
    ref, alive, _ = oracle.gol_run(W, H, gens, seed=seed)
    assert np.array_equal(g.read(s), ref)
    assert heap.get_error() == 0
    heap.close()
