"""GPU parity of batched Nagel-Schreckenberg rings.

Bar: bit-exact occupancy and speeds.  At the configured size (64 rings, lengths
2^12..2^20, 1000 steps) whole-batch oracle runs take minutes, so rings are sampled
and replayed alone in the oracle (rings are independent; the oracle pins that).
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def world(L, thr, seed, heap_bytes=64 << 20, **kw):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import TrafficWorld
    heap = D.Heap(heap_bytes)
    w = TrafficWorld(heap, L, thr, seed, **kw)
    heap.freeze()
    w.init()
    return heap, w


def test_small_batch_per_step():
    L = [16, 23, 300, 4096, 5000]
    thr = [int(d * 2**32) for d in (0.3, 0.6, 0.2, 0.1, 0.3)]
    seed = 77
    heap, w = world(L, thr, seed, ramp_thr=int(0.3 * 2**32))
    for k in (1, 2, 5, 17, 40):
        while w.steps_done < k:
            w.step()
        o, v, cars = oracle.traffic_run(L, thr, k, seed=seed, ramp_thr=int(0.3 * 2**32))
        go, gv = w.read()
        assert np.array_equal(go, o), k
        assert np.array_equal(gv, v), k
        assert heap.count(w.car_type) == cars[-1].sum()
    assert heap.get_error() == 0


def test_deterministic_limit():
    # slow-down and ramps off: a lone car reaches vmax = 5
    L = [100]
    occ = np.zeros(100, np.uint8)
    occ[7] = 1
    heap, w = world(L, [0], 1, slow_thr=0, ramp_thr=0, init_occ=occ, init_v=np.zeros(100, np.uint8))
    for _ in range(10):
        w.step()
    o, v = w.read()
    assert np.nonzero(o)[0].tolist() == [(7 + 1 + 2 + 3 + 4 + 5 * 6) % 100]
    assert v[o.astype(bool)].tolist() == [5]


def test_full_config_sampled_rings():
    from concurrent.futures import ThreadPoolExecutor
    from paper_1810_11765_gb300 import inputs
    L, thr = inputs.traffic_instances()
    seed = inputs.SEED_TRAFFIC
    base = np.concatenate([[0], np.cumsum(L.astype(np.int64))])
    order = np.argsort(L)
    # the two shortest, the median and the two longest rings (about 2^20 cells:
    # the longest gaps and the most cars of the batch), against the oracle run
    # of each ring alone; the oracle (C through ctypes, which releases the GIL)
    # runs in threads while the GPU steps
    sample = [int(order[0]), int(order[1]), int(order[len(L) // 2]), int(order[-2]), int(order[-1])]
    checkpoints = [100, 1000]
    pool = ThreadPoolExecutor(max_workers=len(sample) * len(checkpoints))
    ref = {(k, i): pool.submit(oracle.traffic_run, [L[i]], [thr[i]], k, seed=seed, first_ring=i)
           for k in checkpoints for i in sample}
    heap, w = world(L, thr, seed, heap_bytes=512 << 20)
    for k in checkpoints:
        while w.steps_done < k:
            w.step()
        go, gv = w.read()
        for i in sample:
            o, v, _ = ref[(k, i)].result()
            assert np.array_equal(go[base[i]:base[i + 1]], o), (k, i)
            assert np.array_equal(gv[base[i]:base[i + 1]], v), (k, i)
    pool.shutdown()
    # at any size: cars occupy distinct cells, speeds within [0, 5], count matches
    assert heap.count(w.car_type) == int(go.sum())
    assert gv.max() <= 5 and np.all(gv[~go.astype(bool)] == 0)
    assert heap.get_error() == 0


@pytest.mark.parametrize("flags", [16, 256, 128 | 16, 1024])
def test_launch_flags_keep_semantics(flags):
    """The batch stepped with programmatic dependent launch (16) and / or the
    allocation-policy flags (128, 256, 1024) equals the oracle."""
    L = [16, 23, 300, 4096, 5000]
    thr = [int(d * 2**32) for d in (0.3, 0.6, 0.2, 0.1, 0.3)]
    seed = 78
    heap, w = world(L, thr, seed, ramp_thr=int(0.3 * 2**32))
    heap.set_flags(flags)
    while w.steps_done < 25:
        w.step()
    o, v, cars = oracle.traffic_run(L, thr, 25, seed=seed, ramp_thr=int(0.3 * 2**32))
    go, gv = w.read()
    assert np.array_equal(go, o)
    assert np.array_equal(gv, v)
    assert heap.get_error() == 0


def test_separate_onramp_and_advance_equal_folded():
    """ONRAMP then ADVANCE as two launches, or ONRAMP_ADVANCE (the default) as one,
    over 300 rings (several CTAs' worth for the separate on-ramp kernel): the same
    cars as the oracle."""
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import TrafficWorld

    class Separate(TrafficWorld):
        def step(self):
            self.heap.run_kernel(D.K_TRAFFIC_CLEAR, self.total, self.a)
            self.heap.parallel_do(self.car_type, D.M_TRAFFIC_MOVE, self.a)
            self.heap.run_kernel(D.K_TRAFFIC_ONRAMP, int(self.L.size), self.a)
            self.heap.run_kernel(D.K_TRAFFIC_ADVANCE, 1, self.a)
            self.steps_done += 1

    rng = np.random.default_rng(3)
    L = [int(x) for x in rng.integers(16, 400, 300)]
    thr = [int(d * 2**32) for d in rng.uniform(0.1, 0.3, 300)]
    seed, steps, ramp = 91, 25, int(0.3 * 2**32)
    o, v, cars = oracle.traffic_run(L, thr, steps, seed=seed, ramp_thr=ramp)
    for cls in (Separate, TrafficWorld):
        heap = D.Heap(64 << 20)
        w = cls(heap, L, thr, seed, ramp_thr=ramp)
        heap.freeze()
        w.init()
        for _ in range(steps):
            w.step()
        go, gv = w.read()
        assert np.array_equal(go, o) and np.array_equal(gv, v), cls.__name__
        assert heap.count(w.car_type) == cars[-1].sum()
        assert heap.get_error() == 0
        heap.close()
