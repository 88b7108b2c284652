"""GPU parity of Wa-Tor (Fish / Shark agents, claims by lowest source index).

Bar: bit-exact grids and populations per step against the oracle.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready, host_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def world(heap_bytes=64 << 20, capacity=1):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import WatorWorld
    heap = D.Heap(heap_bytes)
    w = WatorWorld(heap, capacity)
    heap.freeze()
    return heap, w


def test_hand_cases():
    heap, w = world(4 << 20, capacity=3)
    a = w.add(3, 1, 5, init=np.array([[2, 1, 0]], np.uint8))
    b = w.add(3, 1, 5, init=np.array([[1, 0, 1]], np.uint8))
    w.step()
    assert w.read(a).tolist() == [[0, 0, 2]]
    assert w.read(b).tolist() == [[0, 1, 1]]
    assert heap.get_error() == 0


@pytest.mark.parametrize("W,H,steps,seed", [(4, 4, 30, 1), (5, 5, 40, 2), (64, 48, 60, 3), (200, 100, 80, 4)])
def test_random_grids_per_step(W, H, steps, seed):
    heap, w = world(32 << 20)
    s = w.add(W, H, seed)
    g0, _ = oracle.wator_run(W, H, 0, seed=seed)
    assert np.array_equal(w.read(s), g0)
    _, st = oracle.wator_run(W, H, steps, seed=seed)
    for k in range(steps):
        w.step()
        assert w.counts() == (st[k]["fish"], st[k]["sharks"]), k
    ref, _ = oracle.wator_run(W, H, steps, seed=seed)
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    host = host_check(heap, 2)
    assert all(v == 0 for v in host["violations"].values()), host


_FULL_REF = {}


def full_reference():
    """The oracle's run of the configured workload (computed once per session)."""
    from paper_1810_11765_gb300 import inputs
    cfg = inputs.WatorConfig()
    if "ref" not in _FULL_REF:
        _FULL_REF["ref"] = oracle.wator_run(cfg.width, cfg.height, cfg.steps, seed=cfg.seed)
    return cfg, _FULL_REF["ref"]


def test_full_config_1024_500():
    """1024 x 1024 torus, 30 % fish / 5 % sharks, 500 steps (the configured workload)."""
    cfg, (ref, st) = full_reference()
    heap, w = world(256 << 20)
    s = w.add(cfg.width, cfg.height, cfg.seed)
    for k in range(cfg.steps):
        w.step()
        if k % 50 == 49 or k < 5:
            assert w.counts() == (st[k]["fish"], st[k]["sharks"]), k
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    assert all(v == 0 for v in heap.check().values())


@pytest.mark.parametrize("flags", [1024, 256 | 4, 2])
def test_full_config_under_allocation_policies(flags):
    """The configured workload (1024 x 1024, 500 steps) with blocks left to drain
    (1024), with Alg. 1's reading of r and no hint (256 | 4), and without bitmap
    rotation (2): placement changes, the result is the oracle's."""
    cfg, (ref, st) = full_reference()
    heap, w = world(512 << 20)
    heap.set_flags(flags)
    s = w.add(cfg.width, cfg.height, cfg.seed)
    for k in range(cfg.steps):
        w.step()
        if k % 100 == 99:
            assert w.counts() == (st[k]["fish"], st[k]["sharks"]), k
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    assert all(v == 0 for v in heap.check().values())
    host = host_check(heap, 2)
    assert all(v == 0 for v in host["violations"].values()), host


def test_batched_instances_match_alone():
    heap, w = world(64 << 20, capacity=3)
    specs = [(50, 40, 31), (128, 64, 32), (17, 90, 33)]
    slots = [w.add(a, b, sd) for a, b, sd in specs]
    for _ in range(40):
        w.step()
    for slot, (a, b, sd) in zip(slots, specs):
        ref, _ = oracle.wator_run(a, b, 40, seed=sd)
        assert np.array_equal(w.read(slot), ref)
    assert heap.get_error() == 0


@pytest.mark.parametrize("launch,flags", [(dict(), 0), (dict(tpb=128, ctas_per_sm=4, slots_per_thread=2, scan_tiles=2), 0),
                                          (dict(), 8), (dict(tpb=512, ctas_per_sm=1), 12),
                                          (dict(waves=1), 0), (dict(tpb=128, slots_per_thread=2, waves=16), 0),
                                          (dict(), 16), (dict(tpb=128, scan_tiles=2, waves=8), 16),
                                          (dict(tpb=512, ctas_per_sm=1, waves=1), 20),
                                          (dict(), 128), (dict(tpb=128, waves=8), 256 | 16), (dict(waves=1), 384 | 4),
                                          (dict(), 1024), (dict(scan_tiles=5, waves=8), 1024 | 16)])
def test_graph_captured_steps_match_oracle(launch, flags):
    """One step captured as a CUDA graph and replayed: the step index lives in
    device memory, so replays advance the simulation exactly like plain steps."""
    import torch
    W, H, steps, seed = 128, 96, 60, 41
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
        for _ in range(steps):
            g.launch()
        s.synchronize()
        grid = w.read(slot)
        counts = w.counts()
    ref, st = oracle.wator_run(W, H, steps, seed=seed)
    assert np.array_equal(grid, ref)
    assert counts == (st[-1]["fish"], st[-1]["sharks"])
    assert heap.get_error() == 0
    g.close()


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_ablations_finish_with_the_oracle_result(flags):
    """NoCoal, NoShift and both (Sec. 6.4, Fig. 10c) on a 256 x 256 world: slower
    placement, same simulation, no device error."""
    W, H, steps, seed = 256, 256, 40, 0x5EED0003
    heap, w = world(64 << 20)
    heap.set_flags(flags)
    slot = w.add(W, H, seed)
    _, st = oracle.wator_run(W, H, steps, seed=seed)
    for k in range(steps):
        w.step()
        if k % 10 == 9:
            assert w.counts() == (st[k]["fish"], st[k]["sharks"]), k
    ref, _ = oracle.wator_run(W, H, steps, seed=seed)
    assert np.array_equal(w.read(slot), ref)
    assert heap.get_error() == 0
    host = host_check(heap, 2)
    assert all(v == 0 for v in host["violations"].values()), host
    heap.close()


@pytest.mark.parametrize("scan", [1, 2, 3, 4, 5])
def test_enumeration_modes_agree(scan):
    """Tile-count + compaction kernels (1 or 2 tiles per CTA), the single-pass
    look-back kernel and the streamed enumeration inside the choose methods give
    the same snapshots, hence the same simulation."""
    heap, w = world(32 << 20)
    heap.set_launch(scan_tiles=scan)
    s = w.add(160, 120, 55)
    for _ in range(40):
        w.step()
    ref, _ = oracle.wator_run(160, 120, 40, seed=55)
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0


class _Dev:
    """A device buffer given by pointer, for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


def _enumeration(heap, t, ptrs):
    import torch
    R, occ, r = ptrs
    torch.cuda.synchronize()
    n = int(torch.as_tensor(_Dev(r, 1, "<i4"), device="cuda").cpu()[0])
    lst = torch.as_tensor(_Dev(R, max(n, 1), "<i4"), device="cuda")[:n].cpu().numpy().copy()
    snap = torch.as_tensor(_Dev(occ, max(n, 1), "<i8"), device="cuda")[:n].cpu().numpy().copy()
    return lst, snap


@pytest.mark.parametrize("scan_tiles", [1, 3, 5])
def test_enumerate_many_equals_separate_enumerations(scan_tiles):
    """One launch enumerating Fish and Shark gives, per type, the block list and
    occupancy snapshot of a separate dsoa_enumerate (same per-type buffers)."""
    heap, w = world(64 << 20)
    heap.set_launch(scan_tiles=scan_tiles)
    w.add(200, 100, 9)
    for _ in range(15):
        w.step()
    types = (w.fish_type, w.shark_type)
    ptrs = {t: heap.enumerate(t) for t in types}
    sep = {t: _enumeration(heap, t, ptrs[t]) for t in types}
    assert all(len(sep[t][0]) > 0 for t in types)
    for order in ([w.fish_type, w.shark_type], [w.shark_type, w.fish_type]):
        for _ in range(3):            # repeated launches: epochs advance per type
            heap.enumerate_many(order)
            for t in types:
                lst, snap = _enumeration(heap, t, ptrs[t])
                assert np.array_equal(lst, sep[t][0]) and np.array_equal(snap, sep[t][1])
    heap.enumerate(w.fish_type)        # a single-type launch after batched ones
    lst, snap = _enumeration(heap, w.fish_type, ptrs[w.fish_type])
    assert np.array_equal(lst, sep[w.fish_type][0])
    assert heap.get_error() == 0
    heap.close()


@pytest.mark.parametrize("defer", [False, True])
def test_births_in_place_or_deferred_match_oracle(defer):
    """Newborn fish allocated inside Fish.move or by the births kernel after it:
    both give the oracle's populations per step and final grid."""
    W, H, steps, seed = 96, 64, 60, 12
    heap, w = world(32 << 20)
    w.defer_births = defer
    s = w.add(W, H, seed)
    _, st = oracle.wator_run(W, H, steps, seed=seed)
    for k in range(steps):
        w.step()
        assert w.counts() == (st[k]["fish"], st[k]["sharks"]), k
    ref, _ = oracle.wator_run(W, H, steps, seed=seed)
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    host = host_check(heap, 2)
    assert all(v == 0 for v in host["violations"].values()), host
    heap.close()


def test_count_many_matches_count_and_is_capturable():
    """Populations of both types in one launch, inside a captured step graph."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        heap, w = world(64 << 20)
        w.add(128, 96, 21)
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        heap.graph_begin()
        w.step()
        heap.count_many_async([w.fish_type, w.shark_type], out)
        g = heap.graph_end()
        _, st = oracle.wator_run(128, 96, 12, seed=21)
        for k in range(12):
            g.launch()
            got = out.cpu().tolist()
            assert got == [st[k]["fish"], st[k]["sharks"]], k
            assert got == [heap.count(w.fish_type), heap.count(w.shark_type)]
        heap.count_many_async([w.shark_type], out[1:])
        assert int(out[1].item()) == heap.count(w.shark_type)
        g.close()
        heap.close()


def test_full_config_in_the_benchmarked_launch_configuration():
    """The configured workload (1024 x 1024, 500 steps) exactly as the benchmark
    runs it: 512 MiB heap, the autotuned launch shape, each step one captured CUDA
    graph replayed; final grid and populations equal the oracle's."""
    import torch
    from paper_1810_11765_gb300 import autotune, dsoa as D
    from paper_1810_11765_gb300.apps import WatorWorld
    cfg, (ref, st) = full_reference()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        launch = autotune.best_wator_launch(cfg.seed)
        heap = D.Heap(512 << 20)
        w = WatorWorld(heap)
        heap.freeze()
        autotune.apply(heap, launch)
        slot = w.add(cfg.width, cfg.height, cfg.seed)
        heap.graph_begin()
        w.step()
        g = heap.graph_end()
        for _ in range(cfg.steps):
            g.launch()
        assert np.array_equal(w.read(slot), ref)
        assert w.counts() == (st[-1]["fish"], st[-1]["sharks"])
        assert heap.get_error() == 0
        assert all(v == 0 for v in heap.check().values())
        g.close()
        heap.close()


def test_counts_stored_into_mapped_pinned_host_memory():
    """dsoa_count_many_async stores its totals (no pre-zeroing, no copy) into any
    device-writable address: a captured step writes each step's populations
    straight into pinned host memory, repeatedly, and they equal the oracle's."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        heap, w = world(64 << 20)
        w.add(128, 96, 23)
        host = torch.full((2,), -1, dtype=torch.int64).pin_memory()
        heap.graph_begin()
        w.step()
        heap.count_many_async([w.fish_type, w.shark_type], host)
        g = heap.graph_end()
        _, st = oracle.wator_run(128, 96, 15, seed=23)
        for k in range(15):
            g.launch()
            s.synchronize()
            assert host.tolist() == [st[k]["fish"], st[k]["sharks"]], k
        dev = torch.full((3,), 7, dtype=torch.int64, device="cuda")
        heap.count_many_async([w.shark_type, w.fish_type], dev[1:])   # stored, not added
        assert dev.tolist() == [7, st[14]["sharks"], st[14]["fish"]]
        assert heap.get_error() == 0
        g.close()
        heap.close()


def test_separate_advance_launch_equals_folded():
    """The step counter advanced by its own kernel after Shark.move (K_WATOR_ADVANCE)
    or by CTA 0 of Shark.move itself (SHARK_MOVE_ADVANCE, the default): the same
    simulation."""
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import WatorWorld

    class Separate(WatorWorld):
        def step(self):
            a = self.args()
            self.heap.parallel_do(self.fish_type, D.M_WATOR_FISH_CHOOSE, a)
            self.heap.parallel_do_enumerated(self.fish_type, D.M_WATOR_FISH_MOVE, a)
            self.heap.parallel_do(self.shark_type, D.M_WATOR_SHARK_CHOOSE, a)
            self.heap.parallel_do_enumerated(self.shark_type, D.M_WATOR_SHARK_MOVE, a)
            self.heap.run_kernel(D.K_WATOR_ADVANCE, self.table.capacity, a)

    W, H, steps, seed = 96, 64, 30, 17
    heap = D.Heap(32 << 20)
    w = Separate(heap)
    heap.freeze()
    s = w.add(W, H, seed)
    for _ in range(steps):
        w.step()
    ref, _ = oracle.wator_run(W, H, steps, seed=seed)
    assert np.array_equal(w.read(s), ref)
    assert heap.get_error() == 0
    heap.close()
