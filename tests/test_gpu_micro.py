"""GPU parity of the allocator + do-all microbench against the oracle.

Bar: live counts, integer sums and per-object x bit-exact; the fp64 sum of x within
1e-6 relative (the configured tolerance for the fp32 field); allocator invariants
clean at quiescence, checked by the library's device checker and by the independent
host checker of gpu_common.
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


def make(heap_bytes=64 << 20, n=1 << 18, **launch):
    from paper_1810_11765_gb300.apps import Micro
    m = Micro(heap_bytes, SEED, n)
    if launch:
        m.heap.set_launch(**launch)
    return m


def assert_clean(m):
    assert m.heap.get_error() == 0
    dev = m.heap.check()
    assert all(v == 0 for v in dev.values()), dev
    host = host_check(m.heap, 1)
    assert all(v == 0 for v in host["violations"].values()), host
    return host


def compare_round(g, o):
    assert g["live"] == o["live"]
    assert g["sum_id"] == o["sum_id"] % 2**64
    assert g["sum_tag"] == o["sum_tag"]
    assert g["xor_tag"] == o["xor_tag"]
    assert abs(g["sum_x"] - o["sum_x"]) <= 1e-6 * max(abs(o["sum_x"]), 1.0)


def test_full_config_parity():
    """2^18 new per round, 10 rounds, 64 MiB heap: the configured microbench."""
    n, rounds = 1 << 18, 10
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    m = make()
    for r in range(rounds):
        m.new(r)
        if r == 0:
            # no slot handed out twice: n distinct ids land in n distinct slots
            assert m.heap.count(m.type) == n
            _, live0 = m.gather(n)
            assert live0.sum() == n
        m.scale()
        m.delete(r)
        compare_round(m.stats(), ref[r])
        host = assert_clean(m)
        assert host["live"][0] == ref[r]["live"]
        assert m.heap.count(m.type) == ref[r]["live"]
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 4097, 70001])
def test_ragged_sizes(n):
    rounds = 3
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    m = make(heap_bytes=32 << 20, n=n)
    for r in range(rounds):
        m.round(r)
        compare_round(m.stats(), ref[r])
        assert_clean(m)
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    assert np.array_equal(x[live_ref.astype(bool)], x_ref[live_ref.astype(bool)])


@pytest.mark.parametrize("method", ["scalar", "scalar_g2", "spt1", "spt2", "spt4", "bulk"])
def test_scale_variants_agree(method):
    from paper_1810_11765_gb300 import dsoa as D
    n, rounds = 50000, 4
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    spt = {"scalar": 1, "scalar_g2": 2, "spt1": 1, "spt2": 2, "spt4": 4, "bulk": 4}[method]
    m = make(heap_bytes=16 << 20, n=n, slots_per_thread=spt)
    meth = {"scalar": D.M_MICRO_SCALE_SCALAR, "scalar_g2": D.M_MICRO_SCALE_SCALAR,
            "bulk": D.M_MICRO_SCALE_TMA}.get(method, D.M_MICRO_SCALE)
    for r in range(rounds):
        m.round(r, method=meth)
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    assert np.array_equal(x[live_ref.astype(bool)], x_ref[live_ref.astype(bool)])
    assert_clean(m)


@pytest.mark.parametrize("flags", [1, 2, 3, 4, 7, 8, 15, 16, 24, 128, 256, 256 | 4, 384 | 3, 1024, 1024 | 4, 1024 | 1])
def test_ablations_keep_semantics(flags):
    """NoCoal / NoShift / both (Sec. 6.4) change placement and speed, not results:
    every variant, NoShift included, must finish each round with the oracle's
    results and no device error.  Without coalescing every thread of a burst on
    an empty heap may take a block of its own (Alg. 1 slow path), so the heap
    must hold one block per request."""
    n, rounds = 20000, 3
    ref, _, _ = oracle.micro_run(SEED, n, rounds)
    m = make(heap_bytes=64 << 20, n=n)
    m.heap.set_flags(flags)
    for r in range(rounds):
        m.round(r)
        compare_round(m.stats(), ref[r])
        assert_clean(m)


@pytest.mark.parametrize("tpb,ctas,scan,waves", [(64, 1, 1, 1), (128, 4, 2, 2), (512, 2, 1, 4), (512, 8, 2, 16),
                                                 (256, 8, 3, 4), (64, 2, 3, 8), (128, 8, 4, 1), (512, 1, 4, 2),
                                                 (128, 8, 5, 4), (256, 4, 5, 1)])
def test_launch_shapes_keep_semantics(tpb, ctas, scan, waves):
    n, rounds = 30000, 3
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    m = make(heap_bytes=16 << 20, n=n, tpb=tpb, ctas_per_sm=ctas, scan_tiles=scan, waves=waves)
    for r in range(rounds):
        m.round(r)
        compare_round(m.stats(), ref[r])
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    assert np.array_equal(x[live_ref.astype(bool)], x_ref[live_ref.astype(bool)])


def test_empty_heap_operations():
    m = make(heap_bytes=4 << 20, n=0)
    assert m.heap.count(m.type) == 0
    m.scale()
    m.delete(0)
    s = m.stats()
    assert s["live"] == 0 and s["sum_x"] == 0.0
    assert_clean(m)


def test_out_of_memory_is_reported_not_hung():
    """A heap with room for a few blocks: allocation beyond it returns null handles
    and sets DSOA_DEV_OOM; the kernel completes and the heap stays consistent."""
    from paper_1810_11765_gb300 import dsoa as D
    m = make(heap_bytes=64 << 10, n=10000)
    M = m.heap.info()["num_blocks"]
    m.new(0)
    err = m.heap.get_error()
    assert err & D.DEV_OOM
    assert not err & (D.DEV_SPIN | D.DEV_DOUBLE_FREE | D.DEV_BAD_HANDLE)
    live = m.heap.count(m.type)
    assert 0 < live <= 64 * M
    assert live >= 0.9 * 64 * M        # nearly all slots are used before OOM (Sec. 6.5)
    host = host_check(m.heap, 1)
    assert host["live"][0] == live
    assert all(v == 0 for v in host["violations"].values()), host


def test_launch_shape_bounds():
    from paper_1810_11765_gb300 import dsoa as D
    m = make(heap_bytes=4 << 20, n=10)
    for bad in (dict(tpb=1024), dict(tpb=96), dict(ctas_per_sm=64), dict(slots_per_thread=3), dict(waves=17),
                dict(waves=-1), dict(scan_tiles=6)):
        with pytest.raises(D.DsoaError):
            m.heap.set_launch(**bad)


def test_heap_from_torch_buffer():
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    buf = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    heap = D.Heap(buffer=buf)
    m = Micro(0, SEED, 5000, heap=heap)
    ref, _, _ = oracle.micro_run(SEED, 5000, 2)
    for r in range(2):
        m.round(r)
        compare_round(m.stats(), ref[r])
    heap.close()


def test_graph_capture_replays_rounds():
    """A captured round (new / scale / delete) replays with its argument values
    baked in; replaying the round graph of round r reproduces round r."""
    import torch
    from paper_1810_11765_gb300.apps import Micro
    n, rounds = 40000, 5
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m = Micro(16 << 20, SEED, n, stream=s)
        graphs = []
        for r in range(rounds):
            m.heap.graph_begin()
            m.round(r)
            graphs.append(m.heap.graph_end())
        for r in range(rounds):
            graphs[r].launch(s)
        s.synchronize()
        compare_round(m.stats(), ref[-1])
        x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    assert np.array_equal(x[live_ref.astype(bool)], x_ref[live_ref.astype(bool)])


def test_delete_handles_matches_parity_delete():
    """Freeing a host-chosen list of handles (the odd-parity ids of round 0) in one
    kernel gives the same objects as the parity delete do-all."""
    import torch
    n = 30000
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, 1, per_object=True)
    m = make(heap_bytes=16 << 20, n=n)
    m.new(0)
    m.scale()
    hs = m.handles(n)
    kill = torch.from_numpy((live_ref == 0).astype(np.bool_)).cuda()
    m.heap.delete_handles(hs[kill].contiguous(), int(kill.sum()))
    compare_round(m.stats(), ref[0])
    x, live = m.gather(n)
    assert np.array_equal(live, live_ref)
    assert_clean(m)


def test_double_free_and_bad_handles_are_reported_not_fatal():
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    n = 5000
    m = make(heap_bytes=8 << 20, n=n)
    m.new(0)
    hs = m.handles(n)
    first = hs[1:2000:2].contiguous()                   # odd ids: no block becomes empty
    m.heap.delete_handles(first, 1000)
    assert m.heap.get_error() == 0
    m.heap.delete_handles(first, 1000)                  # second free of the same slots
    assert m.heap.get_error() & D.DEV_DOUBLE_FREE
    M = m.heap.info()["num_blocks"]
    bad_u64 = np.array([(200 << 56) | 5, (1 << 56) | ((M + 7) << 6), 0], dtype=np.uint64)
    bad = torch.from_numpy(bad_u64.view(np.int64)).cuda()
    m.heap.delete_handles(bad, 3)                       # unknown type, block past M, null
    assert m.heap.get_error() == D.DEV_BAD_HANDLE
    assert m.heap.count(m.type) == n - 1000
    assert_clean(m)


@pytest.mark.parametrize("r", [1, 2, 5, 16])
def test_lookup_count_r_keeps_semantics_and_stats(r):
    """r (Sec. 4.2, Fig. 11) changes how often new blocks are initialised, never the
    results; type_stats reports blocks and objects consistent with the checkers."""
    n, rounds = 40000, 3
    ref, _, _ = oracle.micro_run(SEED, n, rounds)
    m = make(heap_bytes=16 << 20, n=n)
    m.heap.set_lookups(r)
    for k in range(rounds):
        m.round(k)
        compare_round(m.stats(), ref[k])
    st = m.heap.type_stats(m.type)
    host = assert_clean(m)
    assert st["objects"] == ref[-1]["live"] == host["live"][0]
    assert st["blocks"] == host["blocks_in_use"]
    assert abs(st["fragmentation"] - host["fragmentation"]) < 1e-12
    assert 0.0 <= st["fragmentation"] < 1.0


def test_device_do_visits_every_object_once():
    """device_do (Sec. 2.1): every thread's sequential for-each sees each live object
    exactly once (count and sum of ids equal the oracle's)."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    n, rounds = 20000, 3
    ref, _, _ = oracle.micro_run(SEED, n, rounds)
    m = make(heap_bytes=16 << 20, n=n)
    for k in range(rounds):
        m.round(k)
    threads = 3
    out = torch.zeros(2 * threads, dtype=torch.int64, device="cuda")
    m.heap.run_kernel(D.K_MICRO_DEVICE_DO, threads, m.args(stats=out.data_ptr(), round=m.type))
    o = out.cpu().numpy().reshape(threads, 2)
    assert np.all(o[:, 0] == ref[-1]["live"])
    assert np.all(o[:, 1] == ref[-1]["sum_id"])


def test_atomic_peak_probe_final_words():
    """The L2 atomic-throughput probe: every op's bit k & 63 is cleared by even k and
    set by odd k, so ops on one word commute and the final words are fixed; they are
    recomputed here with numpy from the stated index rule."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    m = make(heap_bytes=4 << 20, n=64)
    nw, n, iters = 1 << 12, 3000, 9
    rng = np.random.default_rng(7)
    init = rng.integers(0, 2**63, size=nw, dtype=np.int64)
    words = torch.from_numpy(init.copy()).cuda()
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.heap.run_kernel(D.K_MICRO_ATOMIC_PEAK, n, m.args(handles_out=words.data_ptr(), n_ids=nw, round=iters,
                                                       stats=sink.data_ptr(), seed=1))
    torch.cuda.synchronize()
    w = init.view(np.uint64).copy()
    i = np.arange(n, dtype=np.uint64)
    for k in range(iters):
        idx = ((i + np.uint64(k * n)) * np.uint64(17)) & np.uint64(nw - 1)
        bit = np.uint64(1) << np.uint64(k & 63)
        if k & 1:
            np.bitwise_or.at(w, idx, bit)
        else:
            np.bitwise_and.at(w, idx, ~bit)
    assert np.array_equal(words.cpu().numpy().view(np.uint64), w)
    with pytest.raises(RuntimeError):
        m.heap.run_kernel(D.K_MICRO_ATOMIC_PEAK, n, m.args(handles_out=words.data_ptr(), n_ids=nw - 1, round=1,
                                                           stats=sink.data_ptr()))
    assert m.heap.get_error() == 0


@pytest.mark.parametrize("scan,flags", [(3, 0), (3, 32), (1, 0), (5, 0)])
def test_heap_beyond_one_wave_of_enumeration_ctas(scan, flags):
    """A 5 GiB heap has more level-1 tiles (~1200) than single-tile look-back CTAs
    fit on the GPU at once (~900): the enumeration runs the multi-tile kernel (CTA
    index orders the look-back), or with DSOA_FLAG_ENUM_TICKETS (32) hands tiles
    out by the ticket counter; the rounds still match the oracle.  The two-kernel
    enumeration runs the same heap."""
    n, rounds = 1 << 18, 3
    ref, _, _ = oracle.micro_run(SEED, n, rounds)
    m = make(heap_bytes=5 << 30, n=n, scan_tiles=scan)
    m.heap.set_flags(flags)
    assert m.heap.info()["num_blocks"] > 4096 * 1100
    for r in range(rounds):
        m.round(r)
        compare_round(m.stats(), ref[r])
    assert m.heap.get_error() == 0
    assert all(v == 0 for v in m.heap.check().values())
    m.heap.close()


def test_doall_at_benchmark_size_every_object():
    """The do-all sweep's size (2^26 objects, > L2) with the vectorised kernel the
    benchmark times: after two do-alls every x equals (id * 1.5f) + id with each
    operation rounded once, checked for all 2^26 objects."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    n = 1 << 26
    m = Micro(int(n * 16 * 1.3) + (64 << 20), SEED, n)
    m.new(0)
    m.heap.parallel_do(m.type, D.M_MICRO_SCALE, m.args())
    m.heap.parallel_do_enumerated(m.type, D.M_MICRO_SCALE, m.args())
    x, live = m.gather(n)
    assert live.all()
    ids = np.arange(n, dtype=np.float32)
    want = (ids * np.float32(1.5)).astype(np.float32) + ids
    assert np.array_equal(x.view(np.uint32), want.astype(np.float32).view(np.uint32))
    assert m.heap.get_error() == 0
    m.heap.close()
    del m
    torch.cuda.empty_cache()


@pytest.mark.parametrize("threads,per_thread", [(1 << 14, 1), (1 << 14, 16), (4096, 64), (1000, 7)])
def test_sequential_news_per_thread_match_oracle(threads, per_thread):
    """The Linux-scalability allocation pattern (Sec. 6.5): every thread creates
    `per_thread` objects one after another (K_MICRO_NEW_EACH).  The objects are
    the ids 0 .. threads * per_thread - 1 of one oracle round, so after the
    round's do-all and parity delete the statistics and per-object x equal the
    oracle's; then delete-all empties the heap."""
    from paper_1810_11765_gb300 import dsoa as D
    n = threads * per_thread
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, 1, per_object=True)
    m = make(heap_bytes=int(n * 16 * 2.2) + (8 << 20), n=n)
    m.heap.run_kernel(D.K_MICRO_NEW_EACH, threads, m.args(round=per_thread, n_ids=m.type))
    assert m.heap.count(m.type) == n
    _, live0 = m.gather(n)
    assert live0.sum() == n                         # every id once: no slot handed out twice
    m.scale()
    m.delete(0)
    compare_round(m.stats(), ref[0])
    x, live = m.gather(n)
    assert np.array_equal(live, live_ref)
    assert np.array_equal(x[live_ref.astype(bool)], x_ref[live_ref.astype(bool)])
    assert_clean(m)
    m.heap.parallel_do(m.type, D.M_MICRO_DELETE_ALL, m.args())
    assert m.heap.count(m.type) == 0
    assert_clean(m)
