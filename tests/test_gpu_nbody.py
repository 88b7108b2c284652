"""GPU parity of the n-body and particle-collision workloads (Body objects, forces
by device_do or by the pairwise tiled kernel, merges by six do-alls).

Bar: bit-exact.  The forces are sums of integers (fixed-point pair terms), so the
GPU's visit order and its partition of the pairs do not change a bit; every other
operation is one IEEE binary32 operation on both sides.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready, host_check

pytestmark = pytest.mark.gpu

SMALL = dict(G=2.0 ** -22, dt=0.25, eps2=2.0 ** -18, rc2=2.0 ** -12, fscale=2.0 ** 40,
             vscale=2.0 ** -8, mass_max=16)


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def cfg(**kw):
    from paper_1810_11765_gb300 import inputs
    d = dict(SMALL)
    d.update(kw)
    return inputs.NBodyConfig(**{k: v for k, v in d.items() if k in inputs.NBodyConfig.__dataclass_fields__})


def world(c, collide, tiled, heap_bytes=64 << 20, all_pairs=False):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import NBodyWorld
    heap = D.Heap(heap_bytes)
    w = NBodyWorld(heap, c, collide=collide, tiled=tiled, all_pairs=all_pairs)
    heap.freeze()
    return heap, w


def oracle_run(c, n, steps, collide, init=None):
    return oracle.nbody_run(n, steps, c.seed, G=c.G, dt=c.dt, eps2=c.eps2, rc2=c.rc2, fscale=c.fscale,
                            vscale=c.vscale, mass_max=c.mass_max, collide=collide, init=init)


@pytest.mark.parametrize("tiled", [False, True])
@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 700, 2000])
def test_nbody_bit_exact(n, tiled):
    c = cfg(seed=100 + n)
    heap, w = world(c, False, tiled)
    w.create(n)
    st0, al0 = w.read()
    ref0, _, _, _ = oracle_run(c, n, 0, False)
    assert np.array_equal(st0, ref0) and al0.all()
    for _ in range(5):
        w.step()
    st, alive = w.read()
    ref, ref_alive, _, _ = oracle_run(c, n, 5, False)
    assert np.array_equal(alive, ref_alive)
    assert np.array_equal(st.view(np.uint32), ref.view(np.uint32))
    assert heap.get_error() == 0
    heap.close()


@pytest.mark.parametrize("tiled,all_pairs", [(False, False), (True, False), (True, True)])
def test_collisions_bit_exact_per_step(tiled, all_pairs):
    """FIND by device_do, by the unordered-pair kernel and by the ordered-pair one."""
    c = cfg(seed=7, G=2.0 ** -24)
    n, steps = 2000, 20
    heap, w = world(c, True, tiled, all_pairs=all_pairs)
    w.create(n)
    _, _, counts, _ = oracle_run(c, n, steps, True)
    for k in range(steps):
        w.step()
        assert w.count() == counts[k + 1], k
    st, alive = w.read()
    ref, ref_alive, _, _ = oracle_run(c, n, steps, True)
    assert counts[-1] < counts[0]
    assert np.array_equal(alive, ref_alive)
    assert np.array_equal(st.view(np.uint32), ref.view(np.uint32))
    assert heap.get_error() == 0
    assert all(v == 0 for v in heap.check().values())
    host = host_check(heap, 1)
    assert all(v == 0 for v in host["violations"].values()), host
    heap.close()


@pytest.mark.parametrize("all_pairs", [False, True])
def test_collisions_with_many_bodies_in_reach(all_pairs):
    """A merge distance of 1/8 gives every body dozens of candidates: the keys of
    both bodies of a pair (register and shared-memory minima) must reproduce the
    oracle's targets, merges and deletions step by step."""
    c = cfg(seed=31, G=2.0 ** -24, rc2=2.0 ** -6)
    n, steps = 1500, 6
    heap, w = world(c, True, True, all_pairs=all_pairs)
    w.create(n)
    _, _, counts, _ = oracle_run(c, n, steps, True)
    for k in range(steps):
        w.step()
        assert w.count() == counts[k + 1], k
    st, alive = w.read()
    ref, ref_alive, _, _ = oracle_run(c, n, steps, True)
    assert counts[-1] < 0.8 * n
    assert np.array_equal(alive, ref_alive)
    assert np.array_equal(st.view(np.uint32), ref.view(np.uint32))
    assert heap.get_error() == 0
    heap.close()


def test_collisions_over_four_slot_blocks_indexed_by_slot():
    """17,000 bodies in blocks of four (4,250 listed blocks, beyond dense
    indexing): FORCE and FIND stage empty slots as mass-0 placeholders at the
    origin, which must never become a target; two collision steps equal the
    oracle's."""
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import NBodyWorld
    c = cfg(seed=5, G=2.0 ** -24, rc2=2.0 ** -12)
    n, steps = 17000, 2
    heap = D.Heap(64 << 20)
    heap.register_type([4])
    heap.set_capacity_mode(D.CAPACITY_PER_TYPE)
    w = NBodyWorld(heap, c, collide=True, tiled=True)
    heap.freeze()
    assert heap.capacity(w.type) == 4
    w.create(n)
    for _ in range(steps):
        w.step()
    st, alive = w.read()
    ref, ref_alive, counts, _ = oracle_run(c, n, steps, True)
    assert counts[-1] < n
    assert np.array_equal(alive, ref_alive)
    assert np.array_equal(st.view(np.uint32), ref.view(np.uint32))
    assert heap.get_error() == 0
    heap.close()


def test_merge_chain_hand_case():
    rc = 2.0 ** -5
    c = cfg(G=0.0, rc2=rc * rc)
    init = np.array([[0.0, 0, 0, 0, 1.0], [0.8 * rc, 0, 0, 0, 2.0], [1.1 * rc, 0, 0, 0, 3.0]], np.float32)
    heap, w = world(c, True, True, 4 << 20)
    w.create(3, init)
    w.step()
    st1, al1 = w.read()
    assert al1.tolist() == [1, 0, 1] and st1[2, 4] == 5.0
    w.step()
    st2, al2 = w.read()
    ref, ref_alive, counts, _ = oracle_run(c, 3, 2, True, init=init)
    assert counts.tolist() == [3, 2, 1]
    assert al2.tolist() == ref_alive.tolist() == [0, 0, 1]
    assert np.array_equal(st2.view(np.uint32), ref.view(np.uint32))
    heap.close()


def test_forces_sum_to_zero_and_match_sampled_bodies_at_full_size():
    """65,536 bodies (the configured size): one FORCE by the unordered-pair and the
    ordered-pair tiled kernels and by the device_do walk; Newton's third law holds
    exactly over all bodies, and sampled bodies (first, last, a ragged spread)
    match the oracle one by one."""
    from paper_1810_11765_gb300 import inputs
    c = inputs.NBodyConfig()
    ids = np.unique(np.concatenate([[0, 1, 63, 64, c.n - 1], np.random.default_rng(5).integers(0, c.n, 27)]))
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import NBodyWorld
    got = {}
    for scheme in ("unordered", "ordered", "walk"):
        heap = D.Heap(512 << 20)
        w = NBodyWorld(heap, c, tiled=scheme != "walk", all_pairs=scheme == "ordered")
        heap.freeze()
        w.create(c.n)
        st0, _ = w.read()
        w.force()
        _, _, F = w.read(forces=True)
        assert np.all(F.sum(0) == 0)
        got[scheme] = F
        assert heap.get_error() == 0
        heap.close()
    assert np.array_equal(got["unordered"], got["walk"])
    assert np.array_equal(got["ordered"], got["walk"])
    ref0, _, _, _ = oracle_run(c, c.n, 0, False)
    assert np.array_equal(st0, ref0)
    want = oracle.nbody_force_on(ref0, ids, G=c.G, eps2=c.eps2, fscale=c.fscale)
    assert np.array_equal(got["unordered"][ids], want)


def _general_init(n, seed):
    """Positions in [-1, 1)^2, masses in [0.5, 20) with fractional parts, so the
    two terms of a pair have different coefficients ((G S m_i) m_j vs (G S m_j) m_i)."""
    rng = np.random.default_rng(seed)
    init = np.zeros((n, 5), np.float32)
    init[:, 0:2] = rng.uniform(-1.0, 1.0, (n, 2))
    init[:, 2:4] = rng.uniform(-2.0 ** -9, 2.0 ** -9, (n, 2))
    init[:, 4] = rng.uniform(0.5, 20.0, n)
    return init


def _forces(c, init, tiled, all_pairs=False, four_slot_blocks=False):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import NBodyWorld
    heap = D.Heap(64 << 20)
    if four_slot_blocks:
        heap.register_type([4])                   # 256-byte blocks: four Bodies per block
        heap.set_capacity_mode(D.CAPACITY_PER_TYPE)
    w = NBodyWorld(heap, c, tiled=tiled, all_pairs=all_pairs)
    heap.freeze()
    if four_slot_blocks:
        assert heap.capacity(w.type) == 4
    w.create(init.shape[0], init)
    w.force()
    st, alive, F = w.read(forces=True)
    assert np.array_equal(st, init) and alive.all()
    assert heap.get_error() == 0
    heap.close()
    return F


@pytest.mark.parametrize("n", [1, 2, 31, 33, 255, 257, 700, 2100])
def test_force_pair_schemes_with_unequal_pair_coefficients(n):
    """G not a power of two and fractional masses: the unordered-pair kernel (one
    evaluation per pair, both bodies' terms), the ordered-pair kernel and the
    device_do walk give the oracle's integers for every body, ragged last tiles
    and single-group cases included."""
    c = cfg(G=float(np.float32(3.1e-7)), fscale=2.0 ** 36)
    init = _general_init(n, 1000 + n)
    want = oracle.nbody_force_on(init, np.arange(n), G=c.G, eps2=c.eps2, fscale=c.fscale)
    for tiled, all_pairs in ((True, False), (True, True), (False, False)):
        assert np.array_equal(_forces(c, init, tiled, all_pairs), want), (tiled, all_pairs)


@pytest.mark.parametrize("n", [12000, 17000])
def test_force_over_four_slot_blocks(n):
    """Four Bodies per block (per-type capacity behind a 4-byte type): 3000 listed
    blocks are indexed densely, 4250 by slot (60 of every 64 indices are empty
    slots staged as mass 0).  Both pair schemes give the oracle's integers."""
    c = cfg(G=float(np.float32(3.1e-7)), fscale=2.0 ** 36)
    init = _general_init(n, 77 + n)
    want = oracle.nbody_force_on(init, np.arange(n), G=c.G, eps2=c.eps2, fscale=c.fscale)
    for all_pairs in (False, True):
        assert np.array_equal(_forces(c, init, True, all_pairs, four_slot_blocks=True), want), all_pairs


def test_inverse_root_sequence_is_exact_on_its_whole_domain(tmp_path):
    """The FORCE kernel's fused-multiply-add sequence for 1/sqrt(d2) gives the bits
    of RN(1 / RN(sqrt d2)) (what the oracle computes) for every binary32 d2 in
    [2^-80, FLT_MAX]: all 1.74 G inputs, compared on the GPU."""
    import ctypes
    import os
    import subprocess
    from conftest import ROOT
    from paper_1810_11765_gb300 import build
    lib = tmp_path / "libinvroot.so"
    subprocess.run([build._nvcc(), *build.ARCH, "-O3", "-I", build.CSRC, "-shared", "-Xcompiler", "-fPIC",
                    "-cudart", "shared", "-o", str(lib), os.path.join(ROOT, "tests", "inv_root_check.cu")],
                   check=True)
    f = ctypes.CDLL(str(lib)).inv_root_mismatches
    f.argtypes, f.restype = [ctypes.c_uint32, ctypes.c_uint32], ctypes.c_longlong
    lo = int(np.float32(2.0 ** -80).view(np.uint32))
    hi = int(np.float32(np.inf).view(np.uint32))          # exclusive: up to FLT_MAX
    assert f(lo, hi) == 0


def test_collision_graph_replay_matches_plain():
    """A collision step (one enumeration, six do-alls) captured as a CUDA graph and
    replayed gives the plain steps' state, bit for bit."""
    import torch
    c = cfg(seed=9, G=2.0 ** -24)
    n, steps = 1500, 12
    finals = []
    for graph in (False, True):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            heap, w = world(c, True, True)
            w.create(n)
            if graph:
                heap.graph_begin()
                w.step()
                g = heap.graph_end()
                for _ in range(steps):
                    g.launch()
                g.close()
            else:
                for _ in range(steps):
                    w.step()
            finals.append(w.read())
            assert heap.get_error() == 0
            heap.close()
    assert np.array_equal(finals[0][0].view(np.uint32), finals[1][0].view(np.uint32))
    ref, ref_alive, _, _ = oracle_run(c, n, steps, True)
    assert np.array_equal(finals[1][1], ref_alive)
    assert np.array_equal(finals[1][0].view(np.uint32), ref.view(np.uint32))


def test_rejects_bad_arguments():
    from paper_1810_11765_gb300 import dsoa as D
    c = cfg()
    heap, w = world(c, True, True, 4 << 20)
    with pytest.raises(D.DsoaError):
        heap.parallel_new(w.type, 10, D.C_NBODY, w.args(n_ids=5))        # n beyond n_ids
    with pytest.raises(D.DsoaError):
        heap.parallel_do(w.type, D.M_NBODY_MOVE, w.args(eps2=0.0))        # no softening
    with pytest.raises(D.DsoaError):
        heap.parallel_do(w.type, D.M_COLL_CLAIM, w.args(handle_of=None))  # claims need the id map
    with pytest.raises(D.DsoaError):
        heap.parallel_do(w.type, D.M_NBODY_FORCE_TILED, w.args(eps2=2.0 ** -81))   # inverse cube may overflow
    heap.close()
