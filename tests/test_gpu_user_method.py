"""User methods on the GPU (Sec. 2.1: parallel_do of any member function).

tests/user_method.cu is a user library built against the public headers: its
methods are registered by DSOA_METHOD when the library loads, and
dsoa_parallel_do runs them like built-in ones.  The microbench with the user's
scale method in place of the built-in one gives the oracle's objects bit for
bit; a user method that allocates objects of another type (and of its own
type, which the do-all's snapshot must not visit) gives the oracle's live set.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from conftest import ROOT
from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu

SEED = 0x5EED0001
SCALE, SPAWN, MARK = 1000, 1001, 1002
OK, INVALID_ARG, UNKNOWN_METHOD = 0, -1, -7


class UserArgs(ctypes.Structure):
    _fields_ = [("other_type", ctypes.c_uint32), ("n_ids", ctypes.c_uint32), ("out", ctypes.c_void_p)]


@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    gpu_ready()
    from paper_1810_11765_gb300 import build, dsoa as D
    D.load()
    out = tmp_path_factory.mktemp("user") / "libuser_methods.so"
    subprocess.run([build._nvcc(), *build.ARCH, "-O3", "-std=c++17", "-I", build.INCLUDE, "-shared",
                    "-Xcompiler", "-fPIC", "-cudart", "shared", "-o", str(out),
                    os.path.join(ROOT, "tests", "user_method.cu"), "-L", build.OUT, "-ldsoa",
                    "-Xlinker", "-rpath," + build.OUT], check=True)
    return ctypes.CDLL(str(out))


def micro(n, heap=None):
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    return Micro(0, SEED, n, heap=heap if heap is not None else D.Heap(64 << 20))


@pytest.mark.parametrize("n,rounds", [(1, 3), (1000, 5), (1 << 18, 10)])
def test_user_scale_method_in_the_microbench(user_lib, n, rounds):
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    m = micro(n)
    launches = m.heap.launches
    for r in range(rounds):
        m.new(r)
        m.heap.parallel_do(m.type, SCALE, UserArgs())
        m.delete(r)
        s = m.stats()
        assert (s["live"], s["xor_tag"]) == (ref[r]["live"], ref[r]["xor_tag"])
    assert m.heap.launches > launches
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))
    assert m.heap.get_error() == 0
    assert all(v == 0 for v in m.heap.check().values())
    m.heap.close()


def test_user_method_allocates_other_and_own_type(user_lib):
    """spawn on the microbench type creates one Tag per live object; spawn on Tag
    itself doubles the Tags exactly (the objects it creates are not visited);
    mark on either type reproduces the oracle's live set."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    n, rounds = 5000, 3
    _, _, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    heap = D.Heap(64 << 20)
    tag = heap.register_type([4])
    m = micro(n, heap)
    for r in range(rounds):
        m.round(r)
    live = int(live_ref.sum())
    heap.parallel_do(m.type, SPAWN, UserArgs(other_type=tag))
    assert heap.count(tag) == live
    heap.parallel_do(tag, SPAWN, UserArgs(other_type=tag))
    assert heap.count(tag) == 2 * live
    for t in (m.type, tag):
        out = torch.zeros(n * rounds, dtype=torch.uint8, device="cuda")
        heap.parallel_do(t, MARK, UserArgs(n_ids=n * rounds, out=out.data_ptr()))
        assert np.array_equal(out.cpu().numpy(), live_ref)
    assert heap.get_error() == 0
    assert all(v == 0 for v in heap.check().values())
    heap.close()


def test_user_method_in_a_captured_graph(user_lib):
    import torch
    n, rounds = 3000, 4
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m = micro(n)
        args = UserArgs()
        m.heap.graph_begin()
        m.heap.parallel_do(m.type, SCALE, args)
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


def test_registration_and_dispatch_errors(user_lib):
    from paper_1810_11765_gb300 import dsoa as D
    L = D.load()
    scale = ctypes.cast(user_lib.user_scale, ctypes.c_void_p).value
    mark = ctypes.cast(user_lib.user_mark, ctypes.c_void_p).value
    assert L.dsoa_register_method(SCALE, scale) == OK            # the same launcher again
    assert L.dsoa_register_method(SCALE, mark) == INVALID_ARG  # id taken by another
    assert L.dsoa_register_method(999, mark) == INVALID_ARG   # below the user range
    assert L.dsoa_register_method(1500, None) == INVALID_ARG
    m = micro(100)
    m.new(0)
    with pytest.raises(D.DsoaError) as e:
        m.heap.parallel_do(m.type, 1999, UserArgs())                   # nothing registered
    assert e.value.code == UNKNOWN_METHOD
    with pytest.raises(D.DsoaError) as e:
        m.heap.parallel_do(m.type, SCALE, D.MicroArgs())               # args of another size
    assert e.value.code == INVALID_ARG
    assert m.heap.get_error() == 0
    m.heap.close()


def test_user_method_covers_subtypes(user_lib):
    """A user do-all on a base type runs on the objects of its subtypes too (one
    snapshot, one launch per type): the microbench split over a base and a
    subtype, scaled by the user's method, equals the oracle."""
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    n, rounds = 4000, 4
    ref, x_ref, live_ref = oracle.micro_run(SEED, n, rounds, per_object=True)
    heap = D.Heap(64 << 20)
    heap.set_capacity_mode(D.CAPACITY_PER_TYPE)
    m = Micro(0, SEED, n, heap=heap, sub_fields=[8, 8], sub_share=0.6)
    for r in range(rounds):
        m.new(r)
        heap.parallel_do(m.type, SCALE, UserArgs())
        m.delete(r)
    assert heap.count(m.sub_type) > 0
    x, live = m.gather(n * rounds)
    assert np.array_equal(live, live_ref)
    sel = live_ref.astype(bool)
    assert np.array_equal(x[sel].view(np.uint32), x_ref[sel].view(np.uint32))
    assert heap.get_error() == 0
    heap.close()


def test_prologue_runs_once_per_do_all_of_a_family(user_lib):
    """A do-all on a type with subtypes launches the method once per member type;
    a method's prologue (per-launch work such as advancing step counters) must
    still run once per dsoa_parallel_do, in plain and in enumerated do-alls."""
    import torch
    from paper_1810_11765_gb300 import dsoa as D
    from paper_1810_11765_gb300.apps import Micro
    TALLY = 1003
    heap = D.Heap(64 << 20)
    m = Micro(0, SEED, 4000, heap=heap, sub_fields=[8], sub_share=0.5)
    m.new(0)
    assert heap.count(m.type) > 0 and heap.count(m.sub_type) > 0
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = UserArgs(out=cnt.data_ptr())
    for k in range(1, 4):
        heap.parallel_do(m.type, TALLY, args)
        torch.cuda.synchronize()
        assert int(cnt.item()) == k
    heap.parallel_do_enumerated(m.type, TALLY, args)
    heap.parallel_do(m.sub_type, TALLY, args)           # the subtype alone: one launch
    torch.cuda.synchronize()
    assert int(cnt.item()) == 5
    assert heap.get_error() == 0
    heap.close()
