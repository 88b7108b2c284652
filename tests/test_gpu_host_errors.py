"""Host-side argument and state errors of the C ABI return codes (no device
fault, no hang): registration after the freeze, bad type / method ids, argument
structs of the wrong size, heaps too small for their metadata."""
import ctypes

import pytest

from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def test_error_codes():
    from paper_1810_11765_gb300 import dsoa as D
    L = D.load()
    heap = D.Heap(8 << 20)
    t = heap.register_type([4, 4, 8])
    heap.freeze()
    fb = (ctypes.c_uint32 * 1)(4)
    out = ctypes.c_int()
    assert L.dsoa_register_type(heap.handle, fb, 1, ctypes.byref(out)) == -2       # FROZEN
    assert L.dsoa_set_capacity_mode(heap.handle, 1) == -2                          # FROZEN
    a = D.MicroArgs()
    assert L.dsoa_parallel_new(heap.handle, 7, 10, D.C_MICRO, ctypes.byref(a), ctypes.sizeof(a)) == -1
    assert L.dsoa_parallel_new(heap.handle, t, 10, 999, ctypes.byref(a), ctypes.sizeof(a)) == -7
    assert L.dsoa_parallel_do(heap.handle, t, 199, ctypes.byref(a), ctypes.sizeof(a)) == -7
    assert L.dsoa_parallel_new(heap.handle, t, 10, D.C_MICRO, ctypes.byref(a), ctypes.sizeof(a) - 8) == -1
    assert L.dsoa_count(heap.handle, -1, ctypes.byref(ctypes.c_uint64())) == -1
    assert L.dsoa_enumerate_many(heap.handle, (ctypes.c_int * 2)(t, t), 2) == -1   # duplicate type
    assert L.dsoa_set_launch(heap.handle, 100, 0, 0, 0, 0) == -1                    # tpb not a multiple of 64
    assert heap.get_error() == 0
    heap.close()
    small = D.Heap(4096)                       # too small for any block plus metadata
    small.register_type([4, 4, 8])
    with pytest.raises(D.DsoaError) as e:
        small.freeze()
    assert e.value.code == -4                  # OOM
    small.close()
    big = D.Heap(8 << 20)
    with pytest.raises(D.DsoaError) as e:
        big.register_type([3])                 # field size not 1, 2, 4, 8 or 16
    assert e.value.code == -1
    for _ in range(16):                        # DSOA_MAX_TYPES
        big.register_type([4])
    with pytest.raises(D.DsoaError) as e:
        big.register_type([4])
    assert e.value.code == -3                  # TOO_MANY_TYPES
    big.close()
