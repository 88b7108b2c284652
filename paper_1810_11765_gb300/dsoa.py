"""Python binding of the C ABI in ``include/dsoa.h`` and ``include/dsoa_apps.h``.

Argument marshalling only: every step of the allocator and the do-all runs in the
CUDA kernels of ``_lib/libdsoa.so``.  There is no CPU fallback; loading fails with
an error when the library has not been built (``paper_1810_11765_gb300.build``).
PyTorch supplies device memory (tensors) and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DSOA_OK = 0
ERRORS = {-1: "invalid argument", -2: "heap layout already frozen", -3: "too many types",
          -4: "heap too small", -5: "CUDA runtime error", -6: "heap layout not frozen",
          -7: "unknown built-in method", -8: "synchronous call during stream capture",
          -9: "heap larger than the fixed no-allocation scratch allows"}

DEV_OOM, DEV_SPIN, DEV_DOUBLE_FREE, DEV_BAD_HANDLE, DEV_BAD_INDEX = 1, 2, 4, 8, 16
FLAG_NO_COALESCE, FLAG_NO_ROTATE, FLAG_NO_HINT, FLAG_FUSED, FLAG_PDL = 1, 2, 4, 8, 16
FLAG_ENUM_TICKETS = 32
FLAG_NO_FRESH_GROUP, FLAG_PAPER_R, FLAG_R_PER_ROUND = 128, 256, 512
FLAG_DRAIN = 1024
CHECK_NAMES = ["hier", "free_xor", "multi_type", "active_subset", "type", "free_word",
               "empty_alloc", "active_exact", "tail_bits", "cap_bits"]
CAPACITY_UNIFORM, CAPACITY_PER_TYPE = 0, 1

# built-in ids (dsoa_apps.h)
C_MICRO, M_MICRO_SCALE, M_MICRO_SCALE_SCALAR, M_MICRO_DELETE = 100, 101, 102, 103
M_MICRO_GATHER, M_MICRO_STATS, M_MICRO_SCALE_TMA, M_MICRO_DELETE_ALL = 104, 105, 106, 107
M_MICRO_HANDLES = 108
K_MICRO_DEVICE_DO = 150
K_MICRO_ATOMIC_PEAK = 151
K_MICRO_NEW_EACH = 152
C_GOL_CELL, M_GOL_SPREAD, M_GOL_REAP, M_GOL_DECIDE, M_GOL_READ, M_GOL_KILL = 200, 201, 202, 203, 204, 205
K_GOL_ADVANCE = 250
M_WATOR_FISH_CHOOSE, M_WATOR_FISH_MOVE, M_WATOR_SHARK_CHOOSE, M_WATOR_SHARK_MOVE = 301, 302, 303, 304
M_WATOR_KILL, K_WATOR_INIT, K_WATOR_ADVANCE = 305, 350, 351
M_WATOR_FISH_MOVE_DEFER, K_WATOR_BIRTHS = 306, 352
M_GOL_DECIDE_ADVANCE, M_WATOR_SHARK_MOVE_ADVANCE = 206, 307
M_TRAFFIC_MOVE, M_TRAFFIC_READ = 401, 402
K_TRAFFIC_INIT, K_TRAFFIC_CLEAR, K_TRAFFIC_ONRAMP, K_TRAFFIC_ADVANCE = 450, 451, 452, 453
K_TRAFFIC_ONRAMP_ADVANCE = 454
C_NBODY, M_NBODY_FORCE, M_NBODY_MOVE = 500, 501, 502
M_COLL_FIND, M_COLL_CLAIM, M_COLL_MERGE, M_COLL_DELETE = 503, 504, 505, 506
M_NBODY_READ, M_NBODY_FORCE_TILED, M_COLL_FIND_TILED = 507, 508, 509
USER_METHOD_MIN, USER_METHOD_MAX = 1000, 1999
NBODY_KEYED_FIND = 1
NBODY_ALL_PAIRS = 2

INST_IDLE, INST_RUN, INST_KILL = 0, 1, 2

P = ctypes.c_void_p
u8p = ctypes.c_void_p


class MicroArgs(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("id_base", ctypes.c_uint32), ("round", ctypes.c_uint32),
                ("x_out", P), ("live_out", P), ("n_ids", ctypes.c_uint64), ("stats", P),
                ("handles_out", P)]


class MicroStats(ctypes.Structure):
    _fields_ = [("live", ctypes.c_uint64), ("sum_id", ctypes.c_uint64), ("sum_tag", ctypes.c_uint64),
                ("xor_tag", ctypes.c_uint64), ("sum_x", ctypes.c_double)]


class Inst(ctypes.Structure):
    _fields_ = [("cellmap", P), ("occ", P), ("claim", P), ("seed", ctypes.c_uint64),
                ("w", ctypes.c_uint32), ("h", ctypes.c_uint32), ("t", ctypes.c_uint32),
                ("state", ctypes.c_uint32)]


class GolArgs(ctypes.Structure):
    _fields_ = [("inst", P), ("init", P), ("n_inst", ctypes.c_uint32), ("target", ctypes.c_uint32),
                ("cell_type", ctypes.c_int32), ("alive_type", ctypes.c_int32)]


class WatorArgs(ctypes.Structure):
    _fields_ = [("inst", P), ("init", P), ("n_inst", ctypes.c_uint32), ("target", ctypes.c_uint32),
                ("fish_type", ctypes.c_int32), ("shark_type", ctypes.c_int32)]


class TrafficArgs(ctypes.Structure):
    _fields_ = [("occ0", P), ("occ1", P), ("vel_out", P), ("ring_base", P), ("ring_thr", P),
                ("init_occ", P), ("init_v", P), ("t_dev", P), ("seed", ctypes.c_uint64),
                ("n_rings", ctypes.c_uint32), ("slow_thr", ctypes.c_uint32),
                ("ramp_thr", ctypes.c_uint32), ("car_type", ctypes.c_int32)]


class NBodyArgs(ctypes.Structure):
    _fields_ = [("handle_of", P), ("init", P), ("out", P), ("alive_out", P), ("force_out", P),
                ("seed", ctypes.c_uint64), ("n_ids", ctypes.c_uint32), ("mass_max", ctypes.c_uint32),
                ("G", ctypes.c_float), ("dt", ctypes.c_float), ("eps2", ctypes.c_float),
                ("rc2", ctypes.c_float), ("fscale", ctypes.c_float), ("vscale", ctypes.c_float),
                ("body_type", ctypes.c_int32), ("flags", ctypes.c_uint32)]


# exported names of include/dsoa.h, in declaration order
ABI_FUNCTIONS = [
    "dsoa_heap_create", "dsoa_heap_create_from", "dsoa_register_type", "dsoa_register_subtype",
    "dsoa_type_base", "dsoa_register_method", "dsoa_heap_freeze",
    "dsoa_heap_info", "dsoa_field_offset", "dsoa_parallel_new", "dsoa_parallel_do",
    "dsoa_parallel_do_enumerated", "dsoa_run_kernel", "dsoa_delete_handles", "dsoa_enumerate",
    "dsoa_enumerate_many", "dsoa_count", "dsoa_count_async", "dsoa_count_many_async",
    "dsoa_free_blocks_async", "dsoa_get_error", "dsoa_check", "dsoa_export_state",
    "dsoa_heap_save", "dsoa_heap_load",
    "dsoa_get_ctx", "dsoa_graph_begin", "dsoa_graph_end", "dsoa_graph_launch",
    "dsoa_graph_destroy", "dsoa_set_launch", "dsoa_set_flags", "dsoa_set_lookups",
    "dsoa_type_stats", "dsoa_launch_count", "dsoa_set_capacity_mode", "dsoa_type_capacity",
    "dsoa_heap_destroy", "dsoa_error_string",
    "dsoa_bitmap_heap_create", "dsoa_bitmap_register_type", "dsoa_bitmap_heap_freeze",
    "dsoa_bitmap_heap_info", "dsoa_bitmap_parallel_new", "dsoa_bitmap_parallel_do",
    "dsoa_bitmap_count", "dsoa_bitmap_check", "dsoa_bitmap_get_error", "dsoa_bitmap_heap_destroy",
    "dsoa_enumerate_noalloc",
]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libdsoa.so (no implicit build, no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with paper_1810_11765_gb300.build.build()")
    L = ctypes.CDLL(p)
    vp, sz, i32, u32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "dsoa_heap_create": [sz, vp, vp], "dsoa_heap_create_from": [vp, sz, vp, vp],
        "dsoa_register_type": [vp, vp, i32, vp], "dsoa_heap_freeze": [vp],
        "dsoa_register_subtype": [vp, i32, vp, i32, vp], "dsoa_type_base": [vp, i32, vp],
        "dsoa_register_method": [i32, vp],
        "dsoa_heap_info": [vp, vp, vp, vp, vp], "dsoa_field_offset": [vp, i32, i32, vp],
        "dsoa_parallel_new": [vp, i32, u64, i32, vp, sz], "dsoa_parallel_do": [vp, i32, i32, vp, sz],
        "dsoa_parallel_do_enumerated": [vp, i32, i32, vp, sz],
        "dsoa_run_kernel": [vp, i32, u64, vp, sz], "dsoa_enumerate": [vp, i32, vp, vp, vp],
        "dsoa_enumerate_many": [vp, vp, i32], "dsoa_count_many_async": [vp, vp, i32, vp],
        "dsoa_delete_handles": [vp, vp, u64],
        "dsoa_count": [vp, i32, vp], "dsoa_count_async": [vp, i32, vp],
        "dsoa_free_blocks_async": [vp, vp], "dsoa_get_error": [vp, vp], "dsoa_check": [vp, vp],
        "dsoa_export_state": [vp, vp, sz, vp, vp], "dsoa_get_ctx": [vp, vp, sz],
        "dsoa_heap_save": [vp, vp, sz, vp], "dsoa_heap_load": [vp, vp, sz],
        "dsoa_graph_begin": [vp], "dsoa_graph_end": [vp, vp], "dsoa_graph_launch": [vp, vp],
        "dsoa_graph_destroy": [vp], "dsoa_set_launch": [vp, i32, i32, i32, i32, i32],
        "dsoa_set_flags": [vp, u32], "dsoa_launch_count": [vp, vp], "dsoa_heap_destroy": [vp],
        "dsoa_set_lookups": [vp, i32], "dsoa_type_stats": [vp, i32, vp],
        "dsoa_set_capacity_mode": [vp, i32], "dsoa_type_capacity": [vp, i32, vp],
        "dsoa_error_string": [i32],
        "dsoa_enumerate_noalloc": [vp, i32, vp, vp, vp, u64],
        "dsoa_bitmap_heap_create": [sz, vp, vp], "dsoa_bitmap_register_type": [vp, vp, i32, vp],
        "dsoa_bitmap_heap_freeze": [vp], "dsoa_bitmap_heap_info": [vp, vp, vp, vp],
        "dsoa_bitmap_parallel_new": [vp, i32, u64, i32, vp, sz],
        "dsoa_bitmap_parallel_do": [vp, i32, i32, vp, sz], "dsoa_bitmap_count": [vp, i32, vp],
        "dsoa_bitmap_check": [vp, vp], "dsoa_bitmap_get_error": [vp, vp],
        "dsoa_bitmap_heap_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "dsoa_error_string" else i32
    if path is None:
        _lib = L
    return L


class DsoaError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")
        self.code = code


def _ok(rc, what):
    if rc != DSOA_OK:
        raise DsoaError(rc, what)


def _addr(x) -> int | None:
    """Device / host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


class Graph:
    def __init__(self, handle):
        self._h = handle

    def launch(self, stream=None):
        _ok(load().dsoa_graph_launch(self._h, _stream_ptr(stream)), "dsoa_graph_launch")

    def close(self):
        if self._h:
            load().dsoa_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Heap:
    """A device heap of 64-slot SOA blocks (dsoa_heap)."""

    def __init__(self, nbytes: int | None = None, stream=None, buffer=None):
        L = load()
        self._h = ctypes.c_void_p()
        self.stream = stream
        sp = _stream_ptr(stream)
        self._buffer = buffer
        if buffer is not None:
            _ok(L.dsoa_heap_create_from(_addr(buffer), buffer.numel() * buffer.element_size(), sp,
                                        ctypes.byref(self._h)), "dsoa_heap_create_from")
        else:
            _ok(L.dsoa_heap_create(int(nbytes), sp, ctypes.byref(self._h)), "dsoa_heap_create")

    @property
    def handle(self):
        return self._h

    def register_type(self, field_bytes) -> int:
        fb = (ctypes.c_uint32 * len(field_bytes))(*field_bytes)
        t = ctypes.c_int()
        _ok(load().dsoa_register_type(self._h, fb, len(field_bytes), ctypes.byref(t)), "dsoa_register_type")
        return t.value

    def register_subtype(self, base: int, extra_field_bytes=()) -> int:
        """A type extending ``base``: base's fields, then ``extra_field_bytes``."""
        n = len(extra_field_bytes)
        fb = (ctypes.c_uint32 * max(n, 1))(*extra_field_bytes)
        t = ctypes.c_int()
        _ok(load().dsoa_register_subtype(self._h, base, fb, n, ctypes.byref(t)), "dsoa_register_subtype")
        return t.value

    def type_base(self, t: int) -> int:
        b = ctypes.c_int()
        _ok(load().dsoa_type_base(self._h, t, ctypes.byref(b)), "dsoa_type_base")
        return b.value

    def freeze(self):
        _ok(load().dsoa_heap_freeze(self._h), "dsoa_heap_freeze")

    def set_capacity_mode(self, mode: int):
        """CAPACITY_UNIFORM (64 slots for every type) or CAPACITY_PER_TYPE (Sec. 3.2 N_T)."""
        _ok(load().dsoa_set_capacity_mode(self._h, mode), "dsoa_set_capacity_mode")

    def capacity(self, t: int) -> int:
        n = ctypes.c_uint32()
        _ok(load().dsoa_type_capacity(self._h, t, ctypes.byref(n)), "dsoa_type_capacity")
        return n.value

    def info(self) -> dict:
        M, bb, nl, meta = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        _ok(load().dsoa_heap_info(self._h, ctypes.byref(M), ctypes.byref(bb), ctypes.byref(nl),
                                  ctypes.byref(meta)), "dsoa_heap_info")
        return {"num_blocks": M.value, "block_bytes": bb.value, "num_levels": nl.value,
                "metadata_bytes": meta.value}

    def field_offset(self, t: int, f: int) -> int:
        o = ctypes.c_uint32()
        _ok(load().dsoa_field_offset(self._h, t, f, ctypes.byref(o)), "dsoa_field_offset")
        return o.value

    def parallel_new(self, t: int, n: int, ctor: int, args):
        _ok(load().dsoa_parallel_new(self._h, t, n, ctor, ctypes.byref(args), ctypes.sizeof(args)),
            "dsoa_parallel_new")

    def parallel_do(self, t: int, method: int, args):
        _ok(load().dsoa_parallel_do(self._h, t, method, ctypes.byref(args), ctypes.sizeof(args)),
            "dsoa_parallel_do")

    def parallel_do_enumerated(self, t: int, method: int, args):
        _ok(load().dsoa_parallel_do_enumerated(self._h, t, method, ctypes.byref(args), ctypes.sizeof(args)),
            "dsoa_parallel_do_enumerated")

    def run_kernel(self, kernel: int, n: int, args):
        _ok(load().dsoa_run_kernel(self._h, kernel, n, ctypes.byref(args), ctypes.sizeof(args)),
            "dsoa_run_kernel")

    def delete_handles(self, handles_dev, n: int):
        _ok(load().dsoa_delete_handles(self._h, _addr(handles_dev), n), "dsoa_delete_handles")

    def enumerate_many(self, types):
        """One enumeration launch for several types (dsoa_enumerate_many)."""
        arr = (ctypes.c_int * len(types))(*types)
        _ok(load().dsoa_enumerate_many(self._h, arr, len(types)), "dsoa_enumerate_many")

    def enumerate(self, t: int):
        R, occ, r = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _ok(load().dsoa_enumerate(self._h, t, ctypes.byref(R), ctypes.byref(occ), ctypes.byref(r)),
            "dsoa_enumerate")
        return R.value, occ.value, r.value

    def count(self, t: int) -> int:
        out = ctypes.c_uint64()
        _ok(load().dsoa_count(self._h, t, ctypes.byref(out)), "dsoa_count")
        return out.value

    def count_many_async(self, types, out_dev):
        """Live objects of each type into out_dev[0..len(types)) (uint64), one launch."""
        arr = (ctypes.c_int * len(types))(*types)
        _ok(load().dsoa_count_many_async(self._h, arr, len(types), _addr(out_dev)), "dsoa_count_many_async")

    def count_async(self, t: int, out_dev):
        _ok(load().dsoa_count_async(self._h, t, _addr(out_dev)), "dsoa_count_async")

    def free_blocks_async(self, out_dev):
        _ok(load().dsoa_free_blocks_async(self._h, _addr(out_dev)), "dsoa_free_blocks_async")

    def get_error(self) -> int:
        e = ctypes.c_int()
        _ok(load().dsoa_get_error(self._h, ctypes.byref(e)), "dsoa_get_error")
        return e.value

    def check(self) -> dict:
        out = (ctypes.c_uint64 * len(CHECK_NAMES))()
        _ok(load().dsoa_check(self._h, out), "dsoa_check")
        return {n: int(out[i]) for i, n in enumerate(CHECK_NAMES)}

    def export_state(self) -> dict:
        need, words = ctypes.c_size_t(), ctypes.c_uint64()
        L = load()
        _ok(L.dsoa_export_state(self._h, None, 0, ctypes.byref(need), ctypes.byref(words)), "dsoa_export_state")
        buf = np.empty(need.value, dtype=np.uint8)
        _ok(L.dsoa_export_state(self._h, buf.ctypes.data, need.value, ctypes.byref(need), ctypes.byref(words)),
            "dsoa_export_state")
        M = self.info()["num_blocks"]
        slot = buf[:M * 8].view(np.uint64)
        btype = buf[M * 8:M * 12].view(np.uint32)
        bm = buf[M * 12:].view(np.uint64).reshape(-1, words.value)
        return {"slot": slot, "btype": btype, "bitmaps": bm}

    def save(self) -> np.ndarray:
        """Checkpoint image of the heap (header + heap bytes) in host memory."""
        need = ctypes.c_size_t()
        L = load()
        _ok(L.dsoa_heap_save(self._h, None, 0, ctypes.byref(need)), "dsoa_heap_save")
        buf = np.empty(need.value, dtype=np.uint8)
        _ok(L.dsoa_heap_save(self._h, buf.ctypes.data, need.value, ctypes.byref(need)), "dsoa_heap_save")
        return buf

    def load_image(self, image: np.ndarray):
        """Restore a checkpoint image taken from a heap of the same layout."""
        img = np.ascontiguousarray(image, dtype=np.uint8)
        _ok(load().dsoa_heap_load(self._h, img.ctypes.data, img.size), "dsoa_heap_load")

    def set_launch(self, tpb=0, ctas_per_sm=0, slots_per_thread=0, scan_tiles=0, waves=0):
        _ok(load().dsoa_set_launch(self._h, tpb, ctas_per_sm, slots_per_thread, scan_tiles, waves),
            "dsoa_set_launch")
        if scan_tiles:
            self._scan_tiles = scan_tiles

    def set_flags(self, flags: int):
        _ok(load().dsoa_set_flags(self._h, flags), "dsoa_set_flags")
        self._flags = flags

    def separate_enumeration(self) -> bool:
        """True unless the do-alls enumerate inside their own kernels (the fused
        cooperative do-all or the streamed enumeration), i.e. when an up-front
        dsoa_enumerate_many serves the following enumerated do-alls."""
        return not (getattr(self, "_flags", 0) & FLAG_FUSED) and getattr(self, "_scan_tiles", 0) != 4

    def set_lookups(self, r: int):
        _ok(load().dsoa_set_lookups(self._h, r), "dsoa_set_lookups")

    def type_stats(self, t: int) -> dict:
        out = (ctypes.c_uint64 * 2)()
        _ok(load().dsoa_type_stats(self._h, t, out), "dsoa_type_stats")
        blocks, objs = int(out[0]), int(out[1])
        cap = self.capacity(t)
        frag = 1.0 - objs / (float(cap) * blocks) if blocks else 0.0
        return {"blocks": blocks, "objects": objs, "fragmentation": frag, "slots": cap * blocks}

    @property
    def launches(self) -> int:
        out = ctypes.c_uint64()
        _ok(load().dsoa_launch_count(self._h, ctypes.byref(out)), "dsoa_launch_count")
        return out.value

    def graph_begin(self):
        _ok(load().dsoa_graph_begin(self._h), "dsoa_graph_begin")

    def graph_end(self) -> Graph:
        g = ctypes.c_void_p()
        _ok(load().dsoa_graph_end(self._h, ctypes.byref(g)), "dsoa_graph_end")
        return Graph(g)

    def close(self):
        if self._h:
            load().dsoa_heap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BitmapHeap:
    """BitmapAlloc (dsoa_bitmap_heap): one array of equal-size AOS records managed by
    a free-slot bitmap and one allocation bitmap per type.  Offers the subset of
    ``Heap``'s methods that the microbench driver uses."""

    def __init__(self, nbytes: int, stream=None):
        self._h = ctypes.c_void_p()
        self.stream = stream
        _ok(load().dsoa_bitmap_heap_create(int(nbytes), _stream_ptr(stream), ctypes.byref(self._h)),
            "dsoa_bitmap_heap_create")

    def register_type(self, field_bytes) -> int:
        fb = (ctypes.c_uint32 * len(field_bytes))(*field_bytes)
        t = ctypes.c_int()
        _ok(load().dsoa_bitmap_register_type(self._h, fb, len(field_bytes), ctypes.byref(t)),
            "dsoa_bitmap_register_type")
        return t.value

    def freeze(self):
        _ok(load().dsoa_bitmap_heap_freeze(self._h), "dsoa_bitmap_heap_freeze")

    def info(self) -> dict:
        n, rb, nl = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
        _ok(load().dsoa_bitmap_heap_info(self._h, ctypes.byref(n), ctypes.byref(rb), ctypes.byref(nl)),
            "dsoa_bitmap_heap_info")
        return {"num_slots": n.value, "record_bytes": rb.value, "num_levels": nl.value}

    def parallel_new(self, t: int, n: int, ctor: int, args):
        _ok(load().dsoa_bitmap_parallel_new(self._h, t, n, ctor, ctypes.byref(args), ctypes.sizeof(args)),
            "dsoa_bitmap_parallel_new")

    def parallel_do(self, t: int, method: int, args):
        _ok(load().dsoa_bitmap_parallel_do(self._h, t, method, ctypes.byref(args), ctypes.sizeof(args)),
            "dsoa_bitmap_parallel_do")

    def count(self, t: int) -> int:
        out = ctypes.c_uint64()
        _ok(load().dsoa_bitmap_count(self._h, t, ctypes.byref(out)), "dsoa_bitmap_count")
        return out.value

    def get_error(self) -> int:
        out = ctypes.c_int()
        _ok(load().dsoa_bitmap_get_error(self._h, ctypes.byref(out)), "dsoa_bitmap_get_error")
        return out.value

    def check(self) -> dict:
        out = (ctypes.c_uint64 * 3)()
        _ok(load().dsoa_bitmap_check(self._h, out), "dsoa_bitmap_check")
        return {"hier": out[0], "free_xor": out[1], "tail": out[2]}

    def close(self):
        if self._h:
            load().dsoa_bitmap_heap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
