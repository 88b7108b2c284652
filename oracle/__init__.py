"""Sequential CPU oracle for the SMMO runtime (DynaSOAr, Springer & Masuhara, ECOOP 2019).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1810_11765_gb300``) and never
imports it.

The C source (``dsoa_oracle.c``) states, per function, the passage it follows and the
pins that check it.  This module only compiles it with gcc and marshals numpy arrays
through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsoa_oracle.c")
_SRC_FRAG = os.path.join(_HERE, "frag_model.c")
_HDR = os.path.join(_HERE, "dsoa_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (plain C11, no fp contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_FRAG), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wextra", "-o", tmp, _SRC, _SRC_FRAG, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class MicroRound(ctypes.Structure):
    _fields_ = [("live", ctypes.c_uint64), ("sum_id", ctypes.c_int64),
                ("sum_tag", ctypes.c_uint64), ("xor_tag", ctypes.c_uint64),
                ("sum_x", ctypes.c_double), ("news", ctypes.c_uint64),
                ("deletes", ctypes.c_uint64)]


class NBodyParams(ctypes.Structure):
    _fields_ = [("G", ctypes.c_float), ("dt", ctypes.c_float), ("eps2", ctypes.c_float),
                ("rc2", ctypes.c_float), ("fscale", ctypes.c_float), ("vscale", ctypes.c_float),
                ("mass_max", ctypes.c_uint32), ("collide", ctypes.c_uint32)]


class WatorStep(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("fish", "sharks", "fish_births", "shark_births", "eaten", "starved",
                 "fish_moves", "shark_moves")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
            lib.orc_philox4x32.argtypes = [P, P, i32, P]
            lib.orc_philox4x32.restype = None
            lib.orc_splitmix64.argtypes = [u64]
            lib.orc_splitmix64.restype = u64
            lib.orc_sm2.argtypes = [u64, u64]
            lib.orc_sm2.restype = u64
            lib.orc_sm3.argtypes = [u64, u64, u64]
            lib.orc_sm3.restype = u64
            lib.orc_micro_run.argtypes = [u64, u32, u32, u64, P, P, P]
            lib.orc_micro_run.restype = i32
            lib.orc_gol_run.argtypes = [u32, u32, P, u64, u32, u64, P, P, P]
            lib.orc_gol_run.restype = i32
            lib.orc_wator_run.argtypes = [u32, u32, P, u64, u32, u32, u64, P, P]
            lib.orc_wator_run.restype = i32
            lib.orc_wator_frag.argtypes = [u32, u32, u64, u32, i32, u32, P, P, P, P]
            lib.orc_wator_frag.restype = i32
            lib.orc_traffic_run.argtypes = [u32, u32, P, P, u64, u32, u32, u32, P, P, u64,
                                            P, P, P]
            lib.orc_traffic_run.restype = i32
            lib.orc_nbody_run.argtypes = [u32, P, u64, P, u32, u64, P, P, P, P]
            lib.orc_nbody_run.restype = i32
            lib.orc_nbody_force_on.argtypes = [u32, P, P, P, u32, P]
            lib.orc_nbody_force_on.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32(_ptr(c), _ptr(k), rounds, _ptr(out))
    return out


def splitmix64(state: int) -> int:
    return int(_load().orc_splitmix64(state & (2**64 - 1)))


def sm2(a: int, b: int) -> int:
    return int(_load().orc_sm2(a & (2**64 - 1), b & (2**64 - 1)))


def sm3(a: int, b: int, c: int) -> int:
    return int(_load().orc_sm3(a & (2**64 - 1), b & (2**64 - 1), c & (2**64 - 1)))


def micro_run(seed: int, n_per_round: int, rounds: int, order_seed: int = 0,
              per_object: bool = False):
    """Microbench rounds.  Returns (list of per-round dicts, x_by_id, live_by_id)."""
    stats = (MicroRound * rounds)()
    total = n_per_round * rounds
    x = np.zeros(total, dtype=np.float32) if per_object else None
    live = np.zeros(total, dtype=np.uint8) if per_object else None
    rc = _load().orc_micro_run(seed, n_per_round, rounds, order_seed,
                               ctypes.cast(stats, ctypes.c_void_p), _ptr(x), _ptr(live))
    if rc != 0:
        raise RuntimeError("oracle microbench failed")
    rows = [{f: getattr(s, f) for f, _ in MicroRound._fields_} for s in stats]
    return rows, x, live


def gol_run(w: int, h: int, gens: int, seed: int = 0, init=None, order_seed: int = 0):
    """Game of Life.  Returns (final grid uint8[h,w], alive counts[gens+1], Alive objects[gens+1])."""
    ini = None if init is None else np.ascontiguousarray(np.asarray(init, dtype=np.uint8).reshape(-1))
    grid = np.zeros(w * h, dtype=np.uint8)
    alive = np.zeros(gens + 1, dtype=np.uint32)
    objs = np.zeros(gens + 1, dtype=np.uint32)
    rc = _load().orc_gol_run(w, h, _ptr(ini), seed, gens, order_seed, _ptr(grid),
                             _ptr(alive), _ptr(objs))
    if rc != 0:
        raise RuntimeError("oracle game of life failed")
    return grid.reshape(h, w), alive, objs


def wator_run(w: int, h: int, steps: int, seed: int = 0, init=None, t0: int = 0,
              order_seed: int = 0):
    """Wa-Tor.  Returns (final grid uint8[h,w], list of per-step dicts)."""
    ini = None if init is None else np.ascontiguousarray(np.asarray(init, dtype=np.uint8).reshape(-1))
    grid = np.zeros(w * h, dtype=np.uint8)
    stats = (WatorStep * max(steps, 1))()
    rc = _load().orc_wator_run(w, h, _ptr(ini), seed, steps, t0, order_seed, _ptr(grid),
                               ctypes.cast(stats, ctypes.c_void_p))
    if rc != 0:
        raise RuntimeError("oracle wa-tor failed")
    rows = [{f: getattr(s, f) for f, _ in WatorStep._fields_} for s in stats[:steps]]
    return grid.reshape(h, w), rows


FRAG_POLICIES = {"first_fit": 0, "best_fit": 1, "random_fit": 2, "hinted_random_fit": 3,
                 "hinted_random_fit_drain": 4}


def wator_frag(w: int, h: int, steps: int, seed: int, policy: str = "first_fit", every: int = 25):
    """Fragmentation of an idealised sequential allocator (frag_model.c) on the
    Wa-Tor run: dict of arrays F, fish, sharks, blocks, one entry per `every` steps."""
    k = steps // every
    F = np.zeros(max(k, 1), dtype=np.float64)
    fish, sharks, blocks = (np.zeros(max(k, 1), dtype=np.uint32) for _ in range(3))
    rc = _load().orc_wator_frag(w, h, seed, steps, FRAG_POLICIES[policy], every, _ptr(F), _ptr(fish),
                                _ptr(sharks), _ptr(blocks))
    if rc != 0:
        raise RuntimeError("oracle fragmentation model failed")
    return {"step": np.arange(1, k + 1) * every, "F": F[:k], "fish": fish[:k], "sharks": sharks[:k],
            "blocks": blocks[:k]}


SLOW_THR = 858993459     # floor(0.20 * 2^32)
RAMP_THR = 214748364     # floor(0.05 * 2^32)


def traffic_run(L, thr, steps: int, seed: int = 0, slow_thr: int = SLOW_THR,
                ramp_thr: int = RAMP_THR, init_occ=None, init_v=None, order_seed: int = 0,
                first_ring: int = 0):
    """Batched Nagel-Schreckenberg rings.  Returns (occ[sum L], v[sum L], cars[(steps+1), n]).
    ``first_ring`` is the batch index of ring 0 (to replay one ring of a batch alone)."""
    Ls = np.ascontiguousarray(np.asarray(L, dtype=np.uint32))
    ths = np.ascontiguousarray(np.asarray(thr, dtype=np.uint32))
    n = Ls.size
    total = int(Ls.astype(np.uint64).sum())
    io = None if init_occ is None else np.ascontiguousarray(np.asarray(init_occ, dtype=np.uint8))
    iv = None if init_v is None else np.ascontiguousarray(np.asarray(init_v, dtype=np.uint8))
    occ = np.zeros(total, dtype=np.uint8)
    v = np.zeros(total, dtype=np.uint8)
    cars = np.zeros((steps + 1, n), dtype=np.uint32)
    rc = _load().orc_traffic_run(n, first_ring, _ptr(Ls), _ptr(ths), seed, steps, slow_thr, ramp_thr,
                                 _ptr(io), _ptr(iv), order_seed, _ptr(occ), _ptr(v), _ptr(cars))
    if rc != 0:
        raise RuntimeError("oracle traffic failed")
    return occ, v, cars


def nbody_run(n: int, steps: int, seed: int = 0, *, G: float, dt: float, eps2: float,
              rc2: float = 0.0, fscale: float = 2.0 ** 40, vscale: float = 2.0 ** -8,
              mass_max: int = 16, collide: bool = False, init=None, order_seed: int = 0):
    """N-body (collide=False) or particle collisions.  Returns (state float32[n,5] by id:
    px, py, vx, vy, m; alive uint8[n]; counts uint32[steps+1]; force sums int64[steps,2])."""
    prm = NBodyParams(G, dt, eps2, rc2, fscale, vscale, mass_max, 1 if collide else 0)
    ini = None if init is None else np.ascontiguousarray(np.asarray(init, dtype=np.float32).reshape(n, 5))
    out = np.zeros((max(n, 1), 5), dtype=np.float32)
    alive = np.zeros(max(n, 1), dtype=np.uint8)
    counts = np.zeros(steps + 1, dtype=np.uint32)
    fsum = np.zeros((max(steps, 1), 2), dtype=np.int64)
    rc = _load().orc_nbody_run(n, _ptr(ini), seed, ctypes.byref(prm), steps, order_seed,
                               _ptr(out), _ptr(alive), _ptr(counts), _ptr(fsum))
    if rc != 0:
        raise RuntimeError("oracle n-body failed")
    return out[:n], alive[:n], counts, fsum[:steps]


def nbody_force_on(state, ids, alive=None, *, G: float, eps2: float, fscale: float = 2.0 ** 40):
    """Fixed-point forces int64[len(ids), 2] of one FORCE do-all on the bodies ``ids``
    of ``state`` (float32[n, 5]), from every other (alive) body."""
    st = np.ascontiguousarray(np.asarray(state, dtype=np.float32))
    n = st.shape[0]
    al = None if alive is None else np.ascontiguousarray(np.asarray(alive, dtype=np.uint8))
    prm = NBodyParams(G, 1.0, eps2, 0.0, fscale, 0.0, 1, 0)
    out = np.zeros((len(ids), 2), dtype=np.int64)
    row = np.zeros(2, dtype=np.int64)
    for k, i in enumerate(ids):
        if _load().orc_nbody_force_on(n, _ptr(st), _ptr(al), ctypes.byref(prm), int(i), _ptr(row)) != 0:
            raise RuntimeError("oracle n-body force failed")
        out[k] = row
    return out
