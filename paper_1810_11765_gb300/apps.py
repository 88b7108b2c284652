"""Workload drivers over the C ABI: microbench, game of life, wa-tor, traffic,
n-body and particle collisions.

Each driver only sequences library calls (``dsoa_parallel_new``, ``dsoa_parallel_do``,
``dsoa_run_kernel``) and owns the plain device arrays of its workload as torch
tensors (grids, handle maps, instance tables).  All per-object work runs in the
library's kernels on the heap's stream, which is the torch stream current when the
heap was created; torch work issued by the drivers stays on that stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import dsoa as D

INST_BYTES = ctypes.sizeof(D.Inst)


def _dev_u8(n, device):
    return torch.zeros(max(int(n), 1), dtype=torch.uint8, device=device)


def _grid_on_device(init, device):
    """An initial grid as a flat uint8 device tensor (host arrays are copied)."""
    if init is None:
        return None
    if isinstance(init, torch.Tensor):
        return init.to(device=device, dtype=torch.uint8).contiguous().view(-1)
    return torch.as_tensor(np.ascontiguousarray(init, dtype=np.uint8).reshape(-1)).to(device)


def _upload(dst: torch.Tensor, offset: int, raw: bytes):
    src = torch.frombuffer(bytearray(raw), dtype=torch.uint8)
    dst[offset:offset + len(raw)].copy_(src)


class InstanceTable:
    """Device table of ``dsoa_inst`` entries (one per instance slot)."""

    def __init__(self, capacity: int, device):
        self.capacity = capacity
        self.dev = _dev_u8(capacity * INST_BYTES, device)
        self.host = (D.Inst * capacity)()
        self.free = list(range(capacity - 1, -1, -1))

    @property
    def ptr(self) -> int:
        return self.dev.data_ptr()

    def put(self, slot: int):
        raw = bytes(memoryview(self.host).cast("B")[slot * INST_BYTES:(slot + 1) * INST_BYTES])
        _upload(self.dev, slot * INST_BYTES, raw)

    def set_state(self, slot: int, state: int):
        # only the 4-byte state word: the step counter t is owned by the device
        off = slot * INST_BYTES + D.Inst.state.offset
        self.host[slot].state = state
        _upload(self.dev, off, int(state).to_bytes(4, "little"))

    def read_t(self, slot: int) -> int:
        off = slot * INST_BYTES + D.Inst.t.offset
        return int(self.dev[off:off + 4].cpu().numpy().view(np.uint32)[0])


# ----------------------------------------------------------------------------- microbench
class Micro:
    """One type {int32 id, float x, int64 tag}; rounds of new / scale / delete.

    With ``sub_fields`` a subtype extending it by those fields is registered too,
    and every round creates its last ``sub_share`` of the objects (the highest
    ids) as subtype objects; the do-alls run on the base type and so cover both."""

    FIELDS = [4, 4, 8]

    def __init__(self, heap_bytes: int, seed: int, n_per_round: int, stream=None, heap=None,
                 sub_fields=None, sub_share: float = 0.5):
        self.heap = heap if heap is not None else D.Heap(heap_bytes, stream)
        self.type = self.heap.register_type(self.FIELDS)
        self.sub_type = None if sub_fields is None else self.heap.register_subtype(self.type, sub_fields)
        self.sub_share = sub_share
        self.heap.freeze()
        self.seed, self.n = seed, n_per_round
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._stats = torch.zeros(ctypes.sizeof(D.MicroStats), dtype=torch.uint8, device=self.device)

    def args(self, **kw) -> D.MicroArgs:
        a = D.MicroArgs(seed=self.seed)
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    def new(self, rnd: int, n: int | None = None):
        n = self.n if n is None else n
        n_sub = 0 if self.sub_type is None else int(n * self.sub_share)
        if n - n_sub:
            self.heap.parallel_new(self.type, n - n_sub, D.C_MICRO, self.args(id_base=rnd * self.n))
        if n_sub:
            self.heap.parallel_new(self.sub_type, n_sub, D.C_MICRO, self.args(id_base=rnd * self.n + n - n_sub))

    def scale(self, method: int = D.M_MICRO_SCALE):
        self.heap.parallel_do(self.type, method, self.args())

    def delete(self, rnd: int):
        self.heap.parallel_do(self.type, D.M_MICRO_DELETE, self.args(round=rnd))

    def round(self, rnd: int, method: int = D.M_MICRO_SCALE):
        self.new(rnd)
        self.scale(method)
        self.delete(rnd)

    def stats(self) -> dict:
        self._stats.zero_()
        self.heap.parallel_do(self.type, D.M_MICRO_STATS, self.args(stats=self._stats.data_ptr()))
        raw = bytes(self._stats.cpu().numpy())
        s = D.MicroStats.from_buffer_copy(raw)
        return {"live": s.live, "sum_id": s.sum_id, "sum_tag": s.sum_tag, "xor_tag": s.xor_tag,
                "sum_x": s.sum_x}

    def handles(self, n_ids: int) -> torch.Tensor:
        """Device tensor of the handle of every live object, indexed by id (0 = dead)."""
        out = torch.zeros(n_ids, dtype=torch.int64, device=self.device)
        self.heap.parallel_do(self.type, D.M_MICRO_HANDLES,
                              self.args(handles_out=out.data_ptr(), n_ids=n_ids))
        return out

    def gather(self, n_ids: int):
        x = torch.zeros(n_ids, dtype=torch.float32, device=self.device)
        live = torch.zeros(n_ids, dtype=torch.uint8, device=self.device)
        self.heap.parallel_do(self.type, D.M_MICRO_GATHER,
                              self.args(x_out=x.data_ptr(), live_out=live.data_ptr(), n_ids=n_ids))
        return x.cpu().numpy(), live.cpu().numpy()


# ----------------------------------------------------------------------------- game of life
class GolWorld:
    """Game of life instances in one heap: Cell per site, Alive per live cell."""

    CELL_FIELDS = [4, 4, 4, 1]   # inst, cell, count, alive
    ALIVE_FIELDS = [4, 4]        # inst, cell

    def __init__(self, heap: D.Heap, capacity: int = 1, types=None):
        self.heap = heap
        if types is None:
            self.cell_type = heap.register_type(self.CELL_FIELDS)
            self.alive_type = heap.register_type(self.ALIVE_FIELDS)
        else:
            self.cell_type, self.alive_type = types
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.table = InstanceTable(capacity, self.device)
        self.bufs = {}

    def args(self, target=0, init=None) -> D.GolArgs:
        return D.GolArgs(inst=self.table.ptr, init=D._addr(init), n_inst=self.table.capacity,
                         target=target, cell_type=self.cell_type, alive_type=self.alive_type)

    def add(self, w: int, h: int, seed: int, init=None) -> int:
        slot = self.table.free.pop()
        n = w * h
        cellmap = torch.zeros(n, dtype=torch.int64, device=self.device)
        occ = _dev_u8(n, self.device)
        self.bufs[slot] = (cellmap, occ)
        e = self.table.host[slot]
        e.cellmap, e.occ, e.claim, e.seed = cellmap.data_ptr(), occ.data_ptr(), None, seed
        e.w, e.h, e.t, e.state = w, h, 0, D.INST_RUN
        self.table.put(slot)
        ini = _grid_on_device(init, self.device)
        self.heap.parallel_new(self.cell_type, n, D.C_GOL_CELL, self.args(slot, ini))
        if ini is not None:
            self.bufs[slot] = (cellmap, occ, ini)   # keep alive until the kernel ran
        return slot

    batch_enumeration = True

    def step(self):
        """One generation.  Spread neither creates nor deletes Alive objects, so
        Reap runs on Spread's snapshot without enumerating again; Cells are never
        created or deleted during a generation, so their snapshot is taken at its
        start together with the Alive snapshot, in one enumeration launch."""
        a = self.args()
        batch = self.batch_enumeration and self.heap.separate_enumeration()
        if batch:
            self.heap.enumerate_many([self.alive_type, self.cell_type])
            self.heap.parallel_do_enumerated(self.alive_type, D.M_GOL_SPREAD, a)
        else:
            self.heap.parallel_do(self.alive_type, D.M_GOL_SPREAD, a)
        self.heap.parallel_do_enumerated(self.alive_type, D.M_GOL_REAP, a)
        # Decide also advances the instances' generation counters (CTA 0)
        if batch:
            self.heap.parallel_do_enumerated(self.cell_type, D.M_GOL_DECIDE_ADVANCE, a)
        else:
            self.heap.parallel_do(self.cell_type, D.M_GOL_DECIDE_ADVANCE, a)

    def read(self, slot: int) -> np.ndarray:
        self.heap.parallel_do(self.cell_type, D.M_GOL_READ, self.args())
        e = self.table.host[slot]
        return self.bufs[slot][1][:e.w * e.h].cpu().numpy().reshape(e.h, e.w)

    def alive_objects(self) -> int:
        return self.heap.count(self.alive_type)

    def remove(self, slot: int):
        self.table.set_state(slot, D.INST_KILL)
        a = self.args()
        self.heap.parallel_do(self.cell_type, D.M_GOL_KILL, a)
        self.heap.parallel_do(self.alive_type, D.M_GOL_KILL, a)
        self.table.set_state(slot, D.INST_IDLE)
        self.table.free.append(slot)
        self.bufs.pop(slot, None)


# ----------------------------------------------------------------------------- wa-tor
class WatorWorld:
    """Wa-Tor instances in one heap: Fish / Shark agents plus per-cell grids."""

    FISH_FIELDS = [4, 4, 4, 4]          # inst, cell, age, target
    SHARK_FIELDS = [4, 4, 4, 4, 4, 4]   # inst, cell, age, energy, target, eat

    def __init__(self, heap: D.Heap, capacity: int = 1, types=None):
        self.heap = heap
        if types is None:
            self.fish_type = heap.register_type(self.FISH_FIELDS)
            self.shark_type = heap.register_type(self.SHARK_FIELDS)
        else:
            self.fish_type, self.shark_type = types
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.table = InstanceTable(capacity, self.device)
        self.bufs = {}

    def args(self, target=0, init=None) -> D.WatorArgs:
        return D.WatorArgs(inst=self.table.ptr, init=D._addr(init), n_inst=self.table.capacity,
                           target=target, fish_type=self.fish_type, shark_type=self.shark_type)

    def add(self, w: int, h: int, seed: int, init=None, t0: int = 0) -> int:
        slot = self.table.free.pop()
        n = w * h
        cellmap = torch.zeros(n, dtype=torch.int64, device=self.device)
        occ = _dev_u8(n, self.device)
        claim = torch.full((n,), -1, dtype=torch.int32, device=self.device)
        ini = _grid_on_device(init, self.device)
        self.bufs[slot] = (cellmap, occ, claim, ini)
        e = self.table.host[slot]
        e.cellmap, e.occ, e.claim, e.seed = cellmap.data_ptr(), occ.data_ptr(), claim.data_ptr(), seed
        e.w, e.h, e.t, e.state = w, h, t0, D.INST_RUN
        self.table.put(slot)
        self.heap.run_kernel(D.K_WATOR_INIT, n, self.args(slot, ini))
        return slot

    batch_enumeration = True
    defer_births = False        # measured slower: the births kernel is an allocation burst

    def step(self):
        """One step.  The choose methods neither create nor delete agents of their
        own type, so each move method runs on its choose method's snapshot; and the
        fish methods neither create nor delete sharks, so the shark snapshot can be
        taken at the start of the step together with the fish snapshot, in one
        enumeration launch.  Newborn fish are created by the births kernel after
        Fish.move (``defer_births``) or inside it."""
        a = self.args()
        if self.batch_enumeration and self.heap.separate_enumeration():
            self.heap.enumerate_many([self.fish_type, self.shark_type])
            self.heap.parallel_do_enumerated(self.fish_type, D.M_WATOR_FISH_CHOOSE, a)
        else:
            self.heap.parallel_do(self.fish_type, D.M_WATOR_FISH_CHOOSE, a)
        if self.defer_births:
            self.heap.parallel_do_enumerated(self.fish_type, D.M_WATOR_FISH_MOVE_DEFER, a)
            self.heap.run_kernel(D.K_WATOR_BIRTHS, self.table.capacity, a)
        else:
            self.heap.parallel_do_enumerated(self.fish_type, D.M_WATOR_FISH_MOVE, a)
        if self.batch_enumeration and self.heap.separate_enumeration():
            self.heap.parallel_do_enumerated(self.shark_type, D.M_WATOR_SHARK_CHOOSE, a)
        else:
            self.heap.parallel_do(self.shark_type, D.M_WATOR_SHARK_CHOOSE, a)
        # Shark.move also advances the instances' step counters (CTA 0)
        self.heap.parallel_do_enumerated(self.shark_type, D.M_WATOR_SHARK_MOVE_ADVANCE, a)

    def read(self, slot: int) -> np.ndarray:
        e = self.table.host[slot]
        return self.bufs[slot][1][:e.w * e.h].cpu().numpy().reshape(e.h, e.w)

    def counts(self):
        return self.heap.count(self.fish_type), self.heap.count(self.shark_type)

    def remove(self, slot: int):
        self.table.set_state(slot, D.INST_KILL)
        a = self.args()
        self.heap.parallel_do(self.fish_type, D.M_WATOR_KILL, a)
        self.heap.parallel_do(self.shark_type, D.M_WATOR_KILL, a)
        self.table.set_state(slot, D.INST_IDLE)
        self.table.free.append(slot)
        self.bufs.pop(slot, None)


# ----------------------------------------------------------------------------- traffic
SLOW_THR = 858993459     # floor(0.20 * 2^32)
RAMP_THR = 214748364     # floor(0.05 * 2^32)


class TrafficWorld:
    """Batched Nagel-Schreckenberg rings; Car {ring, pos, v} objects."""

    CAR_FIELDS = [4, 4, 4]

    def __init__(self, heap: D.Heap, L, thr, seed: int, slow_thr: int = SLOW_THR,
                 ramp_thr: int = RAMP_THR, car_type=None, init_occ=None, init_v=None):
        self.heap = heap
        self.car_type = heap.register_type(self.CAR_FIELDS) if car_type is None else car_type
        self.device = torch.device("cuda", torch.cuda.current_device())
        L = np.asarray(L, dtype=np.uint64)
        self.L = L
        base = np.zeros(L.size + 1, dtype=np.uint64)
        base[1:] = np.cumsum(L)
        self.total = int(base[-1])
        self.base_host = base
        self.ring_base = torch.as_tensor(base.astype(np.int64)).to(self.device)
        self.ring_thr = torch.as_tensor(np.asarray(thr, dtype=np.uint32).view(np.int32)).to(self.device)
        self.occ0 = _dev_u8(self.total, self.device)
        self.occ1 = _dev_u8(self.total, self.device)
        self.vel = _dev_u8(self.total, self.device)
        self.t_dev = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._init = [None if x is None else torch.as_tensor(np.ascontiguousarray(x, dtype=np.uint8)).to(self.device)
                      for x in (init_occ, init_v)]
        self.a = D.TrafficArgs(occ0=self.occ0.data_ptr(), occ1=self.occ1.data_ptr(), vel_out=self.vel.data_ptr(),
                               ring_base=self.ring_base.data_ptr(), ring_thr=self.ring_thr.data_ptr(),
                               init_occ=D._addr(self._init[0]), init_v=D._addr(self._init[1]),
                               t_dev=self.t_dev.data_ptr(), seed=seed, n_rings=int(L.size),
                               slow_thr=slow_thr, ramp_thr=ramp_thr, car_type=self.car_type)
        self.steps_done = 0

    def init(self):
        self.heap.run_kernel(D.K_TRAFFIC_INIT, self.total, self.a)

    def step(self):
        self.heap.run_kernel(D.K_TRAFFIC_CLEAR, self.total, self.a)
        self.heap.parallel_do(self.car_type, D.M_TRAFFIC_MOVE, self.a)
        self.heap.run_kernel(D.K_TRAFFIC_ONRAMP_ADVANCE, int(self.L.size), self.a)
        self.steps_done += 1

    def read(self):
        """(occupancy, speed) per cell, both uint8[total]."""
        self.vel.zero_()
        self.heap.parallel_do(self.car_type, D.M_TRAFFIC_READ, self.a)
        t = int(self.t_dev.cpu().numpy()[0])
        occ = self.occ1 if (t & 1) else self.occ0
        return occ[:self.total].cpu().numpy(), self.vel[:self.total].cpu().numpy()


# ----------------------------------------------------------------------------- n-body
class NBodyWorld:
    """n-body (``collide=False``: FORCE, MOVE) or particle collisions (FORCE, MOVE,
    FIND, CLAIM, MERGE, DELETE) over one Body type.  ``tiled`` selects the pairwise
    shared-memory FORCE kernel instead of the per-thread device_do walk (same
    integers); ``all_pairs`` makes that kernel evaluate every ordered pair instead
    of every unordered pair once (same integers again)."""

    BODY_FIELDS = [4, 4, 4, 4, 4, 4, 8, 8, 4, 4, 4]   # id px py vx vy m fx fy target incoming merged

    def __init__(self, heap: D.Heap, cfg, collide: bool = False, tiled: bool = True, body_type=None,
                 all_pairs: bool = False):
        self.heap = heap
        self.cfg = cfg
        self.collide = collide
        self.tiled = tiled
        self.pair_flags = D.NBODY_ALL_PAIRS if all_pairs else 0
        self.force_method = D.M_NBODY_FORCE_TILED if tiled else D.M_NBODY_FORCE
        self.type = heap.register_type(self.BODY_FIELDS) if body_type is None else body_type
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.n = 0
        self.handle_of = None
        self._init = None

    def args(self, **kw) -> D.NBodyArgs:
        c = self.cfg
        a = D.NBodyArgs(handle_of=D._addr(self.handle_of), seed=c.seed, n_ids=self.n,
                        mass_max=c.mass_max, G=c.G, dt=c.dt, eps2=c.eps2, rc2=c.rc2,
                        fscale=c.fscale, vscale=c.vscale, body_type=self.type,
                        flags=self.pair_flags | (D.NBODY_KEYED_FIND if (self.collide and self.tiled) else 0))
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    def create(self, n: int, init=None):
        """parallel_new<Body>(n): ids 0..n-1, from ``init`` (n x 5 floats) or the seed."""
        self.n = n
        self.handle_of = torch.zeros(max(n, 1), dtype=torch.int64, device=self.device)
        self._init = None
        if init is not None:
            self._init = torch.as_tensor(np.ascontiguousarray(init, dtype=np.float32).reshape(-1)).to(self.device)
        self.heap.parallel_new(self.type, n, D.C_NBODY, self.args(init=D._addr(self._init)))

    def step(self):
        """One step: a single enumeration, every other do-all on its snapshot (no
        Body is created during a step; DELETE only deletes itself)."""
        a = self.args()
        self.heap.parallel_do(self.type, self.force_method, a)
        self.heap.parallel_do_enumerated(self.type, D.M_NBODY_MOVE, a)
        if self.collide:
            find = D.M_COLL_FIND_TILED if self.tiled else D.M_COLL_FIND
            for m in (find, D.M_COLL_CLAIM, D.M_COLL_MERGE, D.M_COLL_DELETE):
                self.heap.parallel_do_enumerated(self.type, m, a)

    def force(self):
        """FORCE alone (adds the pair sums to the force fields, which MOVE clears)."""
        self.heap.parallel_do(self.type, self.force_method, self.args(flags=self.pair_flags))

    def read(self, forces: bool = False):
        """(state float32[n, 5] by id: px py vx vy m, alive uint8[n]) and, with
        ``forces``, the fixed-point forces int64[n, 2]."""
        out = torch.zeros(max(self.n, 1) * 5, dtype=torch.float32, device=self.device)
        alive = torch.zeros(max(self.n, 1), dtype=torch.uint8, device=self.device)
        fo = torch.zeros(max(self.n, 1) * 2, dtype=torch.int64, device=self.device) if forces else None
        self.heap.parallel_do(self.type, D.M_NBODY_READ,
                              self.args(out=out.data_ptr(), alive_out=alive.data_ptr(), force_out=D._addr(fo)))
        res = (out.view(-1, 5)[:self.n].cpu().numpy(), alive[:self.n].cpu().numpy())
        if forces:
            res += (fo.view(-1, 2)[:self.n].cpu().numpy(),)
        return res

    def count(self) -> int:
        return self.heap.count(self.type)
