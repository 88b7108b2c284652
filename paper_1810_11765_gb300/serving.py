"""Continuous-batching server for simulation instances on one shared device heap.

Requests (game-of-life or wa-tor instances of different sizes and step counts) arrive
over time.  Admitted instances live as objects in one heap and are all advanced by
the same launches: one *tick* = one step of every running instance (game-of-life
spread / reap / decide + wa-tor fish and shark choose / move), replayed as one
captured CUDA graph whose kernels read the device instance tables, so admissions and
removals between ticks need no re-capture.  A request is admitted as soon as an
instance slot is free and the heap can hold it: the free-block count is read from the
device's free-block bitmap every tick (asynchronously, into pinned memory) and compared
with the blocks the request needs plus the growth still promised to running
instances.  A finished instance's grid is copied out and its objects are deleted
(KILL do-alls), which returns its blocks to the free bitmap for the next admissions.

Every instance's random numbers are keyed by its own seed and its own step index, so
its result is the same alone and in any mix.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np
import torch

from . import dsoa as D
from .apps import GolWorld, WatorWorld


@dataclasses.dataclass
class Running:
    req: object
    kind: str
    slot: int
    need: int
    steps_done: int = 0
    admitted_s: float = 0.0


@dataclasses.dataclass
class Finished:
    rid: int
    kind: str
    side: int
    steps: int
    seed: int
    arrival_s: float
    admitted_s: float
    done_s: float
    grid: np.ndarray

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def blocks_needed(kind: str, side: int) -> int:
    """Conservative blocks for an instance of side x side cells: game of life = one
    Cell per site + Alive agents for up to half the sites; wa-tor = agents for every
    site (fish can fill the torus when sharks die out) + 25 % for partly filled blocks."""
    n = side * side
    if kind == "gol":
        return math.ceil(n / 64) + math.ceil(n / 128) + 64
    return math.ceil(1.25 * n / 64) + 64


class Server:
    def __init__(self, heap_bytes: int = 64 << 30, capacity: int = 64, max_inflight_ticks: int = 2):
        self.stream = torch.cuda.current_stream()
        if self.stream.cuda_stream == 0:
            raise RuntimeError("Server needs a non-default current stream (CUDA graph capture)")
        self.heap = D.Heap(heap_bytes)
        self.gol = GolWorld(self.heap, capacity)
        self.wator = WatorWorld(self.heap, capacity)
        self.heap.freeze()
        self.total_blocks = self.heap.info()["num_blocks"]
        dev = torch.device("cuda", torch.cuda.current_device())
        self.free_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        self.free_host = torch.zeros(1, dtype=torch.int64).pin_memory()
        self.free_event = None
        self.free_latest = self.total_blocks
        self.max_inflight = max_inflight_ticks
        self.inflight = collections.deque()
        # one tick = one step of every running instance of both kinds
        self.heap.graph_begin()
        self.gol.step()
        self.wator.step()
        self.tick_graph = self.heap.graph_end()
        self.running: list[Running] = []
        self.ticks = 0
        self.instance_steps = 0

    # ------------------------------------------------------------------ admission
    def _poll_free_blocks(self):
        if self.free_event is not None and self.free_event.query():
            self.free_latest = int(self.free_host[0])
            self.free_event = None
        if self.free_event is None:
            self.heap.free_blocks_async(self.free_dev)
            self.free_host.copy_(self.free_dev, non_blocking=True)
            self.free_event = torch.cuda.Event()
            self.free_event.record()

    def can_admit(self, kind: str, side: int) -> bool:
        world = self.gol if kind == "gol" else self.wator
        if not world.table.free:
            return False
        need = blocks_needed(kind, side)
        used = self.total_blocks - self.free_latest
        promised = max(0, sum(r.need for r in self.running) - used)
        return self.free_latest - promised >= need

    def admit(self, req, now_s: float):
        world = self.gol if req.kind == "gol" else self.wator
        slot = world.add(req.side, req.side, req.seed)
        self.running.append(Running(req, req.kind, slot, blocks_needed(req.kind, req.side), 0, now_s))

    # ------------------------------------------------------------------ stepping
    def tick(self):
        self.tick_graph.launch()
        ev = torch.cuda.Event()
        ev.record()
        self.inflight.append(ev)
        while len(self.inflight) > self.max_inflight:
            self.inflight.popleft().synchronize()
        self.ticks += 1
        for r in self.running:
            r.steps_done += 1
        self.instance_steps += len(self.running)

    def _finish(self, r: Running, t0: float) -> Finished:
        world = self.gol if r.kind == "gol" else self.wator
        world.table.set_state(r.slot, D.INST_IDLE)          # stops stepping at the next tick
        grid = world.read(r.slot)                            # synchronises the stream
        world.remove(r.slot)
        q = r.req
        return Finished(q.rid, q.kind, q.side, q.steps, q.seed, q.arrival_s, r.admitted_s,
                        time.perf_counter() - t0, grid)

    def run(self, requests, time_scale: float = 1.0, poll_sleep_s: float = 1e-4):
        """Serve `requests` (inputs.Request, sorted by arrival); arrival times are
        multiplied by time_scale.  Returns (finished list, summary dict)."""
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival_s))
        rejected = [q for q in pending if blocks_needed(q.kind, q.side) > self.total_blocks]
        for q in rejected:
            pending.remove(q)      # can never fit in this heap
        finished = []
        t0 = time.perf_counter()
        while pending or self.running:
            now = time.perf_counter() - t0
            self._poll_free_blocks()
            while pending and pending[0].arrival_s * time_scale <= now and \
                    self.can_admit(pending[0].kind, pending[0].side):
                q = pending.popleft()
                self.admit(q, now)
                self.free_latest -= blocks_needed(q.kind, q.side)   # until the next device read
            if self.running:
                self.tick()
                done = [r for r in self.running if r.steps_done >= r.req.steps]
                for r in done:
                    self.running.remove(r)
                    f = self._finish(r, t0)
                    f.arrival_s *= time_scale
                    finished.append(f)
            elif pending:
                wait = pending[0].arrival_s * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
                else:
                    time.sleep(poll_sleep_s)   # waiting for blocks to be freed
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        lat = np.array([f.latency_s for f in finished]) if finished else np.zeros(1)
        summary = {"requests": len(finished), "rejected": [q.rid for q in rejected],
                   "wall_s": wall, "ticks": self.ticks,
                   "instance_steps": self.instance_steps,
                   "instance_steps_per_s": self.instance_steps / wall if wall else 0.0,
                   "ticks_per_s": self.ticks / wall if wall else 0.0,
                   "p50_latency_s": float(np.percentile(lat, 50)),
                   "p99_latency_s": float(np.percentile(lat, 99)),
                   "device_errors": self.heap.get_error()}
        return finished, summary

    def close(self):
        self.tick_graph.close()
        self.heap.close()
