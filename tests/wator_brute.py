"""An independent, cell-indexed restatement of one Wa-Tor run, for pinning the oracle.

The oracle (``orc_wator_run``) keeps Fish and Shark objects in free-list stores and
visits them in snapshot order.  This module keeps no objects at all: it holds the
world as three per-cell arrays (kind, age, energy) and applies the rules of Table 1
"wa-tor" (Dewdney's predator-prey on a torus) phase by phase, with the readings the
oracle states:

* von Neumann neighbourhood visited N, E, S, W (y grows southwards);
* a mover lists its candidate cells in that order and takes candidate
  ``w0 mod k``, where ``w0`` is word 0 of Philox4x32-10 keyed by the seed
  (low word first) at counter (t, cell, 1, 0) for fish and (t, cell, 2, 0) for
  sharks;
* the lowest source cell wins a contested target;
* every agent of the phase's snapshot ages by one, movers or not; a mover whose
  age reached 3 (fish) or 10 (sharks) leaves a newborn of age 0 behind and
  restarts at 0;
* a shark prefers cells holding fish, refills its energy to 3 when it eats and
  otherwise loses one, and is removed when its energy reaches 0;
* the initial grid draws ``u = w0`` at counter (0xFFFFFFFF, cell, 0, 0):
  u < floor(0.30 * 2^32) fish, else u < floor(0.35 * 2^32) shark, else empty.

Philox itself comes from ``oracle.philox4x32``, which the published Random123
known-answer vectors pin.  Pure Python loops: for tori of a few dozen cells.
"""
from __future__ import annotations

import numpy as np

import oracle

EMPTY, FISH, SHARK = 0, 1, 2
FISH_BREED, SHARK_BREED, SHARK_ENERGY = 3, 10, 3
FISH_THR, SHARK_THR = 1288490188, 1503238553


def draw(seed: int, c0: int, c1: int, c2: int) -> int:
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return int(oracle.philox4x32([c0 & 0xFFFFFFFF, c1, c2, 0], key)[0])


def neighbours(c: int, w: int, h: int):
    x, y = c % w, c // w
    return [((y - 1) % h) * w + x,      # N
            y * w + (x + 1) % w,        # E
            ((y + 1) % h) * w + x,      # S
            y * w + (x - 1) % w]        # W


def initial_grid(w: int, h: int, seed: int) -> np.ndarray:
    g = np.zeros(w * h, np.uint8)
    for c in range(w * h):
        u = draw(seed, 0xFFFFFFFF, c, 0)
        g[c] = FISH if u < FISH_THR else (SHARK if u < SHARK_THR else EMPTY)
    return g


def run(w: int, h: int, steps: int, seed: int, init=None, t0: int = 0):
    """Returns (final grid uint8[h, w], per-step dicts with the oracle's stat keys)."""
    n = w * h
    kind = initial_grid(w, h, seed) if init is None else np.asarray(init, np.uint8).reshape(-1).copy()
    age = np.zeros(n, np.int64)
    energy = np.where(kind == SHARK, SHARK_ENERGY, 0).astype(np.int64)
    stats = []
    for step in range(steps):
        t = t0 + step
        ev = dict(fish_births=0, shark_births=0, eaten=0, starved=0, fish_moves=0, shark_moves=0)

        # fish: choices on the grid at the start of the phase, then the winners move
        movers = [c for c in range(n) if kind[c] == FISH]
        target, best = {}, {}
        for c in movers:
            cand = [d for d in neighbours(c, w, h) if kind[d] == EMPTY]
            if cand:
                tg = cand[draw(seed, t, c, 1) % len(cand)]
                target[c] = tg
                best[tg] = min(best.get(tg, n), c)
        for c in movers:
            a = age[c] + 1
            tg = target.get(c)
            if tg is None or best[tg] != c:
                age[c] = a
                continue
            ev["fish_moves"] += 1
            kind[tg] = FISH
            if a >= FISH_BREED:
                age[tg] = 0
                age[c] = 0                      # the newborn stays behind
                ev["fish_births"] += 1
            else:
                age[tg] = a
                kind[c] = EMPTY
                age[c] = 0

        # sharks: fish neighbours first, else empty ones
        movers = [c for c in range(n) if kind[c] == SHARK]
        target, best, eats = {}, {}, {}
        for c in movers:
            nb = neighbours(c, w, h)
            cand = [d for d in nb if kind[d] == FISH]
            eats[c] = bool(cand)
            if not cand:
                cand = [d for d in nb if kind[d] == EMPTY]
            if cand:
                tg = cand[draw(seed, t, c, 2) % len(cand)]
                target[c] = tg
                best[tg] = min(best.get(tg, n), c)
        for c in movers:
            a, e = age[c] + 1, energy[c]
            tg = target.get(c)
            here = c
            if tg is not None and best[tg] == c:
                ev["shark_moves"] += 1
                if eats[c]:
                    assert kind[tg] == FISH
                    ev["eaten"] += 1
                    e = SHARK_ENERGY
                else:
                    e -= 1
                kind[tg] = SHARK
                here = tg
                if a >= SHARK_BREED:
                    a = 0
                    age[c], energy[c] = 0, SHARK_ENERGY   # the newborn stays behind
                    ev["shark_births"] += 1
                else:
                    kind[c] = EMPTY
                    age[c], energy[c] = 0, 0
            else:
                e -= 1
            age[here], energy[here] = a, e
            if e == 0:
                kind[here] = EMPTY
                age[here] = energy[here] = 0
                ev["starved"] += 1
        ev["fish"] = int((kind == FISH).sum())
        ev["sharks"] = int((kind == SHARK).sum())
        stats.append(ev)
    return kind.reshape(h, w).copy(), stats
