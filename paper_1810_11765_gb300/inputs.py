"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method: it only draws workload parameters
(ring lengths, densities, arrival times, instance sizes and seeds) with numpy's
seeded generator, so that both sides consume identical inputs.  The random numbers
that the workloads themselves draw (Philox4x32 / SplitMix64 keyed by logical ids)
are implemented independently on each side.

Workload recipe (shapes follow the paper's applications, Table 1 and Sec. 6):
  * microbench: 2^18 new per round, 10 rounds, 16-byte objects, 64 MiB heap
  * game of life: 512 x 512 torus, density 1/4, 200 generations
  * wa-tor: 1024 x 1024 torus, 30 % fish / 5 % sharks, 500 steps
  * traffic: 64 rings, length floor(2^(12 + 8u)), density U(0.1, 0.3), 1000 steps
  * n-body / collisions: 65,536 bodies in [-1, 1)^2, integer masses 1..16
  * serving: Poisson arrivals of game-of-life / wa-tor instances, side
    2^U(8, 12), U(100, 1000) steps
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 0x5EED0001

SEED_MICRO = SEED_BASE + 0
SEED_GOL = SEED_BASE + 1
SEED_WATOR = SEED_BASE + 2
SEED_TRAFFIC = SEED_BASE + 3
SEED_SERVING = SEED_BASE + 4
SEED_NBODY = SEED_BASE + 5
SEED_COLLISION = SEED_BASE + 6


@dataclass(frozen=True)
class MicroConfig:
    n_per_round: int = 1 << 18
    rounds: int = 10
    heap_bytes: int = 64 << 20
    seed: int = SEED_MICRO


@dataclass(frozen=True)
class GolConfig:
    width: int = 512
    height: int = 512
    gens: int = 200
    seed: int = SEED_GOL


@dataclass(frozen=True)
class NBodyConfig:
    """n-body / collision parameters (the paper gives none; 65,536 bodies as in its
    n-body listing).  G and fscale are powers of two."""
    n: int = 1 << 16
    steps: int = 10
    G: float = 2.0 ** -30
    dt: float = 0.25
    eps2: float = 2.0 ** -18
    rc2: float = 2.0 ** -18
    fscale: float = 2.0 ** 40
    vscale: float = 2.0 ** -8
    mass_max: int = 16
    seed: int = SEED_NBODY


@dataclass(frozen=True)
class WatorConfig:
    width: int = 1024
    height: int = 1024
    steps: int = 500
    seed: int = SEED_WATOR


def traffic_instances(n_inst: int = 64, log2_min: float = 12.0, log2_max: float = 20.0,
                      dens_min: float = 0.1, dens_max: float = 0.3,
                      seed: int = SEED_TRAFFIC):
    """Ring lengths L_i = floor(2^(log2_min + (log2_max-log2_min) u)) and density
    thresholds thr_i = floor(d_i * 2^32), d_i ~ U(dens_min, dens_max).
    Returns (L uint32[n], thr uint32[n])."""
    rng = np.random.default_rng(seed)
    u = rng.random(n_inst)
    L = np.floor(2.0 ** (log2_min + (log2_max - log2_min) * u)).astype(np.uint32)
    d = dens_min + (dens_max - dens_min) * rng.random(n_inst)
    thr = np.floor(d * 2.0 ** 32).astype(np.uint64).clip(0, 2**32 - 1).astype(np.uint32)
    return L, thr


@dataclass(frozen=True)
class Request:
    rid: int
    kind: str          # "gol" or "wator"
    side: int
    steps: int
    seed: int
    arrival_s: float


def serving_requests(n_req: int, rate_per_s: float, side_log2_min: float = 8.0,
                     side_log2_max: float = 12.0, steps_min: int = 100,
                     steps_max: int = 1000, seed: int = SEED_SERVING):
    """Poisson arrivals (exponential gaps of mean 1/rate), kind 50/50, side
    round(2^U(min,max)), steps U{min..max}, per-request seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_req)
    t = np.cumsum(gaps) - gaps[0]
    kinds = rng.random(n_req) < 0.5
    sides = np.rint(2.0 ** rng.uniform(side_log2_min, side_log2_max, n_req)).astype(np.int64)
    steps = rng.integers(steps_min, steps_max + 1, n_req)
    seeds = rng.integers(1, 2**63 - 1, n_req, dtype=np.int64)
    return [Request(i, "gol" if kinds[i] else "wator", int(sides[i]), int(steps[i]),
                    int(seeds[i]), float(t[i])) for i in range(n_req)]
