"""Pins of the oracle's Game of Life (Cell per site + Alive agent per live cell)."""
import os

import numpy as np
import pytest

import oracle
from conftest import GOLDEN


def load_patterns():
    pats = {}
    with open(os.path.join(GOLDEN, "gol_patterns.txt")) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("# ")]
    i = 0
    while i < len(lines):
        ln = lines[i].split()
        if ln and ln[0] == "pattern":
            name, period, dx, dy = ln[1], int(ln[3]), int(ln[5]), int(ln[7])
            rows = []
            i += 1
            while lines[i].strip() != "end":
                rows.append([1 if ch == "#" else 0 for ch in lines[i].strip()])
                i += 1
            pats[name] = (np.array(rows, dtype=np.uint8), period, dx, dy)
        i += 1
    return pats


PATTERNS = load_patterns()


def place(pat, w, h, x0, y0):
    g = np.zeros((h, w), dtype=np.uint8)
    ph, pw = pat.shape
    g[y0:y0 + ph, x0:x0 + pw] = pat
    return g


def conway_numpy(g, gens):
    """Textbook B3/S23 on a torus via an 8-neighbour roll sum."""
    g = g.astype(np.uint8)
    for _ in range(gens):
        n = sum(np.roll(np.roll(g, dy, 0), dx, 1)
                for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0))
        g = ((n == 3) | ((g == 1) & (n == 2))).astype(np.uint8)
    return g


@pytest.mark.parametrize("name", ["blinker", "block", "beehive", "toad"])
def test_oscillators_and_still_lifes(name):
    pat, period, _, _ = PATTERNS[name]
    g0 = place(pat, 16, 12, 5, 3)
    for k in (1, 2, 3):
        out, alive, objs = oracle.gol_run(16, 12, period * k, init=g0)
        assert np.array_equal(out, g0)
        assert np.array_equal(alive, objs)
    if period == 2:
        mid, _, _ = oracle.gol_run(16, 12, 1, init=g0)
        assert not np.array_equal(mid, g0)


def test_glider_moves_one_diagonal_cell_per_four_generations():
    pat, period, dx, dy = PATTERNS["glider"]
    w, h = 20, 20
    g0 = place(pat, w, h, 2, 2)
    for k in (1, 2, 10):   # 10 periods wrap the glider twice around the 20-torus
        out, alive, objs = oracle.gol_run(w, h, period * k, init=g0)
        assert np.array_equal(out, np.roll(np.roll(g0, dy * k, 0), dx * k, 1))
        assert np.all(alive[::period] == 5)
        assert np.array_equal(alive, objs)


@pytest.mark.parametrize("w,h,gens,seed", [(8, 8, 30, 1), (17, 13, 40, 2), (32, 32, 60, 3),
                                           (3, 3, 10, 4), (1, 5, 5, 5)])
def test_random_grids_match_textbook_rule(w, h, gens, seed):
    rng = np.random.default_rng(seed)
    g0 = (rng.random((h, w)) < 0.35).astype(np.uint8)
    out, alive, objs = oracle.gol_run(w, h, gens, init=g0)
    ref = g0
    for g in range(gens + 1):
        if g > 0:
            ref = conway_numpy(ref, 1)
        assert alive[g] == ref.sum()
    assert np.array_equal(out, ref)
    assert np.array_equal(alive, objs)


def test_seeded_initial_density():
    # initial state: Philox word < 2^30, i.e. Bernoulli(1/4) per cell
    g, alive, _ = oracle.gol_run(256, 256, 0, seed=0x5EED0002)
    n = 256 * 256
    assert abs(int(g.sum()) - n / 4) < 5 * np.sqrt(n * 3 / 16)
    assert alive[0] == g.sum()


def test_order_independence():
    a = oracle.gol_run(48, 40, 25, seed=7)
    for os_ in (3, 11):
        b = oracle.gol_run(48, 40, 25, seed=7, order_seed=os_)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
