"""Pins of the oracle's Wa-Tor choice rule, draw layout and breeding against an
independent cell-indexed brute force (``wator_brute.py``) and hand-derived picks.

The paper only sketches Wa-Tor (Table 1); the readings both sides follow are listed
in ``wator_brute``.  Philox4x32-10 is pinned separately by its published
known-answer vectors, so every expected pick below follows from those vectors and
the stated rule alone.
"""
import numpy as np
import pytest

import oracle
import wator_brute as wb

EMPTY, FISH, SHARK = wb.EMPTY, wb.FISH, wb.SHARK


def _same(w, h, steps, seed, init=None, t0=0):
    a, sa = oracle.wator_run(w, h, steps, seed=seed, init=init, t0=t0)
    b, sb = wb.run(w, h, steps, seed, init=init, t0=t0)
    assert np.array_equal(a, b)
    for k, (x, y) in enumerate(zip(sa, sb)):
        assert x == y, (k, x, y)
    return sa


def _dense(w, h, seed, p_fish, p_shark):
    rng = np.random.default_rng(seed)
    u = rng.random(w * h)
    return np.where(u < p_fish, FISH, np.where(u < p_fish + p_shark, SHARK, EMPTY)).astype(np.uint8)


@pytest.mark.parametrize("w,h,seed", [(4, 4, 11), (4, 4, 12), (5, 5, 13), (5, 5, 14), (5, 4, 15)])
def test_drawn_grids_match_brute_force(w, h, seed):
    _same(w, h, 60, seed)


def test_runs_where_sharks_breed_match_brute_force():
    # fish-rich 5x5 / 6x5 tori: sharks keep eating long enough to reach age 10
    births = 0
    for k, (w, h) in enumerate([(5, 5), (5, 5), (6, 5), (6, 6), (5, 5), (6, 5)]):
        init = _dense(w, h, 100 + k, 0.75, 0.12)
        st = _same(w, h, 80, 0x5EED0003 + k, init=init)
        births += sum(s["shark_births"] for s in st)
    assert births > 0


def test_high_seed_words_and_step_offset_match_brute_force():
    _same(5, 5, 40, 0xDEADBEEF_12345678, init=_dense(5, 5, 7, 0.6, 0.1), t0=1000)


def test_initial_grid_cells_follow_the_draw_layout():
    for seed in (0x5EED0003, 0x1234_0000_0000_0001):
        g, _ = oracle.wator_run(9, 7, 0, seed=seed)
        assert np.array_equal(g.reshape(-1), wb.initial_grid(9, 7, seed))
    # a few cells by hand from the Philox words
    seed = 0x5EED0003
    g, _ = oracle.wator_run(64, 64, 0, seed=seed)
    for c in (0, 1, 63, 64, 2047, 4095):
        u = int(oracle.philox4x32([0xFFFFFFFF, c, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[0])
        want = FISH if u < 1288490188 else (SHARK if u < 1503238553 else EMPTY)
        assert g.reshape(-1)[c] == want


def test_game_of_life_initial_cells_follow_the_draw_layout():
    seed = 0x5EED0002
    g, alive, _ = oracle.gol_run(32, 16, 0, seed=seed)
    flat = g.reshape(-1)
    for c in range(0, 32 * 16, 7):
        u = int(oracle.philox4x32([0xFFFFFFFF, c, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[0])
        assert flat[c] == (1 if u < (1 << 30) else 0)
    assert alive[0] == int(flat.sum())


def _pick(seed, t, cell, stream, cands):
    u = int(oracle.philox4x32([t, cell, stream, 0], [seed & 0xFFFFFFFF, seed >> 32])[0])
    return cands[u % len(cands)]


@pytest.mark.parametrize("seed", [1, 2, 3, 0x5EED0003])
def test_lone_fish_with_four_candidates(seed):
    w = h = 7
    c = 3 * w + 3
    g = np.zeros(w * h, np.uint8)
    g[c] = FISH
    out, st = oracle.wator_run(w, h, 1, seed=seed, init=g, t0=5)
    want = _pick(seed, 5, c, 1, [c - w, c + 1, c + w, c - 1])     # N, E, S, W
    assert out.reshape(-1)[want] == FISH and int(out.sum()) == FISH
    assert st[0]["fish_moves"] == 1


@pytest.mark.parametrize("seed", [4, 5, 6, 7])
def test_fish_with_three_candidates_and_shark_with_four(seed):
    # a shark south of the fish removes S from the fish's candidates; the fish
    # then sits on a cell that is not next to the shark, whose four neighbours
    # are all empty
    w = h = 7
    c = 3 * w + 3
    s = c + w
    g = np.zeros(w * h, np.uint8)
    g[c], g[s] = FISH, SHARK
    out, st = oracle.wator_run(w, h, 1, seed=seed, init=g)
    fish_to = _pick(seed, 0, c, 1, [c - w, c + 1, c - 1])          # N, E, W
    shark_to = _pick(seed, 0, s, 2, [s - w, s + 1, s + w, s - 1])  # N (= c, vacated), E, S, W
    flat = out.reshape(-1)
    assert flat[fish_to] == FISH and flat[shark_to] == SHARK
    assert int((flat != EMPTY).sum()) == 2 and st[0]["eaten"] == 0


@pytest.mark.parametrize("seed", [8, 9, 10, 11])
def test_fish_on_a_ring_has_two_candidates(seed):
    # 7x1 torus: N and S of a cell are the cell itself (occupied), so E and W remain
    g = np.zeros(7, np.uint8)
    g[2] = FISH
    out, _ = oracle.wator_run(7, 1, 1, seed=seed, init=g, t0=3)
    assert out.reshape(-1)[_pick(seed, 3, 2, 1, [3, 1])] == FISH


@pytest.mark.parametrize("seed", [12, 13, 14])
def test_shark_among_four_fish(seed):
    # a shark inside a torus full of fish: no fish can move, the shark eats one of four
    w = h = 5
    g = np.full(w * h, FISH, np.uint8)
    c = 2 * w + 2
    g[c] = SHARK
    out, st = oracle.wator_run(w, h, 1, seed=seed, init=g)
    to = _pick(seed, 0, c, 2, [c - w, c + 1, c + w, c - 1])
    flat = out.reshape(-1)
    assert flat[to] == SHARK and flat[c] == EMPTY
    assert st[0]["eaten"] == 1 and st[0]["fish"] == w * h - 2


@pytest.mark.parametrize("seed", [15, 16, 17, 18])
def test_shark_between_two_fish_and_two_sharks(seed):
    # torus full of fish (none can move) with sharks at c, N of c and E of c: the
    # shark at c lists only its S and W fish; its targets are nobody else's
    w = h = 6
    c = 3 * w + 3
    g = np.full(w * h, FISH, np.uint8)
    g[c] = g[c - w] = g[c + 1] = SHARK
    out, st = oracle.wator_run(w, h, 1, seed=seed, init=g)
    to = _pick(seed, 0, c, 2, [c + w, c - 1])                      # S, W
    flat = out.reshape(-1)
    assert flat[to] == SHARK and flat[c] == EMPTY
    _same(w, h, 1, seed, init=g)


def test_shark_that_eats_every_step_breeds_on_its_tenth_move():
    # a shark inside a torus packed with fish always has a fish neighbour, so it
    # eats on every step and never starves; it breeds on its 10th move
    w = h = 20
    g = np.full(w * h, FISH, np.uint8)
    g[10 * w + 10] = SHARK
    _, st = oracle.wator_run(w, h, 12, seed=42, init=g)
    assert all(s["eaten"] == 1 for s in st[:10])
    assert [s["shark_births"] for s in st[:10]] == [0] * 9 + [1]
    assert [s["sharks"] for s in st[:10]] == [1] * 9 + [2]
    _same(w, h, 12, 42, init=g)


def test_contested_ring_hand_case():
    # 5x1 ring [F, _, F, F, F] (N and S of a cell are the cell itself).  Step 1:
    # fish 0 (east) and fish 2 (west) both want cell 1, the lower source 0 wins.
    # Step 2: fish 1 and fish 4 both want cell 0, fish 1 wins.  Step 3: fish 0
    # and fish 2 want cell 1, fish 0 wins on its third move and leaves a newborn:
    # the ring is full and stays frozen.
    g = np.array([FISH, EMPTY, FISH, FISH, FISH], np.uint8)
    out, st = oracle.wator_run(5, 1, 5, seed=3, init=g)
    assert [s["fish"] for s in st] == [4, 4, 5, 5, 5]
    assert [s["fish_moves"] for s in st] == [1, 1, 1, 0, 0]
    assert [s["fish_births"] for s in st] == [0, 0, 1, 0, 0]
    assert out.reshape(-1).tolist() == [FISH] * 5
    _same(5, 1, 5, 3, init=g)


def test_contested_ring_with_sharks_matches_brute_force():
    _same(7, 1, 12, 21, init=np.array([SHARK, FISH, EMPTY, FISH, SHARK, SHARK, SHARK], np.uint8))
