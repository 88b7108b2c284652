"""Pins of the oracle's Wa-Tor (Fish / Shark agents on a torus).

The paper only sketches Wa-Tor (Table 1); the rules are the readings stated in the
oracle source.  These tests pin them with hand-derived cases on tiny tori, where
the random choice is forced (one candidate), with conservation laws and with
order independence.
"""
import numpy as np
import pytest

import oracle

EMPTY, FISH, SHARK = 0, 1, 2


def test_lone_fish_breeds_on_its_third_move():
    g = np.zeros((32, 32), np.uint8)
    g[10, 10] = FISH
    _, st = oracle.wator_run(32, 32, 3, init=g)
    assert [s["fish"] for s in st] == [1, 1, 2]
    assert [s["fish_births"] for s in st] == [0, 0, 1]


def test_lone_shark_starves_after_three_steps():
    g = np.zeros((32, 32), np.uint8)
    g[5, 7] = SHARK
    out, st = oracle.wator_run(32, 32, 4, init=g)
    assert [s["sharks"] for s in st] == [1, 1, 0, 0]
    assert st[2]["starved"] == 1
    assert out.sum() == 0


def test_shark_eats_forced_fish_then_starves():
    # 1x3 torus (N and S of a cell are the cell itself).  Fish at 1 can only move
    # east to 2; then the shark at 0 sees the fish at 2 (its west neighbour) and
    # eats it.  With energy refilled to 3 it survives steps 1, 2 and starves at 3.
    g = np.array([[SHARK, FISH, EMPTY]], np.uint8)
    out, st = oracle.wator_run(3, 1, 1, init=g)
    assert out.tolist() == [[EMPTY, EMPTY, SHARK]]
    assert st[0]["eaten"] == 1 and st[0]["fish"] == 0
    _, st = oracle.wator_run(3, 1, 5, init=g)
    assert [s["sharks"] for s in st] == [1, 1, 1, 0, 0]


def test_claim_conflict_lowest_source_wins():
    # 1x3 torus, fish at 0 and 2 both can only move into cell 1; the fish from
    # cell 0 (lower index) wins, the one at 2 stays.
    g = np.array([[FISH, EMPTY, FISH]], np.uint8)
    out, st = oracle.wator_run(3, 1, 1, init=g)
    assert out.tolist() == [[EMPTY, FISH, FISH]]
    assert st[0]["fish_moves"] == 1


def test_full_fish_grid_is_frozen():
    g = np.full((3, 3), FISH, np.uint8)
    out, st = oracle.wator_run(3, 3, 12, init=g)
    assert np.array_equal(out, g)
    assert all(s["fish"] == 9 and s["fish_births"] == 0 for s in st)


@pytest.mark.parametrize("w,h,steps,seed", [(4, 4, 40, 1), (5, 5, 60, 2), (64, 48, 80, 3)])
def test_conservation_and_grid_consistency(w, h, steps, seed):
    g0, _ = oracle.wator_run(w, h, 0, seed=seed)
    fish, sharks = int((g0 == FISH).sum()), int((g0 == SHARK).sum())
    out, st = oracle.wator_run(w, h, steps, seed=seed)
    for s in st:
        fish = fish + s["fish_births"] - s["eaten"]
        sharks = sharks + s["shark_births"] - s["starved"]
        assert (s["fish"], s["sharks"]) == (fish, sharks)
        assert s["fish_births"] <= s["fish_moves"] and s["shark_births"] <= s["shark_moves"]
        assert s["eaten"] <= s["shark_moves"]
    assert int((out == FISH).sum()) == fish and int((out == SHARK).sum()) == sharks


def test_initial_densities():
    g, _ = oracle.wator_run(256, 256, 0, seed=0x5EED0003)
    n = 256 * 256
    nf, ns = int((g == FISH).sum()), int((g == SHARK).sum())
    assert abs(nf - 0.30 * n) < 5 * np.sqrt(n * 0.3 * 0.7)
    assert abs(ns - 0.05 * n) < 5 * np.sqrt(n * 0.05 * 0.95)


def test_order_independence():
    a = oracle.wator_run(40, 30, 30, seed=9)
    for os_ in (5, 77):
        b = oracle.wator_run(40, 30, 30, seed=9, order_seed=os_)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1]


def test_step_offset_is_the_philox_step_index():
    # running 10 steps then 10 more from the resulting grid is not the same as
    # 20 steps (ages and energies restart), but the first step of a run with
    # t0 = k must use the Philox counters of step k: two runs from the same grid
    # with different t0 differ.
    a, _ = oracle.wator_run(32, 32, 1, seed=4, t0=0)
    b, _ = oracle.wator_run(32, 32, 1, seed=4, t0=1)
    assert not np.array_equal(a, b)
