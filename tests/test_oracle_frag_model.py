"""Pins of the fragmentation model (oracle/frag_model.c): its Wa-Tor run is the
oracle's (same populations at every record), and its block accounting is exact
for each placement policy (F = 1 - objects / (64 x blocks) within [0, 1), and a
random choice among partly used blocks keeps at least as many blocks as first fit
on the same run)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("policy", ["first_fit", "best_fit", "random_fit", "hinted_random_fit",
                                    "hinted_random_fit_drain"])
@pytest.mark.parametrize("w,h,seed", [(64, 48, 3), (96, 96, 0x5EED0003)])
def test_populations_equal_the_oracle_run(policy, w, h, seed):
    steps, every = 60, 5
    fm = oracle.wator_frag(w, h, steps, seed, policy, every)
    _, st = oracle.wator_run(w, h, steps, seed=seed)
    for i, s in enumerate(fm["step"]):
        assert fm["fish"][i] == st[s - 1]["fish"] and fm["sharks"][i] == st[s - 1]["sharks"], (policy, s)
    live = fm["fish"].astype(np.int64) + fm["sharks"]
    assert np.all(fm["blocks"] * 64 >= live)
    assert np.allclose(fm["F"], 1 - live / (64.0 * fm["blocks"]))
    assert np.all((fm["F"] >= 0) & (fm["F"] < 1))


def test_random_fit_keeps_more_blocks_than_first_fit():
    a = oracle.wator_frag(128, 128, 200, 11, "first_fit", 50)
    b = oracle.wator_frag(128, 128, 200, 11, "random_fit", 50)
    assert np.array_equal(a["fish"], b["fish"])
    assert b["blocks"][-1] >= a["blocks"][-1]


def test_draining_keeps_no_more_blocks_than_the_hinted_policy_it_restricts():
    """Policy 4 is policy 3 with blocks that fell to 8 objects or fewer left out
    of every choice until they fill or empty: on the same run, fewer blocks stay
    in use once the first population wave has receded (both runs see the same
    populations)."""
    a = oracle.wator_frag(256, 256, 300, 11, "hinted_random_fit", 100)
    b = oracle.wator_frag(256, 256, 300, 11, "hinted_random_fit_drain", 100)
    assert np.array_equal(a["fish"], b["fish"]) and np.array_equal(a["sharks"], b["sharks"])
    assert b["blocks"][-1] <= a["blocks"][-1]
    assert b["F"][-1] <= a["F"][-1]
