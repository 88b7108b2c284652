"""Pins of the oracle's allocator microbench (one type {int32 id, float x, int64 tag})."""
import numpy as np
import pytest

import oracle

SEED = 0x5EED0001


def test_expected_live_counts_closed_form():
    # Each live object survives a round with probability 1/2 (a splitmix64 parity),
    # so after round r the expected live count is n * (1 - 2^-(r+1)).
    n, rounds = 1 << 16, 6
    rows, _, _ = oracle.micro_run(SEED, n, rounds)
    for r, row in enumerate(rows):
        expect = n * (1 - 2.0 ** -(r + 1))
        # variance of a sum of independent survivals is below n * (r+1) / 4
        assert abs(row["live"] - expect) < 6 * np.sqrt(n * (r + 1) / 4), (r, row)
        assert row["news"] == n
    # conservation: live = sum(news) - sum(deletes)
    live = 0
    for row in rows:
        live += row["news"] - row["deletes"]
        assert row["live"] == live


def test_x_is_exact_recurrence_within_fp32_bound():
    # In exact arithmetic k applications of x <- 1.5 x + id from x = 0 give
    # x_k = 2 id (1.5^k - 1).  fp32 with one rounding per operation stays within
    # 2k unit roundoffs (relative) of it.
    n, rounds = 4096, 8
    _, x, live = oracle.micro_run(SEED, n, rounds, per_object=True)
    ids = np.arange(n * rounds)
    born = ids // n
    k = rounds - born
    exact = 2.0 * ids * (1.5 ** k - 1.0)
    sel = live.astype(bool) & (ids > 0)
    rel = np.abs(x[sel].astype(np.float64) - exact[sel]) / exact[sel]
    assert sel.sum() > n
    assert np.all(rel <= 2 * k[sel] * 2.0 ** -24)
    # per-operation IEEE single rounding, evaluated with numpy's float32 ops
    ref = np.zeros(n * rounds, dtype=np.float32)
    for r in range(rounds):
        m = born <= r
        ref[m] = (ref[m] * np.float32(1.5)) + ids[m].astype(np.float32)
    assert np.array_equal(x[live.astype(bool)], ref[live.astype(bool)])


def test_survival_set_follows_parity_rule():
    n, rounds = 2048, 5
    _, _, live = oracle.micro_run(SEED, n, rounds, per_object=True)
    for gid in range(0, n * rounds, 37):
        born = gid // n
        alive = all((oracle.sm3(SEED, gid, r) & 1) == 0 for r in range(born, rounds))
        assert bool(live[gid]) == alive


def test_round_sums_match_per_object_state():
    n, rounds = 1000, 4
    rows, x, live = oracle.micro_run(SEED, n, rounds, per_object=True)
    ids = np.nonzero(live)[0]
    last = rows[-1]
    assert last["live"] == ids.size
    assert last["sum_id"] == int(ids.sum())
    tags = [oracle.sm2(SEED, int(i)) for i in ids]
    assert last["sum_tag"] == sum(tags) % 2**64
    xor = 0
    for t in tags:
        xor ^= t
    assert last["xor_tag"] == xor
    assert last["sum_x"] == pytest.approx(float(x[ids].astype(np.float64).sum()), rel=1e-12)


def test_order_independence():
    n, rounds = 3000, 4
    a = oracle.micro_run(SEED, n, rounds, per_object=True)
    for os_ in (1, 99):
        b = oracle.micro_run(SEED, n, rounds, order_seed=os_, per_object=True)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        for ra, rb in zip(a[0], b[0]):
            assert ra["live"] == rb["live"] and ra["sum_id"] == rb["sum_id"]
            assert ra["xor_tag"] == rb["xor_tag"]


def test_empty_round():
    rows, _, _ = oracle.micro_run(SEED, 0, 3)
    assert all(r["live"] == 0 for r in rows)
