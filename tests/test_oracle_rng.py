"""Pins of the oracle's counter-based generators to their published known answers."""
import os

import numpy as np

import oracle
from conftest import GOLDEN


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_philox4x32_known_answers():
    rows = _rows("philox4x32_kat.txt")
    assert len(rows) == 6
    for r in rows:
        rounds = int(r[0])
        vals = [int(x, 16) for x in r[1:]]
        out = oracle.philox4x32(vals[0:4], vals[4:6], rounds)
        assert [int(v) for v in out] == vals[6:10], r


def test_splitmix64_known_answers():
    rows = _rows("splitmix64_kat.txt")
    gamma = 0x9E3779B97F4A7C15
    for k, r in enumerate(rows):
        # output k+1 of the stream started at 0 is sm(state k*gamma)
        assert oracle.splitmix64((k * gamma) % 2**64) == int(r[0], 16)


def test_splitmix_composition():
    # sm2/sm3 are the nested compositions sm(sm(a)^b) and sm(sm2(a,b)^c)
    a, b, c = 0x5EED0001, 12345, 7
    assert oracle.sm2(a, b) == oracle.splitmix64(oracle.splitmix64(a) ^ b)
    assert oracle.sm3(a, b, c) == oracle.splitmix64(oracle.sm2(a, b) ^ c)


def test_philox_threshold_uniformity():
    # A u32 word compared with floor(p * 2^32) is a Bernoulli(p) draw; over 2^14
    # distinct counters the hit rate of p = 0.25 stays within 5 sigma.
    hits = 0
    n = 1 << 14
    for c in range(n):
        hits += int(oracle.philox4x32([0xFFFFFFFF, c, 0, 0], [1, 0])[0] < (1 << 30))
    sigma = np.sqrt(n * 0.25 * 0.75)
    assert abs(hits - n * 0.25) < 5 * sigma
