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


def _splitmix64_py(z):
    """SplitMix64's output for state z (the finaliser: add the golden gamma, then
    xor-shift-multiply twice and a final xor-shift), in Python integers, written
    apart from the oracle's C so that the two check each other."""
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_splitmix_python_restatement_matches_the_known_answers_and_the_oracle():
    """The Python finaliser reproduces the published stream (so it is pinned
    independently of the oracle), and the oracle's sm, sm2 and sm3 equal it and
    its compositions on seeded inputs, among them the microbench tags
    sm2(seed, id) of ids at round boundaries."""
    rows = _rows("splitmix64_kat.txt")
    gamma = 0x9E3779B97F4A7C15
    for k, r in enumerate(rows):
        assert _splitmix64_py((k * gamma) % 2**64) == int(r[0], 16)
    rng = np.random.default_rng(0x5EED0005)
    cases = [(0x5EED0001, i) for i in (0, 1, (1 << 18) - 1, 1 << 18, 9 * (1 << 18) + 5)]
    cases += [(int(x), int(y)) for x, y in rng.integers(0, 2**63, size=(16, 2), dtype=np.int64)]
    for a, b in cases:
        want2 = _splitmix64_py(_splitmix64_py(a) ^ b)
        assert oracle.splitmix64(a) == _splitmix64_py(a)
        assert oracle.sm2(a, b) == want2
        for c in (0, 3, 9):
            assert oracle.sm3(a, b, c) == _splitmix64_py(want2 ^ c)


def test_philox_threshold_uniformity():
    # A u32 word compared with floor(p * 2^32) is a Bernoulli(p) draw; over 2^14
    # distinct counters the hit rate of p = 0.25 stays within 5 sigma.
    hits = 0
    n = 1 << 14
    for c in range(n):
        hits += int(oracle.philox4x32([0xFFFFFFFF, c, 0, 0], [1, 0])[0] < (1 << 30))
    sigma = np.sqrt(n * 0.25 * 0.75)
    assert abs(hits - n * 0.25) < 5 * sigma
