"""Continuous batching: instances admitted while others run, stepped by shared launches.

Each finished instance must equal an oracle run of that instance alone, and the same
request served alone must give the same grid as in the mix.
"""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    gpu_ready()


def serve(reqs, heap_bytes=256 << 20, capacity=8, time_scale=1.0):
    import torch
    from paper_1810_11765_gb300.serving import Server
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        srv = Server(heap_bytes, capacity)
        fin, summary = srv.run(reqs, time_scale=time_scale)
        srv.close()
    return {f.rid: f for f in fin}, summary


def oracle_grid(f):
    if f.kind == "gol":
        return oracle.gol_run(f.side, f.side, f.steps, seed=f.seed)[0]
    return oracle.wator_run(f.side, f.side, f.steps, seed=f.seed)[0]


def test_mixed_stream_matches_oracle_alone():
    from paper_1810_11765_gb300 import inputs
    reqs = inputs.serving_requests(14, rate_per_s=400.0, side_log2_min=4, side_log2_max=6,
                                   steps_min=5, steps_max=40, seed=123)
    fin, summary = serve(reqs, capacity=4)
    assert summary["device_errors"] == 0
    assert len(fin) == len(reqs)
    for f in fin.values():
        assert np.array_equal(f.grid, oracle_grid(f)), (f.rid, f.kind, f.side, f.steps)
        assert f.done_s >= f.admitted_s >= 0
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0


def test_alone_equals_in_the_mix():
    from paper_1810_11765_gb300 import inputs
    reqs = inputs.serving_requests(8, rate_per_s=1000.0, side_log2_min=4, side_log2_max=5.5,
                                   steps_min=10, steps_max=30, seed=7)
    mixed, _ = serve(reqs, capacity=8)
    for q in reqs[:3]:
        alone, _ = serve([q], capacity=1)
        assert np.array_equal(alone[q.rid].grid, mixed[q.rid].grid)


def test_admission_waits_for_blocks():
    """A heap too small for all requests at once: later requests wait until earlier
    instances finish and free their blocks; all still complete correctly."""
    from paper_1810_11765_gb300 import inputs
    reqs = [inputs.Request(i, "wator" if i % 2 else "gol", 48, 12 + i, 1000 + i, 0.0) for i in range(6)]
    fin, summary = serve(reqs, heap_bytes=512 << 10, capacity=6)
    assert summary["device_errors"] == 0
    assert len(fin) == 6
    for f in fin.values():
        assert np.array_equal(f.grid, oracle_grid(f))


def test_configured_stream_sampled():
    """The configured serving stream (24 requests, half game of life and half
    Wa-Tor, sides 2^U(8,12), 100-1000 steps, 64 GiB heap), all arriving at once:
    the three cheapest instances equal the oracle alone, and the largest equals a
    GPU run of it alone."""
    from paper_1810_11765_gb300 import inputs
    reqs = inputs.serving_requests(24, rate_per_s=1e9)
    mixed, summary = serve(reqs, heap_bytes=64 << 30, capacity=32)
    assert summary["device_errors"] == 0 and len(mixed) == 24
    assert max(q.side for q in reqs) > 2048
    for q in sorted(reqs, key=lambda q: q.side * q.side * q.steps)[:3]:
        f = mixed[q.rid]
        assert np.array_equal(f.grid, oracle_grid(f)), (f.rid, f.kind, f.side, f.steps)
    big = max(reqs, key=lambda q: q.side)
    alone, _ = serve([big], heap_bytes=64 << 30, capacity=1)
    assert np.array_equal(alone[big.rid].grid, mixed[big.rid].grid)
