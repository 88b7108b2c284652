"""N>1 host path (replicas only), run as world_size-2 gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1810_11765_gb300.replicas import Replicas, rank_seed
    r = Replicas(backend="gloo")
    r.barrier()
    seconds = 1.0 + rank                       # rank 1 is the slow one
    rate = r.whole_job_rate(100.0, seconds)
    q.put((rank, rank_seed(1000, rank), r.max(float(rank)), rate))
    r.close()


def test_two_gloo_replicas_reduce_time_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = {o[1] for o in out}
    assert len(seeds) == world and 1000 in seeds          # independent replicas, rank 0 = base
    assert all(o[2] == 1.0 for o in out)                  # max over ranks seen by every rank
    assert all(o[3] == pytest.approx(2 * 100.0 / 2.0) for o in out)   # units of all ranks / slowest


def test_single_process_is_world_one():
    from paper_1810_11765_gb300.replicas import Replicas
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r = Replicas()
    assert r.world == 1 and r.max(3.5) == 3.5 and r.whole_job_rate(10, 2.0) == 5.0
    r.close()
