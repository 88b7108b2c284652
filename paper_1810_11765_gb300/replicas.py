"""Multi-GPU policy of the runtime: replicas only.

The SMMO hot path does not shard: a heap lives on one GPU and every do-all runs over
that heap's blocks.  N GPUs run N independent instances (one heap per rank, per-rank
seeds), with no collective on the data path; the host only synchronises ranks around
the timed region and reduces timings (max over ranks) -- weak scaling.  Launched one
process per GPU by torchrun (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* in the
environment); ``backend`` is "nccl" on GPUs and "gloo" for host-only runs and tests.
"""
from __future__ import annotations

import os


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the replica on `rank` (rank 0 runs the configured seed itself)."""
    return base_seed + 7919 * rank


class Replicas:
    def __init__(self, backend: str | None = None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.backend = backend
        if self.world > 1:
            import torch
            import torch.distributed as dist
            be = backend or ("nccl" if torch.cuda.is_available() else "gloo")
            self.backend = be
            if be == "nccl":
                torch.cuda.set_device(self.local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        """Max of a host float over ranks (timings: the slowest rank decides)."""
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def whole_job_rate(self, units_per_rank: float, seconds_this_rank: float) -> float:
        """Units processed by all ranks / max over ranks of the time."""
        return self.world * units_per_rank / self.max(seconds_this_rank)

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()
            self.pg = None
