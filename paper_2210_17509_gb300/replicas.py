"""Independent replicas across ranks (one process per GPU).

The method shards by blocks; on this path the blocks of different ranks never
exchange data, so N ranks run N independent replicas.  The only cross-rank
operations are the benchmark's barrier and the maximum of the per-rank timed
durations (the slowest rank sets the whole-job time).  Works with NCCL on GPUs
and with gloo on CPU (used by the tests).
"""
from __future__ import annotations

import os

import torch


class Replicas:
    def __init__(self, backend: str | None = None, device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.device = device
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                kw = {}
                if backend == "nccl" and device is not None:
                    kw["device_id"] = device
                dist.init_process_group(backend or "gloo", **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, value: float) -> float:
        if self.dist is None:
            return float(value)
        dev = self.device if self.device is not None else torch.device("cpu")
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank: float, ms_max: float) -> float:
        """Whole-job throughput: all ranks' units over the slowest rank's time."""
        return self.world * units_per_rank / (ms_max * 1e-3)

    @property
    def is_root(self) -> bool:
        return self.rank == 0
