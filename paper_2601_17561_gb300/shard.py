"""Weak-scaling shards of the matching job, one rank per GPU.

The CCMM is independent per database row (Section 6.2.3 splits the database in slices across
GPUs), so the job shards by database with no collective on the data path: rank r holds its own
encrypted database shard -- its own MSRLWE database, whose a-part stream is keyed by chunk id r --
and every rank matches the same query batch.  The job's rate is all ranks' comparisons over the
slowest rank's time.  (A deployment would all-gather the query operand once per batch; here every
rank encrypts the same seeded batch.)

The cleartext folding check shards by trial: Philox counters are keyed by the trial index, so
consecutive trial ranges on the ranks are together exactly the single run's trials.
"""
from __future__ import annotations

import torch

from . import synth


def shard_workload(rank: int, n_eyes: int, n_db: int, seed: int = 2, planted_frac: float = 0.05):
    """(rank's database workload, the common query workload).  Database templates are drawn from
    seed + 1000 rank; the queries (and eye ids) from `seed` alone, so every rank sees the same
    batch."""
    W = synth.make_workload(n_eyes=n_eyes, n_db=n_db, seed=seed + 1000 * rank, planted_frac=planted_frac)
    Wq = W if rank == 0 else synth.make_workload(n_eyes=n_eyes, n_db=0, seed=seed)
    return W, Wq


def chunk_id(rank: int) -> int:
    """Chunk id of rank's database: keys its a-part randomness apart from other ranks'."""
    return rank


def job_time_ms(local_ms: float, dist=None, device=None) -> float:
    """The job's time: the maximum of the ranks' times (all-reduce MAX when a process group of
    more than one rank is initialised)."""
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, comparisons_per_rank: int, job_ms: float) -> float:
    """Whole-job comparisons per second (weak scaling: every rank processes its own shard)."""
    return world * comparisons_per_rank / (job_ms / 1e3)


def trial_range(rank: int, world: int, n_trials: int) -> tuple[int, int]:
    """(first trial, number of trials) of rank's share of a run of n_trials trials: consecutive
    ranges, the first n_trials % world ranks one trial longer."""
    base, extra = divmod(int(n_trials), int(world))
    return rank * base + min(rank, extra), base + (1 if rank < extra else 0)


def job_sum(t: torch.Tensor, dist=None) -> torch.Tensor:
    """Counters summed over the ranks (all-reduce SUM when a process group of more than one rank
    is initialised), for reporting."""
    t = t.clone()
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
