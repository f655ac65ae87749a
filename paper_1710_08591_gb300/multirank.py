"""Multi-GPU bookkeeping of the FFT-beam path: one process per GPU, each owning its own
band of frequency channels (channels are independent, Section 3.2: beams are formed per
frequency), so there is no data-path exchange. The only collective is the timing
aggregate: the job's time is the slowest rank's and its work is the sum over ranks.
"""
from __future__ import annotations


def channel_band(nfreq_per_rank: int, rank: int) -> tuple[int, int]:
    """(first channel, channel count) of `rank`'s band under weak scaling."""
    if nfreq_per_rank < 1 or rank < 0:
        raise ValueError("need nfreq_per_rank >= 1 and rank >= 0")
    return rank * nfreq_per_rank, nfreq_per_rank


def band_seed(base_seed: int, rank: int) -> int:
    """Seed of the synthetic voltages of `rank`'s band (distinct data per band)."""
    return base_seed + 1000 * rank


def aggregate(local_ms: float, local_samples: int, device=None) -> tuple[float, int]:
    """(max over ranks of the timed region in ms, total antenna-samples over ranks).

    Without an initialised process group this is the local pair."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms), int(local_samples)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([int(local_samples)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def throughput(max_ms: float, total_samples: int) -> float:
    """Whole-job antenna-samples per second."""
    return total_samples / (max_ms / 1e3)
