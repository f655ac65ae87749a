"""The N>1 path of bench.py on CPU: two gloo ranks with their own channel bands; the job
time is the slowest rank's and the work is summed (no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1710_08591_gb300 import multirank  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f0, nf = multirank.channel_band(1024, rank)
        local_ms = 100.0 + 50.0 * rank                  # rank 1 is the slow one
        local_samples = 384 * nf * 2 * 1024
        mx, total = multirank.aggregate(local_ms, local_samples)
        out.put((rank, f0, nf, mx, total, multirank.band_seed(2, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, f00, nf0, mx0, tot0, s0), (r1, f01, nf1, mx1, tot1, s1) = res
    assert (f00, nf0, f01, nf1) == (0, 1024, 1024, 1024)        # disjoint bands
    assert mx0 == mx1 == 150.0                                  # slowest rank's time
    assert tot0 == tot1 == 2 * 384 * 1024 * 2 * 1024            # summed work
    assert s0 != s1
    assert multirank.throughput(mx0, tot0) == pytest.approx(tot0 / 0.150)


def test_single_process_aggregate_is_local():
    assert multirank.aggregate(12.5, 7) == (12.5, 7)
