"""The multi-process path on CPU: world-size-2 gloo process groups (no GPU).

Covers the host side of what torchrun runs on several GPUs: the voter shards,
the one exchange of a voter-sharded tally (an int32 sum all-reduce of the
partial tallies, exact because d is a sum over voters), and the max over
ranks of the step times. The local tally here is the CPU oracle standing in
for the library's GPU tally (test infrastructure only)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_12976_gb300 import distributed as D


def test_voter_shards_partition():
    for n in (0, 1, 7, 20000, 20001):
        for world in (1, 2, 3, 8):
            spans = [D.voter_shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.voter_shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import oracle
    import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        m, n, k = 60, 1001, 12
        ballots = W.mallows(77, n, m, k, 0.85, W.permutation(78, m))
        a, b = D.voter_shard(n, rank, world)

        def cpu_tally(r, m, flags=0, ctx=None):
            return torch.from_numpy(np.ascontiguousarray(oracle.tally(r.numpy(), m), dtype=np.int32))

        d = D.tally_voter_sharded(torch.from_numpy(ballots[a:b].copy()), m, tally=cpu_tally)
        slow = D.max_over_ranks(0.25 + rank, device="cpu")
        np.save(os.path.join(out_dir, f"d{rank}.npy"), d.numpy())
        np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([slow]))
    finally:
        dist.destroy_process_group()


def test_voter_sharded_tally_gloo(tmp_path):
    """Two ranks, each tallying half of the voters: after the all-reduce both
    hold the whole election's d, equal to the oracle's tally of all ballots;
    the max over ranks sees the slower rank."""
    import oracle
    import workloads as W
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    m, n, k = 60, 1001, 12
    want = oracle.tally(W.mallows(77, n, m, k, 0.85, W.permutation(78, m)), m)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"d{r}.npy"), want), f"rank {r}"
        assert np.load(tmp_path / f"t{r}.npy")[0] == 1.25
