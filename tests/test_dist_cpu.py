"""Multi-process host logic (paper_2608_16960_gb300/dist.py) on CPU with the
gloo backend, world size 2: slowest-rank timing, whole-job throughput, and
view sharding whose adjoint is the all-reduced sum of the ranks' partial
back-projections (checked against the FP64 oracle's adjoint of all rays)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.dist import job_throughput, max_over_ranks, shard, sum_partials

from _util import oracle_rays


def test_shard_covers_every_item_once():
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            blocks = [shard(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def test_single_process_defaults():
    assert max_over_ranks(3.5) == 3.5
    assert job_throughput(100.0, 2.0, 1) == 50.0
    v = torch.ones(3)
    assert torch.equal(sum_partials(v), torch.ones(3))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # slowest rank's time and the whole job's throughput
        t = max_over_ranks(1.0 + rank)
        assert t == float(world)
        assert job_throughput(10.0, t, world) == 10.0 * world / world
        # view sharding: each rank back-projects its block of rays, then the sum
        wl = workloads.tiny()
        st, di = oracle_rays(wl.views[0])
        y = synth.uniform_volume((st.shape[0],), 5).astype(np.float64)
        lo, hi = shard(st.shape[0], rank, world)
        part = torch.tensor(oracle.adjoint(wl.edges, st[lo:hi], di[lo:hi], y[lo:hi]))
        full = sum_partials(part)
        ref = oracle.adjoint(wl.edges, st, di, y)
        assert np.allclose(full.numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        # a rank that gets no rays contributes zeros
        empty = torch.zeros_like(part)
        assert torch.equal(sum_partials(empty), torch.zeros_like(part))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    oracle.build()
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
