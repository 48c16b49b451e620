"""The multi-rank layout of the path (paper_2008_12214_gb300.shard) on two
gloo ranks on CPU: disjoint per-rank targets, shards that cover a global
batch once, the max-over-ranks time and the whole-job rate, and the final
gather; the oracle run on each rank's shard and gathered equals one process
running the whole batch (no collective is needed on the data path)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2008_12214_gb300 import shard


def test_seed_and_shard_layout():
    seeds = [shard.target_seeds(r, 5) for r in range(3)]
    flat = sum(seeds, [])
    assert len(set(flat)) == 15 and flat == list(range(1000, 1015))
    for total, world in ((10, 3), (7, 7), (3, 4), (64, 8)):
        got = []
        for r in range(world):
            s, c = shard.shard(total, r, world)
            got += list(range(s, s + c))
            assert c in (total // world, total // world + 1)
        assert got == list(range(total))
    assert shard.weak_scaling_rate(4, 100, 2.0) == 200.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, total, n, iters, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2008_12214_gb300 import synth
        start, count = shard.shard(total, rank, world)
        t = synth.targets(total, n, n, 2000)[start:start + count]
        ph = synth.init_phases(total, n, n, 2000)[start:start + count]
        mse = np.stack([oracle.gs_run(t[b], ph[b].astype(np.float64), iters)["mse"] for b in range(count)])
        counts = [shard.shard(total, r, world)[1] for r in range(world)]
        gathered = shard.gather_rows(torch.from_numpy(mse), counts)
        slowest = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            np.savez(out_path, mse=gathered.numpy(), slowest=slowest)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_gather_and_time(tmp_path):
    total, n, iters, world = 5, 16, 3, 2
    out = str(tmp_path / "r0.npz")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, total, n, iters, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = np.load(out)
    import oracle
    from paper_2008_12214_gb300 import synth
    t = synth.targets(total, n, n, 2000)
    ph = synth.init_phases(total, n, n, 2000)
    ref = np.stack([oracle.gs_run(t[b], ph[b].astype(np.float64), iters)["mse"] for b in range(total)])
    assert np.array_equal(res["mse"], ref)
    assert float(res["slowest"]) == 11.0
