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


def _dp_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import cnn_oracle as cn
        p = cn.init_params(2)
        names = cn.param_names()
        T, phi = _dp_batch()
        half = T.shape[0] // world
        sl = slice(rank * half, (rank + 1) * half)
        _, g = cn.loss_and_grads(p, T[sl], phi[sl])
        flat = torch.from_numpy(np.concatenate([g[k].ravel() for k in names]))
        shard.average_over_ranks(flat)
        theta = np.concatenate([p[k].ravel() for k in names])
        z = np.zeros_like(theta)
        theta1, _, _ = cn.adam_step(theta, flat.numpy(), z, z, 1, 1e-3)
        if rank == 0:
            np.savez(out_path, g=flat.numpy(), theta=theta1)
    finally:
        dist.destroy_process_group()


def _dp_batch():
    rng = np.random.default_rng(31)
    T = rng.random((4, 8, 8)) * (rng.random((4, 8, 8)) > 0.3)
    phi = rng.uniform(-np.pi, np.pi, (4, 8, 8))
    return T, phi


def _tmp_dir():
    import pathlib
    import tempfile
    return pathlib.Path(tempfile.mkdtemp(prefix="dp_"))


def test_two_gloo_ranks_average_gradients_to_the_whole_batch():
    """Data-parallel training's exchange (shard.average_over_ranks, used by
    warmstart.dp_train_step): two ranks with two images each, FP64 oracle
    gradients of the net; the rank average equals the gradient of the
    four-image batch, and the Adam step from it is the whole batch's."""
    out = str(_tmp_dir() / "dp.npz")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_dp_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = np.load(out)
    from oracle import cnn_oracle as cn
    p = cn.init_params(2)
    names = cn.param_names()
    T, phi = _dp_batch()
    _, g = cn.loss_and_grads(p, T, phi)
    full = np.concatenate([g[k].ravel() for k in names])
    assert np.allclose(res["g"], full, rtol=1e-12, atol=1e-18)
    theta = np.concatenate([p[k].ravel() for k in names])
    z = np.zeros_like(theta)
    theta1, _, _ = cn.adam_step(theta, full, z, z, 1, 1e-3)
    # Adam's first step is lr g / (|g| + eps): components with |g| near eps (1e-8)
    # carry the rounding of the two summation orders at about 1e-15
    assert np.allclose(res["theta"], theta1, rtol=0, atol=1e-13)
