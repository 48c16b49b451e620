"""Learned warm start for GS: training the network of include/hologen_cnn.h on
the engine's own GS phases, and measuring what it gains.

Argument marshalling and loop control only: every step runs in the
library's kernels (GS through hg_run / hg_get_phase, the network through
hg_cnn_*); the targets come from synth.targets_device.

Labels.  The label of a target is the replay phase after `label_iters` GS
iterations (Section 3.2) from a starting phase chosen by `label_start`:
"flat" (phase 0), "fixed" (one seeded random phase shared by every target)
or "random" (GS's own seeded random phase per target).  The first two make
the label a deterministic function of the target.  With `residual` (fixed
starts only) the shared start phase becomes the network's base phase
(hg_cnn_set_base_phase): the network then models e^{i(phi - phi_0)}, the
part of the label that GS added to its start, and its phase output is that
remainder's phase plus phi_0.

Evaluation.  For held-out targets (seeds from 10^6), plain GS from the
seeded random phase runs `ref_iters` iterations; its last MSE is the
reference.  GS started from the network's phase then runs until its MSE
reaches the reference; iterations and wall time (the network's forward
pass included) are compared per target.  GS from a random phase stays the
fallback: a target the warm start does not bring to the reference within
`max_iters` iterations counts as not reached.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import hologen as hg
from . import shard
from . import synth

HELDOUT_BASE = 10 ** 6


def start_phase(kind, T, seed=0):
    """Starting replay phase for labels: None (GS's seeded random phase) or a tensor like T."""
    if kind == "flat":
        return torch.zeros_like(T)
    if kind == "fixed":
        g = torch.Generator(device="cpu").manual_seed(12345 + seed)
        ph = torch.rand(T.shape[1:], generator=g) * (2 * np.pi)
        return ph.to(T.device).expand_as(T).contiguous()
    if kind == "random":
        return None
    raise ValueError(kind)


def gs_labels(plan, T, label_iters=200, label_start="flat"):
    """Replay phase after label_iters GS iterations; T [B][H][W] on the device."""
    plan.run(T, start_phase(label_start, T), label_iters)
    phi = torch.empty_like(T)
    hg.hg_get_phase(plan.h, phi)
    return phi


def train(H, W, pairs, batch=8, lr=1e-3, seed=0, chunk=64, label_iters=200, epochs=1, net=None,
          base_seed=1, log=None, label_start="flat", slm_kind=hg.HG_SLM_BINARY, levels=2, residual=False):
    """Trains on `pairs` (target, GS phase) pairs, generated `chunk` at a time
    (target seeds base_seed ...).  Returns (net, losses per step, seconds)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    if net is None:
        net = hg.CNN(H, W, batch, seed=seed)
    if residual:
        if label_start != "fixed":
            raise ValueError("residual labels need the one shared start phase (label_start='fixed')")
        hg.hg_cnn_set_base_phase(net.h, start_phase("fixed", torch.zeros((1, H, W), device=dev))[0].contiguous())
    plan = hg.Plan(H, W, chunk, slm_kind, levels)
    losses = []
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    lhist = torch.zeros(max(1, pairs // batch * epochs), dtype=torch.float64, device=dev)
    t0 = time.time()
    step = 0
    try:
        for _ in range(epochs):
            for c0 in range(0, pairs - chunk + 1, chunk):
                T = synth.targets_device(chunk, H, W, base_seed + c0, dev)
                if label_start == "random":  # a fresh Philox stream per chunk
                    pl = hg.Plan(H, W, chunk, slm_kind, levels, seed=base_seed + c0)
                    phi = gs_labels(pl, T, label_iters, label_start)
                    pl.sync()
                    pl.close()
                else:
                    phi = gs_labels(plan, T, label_iters, label_start)
                for i in range(0, chunk, batch):
                    hg.hg_cnn_train_step(net.h, T[i:i + batch], phi[i:i + batch], batch, lr, loss)
                    if step < lhist.numel():
                        lhist[step:step + 1].copy_(loss)
                    step += 1
                if log:
                    log("pairs %d loss %.4f" % (c0 + chunk, loss.item()))
        hg.hg_cnn_sync(net.h)
        plan.sync()
    finally:
        plan.close()
    losses = lhist[:step].cpu().numpy().tolist()
    return net, losses, time.time() - t0


def dp_train_step(net, T, phi, batch, lr, grad_buf, loss=None):
    """One data-parallel training step: this rank's gradients of its batch
    (hg_cnn_gradients), averaged over the ranks (shard.average_over_ranks,
    an NCCL all-reduce on GPU ranks; nothing with one rank), then one Adam
    update (hg_cnn_apply_grads), the same on every rank.  grad_buf: float32
    [HG_CNN_NPARAMS] on the net's device; loss (double [1]) gets this rank's
    loss.  Every call is on the current stream, as the net's calls are."""
    hg.hg_cnn_gradients(net.h, T, phi, batch, loss)
    hg.hg_cnn_get_grads(net.h, grad_buf)
    shard.average_over_ranks(grad_buf)
    hg.hg_cnn_apply_grads(net.h, grad_buf, lr)


def evaluate(net, H, W, n, ref_iters=100, max_iters=100, chunk=64, base_seed=HELDOUT_BASE,
             slm_kind=hg.HG_SLM_BINARY, levels=2):
    """Iterations and wall time for GS from the network's phase to reach the
    MSE plain random-phase GS reaches after ref_iters iterations."""
    dev = torch.device("cuda", torch.cuda.current_device())
    chunk = min(chunk, n, net.max_batch)
    plan = hg.Plan(H, W, chunk, slm_kind, levels)
    ref, warm_iters, flat_iters, rand_curve, warm_curve, flat_curve = [], [], [], [], [], []
    t_iter = t_cnn = 0.0
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    try:
        for c0 in range(0, n - chunk + 1, chunk):
            T = synth.targets_device(chunk, H, W, base_seed + c0, dev)
            mse_r = torch.empty((chunk, ref_iters), dtype=torch.float64, device=dev)
            e0.record()
            plan.run(T, None, ref_iters, None, mse_r)  # seeded random phase
            e1.record()
            torch.cuda.synchronize()
            t_iter += e0.elapsed_time(e1) / ref_iters
            phase0 = torch.empty_like(T)
            e0.record()
            hg.hg_cnn_forward(net.h, T, chunk, None, phase0)
            e1.record()
            mse_w = torch.empty((chunk, max_iters), dtype=torch.float64, device=dev)
            plan.run(T, phase0, max_iters, None, mse_w)
            e2.record()
            torch.cuda.synchronize()
            t_cnn += e0.elapsed_time(e1)
            mse_f = torch.empty((chunk, max_iters), dtype=torch.float64, device=dev)
            plan.run(T, torch.zeros_like(T), max_iters, None, mse_f)  # flat phase 0, for context
            plan.sync()
            r = mse_r[:, -1].cpu().numpy()
            for name, m, out in (("warm", mse_w, warm_iters), ("flat", mse_f, flat_iters)):
                mm = m.cpu().numpy()
                for b in range(chunk):
                    hit = np.nonzero(mm[b] <= r[b])[0]
                    out.append(int(hit[0]) + 1 if hit.size else np.inf)
            ref.extend(r.tolist())
            rand_curve.append(mse_r.cpu().numpy() / r[:, None])
            warm_curve.append(mse_w.cpu().numpy() / r[:, None])
            flat_curve.append(mse_f.cpu().numpy() / r[:, None])
    finally:
        plan.close()
    chunks = n // chunk
    t_iter /= chunks
    t_cnn /= chunks
    warm_iters = np.array(warm_iters, dtype=float)
    t_rand = ref_iters * t_iter
    t_warm = t_cnn + np.where(np.isfinite(warm_iters), warm_iters, max_iters) * t_iter
    return dict(n=len(ref), ref_iters=ref_iters, max_iters=max_iters,
                ms_per_gs_iter_batch=t_iter, ms_cnn_batch=t_cnn, batch=chunk,
                reached=float(np.mean(np.isfinite(warm_iters))),
                median_warm_iters=float(np.median(warm_iters)),
                median_flat_iters=float(np.median(np.array(flat_iters, dtype=float))),
                median_speedup=float(np.median(t_rand / t_warm)),
                # mean MSE per iteration, each target's curve divided by its reference
                rel_rand_curve=np.concatenate(rand_curve).mean(axis=0).tolist(),
                rel_warm_curve=np.concatenate(warm_curve).mean(axis=0).tolist(),
                rel_flat_curve=np.concatenate(flat_curve).mean(axis=0).tolist())
