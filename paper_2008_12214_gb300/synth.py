"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module only draws inputs; it holds none of the hologram method's
arithmetic (no normalisation, no transforms, no quantisation).  The paper
measures on no public dataset, so every workload uses these synthetic targets.

Target recipe (amplitude, replay order, zero background):
  * 16 Gaussian blobs: centre uniform over the field, sigma ~ U(2, 20) px,
    peak ~ U(0.2, 1);
  * 8 axis-aligned rectangles: height ~ U[ny/32, ny/4], width ~ U[nx/32, nx/4]
    (at least one pixel), top-left corner uniform over the field (clipped at
    the far edge), amplitude ~ U(0.3, 1);
  * all components summed; float32, NOT normalised (the method's target
    preparation normalises to sum T^2 = 1).
Target b of a batch uses seed base_seed + b (base 1000 by default).
Initial phases are U[0, 2 pi) float32 from the stream (seed, 1).

targets_device() draws the same per-seed parameters and renders them on a
torch device (every component is an outer product of a y profile and an x
profile), for the many targets a training set needs; it equals targets() up
to float32 rounding.
"""
from __future__ import annotations

import numpy as np

BLOBS = 16
RECTS = 8


def _params(ny: int, nx: int, seed: int):
    """Blob and rectangle parameters of target `seed`, in target()'s draw order."""
    rng = np.random.default_rng(seed)
    blobs, rects = [], []
    for _ in range(BLOBS):
        cy = rng.uniform(0, ny)
        cx = rng.uniform(0, nx)
        sigma = rng.uniform(2.0, 20.0)
        peak = rng.uniform(0.2, 1.0)
        blobs.append((cy, cx, sigma, peak))
    for _ in range(RECTS):
        h = max(1, int(round(rng.uniform(ny / 32, ny / 4))))
        w = max(1, int(round(rng.uniform(nx / 32, nx / 4))))
        y0 = int(rng.integers(0, ny))
        x0 = int(rng.integers(0, nx))
        amp = rng.uniform(0.3, 1.0)
        rects.append((h, w, y0, x0, amp))
    return blobs, rects


def targets_device(batch: int, ny: int, nx: int, base_seed: int = 1000, device="cuda"):
    """targets() rendered on `device` as a float32 torch tensor [batch][ny][nx]."""
    import torch
    K = BLOBS + RECTS
    Y = np.zeros((batch, K, ny))
    X = np.zeros((batch, K, nx))
    y = np.arange(ny, dtype=np.float64)
    x = np.arange(nx, dtype=np.float64)
    for b in range(batch):
        blobs, rects = _params(ny, nx, base_seed + b)
        for k, (cy, cx, sigma, peak) in enumerate(blobs):
            Y[b, k] = peak * np.exp(-((y - cy) ** 2) / (2 * sigma * sigma))
            X[b, k] = np.exp(-((x - cx) ** 2) / (2 * sigma * sigma))
        for k, (h, w, y0, x0, amp) in enumerate(rects):
            Y[b, BLOBS + k, y0:y0 + h] = amp
            X[b, BLOBS + k, x0:x0 + w] = 1.0
    Yd = torch.from_numpy(Y.astype(np.float32)).to(device)
    Xd = torch.from_numpy(X.astype(np.float32)).to(device)
    return torch.bmm(Yd.transpose(1, 2), Xd).contiguous()


def target(ny: int, nx: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    y = np.arange(ny, dtype=np.float64)
    x = np.arange(nx, dtype=np.float64)
    t = np.zeros((ny, nx), np.float64)
    for _ in range(BLOBS):
        cy = rng.uniform(0, ny)
        cx = rng.uniform(0, nx)
        sigma = rng.uniform(2.0, 20.0)
        peak = rng.uniform(0.2, 1.0)
        gy = np.exp(-((y - cy) ** 2) / (2 * sigma * sigma))
        gx = np.exp(-((x - cx) ** 2) / (2 * sigma * sigma))
        t += peak * np.outer(gy, gx)
    for _ in range(RECTS):
        h = max(1, int(round(rng.uniform(ny / 32, ny / 4))))
        w = max(1, int(round(rng.uniform(nx / 32, nx / 4))))
        y0 = int(rng.integers(0, ny))
        x0 = int(rng.integers(0, nx))
        amp = rng.uniform(0.3, 1.0)
        t[y0:y0 + h, x0:x0 + w] += amp
    return t.astype(np.float32)


def init_phase(ny: int, nx: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 1])
    return (rng.random((ny, nx)) * (2 * np.pi)).astype(np.float32)


def targets(batch: int, ny: int, nx: int, base_seed: int = 1000) -> np.ndarray:
    return np.stack([target(ny, nx, base_seed + b) for b in range(batch)])


def init_phases(batch: int, ny: int, nx: int, base_seed: int = 1000) -> np.ndarray:
    return np.stack([init_phase(ny, nx, base_seed + b) for b in range(batch)])
