"""FP64 CPU oracle of the learned warm start: an encoder-decoder CNN that maps
a target amplitude to a starting replay phase for GS, its loss, its gradients
and the Adam update.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never imports it.
It shares no code with the CUDA path.

The paper (HoloGen, arXiv:2008.12214) describes no network: it names GS,
weighted GS and OSPR as the generators (Sections 3.2, 3.4) whose starting
replay phase is free.  Everything about the net is therefore a stated
reading, written out here as plain array code:

* Layout: activations [B][H][W][C] (channels fastest); a 3x3 weight is
  [9][Cout][Cin] with tap t = 3*(dy+1) + (dx+1) for dy, dx in {-1, 0, 1}.
* conv3x3 (cross-correlation, zero padding 1):
      y[b,h,w,co] = bias[co] + sum_{t,ci} W[t,co,ci] * x[b, h+dy_t, w+dx_t, ci]
* Net (levels 0..3, widths 32/64/128/256), every 3x3 conv followed by ReLU:
      enc l: two convs (C_{l-1} -> C_l -> C_l), 2x2 average pool between levels;
      dec l (l = 2, 1, 0): nearest 2x upsample of the coarser output, concatenated
      [upsampled, encoder skip] along channels, then two convs -> C_l;
      head: 1x1 conv 32 -> 2 channels (c, s) without ReLU; phase = atan2(s, c).
* Input: T / max(T) per image (the amplitude's scale carries no information,
  Section 3's scale freedom).
* Loss (per image, averaged over the batch), with wT = T^2 / sum T^2:
      L = sum_px wT * |(c, s) - (cos phi, sin phi)|^2 / 2
  i.e. the prediction regresses the label's phasor.  On the unit circle
  |(c, s)| = 1 this is exactly 1 - cos(phase error) weighted by the target
  energy; off it the loss is quadratic, so its gradient stays bounded and
  proportional to the error everywhere.  (Normalising (c, s) first makes the
  gradient grow as 1/|(c, s)|: on a freshly initialised net 0.1 % of the
  pixels then held 40 % of its norm; and a regularised normalisation
  (c, s) / sqrt(c^2 + s^2 + 1) rewards ever larger outputs, on which the
  spatial gradient vanishes.)
* Adam (Kingma & Ba): beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.

Pins (tests/test_cnn_oracle.py): the conv against a direct loop definition;
the adjoint identities <conv(x), g> = <x, dgrad(g)> = <W, wgrad(x, g)>, and
the same for pool / upsample; loss and whole-net gradients against central
finite differences; Adam's first step against its closed form.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (32, 64, 128, 256)
# (name, Cin, Cout) of every 3x3 conv, in parameter order
CONVS = (("e0a", 1, 32), ("e0b", 32, 32), ("e1a", 32, 64), ("e1b", 64, 64),
         ("e2a", 64, 128), ("e2b", 128, 128), ("e3a", 128, 256), ("e3b", 256, 256),
         ("d2a", 384, 128), ("d2b", 128, 128), ("d1a", 192, 64), ("d1b", 64, 64),
         ("d0a", 96, 32), ("d0b", 32, 32))
HEAD = ("head", 32, 2)


def taps():
    """(dy, dx) of tap t = 3*(dy+1) + (dx+1)."""
    return [(t // 3 - 1, t % 3 - 1) for t in range(9)]


# ----------------------------------------------------------------- layers

def conv3x3(x, W, bias=None):
    """x [B,H,W,Ci], W [9,Co,Ci] -> [B,H,W,Co] (zero padding 1)."""
    B, H, Wd, Ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:H + 1, 1:Wd + 1, :] = x
    y = np.zeros((B, H, Wd, W.shape[1]))
    for t, (dy, dx) in enumerate(taps()):
        y += xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :] @ W[t].T
    if bias is not None:
        y += bias
    return y


def conv3x3_dgrad(g, W):
    """Gradient wrt x of sum(g * conv3x3(x, W)): g [B,H,W,Co] -> [B,H,W,Ci]."""
    B, H, Wd, Co = g.shape
    gp = np.zeros((B, H + 2, Wd + 2, Co))
    gp[:, 1:H + 1, 1:Wd + 1, :] = g
    dx = np.zeros((B, H, Wd, W.shape[2]))
    for t, (dy, dxx) in enumerate(taps()):
        # x[h', w'] met g[h' - dy, w' - dx] through tap t
        dx += gp[:, 1 - dy:1 - dy + H, 1 - dxx:1 - dxx + Wd, :] @ W[t]
    return dx


def conv3x3_wgrad(x, g):
    """Gradients wrt W [9,Co,Ci] and bias [Co] of sum(g * conv3x3(x, W, bias))."""
    B, H, Wd, Ci = x.shape
    Co = g.shape[3]
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:H + 1, 1:Wd + 1, :] = x
    dW = np.zeros((9, Co, Ci))
    gf = g.reshape(-1, Co)
    for t, (dy, dx) in enumerate(taps()):
        dW[t] = gf.T @ xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :].reshape(-1, Ci)
    return dW, gf.sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_bwd(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# ------------------------------------------------------------------- loss

def phase_loss(c, s, T, phi):
    """Mean over images of sum wT |(c, s) - e^{i phi}|^2 / 2; returns (L, dc, ds)."""
    B = T.shape[0]
    wT = T ** 2 / (T ** 2).sum(axis=(1, 2), keepdims=True)
    ec, es = c - np.cos(phi), s - np.sin(phi)
    L = (wT * (ec * ec + es * es)).sum() / (2 * B)
    return L, wT * ec / B, wT * es / B


# -------------------------------------------------------------------- net

def init_params(seed=0):
    """He-normal 3x3 weights (std sqrt(2 / (9 Cin))), head std sqrt(1/32), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in CONVS:
        p[name + ".w"] = rng.standard_normal((9, co, ci)) * np.sqrt(2.0 / (9 * ci))
        p[name + ".b"] = np.zeros(co)
    p["head.w"] = rng.standard_normal((2, 32)) * np.sqrt(1.0 / 32)
    p["head.b"] = np.zeros(2)
    return p


def param_names():
    return [n + s for n, _, _ in CONVS for s in (".w", ".b")] + ["head.w", "head.b"]


def net_input(T):
    """T [B,H,W] -> x [B,H,W,1] = T / max T per image."""
    m = T.reshape(T.shape[0], -1).max(axis=1)
    return (T / m[:, None, None])[..., None]


def keep(v):
    return v


def forward(p, x, store=keep):
    """x [B,H,W,1] -> (c, s, cache).  H, W divisible by 8.  `store` is applied
    to every activation the net keeps (identity here; a test may pass a
    rounding to model a storage precision)."""
    a = {}

    def block(name, inp):
        pre = conv3x3(inp, p[name + ".w"], p[name + ".b"])
        out = store(relu(pre))
        a[name + ".in"] = inp
        a[name + ".out"] = out
        return out

    e = []
    h = x
    for l in range(4):
        if l:
            h = store(avgpool2(h))
        h = block("e%da" % l, h)
        h = block("e%db" % l, h)
        e.append(h)
    for l in (2, 1, 0):
        h = np.concatenate([up2(h), e[l]], axis=3)
        h = block("d%da" % l, h)
        h = block("d%db" % l, h)
    a["head.in"] = h
    cs = h @ p["head.w"].T + p["head.b"]
    return cs[..., 0], cs[..., 1], a


def backward(p, a, dc, ds, store=keep):
    """Gradients of the loss wrt every parameter, from dL/dc, dL/ds.  `store`
    as in forward, applied to every activation gradient kept."""
    g = {}
    dcs = np.stack([dc, ds], axis=-1)
    h = a["head.in"]
    g["head.w"] = dcs.reshape(-1, 2).T @ h.reshape(-1, h.shape[3])
    g["head.b"] = dcs.reshape(-1, 2).sum(axis=0)
    dh = dcs @ p["head.w"]

    def block_bwd(name, dout):
        dpre = store(dout * (a[name + ".out"] > 0))
        g[name + ".w"], g[name + ".b"] = conv3x3_wgrad(a[name + ".in"], dpre)
        return store(conv3x3_dgrad(dpre, p[name + ".w"]))

    dskip = {}
    for l in (0, 1, 2):
        dh = block_bwd("d%db" % l, dh)
        dcat = block_bwd("d%da" % l, dh)
        cu = dcat.shape[3] - WIDTHS[l]      # channels of the upsampled part
        dskip[l] = dcat[..., cu:]
        dh = up2_bwd(dcat[..., :cu])
    for l in (3, 2, 1, 0):
        if l < 3:
            dh = dh + dskip[l]
        dh = block_bwd("e%db" % l, dh)
        dh = block_bwd("e%da" % l, dh)
        if l:
            dh = avgpool2_bwd(dh)
    return g


def loss_and_grads(p, T, phi, base=None):
    """Loss and parameter gradients for labels phi; with a base phase [H][W]
    (shared by the images) (c, s) is compared with e^{i(phi - base)}."""
    c, s, a = forward(p, net_input(T))
    L, dc, ds = phase_loss(c, s, T, phi if base is None else phi - base)
    return L, backward(p, a, dc, ds)


def predict_phase(p, T, base=None):
    """Phase of the network's (c, s), plus the base phase if one is given."""
    c, s, _ = forward(p, net_input(T))
    return np.arctan2(s, c) + (0.0 if base is None else base)


# ------------------------------------------------------------------- Adam

def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
