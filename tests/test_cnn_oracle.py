"""Pins of the CNN oracle (oracle/cnn_oracle.py) against definitions that do
not depend on it: a direct loop convolution, adjoint identities, central
finite differences in FP64, and Adam's closed-form first step."""
import numpy as np
import pytest

from oracle import cnn_oracle as cn
from paper_2008_12214_gb300 import synth


def direct_conv(x, W, b):
    """y[b,h,w,co] = bias[co] + sum over the 3x3 window of W * x, zero outside."""
    B, H, Wd, Ci = x.shape
    Co = W.shape[1]
    y = np.zeros((B, H, Wd, Co))
    for n in range(B):
        for h in range(H):
            for w in range(Wd):
                for co in range(Co):
                    acc = b[co]
                    for ky in range(3):
                        for kx in range(3):
                            hh, ww = h + ky - 1, w + kx - 1
                            if 0 <= hh < H and 0 <= ww < Wd:
                                for ci in range(Ci):
                                    acc += W[3 * ky + kx, co, ci] * x[n, hh, ww, ci]
                    y[n, h, w, co] = acc
    return y


def test_conv_matches_direct_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 5, 2))
    W = rng.standard_normal((9, 3, 2))
    b = rng.standard_normal(3)
    assert np.allclose(cn.conv3x3(x, W, b), direct_conv(x, W, b), atol=1e-12)


def test_conv_single_taps_are_shifts_with_zero_fill():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 6, 1))
    for t, (dy, dx) in enumerate(cn.taps()):
        W = np.zeros((9, 1, 1))
        W[t] = 1.0
        y = cn.conv3x3(x, W)[0, :, :, 0]
        for h in range(4):
            for w in range(6):
                hh, ww = h + dy, w + dx
                want = x[0, hh, ww, 0] if 0 <= hh < 4 and 0 <= ww < 6 else 0.0
                assert y[h, w] == want


def test_dgrad_and_wgrad_are_the_adjoints_of_conv():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 5, 7, 3))
    W = rng.standard_normal((9, 4, 3))
    b = rng.standard_normal(4)
    g = rng.standard_normal((2, 5, 7, 4))
    lhs = np.sum(cn.conv3x3(x, W) * g)
    assert np.isclose(lhs, np.sum(x * cn.conv3x3_dgrad(g, W)), rtol=1e-12)
    dW, db = cn.conv3x3_wgrad(x, g)
    assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)
    # the bias enters linearly: d/db sum(g * (conv + b)) = sum of g over pixels
    assert np.isclose(np.sum(cn.conv3x3(x, W, b) * g) - lhs, np.dot(b, db), rtol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 6, 8, 3))
    y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(cn.avgpool2(x) * y), np.sum(x * cn.avgpool2_bwd(y)), rtol=1e-12)
    assert np.isclose(np.sum(cn.up2(y) * x), np.sum(y * cn.up2_bwd(x)), rtol=1e-12)
    assert np.allclose(cn.avgpool2(cn.up2(y)), y, atol=1e-15)
    assert cn.avgpool2(x)[1, 2, 3, 1] == pytest.approx(x[1, 4:6, 6:8, 1].mean(), abs=1e-15)


def test_phase_loss_special_values():
    rng = np.random.default_rng(5)
    T = rng.random((2, 4, 4))
    phi = rng.uniform(-np.pi, np.pi, (2, 4, 4))
    L, dc, ds = cn.phase_loss(np.cos(phi), np.sin(phi), T, phi)
    assert L == pytest.approx(0.0, abs=1e-15) and np.abs(dc).max() < 1e-15 and np.abs(ds).max() < 1e-15
    # on the unit circle the loss is the energy-weighted 1 - cos(phase error)
    L, _, _ = cn.phase_loss(-np.cos(phi), -np.sin(phi), T, phi)
    assert L == pytest.approx(2.0, abs=1e-12)   # sum wT = 1 per image, mean over images
    L, _, _ = cn.phase_loss(-np.sin(phi), np.cos(phi), T, phi)
    assert L == pytest.approx(1.0, abs=1e-12)   # quarter-turn error
    d = rng.uniform(-np.pi, np.pi, (2, 4, 4))
    L, _, _ = cn.phase_loss(np.cos(phi + d), np.sin(phi + d), T, phi)
    wT = T ** 2 / (T ** 2).sum(axis=(1, 2), keepdims=True)
    assert L == pytest.approx((wT * (1 - np.cos(d))).sum() / 2, abs=1e-12)
    # pixels with T = 0 carry no weight
    T0 = T.copy()
    T0[:, :2] = 0
    c, s = rng.standard_normal((2, 2, 4, 4))
    L1, _, _ = cn.phase_loss(c, s, T0, phi)
    c2 = c.copy()
    c2[:, :2] = 5.0
    L2, _, _ = cn.phase_loss(c2, s, T0, phi)
    assert L1 == pytest.approx(L2, abs=1e-15)


def test_phase_loss_gradient_finite_differences():
    rng = np.random.default_rng(6)
    T = rng.random((2, 3, 4))
    phi = rng.uniform(-np.pi, np.pi, (2, 3, 4))
    c, s = rng.standard_normal((2, 2, 3, 4)) * 0.5
    _, dc, ds = cn.phase_loss(c, s, T, phi)
    h = 1e-6
    for arr, grad in ((c, dc), (s, ds)):
        for idx in [(0, 0, 0), (1, 2, 3), (0, 1, 2), (1, 0, 1)]:
            a0 = arr[idx]
            arr[idx] = a0 + h
            Lp = cn.phase_loss(c, s, T, phi)[0]
            arr[idx] = a0 - h
            Lm = cn.phase_loss(c, s, T, phi)[0]
            arr[idx] = a0
            assert grad[idx] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6, abs=1e-11)


def test_net_shapes_and_parameter_count():
    p = cn.init_params(0)
    assert [k for k in p] == cn.param_names()
    n = sum(v.size for v in p.values())
    assert n == 1946338
    T = np.random.default_rng(7).random((1, 16, 24))
    c, s, _ = cn.forward(p, cn.net_input(T))
    assert c.shape == s.shape == (1, 16, 24)
    ph = cn.predict_phase(p, T)
    assert np.all(np.abs(ph) <= np.pi)


def test_whole_net_gradients_finite_differences():
    rng = np.random.default_rng(8)
    p = cn.init_params(3)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    T = rng.random((2, 8, 8)) * (rng.random((2, 8, 8)) > 0.3)
    phi = rng.uniform(-np.pi, np.pi, (2, 8, 8))
    _, g = cn.loss_and_grads(p, T, phi)
    h = 1e-6
    picks = []
    for name in cn.param_names():
        flat = p[name].reshape(-1)
        for j in rng.choice(flat.size, 2, replace=False):
            picks.append((name, int(j)))
    for name, j in picks:
        flat = p[name].reshape(-1)
        v0 = flat[j]
        flat[j] = v0 + h
        Lp = cn.loss_and_grads(p, T, phi)[0]
        flat[j] = v0 - h
        Lm = cn.loss_and_grads(p, T, phi)[0]
        flat[j] = v0
        fd = (Lp - Lm) / (2 * h)
        an = g[name].reshape(-1)[j]
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-9), (name, j, an, fd)


def test_adam_first_step_closed_form_and_second_step():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    m = np.zeros(4)
    v = np.zeros(4)
    th1, m1, v1 = cn.adam_step(th, g, m, v, 1, lr=0.01)
    # step 1: m^ = g, v^ = g^2, so the step is lr * g / (|g| + eps)
    assert np.allclose(th1, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    g2 = np.array([0.1, 0.1, 0.1, 0.1])
    th2, m2, v2 = cn.adam_step(th1, g2, m1, v1, 2, lr=0.01)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    assert np.allclose(th2, th1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-13)


def test_base_phase_reads_the_label_as_its_remainder():
    """With a base phase phi_b the network's (c, s) is compared with the
    label's remainder e^{i(phi - phi_b)}, and the predicted phase is the
    phase of (c, s) plus phi_b: the loss equals the plain loss on the labels
    phi - phi_b, the gradients too, and the phase is shifted by phi_b."""
    H = W = 16
    p = cn.init_params(2)
    T = np.stack([synth.target(H, W, 70 + b) for b in range(2)])
    rng = np.random.default_rng(3)
    phi = rng.uniform(-np.pi, np.pi, (2, H, W))
    base = rng.uniform(0, 2 * np.pi, (H, W))
    L1, g1 = cn.loss_and_grads(p, T, phi, base)
    L2, g2 = cn.loss_and_grads(p, T, phi - base)
    assert L1 == L2 and all(np.array_equal(g1[k], g2[k]) for k in g1)
    # a label equal to the base is a remainder of phase 0: (c, s) = (1, 0) scores 0
    c, s, _ = cn.forward(p, cn.net_input(T))
    assert cn.phase_loss(np.ones_like(c), np.zeros_like(s), T, (base + 0 * phi) - base)[0] == 0.0
    assert np.allclose(cn.predict_phase(p, T, base), cn.predict_phase(p, T) + base, atol=1e-15)
