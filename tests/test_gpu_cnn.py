"""GPU parity of the warm-start network against the FP64 oracle
(oracle/cnn_oracle.py): the tensor-core convolutions layer by layer, the
whole net's outputs, loss and gradients, the fused Adam update, and a short
training run.

Tolerances.  The kernels read BF16 operands exactly and accumulate in FP32,
so a convolution differs from the FP64 oracle (fed the same BF16 values) by
the FP32 accumulation error (~1e-6 relative) plus the rounding of its BF16
output (at most 2^-9 relative per element): single layers are held to the
low-precision bound rel-L2 <= 3e-3 and to 2^-8 relative per element.  The
weight gradient is FP32 end to end: rel-L2 <= 1e-4.  Through the whole net
every activation and activation gradient is stored in BF16 between layers,
and ReLU masks and the cancellation in gradient sums amplify that rounding;
the floor is measured, not guessed: the oracle is run a second time with the
same BF16 storage (its `store` hook), and the net must lie within a small
multiple of that run's distance from the exact oracle."""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as cn
from paper_2008_12214_gb300 import hologen as hg
from paper_2008_12214_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def bf(a):
    """The BF16 value of each element (round to nearest even), as float64."""
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def dev_bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(DEV)


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# B, H, W, Cin, Cout, relu, bias, mask
FWD_CASES = [
    (2, 8, 128, 32, 32, True, True, False),
    (1, 16, 256, 96, 64, True, True, True),
    (2, 32, 16, 384, 128, False, True, False),
    (1, 8, 128, 64, 384, True, False, True),
    (1, 8, 64, 128, 256, True, True, False),
    (3, 4, 128, 192, 96, False, False, False),
]


@pytest.mark.parametrize("B,H,W,Cin,Cout,relu,bias,mask", FWD_CASES)
def test_conv_forward_matches_oracle(B, H, W, Cin, Cout, relu, bias, mask):
    rng = np.random.default_rng(B * 1000 + Cin + Cout)
    x = bf(rng.standard_normal((B, H, W, Cin)))
    w = bf(rng.standard_normal((9, Cout, Cin)) * np.sqrt(2.0 / (9 * Cin)))
    b = rng.standard_normal(Cout).astype(np.float32) if bias else None
    m = bf(rng.standard_normal((B, H, W, Cout))) if mask else None
    ref = cn.conv3x3(x, w, None if b is None else b.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)
    if mask:
        ref = ref * (m > 0)
    y = torch.full((B, H, W, Cout), 7.0, dtype=torch.bfloat16, device=DEV)
    hg.hg_conv3x3_forward(dev_bf16(x), B, H, W, Cin, dev_bf16(w), Cout,
                          None if b is None else torch.from_numpy(b).to(DEV), int(relu),
                          dev_bf16(m) if mask else None, y)
    hg.hg_conv_status()
    got = host(y)
    print("conv fwd", (B, H, W, Cin, Cout), "rel-L2", rel_l2(got, ref))
    assert rel_l2(got, ref) <= 3e-3, rel_l2(got, ref)
    slack = 1e-3 * np.abs(ref).max()
    bad = np.abs(got - ref) > 2.0 ** -8 * np.abs(ref) + slack
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])


@pytest.mark.parametrize("B,H,W,Cin,Cout,mask", [(2, 8, 128, 32, 32, True), (1, 8, 64, 384, 128, False),
                                                 (2, 16, 32, 96, 32, True), (1, 8, 128, 256, 256, True)])
def test_conv_dgrad_matches_oracle(B, H, W, Cin, Cout, mask):
    rng = np.random.default_rng(7 + Cin + Cout)
    dy = bf(rng.standard_normal((B, H, W, Cout)))
    w = bf(rng.standard_normal((9, Cout, Cin)) * np.sqrt(2.0 / (9 * Cin)))
    m = bf(rng.standard_normal((B, H, W, Cin))) if mask else None
    ref = cn.conv3x3_dgrad(dy, w)
    if mask:
        ref = ref * (m > 0)
    w_rot = np.ascontiguousarray(w[::-1].transpose(0, 2, 1))  # [t][ci][co] = w[8 - t][co][ci]
    dx = torch.empty((B, H, W, Cin), dtype=torch.bfloat16, device=DEV)
    hg.hg_conv3x3_dgrad(dev_bf16(dy), B, H, W, Cout, dev_bf16(w_rot), Cin, dev_bf16(m) if mask else None, dx)
    hg.hg_conv_status()
    got = host(dx)
    print("conv dgrad", (B, H, W, Cin, Cout), "rel-L2", rel_l2(got, ref))
    assert rel_l2(got, ref) <= 3e-3, rel_l2(got, ref)


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 8, 128, 32, 32), (1, 16, 64, 96, 64), (2, 16, 16, 384, 128),
                                            (1, 8, 128, 64, 256), (2, 32, 32, 192, 64)])
def test_conv_wgrad_matches_oracle(B, H, W, Cin, Cout):
    rng = np.random.default_rng(11 + Cin * Cout)
    x = bf(rng.standard_normal((B, H, W, Cin)))
    dy = bf(rng.standard_normal((B, H, W, Cout)))
    dw_ref, db_ref = cn.conv3x3_wgrad(x, dy)
    ws = torch.empty(hg.hg_conv3x3_wgrad_workspace(B, H, W, Cin, Cout), dtype=torch.uint8, device=DEV)
    dw = torch.full((9, Cout, Cin), float("nan"), dtype=torch.float32, device=DEV)
    db = torch.full((Cout,), float("nan"), dtype=torch.float32, device=DEV)
    hg.hg_conv3x3_wgrad(dev_bf16(x), dev_bf16(dy), B, H, W, Cin, Cout, dw, db, ws)
    hg.hg_conv_status()
    got, gb = dw.cpu().numpy().astype(np.float64), db.cpu().numpy().astype(np.float64)
    print("conv wgrad", (B, H, W, Cin, Cout), "rel-L2", rel_l2(got, dw_ref), rel_l2(gb, db_ref))
    assert rel_l2(got, dw_ref) <= 1e-4, rel_l2(got, dw_ref)
    assert rel_l2(gb, db_ref) <= 1e-4, rel_l2(gb, db_ref)


def test_conv_rejects_untileable_shapes():
    x = torch.zeros(1 * 8 * 100 * 32, dtype=torch.bfloat16, device=DEV)
    w = torch.zeros(9 * 32 * 32, dtype=torch.bfloat16, device=DEV)
    with pytest.raises(hg.HgError) as e:
        hg.hg_conv3x3_forward(x, 1, 8, 100, 32, w, 32, None, 1, None, x)
    assert e.value.status == 2
    with pytest.raises(hg.HgError) as e:
        hg.hg_conv3x3_forward(x, 1, 8, 128, 48, w, 32, None, 1, None, x)
    assert e.value.status == 2


# ------------------------------------------------------------------ network

def flat(p):
    return np.concatenate([p[k].reshape(-1) for k in cn.param_names()])


def unflat(v):
    p, o = {}, 0
    ref = cn.init_params(0)
    for k in cn.param_names():
        n = ref[k].size
        p[k] = v[o:o + n].reshape(ref[k].shape)
        o += n
    return p


def oracle_view(p32):
    """What the net computes with: the tensor-core layers' weights rounded to
    BF16, everything else the FP32 values."""
    q = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p32.items()}
    for name, _, _ in cn.CONVS[1:]:
        q[name + ".w"] = bf(q[name + ".w"])
    return q


def net_inputs(B, H, W, seed):
    T = np.stack([synth.target(H, W, seed + b) for b in range(B)]).astype(np.float32)
    phi = np.random.default_rng(seed).uniform(-np.pi, np.pi, (B, H, W)).astype(np.float32)
    return T, phi


def test_net_forward_loss_and_gradients_match_oracle():
    B, H, W = 2, 128, 128
    p = cn.init_params(5)
    rng = np.random.default_rng(6)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    p32 = {k: v.astype(np.float32) for k, v in p.items()}
    T, phi = net_inputs(B, H, W, 300)
    net = hg.CNN(H, W, B, seed=1)
    try:
        hg.hg_cnn_set_params(net.h, torch.from_numpy(flat(p32)).to(DEV))
        Td, Pd = torch.from_numpy(T).to(DEV), torch.from_numpy(phi).to(DEV)
        cs = torch.empty((B, H, W, 2), dtype=torch.float32, device=DEV)
        ph = torch.empty((B, H, W), dtype=torch.float32, device=DEV)
        hg.hg_cnn_forward(net.h, Td, B, cs, ph)
        loss = torch.zeros(1, dtype=torch.float64, device=DEV)
        hg.hg_cnn_gradients(net.h, Td, Pd, B, loss)
        g = torch.empty(hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
        hg.hg_cnn_get_grads(net.h, g)
        hg.hg_cnn_sync(net.h)
    finally:
        net.close()
    q = oracle_view(p32)
    T64, phi64 = T.astype(np.float64), phi.astype(np.float64)
    c, s, cache = cn.forward(q, cn.net_input(T64))
    L, dc, ds = cn.phase_loss(c, s, T64, phi64)
    gref = cn.backward(q, cache, dc, ds)
    # the same oracle storing every activation and activation gradient in BF16,
    # as the net does: its distance from the exact oracle is the noise floor
    c2, s2, cache2 = cn.forward(q, cn.net_input(T64), store=bf)
    L2, dc2, ds2 = cn.phase_loss(c2, s2, T64, phi64)
    gsim = cn.backward(q, cache2, dc2, ds2, store=bf)
    got_cs = cs.cpu().numpy().astype(np.float64)
    floor = (rel_l2(c2, c), rel_l2(s2, s))
    errs_cs = (rel_l2(got_cs[..., 0], c), rel_l2(got_cs[..., 1], s))
    print("net cs", errs_cs, "floor", floor, "loss", loss.item(), L, L2)
    assert errs_cs[0] <= 2 * floor[0] + 1e-3 and errs_cs[1] <= 2 * floor[1] + 1e-3, (errs_cs, floor)
    assert np.allclose(ph.cpu().numpy(), np.arctan2(got_cs[..., 1], got_cs[..., 0]), atol=1e-5)
    assert abs(loss.item() - L) <= 2 * abs(L2 - L) + 1e-4 * L, (loss.item(), L, L2)
    gg = unflat(g.cpu().numpy().astype(np.float64))
    errs = {k: (rel_l2(gg[k], gref[k]), rel_l2(gsim[k], gref[k])) for k in cn.param_names()}
    print("net grads (gpu, floor)", {k: (round(a, 4), round(b, 4)) for k, (a, b) in errs.items()})
    bad = {k: v for k, v in errs.items() if v[0] > 3 * v[1] + 5e-3}
    assert not bad, bad


def test_adam_step_matches_oracle():
    B, H, W = 1, 128, 128
    T, phi = net_inputs(B, H, W, 400)
    net = hg.CNN(H, W, B, seed=3)
    try:
        th0 = torch.empty(hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
        hg.hg_cnn_get_params(net.h, th0)
        Td, Pd = torch.from_numpy(T).to(DEV), torch.from_numpy(phi).to(DEV)
        g1 = torch.empty_like(th0)
        th1 = torch.empty_like(th0)
        g2 = torch.empty_like(th0)
        th2 = torch.empty_like(th0)
        hg.hg_cnn_train_step(net.h, Td, Pd, B, 1e-3)
        hg.hg_cnn_get_grads(net.h, g1)
        hg.hg_cnn_get_params(net.h, th1)
        hg.hg_cnn_train_step(net.h, Td, Pd, B, 1e-3)
        hg.hg_cnn_get_grads(net.h, g2)
        hg.hg_cnn_get_params(net.h, th2)
        hg.hg_cnn_sync(net.h)
    finally:
        net.close()
    th0, g1, th1, g2, th2 = (t.cpu().numpy().astype(np.float64) for t in (th0, g1, th1, g2, th2))
    z = np.zeros_like(th0)
    e1, m1, v1 = cn.adam_step(th0, g1, z, z, 1, 1e-3)
    e2, _, _ = cn.adam_step(th1, g2, m1, v1, 2, 1e-3)
    # FP32 arithmetic on values of size ~0.1 with steps of ~1e-3
    assert np.max(np.abs(th1 - e1)) <= 1e-6, np.max(np.abs(th1 - e1))
    assert np.max(np.abs(th2 - e2)) <= 2e-6, np.max(np.abs(th2 - e2))
    assert np.any(th1 != th0)


def test_training_lowers_the_loss_on_gs_phases():
    """A few Adam steps on a fixed batch whose labels are GS replay phases
    (the engine's own): the loss must fall."""
    B, H, W = 4, 128, 128
    T = np.stack([synth.target(H, W, 500 + b) for b in range(B)]).astype(np.float32)
    Td = torch.from_numpy(T).to(DEV)
    plan = hg.Plan(H, W, B)
    plan.run(Td, torch.zeros_like(Td), 50)
    plan.sync()
    phi = torch.empty_like(Td)
    hg.hg_get_phase(plan.h, phi)
    plan.sync()
    plan.close()
    net = hg.CNN(H, W, B, seed=9)
    losses = []
    try:
        loss = torch.zeros(1, dtype=torch.float64, device=DEV)
        for _ in range(60):
            hg.hg_cnn_train_step(net.h, Td, phi, B, 1e-3, loss)
            losses.append(loss.item())
        hg.hg_cnn_sync(net.h)
    finally:
        net.close()
    print("train losses", [round(v, 5) for v in losses])
    assert np.isfinite(losses).all()
    # Adam's first steps overshoot; after them the loss must keep falling
    assert np.mean(losses[-5:]) < 0.9 * losses[0], losses
    assert np.mean(losses[-5:]) < 0.97 * np.mean(losses[10:15]), losses


def test_checkpoint_resume_continues_training_bit_for_bit():
    B, H, W = 2, 128, 128
    T, phi = net_inputs(B, H, W, 600)
    Td, Pd = torch.from_numpy(T).to(DEV), torch.from_numpy(phi).to(DEV)
    a, b = hg.CNN(H, W, B, seed=4), hg.CNN(H, W, B, seed=5)
    try:
        for _ in range(2):
            hg.hg_cnn_train_step(a.h, Td, Pd, B, 1e-3)
        state = torch.empty(3 * hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
        step = hg.hg_cnn_get_state(a.h, state)
        hg.hg_cnn_sync(a.h)
        assert step == 2
        hg.hg_cnn_train_step(a.h, Td, Pd, B, 1e-3)
        hg.hg_cnn_set_state(b.h, state, step)
        hg.hg_cnn_train_step(b.h, Td, Pd, B, 1e-3)
        pa = torch.empty(hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
        pb = torch.empty_like(pa)
        hg.hg_cnn_get_params(a.h, pa)
        hg.hg_cnn_get_params(b.h, pb)
        hg.hg_cnn_sync(a.h)
        hg.hg_cnn_sync(b.h)
    finally:
        a.close()
        b.close()
    assert torch.equal(pa, pb)


def test_data_parallel_step_with_one_rank_is_the_fused_step():
    """warmstart.dp_train_step (gradients, the rank average, hg_cnn_apply_grads)
    with one rank equals hg_cnn_train_step bit for bit over three steps; the
    average over ranks itself is tested on two gloo ranks on CPU."""
    from paper_2008_12214_gb300 import warmstart
    B, H, W = 2, 128, 128
    T, phi = net_inputs(B, H, W, 610)
    Td, Pd = torch.from_numpy(T).to(DEV), torch.from_numpy(phi).to(DEV)
    a, b = hg.CNN(H, W, B, seed=6), hg.CNN(H, W, B, seed=6)
    try:
        g = torch.empty(hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
        la = torch.zeros(1, dtype=torch.float64, device=DEV)
        lb = torch.zeros(1, dtype=torch.float64, device=DEV)
        for _ in range(3):
            hg.hg_cnn_train_step(a.h, Td, Pd, B, 1e-3, la)
            warmstart.dp_train_step(b, Td, Pd, B, 1e-3, g, lb)
        sa = torch.empty(3 * hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
        sb = torch.empty_like(sa)
        ka = hg.hg_cnn_get_state(a.h, sa)
        kb = hg.hg_cnn_get_state(b.h, sb)
        hg.hg_cnn_sync(a.h)
        hg.hg_cnn_sync(b.h)
    finally:
        a.close()
        b.close()
    assert ka == kb == 3
    assert torch.equal(sa, sb) and torch.equal(la, lb)


def test_base_phase_equals_labels_minus_base():
    """hg_cnn_set_base_phase: with a base phase phi_b the loss and gradients
    equal those of the plain net on the labels phi - phi_b (the same float
    subtraction as in the kernel), bit for bit; the forward phase is the
    plain one plus phi_b; removing the base restores the plain net."""
    B, H, W = 2, 128, 128
    T, phi = net_inputs(B, H, W, 500)
    base = np.random.default_rng(8).uniform(0, 2 * np.pi, (H, W)).astype(np.float32)
    resid = (phi - base[None]).astype(np.float32)
    net = hg.CNN(H, W, B, seed=4)
    try:
        Td = torch.from_numpy(T).to(DEV)

        def run(label, with_base):
            hg.hg_cnn_set_base_phase(net.h, torch.from_numpy(base).to(DEV) if with_base else None)
            loss = torch.zeros(1, dtype=torch.float64, device=DEV)
            hg.hg_cnn_gradients(net.h, Td, torch.from_numpy(label).to(DEV), B, loss)
            g = torch.empty(hg.HG_CNN_NPARAMS, dtype=torch.float32, device=DEV)
            hg.hg_cnn_get_grads(net.h, g)
            ph = torch.empty((B, H, W), dtype=torch.float32, device=DEV)
            hg.hg_cnn_forward(net.h, Td, B, None, ph)
            hg.hg_cnn_sync(net.h)
            return loss.item(), g.cpu().numpy(), ph.cpu().numpy()

        Lb, gb, pb = run(phi, True)
        Lr, gr, pr = run(resid, False)
        L0, _, p0 = run(phi, False)
    finally:
        net.close()
    assert Lb == Lr and np.array_equal(gb, gr), (Lb, Lr)
    assert np.array_equal(pb, (pr + base[None]).astype(np.float32))
    assert np.array_equal(p0, pr) and L0 != Lb
