"""The fused iteration loop, one step at a time from the oracle's state
(marked gpu).

Between its first and last iteration hg_run repeats one row pass and one
column pass; at the benchmark's sizes these are the TMA-fed paired row pass in
Hermitian form and the column-pair pass.  hg_debug_loop_step runs exactly those
launches of the plan, fed a hologram H_k.  Every test here feeds the hologram
of the oracle's own run at iteration k (Section 3.2) and checks, per sampled
target:
  * the metrics of iteration k (the replay of H_k): relative 1e-4;
  * the field the row pass leaves, against its definition (the unnormalised
    inverse row DFT of the constrained field F = w T R/|R|, or of its
    Hermitian part F_H) computed here from the oracle's replay field:
    relative L2 <= 1e-5;
  * the next hologram H_{k+1} against the oracle's next step: bit-exact except
    pixels whose back-propagated phase lies within 1e-5 rad of a decision
    boundary (counted and printed);
  * the field the column pass leaves, against the column DFT of the SLM field
    of the GPU's own H_{k+1}: relative L2 <= 1e-5;
  * WGS: the updated weights against the oracle's where I is above 1% of its
    mean (elsewhere w T / sqrt(I) divides by a near-zero |R|); the constrained
    field F (the row pass's output transformed back along x) with the GPU's
    weights on those pixels, relative L2 <= 1e-5; the next hologram against
    the quantisation of the exact inverse DFT of the GPU's own F, bit-exact
    except pixels within 1e-5 rad of a boundary or closer to it than 1e-6 of
    the field's RMS magnitude (wgs_floor_mask: the weights' dynamic range).
The plans are those the workloads use (autotuned, default options); targets
that are not sampled get seeded random holograms and only their metrics are
checked.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2008_12214_gb300 import hologen as hg
from paper_2008_12214_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
BOUND_RAD = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def boundary_mask(h, kind, levels):
    """Pixels whose phase is within 1e-5 rad of a decision boundary."""
    if kind == oracle.SLM_BINARY:
        return np.abs(h.real) <= np.sin(BOUND_RAD) * np.abs(h)
    x = np.angle(h) * levels / (2 * np.pi)
    return np.abs(x - np.floor(x) - 0.5) <= BOUND_RAD * levels / (2 * np.pi)


def wgs_floor_mask(h, kind, levels, rel=1e-6):
    """Pixels whose distance to a decision boundary, in field units, is below
    rel x the field's RMS magnitude (about ten times the FP32 transform's
    absolute error).  Weighted GS gives F a dynamic range in which a fixed
    angle band does not cover that error at pixels of small |h|."""
    floor = rel * np.sqrt(np.mean(np.abs(h) ** 2))
    if kind == oracle.SLM_BINARY:
        return np.abs(h.real) <= floor
    x = np.angle(h) * levels / (2 * np.pi)
    margin = np.abs(x - np.floor(x) - 0.5) * 2 * np.pi / levels  # rad to the boundary
    return np.abs(h) * np.sin(np.minimum(margin, np.pi / 2)) <= floor


def okind(kind):
    return oracle.SLM_BINARY if kind == hg.HG_SLM_BINARY else oracle.SLM_LLEVEL


def phasor(R):
    mag = np.abs(R)
    return np.where(mag > 0, R / np.where(mag > 0, mag, 1.0), 1.0)


def mirror(F):
    """F(-u) of an array in DFT order."""
    return np.roll(F[::-1, ::-1], 1, axis=(0, 1))


def row_field(F_rep, herm):
    """The row pass's output for a constrained field F given in replay order:
    the unnormalised inverse DFT along x of F (or of its Hermitian part) in
    DFT order."""
    nx = F_rep.shape[1]
    F = np.fft.ifftshift(F_rep)
    if herm:
        F = 0.5 * (F + np.conj(mirror(F)))
    return np.fft.ifft(F, axis=1) * nx


def col_field(E_slm):
    """The column pass's output for the field leaving the SLM (natural
    order): the unnormalised forward DFT along y."""
    return np.fft.fft(E_slm, axis=0)


def run_loop_step(plan, t, holos, k=0, weights=None):
    batch, ny, nx = t.shape
    if weights is not None:
        hg.hg_set_weights(plan.h, torch.from_numpy(weights.astype(np.float32)).to(DEV))
    T = torch.from_numpy(t).to(DEV)
    Hin = torch.from_numpy(holos).to(DEV)
    row = torch.empty((batch, ny, nx), dtype=torch.complex64, device=DEV)
    col = torch.empty((batch, ny, nx), dtype=torch.complex64, device=DEV)
    hout = torch.empty((batch, ny, nx), dtype=torch.uint8, device=DEV)
    met = torch.empty((batch, 4), dtype=torch.float64, device=DEV)
    hg.hg_debug_loop_step(plan.h, T, Hin, k, row, hout, col, met)
    plan.sync()
    out = dict(row=row.cpu().numpy(), col=col.cpu().numpy(), holo=hout.cpu().numpy(), met=met.cpu().numpy(),
               variant=(hg.hg_plan_variant(plan.h, 0), hg.hg_plan_variant(plan.h, 1)))
    if plan.algo == hg.HG_WGS:
        w = torch.empty((batch, ny, nx), dtype=torch.float32, device=DEV)
        hg.hg_get_weights(plan.h, w)
        out["w"] = w.cpu().numpy()
    return out


def oracle_state(t_raw, ph0, k, kind, levels, wgs):
    """The oracle's step k: H_k, R_k, the weights w_k it started from and
    w_{k+1}, and the next replay phase."""
    Tn = oracle.prepare_target(t_raw)
    if k == 0:
        phase, w = ph0.astype(np.float64), np.ones(Tn.shape)
    else:
        r = oracle.gs_run(t_raw, ph0.astype(np.float64), k, kind, levels, wgs)
        phase, w = r["phase"], r["w"]
    st = oracle.gs_step(Tn, phase, w if wgs else None, kind, levels, wgs)
    return dict(Tn=Tn, holo=st["holo"], R=st["R"], met=np.array([st["mse"], st["amp_mse"], st["eff"],
                                                                   st["sum_r2"]]),
                w_k=w, w_next=st["w"], phase_next=st["phase"])


def check_sample(g, b, st, kind, levels, wgs, herm, half_col, tag):
    """The per-target checks listed in the module docstring; returns the
    number of boundary pixels quantised differently."""
    ny, nx = st["Tn"].shape
    assert np.allclose(g["met"][b], st["met"], rtol=1e-4, atol=0), (tag, g["met"][b], st["met"])
    w = np.ones((ny, nx))
    good = None
    if wgs:
        R2 = np.abs(st["R"]) ** 2
        I = R2 / R2.sum()
        good = I > 1e-2 * I.mean()
        wg = g["w"][b].astype(np.float64)
        assert rel_l2(wg[good], st["w_next"][good]) <= 1e-5, (tag, "w", rel_l2(wg[good], st["w_next"][good]))
        w = wg
    F = w * st["Tn"] * phasor(st["R"])
    G = row_field(F, herm)
    rows = slice(0, ny // 2 + 1) if herm else slice(0, ny)
    if not wgs:
        e_row = rel_l2(g["row"][b][rows], G[rows])
        assert e_row <= 1e-5, (tag, "row field", e_row)
        nxt = oracle.gs_step(st["Tn"], st["phase_next"], None, kind, levels, False)
        h_next = nxt["h"]
        H_next = nxt["holo"]
        bnd = boundary_mask(h_next, kind, levels)
    else:
        # The literal weight rule divides by |R|, so the largest weights sit
        # where |R| is smallest and its phasor least determined: F's FP32
        # error concentrates on a few pixels that dominate its norm.  The
        # row pass is therefore checked on the constrained field F (its
        # output transformed back along x) where I is above 1% of its mean,
        # and the column pass on the GPU's own F: H_{k+1} against the
        # quantisation of the exact inverse DFT of that F.
        Fg = np.fft.fft(g["row"][b].astype(np.complex128), axis=1) / nx
        Fr = np.fft.ifftshift(F)
        if herm:
            Fr = 0.5 * (Fr + np.conj(mirror(Fr)))
        good = np.fft.ifftshift(good)[rows]
        e_row = rel_l2(Fg[rows][good], Fr[rows][good])
        assert e_row <= 1e-5, (tag, "constrained field where I > 1% of its mean", e_row)
        if herm:
            Fg[ny // 2 + 1:] = np.conj(mirror(Fg))[ny // 2 + 1:]
        h_next = oracle.fft2(Fg, +1)
        H_next = oracle.quantise(h_next, kind, levels)
        bnd = boundary_mask(h_next, kind, levels) | wgs_floor_mask(h_next, kind, levels)
    mism = g["holo"][b] != H_next
    assert not np.any(mism & ~bnd), (tag, "hologram mismatch off the boundary", int(np.sum(mism & ~bnd)))
    step = np.pi if kind == oracle.SLM_BINARY else 2 * np.pi / levels
    C = col_field(np.exp(1j * step * g["holo"][b].astype(np.float64)))
    crows = slice(0, ny // 2 + 1) if half_col else slice(0, ny)
    e_col = rel_l2(g["col"][b][crows], C[crows])
    assert e_col <= 1e-5, (tag, "column field", e_col)
    return int(np.sum(mism)), int(np.sum(bnd)), e_row, e_col


def random_holos(batch, ny, nx, levels, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels, (batch, ny, nx)).astype(np.uint8)


# (ny, nx, batch, kind, levels, algo, sampled targets, iterations k, seed base)
CONFIGS = [
    # the headline workload: binary GS at 1024^2, batch 64
    (1024, 1024, 64, hg.HG_SLM_BINARY, 2, hg.HG_GS, (0, 31, 63), (0, 3, 10), 1000),
    # the 2048^2 x 16 workload and the display size of the mixed batch
    (2048, 2048, 16, hg.HG_SLM_BINARY, 2, hg.HG_GS, (0, 9), (0, 3), 5000),
    (1080, 1920, 16, hg.HG_SLM_BINARY, 2, hg.HG_GS, (0, 7), (0, 3), 6000),
    (512, 512, 16, hg.HG_SLM_BINARY, 2, hg.HG_GS, (2, 15), (0, 3), 7000),
    # weighted GS: 256 levels at 1024^2, and binary (paired rows carry the update)
    (1024, 1024, 1, hg.HG_SLM_LLEVEL, 256, hg.HG_WGS, (0,), (0, 3, 10), 1000),
    (1024, 1024, 4, hg.HG_SLM_BINARY, 2, hg.HG_WGS, (1,), (0, 3), 1100),
    # L-level GS on the unpaired TMA-fed passes
    (1024, 1024, 8, hg.HG_SLM_LLEVEL, 16, hg.HG_GS, (5,), (0, 3), 1200),
]


def cfg_id(c):
    ny, nx, batch, kind, levels, algo = c[:6]
    return "%dx%dx%d-L%d-%s" % (ny, nx, batch, levels, {hg.HG_GS: "gs", hg.HG_WGS: "wgs"}[algo])


@pytest.mark.parametrize("c", CONFIGS, ids=cfg_id)
def test_loop_step_from_oracle_state(c):
    ny, nx, batch, kind, levels, algo, samples, ks, seed = c
    wgs = algo == hg.HG_WGS
    ok = okind(kind)
    t = synth.targets(batch, ny, nx, seed)
    ph0 = synth.init_phases(batch, ny, nx, seed)
    plan = hg.Plan(ny, nx, batch, kind, levels, algo)
    try:
        variant = hg.hg_plan_variant(plan.h, 0), hg.hg_plan_variant(plan.h, 1)
        herm = "+herm" in variant[0]
        half_col = "pair" in variant[0]
        if kind == hg.HG_SLM_BINARY and ny % 2 == 0:
            assert herm, variant  # the binary loop the benchmarks time
        for k in ks:
            holos = random_holos(batch, ny, nx, levels, seed + 17 * k)
            weights = np.ones((batch, ny, nx)) if wgs else None
            states = {}
            for b in samples:
                states[b] = oracle_state(t[b], ph0[b], k, ok, levels, wgs)
                holos[b] = states[b]["holo"]
                if wgs:
                    weights[b] = states[b]["w_k"]
            g = run_loop_step(plan, t, holos, k, weights)
            for b in samples:
                flips, nbnd, e_row, e_col = check_sample(g, b, states[b], ok, levels, wgs, herm, half_col,
                                                         (variant, k, b))
                print("%s k=%d target %d: row rel-L2 %.2e, column rel-L2 %.2e, %d boundary pixels, %d quantised "
                      "differently" % (variant, k, b, e_row, e_col, nbnd, flips))
            others = [b for b in range(batch) if b not in samples][:8]
            for b in others:
                ref = oracle.metrics(oracle.replay(holos[b], ok, levels) * ny * nx,
                                     oracle.prepare_target(t[b]))
                assert np.allclose(g["met"][b, :3], ref[:3], rtol=1e-4, atol=0), (k, b, g["met"][b], ref)
    finally:
        plan.close()


@pytest.mark.parametrize("n,kind,levels", [(512, hg.HG_SLM_BINARY, 2), (1024, hg.HG_SLM_BINARY, 2),
                                           (512, hg.HG_SLM_LLEVEL, 16)])
def test_liu_taghizadeh_loop_step_from_oracle_state(n, kind, levels):
    """LT: the row pass constrains the window of constraint k + 1 with the
    target carrying the replay's energy (sqrt(N) T in unitary units) and
    leaves R free outside it (see oracle.lt_run); fed the oracle's H_k for
    k = 1 and 3 (window fractions 0.4375 and 0.8125 with lt_start 0.25 over
    4 constraints)."""
    batch, f0, grow = 2, 0.25, 4
    ok = okind(kind)
    t = synth.targets(batch, n, n, 4400)
    ph0 = synth.init_phases(batch, n, n, 4400)
    plan = hg.Plan(n, n, batch, kind, levels, hg.HG_LT, lt_start=f0, lt_grow=grow)
    try:
        variant = hg.hg_plan_variant(plan.h, 0), hg.hg_plan_variant(plan.h, 1)
        herm = "+herm" in variant[0]
        half_col = "pair" in variant[0]
        N = n * n
        for k in (1, 3):
            holos = np.empty((batch, n, n), np.uint8)
            for b in range(batch):
                holos[b] = oracle.lt_run(t[b], ph0[b].astype(np.float64), k + 1, f0, grow, ok, levels)["holo"]
            g = run_loop_step(plan, t, holos, k)
            win = oracle.lt_window(n, n, oracle.lt_fraction(k + 1, f0, grow))
            for b in range(batch):
                Tn = oracle.prepare_target(t[b])
                R = oracle.replay_field(holos[b], ok, levels)
                met = oracle.metrics(np.abs(R) ** 2, Tn)
                assert np.allclose(g["met"][b], met, rtol=1e-4, atol=0), (k, b, g["met"][b], met)
                Fu = np.where(win, np.sqrt(N) * Tn * phasor(R), R)  # unitary units
                G = row_field(np.sqrt(N) * Fu, herm)
                rows = slice(0, n // 2 + 1) if herm else slice(0, n)
                e_row = rel_l2(g["row"][b][rows], G[rows])
                assert e_row <= 1e-5, (variant, k, b, e_row)
                h = oracle.fft2(np.fft.ifftshift(Fu), +1)
                H = oracle.quantise(h, ok, levels)
                mism = g["holo"][b] != H
                bnd = boundary_mask(h, ok, levels)
                assert not np.any(mism & ~bnd), (variant, k, b, int(np.sum(mism & ~bnd)))
                step = np.pi if ok == oracle.SLM_BINARY else 2 * np.pi / levels
                C = col_field(np.exp(1j * step * g["holo"][b].astype(np.float64)))
                crows = slice(0, n // 2 + 1) if half_col else slice(0, n)
                assert rel_l2(g["col"][b][crows], C[crows]) <= 1e-5
                print("LT %s k=%d target %d: row rel-L2 %.2e, %d boundary pixels, %d quantised differently"
                      % (variant, k, b, e_row, int(np.sum(bnd)), int(np.sum(mism))))
    finally:
        plan.close()
