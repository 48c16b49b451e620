"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong shift or normalisation)
fails at least one of them.  CPU only.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2008_12214_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sizes_235(limit):
    return [n for n in range(1, limit + 1) if oracle.is_235(n)]


def brute_dft(x, sign):
    """O(n^2) DFT from the definition, exact integer angle reduction."""
    n = x.size
    jk = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(sign * 2j * np.pi * jk / n) @ x


# ---------------------------------------------------------------- FFT (Sec. 2)

@pytest.mark.parametrize("n", sizes_235(60))
def test_fft1d_matches_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        ref = brute_dft(x, sign)
        got = oracle.fft1d(x, sign)
        assert np.linalg.norm(got - ref) <= 1e-13 * max(1.0, np.linalg.norm(ref))


def test_fft1d_rejects_other_primes():
    with pytest.raises(oracle.OracleError):
        oracle.fft1d(np.ones(7, complex))
    assert not oracle.is_235(14) and oracle.is_235(1080) and oracle.is_235(1920)


@pytest.mark.parametrize("ny,nx", [(1, 1), (4, 4), (6, 10), (8, 12), (30, 16), (9, 25), (2, 60)])
def test_fft2_definition_and_library(ny, nx):
    rng = np.random.default_rng(ny * 100 + nx)
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    # eq. fouriertrans2d5c: u pairs with x (columns), v with y (rows), unitary
    Ky = np.exp(-2j * np.pi * (np.outer(np.arange(ny), np.arange(ny)) % ny) / ny)
    Kx = np.exp(-2j * np.pi * (np.outer(np.arange(nx), np.arange(nx)) % nx) / nx)
    ref = Ky @ a @ Kx.T / np.sqrt(nx * ny)
    got = oracle.fft2(a, -1)
    assert np.abs(got - ref).max() < 1e-12
    assert np.abs(got - np.fft.fft2(a, norm="ortho")).max() < 1e-12
    inv = oracle.fft2(a, +1)
    assert np.abs(inv - np.fft.ifft2(a, norm="ortho")).max() < 1e-12


@pytest.mark.parametrize("ny,nx", [(16, 16), (30, 20), (60, 64), (27, 40)])
def test_fft2_parseval_inverse_delta_tone(ny, nx):
    rng = np.random.default_rng(7)
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    A = oracle.fft2(a, -1)
    assert abs(np.sum(np.abs(A) ** 2) - np.sum(np.abs(a) ** 2)) < 1e-10 * np.sum(np.abs(a) ** 2)
    assert np.abs(oracle.fft2(A, +1) - a).max() < 1e-12
    d = np.zeros((ny, nx), complex)
    d[0, 0] = 1
    assert np.abs(oracle.fft2(d) - 1 / np.sqrt(nx * ny)).max() < 1e-14
    # shifted delta -> pure tone e^{-2 pi i (u x0/Nx + v y0/Ny)} / sqrt(N)
    y0, x0 = ny // 3, nx // 5
    d = np.zeros((ny, nx), complex)
    d[y0, x0] = 1
    v = np.arange(ny)[:, None]
    u = np.arange(nx)[None, :]
    tone = np.exp(-2j * np.pi * ((u * x0 % nx) / nx + (v * y0 % ny) / ny)) / np.sqrt(nx * ny)
    assert np.abs(oracle.fft2(d) - tone).max() < 1e-14


@pytest.mark.parametrize("ny,nx", [(4, 4), (6, 10), (5, 9), (8, 3)])
def test_shifts_match_numpy(ny, nx):
    a = np.arange(ny * nx, dtype=float).reshape(ny, nx)
    assert np.array_equal(oracle.shift2d(a, inverse=False), np.fft.fftshift(a))
    assert np.array_equal(oracle.shift2d(a, inverse=True), np.fft.ifftshift(a))


@pytest.mark.parametrize("ny,nx", [(8, 8), (6, 10), (30, 16)])
def test_fftshift_is_checkerboard_modulation_for_even_sizes(ny, nx):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    chk = (-1.0) ** np.add.outer(np.arange(ny), np.arange(nx))
    A = oracle.fft2(a)
    shifted = oracle.shift2d(A.real) + 1j * oracle.shift2d(A.imag)
    assert np.abs(oracle.fft2(a * chk) - shifted).max() < 1e-12


# ------------------------------------------------------ target preparation

def test_prepare_target_normalises_and_rejects_bad_values():
    t = synth.target(32, 48, 5)
    T = oracle.prepare_target(t)
    assert abs(np.sum(T * T) - 1) < 1e-14
    assert np.allclose(T / T.max(), t / t.max(), rtol=1e-7)
    for bad in (-1.0, np.nan, np.inf):
        t2 = t.copy()
        t2[3, 3] = bad
        with pytest.raises(oracle.OracleError):
            oracle.prepare_target(t2)
    with pytest.raises(oracle.OracleError):
        oracle.prepare_target(np.zeros((4, 4), np.float32))


# ------------------------------------------------------------- quantiser

def test_binary_quantiser_is_sign_of_real_part():
    h = np.array([1 + 0j, -1 + 0j, 0j, 1e-300 + 5j, -1e-300 - 5j, 0.3 - 2j, -0.3 + 2j])
    assert list(oracle.quantise(h, oracle.SLM_BINARY)) == [0, 1, 0, 0, 1, 0, 1]


def test_llevel_quantiser_nearest_level_and_wrap():
    L = 8
    step = 2 * np.pi / L
    # exactly on every level, slightly off, the wrap at -pi/pi, and h = 0
    angles = np.concatenate([np.arange(L) * step, np.arange(L) * step + 0.4 * step,
                             np.arange(L) * step - 0.4 * step])
    h = np.exp(1j * angles)
    q = oracle.quantise(h, oracle.SLM_LLEVEL, L)
    assert list(q[:L]) == list(range(L))
    assert list(q[L:2 * L]) == list(range(L))
    assert list(q[2 * L:]) == list(range(L))
    assert oracle.quantise(np.array([0j]), oracle.SLM_LLEVEL, L)[0] == 0
    assert oracle.quantise(np.array([-1 + 0j]), oracle.SLM_LLEVEL, L)[0] == L // 2
    # 256 levels as in the weighted-GS configuration
    rng = np.random.default_rng(1)
    a = rng.uniform(-np.pi, np.pi, 5000)
    q = oracle.quantise(np.exp(1j * a), oracle.SLM_LLEVEL, 256).astype(int)
    err = np.angle(np.exp(1j * (a - q * 2 * np.pi / 256)))
    assert np.abs(err).max() <= np.pi / 256 + 1e-12


def test_llevel_round_half_away_from_zero():
    L = 4
    # arg exactly half-way between levels 0 and 1 (pi/4) and between 0 and 3 (-pi/4)
    h = np.array([1 + 1j, 1 - 1j])
    q = oracle.quantise(h, oracle.SLM_LLEVEL, L)
    assert list(q) == [1, 3]


# ------------------------------------------- hand-worked 4x4 GS iterations

def load_gs_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "gs_4x4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, slm, levels, rc, phase, holo, mse, amp, eff = line.split()
        r, c = map(int, rc.split(","))
        rows.append((name, slm, int(levels), r, c, float(phase),
                     np.array([int(ch) for ch in holo]).reshape(4, 4), float(mse), float(amp),
                     float(eff)))
    return rows


@pytest.mark.parametrize("case", load_gs_golden(), ids=lambda c: c[0])
def test_gs_step_hand_worked_4x4(case):
    name, slm, levels, r, c, phase, holo, mse, amp, eff = case
    t = np.zeros((4, 4), np.float32)
    t[r, c] = 1
    T = oracle.prepare_target(t)
    ph = np.zeros((4, 4))
    ph[r, c] = phase
    kind = oracle.SLM_BINARY if slm == "binary" else oracle.SLM_LLEVEL
    out = oracle.gs_step(T, ph, kind=kind, levels=levels, wgs=True)
    assert np.array_equal(out["holo"], holo)
    assert abs(out["mse"] - mse) < 1e-15
    assert abs(out["amp_mse"] - amp) < 1e-15
    assert abs(out["eff"] - eff) < 1e-14
    assert abs(out["sum_r2"] - 16) < 1e-12          # Parseval: unit-modulus hologram
    if name == "twin_image":
        w = np.ones((4, 4))
        w[2, 3] = np.sqrt(2)
        assert np.abs(out["w"] - w).max() < 1e-14
        I = oracle.replay(out["holo"])
        expect = np.zeros((4, 4))
        expect[2, 3] = expect[2, 1] = 0.5
        assert np.abs(I - expect).max() < 1e-15


def test_wgs_run_hand_worked_twin_image():
    """A whole WGS trajectory derived by hand (binary 4x4, the twin_image case
    of the golden file): the target's single pixel at replay [2][3] with phase
    pi/4.  Each iteration's field is w T e^{i arg R} at that pixel only, so h
    keeps the phases e^{i(pi/4 + pi x/2)} (scaled by w / 4), the hologram stays
    the golden one and the replay splits equally into the pixel and its twin
    [2][1]: I = 1/2 at both and MSE 1/32 at every iteration.  The weight there
    compounds, w_k = w_{k-1} T / sqrt(I) = sqrt(2)^k, and the replay phase
    stays pi/4 at [2][3], -pi/4 at [2][1] and 0 where R = 0."""
    t = np.zeros((4, 4), np.float32)
    t[2, 3] = 1
    ph = np.zeros((4, 4))
    ph[2, 3] = np.pi / 4
    holo = np.array([int(ch) for ch in "0110011001100110"]).reshape(4, 4)
    for k in (1, 2, 3, 5):
        run = oracle.gs_run(t, ph, k, kind=oracle.SLM_BINARY, wgs=True)
        assert np.allclose(run["mse"], 1 / 32, rtol=1e-13, atol=0), run["mse"]
        assert np.array_equal(run["holo"], holo)
        w = np.ones((4, 4))
        w[2, 3] = np.sqrt(2) ** k
        assert np.abs(run["w"] - w).max() < 1e-13 * w.max()
        expect = np.zeros((4, 4))
        expect[2, 3], expect[2, 1] = np.pi / 4, -np.pi / 4
        assert np.abs(run["phase"] - expect).max() < 1e-14
        assert np.allclose(run["eff"], 0.5, rtol=1e-14)


def test_adaptive_ospr_hand_worked_deltas():
    """Adaptive OSPR sequences derived by hand on 4x4 binary targets, for any
    random phases.  A delta at the replay centre is reproduced exactly by every
    subframe (h is constant, H constant, R = 4 at the centre), so each deficit
    target equals T and the time average is T^2: MSE 0.  A delta off the centre
    (replay [2][3]) always splits into itself and its twin [2][1], I = 1/2 at
    both; the deficit at the twin, (n + 1) 0 - S < 0, is clipped to zero, so
    every later subframe aims at the same delta, and the time average keeps
    I = 1/2 at both pixels: MSE 1/32."""
    for r, c, mse in ((2, 2, 0.0), (2, 3, 1 / 32)):
        t = np.zeros((4, 4), np.float32)
        t[r, c] = 1
        for seed in (3, 11):
            out = oracle.adaptive_ospr_run(t, 5, seed, 1)
            assert abs(out["mse"] - mse) < 1e-15, (r, c, seed, out["mse"])
            expect = np.zeros((4, 4))
            if (r, c) == (2, 2):
                expect[2, 2] = 1.0
            else:
                expect[2, 3] = expect[2, 1] = 0.5
            assert np.abs(out["I"] - expect).max() < 1e-15
            for n in range(5):
                Tn = oracle.adaptive_target(oracle.prepare_target(t), out["I"] * n, n + 1) if n else None
                if Tn is not None:
                    assert np.isfinite(Tn).all() and abs(Tn[r, c] - 1.0) < 1e-15
                # each subframe's hologram depends on the column only (h has one frequency)
                assert (out["holo"][n] == out["holo"][n][0]).all()


def test_gs_step_delta_target_any_phase():
    rng = np.random.default_rng(0)
    t = np.zeros((8, 8), np.float32)
    t[4, 4] = 3
    T = oracle.prepare_target(t)
    for _ in range(5):
        out = oracle.gs_step(T, rng.uniform(0, 2 * np.pi, (8, 8)))
        assert out["mse"] < 1e-30 and abs(out["eff"] - 1) < 1e-15


# ------------------------------------------------- properties of GS / OSPR

def test_unquantised_gs_error_is_non_increasing():
    """Error-reduction property (Fienup 1982): with the continuous phase
    projection the replay-plane amplitude error never grows, for any fixed
    scale of T."""
    ny, nx = 24, 30
    t = synth.target(ny, nx, 11)
    T = oracle.prepare_target(t)
    ph = synth.init_phase(ny, nx, 11).astype(np.float64)
    errs = {1.0: [], np.sqrt(ny * nx): []}
    for _ in range(30):
        out = oracle.gs_step(T, ph, kind=oracle.SLM_CONTINUOUS)
        for c in errs:
            errs[c].append(np.sum((np.abs(out["R"]) - c * T) ** 2))
        ph = out["phase"]
    for c, e in errs.items():
        e = np.array(e)
        assert np.all(np.diff(e) <= 1e-12 * e[:-1]), (c, e)
        assert e[-1] < e[0]


def test_binary_replay_is_centro_symmetric():
    ny, nx = 16, 20
    t = synth.target(ny, nx, 4)
    out = oracle.gs_step(oracle.prepare_target(t), synth.init_phase(ny, nx, 4))
    I = np.abs(out["R"]) ** 2
    # replay centre is (ny/2, nx/2): (i, j) <-> (ny - i, nx - j) mod size
    ii = (-np.arange(ny)) % ny
    jj = (-np.arange(nx)) % nx
    assert np.abs(I - I[ii][:, jj]).max() < 1e-12
    I2 = oracle.replay(out["holo"])
    assert abs(I2.sum() - 1) < 1e-14
    assert np.abs(I2 - I / I.sum()).max() < 1e-15


def test_llevel_with_many_levels_approaches_continuous():
    ny, nx = 16, 16
    T = oracle.prepare_target(synth.target(ny, nx, 2))
    ph = synth.init_phase(ny, nx, 2).astype(np.float64)
    cont = oracle.gs_step(T, ph, kind=oracle.SLM_CONTINUOUS)
    prev = None
    for L in (4, 16, 64, 256):
        q = oracle.gs_step(T, ph, kind=oracle.SLM_LLEVEL, levels=L)
        d = np.linalg.norm(q["R"] - cont["R"]) / np.linalg.norm(cont["R"])
        assert d <= 2 * np.pi / L          # each pixel's phase error is <= pi/L
        if prev is not None:
            assert d < prev
        prev = d


def test_wgs_evens_out_uniform_spots():
    """Qualitative weighted-GS check: on an array of equal spots WGS leaves a
    smaller spread of spot intensities than plain GS."""
    ny, nx = 32, 32
    t = np.zeros((ny, nx), np.float32)
    spots = [(8, 8), (8, 20), (20, 8), (20, 20), (14, 26), (26, 14), (12, 12)]
    for (r, c) in spots:
        t[r, c] = 1
    ph0 = synth.init_phase(ny, nx, 9).astype(np.float64)
    res = {}
    for wgs in (False, True):
        out = oracle.gs_run(t, ph0, 40, kind=oracle.SLM_CONTINUOUS, wgs=wgs)
        T = oracle.prepare_target(t)
        o = oracle.gs_step(T, out["phase"], w=out["w"], kind=oracle.SLM_CONTINUOUS, wgs=wgs)
        I = np.abs(o["R"]) ** 2
        v = np.array([I[r, c] for (r, c) in spots])
        res[wgs] = v.std() / v.mean()
    assert res[True] < res[False]


def test_gs_run_equals_repeated_steps():
    ny, nx = 12, 10
    t = synth.target(ny, nx, 3)
    ph0 = synth.init_phase(ny, nx, 3).astype(np.float64)
    run = oracle.gs_run(t, ph0, 4, kind=oracle.SLM_LLEVEL, levels=16, wgs=True)
    T = oracle.prepare_target(t)
    ph, w = ph0, None
    for k in range(4):
        o = oracle.gs_step(T, ph, w=w, kind=oracle.SLM_LLEVEL, levels=16, wgs=True)
        assert o["mse"] == run["mse"][k]
        ph, w = o["phase"], o["w"]
    assert np.array_equal(o["holo"], run["holo"])
    assert np.array_equal(ph, run["phase"]) and np.array_equal(w, run["w"])


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(s, 16) for s in line.split()]
        assert list(oracle.philox4x32_10(v[0:4], v[4:6])) == v[6:10]


def test_random_phase_layout_and_range():
    ph = oracle.random_phase(4, 6, 0x1234_5678_9ABC, 3, 5, 0)
    key = [0x5678_9ABC, 0x1234]
    # one generator call per four consecutive replay pixels, pixel i taking word i mod 4
    for i in (0, 1, 2, 3, 7, 22, 23):
        r = oracle.philox4x32_10([i // 4, 5, 3, 0], key)
        assert ph.flat[i] == pytest.approx(2 * np.pi * (int(r[i % 4]) >> 8) / 2 ** 24, abs=1e-15)
    # the four words of a call are independent draws: no two pixels of a group coincide
    assert len(set(np.round(ph.flat[:4], 12))) == 4
    big = oracle.random_phase(512, 512, 7, 0, 0, 0)
    assert big.min() >= 0 and big.max() < 2 * np.pi
    sigma = 2 * np.pi / np.sqrt(12) / 512          # std of the mean of U[0, 2 pi)
    assert abs(big.mean() - np.pi) < 5 * sigma


def test_ospr_time_average_and_reciprocal_law():
    """Section 3.4: the time-averaged replay of N independent subframes has an
    MSE that falls as 1/N towards the binary floor: fit MSE(N) = a + c/N."""
    ny, nx = 32, 32
    t = synth.target(ny, nx, 21)
    Ns = [1, 2, 4, 8, 16, 24]
    mses = []
    for N in Ns:
        out = oracle.ospr_run(t, N, seed=99, t_index=0)
        mses.append(out["mse"])
        if N == 4:
            I = oracle.replay(out["holo"])
            assert np.abs(I - out["I"]).max() < 1e-15
            ii = (-np.arange(ny)) % ny
            assert np.abs(I - I[ii][:, ii]).max() < 1e-15
    mses = np.array(mses)
    A = np.stack([np.ones(len(Ns)), 1.0 / np.array(Ns)], 1)
    (a, c), *_ = np.linalg.lstsq(A, mses, rcond=None)
    fit = A @ np.array([a, c])
    assert c > 0 and a > 0
    assert np.abs(fit - mses).max() < 0.1 * (mses[0] - mses[-1])


def test_replay_field_and_metrics_helpers_agree_with_step():
    ny, nx = 12, 20
    T = oracle.prepare_target(synth.target(ny, nx, 8))
    for kind, L in ((oracle.SLM_BINARY, 2), (oracle.SLM_LLEVEL, 8)):
        o = oracle.gs_step(T, synth.init_phase(ny, nx, 8), kind=kind, levels=L)
        R = oracle.replay_field(o["holo"], kind, L)
        assert np.abs(R - o["R"]).max() < 1e-13
        m = oracle.metrics(np.abs(R) ** 2, T)
        assert np.allclose(m, [o["mse"], o["amp_mse"], o["eff"], o["sum_r2"]], rtol=1e-12, atol=0)


def test_device_target_generator_matches_the_numpy_one():
    torch = pytest.importorskip("torch")
    from paper_2008_12214_gb300 import synth
    a = synth.targets(3, 64, 96, 4242)
    b = synth.targets_device(3, 64, 96, 4242, "cpu").numpy()
    assert b.shape == a.shape and b.dtype == np.float32
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_adaptive_target_rule():
    """Adaptive OSPR's subframe target: an ideal history (each earlier
    subframe delivered exactly T^2) leaves T unchanged; the deficit is
    clipped at zero; the result is normalised."""
    rng = np.random.default_rng(21)
    T = oracle.prepare_target(rng.random((8, 8)))
    for n in (1, 2, 5):
        Tn = oracle.adaptive_target(T, (n - 1) * T * T, n)
        assert np.allclose(Tn, T, atol=1e-15)
    prev = 3 * T * T
    prev[0, 0] = 10.0  # over-delivered pixel: nothing more asked there
    Tn = oracle.adaptive_target(T, prev, 4)
    assert Tn[0, 0] == 0.0
    assert (Tn ** 2).sum() == pytest.approx(1.0, abs=1e-12)
    d = np.maximum(4 * T * T - prev, 0)
    assert np.allclose(Tn, np.sqrt(d / d.sum()), atol=1e-15)


def test_adaptive_ospr_first_subframe_is_ospr():
    t = synth.target(32, 32, 31)
    a, o = oracle.adaptive_ospr_run(t, 1, 7, 2), oracle.ospr_run(t, 1, 7, 2)
    assert np.array_equal(a["holo"], o["holo"])
    assert a["mse"] == pytest.approx(o["mse"], rel=1e-12)
    a3, o3 = oracle.adaptive_ospr_run(t, 3, 7, 2), oracle.ospr_run(t, 3, 7, 2)
    assert np.array_equal(a3["holo"][0], o3["holo"][0])
    assert not np.array_equal(a3["holo"][2], o3["holo"][2])  # the feedback changes later subframes
    assert np.allclose(a3["I"], sum(oracle.replay(a3["holo"][n]) for n in range(3)) / 3, rtol=1e-12,
                       atol=1e-18)


def test_adaptive_ospr_feedback_lowers_the_time_averaged_error():
    ratios = []
    for b in range(4):
        t = synth.target(32, 32, 2000 + b)
        ratios.append(oracle.adaptive_ospr_run(t, 12, 7, b)["mse"] / oracle.ospr_run(t, 12, 7, b)["mse"])
    assert np.mean(ratios) < 0.8, ratios


def test_lt_window_and_growth():
    W = oracle.lt_window(8, 12, 0.5)
    assert W.sum() == 5 * 7 and W[4, 6] and W[2, 3] and not W[1, 6] and not W[4, 2]
    assert oracle.lt_window(8, 12, 1.0).all()
    assert [oracle.lt_fraction(j, 0.25, 3) for j in range(5)] == [0.25, 0.5, 0.75, 1.0, 1.0]
    W = oracle.lt_window(16, 16, 0.5)
    assert np.array_equal(W, W[::-1, ::-1][np.r_[-1, 0:15]][:, np.r_[-1, 0:15]])  # symmetric under u -> -u


def test_lt_with_a_full_window_is_gs():
    """A window covering the field from the start makes LT plain GS (the
    target's scale does not change a binary or L-level hologram)."""
    t = synth.target(32, 32, 61)
    ph = synth.init_phase(32, 32, 61).astype(np.float64)
    for kind, levels in ((oracle.SLM_BINARY, 2), (oracle.SLM_LLEVEL, 8)):
        lt = oracle.lt_run(t, ph, 4, 1.0, 0, kind, levels)
        gs = oracle.gs_run(t, ph, 4, kind=kind, levels=levels)
        assert np.allclose(lt["mse"], gs["mse"], rtol=1e-9)
        assert np.array_equal(lt["holo"], gs["holo"])


def test_lt_leaves_the_field_outside_the_window_free():
    """With the window frozen at its initial size, iterations only constrain
    the window: the replay outside it is whatever the hologram gives, so the
    error inside the window falls below plain GS's there."""
    t = synth.target(32, 32, 62)
    ph = synth.init_phase(32, 32, 62).astype(np.float64)
    Tn = oracle.prepare_target(t)
    W = oracle.lt_window(32, 32, 0.5)
    lt = oracle.lt_run(t, ph, 12, 0.5, 10 ** 9, oracle.SLM_LLEVEL, 64)
    gs = oracle.gs_run(t, ph, 12, kind=oracle.SLM_LLEVEL, levels=64)

    def win_err(holo):
        I = oracle.replay(holo, oracle.SLM_LLEVEL, 64)
        I_w = I[W] / I[W].sum()
        T_w = Tn[W] ** 2 / (Tn[W] ** 2).sum()
        return np.mean((I_w - T_w) ** 2)

    assert win_err(lt["holo"]) < win_err(gs["holo"])


def test_ospr_mean_intensity_follows_the_arcsine_law():
    """The expected replay of binary OSPR subframes in closed form.  With an
    i.i.d. uniform random phase, h = IFFT2(T e^{i phi}) is (by the central
    limit theorem) circular Gaussian with E[h(x) conj h(x + d)] = C(d) =
    (1/N) sum_u T(u)^2 e^{-2 pi i u d / N}, so Re h has correlation rho(d) =
    Re C(d) / C(0), and the signs b = sign(Re h) of the binary hologram have
    E[b(x) b(x + d)] = (2 / pi) arcsin(rho(d)) (the arcsine law for Gaussian
    pairs).  Then E|R(u)|^2 = sum_d (2 / pi) arcsin(rho(d)) e^{-2 pi i u d / N}.
    The oracle's time average converges to it as 1 / sqrt(subframes)."""
    t = synth.target(32, 32, 77)
    T = oracle.prepare_target(t)
    Td = np.fft.ifftshift(T)
    C = np.fft.fft2(Td * Td) / T.size
    rho = np.real(C) / np.real(C[0, 0])
    P = np.fft.fftshift(np.real(np.fft.fft2((2 / np.pi) * np.arcsin(np.clip(rho, -1, 1)))))
    E = P / P.sum()
    err = []
    for nsub in (2000, 8000):
        I = oracle.ospr_run(t, nsub, 5)["I"]
        err.append(np.linalg.norm(I - E) / np.linalg.norm(E))
    assert err[0] < 0.03 and err[1] < 0.015, err
    assert err[1] < 0.7 * err[0]  # the subframe noise averages out


# --------------------------------------------- GS labels for the warm start


@pytest.mark.parametrize("kind,levels", [(oracle.SLM_BINARY, 2), (oracle.SLM_LLEVEL, 256)])
def test_gs_phase_keeps_the_memory_of_its_start(kind, levels):
    """The warm start's labels are replay phases after 200 GS iterations
    (Section 3.2) grown from one seeded start phase shared by every target.
    GS changes the phase only partly: on the target's support, weighted by
    T^2, the phasor exp(i(phi_200 - phi_0)) still averages to a magnitude near
    0.7, while the GS-200 phases grown from two independent starts are
    uncorrelated (as are the starts themselves).  A label is therefore
    dominated by the shared start, a fixed position-dependent random field
    that a translation-equivariant network cannot produce from the target."""
    n = 128
    a = synth.init_phase(n, n, 1).astype(np.float64)
    b = synth.init_phase(n, n, 2).astype(np.float64)
    t = synth.target(n, n, 1000)
    T = oracle.prepare_target(t)
    w = T * T / np.sum(T * T)

    def corr(x, y):
        return abs(np.sum(w * np.exp(1j * (x - y))))

    pa = oracle.gs_run(t, a, 200, kind, levels)["phase"]
    pb = oracle.gs_run(t, b, 200, kind, levels)["phase"]
    assert corr(pa, a) > 0.6 and corr(pb, b) > 0.6, (corr(pa, a), corr(pb, b))
    assert corr(pa, pb) < 0.1 and corr(a, b) < 0.1, (corr(pa, pb), corr(a, b))


def test_a_useful_gs_start_carries_the_labels_pixel_scale_detail():
    """What a warm start would have to predict (256-level SLM, 128^2): GS
    started from a target's own GS-200 phase (grown from the shared start
    phi_0) is below the GS-100 MSE of a random start after one iteration,
    while phi_0 corrected only by the label's remainder exp(i(phi_200 - phi_0))
    averaged over 2 x 2 blocks needs more than half of those 100 iterations:
    the part of the label that GS adds to phi_0 is pixel-scale."""
    n, kind, levels = 128, oracle.SLM_LLEVEL, 256
    phi0 = synth.init_phase(n, n, 1).astype(np.float64)
    for s in range(2):
        t = synth.target(n, n, 1000 + s)
        T = oracle.prepare_target(t)
        goal = oracle.gs_run(t, synth.init_phase(n, n, 5000 + s).astype(np.float64), 100, kind, levels)["mse"][-1]
        label = oracle.gs_run(t, phi0, 200, kind, levels)["phase"]
        assert oracle.gs_run(t, label, 1, kind, levels)["mse"][0] < 0.99 * goal
        r = np.exp(1j * (label - phi0)) * (T > 0)
        r2 = np.repeat(np.repeat(r.reshape(n // 2, 2, n // 2, 2).mean(axis=(1, 3)), 2, 0), 2, 1)
        mse = oracle.gs_run(t, phi0 + np.angle(r2 + 1e-30), 100, kind, levels)["mse"]
        hit = np.nonzero(mse <= goal)[0]
        assert len(hit) == 0 or hit[0] >= 50, hit[:1]
