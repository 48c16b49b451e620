"""Pins of the oracle's illumination / Fresnel / amplitude-SLM / ROI functions
(Sections 2, 3 and 3.1) against hand-worked values, closed forms and
identities that do not go through the functions' own formulas."""
import os

import numpy as np
import pytest

import oracle
from paper_2008_12214_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pixels(spec):
    return [tuple(map(int, rc.split(","))) for rc in spec.split(";")]


def _roi(spec, n=4):
    if spec == "all":
        return None
    m = np.zeros((n, n), np.uint8)
    kind, arg = spec.split(":")
    if kind == "px":
        for r, c in _pixels(arg):
            m[r, c] = 1
    elif kind == "row":
        m[int(arg), :] = 1
    elif kind == "cols":
        a, b = map(int, arg.split("-"))
        m[:, a:b + 1] = 1
    return m


def load_roi_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "roi_4x4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, tgt, phase, roi, mse, amp, eff, ssim = line.split()
        rows.append((name + "-" + roi, _pixels(tgt), [float(v) for v in phase.split(";")], roi, float(mse), float(amp), float(eff),
                     float(ssim)))
    return rows


@pytest.mark.parametrize("case", load_roi_golden(), ids=lambda c: c[0])
def test_roi_metrics_hand_worked_4x4(case):
    name, pix, phase, roi, mse, amp, eff, ssim = case
    t = np.zeros((4, 4), np.float32)
    ph = np.zeros((4, 4))
    for i, (r, c) in enumerate(pix):
        t[r, c] = 1
        ph[r, c] = phase[min(i, len(phase) - 1)]
    out = oracle.modulated_run(t, ph, 1, oracle.SLM_BINARY, 2, roi=_roi(roi))
    assert abs(out["mse"][0] - mse) < 1e-15
    assert abs(out["amp_mse"][0] - amp) < 1e-15
    assert abs(out["eff"][0] - eff) < 1e-14
    assert abs(out["ssim"][0] - ssim) < 1e-13
    assert abs(out["sum_r2"][0] - 16) < 1e-12
    # the same numbers from the replay of the hologram alone
    ev = oracle.evaluate(out["holo"], t, oracle.SLM_BINARY, 2, roi=_roi(roi))
    assert np.allclose(ev[:4], [mse, amp, eff, ssim], rtol=0, atol=1e-13)


def test_ssim_closed_form_for_an_affine_copy():
    """SSIM(x, a x + b): mu_y = a mu + b, var_y = a^2 var, cov = a var."""
    rng = np.random.default_rng(1)
    x = rng.random(500)
    mu, var = x.mean(), x.var()
    c1, c2 = 1e-4, 9e-4
    for a, b in ((1.0, 0.0), (0.5, 0.1), (2.0, -0.3), (-1.0, 1.0)):
        my = a * mu + b
        expect = (2 * mu * my + c1) * (2 * a * var + c2) / ((mu * mu + my * my + c1) * (var + a * a * var + c2))
        assert abs(oracle.ssim_global(x, a * x + b) - expect) < 1e-14
    assert abs(oracle.ssim_global(x, x) - 1) < 1e-15
    y = rng.random(500)
    assert abs(oracle.ssim_global(x, y) - oracle.ssim_global(y, x)) < 1e-15


def test_roi_metrics_without_roi_are_the_plain_metrics():
    rng = np.random.default_rng(2)
    R2 = rng.random((16, 32)) ** 3
    T = oracle.prepare_target(rng.random((16, 32)).astype(np.float32) * (rng.random((16, 32)) > 0.6))
    a = oracle.roi_metrics(R2, T)
    b = oracle.metrics(R2, T)
    assert np.allclose(a[[0, 1, 2, 4]], b, rtol=1e-12, atol=0)


def test_uniform_far_field_phase_slm_is_plain_gs():
    """No illumination, no Fresnel term, no ROI: the hologram and metrics of
    plain GS (the sqrt(N) target scale does not move a phase decision)."""
    for kind, levels, n in ((oracle.SLM_BINARY, 2, 32), (oracle.SLM_LLEVEL, 8, 24)):
        t = synth.target(n, n, 31)
        ph = synth.init_phase(n, n, 31).astype(np.float64)
        a = oracle.modulated_run(t, ph, 4, kind, levels)
        b = oracle.gs_run(t, ph, 4, kind, levels)
        assert np.mean(a["holo"] != b["holo"]) <= 2.0 / (n * n)
        assert np.allclose(a["mse"], b["mse"], rtol=1e-9, atol=0)
        assert np.allclose(a["amp_mse"], b["amp_mse"], rtol=1e-9, atol=0)


@pytest.mark.parametrize("j", [1, 3])
def test_fresnel_phase_on_the_level_grid_shifts_levels_only(j):
    """Fresnel coefficient c = 2 pi j / L puts the quadratic phase on the
    L-level grid: q(y, x) = (2 pi / L) j r^2 with r^2 = (x - n/2)^2 + (y - n/2)^2.
    The quantiser then picks the far-field level minus j r^2 (mod L) and the
    light leaving the SLM, hence the whole trajectory, is the far field's."""
    L, n = 8, 16
    t = synth.target(n, n, 5)
    ph = synth.init_phase(n, n, 5).astype(np.float64)
    E = oracle.illumination(n, n, fresnel=2 * np.pi * j / L)
    a = oracle.modulated_run(t, ph, 3, oracle.SLM_LLEVEL, L, E=E)
    b = oracle.modulated_run(t, ph, 3, oracle.SLM_LLEVEL, L)
    y, x = np.mgrid[0:n, 0:n]
    r2 = (x - n // 2) ** 2 + (y - n // 2) ** 2
    assert np.mean((a["holo"].astype(int) + j * r2) % L != b["holo"]) <= 2.0 / (n * n)
    assert np.allclose(a["mse"], b["mse"], rtol=1e-9, atol=0)
    # the lens term itself: exp(i q) at the centre is 1, and one pixel off
    # the centre along x it is exp(2 pi i j / L)
    assert abs(E[n // 2, n // 2] - 1) < 1e-15
    assert abs(E[n // 2, n // 2 + 1] - np.exp(2j * np.pi * j / L)) < 1e-14


def test_a_hologram_cancelling_the_lens_focuses_on_the_centre():
    """SLM levels -j r^2 (mod L) under the Fresnel phase (2 pi / L) j r^2 emit a
    plane wave: every photon lands on the replay centre [n/2][n/2]."""
    L, n, j = 16, 32, 5
    y, x = np.mgrid[0:n, 0:n]
    r2 = (x - n // 2) ** 2 + (y - n // 2) ** 2
    holo = ((-j * r2) % L).astype(np.uint8)
    E = oracle.illumination(n, n, fresnel=2 * np.pi * j / L)
    R = np.fft.fftshift(oracle.fft2(oracle.modulated_field(holo, E, oracle.SLM_LLEVEL, L), -1))
    P = np.abs(R) ** 2
    assert abs(P[n // 2, n // 2] - n * n) < 1e-9
    assert P.sum() - P[n // 2, n // 2] < 1e-18 * n * n + 1e-12


def test_uniform_illumination_scales_and_rotates_only():
    """E = a exp(i 2 pi k / L): levels shift by -k, the replay scales by a,
    so the normalised metrics are unchanged and sum |R|^2 = a^2 N (Parseval)."""
    L, n, k, a_ = 8, 32, 3, 2.5
    t = synth.target(n, n, 9)
    ph = synth.init_phase(n, n, 9).astype(np.float64)
    E = np.full((n, n), a_ * np.exp(2j * np.pi * k / L))
    u = oracle.modulated_run(t, ph, 3, oracle.SLM_LLEVEL, L, E=E)
    v = oracle.modulated_run(t, ph, 3, oracle.SLM_LLEVEL, L)
    assert np.mean((u["holo"].astype(int) + k) % L != v["holo"]) <= 2.0 / (n * n)
    assert np.allclose(u["mse"], v["mse"], rtol=1e-9, atol=0)
    assert np.allclose(u["sum_r2"], a_ * a_ * n * n, rtol=1e-12, atol=0)


def test_gaussian_illumination_keeps_phase_decisions_and_energy():
    """A real positive illumination amplitude does not move any phase
    decision of the first iteration; the replay carries sum A^2 (Parseval)."""
    n = 32
    t = synth.target(n, n, 12)
    ph = synth.init_phase(n, n, 12).astype(np.float64)
    y, x = np.mgrid[0:n, 0:n]
    A = np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * (n / 3) ** 2))
    E = oracle.illumination(n, n, amp=A)
    g = oracle.modulated_run(t, ph, 1, oracle.SLM_BINARY, 2, E=E)
    p = oracle.modulated_run(t, ph, 1, oracle.SLM_BINARY, 2)
    assert np.array_equal(g["holo"], p["holo"])
    assert abs(g["sum_r2"][0] - (A * A).sum()) < 1e-10 * (A * A).sum()
    assert 0 < g["eff"][0] <= 1 + 1e-15  # synthetic blobs reach every pixel: support = field


def test_binary_amplitude_is_binary_phase_plus_a_zero_order():
    """Transmittance (1 + b) / 2 for the binary-phase sign b of the same h:
    level 1 exactly where the phase SLM picks 0, and
    R_amp = (R_phase + sqrt(N) delta_centre) / 2."""
    n = 32
    t = synth.target(n, n, 14)
    ph = synth.init_phase(n, n, 14).astype(np.float64)
    a = oracle.modulated_run(t, ph, 1, oracle.SLM_AMPLITUDE, 2)
    b = oracle.modulated_run(t, ph, 1, oracle.SLM_BINARY, 2)
    assert np.array_equal(a["holo"], 1 - b["holo"])
    d = np.zeros((n, n), complex)
    d[n // 2, n // 2] = n
    assert np.abs(a["R"] - (b["R"] + d) / 2).max() < 1e-12


def test_amplitude_quantiser_hand_values():
    """L = 5 levels, clip 2: v = 4 (1/2 + m / 4) with m = Re(h conj E) / |E|^2."""
    h = np.array([0, 2, -2, 1, 6, -0.5, 0.25 + 3j, -6])
    q, s = oracle.quantise_modulated(h, np.ones(h.shape, complex), oracle.SLM_AMPLITUDE, 5, 2.0)
    # m:        0  2  -2  1  6(clamped)  -0.5 (v = 1.5, half away -> 2)  0.25 (v = 2.25)  -6 (clamped)
    assert q.tolist() == [2, 4, 0, 3, 4, 2, 2, 0]
    assert np.allclose(s, q / 4.0)
    # E = 2i: m = Re(h (-2i)) / 4 = Im(h) / 2
    E = np.full(3, 2j)
    q, s = oracle.quantise_modulated(np.array([4j, -1j, 1.0]), E, oracle.SLM_AMPLITUDE, 5, 2.0)
    assert q.tolist() == [4, 2, 2]
    assert np.allclose(s, E * q / 4.0)
    # a dark pixel (E = 0) sits at v = 1/2
    q, _ = oracle.quantise_modulated(np.array([5.0]), np.zeros(1, complex), oracle.SLM_AMPLITUDE, 3, 2.0)
    assert q.tolist() == [1]


def test_phase_quantiser_under_illumination_uses_the_relative_phase():
    h = np.exp(1j * np.array([0.1, 1.7, 3.0, -1.2]))
    E = np.exp(1j * np.array([0.0, np.pi / 2, np.pi, -np.pi / 2]))
    q, s = oracle.quantise_modulated(h, E, oracle.SLM_LLEVEL, 4)
    # relative phases 0.1, 0.129, -0.14, 0.37 -> level 0 each; field = E
    assert q.tolist() == [0, 0, 0, 0]
    assert np.allclose(s, E)
    q, s = oracle.quantise_modulated(h, E, oracle.SLM_BINARY, 2)
    assert q.tolist() == [0, 0, 0, 0]


def test_outside_the_roi_the_replay_is_left_free():
    n = 16
    t = synth.target(n, n, 21)
    ph = synth.init_phase(n, n, 21).astype(np.float64)
    roi = np.zeros((n, n), np.uint8)
    roi[3:12, 5:14] = 1
    out = oracle.modulated_run(t, ph, 2, oracle.SLM_LLEVEL, 4, roi=roi)
    m = roi != 0
    assert np.array_equal(out["F"][~m], out["R"][~m])
    Tn = oracle.roi_target(t, roi)
    assert np.allclose(np.abs(out["F"][m]), n * Tn[m], rtol=1e-12, atol=1e-15)
    assert abs((Tn * Tn).sum() - 1) < 1e-14 and np.all(Tn[~m] == 0)
    full = oracle.modulated_run(t, ph, 2, oracle.SLM_LLEVEL, 4, roi=np.ones((n, n), np.uint8))
    plain = oracle.modulated_run(t, ph, 2, oracle.SLM_LLEVEL, 4)
    assert np.array_equal(full["holo"], plain["holo"]) and np.allclose(full["mse"], plain["mse"], rtol=1e-15)
