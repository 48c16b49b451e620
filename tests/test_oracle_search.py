"""Pins of the oracle's direct search / simulated annealing (Section 3.3):
the incremental error change against full recomputation, the greedy and
local-minimum properties by brute force, the tau -> 0 and tau -> inf limits,
and the tracked replay field."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2008_12214_gb300 import synth


def full_mse(q, T2, kind, levels):
    ny, nx = q.shape
    R = np.fft.fftshift(oracle.fft2(oracle._level_phasors(kind, levels)[q], -1))
    return np.mean((np.abs(R) ** 2 / (ny * nx) - T2) ** 2), R


@pytest.mark.parametrize("kind,levels,shape", [(oracle.SLM_BINARY, 2, (8, 12)), (oracle.SLM_LLEVEL, 4, (6, 10)),
                                               (oracle.SLM_LLEVEL, 5, (9, 8))])
def test_incremental_error_change_is_the_recomputed_difference(kind, levels, shape):
    rng = np.random.default_rng(4)
    ny, nx = shape
    T2 = oracle.prepare_target(rng.random(shape).astype(np.float32)) ** 2
    q = rng.integers(0, levels, shape)
    lv = oracle._level_phasors(kind, levels)
    e0, R = full_mse(q, T2, kind, levels)
    for _ in range(25):
        y, x, qn = rng.integers(0, ny), rng.integers(0, nx), rng.integers(0, levels)
        dE, dR = oracle.search_delta(R, T2, y, x, lv[qn] - lv[q[y, x]])
        q2 = q.copy()
        q2[y, x] = qn
        e1, R1 = full_mse(q2, T2, kind, levels)
        assert abs(dE - (e1 - e0)) <= 1e-15 + 1e-12 * e0
        assert np.abs(R + dR - R1).max() < 1e-13


def test_direct_search_is_greedy_and_ends_in_a_local_minimum():
    """Accepted changes only lower the error, and once a sweep accepts
    nothing, no single-pixel change of the hologram lowers it (checked by
    recomputing every neighbour)."""
    for kind, levels in ((oracle.SLM_BINARY, 2), (oracle.SLM_LLEVEL, 3)):
        t = synth.target(6, 8, 11)
        ph = synth.init_phase(6, 8, 11).astype(np.float64)
        o = oracle.search_run(t, ph, 12, kind, levels)
        m = np.concatenate([[o["mse0"]], o["mse"]])
        assert np.all(np.diff(m) <= 1e-18)
        assert o["accepted"][-1] == 0
        T2 = oracle.prepare_target(t) ** 2
        e0, _ = full_mse(o["holo"].astype(np.int64), T2, kind, levels)
        assert abs(e0 - o["mse"][-1]) < 1e-15
        if kind != oracle.SLM_BINARY:
            continue  # an L-level sweep tries one random level per pixel, not every neighbour
        q = o["holo"].astype(np.int64)
        for y, x in itertools.product(range(6), range(8)):
            q2 = q.copy()
            q2[y, x] ^= 1
            assert full_mse(q2, T2, kind, levels)[0] >= e0 - 1e-18


def test_exhaustive_2x2_direct_search_reaches_a_one_flip_minimum():
    """All 16 binary 2x2 holograms enumerated: the search's end point has no
    better one-flip neighbour, and its error is one of the enumerated ones."""
    t = np.array([[0.2, 1.0], [0.0, 0.5]], np.float32)
    T2 = oracle.prepare_target(t) ** 2
    errs = {}
    for bits in itertools.product((0, 1), repeat=4):
        q = np.array(bits).reshape(2, 2)
        errs[bits] = full_mse(q, T2, oracle.SLM_BINARY, 2)[0]
    for seed in range(4):
        ph = np.random.default_rng(seed).uniform(0, 2 * np.pi, (2, 2))
        o = oracle.search_run(t, ph, 4)
        end = tuple(int(v) for v in o["holo"].ravel())
        assert abs(errs[end] - o["mse"][-1]) < 1e-16
        for i in range(4):
            nb = list(end)
            nb[i] ^= 1
            assert errs[tuple(nb)] >= errs[end] - 1e-18


def test_zero_temperature_annealing_is_direct_search():
    t = synth.target(8, 8, 2)
    ph = synth.init_phase(8, 8, 2).astype(np.float64)
    a = oracle.search_run(t, ph, 3, tau0=0.0, alpha=0.5, seed=9)
    b = oracle.search_run(t, ph, 3)
    assert np.array_equal(a["holo"], b["holo"]) and np.array_equal(a["mse"], b["mse"])


def test_hot_annealing_accepts_nearly_every_change_and_cooling_returns():
    t = synth.target(8, 8, 6)
    ph = synth.init_phase(8, 8, 6).astype(np.float64)
    hot = oracle.search_run(t, ph, 1, tau0=1e6, alpha=1.0, seed=1)
    assert hot["accepted"][0] >= 0.97 * 64
    cool = oracle.search_run(t, ph, 6, tau0=1e-2, alpha=0.05, seed=1)
    # by the last sweeps the temperature is negligible: the search is greedy again
    assert cool["mse"][-1] <= cool["mse"][-2] + 1e-18


def test_tracked_replay_is_the_replay_of_the_final_hologram():
    for kind, levels in ((oracle.SLM_BINARY, 2), (oracle.SLM_LLEVEL, 8)):
        t = synth.target(12, 10, 8)
        ph = synth.init_phase(12, 10, 8).astype(np.float64)
        o = oracle.search_run(t, ph, 3, kind, levels, tau0=1e-3, alpha=0.5, seed=3)
        _, R = full_mse(o["holo"].astype(np.int64), oracle.prepare_target(t) ** 2, kind, levels)
        assert np.abs(o["R"] - R).max() < 1e-12
        # the initial guess is the quantised back-propagation (GS's first half-step)
        h = oracle.fft2(np.fft.ifftshift(oracle.prepare_target(t) * np.exp(1j * ph)), +1)
        q0 = oracle.quantise(h, kind, levels).astype(np.int64)
        assert abs(full_mse(q0, oracle.prepare_target(t) ** 2, kind, levels)[0] - o["mse0"]) < 1e-18
