"""FP64 CPU oracle for the GS / WGS / OSPR hologram generators.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never imports it.
It shares no code with the CUDA path.  The arithmetic lives in
``hologen_oracle.c`` (plain C, double precision); this module compiles it
with gcc on first use and wraps it with ctypes, returning numpy arrays.

Every function cites the passage of arXiv:2008.12214 (HoloGen) it follows in
the C source's header (adaptive OSPR, whose feedback the paper does not spell
out, is a reading written here from the C steps).  Parity status: the FFT,
quantiser, GS step, replay and Philox are pinned by ``tests/test_oracle.py``;
the illumination / Fresnel / amplitude-SLM / region-of-interest functions
(modulated_run, evaluate, roi_metrics, ssim_global) by
``tests/test_oracle_modulation.py`` (hand-worked 4x4 ROI metrics, the SSIM
closed form for an affine copy, the level-grid Fresnel and uniform
illumination identities, binary amplitude = binary phase plus a zero order);
direct search / simulated annealing (search_run, search_delta) by
``tests/test_oracle_search.py`` (the incremental error change against full
recomputation, greedy descent to a one-flip minimum checked by enumeration,
the zero- and high-temperature limits, the tracked replay field);
the OSPR mean intensity by its closed-form expectation (the arcsine law for
the signs of Gaussian pairs), to which the time average converges as
1/sqrt(subframes); whole WGS trajectories by a hand-derived run whose
hologram is stationary while the weight compounds as sqrt(2)^k, and
adaptive-OSPR sequences by hand-derived delta targets (exact reproduction at
the replay centre; off the centre the twin's negative deficit clipped at
every subframe) -- WGS on general targets and the adaptive deficit's effect on
general targets beyond those cases rest on the single-step pins and the
qualitative checks listed there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hologen_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SLM_BINARY, SLM_LLEVEL, SLM_CONTINUOUS = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP over rows/columns)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i = ctypes.c_int
            u32 = ctypes.c_uint32
            u64 = ctypes.c_uint64
            lib.or_is_235.argtypes = [i]
            lib.or_fft1d.argtypes = [i, P, P, i]
            lib.or_fft2d.argtypes = [i, i, P, i]
            lib.or_shift2d.argtypes = [i, i, P, P, i]
            lib.or_shift2d.restype = None
            lib.or_prepare_target.argtypes = [i, P, P]
            lib.or_quantise.argtypes = [i, P, i, i, P]
            lib.or_gs_step.argtypes = [i, i, P, P, P, i, i, i, P, P, P, P, P, P]
            lib.or_gs_run.argtypes = [i, i, P, P, i, i, i, i, P, P, P, P, P, P]
            lib.or_replay.argtypes = [i, i, i, P, i, i, P]
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_philox4x32_10.restype = None
            lib.or_random_phase.argtypes = [i, i, u64, u32, u32, u32, P]
            lib.or_ospr_run.argtypes = [i, i, P, i, u64, u32, P, P, P]
            lib.or_replay_field.argtypes = [i, i, P, i, i, P]
            lib.or_metrics.argtypes = [i, P, P, P]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _ck(st):
    if st != 0:
        raise OracleError("oracle call failed with status %d" % st)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def is_235(n: int) -> bool:
    return bool(_load().or_is_235(int(n)))


def fft1d(x, sign: int = -1) -> np.ndarray:
    """Unnormalised 1D DFT, X[k] = sum_j x[j] exp(sign 2 pi i jk/n)."""
    x = _c128(x)
    out = np.empty_like(x)
    _ck(_load().or_fft1d(x.size, _p(x), _p(out), int(sign)))
    return out


def fft2(a, sign: int = -1) -> np.ndarray:
    """Unitary 2D DFT (eqs. fouriertrans2d5c/d); sign=-1 forward, +1 inverse."""
    a = _c128(a).copy()
    ny, nx = a.shape
    _ck(_load().or_fft2d(ny, nx, _p(a), int(sign)))
    return a


def shift2d(a, inverse: bool = False) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty_like(a)
    _load().or_shift2d(a.shape[0], a.shape[1], _p(a), _p(out), int(bool(inverse)))
    return out


def prepare_target(t_raw) -> np.ndarray:
    t = np.ascontiguousarray(t_raw, dtype=np.float32)
    out = np.empty(t.shape, np.float64)
    _ck(_load().or_prepare_target(t.size, _p(t), _p(out)))
    return out


def quantise(h, kind: int, levels: int = 2) -> np.ndarray:
    h = _c128(h)
    q = np.empty(h.shape, np.uint8)
    _ck(_load().or_quantise(h.size, _p(h), int(kind), int(levels), _p(q)))
    return q


def gs_step(T, phase, w=None, kind=SLM_BINARY, levels=2, wgs=False):
    """One GS/WGS iteration from state (phase, w).  T normalised, replay order.

    Returns dict(h, holo, R, mse, amp_mse, eff, sum_r2, phase, w)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    ny, nx = T.shape
    ph = np.ascontiguousarray(phase, dtype=np.float64)
    w_in = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    h = np.empty((ny, nx), np.complex128)
    holo = np.empty((ny, nx), np.uint8)
    R = np.empty((ny, nx), np.complex128)
    met = np.empty(4, np.float64)
    ph_out = np.empty((ny, nx), np.float64)
    w_out = np.empty((ny, nx), np.float64)
    _ck(_load().or_gs_step(ny, nx, _p(T), _p(ph), _p(w_in), int(kind), int(levels), int(bool(wgs)),
                           _p(h), _p(holo), _p(R), _p(met), _p(ph_out), _p(w_out)))
    return dict(h=h, holo=holo, R=R, mse=met[0], amp_mse=met[1], eff=met[2], sum_r2=met[3],
                phase=ph_out, w=w_out)


def gs_run(t_raw, phase0, iters, kind=SLM_BINARY, levels=2, wgs=False):
    """Whole GS/WGS run; returns dict(holo, mse[iters], amp_mse, eff, phase, w)."""
    t = np.ascontiguousarray(t_raw, dtype=np.float32)
    ny, nx = t.shape
    ph = np.ascontiguousarray(phase0, dtype=np.float64)
    holo = np.empty((ny, nx), np.uint8)
    mse = np.empty(iters, np.float64)
    amp = np.empty(iters, np.float64)
    eff = np.empty(iters, np.float64)
    ph_out = np.empty((ny, nx), np.float64)
    w_out = np.empty((ny, nx), np.float64)
    _ck(_load().or_gs_run(ny, nx, _p(t), _p(ph), int(iters), int(kind), int(levels), int(bool(wgs)),
                          _p(holo), _p(mse), _p(amp), _p(eff), _p(ph_out), _p(w_out)))
    return dict(holo=holo, mse=mse, amp_mse=amp, eff=eff, phase=ph_out, w=w_out)


def replay(holo, kind=SLM_BINARY, levels=2) -> np.ndarray:
    """Normalised replay intensity (sum 1, replay order); holo [count][ny][nx]
    or [ny][nx]; several holograms are time-averaged."""
    h = np.ascontiguousarray(holo, dtype=np.uint8)
    if h.ndim == 2:
        h = h[None]
    c, ny, nx = h.shape
    out = np.empty((ny, nx), np.float64)
    _ck(_load().or_replay(ny, nx, c, _p(h), int(kind), int(levels), _p(out)))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    _load().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def random_phase(ny, nx, seed, t, sub, stream) -> np.ndarray:
    """Seeded U[0, 2 pi) phase map (replay order): pixel r = y nx + x takes
    word r mod 4 of Philox4x32-10 at counter {r // 4, sub, t, stream}."""
    out = np.empty((ny, nx), np.float64)
    _ck(_load().or_random_phase(int(ny), int(nx), int(seed), int(t), int(sub), int(stream), _p(out)))
    return out


def ospr_run(t_raw, nsub, seed, t_index=0):
    """OSPR over nsub subframes; returns dict(holo[nsub], I (normalised time
    average), mse, amp_mse, eff)."""
    t = np.ascontiguousarray(t_raw, dtype=np.float32)
    ny, nx = t.shape
    holo = np.empty((nsub, ny, nx), np.uint8)
    I_out = np.empty((ny, nx), np.float64)
    met = np.empty(4, np.float64)
    _ck(_load().or_ospr_run(ny, nx, _p(t), int(nsub), int(seed), int(t_index), _p(holo), _p(I_out),
                            _p(met)))
    return dict(holo=holo, I=I_out, mse=met[0], amp_mse=met[1], eff=met[2])


def adaptive_target(T, I_prev_sum, n):
    """Target amplitude of adaptive-OSPR subframe n (1-based).  The paper
    (Section 3.4) states only that adaptive OSPR feeds the cumulative error
    back into later subframes; the reading here: after n - 1 subframes whose
    energy-normalised intensities sum to I_prev_sum, subframe n aims at the
    deficit n T^2 - I_prev_sum (T normalised to sum T^2 = 1), clipped at
    zero, so T_n = sqrt(max(n T^2 - I_prev_sum, 0)), normalised to sum 1.
    Subframe 1 is plain OSPR's first subframe."""
    D = np.maximum(n * T * T - I_prev_sum, 0.0)
    s = D.sum()
    return np.sqrt(D / s) if s > 0 else T.copy()


def adaptive_ospr_run(t_raw, nsub, seed, t_index=0):
    """Adaptive OSPR over nsub subframes (random phases as OSPR's, Philox
    counter {pixel, n, t_index, 0}); returns dict(holo[nsub], I (time-averaged
    normalised intensity), mse, amp_mse, eff)."""
    Tn = prepare_target(t_raw)
    ny, nx = Tn.shape
    acc = np.zeros((ny, nx))
    holo = np.empty((nsub, ny, nx), np.uint8)
    for n in range(1, nsub + 1):
        Tt = adaptive_target(Tn, acc, n)
        st = gs_step(Tt, random_phase(ny, nx, seed, t_index, n - 1, 0))
        holo[n - 1] = st["holo"]
        I = np.abs(st["R"]) ** 2
        acc += I / I.sum()
    m = metrics(acc / nsub, Tn)
    return dict(holo=holo, I=acc / nsub, mse=m[0], amp_mse=m[1], eff=m[2])


def lt_fraction(j, f0, grow):
    """Side fraction of the Liu-Taghizadeh window for constraint j (0 = the
    initial field): f0 growing linearly to 1 over `grow` constraints."""
    return 1.0 if grow <= 0 else min(1.0, f0 + (1.0 - f0) * j / grow)


def lt_window(ny, nx, f):
    """Centred window of replay pixels (iy, ix): |iy - ny/2| <= floor(f ny/2)
    and |ix - nx/2| <= floor(f nx/2)."""
    hy, hx = int(np.floor(f * ny / 2)), int(np.floor(f * nx / 2))
    iy = np.arange(ny)[:, None]
    ix = np.arange(nx)[None, :]
    return (np.abs(iy - ny // 2) <= hy) & (np.abs(ix - nx // 2) <= hx)


def lt_run(t_raw, phase0, iters, f0, grow, kind=SLM_BINARY, levels=2):
    """Liu-Taghizadeh GS (Section 3.2: only part of the replay field is
    targeted at first, the targeted region then grows).  Reading: a centred
    window (lt_window) of side fraction lt_fraction(k); inside it the GS
    constraint with the target carrying the replay's total energy
    (sqrt(N) T with sum T^2 = 1, unitary transforms), outside it the replay
    field is left as it is.  The initial field is the windowed target with
    phase0.  Returns dict(holo (last), mse[iters], phase (arg R, last))."""
    Tn = prepare_target(t_raw)
    ny, nx = Tn.shape
    N = ny * nx
    A = np.sqrt(N) * Tn
    F = np.where(lt_window(ny, nx, lt_fraction(0, f0, grow)), A, 0.0) * np.exp(1j * np.asarray(phase0))
    mse = np.empty(iters)
    for k in range(iters):
        h = fft2(np.fft.ifftshift(F), +1)
        H = quantise(h, kind, levels)
        step = np.pi if kind == SLM_BINARY else 2 * np.pi / levels
        R = np.fft.fftshift(fft2(np.exp(1j * step * H), -1))
        mse[k] = metrics(np.abs(R) ** 2, Tn)[0]
        mag = np.abs(R)
        ph = np.where(mag > 0, R / np.where(mag > 0, mag, 1.0), 1.0)
        F = np.where(lt_window(ny, nx, lt_fraction(k + 1, f0, grow)), A * ph, R)
    return dict(holo=H, mse=mse, phase=np.angle(R))


def replay_field(holo, kind=SLM_BINARY, levels=2) -> np.ndarray:
    """Replay field fftshift(FFT2(exp(iH))) (unitary, replay order) of one hologram."""
    h = np.ascontiguousarray(holo, dtype=np.uint8)
    ny, nx = h.shape
    out = np.empty((ny, nx), np.complex128)
    _ck(_load().or_replay_field(ny, nx, _p(h), int(kind), int(levels), _p(out)))
    return out


def metrics(R2, T):
    """(intensity MSE, amplitude MSE, efficiency, sum |R|^2) of an unnormalised
    replay intensity against a normalised target."""
    r = np.ascontiguousarray(R2, dtype=np.float64)
    t = np.ascontiguousarray(T, dtype=np.float64)
    out = np.empty(4, np.float64)
    _ck(_load().or_metrics(r.size, _p(r), _p(t), _p(out)))
    return out


# ------------------------------------------------------------------------
# Illumination, Fresnel holograms, amplitude SLMs, regions of interest
# (Sections 2 and 3.1).  Plain numpy over the pinned primitives above.

SLM_AMPLITUDE = 3


def fresnel_phase(ny, nx, c):
    """Section 2: a Fresnel (mid-field) hologram is the far-field one with an
    extra quadratic phase on the SLM plane.  Reading: q(y, x) = c ((x -
    nx//2)^2 + (y - ny//2)^2) radians, SLM pixel (y, x) in natural order, c
    in radians per squared pixel (pi dx^2 / (lambda z) for pitch dx at
    distance z; c = 0 is the far field)."""
    y = (np.arange(ny) - ny // 2)[:, None].astype(np.float64)
    x = (np.arange(nx) - nx // 2)[None, :].astype(np.float64)
    return c * (x * x + y * y)


def illumination(ny, nx, amp=None, phase=None, fresnel=0.0):
    """Field E(y, x) lighting the SLM (natural order): amplitude `amp` (1 if
    None) and phase `phase` (0 if None) plus the Fresnel term.  The Thrust
    call of Section 4 hands the quantiser the illumination's phases and
    magnitudes; the light leaving SLM pixel (y, x) is E(y, x) times the
    pixel's modulation."""
    a = np.ones((ny, nx)) if amp is None else np.asarray(amp, dtype=np.float64)
    p = np.zeros((ny, nx)) if phase is None else np.asarray(phase, dtype=np.float64)
    return a * np.exp(1j * (p + fresnel_phase(ny, nx, fresnel)))


def round_half_away(v):
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def quantise_modulated(h, E, kind, levels=2, clip=2.0):
    """Nearest SLM state for the wanted field h (unitary) under illumination E.
    Returns (levels uint8, field leaving the SLM).

    Phase SLMs (binary {0, pi} or L levels on the full circle): the state
    nearest h / E in phase, i.e. the quantiser of Section 4 applied to
    h conj(E) (its argument less the illumination's), giving E exp(i H).
    Amplitude SLMs (transmittance l / (L - 1), l < L; Fig. 1's amplitude
    modulation): the least-squares real transmittance m = Re(h conj E) /
    |E|^2 (0 where E = 0) is mapped from [-clip, clip] to [0, 1] by
    v = 1/2 + m / (2 clip) and rounded half away from zero to the nearest
    level, clamped to [0, L - 1]; the field is E l / (L - 1).  With L = 2
    that is l = 1 exactly where Re(h conj E) >= 0, whatever `clip`."""
    h = np.asarray(h, dtype=np.complex128)
    hm = h * np.conj(E)
    if kind == SLM_AMPLITUDE:
        e2 = np.abs(E) ** 2
        m = np.where(e2 > 0, hm.real / np.where(e2 > 0, e2, 1.0), 0.0)
        v = (levels - 1) * (0.5 + m / (2.0 * clip))
        q = np.clip(round_half_away(v), 0, levels - 1).astype(np.uint8)
        return q, E * (q / (levels - 1.0))
    q = quantise(hm, kind, levels)
    step = np.pi if kind == SLM_BINARY else 2 * np.pi / levels
    return q, E * np.exp(1j * step * q)


def modulated_field(holo, E, kind, levels=2):
    """Field leaving the SLM for given levels under illumination E."""
    q = np.asarray(holo, dtype=np.float64)
    if kind == SLM_AMPLITUDE:
        return E * (q / (levels - 1.0))
    step = np.pi if kind == SLM_BINARY else 2 * np.pi / levels
    return E * np.exp(1j * step * q)


def ssim_global(x, y, k1=0.01, k2=0.03, L=1.0):
    """SSIM of Section 3.1 over whole images: means, (population) variances
    and covariance of x and y, c1 = (k1 L)^2, c2 = (k2 L)^2."""
    x = np.asarray(x, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    mx, my = x.mean(), y.mean()
    vx, vy = ((x - mx) ** 2).mean(), ((y - my) ** 2).mean()
    cxy = ((x - mx) * (y - my)).mean()
    c1, c2 = (k1 * L) ** 2, (k2 * L) ** 2
    return (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2))


def roi_target(t_raw, roi=None):
    """Target restricted to the region of interest (replay order) and
    normalised there: sum over the ROI of T^2 = 1, T = 0 outside."""
    t = np.asarray(t_raw, dtype=np.float64)
    if roi is not None:
        t = np.where(np.asarray(roi) != 0, t, 0.0)
    return t / np.sqrt((t * t).sum())


def roi_metrics(R2, Tn, roi=None):
    """Metrics of Section 3.1 restricted to the region of interest, for an
    unnormalised replay intensity R2 = |R|^2 and the ROI-normalised target
    Tn (roi_target).  The scale freedom of Section 3 is taken over the ROI:
    I = |R|^2 / sum_ROI |R|^2, so sum_ROI I = sum_ROI T^2 = 1.  Returns
    (intensity MSE, amplitude MSE of eq. mse on sqrt(I) vs T, efficiency,
    SSIM, sum |R|^2): means over the ROI's pixels; efficiency = energy on
    the target's support inside the ROI over all replay energy; SSIM on the
    amplitudes T / max T and sqrt(I) / max T over the ROI (dynamic range 1)."""
    R2 = np.asarray(R2, dtype=np.float64)
    Tn = np.asarray(Tn, dtype=np.float64)
    m = np.ones(R2.shape, bool) if roi is None else np.asarray(roi) != 0
    I = R2[m] / R2[m].sum()
    t = Tn[m]
    mse = ((I - t * t) ** 2).mean()
    amp = ((np.sqrt(I) - t) ** 2).mean()
    eff = R2[m][t > 0].sum() / R2.sum()
    tmax = t.max()
    ssim = ssim_global(t / tmax, np.sqrt(I) / tmax)
    return np.array([mse, amp, eff, ssim, R2.sum()])


def modulated_run(t_raw, phase0, iters, kind=SLM_BINARY, levels=2, E=None, roi=None, clip=2.0):
    """GS (Section 3.2) with an illuminated (and Fresnel) SLM plane, phase or
    amplitude SLM levels, and a region of interest.  Readings:
      * the target is restricted to the ROI and normalised there (roi_target);
        inside the ROI the replay constraint uses sqrt(N) T (the replay's
        energy of a unit-modulus hologram, unitary transforms), outside it
        the replay field is left free (Section 3's amplitude freedom);
      * the initial field is sqrt(N) T exp(i phase0);
      * h = IFFT2(ifftshift F) is quantised by quantise_modulated under the
        illumination E (natural SLM order; uniform 1 if None), the replay is
        R = fftshift(FFT2(field leaving the SLM));
      * metrics per iteration: roi_metrics.
    Returns dict(holo (last), mse, amp_mse, eff, ssim, sum_r2 [iters], R
    (last replay field), F (the constraint field the next iteration starts
    from))."""
    Tn = roi_target(t_raw, roi)
    ny, nx = Tn.shape
    N = ny * nx
    if E is None:
        E = np.ones((ny, nx), np.complex128)
    inside = np.ones((ny, nx), bool) if roi is None else np.asarray(roi) != 0
    A = np.sqrt(N) * Tn
    F = A * np.exp(1j * np.asarray(phase0, dtype=np.float64))
    out = np.empty((5, iters))
    for k in range(iters):
        h = fft2(np.fft.ifftshift(F), +1)
        q, s = quantise_modulated(h, E, kind, levels, clip)
        R = np.fft.fftshift(fft2(s, -1))
        out[:, k] = roi_metrics(np.abs(R) ** 2, Tn, roi)
        mag = np.abs(R)
        ph = np.where(mag > 0, R / np.where(mag > 0, mag, 1.0), 1.0)
        F = np.where(inside, A * ph, R)
    return dict(holo=q, mse=out[0], amp_mse=out[1], eff=out[2], ssim=out[3], sum_r2=out[4], R=R, F=F)


def evaluate(holo, t_raw, kind=SLM_BINARY, levels=2, E=None, roi=None):
    """roi_metrics of the replay of given holograms (levels, natural order)
    under illumination E, against the ROI-normalised target."""
    q = np.asarray(holo)
    ny, nx = q.shape
    if E is None:
        E = np.ones((ny, nx), np.complex128)
    R = np.fft.fftshift(fft2(modulated_field(q, E, kind, levels), -1))
    return roi_metrics(np.abs(R) ** 2, roi_target(t_raw, roi), roi)


# ------------------------------------------------------------------------
# Holographic search algorithms (Section 3.3): direct search and simulated
# annealing over single-pixel changes of a phase hologram.

def _level_phasors(kind, levels):
    step = np.pi if kind == SLM_BINARY else 2 * np.pi / levels
    return np.exp(1j * step * np.arange(2 if kind == SLM_BINARY else levels))


def search_delta(R, T2, y, x, ds):
    """Change of the intensity MSE when SLM pixel (y, x) changes its field by
    ds (unitary replay R in replay order, T2 = T^2 normalised, sum |R|^2 = N
    for a phase hologram so I = |R|^2 / N).  The replay changes by
    dR(ky, kx) = ds exp(-2 pi i (ky y / ny + kx x / nx)) / sqrt(N) with
    (ky, kx) the frequency of replay pixel (iy, ix) = fftshift order, and
    I by a = (2 Re(R conj dR) + |dR|^2) / N, so the MSE changes by
    mean(a (2 (I - T2) + a)).  Returns (dE, dR)."""
    ny, nx = R.shape
    N = ny * nx
    ky = ((np.arange(ny) - ny // 2) % ny).astype(np.int64)
    kx = ((np.arange(nx) - nx // 2) % nx).astype(np.int64)
    ph = ((ky * y) % ny)[:, None] / ny + ((kx * x) % nx)[None, :] / nx
    dR = ds * np.exp(-2j * np.pi * ph) / np.sqrt(N)
    a = (2 * (R.real * dR.real + R.imag * dR.imag) + (dR.real ** 2 + dR.imag ** 2)) / N
    I = (R.real ** 2 + R.imag ** 2) / N
    return float(np.mean(a * (2 * (I - T2) + a))), dR


def search_run(t_raw, phase0, sweeps, kind=SLM_BINARY, levels=2, tau0=0.0, alpha=1.0, seed=0, t_index=0):
    """Direct search (tau0 = 0) and simulated annealing (Section 3.3: trial
    changes accepted when they lower Error(T, R), and under annealing also
    with a temperature-dependent probability when they raise it).  Readings:
      * the initial guess is the quantised back-propagation of the target with
        phase0 (GS's first half-step): H0 = Q(IFFT2(ifftshift(T e^{i phase0})));
      * a sweep visits every SLM pixel once in raster order (p = y nx + x);
        the trial change is the other binary level, or for L levels level
        (q + 1 + r1 mod (L - 1)) mod L;
      * Error is the intensity MSE (energy normalised);
      * accept when dE < 0, or when tau_s > 0 and u < exp(-dE / tau_s), with
        tau_s = tau0 * MSE(H0) * alpha^s for sweep s;
      * (u, r1): Philox4x32-10 words 0 and 1 at counter {p, s, t_index, 2},
        key seed; u = (word0 >> 8) 2^-24.
    Returns dict(holo, mse[sweeps] (after each sweep), accepted[sweeps],
    mse0, R (tracked replay field, replay order))."""
    Tn = prepare_target(t_raw)
    ny, nx = Tn.shape
    N = ny * nx
    h = fft2(np.fft.ifftshift(Tn * np.exp(1j * np.asarray(phase0, dtype=np.float64))), +1)
    q = quantise(h, kind, levels).astype(np.int64)
    lv = _level_phasors(kind, levels)
    R = np.fft.fftshift(fft2(lv[q], -1))
    T2 = Tn * Tn
    mse0 = float(np.mean(((R.real ** 2 + R.imag ** 2) / N - T2) ** 2))
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    mse, acc = np.empty(sweeps), np.zeros(sweeps, np.int64)
    for s in range(sweeps):
        tau = tau0 * mse0 * alpha ** s
        for p in range(N):
            y, x = divmod(p, nx)
            r = philox4x32_10(np.array([p, s, t_index, 2], np.uint32), key)
            qn = 1 - q[y, x] if kind == SLM_BINARY else (q[y, x] + 1 + int(r[1]) % (levels - 1)) % levels
            dE, dR = search_delta(R, T2, y, x, lv[qn] - lv[q[y, x]])
            u = float(int(r[0]) >> 8) * (1.0 / 16777216.0)
            if dE < 0 or (tau > 0 and u < np.exp(-dE / tau)):
                R = R + dR
                q[y, x] = qn
                acc[s] += 1
        mse[s] = np.mean(((R.real ** 2 + R.imag ** 2) / N - T2) ** 2)
    return dict(holo=q.astype(np.uint8), mse=mse, accepted=acc, mse0=mse0, R=R)
