/*
 * hologen_oracle.c -- plain FP64 CPU oracle for the iterative Fourier-transform
 * hologram generators (Gerchberg-Saxton, weighted GS, OSPR).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * path.  Everything here is written for readability, not speed: a recursive
 * mixed-radix DFT, per-pixel loops, double precision throughout.
 *
 * Paper: "HoloGen: An open-source toolbox for high-speed hologram generation"
 * (Christopher, Kadis, Gordon, Wilkinson), arXiv:2008.12214.
 *
 * What each function follows
 *   or_fft1d / or_fft2d    Section 2, eqs. (fouriertrans2d5c/d): unitary 2D DFT,
 *                          1/sqrt(Nx Ny) in both directions, e^{-2 pi i} forward.
 *                          Evaluated by recursive decimation in time over the
 *                          prime factors 2, 3 and 5 (Section 3, the O(N log N)
 *                          remark; Cooley-Tukey).
 *   or_quantise            Section 3 (quantisation) and Fig. 1 / Listing 1
 *                          (nearest-level phase SLM).  Binary SLM {0, pi}:
 *                          level 0 iff Re h >= 0.  L-level full-circle SLM:
 *                          level = round-half-away(arg h / (2 pi / L)) mod L.
 *                          CONTINUOUS (oracle-only pin aid): phasor h/|h|.
 *   or_gs_step / or_gs_run Section 3.2 (IFTA, Gerchberg-Saxton and weighted GS),
 *                          metrics from Section 3.1 eq. (mse) plus the intensity
 *                          MSE with energy normalisation (scale freedom, Sec. 3).
 *   or_ospr_run            Section 3.4 (one-step phase retrieval, time average
 *                          of independent random-phase binary subframes).
 *   or_philox4x32_10       Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 *                          as easy as 1, 2, 3" (SC'11): the Philox4x32-10
 *                          counter-based generator, used to draw OSPR subframe
 *                          phases and default initial phases.
 *
 * Conventions (readings where the paper is silent)
 *   arrays are [ny][nx], x fastest; complex arrays interleave (re, im) doubles.
 *   The replay field is fftshift(FFT2(exp(iH))); the target lives in replay
 *   order, so the back-propagation is IFFT2(ifftshift(F)).
 *   T is normalised to sum T^2 = 1.  Replay intensity I = s |R|^2 with
 *   s = sum T^2 / sum |R|^2 (energy match).
 *   Intensity MSE = mean((I - T^2)^2); amplitude MSE (eq. mse) =
 *   mean((sqrt(I) - T)^2); efficiency = sum_{T>0} |R|^2 / sum |R|^2.
 *   Next replay phase = arg R (R == 0 -> 0).
 *   WGS: w <- w * T / sqrt(I) where T > 0 and sqrt(I) > 1e-300, else w kept.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SIZE 2
#define OR_ERR_MEM 3

enum { OR_SLM_BINARY = 0, OR_SLM_LLEVEL = 1, OR_SLM_CONTINUOUS = 2 };

static const long double OR_TWO_PI = 6.283185307179586476925286766559005768L;

/* ------------------------------------------------------------------------- */
/* Unitary DFT (Section 2, eqs. fouriertrans2d5c / fouriertrans2d5d)          */
/* ------------------------------------------------------------------------- */

static int smallest_factor(int n) {
    if (n % 2 == 0) return 2;
    if (n % 3 == 0) return 3;
    if (n % 5 == 0) return 5;
    return 0;
}

/* 1 if n >= 1 factors into 2, 3 and 5 only. */
int or_is_235(int n) {
    if (n < 1) return 0;
    while (n > 1) {
        int p = smallest_factor(n);
        if (!p) return 0;
        n /= p;
    }
    return 1;
}

/* w[e] = exp(sign * 2 pi i e / n) for e in [0, n): the angle is reduced as an
 * exact integer ratio and evaluated in long double before rounding to double. */
static cplx *twiddle_table(int n, int sign) {
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!w) return NULL;
    for (int e = 0; e < n; ++e) {
        long double a = OR_TWO_PI * (long double)e / (long double)n;
        w[e] = (double)cosl(a) + I * (double)(sign * sinl(a));
    }
    return w;
}

/*
 * Recursive decimation in time.  X[k] = sum_j x[j] W_n^{jk}, W_n = e^{sign 2pi i/n}.
 * With p the smallest prime factor of n and m = n/p, the p sub-sequences
 * x[p j + r] (r < p) are transformed to Y_r[k] (length m), then
 *   X[k + m q] = sum_r W_n^{r (k + m q)} Y_r[k],   k < m, q < p.
 * W is the table for the top-level length N; W_n^e = W[e * (N / n)].
 */
static void dft_rec(const cplx *x, ptrdiff_t stride, int n, cplx *X,
                    const cplx *W, int N) {
    if (n == 1) {
        X[0] = x[0];
        return;
    }
    int p = smallest_factor(n);
    int m = n / p;
    for (int r = 0; r < p; ++r) dft_rec(x + r * stride, stride * p, m, X + r * m, W, N);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    int step = N / n;
    for (int q = 0; q < p; ++q) {
        for (int k = 0; k < m; ++k) {
            int kk = k + m * q;
            cplx acc = 0;
            for (int r = 0; r < p; ++r) {
                long e = ((long)r * kk) % n;
                acc += W[e * step] * X[r * m + k];
            }
            tmp[kk] = acc;
        }
    }
    memcpy(X, tmp, sizeof(cplx) * (size_t)n);
    free(tmp);
}

/* Unnormalised 1D DFT of n points with exponent sign `sign` (-1 forward). */
int or_fft1d(int n, const double *in_ri, double *out_ri, int sign) {
    if (!or_is_235(n) || (sign != 1 && sign != -1)) return OR_ERR_SIZE;
    cplx *W = twiddle_table(n, sign);
    cplx *x = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *X = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!W || !x || !X) { free(W); free(x); free(X); return OR_ERR_MEM; }
    for (int j = 0; j < n; ++j) x[j] = in_ri[2 * j] + I * in_ri[2 * j + 1];
    dft_rec(x, 1, n, X, W, n);
    for (int k = 0; k < n; ++k) { out_ri[2 * k] = creal(X[k]); out_ri[2 * k + 1] = cimag(X[k]); }
    free(W); free(x); free(X);
    return OR_OK;
}

/* Unitary 2D DFT in place on a[ny][nx]: 1D transforms along every row, then
 * along every column, then a 1/sqrt(nx ny) scale (eqs. fouriertrans2d5c/d). */
static int fft2d_c(int ny, int nx, cplx *a, int sign) {
    if (!or_is_235(ny) || !or_is_235(nx)) return OR_ERR_SIZE;
    cplx *Wx = twiddle_table(nx, sign);
    cplx *Wy = twiddle_table(ny, sign);
    if (!Wx || !Wy) { free(Wx); free(Wy); return OR_ERR_MEM; }
    int err = 0;
#pragma omp parallel
    {
        int nmax = nx > ny ? nx : ny;
        cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)nmax);
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)nmax);
        int ok = line && out;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(static)
        for (int y = 0; y < ny; ++y) {
            if (!ok) continue;
            dft_rec(a + (size_t)y * nx, 1, nx, out, Wx, nx);
            memcpy(a + (size_t)y * nx, out, sizeof(cplx) * (size_t)nx);
        }
#pragma omp for schedule(static)
        for (int x = 0; x < nx; ++x) {
            if (!ok) continue;
            for (int y = 0; y < ny; ++y) line[y] = a[(size_t)y * nx + x];
            dft_rec(line, 1, ny, out, Wy, ny);
            for (int y = 0; y < ny; ++y) a[(size_t)y * nx + x] = out[y];
        }
        free(line);
        free(out);
    }
    free(Wx);
    free(Wy);
    if (err) return OR_ERR_MEM;
    double scale = 1.0 / sqrt((double)nx * (double)ny);
    for (size_t i = 0; i < (size_t)nx * ny; ++i) a[i] *= scale;
    return OR_OK;
}

int or_fft2d(int ny, int nx, double *a_ri, int sign) {
    if (sign != 1 && sign != -1) return OR_ERR_ARG;
    size_t n = (size_t)nx * ny;
    cplx *a = (cplx *)malloc(sizeof(cplx) * n);
    if (!a) return OR_ERR_MEM;
    for (size_t i = 0; i < n; ++i) a[i] = a_ri[2 * i] + I * a_ri[2 * i + 1];
    int st = fft2d_c(ny, nx, a, sign);
    for (size_t i = 0; i < n; ++i) { a_ri[2 * i] = creal(a[i]); a_ri[2 * i + 1] = cimag(a[i]); }
    free(a);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Shifts between replay order (zero frequency at the centre) and DFT order.  */
/* fftshift:  out[i] = in[(i - n/2) mod n];  ifftshift: out[i] = in[(i + n/2) mod n]
 * (integer n/2, applied along both axes).                                    */
/* ------------------------------------------------------------------------- */

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

static void shift2d_c(int ny, int nx, const cplx *in, cplx *out, int inverse) {
    int dy = inverse ? ny / 2 : -(ny / 2), dx = inverse ? nx / 2 : -(nx / 2);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            out[(size_t)y * nx + x] = in[(size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx)];
}

static void shift2d_r(int ny, int nx, const double *in, double *out, int inverse) {
    int dy = inverse ? ny / 2 : -(ny / 2), dx = inverse ? nx / 2 : -(nx / 2);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            out[(size_t)y * nx + x] = in[(size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx)];
}

/* Real-array shift exported for tests: inverse = 0 -> fftshift, 1 -> ifftshift. */
void or_shift2d(int ny, int nx, const double *in, double *out, int inverse) {
    shift2d_r(ny, nx, in, out, inverse);
}

/* ------------------------------------------------------------------------- */
/* Target preparation: T <- T / sqrt(sum T^2) (scale freedom, Section 3).     */
/* ------------------------------------------------------------------------- */

int or_prepare_target(int n, const float *t_raw, double *t_out) {
    double s = 0;
    for (int i = 0; i < n; ++i) {
        if (!(t_raw[i] >= 0.0f) || isinf(t_raw[i])) return OR_ERR_ARG;   /* NaN, <0, inf */
        s += (double)t_raw[i] * (double)t_raw[i];
    }
    if (!(s > 0)) return OR_ERR_ARG;
    double r = 1.0 / sqrt(s);
    for (int i = 0; i < n; ++i) t_out[i] = (double)t_raw[i] * r;
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* SLM quantisation (Section 3; Fig. 1; Listing 1 read as nearest level).     */
/* ------------------------------------------------------------------------- */

static double round_half_away(double v) { return v >= 0 ? floor(v + 0.5) : -floor(-v + 0.5); }

/* Level index of one back-propagated SLM-plane value h. */
static int quantise_one(cplx h, int kind, int levels) {
    if (kind == OR_SLM_BINARY) return creal(h) >= 0.0 ? 0 : 1;
    double a = atan2(cimag(h), creal(h));                 /* (-pi, pi] */
    double q = round_half_away(a / ((double)OR_TWO_PI / levels));
    int qi = (int)q % levels;
    return qi < 0 ? qi + levels : qi;
}

/* Unit phasor the SLM displays for a level index. */
static cplx level_phasor(int q, int kind, int levels) {
    if (kind == OR_SLM_BINARY) return q ? -1.0 : 1.0;
    long double a = OR_TWO_PI * (long double)q / (long double)levels;
    return (double)cosl(a) + I * (double)sinl(a);
}

static cplx slm_phasor(cplx h, int kind, int levels, uint8_t *level_out) {
    if (kind == OR_SLM_CONTINUOUS) {
        double m = cabs(h);
        if (level_out) *level_out = 0;
        return m > 0 ? h / m : 1.0;
    }
    int q = quantise_one(h, kind, levels);
    if (level_out) *level_out = (uint8_t)q;
    return level_phasor(q, kind, levels);
}

static int slm_ok(int kind, int levels) {
    if (kind == OR_SLM_BINARY) return 1;
    if (kind == OR_SLM_LLEVEL) return levels >= 2 && levels <= 256;
    return kind == OR_SLM_CONTINUOUS;
}

/* Level indices of n back-propagated values. */
int or_quantise(int n, const double *h_ri, int kind, int levels, uint8_t *q_out) {
    if (!slm_ok(kind, levels) || kind == OR_SLM_CONTINUOUS) return OR_ERR_ARG;
    for (int i = 0; i < n; ++i) q_out[i] = (uint8_t)quantise_one(h_ri[2 * i] + I * h_ri[2 * i + 1], kind, levels);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Replay field and metrics.                                                  */
/* ------------------------------------------------------------------------- */

/* R = fftshift(FFT2(e)) for an SLM-plane field e (unitary, eq. fouriertrans2d5c). */
static int replay_of(int ny, int nx, const cplx *e, cplx *R) {
    size_t n = (size_t)nx * ny;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
    if (!tmp) return OR_ERR_MEM;
    memcpy(tmp, e, sizeof(cplx) * n);
    int st = fft2d_c(ny, nx, tmp, -1);
    if (st == OR_OK) shift2d_c(ny, nx, tmp, R, 0);
    free(tmp);
    return st;
}

/* metrics[0] intensity MSE, [1] amplitude MSE (eq. mse), [2] efficiency,
 * [3] sum |R|^2, given replay intensity |R|^2 (unnormalised) and normalised T. */
static void metrics_of(size_t n, const double *R2, const double *T, double *metrics) {
    double sT2 = 0, sR2 = 0, sIn = 0;
    for (size_t i = 0; i < n; ++i) { sT2 += T[i] * T[i]; sR2 += R2[i]; if (T[i] > 0) sIn += R2[i]; }
    double s = sR2 > 0 ? sT2 / sR2 : 0.0;
    double mse = 0, amp = 0;
    for (size_t i = 0; i < n; ++i) {
        double Ii = s * R2[i];
        double d = Ii - T[i] * T[i];
        double a = sqrt(Ii) - T[i];
        mse += d * d;
        amp += a * a;
    }
    metrics[0] = mse / (double)n;
    metrics[1] = amp / (double)n;
    metrics[2] = sR2 > 0 ? sIn / sR2 : 0.0;
    metrics[3] = sR2;
}

/* ------------------------------------------------------------------------- */
/* One Gerchberg-Saxton / weighted-GS iteration (Section 3.2).                */
/* ------------------------------------------------------------------------- */

/*
 * Inputs: T (normalised, replay order), phase_in (replay order, radians),
 * w_in (WGS weights, replay order; NULL = all ones).
 *   F = w T e^{i phase}; h = IFFT2(ifftshift(F)); H = Q(h);
 *   R = fftshift(FFT2(e^{iH})); metrics; phase_out = arg R;
 *   wgs: w_out = w T / sqrt(I) where T > 0 and sqrt(I) > 1e-300.
 * Outputs (each may be NULL): h_out (SLM plane, DFT order = natural SLM
 * order), holo_out (level index), R_out (replay order, unnormalised),
 * metrics_out[4], phase_out, w_out.
 */
int or_gs_step(int ny, int nx, const double *T, const double *phase_in, const double *w_in,
               int kind, int levels, int wgs, double *h_out, uint8_t *holo_out, double *R_out,
               double *metrics_out, double *phase_out, double *w_out) {
    if (ny < 1 || nx < 1 || !T || !phase_in) return OR_ERR_ARG;
    if (!or_is_235(ny) || !or_is_235(nx)) return OR_ERR_SIZE;
    if (!slm_ok(kind, levels)) return OR_ERR_ARG;
    size_t n = (size_t)nx * ny;
    cplx *F = (cplx *)malloc(sizeof(cplx) * n);
    cplx *h = (cplx *)malloc(sizeof(cplx) * n);
    cplx *R = (cplx *)malloc(sizeof(cplx) * n);
    double *R2 = (double *)malloc(sizeof(double) * n);
    if (!F || !h || !R || !R2) { free(F); free(h); free(R); free(R2); return OR_ERR_MEM; }

    for (size_t i = 0; i < n; ++i) {
        double w = w_in ? w_in[i] : 1.0;
        F[i] = w * T[i] * cexp(I * phase_in[i]);
    }
    shift2d_c(ny, nx, F, h, 1);                       /* ifftshift */
    int st = fft2d_c(ny, nx, h, +1);                  /* inverse, unitary */
    if (st) goto done;
    if (h_out) for (size_t i = 0; i < n; ++i) { h_out[2 * i] = creal(h[i]); h_out[2 * i + 1] = cimag(h[i]); }
    for (size_t i = 0; i < n; ++i) {
        uint8_t q;
        F[i] = slm_phasor(h[i], kind, levels, &q);    /* F reused as e^{iH} */
        if (holo_out) holo_out[i] = q;
    }
    st = replay_of(ny, nx, F, R);
    if (st) goto done;
    for (size_t i = 0; i < n; ++i) R2[i] = creal(R[i]) * creal(R[i]) + cimag(R[i]) * cimag(R[i]);
    double met[4];
    metrics_of(n, R2, T, met);
    if (metrics_out) memcpy(metrics_out, met, sizeof met);
    if (R_out) for (size_t i = 0; i < n; ++i) { R_out[2 * i] = creal(R[i]); R_out[2 * i + 1] = cimag(R[i]); }
    if (phase_out)
        for (size_t i = 0; i < n; ++i) phase_out[i] = (R2[i] > 0) ? carg(R[i]) : 0.0;
    if (w_out) {
        double s = met[3] > 0 ? 1.0 / met[3] : 0.0;   /* sum T^2 = 1 */
        for (size_t i = 0; i < n; ++i) {
            double w = w_in ? w_in[i] : 1.0;
            double amp = sqrt(s * R2[i]);
            w_out[i] = (wgs && T[i] > 0 && amp > 1e-300) ? w * T[i] / amp : w;
        }
    }
done:
    free(F); free(h); free(R); free(R2);
    return st;
}

/*
 * A whole GS / WGS run of `iters` iterations from phase0 (replay order).
 * t_raw: raw non-negative target in replay order (normalised here).
 * Per iteration k: mse_out[k] (intensity MSE), amp_out[k] (eq. mse),
 * eff_out[k]; after the run: holo_out (last hologram), phase_out (arg of the
 * last replay field), w_out (weights after the last update).  Any output may
 * be NULL.
 */
int or_gs_run(int ny, int nx, const float *t_raw, const double *phase0, int iters, int kind,
              int levels, int wgs, uint8_t *holo_out, double *mse_out, double *amp_out,
              double *eff_out, double *phase_out, double *w_out) {
    if (ny < 1 || nx < 1 || iters < 1 || !t_raw || !phase0) return OR_ERR_ARG;
    size_t n = (size_t)nx * ny;
    double *T = (double *)malloc(sizeof(double) * n);
    double *ph = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    double *w2 = (double *)malloc(sizeof(double) * n);
    if (!T || !ph || !w || !w2) { free(T); free(ph); free(w); free(w2); return OR_ERR_MEM; }
    int st = or_prepare_target((int)n, t_raw, T);
    if (st) goto done;
    memcpy(ph, phase0, sizeof(double) * n);
    for (size_t i = 0; i < n; ++i) w[i] = 1.0;
    for (int k = 0; k < iters; ++k) {
        double met[4];
        st = or_gs_step(ny, nx, T, ph, w, kind, levels, wgs, NULL,
                        k == iters - 1 ? holo_out : NULL, NULL, met, ph, w2);
        if (st) goto done;
        memcpy(w, w2, sizeof(double) * n);
        if (mse_out) mse_out[k] = met[0];
        if (amp_out) amp_out[k] = met[1];
        if (eff_out) eff_out[k] = met[2];
    }
    if (phase_out) memcpy(phase_out, ph, sizeof(double) * n);
    if (w_out) memcpy(w_out, w, sizeof(double) * n);
done:
    free(T); free(ph); free(w); free(w2);
    return st;
}

/* Normalised replay intensity s|R|^2 (sum = 1), replay order, of a hologram of
 * level indices.  `count` holograms of one target are averaged (OSPR time
 * average, Section 3.4); count = 1 for a single hologram. */
int or_replay(int ny, int nx, int count, const uint8_t *holo, int kind, int levels, double *I_out) {
    if (ny < 1 || nx < 1 || count < 1 || !holo || !I_out) return OR_ERR_ARG;
    if (!slm_ok(kind, levels) || kind == OR_SLM_CONTINUOUS) return OR_ERR_ARG;
    size_t n = (size_t)nx * ny;
    cplx *e = (cplx *)malloc(sizeof(cplx) * n);
    cplx *R = (cplx *)malloc(sizeof(cplx) * n);
    if (!e || !R) { free(e); free(R); return OR_ERR_MEM; }
    for (size_t i = 0; i < n; ++i) I_out[i] = 0;
    int st = OR_OK;
    for (int c = 0; c < count; ++c) {
        for (size_t i = 0; i < n; ++i) e[i] = level_phasor(holo[c * n + i], kind, levels);
        st = replay_of(ny, nx, e, R);
        if (st) break;
        for (size_t i = 0; i < n; ++i) I_out[i] += creal(R[i]) * creal(R[i]) + cimag(R[i]) * cimag(R[i]);
    }
    if (st == OR_OK) {
        double s = 0;
        for (size_t i = 0; i < n; ++i) s += I_out[i];
        for (size_t i = 0; i < n; ++i) I_out[i] = s > 0 ? I_out[i] / s : 0.0;
    }
    free(e); free(R);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11).                                      */
/* ------------------------------------------------------------------------- */

/* Ten rounds of the Philox 4x32 bijection on counter c under key k.  Each
 * round multiplies words 0 and 2 by the Philox constants, mixes the high
 * halves with words 1, 3 and the key, and the key is bumped by the Weyl
 * constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Seeded random phase in [0, 2 pi) for every replay pixel (y, x), replay order.
 * Pixel r = y*nx + x takes output word (r mod 4) of one generator call per
 * group of four consecutive pixels:
 *   w = philox(ctr = {floor(r / 4), sub, t, stream}, key = {seed lo, seed hi})
 *   u = (w[r mod 4] >> 8) * 2^-24,  phase = 2 pi u.
 * stream 0: OSPR subframe `sub` of target t; stream 1: GS initial phase.
 * (The paper asks only for random phases, Section 3.4; the counter layout is
 * this implementation's.)
 */
int or_random_phase(int ny, int nx, uint64_t seed, uint32_t t, uint32_t sub, uint32_t stream,
                    double *phase_out) {
    if (ny < 1 || nx < 1 || !phase_out) return OR_ERR_ARG;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (size_t i = 0; i < (size_t)nx * ny; ++i) {
        uint32_t ctr[4] = {(uint32_t)(i / 4), sub, t, stream}, r[4];
        or_philox4x32_10(ctr, key, r);
        double u = (double)(r[i % 4] >> 8) * (1.0 / 16777216.0);
        phase_out[i] = (double)(OR_TWO_PI * (long double)u);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* OSPR (Section 3.4): nsub independent binary subframes, time-averaged.      */
/* ------------------------------------------------------------------------- */

/*
 * For subframe n < nsub: phase_n from or_random_phase(seed, t_index, n, 0);
 * F = T e^{i phase_n}; h = IFFT2(ifftshift(F)); binary H; R_n = fftshift(FFT2(e^{iH})).
 * I_avg = mean_n |R_n|^2, normalised to sum 1; metrics of I_avg against T
 * (metrics_out[4] as in or_gs_step, with |R|^2 replaced by I_avg).
 * holo_out [nsub][ny][nx] and I_out (normalised I_avg, replay order) may be NULL.
 */
int or_ospr_run(int ny, int nx, const float *t_raw, int nsub, uint64_t seed, uint32_t t_index,
                uint8_t *holo_out, double *I_out, double *metrics_out) {
    if (ny < 1 || nx < 1 || nsub < 1 || !t_raw) return OR_ERR_ARG;
    size_t n = (size_t)nx * ny;
    double *T = (double *)malloc(sizeof(double) * n);
    double *ph = (double *)malloc(sizeof(double) * n);
    double *Rri = (double *)malloc(sizeof(double) * 2 * n);
    double *acc = (double *)calloc(n, sizeof(double));
    if (!T || !ph || !Rri || !acc) { free(T); free(ph); free(Rri); free(acc); return OR_ERR_MEM; }
    int st = or_prepare_target((int)n, t_raw, T);
    for (int s = 0; s < nsub && st == OR_OK; ++s) {
        st = or_random_phase(ny, nx, seed, t_index, (uint32_t)s, 0, ph);
        if (st) break;
        st = or_gs_step(ny, nx, T, ph, NULL, OR_SLM_BINARY, 2, 0, NULL,
                        holo_out ? holo_out + (size_t)s * n : NULL, Rri, NULL, NULL, NULL);
        if (st) break;
        for (size_t i = 0; i < n; ++i) acc[i] += Rri[2 * i] * Rri[2 * i] + Rri[2 * i + 1] * Rri[2 * i + 1];
    }
    if (st == OR_OK) {
        for (size_t i = 0; i < n; ++i) acc[i] /= (double)nsub;
        double met[4];
        metrics_of(n, acc, T, met);
        if (metrics_out) memcpy(metrics_out, met, sizeof met);
        if (I_out) {
            double s = met[3] > 0 ? 1.0 / met[3] : 0.0;
            for (size_t i = 0; i < n; ++i) I_out[i] = acc[i] * s;
        }
    }
    free(T); free(ph); free(Rri); free(acc);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Helpers for checking a given hologram.                                     */
/* ------------------------------------------------------------------------- */

/* Replay field R = fftshift(FFT2(e^{iH})) (unitary, replay order) of one
 * hologram of level indices. */
int or_replay_field(int ny, int nx, const uint8_t *holo, int kind, int levels, double *R_out) {
    if (ny < 1 || nx < 1 || !holo || !R_out) return OR_ERR_ARG;
    if (!slm_ok(kind, levels) || kind == OR_SLM_CONTINUOUS) return OR_ERR_ARG;
    size_t n = (size_t)nx * ny;
    cplx *e = (cplx *)malloc(sizeof(cplx) * n);
    cplx *R = (cplx *)malloc(sizeof(cplx) * n);
    if (!e || !R) { free(e); free(R); return OR_ERR_MEM; }
    for (size_t i = 0; i < n; ++i) e[i] = level_phasor(holo[i], kind, levels);
    int st = replay_of(ny, nx, e, R);
    if (st == OR_OK)
        for (size_t i = 0; i < n; ++i) { R_out[2 * i] = creal(R[i]); R_out[2 * i + 1] = cimag(R[i]); }
    free(e); free(R);
    return st;
}

/* metrics[4] (as in or_gs_step) of an unnormalised replay intensity R2 against
 * a normalised target T. */
int or_metrics(int n, const double *R2, const double *T, double *metrics_out) {
    if (n < 1 || !R2 || !T || !metrics_out) return OR_ERR_ARG;
    metrics_of((size_t)n, R2, T, metrics_out);
    return OR_OK;
}
