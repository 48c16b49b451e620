// hg_kernels.cuh -- the fused passes of one GS / WGS / OSPR iteration.
//
// The field lives in DFT order as complex64 [item][ny][nx].  One iteration of
// Section 3.2 (Gerchberg-Saxton) is two passes over it:
//   row pass    : FFT of every row (completing R = FFT2(e^{iH}) of eq.
//                 fouriertrans2d5c), the metrics of Section 3.1 and the replay
//                 amplitude constraint F = w T R/|R| (+ weight update for
//                 weighted GS), then the inverse FFT of every row (starting
//                 h = IFFT2(F), eq. fouriertrans2d5d);
//   column pass : inverse FFT of every column (completing h), quantisation to
//                 the SLM levels (Section 3, Fig. 1), then the FFT of every
//                 column of e^{iH}.
// HEAD starts a run (F from the target and the initial phase), TAIL ends it
// (last metrics, replay phase), AVG time-averages subframe intensities
// (OSPR, Section 3.4, and replay of given holograms).
// Every kernel is persistent: a grid of whole-GPU size walks the panels
// (LINES rows, or C columns, of one item) in a fixed order.
#pragma once
#include "hg_fft.cuh"

namespace hg {

enum RowRole { ROW_HEAD = 0, ROW_ITER = 1, ROW_TAIL = 2, ROW_AVG = 3, ROW_ADAPT = 4, ROW_ADFIN = 5 };
enum ColRole { COL_GS_BIN = 0, COL_GS_LVL = 1, COL_HOLO_BIN = 2, COL_HOLO_LVL = 3, COL_GS_MOD = 4, COL_HOLO_MOD = 5 };

constexpr int NMET = 4;  // per-panel partial sums: (I-T^2)^2, (sqrt I - T)^2, |R|^2 in T>0, |R|^2

struct RowArgs {
    int ny, nx;
    int items;             // line sets: targets (ITER/TAIL/AVG) or chains (HEAD)
    int nsub;              // chains per target (OSPR subframes), 1 otherwise
    float2 *field;         // [chains][ny][nx] DFT order
    const float *T;        // prepared targets [targets][ny][nx], DFT order, sum T^2 = 1
    float *w;              // weighted-GS weights [targets][ny][nx] DFT order, or null
    const float *phase;    // HEAD: initial replay phase (replay order) or null = Philox
    uint32_t seed_lo, seed_hi, stream_id;
    int item0;  // Philox target index of item 0 (a chunk of a larger batch starts past 0)
    double *part;          // metric partials [targets][panels][NMET] or null
    float *phase_out;      // TAIL: arg R, replay order, or null
    float2 *R_out;         // TAIL: replay field, replay order, unitary scale, or null
    float *I_out;          // AVG: normalised intensity, replay order, or null
    const float2 *tw;      // W_nx^e, e < nx (forward roots)
    float invN, invN2, NN, invSqrtN;
    int herm;              // paired binary rows: write only the Hermitian part of F (rows y <= ny/2)
    float *acc;            // ADAPT / ADFIN: summed normalised intensities [targets][ny][nx], DFT order
    int sub;               // ADAPT: subframes delivered so far (index of the next one)
    // Liu-Taghizadeh window (HEAD / ITER): lt_amp > 0 constrains only replay pixels
    // within lt_hy rows and lt_hx columns of the centre, with the target scaled by
    // lt_amp; the field outside stays free.  lt_amp == 0: plain GS.
    float lt_amp;
    int lt_hy, lt_hx;
    // Modulated plans (illuminated / Fresnel / amplitude SLM, region of
    // interest): gen != 0 scores iterations with the eight sums of
    // gen_sums8 (the replay energy is not known in advance), and roi (DFT
    // order, shared by the items; null = the whole field) limits the replay
    // constraint, with lt_amp as the target scale
    const uint8_t *roi;
    int gen;
};

constexpr int NMET_GEN = 8;  // modulated plans: per-panel sums, see the metrics of ROW_ITER

// Is DFT-order pixel (y, x) inside the Liu-Taghizadeh window?  Its replay
// offsets from the centre are min(y, ny - y) and min(x, nx - x).
__device__ __forceinline__ bool lt_in(const RowArgs &a, int y, int x) {
    return min(y, a.ny - y) <= a.lt_hy && min(x, a.nx - x) <= a.lt_hx;
}

struct ColArgs {
    int ny, nx;
    int items;
    float2 *field;
    uint8_t *holo;         // GS: hologram out (null = skip); HOLO: hologram in
    float2 *h_out;         // GS: SLM-plane field before quantisation (unitary), or null
    const float2 *lvl;     // L-level phasors exp(2 pi i q / L)
    int levels;
    float qscale;          // L / (2 pi)
    const float2 *tw;      // W_ny^e, e < ny
    float invSqrtN;
    int half;              // store only rows y <= ny/2 of the result (binary GS whose next
                           // row pass rebuilds rows ny - y from the Hermitian symmetry)
    int half_in;           // the field holds rows y <= ny/2 of a field whose columns are
                           // Hermitian: read those, take row ny - y as conj(row y)
    // MOD roles: illumination E of the SLM plane (natural order [ny][nx]),
    // SLM kind (0 binary phase, 1 L-level phase, 2 amplitude with lvl[q] =
    // q / (L - 1)) and the amplitude map's gain 1 / (2 clip N)
    const float2 *illum;
    int kind;
    float amp_gain;
};

// Sum four per-thread float partials over the block in a fixed order (lanes
// in float, warps in double) and store them at dst (thread 0).  All threads
// must call.
__device__ __forceinline__ void block_sum4(float a0, float a1, float a2, float a3, double *red,
                                           double *dst, int nthreads) {
    float d[NMET] = {a0, a1, a2, a3};
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
        for (int m = 0; m < NMET; ++m) d[m] += __shfl_down_sync(0xffffffffu, d[m], off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < NMET; ++m) red[warp * NMET + m] = (double)d[m];
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[NMET] = {0, 0, 0, 0};
        for (int w = 0; w < (nthreads + 31) / 32; ++w)
#pragma unroll
            for (int m = 0; m < NMET; ++m) s[m] += red[w * NMET + m];
#pragma unroll
        for (int m = 0; m < NMET; ++m) dst[m] = s[m];
    }
    __syncthreads();
}

template <class P, int LINES>
struct RowCfg {
    static constexpr int THREADS = P::TL * LINES;
    static constexpr bool WARP_SYNC = (P::TL <= 32) && (32 % P::TL == 0);
    static_assert(THREADS % 32 == 0, "row CTA must be whole warps");
    static constexpr size_t SMEM =
        sizeof(float2) * LINES * P::SLOTS + sizeof(double) * NMET * (THREADS / 32);
};

template <class P, int C>
struct ColCfg {
    static constexpr int THREADS = P::TL * C;
    static_assert(THREADS % 32 == 0, "column CTA must be whole warps");
    static constexpr size_t SMEM = sizeof(float2) * C * P::SLOTS;
};

// --------------------------------------------------------------- row pass
// H: Hermitian form of HEAD / AVG (binary OSPR): rows y <= ny/2 only, each
// with its mirror row ny - y (see herm_constrain).  Kernels: k_row (H false)
// and k_row_h (H true), sharing this body.
template <class P, int ROLE, int LINES, bool H>
__device__ __forceinline__ void row_body(const RowArgs &a) {
    using Cfg = RowCfg<P, LINES>;
    constexpr int TL = P::TL, E = P::E, NX = P::N;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    double *red = reinterpret_cast<double *>(sm + LINES * P::SLOTS);
    const int tid = threadIdx.x;
    const int line = tid / TL, t = tid - line * TL;
    float2 *smb = sm + line * P::SLOTS;
    auto sync = []() {
        if constexpr (Cfg::WARP_SYNC) __syncwarp();
        else __syncthreads();
    };
    const int ny = a.ny;
    const int rows = H ? ny / 2 + 1 : ny;
    const int ppt = (rows + LINES - 1) / LINES;
    const int total = a.items * ppt;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int item = p / ppt, pan = p - item * ppt;
        const int y = pan * LINES + line;
        const bool act = y < rows;
        const int yc = act ? y : rows - 1;
        const int iy = (yc + ny / 2) % ny;  // replay row of DFT row yc
        float2 v[E];
        if constexpr (ROLE == ROW_HEAD) {
            const int b = item / a.nsub, sub = item - b * a.nsub;
            const float *Tr = a.T + ((size_t)b * ny + yc) * NX;
            const float *wr = a.w ? a.w + ((size_t)b * ny + yc) * NX : nullptr;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int x = t + TL * e;
                const int ix = (x + NX / 2) % NX;
                float amp = Tr[x];
                if (wr) amp *= wr[x];
                if (a.lt_amp > 0.f) amp = lt_in(a, yc, x) ? amp * a.lt_amp : 0.f;
                float s, c;
                if (a.phase) {
                    // phase in half-turns: the reduction is exact, no large-argument path
                    sincospif(__ldg(a.phase + ((size_t)b * ny + iy) * NX + ix) * 0.318309886183790672f,
                              &s, &c);
                } else {
                    sincospif(philox_phase2u((uint32_t)(iy * NX + ix), (uint32_t)sub, (uint32_t)(a.item0 + b),
                                             a.stream_id, a.seed_lo, a.seed_hi),
                              &s, &c);  // pi * 2u
                }
                v[e] = make_float2(amp * c, amp * s);
                if constexpr (H) {  // F_H = (F(u) + conj F(-u)) / 2, u' = (ny - y, nx - x)
                    const int ym = (ny - yc) % ny, iym = (ym + ny / 2) % ny;
                    const int xm = (NX - x) % NX, ixm = (xm + NX / 2) % NX;
                    float snm, csm;
                    if (a.phase) {
                        sincospif(__ldg(a.phase + ((size_t)b * ny + iym) * NX + ixm) * 0.318309886183790672f,
                                  &snm, &csm);
                    } else {
                        sincospif(philox_phase2u((uint32_t)(iym * NX + ixm), (uint32_t)sub, (uint32_t)(a.item0 + b),
                                                 a.stream_id, a.seed_lo, a.seed_hi),
                                  &snm, &csm);
                    }
                    float am = a.T[((size_t)b * ny + ym) * NX + xm];
                    if (a.w) am *= a.w[((size_t)b * ny + ym) * NX + xm];
                    v[e] = make_float2(0.5f * fmaf(am, csm, v[e].x), 0.5f * fmaf(-am, snm, v[e].y));
                }
            });
            line_fft<P, +1, 1>(v, smb, a.tw, t, sync);
            if (act) {
                float2 *fr = a.field + ((size_t)item * ny + y) * NX;
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    fr[t + TL * e] = v[e];
                });
            }
        } else if constexpr (ROLE == ROW_ITER || ROLE == ROW_TAIL) {
            const float2 *fr = a.field + ((size_t)item * ny + yc) * NX;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                v[e] = fr[t + TL * e];
            });
            line_fft<P, -1, 1>(v, smb, a.tw, t, sync);
            const float *Tr = a.T + ((size_t)item * ny + yc) * NX;
            float *wr = a.w ? a.w + ((size_t)item * ny + yc) * NX : nullptr;
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            float acc4 = 0.f, acc5 = 0.f, acc6 = 0.f, acc7 = 0.f;
            const uint8_t *roir = a.roi ? a.roi + (size_t)yc * NX : nullptr;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int x = t + TL * e;
                const float Tv = act ? Tr[x] : 0.f;
                const float2 r = v[e];
                const float m2 = fmaf(r.x, r.x, r.y * r.y);  // |R|^2 before the 1/N scale
                const float e2 = m2 * a.invN;                 // unitary |R|^2
                const bool in = !roir || roir[x] != 0;
                if (a.gen) {
                    // sums over the ROI of e2, e2^2, e2 T^2, sqrt(e2) T and e2 on T > 0,
                    // e2 over the field, T^4 and T^2; the intensity scale (ROI
                    // energy match) is applied when the panels are combined
                    if (act) {
                        acc5 += e2;
                        if (in) {
                            const float t2 = Tv * Tv;
                            acc0 += e2;
                            acc1 = fmaf(e2, e2, acc1);
                            acc2 = fmaf(e2, t2, acc2);
                            acc3 = fmaf(sqrtf(e2), Tv, acc3);
                            if (Tv > 0.f) acc4 += e2;
                            acc6 = fmaf(t2, t2, acc6);
                            acc7 += t2;
                        }
                    }
                } else {
                    const float I = m2 * a.invN2;  // normalised intensity
                    const float d = I - Tv * Tv;
                    const float am = sqrtf(I) - Tv;
                    if (act) {
                        acc0 = fmaf(d, d, acc0);
                        acc1 = fmaf(am, am, acc1);
                        acc3 += e2;
                        if (Tv > 0.f) acc2 += e2;
                    }
                }
                const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
                float wv = 1.f;
                if (wr) {
                    wv = act ? wr[x] : 1.f;
                    if (Tv > 0.f && m2 > 0.f) wv = wv * Tv * (a.NN * rs);  // w T / sqrt(I)
                    if (act) wr[x] = wv;
                }
                if constexpr (ROLE == ROW_ITER) {
                    if (a.lt_amp > 0.f && (!in || !lt_in(a, yc, x))) {
                        v[e] = r;  // outside the window / region of interest: left free
                    } else {
                        const float g = (a.lt_amp > 0.f ? a.lt_amp : 1.f) * Tv * wv;
                        v[e] = m2 > 0.f ? make_float2(g * r.x * rs, g * r.y * rs) : make_float2(g, 0.f);
                    }
                } else {
                    if (act) {
                        const int ix = (x + NX / 2) % NX;
                        const size_t o = ((size_t)item * ny + iy) * NX + ix;
                        if (a.phase_out) a.phase_out[o] = m2 > 0.f ? atan2f(r.y, r.x) : 0.f;
                        if (a.R_out) a.R_out[o] = make_float2(r.x * a.invSqrtN, r.y * a.invSqrtN);
                    }
                }
            });
            if constexpr (ROLE == ROW_ITER) {
                line_fft<P, +1, 1>(v, smb, a.tw, t, sync);
                if (act) {
                    float2 *fw = a.field + ((size_t)item * ny + y) * NX;
                    static_for<0, E>([&](auto ec) {
                        constexpr int e = decltype(ec)::value;
                        fw[t + TL * e] = v[e];
                    });
                }
            }
            if (a.part) {
                if (a.gen) {
                    double *dst = a.part + ((size_t)item * ppt + pan) * NMET_GEN;
                    block_sum4(acc0, acc1, acc2, acc3, red, dst, Cfg::THREADS);
                    block_sum4(acc4, acc5, acc6, acc7, red, dst + NMET, Cfg::THREADS);
                } else {
                    block_sum4(acc0, acc1, acc2, acc3, red,
                               a.part + ((size_t)item * ppt + pan) * NMET, Cfg::THREADS);
                }
            }
        } else if constexpr (ROLE == ROW_ADAPT || ROLE == ROW_ADFIN) {
            // adaptive OSPR: replay of the subframe just quantised, its normalised
            // intensity added to the running sum; ADAPT then forms the next
            // subframe's target from the deficit sqrt(max((sub + 1) T^2 - sum, 0))
            // with its random phase and starts its inverse FFT; ADFIN scores the
            // time average sum / nsub
            const float2 *fr = a.field + ((size_t)item * ny + yc) * NX;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                v[e] = fr[t + TL * e];
            });
            line_fft<P, -1, 1>(v, smb, a.tw, t, sync);
            const float *Tr = a.T + ((size_t)item * ny + yc) * NX;
            float *ar = a.acc + ((size_t)item * ny + yc) * NX;
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            const float inv_sub = 1.0f / (float)a.nsub;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int x = t + TL * e;
                const float m2 = fmaf(v[e].x, v[e].x, v[e].y * v[e].y);
                const float sum = (act ? ar[x] : 0.f) + m2 * a.invN2;
                const float Tv = act ? Tr[x] : 0.f;
                if constexpr (ROLE == ROW_ADAPT) {
                    if (act) ar[x] = sum;
                    const float amp = sqrtf(fmaxf(fmaf((float)(a.sub + 1), Tv * Tv, -sum), 0.f));
                    const int ix = (x + NX / 2) % NX;
                    float s, c;
                    sincospif(philox_phase2u((uint32_t)(iy * NX + ix), (uint32_t)a.sub, (uint32_t)(a.item0 + item),
                                             a.stream_id, a.seed_lo, a.seed_hi),
                              &s, &c);  // pi * 2u
                    v[e] = make_float2(amp * c, amp * s);
                } else {
                    const float I = sum * inv_sub;
                    if (act && a.I_out) a.I_out[((size_t)item * ny + iy) * NX + (x + NX / 2) % NX] = I;
                    if (act) {
                        const float d = I - Tv * Tv;
                        const float am = sqrtf(I) - Tv;
                        const float e2 = I * a.NN;  // unitary |R|^2 of the average
                        acc0 = fmaf(d, d, acc0);
                        acc1 = fmaf(am, am, acc1);
                        acc3 += e2;
                        if (Tv > 0.f) acc2 += e2;
                    }
                }
            });
            if constexpr (ROLE == ROW_ADAPT) {
                line_fft<P, +1, 1>(v, smb, a.tw, t, sync);
                if (act) {
                    float2 *fw = a.field + ((size_t)item * ny + y) * NX;
                    static_for<0, E>([&](auto ec) {
                        constexpr int e = decltype(ec)::value;
                        fw[t + TL * e] = v[e];
                    });
                }
            } else if (a.part) {
                block_sum4(acc0, acc1, acc2, acc3, red, a.part + ((size_t)item * ppt + pan) * NMET, Cfg::THREADS);
            }
        } else {  // ROW_AVG
            float acc[E];
            static_for<0, E>([&](auto ec) { acc[decltype(ec)::value] = 0.f; });
            for (int n = 0; n < a.nsub; ++n) {
                const float2 *fr = a.field + ((size_t)(item * a.nsub + n) * ny + yc) * NX;
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    v[e] = fr[t + TL * e];
                });
                line_fft<P, -1, 1>(v, smb, a.tw, t, sync);
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    acc[e] = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, acc[e]));
                });
            }
            const float inv_sub = 1.0f / (float)a.nsub;
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            const float *Tr = a.T ? a.T + ((size_t)item * ny + yc) * NX : nullptr;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int x = t + TL * e;
                const float I = acc[e] * inv_sub * a.invN2;
                if (act && a.I_out) {
                    const int ix = (x + NX / 2) % NX;
                    a.I_out[((size_t)item * ny + iy) * NX + ix] = I;
                }
                if (Tr && act) {
                    const float Tv = Tr[x];
                    const float d = I - Tv * Tv;
                    const float am = sqrtf(I) - Tv;
                    const float e2 = acc[e] * inv_sub * a.invN;
                    acc0 = fmaf(d, d, acc0);
                    acc1 = fmaf(am, am, acc1);
                    acc3 += e2;
                    if (Tv > 0.f) acc2 += e2;
                }
            });
            if constexpr (H) {
                // the intensity of mirror pixel (ny - y, nx - x) equals that of (y, x)
                const int ym = (ny - yc) % ny, iym = (ym + ny / 2) % ny;
                if (act && ym != yc) {
                    const float *Tm = a.T ? a.T + ((size_t)item * ny + ym) * NX : nullptr;
                    float *Im = a.I_out ? a.I_out + ((size_t)item * ny + iym) * NX : nullptr;
                    static_for<0, E>([&](auto ec) {
                        constexpr int e = decltype(ec)::value;
                        const int xm = (NX - (t + TL * e)) % NX;
                        const float I = acc[e] * inv_sub * a.invN2;
                        if (Im) Im[(xm + NX / 2) % NX] = I;
                        if (Tm) {
                            const float Tv = Tm[xm];
                            const float d = I - Tv * Tv;
                            const float am = sqrtf(I) - Tv;
                            const float e2 = acc[e] * inv_sub * a.invN;
                            acc0 = fmaf(d, d, acc0);
                            acc1 = fmaf(am, am, acc1);
                            acc3 += e2;
                            if (Tv > 0.f) acc2 += e2;
                        }
                    });
                }
            }
            if (a.part)
                block_sum4(acc0, acc1, acc2, acc3, red,
                           a.part + ((size_t)item * ppt + pan) * NMET, Cfg::THREADS);
        }
    }
}

template <class P, int ROLE, int LINES>
__global__ void __launch_bounds__(P::TL *LINES) k_row(const RowArgs a) {
    row_body<P, ROLE, LINES, false>(a);
}
template <class P, int ROLE, int LINES>
__global__ void __launch_bounds__(P::TL *LINES, ROLE == ROW_HEAD ? 2 : 1) k_row_h(const RowArgs a) {
    row_body<P, ROLE, LINES, true>(a);
}

// ------------------------------------------------------------ column pass
template <class P, int ROLE, int C>
__global__ void __launch_bounds__(P::TL *C) k_col(const ColArgs a) {
    constexpr int TL = P::TL, E = P::E, NY = P::N;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int tid = threadIdx.x, c = tid % C, t = tid / C;
    float2 *smb = sm + c;
    auto sync = []() { __syncthreads(); };
    const int nx = a.nx;
    const int ppt = (nx + C - 1) / C;
    const int total = a.items * ppt;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int item = p / ppt, pan = p - item * ppt;
        const int x = pan * C + c;
        const bool act = x < nx;
        const int xc = act ? x : nx - 1;
        const size_t base = (size_t)item * NY * nx;
        float2 v[E];
        if constexpr (ROLE == COL_GS_BIN || ROLE == COL_GS_LVL || ROLE == COL_GS_MOD) {
            const float2 *fc = a.field + base + xc;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                v[e] = fc[(t + TL * e) * nx];
            });
            line_fft<P, +1, C>(v, smb, a.tw, t, sync);
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int o = (t + TL * e) * nx + x;
                const float2 h = v[e];
                int q;
                float2 ph;
                if constexpr (ROLE == COL_GS_MOD) {
                    // the level nearest h / E: phase SLMs decide on h conj(E), the
                    // amplitude SLM on the least-squares transmittance
                    // Re(h conj E) / |E|^2 mapped to [0, L - 1]; the light leaving
                    // the SLM is E times the level
                    const float2 E = __ldg(a.illum + (size_t)(t + TL * e) * nx + xc);
                    const float hr = fmaf(h.x, E.x, h.y * E.y), hi = fmaf(h.y, E.x, -h.x * E.y);
                    if (a.kind == 2) {
                        const float e2 = fmaf(E.x, E.x, E.y * E.y);
                        const float m = e2 > 0.f ? hr / e2 : 0.f;
                        const float lv = (float)(a.levels - 1) * fmaf(m, a.amp_gain, 0.5f);
                        q = (int)roundf(fminf(fmaxf(lv, 0.f), (float)(a.levels - 1)));
                        const float tr = __ldg(a.lvl + q).x;
                        ph = make_float2(E.x * tr, E.y * tr);
                    } else {
                        float2 l;
                        if (a.kind == 0) {
                            q = hr >= 0.f ? 0 : 1;
                            l = make_float2(q ? -1.f : 1.f, 0.f);
                        } else {
                            q = (int)roundf(atan2f(hi, hr) * a.qscale) % a.levels;
                            if (q < 0) q += a.levels;
                            l = __ldg(a.lvl + q);
                        }
                        ph = make_float2(E.x * l.x - E.y * l.y, fmaf(E.x, l.y, E.y * l.x));
                    }
                } else if constexpr (ROLE == COL_GS_BIN) {
                    q = h.x >= 0.f ? 0 : 1;
                    ph = make_float2(q ? -1.f : 1.f, 0.f);
                } else {
                    q = (int)roundf(atan2f(h.y, h.x) * a.qscale) % a.levels;
                    if (q < 0) q += a.levels;
                    ph = __ldg(a.lvl + q);
                }
                if (act) {
                    if (a.h_out) a.h_out[base + o] = make_float2(h.x * a.invSqrtN, h.y * a.invSqrtN);
                    if (a.holo) a.holo[base + o] = (uint8_t)q;
                }
                v[e] = ph;
            });
        } else {
            const uint8_t *hc = a.holo + base + xc;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int q = hc[(t + TL * e) * nx];
                if constexpr (ROLE == COL_HOLO_BIN) {
                    v[e] = make_float2(q ? -1.f : 1.f, 0.f);
                } else if constexpr (ROLE == COL_HOLO_MOD) {
                    const float2 E = __ldg(a.illum + (size_t)(t + TL * e) * nx + xc);
                    const float2 l = a.kind == 0 ? make_float2(q ? -1.f : 1.f, 0.f)
                                                 : __ldg(a.lvl + (q < a.levels ? q : 0));
                    v[e] = make_float2(E.x * l.x - E.y * l.y, fmaf(E.x, l.y, E.y * l.x));
                } else {
                    v[e] = __ldg(a.lvl + (q < a.levels ? q : 0));
                }
            });
        }
        line_fft<P, -1, C>(v, smb, a.tw, t, sync);
        if (act) {
            float2 *fw = a.field + base + x;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                fw[(t + TL * e) * nx] = v[e];
            });
        }
    }
}

// ----------------------------------------------------- per-length dispatch

struct LineOps {
    int N;
    int row_threads, row_lines, col_threads, col_c;
    size_t row_smem, col_smem;
    int row_blocks_per_sm, col_blocks_per_sm;  // filled by init
    cudaError_t (*init)(LineOps *self);        // per device: smem attributes, occupancy
    void (*row)(int role, const RowArgs &a, int grid, cudaStream_t s);
    void (*col)(int role, const ColArgs &a, int grid, cudaStream_t s);
};

// HERM: also instantiate the Hermitian HEAD / AVG rows (power-of-two lengths
// that have a column-pair pass).
template <class P, int LINES, int C, bool HERM = false>
struct OpsImpl {
    using RC = RowCfg<P, LINES>;
    using CC = ColCfg<P, C>;
    static cudaError_t init(LineOps *self) {
        cudaError_t e = cudaSuccess;
        auto set = [&](const void *f, size_t smem) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        };
        set((const void *)k_row<P, ROW_HEAD, LINES>, RC::SMEM);
        set((const void *)k_row<P, ROW_ITER, LINES>, RC::SMEM);
        set((const void *)k_row<P, ROW_TAIL, LINES>, RC::SMEM);
        set((const void *)k_row<P, ROW_AVG, LINES>, RC::SMEM);
        set((const void *)k_row<P, ROW_ADAPT, LINES>, RC::SMEM);
        set((const void *)k_row<P, ROW_ADFIN, LINES>, RC::SMEM);
        if constexpr (HERM) {
            set((const void *)k_row_h<P, ROW_HEAD, LINES>, RC::SMEM);
            set((const void *)k_row_h<P, ROW_AVG, LINES>, RC::SMEM);
        }
        set((const void *)k_col<P, COL_GS_BIN, C>, CC::SMEM);
        set((const void *)k_col<P, COL_GS_LVL, C>, CC::SMEM);
        set((const void *)k_col<P, COL_HOLO_BIN, C>, CC::SMEM);
        set((const void *)k_col<P, COL_HOLO_LVL, C>, CC::SMEM);
        set((const void *)k_col<P, COL_GS_MOD, C>, CC::SMEM);
        set((const void *)k_col<P, COL_HOLO_MOD, C>, CC::SMEM);
        if (e != cudaSuccess) return e;
        int rb = 0, cb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rb, k_row<P, ROW_ITER, LINES>,
                                                          RC::THREADS, RC::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cb, k_col<P, COL_GS_BIN, C>, CC::THREADS,
                                                          CC::SMEM);
        if (e != cudaSuccess) return e;
        self->row_blocks_per_sm = rb > 0 ? rb : 1;
        self->col_blocks_per_sm = cb > 0 ? cb : 1;
        return cudaSuccess;
    }
    static void row(int role, const RowArgs &a, int grid, cudaStream_t s) {
        if constexpr (HERM) {
            if (a.herm && role == ROW_HEAD) {
                k_row_h<P, ROW_HEAD, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a);
                return;
            }
            if (a.herm && role == ROW_AVG) {
                k_row_h<P, ROW_AVG, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a);
                return;
            }
        }
        switch (role) {
            case ROW_HEAD: k_row<P, ROW_HEAD, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a); break;
            case ROW_ITER: k_row<P, ROW_ITER, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a); break;
            case ROW_TAIL: k_row<P, ROW_TAIL, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a); break;
            case ROW_ADAPT: k_row<P, ROW_ADAPT, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a); break;
            case ROW_ADFIN: k_row<P, ROW_ADFIN, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a); break;
            default: k_row<P, ROW_AVG, LINES><<<grid, RC::THREADS, RC::SMEM, s>>>(a); break;
        }
    }
    static void col(int role, const ColArgs &a, int grid, cudaStream_t s) {
        switch (role) {
            case COL_GS_BIN: k_col<P, COL_GS_BIN, C><<<grid, CC::THREADS, CC::SMEM, s>>>(a); break;
            case COL_GS_LVL: k_col<P, COL_GS_LVL, C><<<grid, CC::THREADS, CC::SMEM, s>>>(a); break;
            case COL_HOLO_BIN: k_col<P, COL_HOLO_BIN, C><<<grid, CC::THREADS, CC::SMEM, s>>>(a); break;
            case COL_GS_MOD: k_col<P, COL_GS_MOD, C><<<grid, CC::THREADS, CC::SMEM, s>>>(a); break;
            case COL_HOLO_MOD: k_col<P, COL_HOLO_MOD, C><<<grid, CC::THREADS, CC::SMEM, s>>>(a); break;
            default: k_col<P, COL_HOLO_LVL, C><<<grid, CC::THREADS, CC::SMEM, s>>>(a); break;
        }
    }
    static LineOps make() {
        LineOps o{};
        o.N = P::N;
        o.row_threads = RC::THREADS;
        o.row_lines = LINES;
        o.col_threads = CC::THREADS;
        o.col_c = C;
        o.row_smem = RC::SMEM;
        o.col_smem = CC::SMEM;
        o.init = &init;
        o.row = &row;
        o.col = &col;
        return o;
    }
};

// Registry (one translation unit per group of lengths).
const LineOps *ops_small(int n);
const LineOps *ops_mid(int n);
const LineOps *ops_1024(int n);
const LineOps *ops_2048(int n);
const LineOps *ops_hd(int n);

}  // namespace hg
