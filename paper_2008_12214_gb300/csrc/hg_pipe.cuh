// hg_pipe.cuh -- TMA-fed, warp-specialised versions of the two passes of a
// GS / WGS iteration (same arithmetic as k_row ROW_ITER and k_col COL_GS_*).
//
// A CTA has NG independent groups of threads; each group owns a ring of D
// shared-memory slots.  The group's leader thread streams the group's panels
// into its ring with the bulk-copy engine (row panels are contiguous and go
// through cp.async.bulk; column panels are 2D tiles of the [rows][2 nx floats]
// field and go through cp.async.bulk.tensor.2d with a tensor map), each slot
// completing an mbarrier with the copy's transaction count.  A group uses
// slot k % D for its k-th panel and refills it with panel k + D as soon as
// the panel's transforms are done, so D - 1 copies are always in flight
// while the group computes.  The transforms exchange data in place inside the
// slot with a swizzled layout; results are written back with ordinary
// coalesced stores.
//
// Every wait is bounded by %globaltimer: a wait that runs past the limit
// sets the error flag and makes the CTA abort; before leaving, each group's
// leader waits (bounded) for the copies it still has in flight.
#pragma once
#include <cuda.h>

#include "hg_kernels.cuh"

namespace hg {

constexpr unsigned ERR_TIMEOUT_BIT = 4u;

struct PipeArgs {
    unsigned *err;                 // device error word (bit ERR_TIMEOUT_BIT)
    unsigned long long wait_ns;    // bound on any single wait
    int drop_job;                  // fault-injection hook: this job is never issued (-1: none)
};

// Index of the mirror sample (N - x) mod N, for any line length N.
template <int N>
__device__ __forceinline__ int mirror_idx(int x) {
    if constexpr ((N & (N - 1)) == 0) return (N - x) & (N - 1);
    else return x ? N - x : 0;
}

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of `bar` with the given parity to complete; false when
// `limit_ns` passes first or another thread of the CTA raised `abort`.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                          volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if ((abort && *abort) || global_ns() - t0 > limit_ns) return false;
    }
}
// 1D bulk copy global -> shared, completing `bytes` on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// 2D tensor tile global -> shared at coordinates (x, y) of the tensor map.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Sum four per-thread float partials over a consumer group of GT threads in a
// fixed order: lanes and warps combine in float (at most GT partial sums of
// E terms each), the group total is stored as double by thread 0 and every
// reduction across panels is done in double.  (Double shuffles or additions
// here would occupy the FP64 pipe, which is narrow on this GPU.)
// float -> double on the integer pipes (IEEE 754 binary32 -> binary64, exact):
// a normal float's biased exponent is raised by 1023 - 127 = 896 and its 23
// fraction bits become the top of the 52-bit fraction; a subnormal m 2^-149
// is renormalised at its leading bit p (exponent p - 149); zeros keep their
// sign and infinities / NaNs keep exponent all-ones and the payload.  The
// group totals would otherwise hold their group's barrier on the narrow FP64
// pipe (a select between two paths still executes the conversion).
__device__ __forceinline__ double f2d_exact(float x) {
    const uint32_t u = __float_as_uint(x), m = u & 0x7fffffffu;
    const unsigned long long sgn = ((unsigned long long)(u & 0x80000000u)) << 32;
    unsigned long long d;
    if (m >= 0x00800000u && m < 0x7f800000u) {
        d = (((unsigned long long)m) << 29) + (896ull << 52);
    } else if (m >= 0x7f800000u) {
        d = (0x7ffull << 52) | (((unsigned long long)(m & 0x007fffffu)) << 29);
    } else if (m == 0u) {
        d = 0ull;
    } else {
        const int pb = 31 - __clz((int)m);  // leading bit, 0 .. 22
        d = ((unsigned long long)(pb + 874) << 52) |
            ((((unsigned long long)m) << (52 - pb)) & ((1ull << 52) - 1));
    }
    return __longlong_as_double((long long)(sgn | d));
}

template <int GT, class SYNC>
__device__ __forceinline__ void group_sum4(float a0, float a1, float a2, float a3, double *red,
                                           double *dst, int gt, SYNC gsync) {
    float d[NMET] = {a0, a1, a2, a3};
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
        for (int m = 0; m < NMET; ++m) d[m] += __shfl_down_sync(0xffffffffu, d[m], off);
    if constexpr (GT == 32) {
        if (gt == 0)
#pragma unroll
            for (int m = 0; m < NMET; ++m) dst[m] = f2d_exact(d[m]);
    } else {
        float *redf = reinterpret_cast<float *>(red);
        const int lane = gt & 31, w = gt >> 5;
        if (lane == 0)
#pragma unroll
            for (int m = 0; m < NMET; ++m) redf[w * NMET + m] = d[m];
        gsync();
        if (gt == 0) {
            // the group's few warp sums in float (one rounding each), then one
            // exact conversion on the integer pipes: FP64 work here would hold
            // the group's barrier on the narrow FP64 pipe
            float s[NMET] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < GT / 32; ++q)
#pragma unroll
                for (int m = 0; m < NMET; ++m) s[m] += redf[q * NMET + m];
#pragma unroll
            for (int m = 0; m < NMET; ++m) dst[m] = f2d_exact(s[m]);
        }
        gsync();
    }
}

// -------------------------------------------------------------- row pass
template <class P, int LINES, int NG, int D, int SWZ>
struct RowPipeCfg {
    static constexpr int GT = P::TL * LINES;
    static_assert(GT % 32 == 0, "row group must be whole warps");
    static constexpr int GW = GT / 32;
    static constexpr int THREADS = NG * GT;
    static constexpr int SLOT_F = LINES * P::N * 8;
    static constexpr int SLOT_T = LINES * P::N * 4;
    static constexpr int RED = NG * GW * NMET * 8;
    static constexpr size_t smem_for(int slot) {
        return 1024 + (size_t)NG * D * slot + RED + NG * D * 8 + 4 * (NG + 1) + 256;
    }
    // region-of-interest rows (1 B/px) come in with the panel when a row is a
    // whole number of 16-byte units and the larger ring still fits in 227 KB;
    // otherwise they are read from global memory
    static constexpr int SLOT_FT = (SLOT_F + SLOT_T + 127) / 128 * 128;
    static constexpr int SLOT_FTR = (SLOT_F + SLOT_T + LINES * P::N + 127) / 128 * 128;
    static constexpr bool ROI_SM = P::N % 16 == 0 && smem_for(SLOT_FTR) <= 227 * 1024;
    static constexpr int SLOT = ROI_SM ? SLOT_FTR : SLOT_FT;
    static constexpr size_t SMEM = smem_for(SLOT);
};

// GEN: the modulated plans' row pass (a.gen: eight metric sums, region of
// interest, no weights, a window that covers the field); otherwise the plain
// GS / WGS / LT pass (four sums, no region of interest).
template <class P, int LINES, int NG, int D, int SWZ, bool GEN>
__global__ void __launch_bounds__(RowPipeCfg<P, LINES, NG, D, SWZ>::THREADS, 1)
    k_row_pipe(const RowArgs a, const PipeArgs pa) {
    using Cfg = RowPipeCfg<P, LINES, NG, D, SWZ>;
    using LAY = Swz<SWZ>;
    constexpr int TL = P::TL, E = P::E, NX = P::N, GT = Cfg::GT;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    double *red = reinterpret_cast<double *>(base + (size_t)NG * D * Cfg::SLOT);
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(red) + Cfg::RED);
    volatile int *flags = reinterpret_cast<volatile int *>(full + NG * D);
    volatile int *abort = flags + NG;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NG * D; ++i) mbar_init(full + i, 1);
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int ny = a.ny;
    const int ppt = (ny + LINES - 1) / LINES;
    const int J = a.items * ppt;
    const int g = tid / GT, gt = tid - g * GT;
    const int line = gt / TL, t = gt - line * TL;
    unsigned char *ring = base + (size_t)g * D * Cfg::SLOT;
    uint64_t *gfull = full + g * D;
    auto gsync = [g]() {
        if constexpr (Cfg::GW == 1) __syncwarp();
        else named_sync(1 + g, GT);
    };
    auto job = [&](int k) { return (int)blockIdx.x + (g + NG * k) * (int)gridDim.x; };
    auto issue = [&](int k) {  // copy the group's k-th panel (field, target and ROI rows)
        const int j = job(k);
        if (j >= J || j == pa.drop_job) return;
        const int item = j / ppt, pan = j - item * ppt, y0 = pan * LINES;
        const int nl = min(LINES, ny - y0);
        const uint32_t bf = (uint32_t)(nl * NX * 8), bt = (uint32_t)(nl * NX * 4);
        const uint32_t br = GEN && Cfg::ROI_SM && a.roi ? (uint32_t)(nl * NX) : 0u;
        unsigned char *sl = ring + (size_t)(k % D) * Cfg::SLOT;
        mbar_expect_tx(gfull + k % D, bf + bt + br);
        bulk_g2s(sl, a.field + ((size_t)item * ny + y0) * NX, bf, gfull + k % D);
        bulk_g2s(sl + Cfg::SLOT_F, a.T + ((size_t)item * ny + y0) * NX, bt, gfull + k % D);
        if (br) bulk_g2s(sl + Cfg::SLOT_F + Cfg::SLOT_T, a.roi + (size_t)y0 * NX, br, gfull + k % D);
    };
    auto drain = [&](int k0, int k1) {
        for (int q = k0; q < k1; ++q) {
            const int j = job(q);
            if (j < J && j != pa.drop_job) mbar_wait(gfull + q % D, (q / D) & 1, pa.wait_ns, nullptr);
        }
    };
    if (gt == 0)
        for (int k = 0; k < D; ++k) issue(k);

    for (int k = 0;; ++k) {
        const int j = job(k);
        if (j >= J) break;
        if (gt == 0) {
            bool ok = !*abort && mbar_wait(gfull + k % D, (k / D) & 1, pa.wait_ns, abort);
            if (!ok) {
                atomicOr(pa.err, ERR_TIMEOUT_BIT);
                *abort = 1;
            }
            flags[g] = ok;
        }
        gsync();
        if (!flags[g]) {
            if (gt == 0) drain(k, k + D);
            break;
        }
        const int item = j / ppt, pan = j - item * ppt;
        const int y = pan * LINES + line;
        const bool act = y < ny;
        unsigned char *sl = ring + (size_t)(k % D) * Cfg::SLOT;
        float2 *sf = reinterpret_cast<float2 *>(sl) + line * NX;  // also the exchange buffer
        const float *sT = reinterpret_cast<const float *>(sl + Cfg::SLOT_F) + line * NX;
        float2 v[E];
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            v[e] = sf[t + TL * e];
        });
        line_fft<P, -1, 1, LAY>(v, sf, a.tw, t, gsync);
        float *wr = !GEN && a.w ? a.w + ((size_t)item * ny + (act ? y : ny - 1)) * NX : nullptr;
        // region-of-interest flags of this thread's E samples, one bit each
        static_assert(E <= 32, "one flag bit per sample");
        uint32_t inm = 0xffffffffu;
        if (GEN && a.roi) {
            const uint8_t *roir = Cfg::ROI_SM ? sl + Cfg::SLOT_F + Cfg::SLOT_T + line * NX
                                              : a.roi + (size_t)(act ? y : ny - 1) * NX;
            inm = 0u;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                inm |= (roir[t + TL * e] != 0 ? 1u : 0u) << e;
            });
        }
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
        float acc4 = 0.f, acc5 = 0.f, acc6 = 0.f, acc7 = 0.f;
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const int x = t + TL * e;
            const float Tv = act ? sT[x] : 0.f;
            const float2 r = v[e];
            const float m2 = fmaf(r.x, r.x, r.y * r.y);
            const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
            const float e2 = m2 * a.invN;
            const bool in = (inm >> e) & 1u;
            if constexpr (GEN) {  // modulated plan: the eight sums of the generic row pass
                if (act) {
                    acc5 += e2;
                    if (in) {
                        const float t2 = Tv * Tv;
                        acc0 += e2;
                        acc1 = fmaf(e2, e2, acc1);
                        acc2 = fmaf(e2, t2, acc2);
                        acc3 = fmaf(m2 * rs, Tv * a.invSqrtN, acc3);  // sqrt(e2) T
                        if (Tv > 0.f) acc4 += e2;
                        acc6 = fmaf(t2, t2, acc6);
                        acc7 += t2;
                    }
                }
            } else {
                const float I = m2 * a.invN2;
                const float d = I - Tv * Tv;
                const float am = fmaf(m2 * rs, a.invSqrtN * a.invSqrtN, -Tv);  // sqrt(I) - T
                if (act) {
                    acc0 = fmaf(d, d, acc0);
                    acc1 = fmaf(am, am, acc1);
                    acc3 += e2;
                    if (Tv > 0.f) acc2 += e2;
                }
            }
            float wv = 1.f;
            if (wr) {
                wv = act ? wr[x] : 1.f;
                if (Tv > 0.f && m2 > 0.f) wv = wv * Tv * (a.NN * rs);
                if (act) wr[x] = wv;
            }
            // a modulated plan scales T by its lt_amp (the replay energy of a
            // unit-modulus hologram) with a window that covers the field, and
            // leaves pixels outside the region of interest free; LT scales T
            // the same way and leaves pixels outside its window free
            const bool lt = GEN || a.lt_amp > 0.f;
            const float gm = (lt ? a.lt_amp : 1.f) * Tv * wv;
            if (lt && (!in || (!GEN && !lt_in(a, y, x)))) v[e] = r;
            else v[e] = m2 > 0.f ? make_float2(gm * r.x * rs, gm * r.y * rs) : make_float2(gm, 0.f);
        });
        line_fft<P, +1, 1, LAY>(v, sf, a.tw, t, gsync);
        gsync();
        if (gt == 0) issue(k + D);  // slot fully consumed: refill it
        if (act) {
            float2 *fw = a.field + ((size_t)item * ny + y) * NX;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                fw[t + TL * e] = v[e];
            });
        }
        if (a.part) {
            if constexpr (GEN) {
                double *dst = a.part + ((size_t)item * ppt + pan) * NMET_GEN;
                group_sum4<GT>(acc0, acc1, acc2, acc3, red + (size_t)g * Cfg::GW * NMET, dst, gt, gsync);
                group_sum4<GT>(acc4, acc5, acc6, acc7, red + (size_t)g * Cfg::GW * NMET, dst + NMET, gt, gsync);
            } else {
                group_sum4<GT>(acc0, acc1, acc2, acc3, red + (size_t)g * Cfg::GW * NMET,
                               a.part + ((size_t)item * ppt + pan) * NMET, gt, gsync);
            }
        }
    }
}

// --------------------------------------------------- paired row pass (binary)
// For a binary SLM e^{iH} is real, so after the column FFTs every column is
// Hermitian in ky: C[ny - ky][x] = conj(C[ky][x]), hence for the full 2D
// transform R[ny - ky][kx] = conj(R[ky][(nx - kx) % nx]).  The column pass then
// stores rows ky <= ny/2 only, and this pass handles the rows (ky, ny - ky) of
// one panel with a single forward row FFT: row ny - ky's spectrum is the
// conjugated reversal of row ky's, fetched through shared memory.  The
// self-conjugate rows 0 and ny/2 are panels of their own.  Each panel then
// applies the constraint to its rows and runs their inverse FFTs, as the
// plain row pass does.
// Constraint of one replay row held as E samples per thread (binary pairs):
// metric partials, optional weight update, F = w T R / |R| in place.
template <class P>
__device__ __forceinline__ void pair_constrain(float2 (&w)[P::E], const float *sT, float *wr,
                                               const RowArgs &a, int t, int yrow, float &acc0, float &acc1,
                                               float &acc2, float &acc3) {
    static_for<0, P::E>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const int x = t + P::TL * e;
        const float Tv = sT[x];
        const float2 r = w[e];
        const float m2 = fmaf(r.x, r.x, r.y * r.y);
        const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
        const float I = m2 * a.invN2;
        const float d = I - Tv * Tv;
        const float am = fmaf(m2 * rs, a.invSqrtN * a.invSqrtN, -Tv);
        const float e2 = m2 * a.invN;
        acc0 = fmaf(d, d, acc0);
        acc1 = fmaf(am, am, acc1);
        acc3 += e2;
        if (Tv > 0.f) acc2 += e2;
        float wv = 1.f;
        if (wr) {
            wv = wr[x];
            if (Tv > 0.f && m2 > 0.f) wv = wv * Tv * (a.NN * rs);
            wr[x] = wv;
        }
        const float gm = (a.lt_amp > 0.f ? a.lt_amp : 1.f) * Tv * wv;
        if (a.lt_amp > 0.f && !lt_in(a, yrow, x)) w[e] = r;  // outside the window: left free
        else w[e] = m2 > 0.f ? make_float2(gm * r.x * rs, gm * r.y * rs) : make_float2(gm, 0.f);
    });
}

// Inverse row FFT of one row (exchange in `xbuf`) and its store.
template <class P, class LAY, class SYNC>
__device__ __forceinline__ void pair_finish(float2 (&w)[P::E], float2 *xbuf, const float2 *tw, int t,
                                            SYNC gsync, float2 *fw) {
    line_fft<P, +1, 1, LAY>(w, xbuf, tw, t, gsync);
    static_for<0, P::E>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        fw[t + P::TL * e] = w[e];
    });
}

// Hermitian form of the binary constraint.  The binary quantiser reads only
// Re h, and Re IFFT2(F) = IFFT2(F_H) with F_H(u) = (F(u) + conj F(-u)) / 2.
// For a binary SLM the replay is Hermitian, R(-u) = conj R(u), so
// F_H(u) = (wT(u) + wT(-u)) / 2 * R(u) / |R(u)|: the same constraint with a
// symmetrised target, and F_H is Hermitian, so after the inverse row FFTs
// row ny - y of the field is conj(row y).  Each thread takes its pixel u of
// row p together with the mirror u' = (ny - p, nx - x): |R(u')| = |R(u)|, so
// both pixels' metrics and weight updates come from the one spectrum, and
// only row p of F_H is transformed and stored.  sTm: targets of row ny - p
// (row p itself for the self-mirrored rows 0 and ny/2); wold_m: the mirror
// row's weights before this pass (for self-mirrored rows a shared-memory
// copy, since other threads update the row in place); store_m: write the
// mirror's updated weight (partner rows only).
template <class P, bool GEN>
__device__ __forceinline__ void herm_constrain(float2 (&w)[P::E], const float *sT, const float *sTm, float *wr,
                                               const float *wold_m, float *wrm, bool partner,
                                               const RowArgs &a, int t, int yrow, float &acc0, float &acc1,
                                               float &acc2, float &acc3) {
    static_for<0, P::E>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const int x = t + P::TL * e;
        const int xm = mirror_idx<P::N>(x);
        const float Tv = sT[x], Tm = sTm[xm];
        const float2 r = w[e];
        const float m2 = fmaf(r.x, r.x, r.y * r.y);
        const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
        const float I = m2 * a.invN2;
        const float amp = m2 * rs * (a.invSqrtN * a.invSqrtN);
        const float e2 = m2 * a.invN;
        const float d = I - Tv * Tv, am = amp - Tv;
        acc0 = fmaf(d, d, acc0);
        acc1 = fmaf(am, am, acc1);
        acc3 += e2;
        if (Tv > 0.f) acc2 += e2;
        if (partner) {
            const float dm = I - Tm * Tm, amm = amp - Tm;
            acc0 = fmaf(dm, dm, acc0);
            acc1 = fmaf(amm, amm, acc1);
            acc3 += e2;
            if (Tm > 0.f) acc2 += e2;
        }
        if constexpr (GEN) {
            float wv = 1.f, wm = 1.f;
            if (wr) {
                wv = wr[x];
                if (Tv > 0.f && m2 > 0.f) wv = wv * Tv * (a.NN * rs);
                wr[x] = wv;
                wm = wold_m[xm];
                if (Tm > 0.f && m2 > 0.f) wm = wm * Tm * (a.NN * rs);
                if (partner) wrm[xm] = wm;
            }
            const float gm = (a.lt_amp > 0.f ? a.lt_amp : 1.f) * 0.5f * fmaf(Tv, wv, Tm * wm);
            // the window is symmetric under u -> -u: outside it F_H = R
            if (a.lt_amp > 0.f && !lt_in(a, yrow, x)) w[e] = r;
            else w[e] = m2 > 0.f ? make_float2(gm * r.x * rs, gm * r.y * rs) : make_float2(gm, 0.f);
        } else {  // plain GS: no weights, no window
            const float gm = 0.5f * (Tv + Tm);
            w[e] = m2 > 0.f ? make_float2(gm * r.x * rs, gm * r.y * rs) : make_float2(gm, 0.f);
        }
    });
}

template <class P, int NG, int D, int SWZ>
struct PairPipeCfg {
    static constexpr int GT = P::TL;
    static_assert(GT % 32 == 0, "paired row group must be whole warps");
    static constexpr int GW = GT / 32;
    static constexpr int THREADS = NG * GT;
    static constexpr int SLOT_F = P::N * 8;
    static constexpr int SLOT = SLOT_F + 2 * P::N * 4;  // field row ky, targets of both rows
    static constexpr int RED = NG * GW * NMET * 8;
    static constexpr size_t SMEM = 1024 + (size_t)NG * D * SLOT + RED + NG * D * 8 + 4 * (NG + 1) + 256;
};

// MODE 0: paired rows (full F); 1: Hermitian form, any plan (weights, window);
// 2: Hermitian form of plain GS (no weights, no window), compiled without
// those paths; 3: Hermitian HEAD, the first field F_H of a run from the
// target and the initial replay phase (or Philox phases), rows ky <= ny/2,
// inverse row FFT; 4: Hermitian TAIL, the forward row FFT of a binary
// column-transformed field (rows ky <= ny/2), metrics and weights of both
// pixels u and -u, and optionally arg R and R at both (no inverse FFT, no
// store); 5: Hermitian time average (binary OSPR, Section 3.4): a job is one
// row ky <= ny/2 of one target, whose nsub subframe rows the group streams in
// order, summing |R|^2 in registers; after the last one it writes the
// normalised intensity of u and -u and the metrics; 6 and 7: adaptive OSPR in
// Hermitian form, 6 the replay of the subframe just quantised added to the
// running intensity sum, then the next subframe's deficit target with its
// Philox phases and the inverse row FFT, 7 the last subframe's replay and the
// metrics of the time average.
template <class P, int NG, int D, int SWZ, int MODE, int MINB = 1>
__global__ void __launch_bounds__(PairPipeCfg<P, NG, D, SWZ>::THREADS, MINB)
    k_row_pipe_pair(const RowArgs a, const PipeArgs pa) {
    constexpr bool HERM = MODE != 0;
    using Cfg = PairPipeCfg<P, NG, D, SWZ>;
    using LAY = Swz<SWZ>;
    constexpr int TL = P::TL, E = P::E, NX = P::N, GT = Cfg::GT;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    double *red = reinterpret_cast<double *>(base + (size_t)NG * D * Cfg::SLOT);
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(red) + Cfg::RED);
    volatile int *flags = reinterpret_cast<volatile int *>(full + NG * D);
    volatile int *abort = flags + NG;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NG * D; ++i) mbar_init(full + i, 1);
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // panels per item: p = 0 (row 0 alone), 1 .. ny/2 - 1 (rows p and ny - p),
    // ny/2 (row ny/2 alone)
    const int ny = a.ny, hy = ny / 2;
    const int ppt = hy + 1;
    const int J = a.items * ppt;
    const int g = tid / GT, t = tid - g * GT;
    unsigned char *ring = base + (size_t)g * D * Cfg::SLOT;
    uint64_t *gfull = full + g * D;
    auto gsync = [g]() {
        if constexpr (Cfg::GW == 1) __syncwarp();
        else named_sync(1 + g, GT);
    };
    auto job = [&](int k) { return (int)blockIdx.x + (g + NG * k) * (int)gridDim.x; };
    // the group's k-th panel belongs to job jstep(k); MODE 5 takes nsub panels
    // (the job's subframes, in order) per job
    const int per = MODE == 5 ? a.nsub : 1;
    auto jstep = [&](int k) { return job(k / per); };
    auto issue = [&](int k) {
        const int j = jstep(k);
        if (j >= J || j == pa.drop_job) return;
        const int item = j / ppt, pan = j - item * ppt;
        const bool partner = pan != 0 && pan != hy;
        unsigned char *sl = ring + (size_t)(k % D) * Cfg::SLOT;
        if constexpr (MODE == 5) {
            // subframe n's row, and with the last subframe the target rows
            const int n = k % per;
            const bool last = n == per - 1;
            mbar_expect_tx(gfull + k % D, (uint32_t)(NX * 8 + (last ? NX * 4 * (partner ? 2 : 1) : 0)));
            bulk_g2s(sl, a.field + ((size_t)(item * per + n) * ny + pan) * NX, NX * 8, gfull + k % D);
            if (last) {
                bulk_g2s(sl + Cfg::SLOT_F, a.T + ((size_t)item * ny + pan) * NX, NX * 4, gfull + k % D);
                if (partner)
                    bulk_g2s(sl + Cfg::SLOT_F + NX * 4, a.T + ((size_t)item * ny + ny - pan) * NX, NX * 4,
                             gfull + k % D);
            }
            return;
        }
        if constexpr (MODE == 3) {
            // replay rows of DFT rows pan and ny - pan: phases, then the targets
            const int b = item / a.nsub, ym = (ny - pan) % ny;
            const int iy = (pan + hy) % ny, iym = (ym + hy) % ny;
            const uint32_t rows = partner ? 2u : 1u;
            mbar_expect_tx(gfull + k % D, (uint32_t)(NX * 4) * rows * (a.phase ? 2u : 1u));
            if (a.phase) {
                bulk_g2s(sl, a.phase + ((size_t)b * ny + iy) * NX, NX * 4, gfull + k % D);
                if (partner) bulk_g2s(sl + NX * 4, a.phase + ((size_t)b * ny + iym) * NX, NX * 4, gfull + k % D);
            }
            bulk_g2s(sl + Cfg::SLOT_F, a.T + ((size_t)b * ny + pan) * NX, NX * 4, gfull + k % D);
            if (partner)
                bulk_g2s(sl + Cfg::SLOT_F + NX * 4, a.T + ((size_t)b * ny + ym) * NX, NX * 4, gfull + k % D);
            return;
        }
        mbar_expect_tx(gfull + k % D, (uint32_t)(NX * (partner ? 16 : 12)));
        bulk_g2s(sl, a.field + ((size_t)item * ny + pan) * NX, NX * 8, gfull + k % D);
        bulk_g2s(sl + Cfg::SLOT_F, a.T + ((size_t)item * ny + pan) * NX, NX * 4, gfull + k % D);
        if (partner)
            bulk_g2s(sl + Cfg::SLOT_F + NX * 4, a.T + ((size_t)item * ny + ny - pan) * NX, NX * 4,
                     gfull + k % D);
    };
    auto drain = [&](int k0, int k1) {
        for (int q = k0; q < k1; ++q) {
            const int j = jstep(q);
            if (j < J && j != pa.drop_job) mbar_wait(gfull + q % D, (q / D) & 1, pa.wait_ns, nullptr);
        }
    };
    if (t == 0)
        for (int k = 0; k < D; ++k) issue(k);

    float accI[E];  // MODE 5: sum over the subframes of |R|^2
    for (int k = 0;; ++k) {
        const int j = jstep(k);
        if (j >= J) break;
        if (t == 0) {
            bool ok = !*abort && mbar_wait(gfull + k % D, (k / D) & 1, pa.wait_ns, abort);
            if (!ok) {
                atomicOr(pa.err, ERR_TIMEOUT_BIT);
                *abort = 1;
            }
            flags[g] = ok;
        }
        gsync();
        if (!flags[g]) {
            if (t == 0) drain(k, k + D);
            break;
        }
        const int item = j / ppt, pan = j - item * ppt;
        const bool partner = pan != 0 && pan != hy;
        unsigned char *sl = ring + (size_t)(k % D) * Cfg::SLOT;
        float2 *sf = reinterpret_cast<float2 *>(sl);  // field row, then exchange buffer
        const float *sTa = reinterpret_cast<const float *>(sl + Cfg::SLOT_F);
        float2 *park = reinterpret_cast<float2 *>(sl + Cfg::SLOT_F);  // row ny - p after use of T
        float2 v[E];
        if constexpr (MODE == 3) {
            // F_H(u) = (F(u) + conj F(-u)) / 2 with F = w T e^{i phi} (A w T inside
            // the Liu-Taghizadeh window, 0 outside; the window is symmetric)
            const float *sP = reinterpret_cast<const float *>(sl);
            const float *sPm = partner ? sP + NX : sP;
            const float *sTm = partner ? sTa + NX : sTa;
            const int b = item / a.nsub, sub = item - b * a.nsub;
            const int ym = (ny - pan) % ny, iy = (pan + hy) % ny, iym = (ym + hy) % ny;
            const float *wr = a.w ? a.w + ((size_t)b * ny + pan) * NX : nullptr;
            const float *wrm = a.w ? a.w + ((size_t)b * ny + ym) * NX : nullptr;
            if (!a.phase) {
                // drawn phases: one generator call per four pixels of each replay row
                // (the phase map's definition), stored as 2u where the phase rows would be
                float4 *wP = reinterpret_cast<float4 *>(sl);
                const int nrow = partner ? 2 : 1;
                for (int gi = t; gi < nrow * (NX / 4); gi += TL) {
                    const int rr = gi / (NX / 4), g4 = gi - rr * (NX / 4);
                    const uint4 w = philox4((uint32_t)((rr ? iym : iy) * (NX / 4) + g4), (uint32_t)sub, (uint32_t)(a.item0 + b),
                                            a.stream_id, a.seed_lo, a.seed_hi);
                    constexpr float k = 1.0f / 8388608.0f;
                    wP[gi] = make_float4((float)(w.x >> 8) * k, (float)(w.y >> 8) * k, (float)(w.z >> 8) * k,
                                         (float)(w.w >> 8) * k);
                }
                gsync();
            }
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const int x = t + TL * e, xm = mirror_idx<NX>(x);
                const int ix = (x + NX / 2) % NX, ixm = (xm + NX / 2) % NX;
                float amp = sTa[x], am = sTm[xm];
                if (wr) {
                    amp *= wr[x];
                    am *= wrm[xm];
                }
                if (a.lt_amp > 0.f) {
                    const bool in = lt_in(a, pan, x);
                    amp = in ? amp * a.lt_amp : 0.f;
                    am = in ? am * a.lt_amp : 0.f;
                }
                float s, c, sm, cm;
                if (a.phase) {
                    // phase in half-turns: the reduction is exact, no large-argument path
                    sincospif(sP[ix] * 0.318309886183790672f, &s, &c);
                    sincospif(sPm[ixm] * 0.318309886183790672f, &sm, &cm);
                } else {
                    sincospif(sP[ix], &s, &c);  // pi * 2u
                    sincospif(sPm[ixm], &sm, &cm);
                }
                v[e] = make_float2(0.5f * fmaf(am, cm, amp * c), 0.5f * fmaf(-am, sm, amp * s));
            });
            pair_finish<P, LAY>(v, sf, a.tw, t, gsync, a.field + ((size_t)item * ny + pan) * NX);
            gsync();
            if (t == 0) issue(k + D);
            continue;
        }
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            v[e] = sf[t + TL * e];
        });
        line_fft<P, -1, 1, LAY>(v, sf, a.tw, t, gsync);
        if constexpr (MODE == 5) {
            const int n = k % per;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                accI[e] = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, n ? accI[e] : 0.f));
            });
            if (n == per - 1) {
                // normalised time-averaged intensity of u and of -u (the same), metrics
                const float inv_sub = 1.0f / (float)per;
                const float *sTm = partner ? sTa + NX : sTa;
                const int ym = (ny - pan) % ny, iy = (pan + hy) % ny, iym = (ym + hy) % ny;
                float *Io = a.I_out ? a.I_out + (size_t)item * ny * NX : nullptr;
                float m0 = 0.f, m1 = 0.f, m2s = 0.f, m3 = 0.f;
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    const int x = t + TL * e, xm = mirror_idx<NX>(x);
                    const float I = accI[e] * inv_sub * a.invN2;
                    const float e2 = accI[e] * inv_sub * a.invN;
                    const float Tv = sTa[x];
                    const float d = I - Tv * Tv, am = sqrtf(I) - Tv;
                    m0 = fmaf(d, d, m0);
                    m1 = fmaf(am, am, m1);
                    m3 += e2;
                    if (Tv > 0.f) m2s += e2;
                    if (Io) Io[(size_t)iy * NX + (x + NX / 2) % NX] = I;
                    if (partner) {
                        const float Tm = sTm[xm];
                        const float dm = I - Tm * Tm, amm = sqrtf(I) - Tm;
                        m0 = fmaf(dm, dm, m0);
                        m1 = fmaf(amm, amm, m1);
                        m3 += e2;
                        if (Tm > 0.f) m2s += e2;
                        if (Io) Io[(size_t)iym * NX + (xm + NX / 2) % NX] = I;
                    }
                });
                if (a.part)
                    group_sum4<GT>(m0, m1, m2s, m3, red + (size_t)g * Cfg::GW * NMET,
                                   a.part + ((size_t)item * ppt + pan) * NMET, t, gsync);
            }
            gsync();
            if (t == 0) issue(k + D);
            continue;
        }
        if constexpr (MODE == 6 || MODE == 7) {
            // adaptive OSPR: every subframe's replay is Hermitian, so the running
            // sum S of the energy-normalised intensities is symmetric, S(-u) = S(u),
            // and is kept for rows ky <= ny/2 only (a.acc, DFT order)
            float *ar = a.acc + ((size_t)item * ny + pan) * NX;
            const float *sTm = partner ? sTa + NX : sTa;
            const int ym = (ny - pan) % ny, iy = (pan + hy) % ny, iym = (ym + hy) % ny;
            float sum[E];
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const float2 r = v[e];
                sum[e] = ar[t + TL * e] + fmaf(r.x, r.x, r.y * r.y) * a.invN2;
            });
            if constexpr (MODE == 6) {
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    ar[t + TL * e] = sum[e];
                });
                // the next subframe: target sqrt(max((sub + 1) T^2 - S, 0)) at u and -u,
                // its Philox phases drawn four per call into the (consumed) field area
                gsync();
                float4 *wP = reinterpret_cast<float4 *>(sl);
                for (int gi = t; gi < (partner ? 2 : 1) * (NX / 4); gi += TL) {
                    const int rr = gi / (NX / 4), g4 = gi - rr * (NX / 4);
                    const uint4 w = philox4((uint32_t)((rr ? iym : iy) * (NX / 4) + g4), (uint32_t)a.sub,
                                            (uint32_t)(a.item0 + item), a.stream_id, a.seed_lo, a.seed_hi);
                    constexpr float kk = 1.0f / 8388608.0f;
                    wP[gi] = make_float4((float)(w.x >> 8) * kk, (float)(w.y >> 8) * kk, (float)(w.z >> 8) * kk,
                                         (float)(w.w >> 8) * kk);
                }
                gsync();
                const float *sP = reinterpret_cast<const float *>(sl);
                const float *sPm = partner ? sP + NX : sP;
                const float nn = (float)(a.sub + 1);
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    const int x = t + TL * e, xm = mirror_idx<NX>(x);
                    const float Tv = sTa[x], Tm = sTm[xm];
                    const float amp = sqrtf(fmaxf(fmaf(nn, Tv * Tv, -sum[e]), 0.f));
                    const float am = sqrtf(fmaxf(fmaf(nn, Tm * Tm, -sum[e]), 0.f));
                    float sn, cs, snm, csm;
                    sincospif(sP[(x + NX / 2) % NX], &sn, &cs);  // pi * 2u
                    sincospif(sPm[(xm + NX / 2) % NX], &snm, &csm);
                    v[e] = make_float2(0.5f * fmaf(am, csm, amp * cs), 0.5f * fmaf(-am, snm, amp * sn));
                });
                pair_finish<P, LAY>(v, sf, a.tw, t, gsync, a.field + ((size_t)item * ny + pan) * NX);
            } else {
                // the time average S / nsub of u and -u, scored as in the plain OSPR average
                const float inv_sub = 1.0f / (float)a.nsub;
                float *Io = a.I_out ? a.I_out + (size_t)item * ny * NX : nullptr;
                float m0 = 0.f, m1 = 0.f, m2s = 0.f, m3 = 0.f;
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    const int x = t + TL * e, xm = mirror_idx<NX>(x);
                    const float I = sum[e] * inv_sub;
                    const float e2 = I * a.NN;
                    const float Tv = sTa[x];
                    const float d = I - Tv * Tv, am = sqrtf(I) - Tv;
                    m0 = fmaf(d, d, m0);
                    m1 = fmaf(am, am, m1);
                    m3 += e2;
                    if (Tv > 0.f) m2s += e2;
                    if (Io) Io[(size_t)iy * NX + (x + NX / 2) % NX] = I;
                    if (partner) {
                        const float Tm = sTm[xm];
                        const float dm = I - Tm * Tm, amm = sqrtf(I) - Tm;
                        m0 = fmaf(dm, dm, m0);
                        m1 = fmaf(amm, amm, m1);
                        m3 += e2;
                        if (Tm > 0.f) m2s += e2;
                        if (Io) Io[(size_t)iym * NX + (xm + NX / 2) % NX] = I;
                    }
                });
                if (a.part)
                    group_sum4<GT>(m0, m1, m2s, m3, red + (size_t)g * Cfg::GW * NMET,
                                   a.part + ((size_t)item * ppt + pan) * NMET, t, gsync);
            }
            gsync();
            if (t == 0) issue(k + D);
            continue;
        }
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
        if constexpr (MODE == 4) {
            // outputs at u (this row) and -u (row ny - pan, R(-u) = conj R(u));
            // the mirror pixels of the self-conjugate rows are this row's own
            if (a.phase_out || a.R_out) {
                const int ym = (ny - pan) % ny, iy = (pan + hy) % ny, iym = (ym + hy) % ny;
                const size_t ob = (size_t)item * ny * NX;
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    const int x = t + TL * e, xm = mirror_idx<NX>(x);
                    const int ix = (x + NX / 2) % NX, ixm = (xm + NX / 2) % NX;
                    const float2 r = v[e];
                    const bool nz = fmaf(r.x, r.x, r.y * r.y) > 0.f;
                    if (a.phase_out) {
                        a.phase_out[ob + (size_t)iy * NX + ix] = nz ? atan2f(r.y, r.x) : 0.f;
                        if (partner) a.phase_out[ob + (size_t)iym * NX + ixm] = nz ? atan2f(-r.y, r.x) : 0.f;
                    }
                    if (a.R_out) {
                        a.R_out[ob + (size_t)iy * NX + ix] = make_float2(r.x * a.invSqrtN, r.y * a.invSqrtN);
                        if (partner)
                            a.R_out[ob + (size_t)iym * NX + ixm] = make_float2(r.x * a.invSqrtN, -r.y * a.invSqrtN);
                    }
                });
            }
        }
        if constexpr (HERM) {
            float *wrp = nullptr, *wrm = nullptr;
            const float *wold = nullptr;
            if constexpr (MODE == 1 || MODE == 4) {
                wrp = a.w ? a.w + ((size_t)item * ny + pan) * NX : nullptr;
                wrm = a.w && partner ? a.w + ((size_t)item * ny + ny - pan) * NX : nullptr;
                wold = wrm;
                if (a.w && !partner) {  // self-mirrored row: keep its old weights for the mirror reads
                    float *sW = const_cast<float *>(sTa) + NX;
                    static_for<0, E>([&](auto ec) {
                        constexpr int e = decltype(ec)::value;
                        sW[t + TL * e] = wrp[t + TL * e];
                    });
                    gsync();
                    wold = sW;
                }
            }
            herm_constrain<P, MODE != 2>(v, sTa, partner ? sTa + NX : sTa, wrp, wold, wrm, partner, a, t, pan,
                                         acc0, acc1, acc2, acc3);
            if constexpr (MODE != 4)
                pair_finish<P, LAY>(v, sf, a.tw, t, gsync, a.field + ((size_t)item * ny + pan) * NX);
            gsync();
            if (t == 0) issue(k + D);
            if (a.part)
                group_sum4<GT>(acc0, acc1, acc2, acc3, red + (size_t)g * Cfg::GW * NMET,
                               a.part + ((size_t)item * ppt + pan) * NMET, t, gsync);
            continue;
        } else {
        if (partner) {
            // spectrum of row ny - p: conj(X[(nx - kx) % nx]), through shared memory;
            // its constraint is applied now and the result parked where the
            // (consumed) targets were
            gsync();
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                sf[t + TL * e] = v[e];
            });
            gsync();
            float2 vb[E];
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                const float2 q = sf[mirror_idx<NX>(t + TL * e)];
                vb[e] = make_float2(q.x, -q.y);
            });
            pair_constrain<P>(vb, sTa + NX, a.w ? a.w + ((size_t)item * ny + ny - pan) * NX : nullptr, a,
                              t, ny - pan, acc0, acc1, acc2, acc3);
            pair_constrain<P>(v, sTa, a.w ? a.w + ((size_t)item * ny + pan) * NX : nullptr, a, t, pan, acc0,
                              acc1, acc2, acc3);
            gsync();
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                park[t + TL * e] = vb[e];
            });
        } else {
            pair_constrain<P>(v, sTa, a.w ? a.w + ((size_t)item * ny + pan) * NX : nullptr, a, t, pan, acc0,
                              acc1, acc2, acc3);
        }
#pragma unroll 1
        for (int r = 0; r < (partner ? 2 : 1); ++r) {
            if (r == 1)
                static_for<0, E>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    v[e] = park[t + TL * e];
                });
            pair_finish<P, LAY>(v, sf, a.tw, t, gsync,
                                a.field + ((size_t)item * ny + (r ? ny - pan : pan)) * NX);
        }
        gsync();
        if (t == 0) issue(k + D);  // slot fully consumed: refill it
        if (a.part)
            group_sum4<GT>(acc0, acc1, acc2, acc3, red + (size_t)g * Cfg::GW * NMET,
                           a.part + ((size_t)item * ppt + pan) * NMET, t, gsync);
        }
    }
}

// ----------------------------------------------------------- column pass
template <class P, int C, int NG, int D, int SWZ, int BOXR, bool EB = false>
struct ColPipeCfg {
    static constexpr int GT = P::TL * C;
    static_assert(GT % 32 == 0, "column group must be whole warps");
    static_assert(P::N % BOXR == 0 && BOXR <= 256, "box rows must tile the column");
    static constexpr int THREADS = NG * GT;
    static constexpr int SLOT = P::N * C * 8;
    // EB: each group also holds the illumination tile of its panel
    static constexpr int NE = EB ? NG : 0;
    static constexpr size_t SMEM = 1024 + (size_t)(NG * D + NE) * SLOT + (NG * D + NE) * 8 + 4 * (NG + 1) + 256;
};

// Column pass of the GS loop (binary, L-level or modulated quantiser): each
// group of TL x C threads transforms C columns of one target per job, with the
// panels brought in by tensor copies through a ring of D slots.  EB (modulated
// plans): the illumination tile of the job's panel (C columns x all rows of E,
// a second tensor map over [ny][nx] float2) is copied into the group's own
// buffer at the start of the job, so the quantiser reads E from shared memory;
// the copy overlaps the inverse transform.
template <class P, int ROLE, int C, int NG, int D, int SWZ, int BOXR, int MINB = 1, bool EB = false>
__global__ void __launch_bounds__(ColPipeCfg<P, C, NG, D, SWZ, BOXR, EB>::THREADS, MINB)
    k_col_pipe(const ColArgs a, const PipeArgs pa, const __grid_constant__ CUtensorMap tmap,
               const __grid_constant__ CUtensorMap emap) {
    static_assert(!EB || ROLE == COL_GS_MOD, "illumination tiles serve the modulated quantiser");
    using Cfg = ColPipeCfg<P, C, NG, D, SWZ, BOXR, EB>;
    using LAY = Swz<SWZ>;
    constexpr int TL = P::TL, E = P::E, NY = P::N, GT = Cfg::GT;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *ebuf = base + (size_t)NG * D * Cfg::SLOT;
    uint64_t *full = reinterpret_cast<uint64_t *>(ebuf + (size_t)Cfg::NE * Cfg::SLOT);
    uint64_t *ebar = full + NG * D;
    volatile int *flags = reinterpret_cast<volatile int *>(ebar + Cfg::NE);
    volatile int *abort = flags + NG;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NG * D + Cfg::NE; ++i) mbar_init(full + i, 1);
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int nx = a.nx;
    const int ppt = (nx + C - 1) / C;
    const int J = a.items * ppt;
    const int g = tid / GT, gt = tid - g * GT;
    const int c = gt % C, t = gt / C;
    unsigned char *ring = base + (size_t)g * D * Cfg::SLOT;
    uint64_t *gfull = full + g * D;
    auto gsync = [g]() { named_sync(1 + g, GT); };
    auto job = [&](int k) { return (int)blockIdx.x + (g + NG * k) * (int)gridDim.x; };
    // rows to bring in: all, or 0 .. ny/2 of a Hermitian-column field, as whole
    // boxes plus (when one row is left over) a single-row bulk copy
    const int rows_in = a.half_in ? NY / 2 + 1 : NY;
    const int nbox = rows_in / BOXR, rem = rows_in - nbox * BOXR;
    const int nbox_t = nbox + (rem > 1 ? 1 : 0);
    const uint32_t slot_bytes = (uint32_t)(nbox_t * BOXR * C * 8 + (rem == 1 ? C * 8 : 0));
    auto issue = [&](int k) {  // copy the group's k-th panel: C columns, the rows above
        const int j = job(k);
        if (j >= J || j == pa.drop_job) return;
        const int item = j / ppt, pan = j - item * ppt;
        unsigned char *sl = ring + (size_t)(k % D) * Cfg::SLOT;
        mbar_expect_tx(gfull + k % D, slot_bytes);
#pragma unroll 1
        for (int r = 0; r < nbox_t; ++r)
            tma_load_2d(sl + (size_t)r * BOXR * C * 8, &tmap, 2 * pan * C, item * NY + r * BOXR,
                        gfull + k % D);
        if (rem == 1)
            bulk_g2s(sl + (size_t)nbox * BOXR * C * 8, a.field + ((size_t)item * NY + nbox * BOXR) * nx + pan * C,
                     C * 8, gfull + k % D);
    };
    auto drain = [&](int k0, int k1) {
        for (int q = k0; q < k1; ++q) {
            const int j = job(q);
            if (j < J && j != pa.drop_job) mbar_wait(gfull + q % D, (q / D) & 1, pa.wait_ns, nullptr);
        }
    };
    if (gt == 0)
        for (int k = 0; k < D; ++k) issue(k);

    for (int k = 0;; ++k) {
        const int j = job(k);
        if (j >= J) break;
        if (gt == 0) {
            bool ok = !*abort && mbar_wait(gfull + k % D, (k / D) & 1, pa.wait_ns, abort);
            if (!ok) {
                atomicOr(pa.err, ERR_TIMEOUT_BIT);
                *abort = 1;
            }
            flags[g] = ok;
        }
        gsync();
        if (!flags[g]) {
            if (gt == 0) drain(k, k + D);
            break;
        }
        const int item = j / ppt, pan = j - item * ppt;
        const int x = pan * C + c;
        const bool act = x < nx;
        const float2 *se = reinterpret_cast<const float2 *>(ebuf + (size_t)g * Cfg::SLOT);
        if constexpr (EB) {
            // the previous job's readers of this buffer passed the group
            // barriers of its forward transform
            if (gt == 0) {
                mbar_expect_tx(ebar + g, (uint32_t)(NY * C * 8));
#pragma unroll 1
                for (int r = 0; r < NY / BOXR; ++r)
                    tma_load_2d(ebuf + (size_t)g * Cfg::SLOT + (size_t)r * BOXR * C * 8, &emap, 2 * pan * C,
                                r * BOXR, ebar + g);
            }
        }
        float2 *sl = reinterpret_cast<float2 *>(ring + (size_t)(k % D) * Cfg::SLOT);
        float2 v[E];
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const int n = t + TL * e;
            if (a.half_in && n > NY / 2) {
                const float2 q = sl[(NY - n) * C + c];
                v[e] = make_float2(q.x, -q.y);
            } else {
                v[e] = sl[n * C + c];
            }
        });
        line_fft<P, +1, C, LAY>(v, sl + c, a.tw, t, gsync);
        if constexpr (EB) {
            if (gt == 0) {
                bool ok = !*abort && mbar_wait(ebar + g, k & 1, pa.wait_ns, abort);
                if (!ok) {
                    atomicOr(pa.err, ERR_TIMEOUT_BIT);
                    *abort = 1;
                    mbar_wait(ebar + g, k & 1, pa.wait_ns, nullptr);  // the copy still lands here
                }
                flags[g] = ok;
            }
            gsync();
            if (!flags[g]) {
                if (gt == 0) drain(k + 1, k + D);
                break;
            }
        }
        const size_t base_o = (size_t)item * NY * nx;
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const int o = (t + TL * e) * nx + x;
            const float2 h = v[e];
            int q;
            float2 ph;
            if constexpr (ROLE == COL_GS_MOD) {
                // as the generic column pass: the level nearest h / E, light E x level
                const float2 E = EB ? se[(t + TL * e) * C + c]
                                    : __ldg(a.illum + (size_t)(t + TL * e) * nx + (act ? x : nx - 1));
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
                if (a.h_out) a.h_out[base_o + o] = make_float2(h.x * a.invSqrtN, h.y * a.invSqrtN);
                if (a.holo) a.holo[base_o + o] = (uint8_t)q;
            }
            v[e] = ph;
        });
        line_fft<P, -1, C, LAY>(v, sl + c, a.tw, t, gsync);
        gsync();
        if (gt == 0) issue(k + D);  // slot fully consumed: refill it
        if (act) {
            float2 *fw = a.field + base_o + x;
            static_for<0, E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                if (!a.half || t + TL * e <= NY / 2) fw[(t + TL * e) * nx] = v[e];
            });
        }
    }
}


// -------------------------- column pass of the Hermitian binary loop (pairs)
// In the Hermitian loop (see herm_constrain) every column of the field is
// Hermitian in ky, so its inverse FFT is real, and so is its binary
// hologram; two columns a and b therefore share every transform.  The
// inverse FFT of A + iB gives a + ib, whose signs are the two columns'
// binary levels; the forward FFT of z = qa + i qb gives Z, and
// QA[k] = (Z[k] + conj Z[N-k]) / 2, QB[k] = (Z[k] - conj Z[N-k]) / (2i).
// Reads rows 0 .. ny/2 (the rest by conjugation), writes rows <= ny/2 (all
// rows when a.half == 0).  C columns (C/2 pairs) per CTA, ring depth D.
template <class P, int C, int D, int SWZ, int BOXR>
struct ColHermCfg {
    static constexpr int CP = C / 2;
    static constexpr int GT = P::TL * CP;
    static_assert(C % 2 == 0 && GT % 32 == 0, "column pairs must fill whole warps");
    static_assert(BOXR <= 256, "box rows");
    static constexpr int THREADS = GT;
    static constexpr int ROWS_IN = P::N / 2 + 1;
    static constexpr int NBOX = ROWS_IN / BOXR, REM = ROWS_IN - NBOX * BOXR;
    static constexpr int NBOX_T = NBOX + (REM > 1 ? 1 : 0);
    static constexpr int LOAD = NBOX_T * BOXR * C * 8 + (REM == 1 ? C * 8 : 0);
    static constexpr int XCH = P::N * CP * 8;
    static constexpr int SLOT = ((LOAD > XCH ? LOAD : XCH) + 1023) / 1024 * 1024;
    static constexpr size_t SMEM = 1024 + (size_t)D * SLOT + D * 8 + 16 + 256;
};

template <class P, int C, int D, int SWZ, int BOXR, int MINB = 1>
__global__ void __launch_bounds__(ColHermCfg<P, C, D, SWZ, BOXR>::THREADS, MINB)
    k_col_pipe_herm(const ColArgs a, const PipeArgs pa, const __grid_constant__ CUtensorMap tmap) {
    using Cfg = ColHermCfg<P, C, D, SWZ, BOXR>;
    using LAY = Swz<SWZ>;
    constexpr int TL = P::TL, E = P::E, NY = P::N, CP = Cfg::CP, HY = NY / 2;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + (size_t)D * Cfg::SLOT);
    volatile int *flags = reinterpret_cast<volatile int *>(full + D);
    volatile int *abort = flags + 1;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < D; ++i) mbar_init(full + i, 1);
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int nx = a.nx;
    const int ppt = (nx + C - 1) / C;
    const int J = a.items * ppt;
    const int cp = tid % CP, t = tid / CP;
    auto sync = []() { __syncthreads(); };
    auto job = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
    auto issue = [&](int k) {
        const int j = job(k);
        if (j >= J || j == pa.drop_job) return;
        const int item = j / ppt, pan = j - item * ppt;
        unsigned char *sl = base + (size_t)(k % D) * Cfg::SLOT;
        mbar_expect_tx(full + k % D, (uint32_t)Cfg::LOAD);
#pragma unroll 1
        for (int r = 0; r < Cfg::NBOX_T; ++r)
            tma_load_2d(sl + (size_t)r * BOXR * C * 8, &tmap, 2 * pan * C, item * NY + r * BOXR, full + k % D);
        if constexpr (Cfg::REM == 1)
            bulk_g2s(sl + (size_t)Cfg::NBOX * BOXR * C * 8,
                     a.field + ((size_t)item * NY + Cfg::NBOX * BOXR) * nx + pan * C, C * 8, full + k % D);
    };
    auto drain = [&](int k0, int k1) {
        for (int q = k0; q < k1; ++q) {
            const int j = job(q);
            if (j < J && j != pa.drop_job) mbar_wait(full + q % D, (q / D) & 1, pa.wait_ns, nullptr);
        }
    };
    if (tid == 0)
        for (int k = 0; k < D; ++k) issue(k);

    for (int k = 0;; ++k) {
        const int j = job(k);
        if (j >= J) break;
        if (tid == 0) {
            bool ok = !*abort && mbar_wait(full + k % D, (k / D) & 1, pa.wait_ns, abort);
            if (!ok) {
                atomicOr(pa.err, ERR_TIMEOUT_BIT);
                *abort = 1;
            }
            flags[0] = ok;
        }
        sync();
        if (!flags[0]) {
            if (tid == 0) drain(k, k + D);
            break;
        }
        const int item = j / ppt, pan = j - item * ppt;
        const int xa = pan * C + 2 * cp;
        const bool act = xa + 1 < nx;
        float2 *sl = reinterpret_cast<float2 *>(base + (size_t)(k % D) * Cfg::SLOT);
        float2 v[E];
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const int n = t + TL * e;
            float2 A, B;
            if (n <= HY) {
                A = sl[n * C + 2 * cp];
                B = sl[n * C + 2 * cp + 1];
            } else {
                const float2 qa = sl[(NY - n) * C + 2 * cp], qb = sl[(NY - n) * C + 2 * cp + 1];
                A = make_float2(qa.x, -qa.y);
                B = make_float2(qb.x, -qb.y);
            }
            v[e] = make_float2(A.x - B.y, A.y + B.x);  // A + iB
        });
        line_fft<P, +1, CP, LAY>(v, sl + cp, a.tw, t, sync);
        const size_t base_o = (size_t)item * NY * nx;
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const int n = t + TL * e;
            const int qa = v[e].x >= 0.f ? 0 : 1, qb = v[e].y >= 0.f ? 0 : 1;
            if (act && a.holo)
                *reinterpret_cast<uint16_t *>(a.holo + base_o + (size_t)n * nx + xa) = (uint16_t)(qa | (qb << 8));
            v[e] = make_float2(qa ? -1.f : 1.f, qb ? -1.f : 1.f);
        });
        line_fft<P, -1, CP, LAY>(v, sl + cp, a.tw, t, sync);
        // separate the two spectra through Z[N - k]
        sync();
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            sl[(t + TL * e) * CP + cp] = v[e];
        });
        sync();
        float4 *fw = reinterpret_cast<float4 *>(a.field + base_o + xa);
        static_for<0, E>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            const int kk = t + TL * e;
            const float2 z = v[e], zm = sl[mirror_idx<NY>(kk) * CP + cp];
            if (act && (!a.half || kk <= HY))
                fw[(size_t)kk * nx / 2] = make_float4(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y),
                                                     0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
        });
        sync();
        if (tid == 0) issue(k + D);  // slot fully consumed: refill it
    }
}

// --------------------------------------------------------- dispatch glue

struct PipeOps {
    int N;
    const char *name;
    int row_threads, col_threads, col_c, col_boxr, row_lines;
    size_t row_smem, col_smem;
    int row_blocks_per_sm, col_blocks_per_sm;
    int col_mod_blocks_per_sm;  // CTAs per SM of the modulated column pass
    int col_emap;               // the modulated column pass reads E through a tensor map
    int paired;  // row pass is k_row_pipe_pair (binary SLM, even ny, half-row column stores)
    cudaError_t (*init)(PipeOps *self);
    void (*row_iter)(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s);  // may be null
    void (*col_gs)(int role, const ColArgs &a, const PipeArgs &pa, const CUtensorMap &m, const CUtensorMap &em,
                   int grid, cudaStream_t s);  // may be null
    // column pass of the Hermitian binary loop, two columns per transform (may be null);
    // its tensor map has boxes of herm_c columns x herm_boxr rows
    void (*col_herm)(const ColArgs &a, const PipeArgs &pa, const CUtensorMap &m, int grid, cudaStream_t s);
    int herm_c, herm_boxr, herm_blocks_per_sm;
    // Hermitian head and tail of the binary loop on the paired row kernel
    // (rows ky <= ny/2; may be null)
    void (*row_head)(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s);
    void (*row_tail)(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s);
    // Hermitian OSPR time average on the paired row kernel (may be null)
    void (*row_avg)(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s);
    // Hermitian adaptive-OSPR step (last: the final average) on the paired row kernel (may be null)
    void (*row_adapt)(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s, bool last);
};

// Row pass: plan P, LINES rows per group, NGR groups, ring depth DR, swizzle
// SWZR (LINES == 0: no TMA-fed row pass).  Column pass: plan PC, C columns per
// group, NGC groups, ring depth DC, swizzle SWZC, BOXR rows per tensor copy,
// at least MINBC CTAs per SM (the register budget); EBC: the modulated
// quantiser reads the illumination from a shared-memory tile per group.
template <class P, int LINES, int NGR, int DR, int SWZR, class PC, int C, int NGC, int DC, int SWZC,
          int BOXR, int MINBC = 1, bool EBC = false>
struct PipeImpl {
    using CC = ColPipeCfg<PC, C, NGC, DC, SWZC, BOXR>;
    using CCM = ColPipeCfg<PC, C, NGC, DC, SWZC, BOXR, EBC>;  // the modulated pass
    template <int ROLE, bool EB = false>
    static constexpr auto col_kernel() { return k_col_pipe<PC, ROLE, C, NGC, DC, SWZC, BOXR, MINBC, EB>; }
    static cudaError_t init(PipeOps *self) {
        cudaError_t e = cudaSuccess;
        int rb = 1, cb = 0, mb = 0;
        if constexpr (LINES > 0) {
            using RC = RowPipeCfg<P, LINES, NGR, DR, SWZR>;
            for (const void *f : {(const void *)k_row_pipe<P, LINES, NGR, DR, SWZR, false>,
                                  (const void *)k_row_pipe<P, LINES, NGR, DR, SWZR, true>})
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::SMEM);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &rb, k_row_pipe<P, LINES, NGR, DR, SWZR, false>, RC::THREADS, RC::SMEM);
        }
        for (const void *f : {(const void *)col_kernel<COL_GS_BIN>(), (const void *)col_kernel<COL_GS_LVL>()})
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void *)col_kernel<COL_GS_MOD, EBC>(),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CCM::SMEM);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cb, col_kernel<COL_GS_BIN>(), CC::THREADS,
                                                              CC::SMEM);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mb, col_kernel<COL_GS_MOD, EBC>(), CCM::THREADS,
                                                              CCM::SMEM);
        if (e != cudaSuccess) return e;
        if (rb < 1 || cb < 1 || mb < 1) return cudaErrorInvalidConfiguration;
        self->row_blocks_per_sm = rb;
        self->col_blocks_per_sm = cb;
        self->col_mod_blocks_per_sm = mb;
        return cudaSuccess;
    }
    static void row_iter(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s) {
        if constexpr (LINES > 0) {
            using RC = RowPipeCfg<P, LINES, NGR, DR, SWZR>;
            if (a.gen) k_row_pipe<P, LINES, NGR, DR, SWZR, true><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
            else k_row_pipe<P, LINES, NGR, DR, SWZR, false><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
        }
    }
    // em: the illumination's tensor map (boxes as the field's), read by the
    // modulated pass of an EBC variant
    static void col_gs(int role, const ColArgs &a, const PipeArgs &pa, const CUtensorMap &m, const CUtensorMap &em,
                       int grid, cudaStream_t s) {
        if (role == COL_GS_BIN)
            col_kernel<COL_GS_BIN>()<<<grid, CC::THREADS, CC::SMEM, s>>>(a, pa, m, m);
        else if (role == COL_GS_MOD)
            col_kernel<COL_GS_MOD, EBC>()<<<grid, CCM::THREADS, CCM::SMEM, s>>>(a, pa, m, em);
        else
            col_kernel<COL_GS_LVL>()<<<grid, CC::THREADS, CC::SMEM, s>>>(a, pa, m, m);
    }
    static PipeOps make(const char *name) {
        PipeOps o{};
        o.N = P::N;
        o.name = name;
        o.col_threads = CC::THREADS;
        o.col_c = C;
        o.col_boxr = BOXR;
        o.col_smem = CC::SMEM;
        o.col_emap = EBC;
        o.row_lines = LINES;
        if constexpr (LINES > 0) {
            using RC = RowPipeCfg<P, LINES, NGR, DR, SWZR>;
            o.row_threads = RC::THREADS;
            o.row_smem = RC::SMEM;
            o.row_iter = &row_iter;
        }
        o.init = &init;
        o.col_gs = &col_gs;
        return o;
    }
};


// A paired-row variant: plan P (TL a multiple of 32), NG groups, ring depth D,
// swizzle SWZ, at least MINB CTAs per SM (the register budget), and the
// column pass of another variant `col`.
template <class P, int NG, int D, int SWZ, int MINB = 1>
struct PairImpl {
    using RC = PairPipeCfg<P, NG, D, SWZ>;
    static cudaError_t init_row(int *blocks) {
        cudaError_t e = cudaSuccess;
        for (const void *f : {(const void *)k_row_pipe_pair<P, NG, D, SWZ, 0, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 1, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 2, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 3, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 4, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 5, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 6, MINB>,
                              (const void *)k_row_pipe_pair<P, NG, D, SWZ, 7, MINB>})
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::SMEM);
        // the block count of the general Hermitian kernel (the most registers)
        // sizes the grid of every mode
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_row_pipe_pair<P, NG, D, SWZ, 1, MINB>,
                                                              RC::THREADS, RC::SMEM);
        return e;
    }
    static void row_iter(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s) {
        if (!a.herm) k_row_pipe_pair<P, NG, D, SWZ, 0, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
        else if (a.w || a.lt_amp > 0.f)
            k_row_pipe_pair<P, NG, D, SWZ, 1, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
        else k_row_pipe_pair<P, NG, D, SWZ, 2, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
    }
    static void row_head(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s) {
        k_row_pipe_pair<P, NG, D, SWZ, 3, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
    }
    static void row_tail(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s) {
        k_row_pipe_pair<P, NG, D, SWZ, 4, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
    }
    static void row_avg(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s) {
        k_row_pipe_pair<P, NG, D, SWZ, 5, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
    }
    static void row_adapt(const RowArgs &a, const PipeArgs &pa, int grid, cudaStream_t s, bool last) {
        if (last) k_row_pipe_pair<P, NG, D, SWZ, 7, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
        else k_row_pipe_pair<P, NG, D, SWZ, 6, MINB><<<grid, RC::THREADS, RC::SMEM, s>>>(a, pa);
    }
};

// Column-pair Hermitian column pass launcher (see k_col_pipe_herm); MINB:
// at least that many CTAs per SM (the register budget).
template <class P, int C, int D, int SWZ, int BOXR, int MINB = 1>
struct HermImpl {
    using CC = ColHermCfg<P, C, D, SWZ, BOXR>;
    static constexpr int COLS = C, BOX_ROWS = BOXR;
    static cudaError_t init(int *blocks) {
        cudaError_t e = cudaFuncSetAttribute((const void *)k_col_pipe_herm<P, C, D, SWZ, BOXR, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::SMEM);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_col_pipe_herm<P, C, D, SWZ, BOXR, MINB>,
                                                              CC::THREADS, CC::SMEM);
        return e;
    }
    static void launch(const ColArgs &a, const PipeArgs &pa, const CUtensorMap &m, int grid, cudaStream_t s) {
        k_col_pipe_herm<P, C, D, SWZ, BOXR, MINB><<<grid, CC::THREADS, CC::SMEM, s>>>(a, pa, m);
    }
};

struct NoHerm {
    static constexpr int COLS = 0, BOX_ROWS = 0;
    static cudaError_t init(int *blocks) {
        *blocks = 0;
        return cudaSuccess;
    }
    static constexpr void (*launch)(const ColArgs &, const PipeArgs &, const CUtensorMap &, int,
                                    cudaStream_t) = nullptr;
};

// Combines a paired row pass with the column pass of an existing variant and
// optionally a column-pair pass for the Hermitian binary loop.
template <class PAIR, const PipeOps *COL, class HERM = NoHerm>
struct PairedOps {
    static cudaError_t init(PipeOps *self) {
        cudaError_t e = COL->init(const_cast<PipeOps *>(COL));
        if (e != cudaSuccess) return e;
        int rb = 0, hb = 0;
        e = PAIR::init_row(&rb);
        if (e == cudaSuccess) e = HERM::init(&hb);
        if (e != cudaSuccess) return e;
        if (rb < 1) return cudaErrorInvalidConfiguration;
        self->row_blocks_per_sm = rb;
        self->col_blocks_per_sm = COL->col_blocks_per_sm;
        self->col_mod_blocks_per_sm = COL->col_mod_blocks_per_sm;
        self->herm_blocks_per_sm = hb;
        if (hb < 1) self->col_herm = nullptr;
        return cudaSuccess;
    }
    static PipeOps make(const char *name) {
        PipeOps o = *COL;
        o.name = name;
        o.paired = 1;
        o.row_lines = 2;  // two rows per panel except the self-conjugate rows 0 and ny/2
        o.row_threads = PAIR::RC::THREADS;
        o.row_smem = PAIR::RC::SMEM;
        o.row_iter = &PAIR::row_iter;
        o.row_head = &PAIR::row_head;
        o.row_tail = &PAIR::row_tail;
        o.row_avg = &PAIR::row_avg;
        o.row_adapt = &PAIR::row_adapt;
        o.col_herm = HERM::launch;
        o.herm_c = HERM::COLS;
        o.herm_boxr = HERM::BOX_ROWS;
        o.init = &init;
        return o;
    }
};

// A column variant that also offers the column-pair pass of the Hermitian
// binary loop for its column length (lengths without a paired row pass).
template <const PipeOps *BASE, class HERM>
struct WithHerm {
    static cudaError_t init(PipeOps *self) {
        cudaError_t e = BASE->init(const_cast<PipeOps *>(BASE));
        if (e != cudaSuccess) return e;
        int hb = 0;
        e = HERM::init(&hb);
        if (e != cudaSuccess) return e;
        self->row_blocks_per_sm = BASE->row_blocks_per_sm;
        self->col_blocks_per_sm = BASE->col_blocks_per_sm;
        self->col_mod_blocks_per_sm = BASE->col_mod_blocks_per_sm;
        self->herm_blocks_per_sm = hb;
        if (hb < 1) self->col_herm = nullptr;
        return cudaSuccess;
    }
    static PipeOps make(const char *name) {
        PipeOps o = *BASE;
        o.name = name;
        o.col_herm = HERM::launch;
        o.herm_c = HERM::COLS;
        o.herm_boxr = HERM::BOX_ROWS;
        o.init = &init;
        return o;
    }
};

// Candidate pipelined variants for a line length (count returned, up to max
// written); the first is the default when autotuning is off.
int pipe_ops_mid(int n, const PipeOps **out, int max);
int pipe_ops_1024(int n, const PipeOps **out, int max);
int pipe_ops_2048(int n, const PipeOps **out, int max);
int pipe_ops_hd(int n, const PipeOps **out, int max);

}  // namespace hg
