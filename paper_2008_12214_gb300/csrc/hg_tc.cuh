// hg_tc.cuh -- the row pass of a GS iteration with its radix-32 DFT stages on
// the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// A 1024-point row transform is two radix-32 stages (four-step, as in the
// CUDA-core engine).  Four rows form one tile: each stage is one GEMM
//   D[128 x 64] = A[128 x 64] . B[64 x 64]^T
// where the 128 GEMM rows are the tile's 4 x 32 length-32 vectors, the 64
// columns are those vectors' interleaved (re, im) parts, and B is the 32-point
// DFT matrix in real form (B[2k][2n] = Re W, B[2k][2n+1] = -Im W,
// B[2k+1][2n] = Im W, B[2k+1][2n+1] = Re W, W = exp(DIR 2 pi i n k / 32)).
// Operands are FP16 or BF16 with FP32 accumulation; the "split" precisions
// write every operand as hi + lo and accumulate hi.hi + hi.lo + lo.hi, which
// keeps about 22 (FP16) or 16 (BF16) significant bits.  Each warp's rows are
// scaled by a power of two before rounding (exact; keeps FP16 in range).
// Stage 0 writes A K-major (a thread writes its own vector); stage 1 needs the
// transposed vectors and writes A MN-major (16-byte stores).  Twiddles, the
// replay constraint and the metrics stay in FP32 on the CUDA cores.
//
// Shared-memory operand layouts (no swizzle, canonical 8-row x 16-byte core
// matrices): K-major element (r, k) at (r/8)*1024 + (k/8)*128 + (r%8)*16 +
// (k%8)*2 (LBO 128 = K step, SBO 1024 = 8-row step); MN-major element (m, k)
// at (m/8)*1152 + (k/8)*144 + (k%8)*16 + (m%8)*2 (LBO 144 = K step, SBO 1152 =
// 8-row step; 16 bytes of padding per K group spread the stores over banks).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "hg_kernels.cuh"

namespace hg {

template <int PREC>
struct TcPrec;  // 1 FP16 hi+lo, 2 FP16, 3 BF16 hi+lo, 4 BF16
template <>
struct TcPrec<1> {
    using T = __half;
    static constexpr bool SPLIT = true;
    static constexpr uint32_t FMT = 0;
};
template <>
struct TcPrec<2> {
    using T = __half;
    static constexpr bool SPLIT = false;
    static constexpr uint32_t FMT = 0;
};
template <>
struct TcPrec<3> {
    using T = __nv_bfloat16;
    static constexpr bool SPLIT = true;
    static constexpr uint32_t FMT = 1;
};
template <>
struct TcPrec<4> {
    using T = __nv_bfloat16;
    static constexpr bool SPLIT = false;
    static constexpr uint32_t FMT = 1;
};

__device__ __forceinline__ __half tc_cvt(float x, __half *) { return __float2half_rn(x); }
__device__ __forceinline__ __nv_bfloat16 tc_cvt(float x, __nv_bfloat16 *) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float tc_back(__half h) { return __half2float(h); }
__device__ __forceinline__ float tc_back(__nv_bfloat16 h) { return __bfloat162float(h); }

constexpr int TC_N = 1024;      // row length served
constexpr int TC_B = 8192;      // one 64 x 64 16-bit matrix
constexpr int TC_A0 = 16384;    // 128 x 64, K-major
constexpr int TC_A1 = 18432;    // 128 x 64, MN-major with padding
// Shared-memory layout per precision: the 4 B matrices, then the stage-0 and
// stage-1 A operands (a low half of each only for the hi+lo precisions), then
// the barrier, TMEM slot, flag and reduction.  Without the low halves a CTA
// needs 69 KB instead of 104 KB, so three fit on an SM instead of two.
template <bool SPLIT>
struct TcLayout {
    static constexpr int NA = SPLIT ? 2 : 1;
    static constexpr int A0 = 4 * TC_B;
    static constexpr int A1 = A0 + NA * TC_A0;
    static constexpr int BAR = A1 + NA * TC_A1;
    static constexpr int SMEM = 1024 + BAR + 256;
    static_assert(TC_A0 + TC_A1 >= 4 * 1024 * 8, "the 2048 exchange buffer reuses the operand memory");
};

struct TcArgs {
    const uint4 *bmats;  // [fwd hi, fwd lo, inv hi, inv lo], each 64 x 64 K-major canonical
    unsigned *err;
    unsigned long long wait_ns;
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Row `lane` of this warp's 32 tensor-memory lanes, 64 FP32 columns.
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float (&d)[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
        "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63},"
        " [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]),
          "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
          "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
          "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
          "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 64; ++j) d[j] = __uint_as_float(r[j]);
}

// Power-of-two scale that brings the warp's largest |component| near 2^14.
__device__ __forceinline__ float tc_warp_scale(const float2 (&v)[32]) {
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < 32; ++e) m = fmaxf(m, fmaxf(fabsf(v[e].x), fabsf(v[e].y)));
#pragma unroll
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (!(m > 0.f) || isinf(m)) return 1.f;
    int ex;
    frexpf(m, &ex);  // m = f * 2^ex, f in [0.5, 1)
    // both the scale and its inverse must stay finite normal floats: rows of
    // denormal values (targets' far tails) would otherwise scale to infinity
    const int sh = max(-126, min(126, 14 - ex));
    return ldexpf(1.f, sh);
}

template <class T>
__device__ __forceinline__ uint32_t tc_pack(T a, T b) {
    return (uint32_t)(*reinterpret_cast<uint16_t *>(&a)) | ((uint32_t)(*reinterpret_cast<uint16_t *>(&b)) << 16);
}

// One radix-32 GEMM stage's MMAs, issued by one thread: K = 64 as 4 steps.
template <class PR>
__device__ __forceinline__ void tc_issue(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, bool mn_major,
                                         uint32_t b_hi, uint32_t b_lo) {
    const uint32_t idesc = (1u << 4) | (PR::FMT << 7) | (PR::FMT << 10) | ((mn_major ? 1u : 0u) << 15) |
                           ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const uint32_t ao = mn_major ? s * 288 : s * 256;
        const uint32_t albo = mn_major ? 144 : 128, asbo = mn_major ? 1152 : 1024;
        const uint64_t ah = tc_desc(a_hi + ao, albo, asbo);
        const uint64_t bh = tc_desc(b_hi + s * 256, 128, 1024);
        tc_mma(tmem, ah, bh, idesc, s > 0);
        if constexpr (PR::SPLIT) {
            tc_mma(tmem, ah, tc_desc(b_lo + s * 256, 128, 1024), idesc, 1);
            tc_mma(tmem, tc_desc(a_lo + ao, albo, asbo), bh, idesc, 1);
        }
    }
}

struct TcCtx {
    unsigned char *sm;   // 1024-aligned base
    uint64_t *bar;
    volatile int *flag;  // thread 0's wait result, shared with the CTA
    uint32_t tmem;
    uint32_t phase;
    bool ok;
};

// Thread 0 waits (bounded) for the MMAs committed to c.bar and shares the
// outcome, so every thread of the CTA takes the same path afterwards.
__device__ __forceinline__ bool tc_wait(TcCtx &c, unsigned long long limit, unsigned *err) {
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait(c.bar, c.phase, limit, nullptr);
        if (!ok) atomicOr(err, ERR_TIMEOUT_BIT);
        *c.flag = ok;
    }
    c.phase ^= 1u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *c.flag != 0;
}

// Forward (DIR = -1) or inverse (+1) 1024-point transform of the 4 lines held
// by the CTA (warp r holds line r, thread `lane` samples lane + 32 e on entry
// and on exit), unnormalised like the CUDA-core engine.  tw holds the roots of
// order 1024 * TWS (W_1024^j = tw[TWS j]).
template <int PREC, int DIR, int TWS = 1>
__device__ __forceinline__ void tc_fft(float2 (&v)[32], TcCtx &c, const float2 *__restrict__ tw,
                                       const TcArgs &ta) {
    using PR = TcPrec<PREC>;
    using T = typename PR::T;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    using L = TcLayout<PR::SPLIT>;
    unsigned char *B0 = c.sm + (DIR < 0 ? 0 : 2 * TC_B);
    unsigned char *A0h = c.sm + L::A0, *A0l = A0h + TC_A0;  // low halves: hi+lo precisions only
    unsigned char *A1h = c.sm + L::A1, *A1l = A1h + TC_A1;
    T *tag = nullptr;

    // ---- stage 0: vector (warp, lane), DFT over n2 = e
    const float s0 = tc_warp_scale(v);
    const int m = tid;
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // K chunk j: complex n2 = 4j .. 4j+3
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float re = v[4 * j + q].x * s0, im = v[4 * j + q].y * s0;
            const T hr = tc_cvt(re, tag), hi = tc_cvt(im, tag);
            h[q] = tc_pack(hr, hi);
            if constexpr (PR::SPLIT) l[q] = tc_pack(tc_cvt(re - tc_back(hr), tag), tc_cvt(im - tc_back(hi), tag));
        }
        const int off = (m >> 3) * 1024 + j * 128 + (m & 7) * 16;
        *reinterpret_cast<uint4 *>(A0h + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if constexpr (PR::SPLIT) *reinterpret_cast<uint4 *>(A0l + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        tc_issue<PR>(c.tmem, smem_addr(A0h), smem_addr(A0l), false, smem_addr(B0), smem_addr(B0 + TC_B));
        tc_commit(c.bar);
    }
    c.ok = tc_wait(c, ta.wait_ns, ta.err) && c.ok;
    if (!c.ok) return;  // uniform across the CTA
    float d[64];
    tc_ld64(c.tmem + ((uint32_t)(warp * 32) << 16), d);
    const float inv0 = 1.f / s0;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
        float2 y = make_float2(d[2 * k2] * inv0, d[2 * k2 + 1] * inv0);
        if (k2) y = cmul_root<DIR>(y, __ldg(tw + TWS * lane * k2));  // W_1024^{n1 k2}
        v[k2] = y;
    }
    // ---- stage 1: vector (warp, k2), DFT over n1 = lane; operand written MN-major
    const float s1 = tc_warp_scale(v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {      // k2 = 8g .. 8g+7 (8 consecutive M rows)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {  // re / im: K index 2 lane + cc
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float a0 = (cc ? v[8 * g + 2 * q].y : v[8 * g + 2 * q].x) * s1;
                const float a1 = (cc ? v[8 * g + 2 * q + 1].y : v[8 * g + 2 * q + 1].x) * s1;
                const T h0 = tc_cvt(a0, tag), h1 = tc_cvt(a1, tag);
                h[q] = tc_pack(h0, h1);
                if constexpr (PR::SPLIT) l[q] = tc_pack(tc_cvt(a0 - tc_back(h0), tag), tc_cvt(a1 - tc_back(h1), tag));
            }
            const int k = 2 * lane + cc;
            const int off = (warp * 4 + g) * 1152 + (k >> 3) * 144 + (k & 7) * 16;
            *reinterpret_cast<uint4 *>(A1h + off) = make_uint4(h[0], h[1], h[2], h[3]);
            if constexpr (PR::SPLIT) *reinterpret_cast<uint4 *>(A1l + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        tc_issue<PR>(c.tmem, smem_addr(A1h), smem_addr(A1l), true, smem_addr(B0), smem_addr(B0 + TC_B));
        tc_commit(c.bar);
    }
    c.ok = tc_wait(c, ta.wait_ns, ta.err) && c.ok;
    if (!c.ok) return;
    tc_ld64(c.tmem + ((uint32_t)(warp * 32) << 16), d);
    const float inv1 = 1.f / s1;
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) v[k1] = make_float2(d[2 * k1] * inv1, d[2 * k1 + 1] * inv1);
    tc_fence_before();  // the next stage's MMA overwrites tensor memory after a barrier
}

// Radix-2 step between the two 1024-point halves of 2048-point rows: the CTA
// holds rows as (even, odd) sample warps 2r, 2r+1, and xbuf (4 x 1024 float2,
// reused operand memory) carries each warp's values to its partner.
//   forward (after the halves' FFTs E, O): X[k] = E + W^k O, X[k+1024] = E - W^k O
//     (the even warp keeps k < 1024, the odd warp k >= 1024);
//   inverse (before the halves' IFFTs): E = X[k] + X[k+1024],
//     O = (X[k] - X[k+1024]) W^{-k}, W = exp(-2 pi i / 2048).
template <int DIR>
__device__ __forceinline__ void tc_radix2(float2 (&v)[32], float2 *xbuf, const float2 *__restrict__ tw) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, odd = warp & 1;
    if (DIR < 0 && odd) {
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = cmul_root<-1>(v[e], __ldg(tw + lane + 32 * e));
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 32; ++e) xbuf[warp * 1024 + lane + 32 * e] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const int k = lane + 32 * e;
        const float2 o = xbuf[(warp ^ 1) * 1024 + k];
        if (DIR < 0) {
            v[e] = odd ? make_float2(o.x - v[e].x, o.y - v[e].y) : make_float2(v[e].x + o.x, v[e].y + o.y);
        } else {
            v[e] = odd ? cmul_root<+1>(make_float2(o.x - v[e].x, o.y - v[e].y), __ldg(tw + k))
                       : make_float2(v[e].x + o.x, v[e].y + o.y);
        }
    }
    __syncthreads();
}

// Row pass on tensor cores for 1024- or 2048-sample rows: ROW_ITER (forward
// transform, metrics, constraint and weight update, inverse transform) or
// ROW_TAIL (forward transform, metrics, replay field / phase / weights).  A
// CTA holds 4 rows of 1024 (warp = row), or 2 rows of 2048 as their even and
// odd samples (warps 2r, 2r+1) joined by tc_radix2.
template <int PREC, int ROLE, int NX>
__global__ void __launch_bounds__(128, 1) k_row_tc(const RowArgs a, const TcArgs ta) {
    static_assert(NX == 1024 || NX == 2048, "tensor-core rows are 1024 or 2048 samples");
    extern __shared__ unsigned char smraw[];
    unsigned char *sm = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + TcLayout<TcPrec<PREC>::SPLIT>::BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    volatile int *flag = reinterpret_cast<volatile int *>(tslot + 1);
    double *red = reinterpret_cast<double *>(bar + 2);  // [4 warps][NMET]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int RPC = NX == 1024 ? 4 : 2;     // rows per CTA panel
    constexpr int TWS = NX / 1024;              // twiddle stride
    const int half = NX == 2048 ? (warp & 1) : 0;  // 2048: even / odd samples of a row
    float2 *xbuf = reinterpret_cast<float2 *>(sm + 4 * TC_B);  // operand memory, free between transforms

    for (int i = tid; i < 4 * TC_B / 16; i += 128) reinterpret_cast<uint4 *>(sm)[i] = ta.bmats[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    TcCtx c{sm, bar, flag, *tslot, 0u, true};

    const int ny = a.ny;
    const int ppt = ny / RPC;
    const int J = a.items * ppt;
    for (int p = blockIdx.x; p < J && c.ok; p += gridDim.x) {
        const int item = p / ppt, pan = p - item * ppt;
        const int y = pan * RPC + (NX == 1024 ? warp : warp >> 1);
        const int iy = (y + ny / 2) % ny;
        const float2 *fr = a.field + ((size_t)item * ny + y) * NX;
        float2 v[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = fr[TWS * (lane + 32 * e) + half];
        tc_fft<PREC, -1, TWS>(v, c, a.tw, ta);
        if (!c.ok) break;
        if constexpr (NX == 2048) tc_radix2<-1>(v, xbuf, a.tw);
        const float *Tr = a.T + ((size_t)item * ny + y) * NX;
        float *wr = a.w ? a.w + ((size_t)item * ny + y) * NX : nullptr;
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int x = half * 1024 + lane + 32 * e;
            const float Tv = Tr[x];
            const float2 r = v[e];
            const float m2 = fmaf(r.x, r.x, r.y * r.y);
            const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
            const float I = m2 * a.invN2;
            const float dd = I - Tv * Tv;
            const float am = fmaf(m2 * rs, a.invSqrtN * a.invSqrtN, -Tv);
            const float e2 = m2 * a.invN;
            acc0 = fmaf(dd, dd, acc0);
            acc1 = fmaf(am, am, acc1);
            acc3 += e2;
            if (Tv > 0.f) acc2 += e2;
            float wv = 1.f;
            if (wr) {
                wv = wr[x];
                if (Tv > 0.f && m2 > 0.f) wv = wv * Tv * (a.NN * rs);
                wr[x] = wv;
            }
            if constexpr (ROLE == ROW_ITER) {
                const float gm = Tv * wv;
                v[e] = m2 > 0.f ? make_float2(gm * r.x * rs, gm * r.y * rs) : make_float2(gm, 0.f);
            } else {
                const int ix = (x + NX / 2) % NX;
                const size_t o = ((size_t)item * ny + iy) * NX + ix;
                if (a.phase_out) a.phase_out[o] = m2 > 0.f ? atan2f(r.y, r.x) : 0.f;
                if (a.R_out) a.R_out[o] = make_float2(r.x * a.invSqrtN, r.y * a.invSqrtN);
            }
        }
        if constexpr (ROLE == ROW_ITER) {
            if constexpr (NX == 2048) tc_radix2<+1>(v, xbuf, a.tw);
            tc_fft<PREC, +1, TWS>(v, c, a.tw, ta);
            if (!c.ok) break;
            float2 *fw = a.field + ((size_t)item * ny + y) * NX;
#pragma unroll
            for (int e = 0; e < 32; ++e) fw[TWS * (lane + 32 * e) + half] = v[e];
        }
        if (a.part) {  // per-panel partial sums: warps in fixed order
            float dm[NMET] = {acc0, acc1, acc2, acc3};
#pragma unroll
            for (int off = 16; off; off >>= 1)
#pragma unroll
                for (int q = 0; q < NMET; ++q) dm[q] += __shfl_down_sync(0xffffffffu, dm[q], off);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < NMET; ++q) red[warp * NMET + q] = (double)dm[q];
            __syncthreads();
            if (tid == 0)
                for (int q = 0; q < NMET; ++q)
                    a.part[((size_t)item * ppt + pan) * NMET + q] =
                        red[q] + red[NMET + q] + red[2 * NMET + q] + red[3 * NMET + q];
            __syncthreads();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(c.tmem));
}

// Host side: fill the four DFT-32 operand matrices (forward hi/lo, inverse
// hi/lo) in the K-major canonical layout, 16-bit values, for a precision.
void tc_make_bmats(int prec, uint16_t *out /* 4 * 4096 */);

// Launchers (the grid is persistent: blocks <= 2 per SM by shared memory).
void tc_launch_row(int prec, int role, const RowArgs &a, const TcArgs &ta, int grid, cudaStream_t s);
cudaError_t tc_init(int *blocks_per_sm);

}  // namespace hg
