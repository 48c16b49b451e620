// cnn_conv.cuh -- tensor-core 3x3 convolutions of the warm-start network:
// implicit-GEMM forward (also the data gradient) and the weight gradient,
// tcgen05.mma kind::f16 on BF16 operands with FP32 accumulators in tensor
// memory, operands brought into shared memory by TMA.
//
// Activations are NHWC BF16 [B][H][W][C] (channels fastest, C % 32 == 0).
// A 3x3 weight is [9][Cout][Cin] with tap t = 3*(dy+1) + (dx+1):
//   y[b,h,w,co] = bias[co] + sum_{t,ci} W[t,co,ci] x[b, h+dy, w+dx, ci]
// (zero outside the image).  The data gradient of that layer is the same
// operation on dY with the weights Wt[t][ci][co] = W[8-t][co][ci].
//
// Forward as a GEMM: M = 128 pixels of a tile (one row segment, or whole rows
// when W < 128), N = Cout, K = 9 taps x Cin.  Each K slice is one tap and 32
// channels: the A slice is a 4D TMA box {32 ch, BW px, BH rows, 1} taken at
// the tap's shifted coordinates, so the zero padding is the TMA's
// out-of-bounds fill; the B slice is {32 ci, NB rows of W, 1 tap}.  Both are
// K-major with the 64-byte swizzle (8 rows x 64 B atoms, SBO 512).
//
// Weight gradient as a GEMM: M = 128 rows of (tap, ci) pairs, N = Cout,
// K = pixels.  A and B are MN-major (channels contiguous, 64-byte swizzle,
// 32-channel atoms 4 KB apart = LBO, 8-pixel groups 512 B apart = SBO); a
// 64-pixel K slice is one box per 32-channel atom.  The pixels are split
// over CTAs and each CTA writes its FP32 partial sums; a separate kernel
// adds the partials in a fixed order (deterministic).
//
// Roles (192 threads): warp 0 issues TMA, warp 1 allocates tensor memory and
// issues the MMAs (one thread), warps 2..5 drain the accumulators.  Every
// wait is bounded by wait_ns; on expiry the CTA raises the error bit, stops,
// waits (bounded) for its copies and MMAs in flight and frees its tensor
// memory.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hg_pipe.cuh"

namespace hg {

constexpr int CV_THREADS = 192;
constexpr int CV_ASLOT = 8192;    // 128 rows x 64 B
constexpr int CV_WG_KP = 64;      // pixels per weight-gradient K slice
constexpr int CV_WG_ATOM = 4096;  // 64 pixels x 64 B

struct ConvFwdArgs {
    int B, H, W, Cin, N;      // N: output channels
    int bw, bh;               // A box: pixels per row, rows (bw * bh == 128)
    int nb, nbox;             // B box rows, boxes per slice (nb * nbox == N)
    int stages, tiles;
    int nbuf;                 // accumulator buffers in tensor memory (1 or 2)
    uint32_t tmem_cols;
    const float *bias;        // [N] or null
    int relu;
    const __nv_bfloat16 *mask;  // [B][H][W][N]: output *= (mask > 0), or null
    __nv_bfloat16 *out;       // [B][H][W][N]
    unsigned *err;
    unsigned long long wait_ns;
};

struct ConvWgArgs {
    int B, H, W, Cin, Cout;
    int kw, kh;               // K-slice box: pixels per row, rows (kw * kh == 64)
    int mtiles, splits, chunks, per_split, stages;
    uint32_t tmem_cols;
    float *partial;           // [splits][9*Cin][Cout]
    unsigned *err;
    unsigned long long wait_ns;
};

__device__ __forceinline__ uint64_t cv_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (4ull << 61);  // 64-byte swizzle
}
__device__ __forceinline__ uint32_t cv_idesc(int M, int N, bool mn_major) {
    const uint32_t mj = mn_major ? 1u : 0u;
    return (1u << 4) | (1u << 7) | (1u << 10) | (mj << 15) | (mj << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void cv_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void cv_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void cv_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void cv_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
// 32 FP32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void cv_ld32(uint32_t taddr, float (&d)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = __uint_as_float(r[j]);
}

// Shared-memory layout of both kernels: [A slots][B slots] (1024-aligned),
// then barriers and the control words.
struct CvShared {
    uint64_t *full, *empty, *tfull, *tempty, *done;
    volatile int *abort;
    uint32_t *tmem;
};
__device__ __forceinline__ CvShared cv_carve(unsigned char *ctl, int stages) {
    CvShared s;
    s.full = reinterpret_cast<uint64_t *>(ctl);
    s.empty = s.full + stages;
    s.tfull = s.empty + stages;
    s.tempty = s.tfull + 2;
    s.done = s.tempty + 2;
    s.abort = reinterpret_cast<volatile int *>(s.done + 1);
    s.tmem = reinterpret_cast<uint32_t *>(s.done + 2);
    return s;
}
// After an abort: wait (bounded) for the last stages' copies, which may still
// be landing in shared memory, before the CTA exits.
__device__ __forceinline__ void cv_drain(uint64_t *full, int S, long issued, unsigned long long wait_ns) {
    const long first = issued > S ? issued - S : 0;
    for (long q = first; q < issued; ++q) mbar_wait(full + (int)(q % S), (uint32_t)((q / S) & 1), wait_ns, nullptr);
}
constexpr int CV_CTL_BYTES = 8 * (2 * 12 + 2 + 2 + 1) + 16;  // up to 12 stages

#ifdef HG_CONV_KERNELS  // the kernels are compiled in cnn_conv.cu only

// Forward / data-gradient convolution, persistent over 128-pixel tiles.
__global__ void __launch_bounds__(CV_THREADS, 1)
    k_conv_fwd(const ConvFwdArgs a, const __grid_constant__ CUtensorMap amap,
               const __grid_constant__ CUtensorMap bmap) {
    extern __shared__ unsigned char cv_smraw[];
    unsigned char *base = cv_smraw + ((1024 - (smem_addr(cv_smraw) & 1023)) & 1023);
    const int S = a.stages;
    const uint32_t bslot = (uint32_t)a.N * 64;
    unsigned char *sA = base;
    unsigned char *sB = base + (size_t)S * CV_ASLOT;
    CvShared sh = cv_carve(sB + (size_t)S * bslot, S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(sh.full + i, 1);
            mbar_init(sh.empty + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(sh.tfull + i, 1);
            mbar_init(sh.tempty + i, 4);
        }
        mbar_init(sh.done, 1);
        *sh.abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(sh.tmem)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    cv_fence_before();
    __syncthreads();
    cv_fence_after();
    const uint32_t tmem = *sh.tmem;

    const int cch = a.Cin / 32;
    const int nk = 9 * cch;
    const int rows_per_tile = a.bh;
    const int xtiles = a.W / a.bw;  // tiles per row band
    auto tile_origin = [&](int tile, int &b, int &y0, int &x0) {
        const int bands = a.H / rows_per_tile;
        const int xt = tile % xtiles;
        const int r = tile / xtiles;
        y0 = (r % bands) * rows_per_tile;
        b = r / bands;
        x0 = xt * a.bw;
    };
    auto fail = [&]() {
        atomicOr(a.err, ERR_TIMEOUT_BIT);
        *sh.abort = 1;
    };

    long issued_stages = 0;  // producer: TMA stages issued (drained on abort)
    if (warp == 0) {
        if (lane == 0) {
            long &it = issued_stages;
            bool ok = true;
            for (int tile = blockIdx.x; tile < a.tiles && ok; tile += gridDim.x) {
                int b, y0, x0;
                tile_origin(tile, b, y0, x0);
                for (int ks = 0; ks < nk; ++ks, ++it) {
                    const int slot = (int)(it % S);
                    const long round = it / S;
                    if (round > 0 && !mbar_wait(sh.empty + slot, (uint32_t)((round - 1) & 1), a.wait_ns, sh.abort)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const int tap = ks / cch, cc = ks - tap * cch;
                    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                    mbar_expect_tx(sh.full + slot, CV_ASLOT + bslot);
                    tma_load_4d(sA + (size_t)slot * CV_ASLOT, &amap, cc * 32, x0 + dx, y0 + dy, b,
                                sh.full + slot);
                    for (int q = 0; q < a.nbox; ++q)
                        tma_load_3d(sB + (size_t)slot * bslot + (size_t)q * a.nb * 64, &bmap, cc * 32, q * a.nb,
                                    tap, sh.full + slot);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            long it = 0;
            int local = 0;
            bool issued = false, ok = true;
            const int nparts = a.N > 256 ? 2 : 1;
            const int npart = a.N / nparts;
            const uint32_t idesc = cv_idesc(128, npart, false);
            for (int tile = blockIdx.x; tile < a.tiles && ok; tile += gridDim.x, ++local) {
                const int buf = a.nbuf == 2 ? (local & 1) : 0;
                const int use = a.nbuf == 2 ? (local >> 1) : local;
                if (use > 0 && !mbar_wait(sh.tempty + buf, (uint32_t)((use - 1) & 1), a.wait_ns, sh.abort)) {
                    fail();
                    break;
                }
                cv_fence_after();
                const uint32_t dcol = tmem + (uint32_t)(buf * a.N);
                for (int ks = 0; ks < nk; ++ks, ++it) {
                    const int slot = (int)(it % S);
                    if (!mbar_wait(sh.full + slot, (uint32_t)((it / S) & 1), a.wait_ns, sh.abort)) {
                        fail();
                        ok = false;
                        break;
                    }
                    cv_fence_after();
                    const uint32_t aa = smem_addr(sA + (size_t)slot * CV_ASLOT);
                    const uint32_t bb = smem_addr(sB + (size_t)slot * bslot);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t ad = cv_desc(aa + kk * 32, 16, 512);
                        for (int p = 0; p < nparts; ++p)
                            cv_mma(dcol + p * npart, ad, cv_desc(bb + (uint32_t)(p * npart * 64) + kk * 32, 16, 512),
                                   idesc, (ks | kk) ? 1u : 0u);
                    }
                    issued = true;
                    cv_commit(sh.empty + slot);  // the slot is free once these MMAs have read it
                }
                if (ok) cv_commit(sh.tfull + buf);
            }
            if (issued) {  // no MMA may still run when the tensor memory is released
                cv_commit(sh.done);
                mbar_wait(sh.done, 0, a.wait_ns, nullptr);
            }
        }
    } else {
        // epilogue: warp w reads tensor-memory lanes 32*(w%4) .. +31 = tile rows
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;
        int local = 0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, ++local) {
            const int buf = a.nbuf == 2 ? (local & 1) : 0;
            const int use = a.nbuf == 2 ? (local >> 1) : local;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(sh.tfull + buf, (uint32_t)(use & 1), a.wait_ns, sh.abort);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) fail();
                break;
            }
            cv_fence_after();
            int b, y0, x0;
            tile_origin(tile, b, y0, x0);
            const int x = x0 + m % a.bw, y = y0 + m / a.bw;
            const size_t pix = ((size_t)b * a.H + y) * a.W + x;
            __nv_bfloat16 *orow = a.out + pix * a.N;
            const __nv_bfloat16 *mrow = a.mask ? a.mask + pix * a.N : nullptr;
            const uint32_t lrow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * a.N);
            for (int c0 = 0; c0 < a.N; c0 += 32) {
                float v[32];
                cv_ld32(lrow + c0, v);
                if (a.bias) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] += __ldg(a.bias + c0 + j);
                }
                if (a.relu) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
                }
                if (mrow) {
                    uint4 mq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) mq[q] = __ldg(reinterpret_cast<const uint4 *>(mrow + c0) + q);
                    const __nv_bfloat16 *mv = reinterpret_cast<const __nv_bfloat16 *>(mq);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (!(__bfloat162float(mv[j]) > 0.f)) v[j] = 0.f;
                }
                uint4 oq[4];
                __nv_bfloat162 *ov = reinterpret_cast<__nv_bfloat162 *>(oq);
#pragma unroll
                for (int j = 0; j < 16; ++j) ov[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
#pragma unroll
                for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(orow + c0)[q] = oq[q];
            }
            cv_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(sh.tempty + buf);
        }
    }
    cv_fence_before();
    __syncthreads();
    if (*sh.abort && tid == 0) cv_drain(sh.full, S, issued_stages, a.wait_ns);
    if (warp == 1) {
        cv_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    }
}

// Weight gradient, one (M tile, pixel split) per CTA: FP32 partial sums
// partial[split][t*Cin + ci][co] = sum over the split's pixels of
// x[p + shift_t][ci] * dy[p][co].
__global__ void __launch_bounds__(CV_THREADS, 1)
    k_conv_wgrad(const ConvWgArgs a, const __grid_constant__ CUtensorMap xmap,
                 const __grid_constant__ CUtensorMap gmap) {
    extern __shared__ unsigned char cv_smraw[];
    unsigned char *base = cv_smraw + ((1024 - (smem_addr(cv_smraw) & 1023)) & 1023);
    const int S = a.stages;
    const uint32_t aslot = 4 * CV_WG_ATOM;
    const uint32_t bslot = (uint32_t)(a.Cout / 32) * CV_WG_ATOM;
    unsigned char *sA = base;
    unsigned char *sB = base + (size_t)S * aslot;
    CvShared sh = cv_carve(sB + (size_t)S * bslot, S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x % a.mtiles, split = blockIdx.x / a.mtiles;
    const int q0 = split * a.per_split;
    const int q1 = min(a.chunks, q0 + a.per_split);
    const int cch = a.Cin / 32;
    const int rows = 9 * a.Cin;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(sh.full + i, 1);
            mbar_init(sh.empty + i, 1);
        }
        mbar_init(sh.tfull, 1);
        mbar_init(sh.done, 1);
        *sh.abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(sh.tmem)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    cv_fence_before();
    __syncthreads();
    cv_fence_after();
    const uint32_t tmem = *sh.tmem;
    auto fail = [&]() {
        atomicOr(a.err, ERR_TIMEOUT_BIT);
        *sh.abort = 1;
    };
    // pixel chunk q -> (b, y0, x0) of a kw x kh box
    const int xch = a.W / a.kw, bands = a.H / a.kh;
    auto chunk_origin = [&](int q, int &b, int &y0, int &x0) {
        const int xc = q % xch;
        const int r = q / xch;
        y0 = (r % bands) * a.kh;
        b = r / bands;
        x0 = xc * a.kw;
    };
    int natoms = 0;  // atoms of this M tile that hold real (tap, ci) rows
    for (int j = 0; j < 4; ++j)
        if ((mt * 4 + j) * 32 < rows) ++natoms;

    long issued_stages = 0;
    if (warp == 0) {
        if (lane == 0) {
            long &it = issued_stages;
            for (int q = q0; q < q1; ++q, ++it) {
                const int slot = (int)(it % S);
                const long round = it / S;
                if (round > 0 && !mbar_wait(sh.empty + slot, (uint32_t)((round - 1) & 1), a.wait_ns, sh.abort)) {
                    fail();
                    break;
                }
                int b, y0, x0;
                chunk_origin(q, b, y0, x0);
                mbar_expect_tx(sh.full + slot, (uint32_t)natoms * CV_WG_ATOM + bslot);
                for (int j = 0; j < natoms; ++j) {
                    const int ga = mt * 4 + j;
                    const int tap = ga / cch, c0 = (ga - tap * cch) * 32;
                    tma_load_4d(sA + (size_t)slot * aslot + (size_t)j * CV_WG_ATOM, &xmap, c0, x0 + tap % 3 - 1,
                                y0 + tap / 3 - 1, b, sh.full + slot);
                }
                for (int j = 0; j < a.Cout / 32; ++j)
                    tma_load_4d(sB + (size_t)slot * bslot + (size_t)j * CV_WG_ATOM, &gmap, j * 32, x0, y0, b,
                                sh.full + slot);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = cv_idesc(128, a.Cout, true);
            bool issued = false, ok = true;
            long it = 0;
            for (int q = q0; q < q1; ++q, ++it) {
                const int slot = (int)(it % S);
                if (!mbar_wait(sh.full + slot, (uint32_t)((it / S) & 1), a.wait_ns, sh.abort)) {
                    fail();
                    ok = false;
                    break;
                }
                cv_fence_after();
                const uint32_t aa = smem_addr(sA + (size_t)slot * aslot);
                const uint32_t bb = smem_addr(sB + (size_t)slot * bslot);
#pragma unroll
                for (int k = 0; k < CV_WG_KP / 16; ++k)
                    cv_mma(tmem, cv_desc(aa + k * 1024, CV_WG_ATOM, 512), cv_desc(bb + k * 1024, CV_WG_ATOM, 512),
                           idesc, (q > q0 || k) ? 1u : 0u);
                issued = true;
                cv_commit(sh.empty + slot);
            }
            if (ok && issued) cv_commit(sh.tfull);
            if (issued) {
                cv_commit(sh.done);
                mbar_wait(sh.done, 0, a.wait_ns, nullptr);
            }
        }
    } else if (q1 > q0) {
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;
        bool ok = true;
        if (lane == 0) ok = mbar_wait(sh.tfull, 0, a.wait_ns, sh.abort);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
            if (lane == 0) fail();
        } else {
            cv_fence_after();
            const int grow = mt * 128 + r;
            float *prow = a.partial + ((size_t)split * rows + grow) * a.Cout;
            const uint32_t lrow = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int c0 = 0; c0 < a.Cout; c0 += 32) {
                float v[32];
                cv_ld32(lrow + c0, v);
                if (grow < rows) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        reinterpret_cast<float4 *>(prow + c0)[q] =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
    }
    cv_fence_before();
    __syncthreads();
    if (*sh.abort && tid == 0) cv_drain(sh.full, S, issued_stages, a.wait_ns);
    if (warp == 1) {
        cv_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    }
}

#endif  // HG_CONV_KERNELS

}  // namespace hg

namespace hg {
// Host launchers (cnn_conv.cu).  All pointers device; `err` a device word
// that receives the timeout bit.  Return cudaErrorInvalidValue for shapes
// the kernels do not tile.
cudaError_t conv_fwd_launch(const __nv_bfloat16 *x, int B, int H, int W, int Cin, const __nv_bfloat16 *w, int N,
                            const float *bias, int relu, const __nv_bfloat16 *mask, __nv_bfloat16 *out,
                            unsigned *err, unsigned long long wait_ns, cudaStream_t s);
bool conv_fwd_shape_ok(int B, int H, int W, int Cin, int N);
size_t conv_wgrad_workspace(int B, int H, int W, int Cin, int Cout);
bool conv_wgrad_shape_ok(int B, int H, int W, int Cin, int Cout);
// Partial sums into `ws`, then the fixed-order reduction into dw [9][Cout][Cin]
// (and db [Cout] from dy when db is not null, through the tail of `ws`).
cudaError_t conv_wgrad_launch(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int H, int W, int Cin,
                              int Cout, float *dw, float *db, void *ws, size_t ws_bytes, unsigned *err,
                              unsigned long long wait_ns, cudaStream_t s);
// Per-channel sums of a [npx][C] BF16 tensor into out[C] (fixed order), using
// `part` (chan_sum_blocks(npx) * C floats) for the block partials.
int chan_sum_blocks(long npx);
cudaError_t chan_sum_launch(const __nv_bfloat16 *x, long npx, int C, float *part, float *out, cudaStream_t s);
int conv_launches_per_wgrad(bool with_bias);
}  // namespace hg
