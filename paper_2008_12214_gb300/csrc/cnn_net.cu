// cnn_net.cu -- the warm-start network of include/hologen_cnn.h: its
// parameters and activations in device memory, the CUDA-core kernels around
// the tensor-core convolutions (first layer with one input channel,
// pooling, upsample + concatenation, the head with the loss, per-image
// statistics, the fused Adam update), and the forward / backward sequences.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cnn_conv.cuh"
#include "hologen_cnn.h"

namespace hg {
namespace {

// ----------------------------------------------------------- parameter table

constexpr int kConvs = 14;
constexpr int kCin[kConvs] = {1, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32};
constexpr int kCout[kConvs] = {32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32};

struct LayerDesc {
    int cin, cout;
    long w_off, b_off;  // in the FP32 parameter vector
    long bf_off;        // in the BF16 weight copies (tensor-core layers; -1 for the first)
};
struct ParamTable {
    LayerDesc l[kConvs];
    long head_w, head_b, n, nbf;
};
constexpr ParamTable make_table() {
    ParamTable t{};
    long off = 0, bf = 0;
    for (int i = 0; i < kConvs; ++i) {
        t.l[i].cin = kCin[i];
        t.l[i].cout = kCout[i];
        t.l[i].w_off = off;
        off += 9L * kCin[i] * kCout[i];
        t.l[i].b_off = off;
        off += kCout[i];
        if (i == 0) {
            t.l[i].bf_off = -1;
        } else {
            t.l[i].bf_off = bf;
            bf += 9L * kCin[i] * kCout[i];
        }
    }
    t.head_w = off;
    off += 64;
    t.head_b = off;
    off += 2;
    t.n = off;
    t.nbf = bf;
    return t;
}
constexpr ParamTable kTab = make_table();
static_assert(kTab.n == HG_CNN_NPARAMS, "parameter count of the header");
__constant__ ParamTable c_tab = make_table();

enum : unsigned { CNN_ERR_BAD = 1u, CNN_ERR_ZERO = 2u };
constexpr int kStatBlocks = 64;
constexpr int kFirstPartN = 9 * 32 + 32;  // first-layer weight and bias partials
constexpr int kHeadPartN = 68;           // 32 + 32 + 2 head gradients, loss, pad

int ew_blocks(long n, int nsm) {
    long b = (n + 255) / 256;
    const long cap = (long)nsm * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// ------------------------------------------------------------------ kernels

// Per image: max T and sum T^2 partials; flags negative / NaN / infinite values.
__global__ void k_img_stats_part(const float *__restrict__ T, long npx, float *pmax, double *psum, unsigned *err) {
    __shared__ float smax[8];
    __shared__ double ssum[8];
    const int b = blockIdx.y;
    const float *tb = T + (size_t)b * npx;
    float mx = 0.f, sf = 0.f;
    bool bad = false;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < npx; i += (long)kStatBlocks * blockDim.x) {
        const float v = tb[i];
        if (!(v >= 0.f) || isinf(v)) bad = true;
        mx = fmaxf(mx, v);
        sf = fmaf(v, v, sf);
    }
    if (bad) atomicOr(err, CNN_ERR_BAD);
    double s = sf;
    for (int o = 16; o; o >>= 1) {
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = mx;
        ssum[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            smax[0] = fmaxf(smax[0], smax[w]);
            ssum[0] += ssum[w];
        }
        pmax[b * kStatBlocks + blockIdx.x] = smax[0];
        psum[b * kStatBlocks + blockIdx.x] = ssum[0];
    }
}

__global__ void k_img_stats_final(const float *pmax, const double *psum, int B, float *inv_max, float *inv_sumsq,
                                  unsigned *err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float mx = 0.f;
    double s = 0;
    for (int i = 0; i < kStatBlocks; ++i) {
        mx = fmaxf(mx, pmax[b * kStatBlocks + i]);
        s += psum[b * kStatBlocks + i];
    }
    if (mx > 0.f && s > 0) {
        inv_max[b] = 1.f / mx;
        inv_sumsq[b] = (float)(1.0 / s);
    } else {
        inv_max[b] = 0.f;
        inv_sumsq[b] = 0.f;
        atomicOr(err, CNN_ERR_ZERO);
    }
}

// x at (b, y, x) of the net input (T / max T), zero outside the image.
__device__ __forceinline__ float net_in(const float *T, const float *inv_max, int b, int H, int W, int y, int x) {
    if (y < 0 || y >= H || x < 0 || x >= W) return 0.f;
    return T[((size_t)b * H + y) * W + x] * inv_max[b];
}

// First convolution (1 -> 32 channels) + ReLU, one pixel per thread.
__global__ void __launch_bounds__(256)
    k_first_fwd(const float *__restrict__ T, const float *__restrict__ inv_max, const float *__restrict__ theta,
                int B, int H, int W, __nv_bfloat16 *__restrict__ out) {
    __shared__ float sw[9 * 32 + 32];
    for (int i = threadIdx.x; i < 9 * 32 + 32; i += blockDim.x) sw[i] = theta[c_tab.l[0].w_off + i];
    __syncthreads();
    const long npx = (long)B * H * W;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < npx; p += (long)gridDim.x * blockDim.x) {
        const int b = (int)(p / ((long)H * W));
        const int r = (int)(p - (long)b * H * W);
        const int y = r / W, x = r - y * W;
        float xin[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) xin[t] = net_in(T, inv_max, b, H, W, y + t / 3 - 1, x + t % 3 - 1);
        uint4 oq[4];
        __nv_bfloat162 *ov = reinterpret_cast<__nv_bfloat162 *>(oq);
#pragma unroll
        for (int co = 0; co < 32; co += 2) {
            float a0 = sw[288 + co], a1 = sw[288 + co + 1];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                a0 = fmaf(sw[t * 32 + co], xin[t], a0);
                a1 = fmaf(sw[t * 32 + co + 1], xin[t], a1);
            }
            ov[co / 2] = __floats2bfloat162_rn(fmaxf(a0, 0.f), fmaxf(a1, 0.f));
        }
        uint4 *o = reinterpret_cast<uint4 *>(out + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = oq[q];
    }
}

// First convolution's weight and bias gradient partials: part[block][t*32+co]
// and part[block][288+co]; lane = output channel, warp = pixel lane.
__global__ void __launch_bounds__(256)
    k_first_wgrad_part(const float *__restrict__ T, const float *__restrict__ inv_max,
                       const __nv_bfloat16 *__restrict__ dpre, int B, int H, int W, float *__restrict__ part) {
    __shared__ float red[8][kFirstPartN];
    const int co = threadIdx.x & 31, pl = threadIdx.x >> 5;
    float acc[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) acc[t] = 0.f;
    const long npx = (long)B * H * W;
    for (long p = (long)blockIdx.x * 8 + pl; p < npx; p += (long)gridDim.x * 8) {
        const int b = (int)(p / ((long)H * W));
        const int r = (int)(p - (long)b * H * W);
        const int y = r / W, x = r - y * W;
        const float d = __bfloat162float(dpre[p * 32 + co]);
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] = fmaf(d, net_in(T, inv_max, b, H, W, y + t / 3 - 1, x + t % 3 - 1), acc[t]);
        acc[9] += d;
    }
#pragma unroll
    for (int t = 0; t < 10; ++t) red[pl][t * 32 + co] = acc[t];
    __syncthreads();
    for (int i = threadIdx.x; i < kFirstPartN; i += blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < 8; ++q) s += red[q][i];
        part[(size_t)blockIdx.x * kFirstPartN + i] = s;
    }
}

// Fixed-order sum of `blocks` partial rows of length n into out[n].
__global__ void k_rows_sum(const float *__restrict__ part, int blocks, int n, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * n + i];
    out[i] = (float)s;
}

// 2x2 average pooling, [B][H][W][C] -> [B][H/2][W/2][C]; 8 channels per thread.
__global__ void k_pool(const __nv_bfloat16 *__restrict__ in, int B, int H, int W, int C,
                       __nv_bfloat16 *__restrict__ out) {
    const int H2 = H / 2, W2 = W / 2, C8 = C / 8;
    const long n = (long)B * H2 * W2 * C8;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int c8 = (int)(i % C8);
        const long p = i / C8;
        const int x = (int)(p % W2);
        const long q = p / W2;
        const int y = (int)(q % H2), b = (int)(q / H2);
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const size_t src = (((size_t)b * H + 2 * y + (d >> 1)) * W + 2 * x + (d & 1)) * C + c8 * 8;
            const uint4 v = *reinterpret_cast<const uint4 *>(in + src);
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += __bfloat162float(h[j]);
        }
        uint4 o;
        __nv_bfloat162 *ov = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
        for (int j = 0; j < 4; ++j) ov[j] = __floats2bfloat162_rn(0.25f * s[2 * j], 0.25f * s[2 * j + 1]);
        *reinterpret_cast<uint4 *>(out + p * C + c8 * 8) = o;
    }
}

// out[B][H][W][Cu+Cs] = [up2(coarse [B][H/2][W/2][Cu]), skip [B][H][W][Cs]].
__global__ void k_upcat(const __nv_bfloat16 *__restrict__ coarse, const __nv_bfloat16 *__restrict__ skip, int B,
                        int H, int W, int Cu, int Cs, __nv_bfloat16 *__restrict__ out) {
    const int C = Cu + Cs, C8 = C / 8;
    const long n = (long)B * H * W * C8;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8) * 8;
        const long p = i / C8;
        const int x = (int)(p % W);
        const long q = p / W;
        const int y = (int)(q % H), b = (int)(q / H);
        uint4 v;
        if (c < Cu)
            v = *reinterpret_cast<const uint4 *>(coarse + (((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * Cu + c);
        else
            v = *reinterpret_cast<const uint4 *>(skip + (size_t)p * Cs + (c - Cu));
        *reinterpret_cast<uint4 *>(out + (size_t)p * C + c) = v;
    }
}

// Backward of k_upcat: dcoarse = (sum over each 2x2 block of dcat[:, :Cu]) * (cmask > 0)
// and dskip = dcat[:, Cu:].
__global__ void k_upcat_bwd(const __nv_bfloat16 *__restrict__ dcat, const __nv_bfloat16 *__restrict__ cmask, int B,
                            int H, int W, int Cu, int Cs, __nv_bfloat16 *__restrict__ dcoarse,
                            __nv_bfloat16 *__restrict__ dskip) {
    const int C = Cu + Cs, H2 = H / 2, W2 = W / 2;
    const long n1 = (long)B * H2 * W2 * (Cu / 8), n2 = (long)B * H * W * (Cs / 8);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n1 + n2; i += (long)gridDim.x * blockDim.x) {
        if (i < n1) {
            const int c = (int)(i % (Cu / 8)) * 8;
            const long p = i / (Cu / 8);
            const int x = (int)(p % W2);
            const long q = p / W2;
            const int y = (int)(q % H2), b = (int)(q / H2);
            float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const size_t src = (((size_t)b * H + 2 * y + (d >> 1)) * W + 2 * x + (d & 1)) * C + c;
                const uint4 v = *reinterpret_cast<const uint4 *>(dcat + src);
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
                for (int j = 0; j < 8; ++j) s[j] += __bfloat162float(h[j]);
            }
            const uint4 mv = *reinterpret_cast<const uint4 *>(cmask + (size_t)p * Cu + c);
            const __nv_bfloat16 *m = reinterpret_cast<const __nv_bfloat16 *>(&mv);
            uint4 o;
            __nv_bfloat162 *ov = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                ov[j] = __floats2bfloat162_rn(__bfloat162float(m[2 * j]) > 0.f ? s[2 * j] : 0.f,
                                              __bfloat162float(m[2 * j + 1]) > 0.f ? s[2 * j + 1] : 0.f);
            *reinterpret_cast<uint4 *>(dcoarse + (size_t)p * Cu + c) = o;
        } else {
            const long k = i - n1;
            const int c = (int)(k % (Cs / 8)) * 8;
            const long p = k / (Cs / 8);
            *reinterpret_cast<uint4 *>(dskip + (size_t)p * Cs + c) =
                *reinterpret_cast<const uint4 *>(dcat + (size_t)p * C + Cu + c);
        }
    }
}

// dpre = (dpool[p/2] / 4 + dskip[p]) * (act > 0), all [.][.][.][C].
__global__ void k_pool_bwd_add(const __nv_bfloat16 *__restrict__ dpool, const __nv_bfloat16 *__restrict__ dskip,
                               const __nv_bfloat16 *__restrict__ act, int B, int H, int W, int C,
                               __nv_bfloat16 *__restrict__ dpre) {
    const int C8 = C / 8;
    const long n = (long)B * H * W * C8;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8) * 8;
        const long p = i / C8;
        const int x = (int)(p % W);
        const long q = p / W;
        const int y = (int)(q % H), b = (int)(q / H);
        const uint4 pv =
            *reinterpret_cast<const uint4 *>(dpool + (((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c);
        const uint4 sv = *reinterpret_cast<const uint4 *>(dskip + (size_t)p * C + c);
        const uint4 av = *reinterpret_cast<const uint4 *>(act + (size_t)p * C + c);
        const __nv_bfloat16 *ph = reinterpret_cast<const __nv_bfloat16 *>(&pv);
        const __nv_bfloat16 *sh = reinterpret_cast<const __nv_bfloat16 *>(&sv);
        const __nv_bfloat16 *ah = reinterpret_cast<const __nv_bfloat16 *>(&av);
        uint4 o;
        __nv_bfloat162 *ov = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v0 = 0.25f * __bfloat162float(ph[2 * j]) + __bfloat162float(sh[2 * j]);
            float v1 = 0.25f * __bfloat162float(ph[2 * j + 1]) + __bfloat162float(sh[2 * j + 1]);
            if (!(__bfloat162float(ah[2 * j]) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(ah[2 * j + 1]) > 0.f)) v1 = 0.f;
            ov[j] = __floats2bfloat162_rn(v0, v1);
        }
        *reinterpret_cast<uint4 *>(dpre + (size_t)p * C + c) = o;
    }
}

// Head: (c, s) = Wh h + bh per pixel.  With a label phi: the loss
// wT |(c, s) - e^{i (phi - phi_b)}|^2 / (2 B), wT = T^2 / sum T^2 (phi_b:
// the optional base phase [H][W], else 0), its gradient through the head
// (dpre of the last convolution, masked by h > 0) and block partials
// {sum dc h[32], sum ds h[32], sum dc, sum ds, loss}.  phase_out gets
// atan2(s, c) + phi_b.
constexpr int HEAD_THREADS = 256;
__global__ void __launch_bounds__(HEAD_THREADS)
    k_head(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ theta, const float *__restrict__ T,
           const float *__restrict__ phi, const float *__restrict__ inv_sumsq, int B, long npx_img, float invB,
           __nv_bfloat16 *__restrict__ dpre, float2 *__restrict__ cs_out, float *__restrict__ phase_out,
           float *__restrict__ part, const float *__restrict__ base) {
    __shared__ float sw[66];
    __shared__ float red[HEAD_THREADS / 32][kHeadPartN];
    if (threadIdx.x < 66) sw[threadIdx.x] = theta[c_tab.head_w + threadIdx.x];
    __syncthreads();
    const bool train = phi != nullptr;
    float g[kHeadPartN];
#pragma unroll
    for (int j = 0; j < kHeadPartN; ++j) g[j] = 0.f;
    const long npx = npx_img * B;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < npx; p += (long)gridDim.x * blockDim.x) {
        float hv[32];
        const uint4 *hq = reinterpret_cast<const uint4 *>(h + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = hq[q];
            const __nv_bfloat16 *hh = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) hv[q * 8 + j] = __bfloat162float(hh[j]);
        }
        float c = sw[64], s = sw[65];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            c = fmaf(sw[j], hv[j], c);
            s = fmaf(sw[32 + j], hv[j], s);
        }
        if (cs_out) cs_out[p] = make_float2(c, s);
        const float pb = base ? base[p % npx_img] : 0.f;
        if (phase_out) phase_out[p] = atan2f(s, c) + pb;
        if (!train) continue;
        const int b = (int)(p / npx_img);
        const float t = T[p];
        const float wT = t * t * inv_sumsq[b];
        float sp, cp;
        sincosf(phi[p] - pb, &sp, &cp);
        const float ec = c - cp, es = s - sp;
        g[66] += 0.5f * wT * (ec * ec + es * es) * invB;
        const float dc = wT * ec * invB, ds = wT * es * invB;
        uint4 oq[4];
        __nv_bfloat162 *ov = reinterpret_cast<__nv_bfloat162 *>(oq);
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const float d0 = hv[j] > 0.f ? dc * sw[j] + ds * sw[32 + j] : 0.f;
            const float d1 = hv[j + 1] > 0.f ? dc * sw[j + 1] + ds * sw[32 + j + 1] : 0.f;
            ov[j / 2] = __floats2bfloat162_rn(d0, d1);
        }
        uint4 *o = reinterpret_cast<uint4 *>(dpre + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = oq[q];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            g[j] = fmaf(dc, hv[j], g[j]);
            g[32 + j] = fmaf(ds, hv[j], g[32 + j]);
        }
        g[64] += dc;
        g[65] += ds;
    }
    if (!train) return;
#pragma unroll
    for (int j = 0; j < kHeadPartN; ++j) {
        float v = g[j];
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][j] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kHeadPartN; j += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < HEAD_THREADS / 32; ++w) s += red[w][j];
        part[(size_t)blockIdx.x * kHeadPartN + j] = s;
    }
}

// Fixed-order sum of the head partials: gradients of the head parameters
// into grad[head_w .. head_b + 1], the loss into *loss (double).
__global__ void k_head_final(const float *__restrict__ part, int blocks, float *__restrict__ grad, double *loss) {
    const int j = threadIdx.x;
    if (j >= 67) return;
    double s = 0;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * kHeadPartN + j];
    if (j < 66) grad[c_tab.head_w + j] = (float)s;
    else if (loss) *loss = s;
}

// Position of parameter i: conv layer (or -1 for the head), and whether it is a weight.
__device__ __forceinline__ int layer_of(long i, bool *is_w) {
    for (int l = 0; l < kConvs; ++l) {
        if (i < c_tab.l[l].b_off) {
            *is_w = true;
            return l;
        }
        if (i < c_tab.l[l].b_off + c_tab.l[l].cout) {
            *is_w = false;
            return l;
        }
    }
    *is_w = i < c_tab.head_b;
    return -1;
}

// Fused Adam step over the whole parameter vector (update = 0: only refresh
// the BF16 copies), writing the BF16 forward weights [9][Cout][Cin] and the
// rotated transposed copies [9][Cin][Cout] of the tensor-core layers.
__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m,
                       float *__restrict__ v, long n, int update, float lr, float b1, float b2, float eps, float bc1,
                       float bc2, __nv_bfloat16 *__restrict__ wf, __nv_bfloat16 *__restrict__ wt) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float th = theta[i];
        if (update) {
            const float gi = grad[i];
            const float mi = b1 * m[i] + (1.f - b1) * gi;
            const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            th -= lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
            theta[i] = th;
        }
        bool is_w;
        const int l = layer_of(i, &is_w);
        if (l > 0 && is_w) {
            const LayerDesc d = c_tab.l[l];
            const long k = i - d.w_off;
            const int ci = (int)(k % d.cin);
            const long r = k / d.cin;
            const int co = (int)(r % d.cout), t = (int)(r / d.cout);
            const __nv_bfloat16 hb = __float2bfloat16_rn(th);
            wf[d.bf_off + k] = hb;
            wt[d.bf_off + ((long)(8 - t) * d.cin + ci) * d.cout + co] = hb;
        }
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// He-normal initialisation (Box-Muller on SplitMix64 of (seed, i)); zero biases.
__global__ void k_init_params(float *theta, long n, uint64_t seed) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        bool is_w;
        const int l = layer_of(i, &is_w);
        float val = 0.f;
        if (is_w) {
            const float sd = l >= 0 ? sqrtf(2.f / (9.f * c_tab.l[l].cin)) : sqrtf(1.f / 32.f);
            const uint64_t z = mix64(seed ^ mix64((uint64_t)i));
            const float u1 = ((float)(z >> 40) + 1.f) * (1.f / 16777217.f);
            const float u2 = (float)((z >> 16) & 0xFFFFFF) * (1.f / 16777216.f);
            val = sd * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
        }
        theta[i] = val;
    }
}

}  // namespace
}  // namespace hg

using namespace hg;

// --------------------------------------------------------------------- net

struct hg_cnn_s {
    int dev = 0, H = 0, W = 0, maxB = 0, nsm = 0;
    cudaStream_t s = nullptr;
    unsigned long long wait_ns = 2000000000ull;
    long step = 0;
    int launches = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wf = nullptr, *wt = nullptr;
    // forward activations (post-ReLU), per level
    __nv_bfloat16 *A[4][2] = {}, *P[3] = {}, *C[3] = {}, *D[3][2] = {};
    // backward scratch per level
    __nv_bfloat16 *G[4][3] = {}, *DS[3] = {};
    float *inv_max = nullptr, *inv_sumsq = nullptr, *pmax = nullptr;
    double *psum = nullptr;
    float *first_part = nullptr, *head_part = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    unsigned *err = nullptr;
    double *loss = nullptr;
    float *base = nullptr;       // optional base phase [H][W] (see hg_cnn_set_base_phase)
    float *base_buf = nullptr;   // its storage, allocated at the first set
    std::vector<void *> owned;
};

namespace {

constexpr int kWidth[4] = {32, 64, 128, 256};
constexpr int kCatC[3] = {96, 192, 384};
constexpr int kGcC[4] = {96, 192, 384, 128};

hg_status st_of(cudaError_t e) {
    if (e == cudaSuccess) return HG_OK;
    if (e == cudaErrorMemoryAllocation) return HG_ERR_OOM;
    if (e == cudaErrorInvalidValue) return HG_ERR_UNSUPPORTED_SIZE;
    return HG_ERR_CUDA;
}

#define CN_CK(x)                                  \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return st_of(e_);  \
    } while (0)

bool net_shape_ok(int H, int W) {
    if (H < 8 || W < 8 || H % 8 || W % 8) return false;
    for (int l = 0; l < 4; ++l) {
        const int h = H >> l, w = W >> l;
        if (!conv_fwd_shape_ok(1, h, w, 32, 32) || !conv_wgrad_shape_ok(1, h, w, 32, 32)) return false;
    }
    return true;
}

template <class T>
cudaError_t alloc(hg_cnn n, T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) n->owned.push_back(*p);
    return e;
}

long lvl_px(hg_cnn n, int B, int l) { return (long)B * (n->H >> l) * (n->W >> l); }

cudaError_t conv(hg_cnn n, int layer, const __nv_bfloat16 *x, int B, int l, const __nv_bfloat16 *mask,
                 __nv_bfloat16 *out) {
    const LayerDesc &d = kTab.l[layer];
    n->launches++;
    return conv_fwd_launch(x, B, n->H >> l, n->W >> l, d.cin, n->wf + d.bf_off, d.cout, n->theta + d.b_off, 1, mask,
                           out, n->err, n->wait_ns, n->s);
}

cudaError_t dgrad(hg_cnn n, int layer, const __nv_bfloat16 *dy, int B, int l, const __nv_bfloat16 *mask,
                  __nv_bfloat16 *dx) {
    const LayerDesc &d = kTab.l[layer];
    n->launches++;
    return conv_fwd_launch(dy, B, n->H >> l, n->W >> l, d.cout, n->wt + d.bf_off, d.cin, nullptr, 0, mask, dx,
                           n->err, n->wait_ns, n->s);
}

cudaError_t wgrad(hg_cnn n, int layer, const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int l) {
    const LayerDesc &d = kTab.l[layer];
    n->launches += conv_launches_per_wgrad(true);
    return conv_wgrad_launch(x, dy, B, n->H >> l, n->W >> l, d.cin, d.cout, n->grad + d.w_off, n->grad + d.b_off,
                             n->ws, n->ws_bytes, n->err, n->wait_ns, n->s);
}

cudaError_t enqueue_forward(hg_cnn n, const float *T, int B) {
    const long npx0 = lvl_px(n, B, 0);
    k_img_stats_part<<<dim3(kStatBlocks, B), 256, 0, n->s>>>(T, (long)n->H * n->W, n->pmax, n->psum, n->err);
    k_img_stats_final<<<(B + 127) / 128, 128, 0, n->s>>>(n->pmax, n->psum, B, n->inv_max, n->inv_sumsq, n->err);
    k_first_fwd<<<ew_blocks(npx0, n->nsm), 256, 0, n->s>>>(T, n->inv_max, n->theta, B, n->H, n->W, n->A[0][0]);
    n->launches += 3;
    cudaError_t e;
    // encoder (layers 1..7: e0b e1a e1b e2a e2b e3a e3b)
    if ((e = conv(n, 1, n->A[0][0], B, 0, nullptr, n->A[0][1])) != cudaSuccess) return e;
    for (int l = 1; l < 4; ++l) {
        const int Hp = n->H >> (l - 1), Wp = n->W >> (l - 1), Cp = kWidth[l - 1];
        k_pool<<<ew_blocks(lvl_px(n, B, l) * Cp / 8, n->nsm), 256, 0, n->s>>>(n->A[l - 1][1], B, Hp, Wp, Cp,
                                                                              n->P[l - 1]);
        n->launches++;
        if ((e = conv(n, 2 * l, n->P[l - 1], B, l, nullptr, n->A[l][0])) != cudaSuccess) return e;
        if ((e = conv(n, 2 * l + 1, n->A[l][0], B, l, nullptr, n->A[l][1])) != cudaSuccess) return e;
    }
    // decoder (layers 8..13: d2a d2b d1a d1b d0a d0b)
    const __nv_bfloat16 *coarse = n->A[3][1];
    for (int l = 2; l >= 0; --l) {
        const int Hl = n->H >> l, Wl = n->W >> l, Cu = kWidth[l + 1], Cs = kWidth[l];
        k_upcat<<<ew_blocks(lvl_px(n, B, l) * (Cu + Cs) / 8, n->nsm), 256, 0, n->s>>>(coarse, n->A[l][1], B, Hl, Wl,
                                                                                      Cu, Cs, n->C[l]);
        n->launches++;
        const int la = 8 + 2 * (2 - l);
        if ((e = conv(n, la, n->C[l], B, l, nullptr, n->D[l][0])) != cudaSuccess) return e;
        if ((e = conv(n, la + 1, n->D[l][0], B, l, nullptr, n->D[l][1])) != cudaSuccess) return e;
        coarse = n->D[l][1];
    }
    return cudaGetLastError();
}

int head_blocks(hg_cnn n, long npx) {
    long b = (npx + HEAD_THREADS - 1) / HEAD_THREADS;
    const long cap = (long)n->nsm * 4;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

cudaError_t enqueue_backward(hg_cnn n, const float *T, const float *phi, int B, double *loss_out) {
    const long npx0 = lvl_px(n, B, 0);
    const int hb = head_blocks(n, npx0);
    k_head<<<hb, HEAD_THREADS, 0, n->s>>>(n->D[0][1], n->theta, T, phi, n->inv_sumsq, B, (long)n->H * n->W,
                                          1.f / (float)B, n->G[0][0], nullptr, nullptr, n->head_part, n->base);
    k_head_final<<<1, 96, 0, n->s>>>(n->head_part, hb, n->grad, loss_out ? loss_out : n->loss);
    n->launches += 2;
    cudaError_t e;
    // decoder, finest first: G[l][0] = dpre of d_lb on entry
    for (int l = 0; l <= 2; ++l) {
        const int la = 8 + 2 * (2 - l);
        if ((e = wgrad(n, la + 1, n->D[l][0], n->G[l][0], B, l)) != cudaSuccess) return e;
        if ((e = dgrad(n, la + 1, n->G[l][0], B, l, n->D[l][0], n->G[l][1])) != cudaSuccess) return e;
        if ((e = wgrad(n, la, n->C[l], n->G[l][1], B, l)) != cudaSuccess) return e;
        if ((e = dgrad(n, la, n->G[l][1], B, l, nullptr, n->G[l][2])) != cudaSuccess) return e;
        // split the concatenation: upsampled part -> dpre of the coarser output
        const __nv_bfloat16 *cmask = l < 2 ? n->D[l + 1][1] : n->A[3][1];
        const int Cu = kWidth[l + 1], Cs = kWidth[l];
        const long nn = lvl_px(n, B, l + 1) * (Cu / 8) + lvl_px(n, B, l) * (Cs / 8);
        k_upcat_bwd<<<ew_blocks(nn, n->nsm), 256, 0, n->s>>>(n->G[l][2], cmask, B, n->H >> l, n->W >> l, Cu, Cs,
                                                             n->G[l + 1][0], n->DS[l]);
        n->launches++;
    }
    // encoder, coarsest first: G[l][0] = dpre of e_lb on entry
    for (int l = 3; l >= 0; --l) {
        if ((e = wgrad(n, 2 * l + 1, n->A[l][0], n->G[l][0], B, l)) != cudaSuccess) return e;
        if ((e = dgrad(n, 2 * l + 1, n->G[l][0], B, l, n->A[l][0], n->G[l][1])) != cudaSuccess) return e;
        if (l == 0) break;
        if ((e = wgrad(n, 2 * l, n->P[l - 1], n->G[l][1], B, l)) != cudaSuccess) return e;
        if ((e = dgrad(n, 2 * l, n->G[l][1], B, l, nullptr, n->G[l][2])) != cudaSuccess) return e;
        const int Cp = kWidth[l - 1];
        k_pool_bwd_add<<<ew_blocks(lvl_px(n, B, l - 1) * Cp / 8, n->nsm), 256, 0, n->s>>>(
            n->G[l][2], n->DS[l - 1], n->A[l - 1][1], B, n->H >> (l - 1), n->W >> (l - 1), Cp, n->G[l - 1][0]);
        n->launches++;
    }
    // first layer: G[0][1] = dpre of e0a
    const int fb = ew_blocks(npx0 / 8, n->nsm);
    k_first_wgrad_part<<<fb, 256, 0, n->s>>>(T, n->inv_max, n->G[0][1], B, n->H, n->W, n->first_part);
    // weights [9][32][1] = [t][co] and bias [32] are contiguous in the vector
    k_rows_sum<<<(kFirstPartN + 127) / 128, 128, 0, n->s>>>(n->first_part, fb, kFirstPartN, n->grad + kTab.l[0].w_off);
    n->launches += 2;
    return cudaGetLastError();
}

cudaError_t refresh_bf16(hg_cnn n) {
    k_adam<<<ew_blocks(kTab.n, n->nsm), 256, 0, n->s>>>(n->theta, n->grad, n->m, n->v, kTab.n, 0, 0.f, 0.f, 0.f, 0.f,
                                                        0.f, 0.f, n->wf, n->wt);
    n->launches++;
    return cudaGetLastError();
}

struct CnnGuard {
    int prev = -1;
    explicit CnnGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~CnnGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

void hg_cnn_destroy(hg_cnn n) {
    if (!n) return;
    CnnGuard g(n->dev);
    cudaStreamSynchronize(n->s);
    for (void *p : n->owned) cudaFree(p);
    delete n;
}

hg_status hg_cnn_create(hg_cnn *out, int H, int W, int maxB, uint64_t seed, void *stream) {
    if (!out) return HG_ERR_INVALID_ARG;
    *out = nullptr;
    if (maxB < 1 || H < 1 || W < 1) return HG_ERR_INVALID_ARG;
    if (!net_shape_ok(H, W)) return HG_ERR_UNSUPPORTED_SIZE;
    hg_cnn n = new (std::nothrow) hg_cnn_s();
    if (!n) return HG_ERR_OOM;
    n->H = H;
    n->W = W;
    n->maxB = maxB;
    n->s = (cudaStream_t)stream;
    auto fail = [&](cudaError_t e) {
        hg_cnn_destroy(n);
        return st_of(e);
    };
    cudaError_t e = cudaGetDevice(&n->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->nsm, cudaDevAttrMultiProcessorCount, n->dev);
    if (e != cudaSuccess) return fail(e);
    const long NP = kTab.n;
    if ((e = alloc(n, &n->theta, NP)) || (e = alloc(n, &n->grad, NP)) || (e = alloc(n, &n->m, NP)) ||
        (e = alloc(n, &n->v, NP)) || (e = alloc(n, &n->wf, kTab.nbf)) || (e = alloc(n, &n->wt, kTab.nbf)))
        return fail(e);
    for (int l = 0; l < 4; ++l) {
        const long px = lvl_px(n, maxB, l);
        if ((e = alloc(n, &n->A[l][0], px * kWidth[l])) || (e = alloc(n, &n->A[l][1], px * kWidth[l])))
            return fail(e);
        if ((e = alloc(n, &n->G[l][0], px * kWidth[l])) || (e = alloc(n, &n->G[l][1], px * kWidth[l])) ||
            (e = alloc(n, &n->G[l][2], px * kGcC[l])))
            return fail(e);
        if (l < 3) {
            if ((e = alloc(n, &n->C[l], px * kCatC[l])) || (e = alloc(n, &n->D[l][0], px * kWidth[l])) ||
                (e = alloc(n, &n->D[l][1], px * kWidth[l])) || (e = alloc(n, &n->DS[l], px * kWidth[l])) ||
                (e = alloc(n, &n->P[l], lvl_px(n, maxB, l + 1) * kWidth[l])))
                return fail(e);
        }
    }
    size_t ws = 0;
    for (int i = 1; i < kConvs; ++i) {
        const int l = i <= 7 ? i / 2 : (13 - i) / 2;  // level of layer i
        const size_t b = conv_wgrad_workspace(maxB, H >> l, W >> l, kTab.l[i].cin, kTab.l[i].cout);
        if (!b) return fail(cudaErrorInvalidValue);
        if (b > ws) ws = b;
    }
    n->ws_bytes = ws;
    if ((e = alloc(n, (char **)&n->ws, ws))) return fail(e);
    const long fbmax = ew_blocks(lvl_px(n, maxB, 0) / 8, n->nsm);
    if ((e = alloc(n, &n->first_part, fbmax * kFirstPartN)) ||
        (e = alloc(n, &n->head_part, (long)n->nsm * 4 * kHeadPartN)) || (e = alloc(n, &n->inv_max, maxB)) ||
        (e = alloc(n, &n->inv_sumsq, maxB)) || (e = alloc(n, &n->pmax, (long)maxB * kStatBlocks)) ||
        (e = alloc(n, &n->psum, (long)maxB * kStatBlocks)) || (e = alloc(n, &n->err, 1)) ||
        (e = alloc(n, &n->loss, 1)))
        return fail(e);
    if ((e = cudaMemsetAsync(n->err, 0, sizeof(unsigned), n->s)) ||
        (e = cudaMemsetAsync(n->m, 0, sizeof(float) * NP, n->s)) ||
        (e = cudaMemsetAsync(n->v, 0, sizeof(float) * NP, n->s)) ||
        (e = cudaMemsetAsync(n->grad, 0, sizeof(float) * NP, n->s)))
        return fail(e);
    k_init_params<<<ew_blocks(NP, n->nsm), 256, 0, n->s>>>(n->theta, NP, seed);
    if ((e = refresh_bf16(n)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(n->s)) != cudaSuccess) return fail(e);
    *out = n;
    return HG_OK;
}

hg_status hg_cnn_set_params(hg_cnn n, const float *params) {
    if (!n || !params) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    n->launches = 0;
    CN_CK(cudaMemcpyAsync(n->theta, params, sizeof(float) * kTab.n, cudaMemcpyDeviceToDevice, n->s));
    CN_CK(refresh_bf16(n));
    return HG_OK;
}

hg_status hg_cnn_get_params(hg_cnn n, float *params) {
    if (!n || !params) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    CN_CK(cudaMemcpyAsync(params, n->theta, sizeof(float) * kTab.n, cudaMemcpyDeviceToDevice, n->s));
    return HG_OK;
}

hg_status hg_cnn_get_state(hg_cnn n, float *state, int64_t *step) {
    if (!n || !state || !step) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    const size_t b = sizeof(float) * kTab.n;
    CN_CK(cudaMemcpyAsync(state, n->theta, b, cudaMemcpyDeviceToDevice, n->s));
    CN_CK(cudaMemcpyAsync(state + kTab.n, n->m, b, cudaMemcpyDeviceToDevice, n->s));
    CN_CK(cudaMemcpyAsync(state + 2 * kTab.n, n->v, b, cudaMemcpyDeviceToDevice, n->s));
    *step = n->step;
    return HG_OK;
}

hg_status hg_cnn_set_state(hg_cnn n, const float *state, int64_t step) {
    if (!n || !state || step < 0) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    n->launches = 0;
    const size_t b = sizeof(float) * kTab.n;
    CN_CK(cudaMemcpyAsync(n->theta, state, b, cudaMemcpyDeviceToDevice, n->s));
    CN_CK(cudaMemcpyAsync(n->m, state + kTab.n, b, cudaMemcpyDeviceToDevice, n->s));
    CN_CK(cudaMemcpyAsync(n->v, state + 2 * kTab.n, b, cudaMemcpyDeviceToDevice, n->s));
    n->step = step;
    CN_CK(refresh_bf16(n));
    return HG_OK;
}

hg_status hg_cnn_set_base_phase(hg_cnn n, const float *base) {
    if (!n) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    if (!base) {
        CN_CK(cudaStreamSynchronize(n->s));
        n->base = nullptr;
        return HG_OK;
    }
    const long npx = (long)n->H * n->W;
    if (!n->base_buf) CN_CK(alloc(n, &n->base_buf, npx));
    CN_CK(cudaMemcpyAsync(n->base_buf, base, sizeof(float) * npx, cudaMemcpyDefault, n->s));
    CN_CK(cudaStreamSynchronize(n->s));
    n->base = n->base_buf;
    return HG_OK;
}

hg_status hg_cnn_get_grads(hg_cnn n, float *grads) {
    if (!n || !grads) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    CN_CK(cudaMemcpyAsync(grads, n->grad, sizeof(float) * kTab.n, cudaMemcpyDeviceToDevice, n->s));
    return HG_OK;
}

hg_status hg_cnn_forward(hg_cnn n, const float *T, int B, float *cs_out, float *phase_out) {
    if (!n || !T || B < 1 || B > n->maxB) return HG_ERR_INVALID_ARG;
    nvtxRangePushA("hg_cnn_forward");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    CnnGuard g(n->dev);
    n->launches = 0;
    CN_CK(enqueue_forward(n, T, B));
    const long npx0 = lvl_px(n, B, 0);
    k_head<<<head_blocks(n, npx0), HEAD_THREADS, 0, n->s>>>(n->D[0][1], n->theta, nullptr, nullptr, nullptr, B,
                                                            (long)n->H * n->W, 1.f, nullptr, (float2 *)cs_out,
                                                            phase_out, nullptr, n->base);
    n->launches++;
    CN_CK(cudaGetLastError());
    return HG_OK;
}

hg_status hg_cnn_gradients(hg_cnn n, const float *T, const float *phi, int B, double *loss_out) {
    if (!n || !T || !phi || B < 1 || B > n->maxB) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    n->launches = 0;
    CN_CK(enqueue_forward(n, T, B));
    CN_CK(enqueue_backward(n, T, phi, B, loss_out));
    return HG_OK;
}

hg_status hg_cnn_train_step(hg_cnn n, const float *T, const float *phi, int B, float lr, double *loss_out) {
    if (!n || !T || !phi || B < 1 || B > n->maxB || !(lr > 0.f)) return HG_ERR_INVALID_ARG;
    nvtxRangePushA("hg_cnn_train_step");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    CnnGuard g(n->dev);
    n->launches = 0;
    CN_CK(enqueue_forward(n, T, B));
    CN_CK(enqueue_backward(n, T, phi, B, loss_out));
    n->step++;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 / (1.0 - std::pow(b1, (double)n->step)));
    const float bc2 = (float)(1.0 / (1.0 - std::pow(b2, (double)n->step)));
    k_adam<<<ew_blocks(kTab.n, n->nsm), 256, 0, n->s>>>(n->theta, n->grad, n->m, n->v, kTab.n, 1, lr, (float)b1,
                                                        (float)b2, 1e-8f, bc1, bc2, n->wf, n->wt);
    n->launches++;
    CN_CK(cudaGetLastError());
    return HG_OK;
}

hg_status hg_cnn_apply_grads(hg_cnn n, const float *grads, float lr) {
    if (!n || !grads || !(lr > 0.f)) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    n->launches = 0;
    CN_CK(cudaMemcpyAsync(n->grad, grads, sizeof(float) * kTab.n, cudaMemcpyDefault, n->s));
    n->step++;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 / (1.0 - std::pow(b1, (double)n->step)));
    const float bc2 = (float)(1.0 / (1.0 - std::pow(b2, (double)n->step)));
    k_adam<<<ew_blocks(kTab.n, n->nsm), 256, 0, n->s>>>(n->theta, n->grad, n->m, n->v, kTab.n, 1, lr, (float)b1,
                                                        (float)b2, 1e-8f, bc1, bc2, n->wf, n->wt);
    n->launches++;
    CN_CK(cudaGetLastError());
    return HG_OK;
}

hg_status hg_cnn_sync(hg_cnn n) {
    if (!n) return HG_ERR_INVALID_ARG;
    CnnGuard g(n->dev);
    CN_CK(cudaStreamSynchronize(n->s));
    unsigned h = 0;
    CN_CK(cudaMemcpy(&h, n->err, sizeof h, cudaMemcpyDeviceToHost));
    if (h) CN_CK(cudaMemset(n->err, 0, sizeof(unsigned)));
    if (h & ERR_TIMEOUT_BIT) return HG_ERR_TIMEOUT;
    if (h & CNN_ERR_BAD) return HG_ERR_INVALID_ARG;
    if (h & CNN_ERR_ZERO) return HG_ERR_NUMERIC;
    return HG_OK;
}

int hg_cnn_launch_count(hg_cnn n) { return n ? n->launches : 0; }

}  // extern "C"
