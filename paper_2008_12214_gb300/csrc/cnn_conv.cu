// cnn_conv.cu -- host side of the tensor-core convolutions: tensor maps, tile
// and pipeline sizing, the fixed-order reductions of the weight gradient,
// and the layer-level C ABI of include/hologen_cnn.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#define HG_CONV_KERNELS
#include "cnn_conv.cuh"
#include "hologen_cnn.h"

namespace hg {
namespace {

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    });
    return fn;
}

constexpr int kMaxDevices = 64;
constexpr int kSmemCap = 220 * 1024;  // dynamic shared memory a conv CTA may take
constexpr int kMaxStages = 12;
constexpr int kWgTargetCtas = 304;    // weight-gradient CTAs aimed for (fixed: the workspace depends on it)
std::mutex g_mu;
int g_nsm[kMaxDevices];
bool g_attr[kMaxDevices];

cudaError_t device_setup(int *nsm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_attr[dev]) {
        if ((e = cudaDeviceGetAttribute(&g_nsm[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_conv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_conv_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)) !=
            cudaSuccess)
            return e;
        g_attr[dev] = true;
    }
    *nsm = g_nsm[dev];
    return cudaSuccess;
}

uint32_t pow2_cols(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// 4D map of an activation tensor [B][H][W][C] (BF16), box {32, bw, bh, 1}.
bool act_map(CUtensorMap *m, const void *p, int B, int H, int W, int C, int bw, int bh) {
    EncodeFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t gd[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t gs[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {32, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(p), gd, gs, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D map of a weight tensor [9][N][K] (BF16), box {32, nb, 1}.
bool wt_map(CUtensorMap *m, const void *p, int N, int K, int nb) {
    EncodeFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t gd[3] = {(cuuint64_t)K, (cuuint64_t)N, 9};
    const cuuint64_t gs[2] = {(cuuint64_t)K * 2, (cuuint64_t)N * K * 2};
    const cuuint32_t box[3] = {32, (cuuint32_t)nb, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(p), gd, gs, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// A box of `pix` pixels: whole row segments of `pix` when W >= pix, else
// pix / W whole rows.
bool box_shape(int H, int W, int pix, int *bw, int *bh) {
    if (W >= pix) {
        if (W % pix) return false;
        *bw = pix;
        *bh = 1;
    } else {
        if (pix % W) return false;
        *bw = W;
        *bh = pix / W;
        if (H % *bh) return false;
    }
    return true;
}

struct WgPlan {
    int kw, kh, mtiles, splits, chunks, per_split;
};
bool wg_plan(int B, int H, int W, int Cin, int Cout, WgPlan *p) {
    if (B < 1 || Cin < 32 || Cin % 32 || Cout < 32 || Cout % 32 || Cout > 256) return false;
    if (!box_shape(H, W, CV_WG_KP, &p->kw, &p->kh)) return false;
    p->chunks = (int)((long)B * H * W / CV_WG_KP);
    p->mtiles = (9 * Cin + 127) / 128;
    int splits = (kWgTargetCtas + p->mtiles - 1) / p->mtiles;
    if (splits > p->chunks) splits = p->chunks;
    if (splits < 1) splits = 1;
    p->per_split = (p->chunks + splits - 1) / splits;
    p->splits = (p->chunks + p->per_split - 1) / p->per_split;  // every split non-empty
    return true;
}

// dw[t][co][ci] = sum over splits (in order) of partial[s][t*Cin + ci][co].
__global__ void k_wg_reduce(const float *__restrict__ part, int splits, int Cin, int Cout, float *__restrict__ dw) {
    const int rows = 9 * Cin;
    const long n = (long)rows * Cout;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int row = (int)(i / Cout), co = (int)(i - (long)row * Cout);
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) acc += part[((size_t)s * rows + row) * Cout + co];
        const int t = row / Cin, ci = row - t * Cin;
        dw[((size_t)t * Cout + co) * Cin + ci] = acc;
    }
}

constexpr int CS_THREADS = 256;

// Block partials of per-channel sums: part[block][c], pixels split over blocks.
__global__ void __launch_bounds__(CS_THREADS)
    k_chan_part(const __nv_bfloat16 *__restrict__ x, long npx, int C, float *__restrict__ part) {
    __shared__ float red[CS_THREADS];
    const int P = CS_THREADS / C;  // pixel lanes (C divides 256)
    const int c = threadIdx.x % C, pl = threadIdx.x / C;
    float acc = 0.f;
    if (pl < P)
        for (long p = (long)blockIdx.x * P + pl; p < npx; p += (long)gridDim.x * P)
            acc += __bfloat162float(x[p * C + c]);
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int q = 0; q < P; ++q) s += red[q * C + threadIdx.x];
        part[(size_t)blockIdx.x * C + threadIdx.x] = s;
    }
}

__global__ void k_chan_final(const float *__restrict__ part, int blocks, int C, float *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double s = 0;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * C + c];
    out[c] = (float)s;
}

}  // namespace

bool conv_fwd_shape_ok(int B, int H, int W, int Cin, int N) {
    int bw, bh;
    if (B < 1 || H < 1 || W < 1 || Cin < 32 || Cin % 32 || N < 32 || N % 32 || N > 512) return false;
    return box_shape(H, W, 128, &bw, &bh);
}

cudaError_t conv_fwd_launch(const __nv_bfloat16 *x, int B, int H, int W, int Cin, const __nv_bfloat16 *w, int N,
                            const float *bias, int relu, const __nv_bfloat16 *mask, __nv_bfloat16 *out,
                            unsigned *err, unsigned long long wait_ns, cudaStream_t s) {
    if (!conv_fwd_shape_ok(B, H, W, Cin, N) || !x || !w || !out || !err) return cudaErrorInvalidValue;
    if (!aligned16(x) || !aligned16(w) || !aligned16(out) || (mask && !aligned16(mask)) || (bias && ((uintptr_t)bias & 3)))
        return cudaErrorInvalidValue;
    int nsm = 0;
    cudaError_t e = device_setup(&nsm);
    if (e != cudaSuccess) return e;
    ConvFwdArgs a{};
    a.B = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.N = N;
    box_shape(H, W, 128, &a.bw, &a.bh);
    a.nbox = N > 256 ? 2 : 1;
    a.nb = N / a.nbox;
    a.tiles = (int)((long)B * H * W / 128);
    a.nbuf = 2 * N <= 512 ? 2 : 1;
    a.tmem_cols = pow2_cols(a.nbuf * N);
    const int stage = CV_ASLOT + N * 64;
    int S = (kSmemCap - 1024 - CV_CTL_BYTES) / stage;
    if (S > kMaxStages) S = kMaxStages;
    if (S < 2) return cudaErrorInvalidValue;
    a.stages = S;
    a.bias = bias;
    a.relu = relu;
    a.mask = mask;
    a.out = out;
    a.err = err;
    a.wait_ns = wait_ns;
    CUtensorMap am, bm;
    if (!act_map(&am, x, B, H, W, Cin, a.bw, a.bh) || !wt_map(&bm, w, N, Cin, a.nb)) return cudaErrorInvalidValue;
    const size_t smem = 1024 + (size_t)S * stage + CV_CTL_BYTES;
    // one CTA per SM: the tensor-memory columns of two CTAs could exceed 512
    const int grid = a.tiles < nsm ? a.tiles : nsm;
    k_conv_fwd<<<grid, CV_THREADS, smem, s>>>(a, am, bm);
    return cudaGetLastError();
}

bool conv_wgrad_shape_ok(int B, int H, int W, int Cin, int Cout) {
    WgPlan p;
    return wg_plan(B, H, W, Cin, Cout, &p);
}

int chan_sum_blocks(long npx) {
    long b = npx / 2048;
    if (b < 1) b = 1;
    if (b > 512) b = 512;
    return (int)b;
}

size_t conv_wgrad_workspace(int B, int H, int W, int Cin, int Cout) {
    WgPlan p;
    if (!wg_plan(B, H, W, Cin, Cout, &p)) return 0;
    const long npx = (long)B * H * W;
    return sizeof(float) * ((size_t)p.splits * 9 * Cin * Cout + (size_t)chan_sum_blocks(npx) * Cout) + 256;
}

cudaError_t chan_sum_launch(const __nv_bfloat16 *x, long npx, int C, float *part, float *out, cudaStream_t s) {
    if (C < 1 || C > CS_THREADS || CS_THREADS % C) return cudaErrorInvalidValue;
    const int blocks = chan_sum_blocks(npx);
    k_chan_part<<<blocks, CS_THREADS, 0, s>>>(x, npx, C, part);
    k_chan_final<<<(C + 127) / 128, 128, 0, s>>>(part, blocks, C, out);
    return cudaGetLastError();
}

int conv_launches_per_wgrad(bool with_bias) { return with_bias ? 4 : 2; }

cudaError_t conv_wgrad_launch(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, int B, int H, int W, int Cin,
                              int Cout, float *dw, float *db, void *ws, size_t ws_bytes, unsigned *err,
                              unsigned long long wait_ns, cudaStream_t s) {
    WgPlan p;
    if (!wg_plan(B, H, W, Cin, Cout, &p) || !x || !dy || !dw || !ws || !err) return cudaErrorInvalidValue;
    if (ws_bytes < conv_wgrad_workspace(B, H, W, Cin, Cout) || !aligned16(x) || !aligned16(dy) || !aligned16(ws))
        return cudaErrorInvalidValue;
    int nsm = 0;
    cudaError_t e = device_setup(&nsm);
    if (e != cudaSuccess) return e;
    ConvWgArgs a{};
    a.B = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.kw = p.kw;
    a.kh = p.kh;
    a.mtiles = p.mtiles;
    a.splits = p.splits;
    a.chunks = p.chunks;
    a.per_split = p.per_split;
    a.tmem_cols = pow2_cols(Cout);
    const int stage = 4 * CV_WG_ATOM + (Cout / 32) * CV_WG_ATOM;
    int S = (kSmemCap - 1024 - CV_CTL_BYTES) / stage;
    if (S > kMaxStages) S = kMaxStages;
    a.stages = S;
    a.partial = (float *)ws;
    a.err = err;
    a.wait_ns = wait_ns;
    CUtensorMap xm, gm;
    if (!act_map(&xm, x, B, H, W, Cin, p.kw, p.kh) || !act_map(&gm, dy, B, H, W, Cout, p.kw, p.kh))
        return cudaErrorInvalidValue;
    const size_t smem = 1024 + (size_t)S * stage + CV_CTL_BYTES;
    k_conv_wgrad<<<p.mtiles * p.splits, CV_THREADS, smem, s>>>(a, xm, gm);
    const long n = 9L * Cin * Cout;
    int rb = (int)((n + 255) / 256);
    if (rb > nsm * 8) rb = nsm * 8;
    k_wg_reduce<<<rb, 256, 0, s>>>(a.partial, p.splits, Cin, Cout, dw);
    if (db) {
        float *cpart = a.partial + (size_t)p.splits * 9 * Cin * Cout;
        e = chan_sum_launch(dy, (long)B * H * W, Cout, cpart, db, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace hg

// ------------------------------------------------------------ layer ABI

namespace {
__device__ unsigned g_conv_err;  // timeout bit of the layer-level calls (per device)

hg_status conv_err_ptr(unsigned **p) {
    if (cudaGetSymbolAddress((void **)p, g_conv_err) != cudaSuccess) return HG_ERR_CUDA;
    return HG_OK;
}
hg_status map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return HG_OK;
    if (e == cudaErrorInvalidValue) return HG_ERR_UNSUPPORTED_SIZE;
    if (e == cudaErrorMemoryAllocation) return HG_ERR_OOM;
    return HG_ERR_CUDA;
}
constexpr unsigned long long kLayerWaitNs = 2000000000ull;
}  // namespace

extern "C" {

hg_status hg_conv3x3_forward(const uint16_t *x, int B, int H, int W, int Cin, const uint16_t *w, int Cout,
                             const float *bias, int relu, const uint16_t *mask, uint16_t *y, void *stream) {
    if (!x || !w || !y) return HG_ERR_INVALID_ARG;
    if (!hg::conv_fwd_shape_ok(B, H, W, Cin, Cout)) return HG_ERR_UNSUPPORTED_SIZE;
    unsigned *err;
    hg_status st = conv_err_ptr(&err);
    if (st != HG_OK) return st;
    return map_cuda(hg::conv_fwd_launch((const __nv_bfloat16 *)x, B, H, W, Cin, (const __nv_bfloat16 *)w, Cout,
                                        bias, relu, (const __nv_bfloat16 *)mask, (__nv_bfloat16 *)y, err,
                                        kLayerWaitNs, (cudaStream_t)stream));
}

hg_status hg_conv3x3_dgrad(const uint16_t *dy, int B, int H, int W, int Cout, const uint16_t *w_rot, int Cin,
                           const uint16_t *mask, uint16_t *dx, void *stream) {
    return hg_conv3x3_forward(dy, B, H, W, Cout, w_rot, Cin, nullptr, 0, mask, dx, stream);
}

size_t hg_conv3x3_wgrad_workspace(int B, int H, int W, int Cin, int Cout) {
    return hg::conv_wgrad_workspace(B, H, W, Cin, Cout);
}

hg_status hg_conv3x3_wgrad(const uint16_t *x, const uint16_t *dy, int B, int H, int W, int Cin, int Cout,
                           float *dw, float *db, void *workspace, size_t workspace_bytes, void *stream) {
    if (!x || !dy || !dw || !workspace) return HG_ERR_INVALID_ARG;
    if (!hg::conv_wgrad_shape_ok(B, H, W, Cin, Cout)) return HG_ERR_UNSUPPORTED_SIZE;
    if (workspace_bytes < hg::conv_wgrad_workspace(B, H, W, Cin, Cout)) return HG_ERR_INVALID_ARG;
    unsigned *err;
    hg_status st = conv_err_ptr(&err);
    if (st != HG_OK) return st;
    return map_cuda(hg::conv_wgrad_launch((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)dy, B, H, W, Cin, Cout,
                                          dw, db, workspace, workspace_bytes, err, kLayerWaitNs,
                                          (cudaStream_t)stream));
}

hg_status hg_conv_status(void *stream) {
    unsigned *err;
    hg_status st = conv_err_ptr(&err);
    if (st != HG_OK) return st;
    unsigned h = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HG_ERR_CUDA;
    if (cudaMemcpy(&h, err, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ERR_CUDA;
    if (h) {
        const unsigned zero = 0;
        if (cudaMemcpy(err, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) return HG_ERR_CUDA;
        return HG_ERR_TIMEOUT;
    }
    return HG_OK;
}

}  // extern "C"
