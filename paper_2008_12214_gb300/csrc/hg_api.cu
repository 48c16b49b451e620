// hg_api.cu -- the C ABI of include/hologen.h: plans, workspace, the launch
// sequence of a run, and the small non-transform kernels (target preparation,
// metric reduction, weight fill).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hg_pipe.cuh"
#include "hg_search.cuh"
#include "hg_tc.cuh"
#include "hologen.h"

using namespace hg;

// NVTX range around a host call (visible to Nsight tools; free without one).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// ------------------------------------------------------------------ kernels

namespace {

enum ErrBits : unsigned { ERR_BAD_VALUE = 1u, ERR_ZERO_ENERGY = 2u };
static_assert(ERR_TIMEOUT_BIT == 4u, "error bits must be distinct");

constexpr int PREP_THREADS = 256;
constexpr int PREP_BLOCKS = 64;  // per target

// Partial sums of T^2 per (target, block), fixed order: each thread sums its
// strided elements in float, threads and warps combine in double.  Flags
// negative, NaN and infinite values.
__global__ void __launch_bounds__(PREP_THREADS)
k_prep_sum(const float *__restrict__ t_raw, int npx, const uint8_t *__restrict__ roi, double *part,
           unsigned *err) {
    __shared__ double red[PREP_THREADS / 32];
    const int b = blockIdx.y;
    const float *tb = t_raw + (size_t)b * npx;
    float sf = 0.f;
    bool bad = false;
    for (int i = blockIdx.x * PREP_THREADS + threadIdx.x; i < npx; i += PREP_BLOCKS * PREP_THREADS) {
        const float v = tb[i];
        if (!(v >= 0.f) || isinf(v)) bad = true;
        if (!roi || roi[i]) sf = fmaf(v, v, sf);
    }
    double s = sf;
    if (bad) atomicOr(err, ERR_BAD_VALUE);
    for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0;
        for (int w = 0; w < PREP_THREADS / 32; ++w) tot += red[w];
        part[(size_t)b * PREP_BLOCKS + blockIdx.x] = tot;
    }
}

// scale[b] = 1 / sqrt(sum T^2) (0 and a flag for an all-zero target).
__global__ void k_prep_scale(const double *part, int batch, double *scale, unsigned *err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    double s = 0;
    for (int i = 0; i < PREP_BLOCKS; ++i) s += part[(size_t)b * PREP_BLOCKS + i];
    if (s > 0) {
        scale[b] = 1.0 / sqrt(s);
    } else {
        scale[b] = 0;
        atomicOr(err, ERR_ZERO_ENERGY);
    }
}

// Prepared target in DFT order: Tf[b][y][x] = T[b][(y+ny/2)%ny][(x+nx/2)%nx] * scale[b],
// rounded to float with the support T > 0 preserved.  One CTA per output row
// (block b * ny + y): the source row is read as two contiguous halves.
__global__ void k_prep_apply(const float *__restrict__ t_raw, int ny, int nx, int batch,
                             const double *scale, const uint8_t *__restrict__ roi, float *__restrict__ tf) {
    const int b = blockIdx.x / ny, y = blockIdx.x - b * ny;
    if (b >= batch) return;
    const int iy = y + ny / 2 < ny ? y + ny / 2 : y + ny / 2 - ny;
    const float sc = (float)scale[b];
    const float *src = t_raw + ((size_t)b * ny + iy) * nx;
    const uint8_t *rr = roi ? roi + (size_t)iy * nx : nullptr;
    float *dst = tf + ((size_t)b * ny + y) * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const int ix = x + nx / 2 < nx ? x + nx / 2 : x + nx / 2 - nx;
        const float v = (!rr || rr[ix]) ? src[ix] : 0.f;  // target restricted to the ROI
        float tv = v * sc;
        // keep the support {T > 0} of the input exactly: a positive value whose
        // scaled float underflows becomes the smallest positive float
        if (v > 0.f && !(tv > 0.f)) tv = __int_as_float(1);
        dst[x] = tv;
    }
}

// DFT-order <-> replay-order copies of a real [batch][ny][nx] array.
// to_dft: dst[y][x] = src[(y+ny/2)%ny][(x+nx/2)%nx]; else the inverse map.
__global__ void k_reorder(const float *__restrict__ src, float *__restrict__ dst, int ny, int nx,
                          int batch, int to_dft) {
    const size_t npx = (size_t)ny * nx, total = npx * batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / npx);
        const int rem = (int)(i - (size_t)b * npx);
        const int y = rem / nx, x = rem - y * nx;
        const size_t r = (size_t)b * npx + (size_t)((y + ny / 2) % ny) * nx + (x + nx / 2) % nx;
        if (to_dft) dst[i] = src[r];
        else dst[r] = src[i];
    }
}

// Deterministic pseudo-random fill in [lo, lo + span) (autotuner inputs).
__global__ void k_fill_hash(float *p, size_t n, float lo, float span) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u;
        h ^= h >> 15;
        h *= 0x85EBCA77u;
        h ^= h >> 13;
        p[i] = lo + span * (float)(h >> 8) * (1.0f / 16777216.0f);
    }
}

__global__ void k_fill(float *p, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// metrics[b][k][4] from the per-panel partials: slot k holds
// [batch][panels_k][4] at part + k * batch * stride * 4, where panels_k is
// `panels` for k < iters - 1 and `panels_last` for the last slot.  Output:
// {sum d^2 / N, sum a^2 / N, in / total, total}; also mse_out[b][k].
__global__ void k_reduce(const double *part, int iters, int batch, int stride, int panels,
                         int panels_last, double invN, double *metrics, double *mse_out) {
    // one warp per (iteration, target): lane l sums panels l, l+32, ...; the
    // 32 lane sums are combined by a fixed shuffle tree
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= iters * batch) return;
    const int k = w / batch, b = w - k * batch;
    const int np = k == iters - 1 ? panels_last : panels;
    const double *p = part + ((size_t)k * batch * stride + (size_t)b * np) * NMET;
    double s[NMET] = {0, 0, 0, 0};
    for (int q = lane; q < np; q += 32)
        for (int m = 0; m < NMET; ++m) s[m] += p[(size_t)q * NMET + m];
    for (int off = 16; off; off >>= 1)
        for (int m = 0; m < NMET; ++m) s[m] += __shfl_down_sync(0xffffffffu, s[m], off);
    if (lane) return;
    double *o = metrics + ((size_t)b * iters + k) * NMET;
    o[0] = s[0] * invN;
    o[1] = s[1] * invN;
    o[2] = s[3] > 0 ? s[2] / s[3] : 0.0;
    o[3] = s[3];
    if (mse_out) mse_out[(size_t)b * iters + k] = o[0];
}

// metrics[b][k][4] of a modulated plan from its eight per-panel sums (see
// ROW_ITER): with g0 = sum_ROI |R|^2, g1 = sum_ROI |R|^4, g2 = sum_ROI |R|^2
// T^2, g3 = sum_ROI |R| T, g4 = sum_{ROI, T>0} |R|^2, g5 = sum |R|^2, g6 =
// sum T^4, g7 = sum T^2 (unitary |R|), the intensity I = s |R|^2 with the
// ROI energy match s = g7 / g0 gives
//   intensity MSE = (s^2 g1 - 2 s g2 + g6) / n_roi,
//   amplitude MSE = (s g0 - 2 sqrt(s) g3 + g7) / n_roi,
//   efficiency g4 / g5, and g5 itself.
__global__ void k_reduce_gen(const double *part, int iters, int batch, int stride, int panels,
                             int panels_last, const unsigned long long *nroi, double *metrics, double *mse_out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= iters * batch) return;
    const int k = w / batch, b = w - k * batch;
    const int np = k == iters - 1 ? panels_last : panels;
    const double *p = part + ((size_t)k * batch * stride + (size_t)b * np) * NMET_GEN;
    double g[NMET_GEN] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = lane; q < np; q += 32)
        for (int m = 0; m < NMET_GEN; ++m) g[m] += p[(size_t)q * NMET_GEN + m];
    for (int off = 16; off; off >>= 1)
        for (int m = 0; m < NMET_GEN; ++m) g[m] += __shfl_down_sync(0xffffffffu, g[m], off);
    if (lane) return;
    const double s = g[0] > 0 ? g[7] / g[0] : 0.0;
    const double inv_nroi = *nroi ? 1.0 / (double)*nroi : 0.0;
    double *o = metrics + ((size_t)b * iters + k) * NMET;
    o[0] = fmax(s * s * g[1] - 2.0 * s * g[2] + g[6], 0.0) * inv_nroi;
    o[1] = fmax(s * g[0] - 2.0 * sqrt(s) * g[3] + g[7], 0.0) * inv_nroi;
    o[2] = g[5] > 0 ? g[4] / g[5] : 0.0;
    o[3] = g[5];
    if (mse_out) mse_out[(size_t)b * iters + k] = o[0];
}

// Illumination of the SLM plane: E = amp exp(i (phase + c ((x - nx/2)^2 +
// (y - ny/2)^2))) in natural order, the phase summed in double (the Fresnel
// term reaches millions of radians).  amp / phase may be null (1 / 0);
// a negative or non-finite amplitude or phase sets ERR_BAD_VALUE.
__global__ void k_illum(const float *amp, const float *phase, int ny, int nx, double c, float2 *E,
                        unsigned *err) {
    const size_t n = (size_t)ny * nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i - (size_t)y * nx);
        const float a = amp ? amp[i] : 1.f, f = phase ? phase[i] : 0.f;
        if (!(a >= 0.f) || isinf(a) || !isfinite(f)) atomicOr(err, ERR_BAD_VALUE);
        const double dx = x - nx / 2, dy = y - ny / 2;
        double sn, cs;
        sincos((double)f + c * (dx * dx + dy * dy), &sn, &cs);
        E[i] = make_float2((float)(a * cs), (float)(a * sn));
    }
}

// Region of interest: DFT-order copy of a replay-order mask and its pixel
// count (*count zeroed before; integer sums, so the order does not matter).
__global__ void k_roi_dft(const uint8_t *roi, int ny, int nx, uint8_t *dft, unsigned long long *count) {
    const size_t n = (size_t)ny * nx;
    unsigned c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i - (size_t)y * nx);
        const uint8_t v = roi[(size_t)((y + ny / 2) % ny) * nx + (x + nx / 2) % nx] ? 1 : 0;
        dft[i] = v;
        c += v;
    }
    for (int off = 16; off; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// ---------------------------------------------------- evaluation of holograms
// Metrics of given holograms over the region of interest (Section 3.1): the
// replay intensity (any scale) I0, the raw target t (replay order).  Pass 1
// per (block, item): sum_ROI I0, sum I0, sum_ROI t^2, sum_{ROI, t>0} I0 and
// max_ROI t.  Pass 2 scales I = I0 / sum_ROI I0 and T = t / sqrt(sum_ROI t^2)
// and sums over the ROI (I - T^2)^2, (sqrt I - T)^2 and the moments of
// x = T / max T, y = sqrt(I) / max T: x, y, x^2, y^2, x y.  Threads sum in
// float over a fixed stride, blocks in double, items in a fixed order.
constexpr int EV_THREADS = 256, EV_BLOCKS = 64, EV_S1 = 5, EV_S2 = 7;

template <int K>
__device__ void ev_block_sum(float (&v)[K], double *dst) {
    __shared__ double red[EV_THREADS / 32][K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
        float x = v[m];
        for (int off = 16; off; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][m] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0;
        for (int w = 0; w < EV_THREADS / 32; ++w) s += red[w][threadIdx.x];
        dst[threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(EV_THREADS)
k_eval1(const float *I0, const float *t, const uint8_t *roi, int npx, double *part, unsigned *err) {
    const int b = blockIdx.y;
    const float *Ib = I0 + (size_t)b * npx;
    const float *tb = t ? t + (size_t)b * npx : nullptr;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    float tmax = 0.f;
    bool bad = false;
    for (int i = blockIdx.x * EV_THREADS + threadIdx.x; i < npx; i += EV_BLOCKS * EV_THREADS) {
        const float I = Ib[i];
        v[1] += I;
        if (roi && !roi[i]) continue;
        v[0] += I;
        if (tb) {
            const float tv = tb[i];
            if (!(tv >= 0.f) || isinf(tv)) bad = true;
            v[2] = fmaf(tv, tv, v[2]);
            if (tv > 0.f) v[3] += I;
            tmax = fmaxf(tmax, tv);
        }
    }
    if (bad) atomicOr(err, ERR_BAD_VALUE);
    double *dst = part + ((size_t)b * EV_BLOCKS + blockIdx.x) * EV_S1;
    ev_block_sum<4>(v, dst);
    for (int off = 16; off; off >>= 1) tmax = fmaxf(tmax, __shfl_down_sync(0xffffffffu, tmax, off));
    __shared__ float mx[EV_THREADS / 32];
    if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = tmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < EV_THREADS / 32; ++w) m = fmaxf(m, mx[w]);
        dst[4] = m;
    }
}

// Item totals of pass 1: {sum_ROI I0, sum I0, sum_ROI t^2, sum_{ROI,t>0} I0, max t}.
__device__ void ev_totals(const double *part1, int b, double (&g)[EV_S1]) {
    for (int m = 0; m < EV_S1; ++m) g[m] = 0;
    for (int k = 0; k < EV_BLOCKS; ++k) {
        const double *q = part1 + ((size_t)b * EV_BLOCKS + k) * EV_S1;
        for (int m = 0; m < 4; ++m) g[m] += q[m];
        g[4] = fmax(g[4], q[4]);
    }
}

// I_out (optional): I0 / sum I0 (normalised over the whole field).
__global__ void __launch_bounds__(EV_THREADS)
k_eval2(const float *I0, const float *t, const uint8_t *roi, int npx, const double *part1, double *part2,
        float *I_out) {
    const int b = blockIdx.y;
    __shared__ float sc[4];
    if (threadIdx.x == 0) {
        double g[EV_S1];
        ev_totals(part1, b, g);
        const double tsc = g[2] > 0 ? 1.0 / sqrt(g[2]) : 0.0;
        const double tm = g[4] * tsc;
        sc[0] = g[0] > 0 ? (float)(1.0 / g[0]) : 0.f;  // ROI energy match (sum_ROI T^2 = 1)
        sc[1] = (float)tsc;
        sc[2] = tm > 0 ? (float)(1.0 / tm) : 0.f;
        sc[3] = g[1] > 0 ? (float)(1.0 / g[1]) : 0.f;
    }
    __syncthreads();
    const float s = sc[0], tsc = sc[1], inv_tm = sc[2], s_all = sc[3];
    const float *Ib = I0 + (size_t)b * npx;
    const float *tb = t ? t + (size_t)b * npx : nullptr;
    float v[EV_S2] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = blockIdx.x * EV_THREADS + threadIdx.x; i < npx; i += EV_BLOCKS * EV_THREADS) {
        const float I0v = Ib[i];
        if (I_out) I_out[(size_t)b * npx + i] = I0v * s_all;
        if (!tb || (roi && !roi[i])) continue;
        const float I = I0v * s, T = tb[i] * tsc;
        const float d = I - T * T, am = sqrtf(I) - T;
        const float x = T * inv_tm, y = sqrtf(I) * inv_tm;
        v[0] = fmaf(d, d, v[0]);
        v[1] = fmaf(am, am, v[1]);
        v[2] += x;
        v[3] += y;
        v[4] = fmaf(x, x, v[4]);
        v[5] = fmaf(y, y, v[5]);
        v[6] = fmaf(x, y, v[6]);
    }
    if (part2) ev_block_sum<EV_S2>(v, part2 + ((size_t)b * EV_BLOCKS + blockIdx.x) * EV_S2);
}

// out[b][5] = {intensity MSE, amplitude MSE, efficiency, SSIM, sum |R|^2}:
// SSIM of Section 3.1 with c1 = 0.01^2, c2 = 0.03^2 (dynamic range 1);
// sum |R|^2 in unitary units = N sum I0 for I0 = |R|^2 / N.
__global__ void k_eval_fin(const double *part1, const double *part2, int batch, const unsigned long long *nroi,
                           double N, double *out, unsigned *err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double n_roi = nroi ? (double)*nroi : N;
    double g[EV_S1], h[EV_S2] = {0, 0, 0, 0, 0, 0, 0};
    ev_totals(part1, b, g);
    if (!(g[2] > 0)) atomicOr(err, ERR_ZERO_ENERGY);  // no target energy in the region of interest
    for (int k = 0; k < EV_BLOCKS; ++k)
        for (int m = 0; m < EV_S2; ++m) h[m] += part2[((size_t)b * EV_BLOCKS + k) * EV_S2 + m];
    const double mx = h[2] / n_roi, my = h[3] / n_roi;
    const double vx = fmax(h[4] / n_roi - mx * mx, 0.0), vy = fmax(h[5] / n_roi - my * my, 0.0);
    const double cxy = h[6] / n_roi - mx * my;
    const double c1 = 1e-4, c2 = 9e-4;
    double *o = out + (size_t)b * 5;
    o[0] = h[0] / n_roi;
    o[1] = h[1] / n_roi;
    o[2] = g[1] > 0 ? g[3] / g[1] : 0.0;
    o[3] = (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2));
    o[4] = g[1] * N;
}

// ------------------------------------------------------------ registry

const LineOps *find_ops(int n) {
    const LineOps *o = ops_small(n);
    if (!o) o = ops_mid(n);
    if (!o) o = ops_1024(n);
    if (!o) o = ops_2048(n);
    if (!o) o = ops_hd(n);
    return o;
}

int pipe_candidates(int n, const PipeOps **out, int max) {
    int k = pipe_ops_mid(n, out, max);
    if (!k) k = pipe_ops_1024(n, out, max);
    if (!k) k = pipe_ops_2048(n, out, max);
    if (!k) k = pipe_ops_hd(n, out, max);
    return k;
}

// Row panels per item of a TMA-fed row pass.
int row_panels(const PipeOps *o, int ny) {
    return o->paired ? ny / 2 + 1 : (ny + o->row_lines - 1) / o->row_lines;
}

// Autotuner cache: (device, ny, nx, items, slm kind) -> chosen candidates.
struct TuneEntry {
    int dev, ny, nx, items, kind;  // kind, + 8 for modulated plans (no paired candidates), + 16 more
                                   // when their column pass stays generic
    const PipeOps *row, *col;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

std::mutex g_init_mu;
constexpr int kMaxDev = 64;
constexpr int kMaxOps = 64;
const LineOps *g_inited[kMaxDev][kMaxOps];

const PipeOps *g_pinited[kMaxDev][kMaxOps];

cudaError_t ensure_pipe_init(int dev, const PipeOps *o) {
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    for (int i = 0; i < kMaxOps; ++i) {
        if (g_pinited[dev][i] == o) return cudaSuccess;
        if (!g_pinited[dev][i]) {
            cudaError_t e = o->init(const_cast<PipeOps *>(o));
            if (e == cudaSuccess) g_pinited[dev][i] = o;
            else cudaGetLastError();  // a candidate this device cannot run is skipped: clear its error
            return e;
        }
    }
    return cudaErrorUnknown;
}

bool g_tc_inited[kMaxDev];
int g_tc_blocks[kMaxDev];

cudaError_t ensure_tc_init(int dev, int *blocks) {
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (!g_tc_inited[dev]) {
        cudaError_t e = tc_init(&g_tc_blocks[dev]);
        if (e != cudaSuccess) return e;
        g_tc_inited[dev] = true;
    }
    *blocks = g_tc_blocks[dev] > 0 ? g_tc_blocks[dev] : 1;
    return cudaSuccess;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Per-device one-time kernel attributes for a line length.
cudaError_t ensure_init(int dev, const LineOps *o) {
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    for (int i = 0; i < kMaxOps; ++i) {
        if (g_inited[dev][i] == o) return cudaSuccess;
        if (!g_inited[dev][i]) {
            cudaError_t e = o->init(const_cast<LineOps *>(o));
            if (e == cudaSuccess) g_inited[dev][i] = o;
            return e;
        }
    }
    return cudaErrorUnknown;
}

}  // namespace

// ------------------------------------------------------------------ plan

struct hg_plan_s {
    int dev = 0, ny = 0, nx = 0, batch = 0, algo = 0, kind = 0, levels = 2, nsub = 1;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;     // user stream (may be the legacy default)
    cudaStream_t cap_stream = nullptr; // private stream used only for graph capture
    int use_graph = 1;
    const LineOps *rops = nullptr, *cops = nullptr;
    const PipeOps *prow = nullptr, *pcol = nullptr;  // pipelined passes (null: generic)
    float tune_ms[8] = {0};                          // autotuner timings: row cands (+ implied column), col cands
    int tc_prec = 0;                                 // tensor-core row pass precision (0: FP32 engine)
    uint4 *tc_b = nullptr;                           // DFT-32 operand matrices
    int tc_blocks = 1, ppt_tc = 0;
    CUtensorMap cmap;                                // field as [chains*ny][2*nx] floats
    CUtensorMap cmap_herm;                           // same field, tiles of the column-pair Hermitian pass
    CUtensorMap emap;                                // modulated: E as [ny][2*nx] floats, tiles as cmap's
    bool use_herm_col = false;                       // Hermitian loop: column pairs share transforms
    const PipeOps *hops = nullptr;                   // variant providing the column-pair pass
    bool ospr_herm = false;                          // binary OSPR in Hermitian form
    float lt_start = 1.f;                            // LT window: initial side fraction, growth length
    int lt_grow = 1;
    bool mod = false;                                // illuminated / Fresnel / amplitude SLM / ROI plan
    float2 *illum = nullptr;                         // modulated: SLM-plane illumination, natural order
    uint8_t *roi_rep = nullptr, *roi_dft = nullptr;  // modulated: region of interest (null: whole field)
    unsigned long long *nroi = nullptr;              // modulated: pixels in the region of interest (device)
    float fresnel = 0.f, amp_clip = 2.f;
    double *ev_part = nullptr;                       // hg_evaluate: pass partials
    float *ev_buf = nullptr;                         // hg_evaluate: replay intensity
    SearchLayout slay{};                             // direct search / annealing: CTA layout
    float2 *rbuf = nullptr;                          // direct search / annealing: initial replay fields
    uint8_t *sholo = nullptr;                        // direct search / annealing: holograms (no holo_out)
    double sa_temp = 0, sa_cool = 1;
    float *acc = nullptr;                            // adaptive OSPR: summed subframe intensities
    uint8_t *holo_tmp = nullptr;                     // adaptive OSPR: one subframe's holograms
    unsigned long long wait_ns = 2000000000ull;      // bound on a device-side wait
    int drop_job = -1;                               // fault-injection hook
    int nsm = 0, ppt = 0, ppt_pipe = 0, ppt_max = 0;
    // per-pass CUDA-event timing (hg_profile_enable): pairs around each row
    // and column pass of the iteration loop, kind 0 = row, 1 = column
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_used = 0;
    size_t npx = 0;
    int nchains = 0;
    float2 *field = nullptr;
    float *tf = nullptr, *w = nullptr;
    double *part = nullptr;
    int part_iters = 0;
    double *metrics = nullptr;
    int metrics_iters = 0;
    double *sum_part = nullptr, *scale = nullptr;
    unsigned *err = nullptr;
    float2 *twx = nullptr, *twy = nullptr, *lvl = nullptr;
    void *stage = nullptr;
    size_t stage_bytes = 0;
    bool weights_preset = false, have_run = false;
    bool field_from_run = false;  // field holds the last GS/WGS run's final column pass
    int last_iters = 0, launches = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_iters = -1;
    double *g_part = nullptr;
    char vname[2][128] = {};
    // hg_run with host buffers: the batch runs as chunks, each a view of this
    // plan (its own batch size, pointers into this plan's per-target buffers,
    // its own loop graph), so that one chunk's copies overlap another's
    // iterations; the copies go on two streams of their own
    bool is_view = false;
    int item0 = 0;  // a view: index of its first target in the plan's batch (Philox counters)
    int host_chunks = 0;
    std::vector<hg_plan_s *> views;
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
    std::vector<cudaEvent_t> chunk_ev;  // per chunk: inputs copied, iterations done
    // the default schedule's model, measured on the first chunked call with
    // x_iters iterations: per target, the input copy (x_in), the iterations
    // (x_it) and the output copy (x_out), and the fixed cost of one chunk
    // (x_fix), all in ms; timing events of that call
    int x_iters = 0;
    double x_in = 0, x_it = 0, x_out = 0, x_fix = 0;
    std::vector<cudaEvent_t> x_ev;
};

namespace {

#define HG_CK(x)                                   \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return map_err(e_); \
    } while (0)

hg_status map_err(cudaError_t e) {
    if (e == cudaSuccess) return HG_OK;
    if (e == cudaErrorMemoryAllocation) return HG_ERR_OOM;
    return HG_ERR_CUDA;
}

// Forward roots W_n^e = exp(-2 pi i e / n), e < n: angle reduced as an exact
// integer ratio, evaluated in long double, rounded to float.
hg_status make_twiddles(int n, float2 **out) {
    float2 *h = (float2 *)malloc(sizeof(float2) * n);
    if (!h) return HG_ERR_OOM;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int e = 0; e < n; ++e) {
        long double a = two_pi * (long double)e / (long double)n;
        h[e] = make_float2((float)cosl(a), (float)-sinl(a));
    }
    cudaError_t ce = cudaMalloc(out, sizeof(float2) * n);
    if (ce == cudaSuccess) ce = cudaMemcpy(*out, h, sizeof(float2) * n, cudaMemcpyHostToDevice);
    free(h);
    return map_err(ce);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

hg_status ensure_stage(hg_plan p, size_t bytes) {
    if (p->stage_bytes >= bytes) return HG_OK;
    if (p->stage) cudaFree(p->stage);
    p->stage = nullptr;
    p->stage_bytes = 0;
    HG_CK(cudaMalloc(&p->stage, bytes));
    p->stage_bytes = bytes;
    return HG_OK;
}

// doubles per panel in the metric partials
int part_stride(hg_plan p) { return p->mod ? NMET_GEN : NMET; }

hg_status ensure_part(hg_plan p, int iters) {
    if (p->part_iters >= iters) return HG_OK;
    if (p->part) cudaFree(p->part);
    p->part = nullptr;
    p->part_iters = 0;
    HG_CK(cudaMalloc(&p->part, sizeof(double) * part_stride(p) * (size_t)iters * p->batch * p->ppt_max));
    p->part_iters = iters;
    return HG_OK;
}

hg_status ensure_metrics(hg_plan p, int iters) {
    if (p->metrics_iters >= iters) return HG_OK;
    if (p->metrics) cudaFree(p->metrics);
    p->metrics = nullptr;
    p->metrics_iters = 0;
    HG_CK(cudaMalloc(&p->metrics, sizeof(double) * NMET * (size_t)iters * p->batch));
    p->metrics_iters = iters;
    return HG_OK;
}

RowArgs row_args(hg_plan p) {
    RowArgs a{};
    a.ny = p->ny;
    a.nx = p->nx;
    a.items = p->batch;
    a.nsub = 1;
    a.field = p->field;
    a.T = p->tf;
    a.w = p->w;
    a.seed_lo = (uint32_t)p->seed;
    a.seed_hi = (uint32_t)(p->seed >> 32);
    a.stream_id = 1;
    a.item0 = p->item0;
    a.tw = p->twx;
    const double N = (double)p->npx;
    a.invN = (float)(1.0 / N);
    a.invN2 = (float)(1.0 / (N * N));
    a.NN = (float)N;
    a.invSqrtN = (float)(1.0 / std::sqrt(N));
    a.lt_amp = 0.f;
    a.lt_hy = p->ny;
    a.lt_hx = p->nx;
    if (p->mod) {
        a.gen = 1;
        a.roi = p->roi_dft;
        a.lt_amp = (float)p->npx;  // target carrying the replay energy of a unit-modulus hologram
    }
    return a;
}

// Liu-Taghizadeh window of constraint j (0: the first field) into a.
void lt_set(hg_plan p, RowArgs &a, int j) {
    if (p->algo != HG_LT) return;
    const double f = std::min(1.0, (double)p->lt_start + (1.0 - (double)p->lt_start) * j / p->lt_grow);
    a.lt_amp = (float)p->npx;  // target scaled to the replay's energy (unnormalised transforms)
    a.lt_hy = (int)std::floor(f * p->ny / 2);
    a.lt_hx = (int)std::floor(f * p->nx / 2);
}

ColArgs col_args(hg_plan p) {
    ColArgs a{};
    a.ny = p->ny;
    a.nx = p->nx;
    a.items = p->batch;
    a.field = p->field;
    a.lvl = p->lvl;
    a.levels = p->levels;
    a.qscale = (float)((double)p->levels / 6.283185307179586476925286766559005768);
    a.tw = p->twy;
    a.invSqrtN = (float)(1.0 / std::sqrt((double)p->npx));
    a.illum = p->illum;
    a.kind = p->kind;
    // the column pass holds N times the unitary field of a target scaled by sqrt(N)
    a.amp_gain = (float)(1.0 / (2.0 * (double)p->amp_clip * (double)p->npx));
    return a;
}

int grid_for(int blocks_per_sm, int nsm, long work) {
    long g = (long)blocks_per_sm * nsm;
    if (g > work) g = work;
    return g < 1 ? 1 : (int)g;
}

void launch_row(hg_plan p, int role, const RowArgs &a, cudaStream_t s) {
    const long work = (long)a.items * p->ppt;
    p->rops->row(role, a, grid_for(p->rops->row_blocks_per_sm, p->nsm, work), s);
    p->launches++;
}

void launch_col(hg_plan p, int role, const ColArgs &a, cudaStream_t s) {
    const long work = (long)a.items * ((p->nx + p->cops->col_c - 1) / p->cops->col_c);
    p->cops->col(role, a, grid_for(p->cops->col_blocks_per_sm, p->nsm, work), s);
    p->launches++;
}

PipeArgs pipe_args(hg_plan p) {
    PipeArgs pa{};
    pa.err = p->err;
    pa.wait_ns = p->wait_ns;
    pa.drop_job = p->drop_job;
    return pa;
}

struct ProfScope {  // records an event pair around one pass launch when profiling
    hg_plan p;
    cudaStream_t s;
    size_t slot = (size_t)-1;
    ProfScope(hg_plan p_, cudaStream_t s_, int kind) : p(p_), s(s_) {
        if (p->prof_on && 2 * (p->prof_used + 1) <= p->prof_ev.size()) {
            slot = p->prof_used++;
            p->prof_kind[slot] = kind;
            cudaEventRecord(p->prof_ev[2 * slot], s);
        }
    }
    ~ProfScope() {
        if (slot != (size_t)-1) cudaEventRecord(p->prof_ev[2 * slot + 1], s);
    }
};

TcArgs tc_args(hg_plan p) {
    TcArgs t{};
    t.bmats = p->tc_b;
    t.err = p->err;
    t.wait_ns = p->wait_ns;
    return t;
}

void launch_row_tc(hg_plan p, int role, const RowArgs &a, cudaStream_t s) {
    tc_launch_row(p->tc_prec, role, a, tc_args(p), grid_for(p->tc_blocks, p->nsm, (long)a.items * p->ppt_tc), s);
    p->launches++;
}

void launch_row_iter(hg_plan p, const RowArgs &a, cudaStream_t s) {
    ProfScope ps(p, s, 0);
    if (p->tc_prec) {
        launch_row_tc(p, ROW_ITER, a, s);
    } else if (p->prow) {
        const long work = (long)a.items * p->ppt_pipe;
        p->prow->row_iter(a, pipe_args(p), grid_for(p->prow->row_blocks_per_sm, p->nsm, work), s);
        p->launches++;
    } else {
        launch_row(p, ROW_ITER, a, s);
    }
}

void launch_col_herm(hg_plan p, const ColArgs &a, cudaStream_t s) {
    ProfScope ps(p, s, 1);
    const PipeOps *h = p->hops;
    const long work = (long)a.items * ((p->nx + h->herm_c - 1) / h->herm_c);
    h->col_herm(a, pipe_args(p), p->cmap_herm, grid_for(h->herm_blocks_per_sm, p->nsm, work), s);
    p->launches++;
}

int col_blocks(const PipeOps *pc, int role) {
    return role == COL_GS_MOD ? pc->col_mod_blocks_per_sm : pc->col_blocks_per_sm;
}

void launch_col_gs(hg_plan p, int role, const ColArgs &a, cudaStream_t s) {
    ProfScope ps(p, s, 1);
    if (p->pcol) {
        const long work = (long)a.items * ((p->nx + p->pcol->col_c - 1) / p->pcol->col_c);
        p->pcol->col_gs(role, a, pipe_args(p), p->cmap, p->emap, grid_for(col_blocks(p->pcol, role), p->nsm, work),
                        s);
        p->launches++;
    } else {
        launch_col(p, role, a, s);
    }
}

int ew_grid(hg_plan p, size_t n) {
    size_t g = (n + 255) / 256;
    size_t cap = (size_t)p->nsm * 8;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// Target preparation (normalise to sum T^2 = 1, move to DFT order).
void enqueue_prep(hg_plan p, const float *target) {
    dim3 g(PREP_BLOCKS, p->batch);
    k_prep_sum<<<g, PREP_THREADS, 0, p->stream>>>(target, (int)p->npx, p->roi_rep, p->sum_part, p->err);
    k_prep_scale<<<(p->batch + 127) / 128, 128, 0, p->stream>>>(p->sum_part, p->batch, p->scale,
                                                                 p->err);
    k_prep_apply<<<(unsigned)(p->ny * p->batch), 256, 0, p->stream>>>(target, p->ny, p->nx, p->batch, p->scale,
                                                                      p->roi_rep, p->tf);
    p->launches += 3;
}

int col_role_gs(hg_plan p) {
    return p->mod ? COL_GS_MOD : p->kind == HG_SLM_BINARY ? COL_GS_BIN : COL_GS_LVL;
}
int col_role_holo(hg_plan p) {
    return p->mod ? COL_HOLO_MOD : p->kind == HG_SLM_BINARY ? COL_HOLO_BIN : COL_HOLO_LVL;
}

bool is_ospr(int algo) { return algo == HG_OSPR || algo == HG_ADOSPR; }
bool is_search(int algo) { return algo == HG_DS || algo == HG_SA; }

// Binary GS with the paired row pass and a TMA-fed column pass: the row pass
// writes only the Hermitian part of F (rows ky <= ny/2) and the next column
// pass reads those rows back (see herm_constrain).
bool herm_loop(hg_plan p) {
    return p->prow && p->prow->paired && p->pcol && p->kind == HG_SLM_BINARY;
}

// The Hermitian binary loop also starts and ends in Hermitian form: the head
// writes rows ky <= ny/2 of F_H, and the tail reads rows ky <= ny/2 of the
// last column pass (both on the paired row kernel).
bool herm_ends(hg_plan p) { return herm_loop(p) && p->prow->row_head && p->prow->row_tail; }

// Binary OSPR in Hermitian form: head and time average on the paired row
// kernel of the variant that provides the column-pair pass.
bool ospr_pair_ends(hg_plan p) { return p->ospr_herm && p->hops->row_head && p->hops->row_avg; }
bool adospr_pair(hg_plan p) { return p->algo == HG_ADOSPR && ospr_pair_ends(p) && p->hops->row_adapt; }

void launch_adapt(hg_plan p, const RowArgs &a, bool last, cudaStream_t s) {
    const long work = (long)a.items * (p->ny / 2 + 1);
    p->hops->row_adapt(a, pipe_args(p), grid_for(p->hops->row_blocks_per_sm, p->nsm, work), s, last);
    p->launches++;
}

void launch_ospr_end(hg_plan p, bool head, const RowArgs &a, cudaStream_t s) {
    const long work = (long)a.items * (p->ny / 2 + 1);
    const int grid = grid_for(p->hops->row_blocks_per_sm, p->nsm, work);
    if (head) p->hops->row_head(a, pipe_args(p), grid, s);
    else p->hops->row_avg(a, pipe_args(p), grid, s);
    p->launches++;
}

void launch_pair_end(hg_plan p, bool head, const RowArgs &a, cudaStream_t s) {
    const long work = (long)a.items * p->ppt_pipe;
    const int grid = grid_for(p->prow->row_blocks_per_sm, p->nsm, work);
    if (head) p->prow->row_head(a, pipe_args(p), grid, s);
    else p->prow->row_tail(a, pipe_args(p), grid, s);
    p->launches++;
}

// The middle of a GS run: for k = 0 .. iters-2, column pass k then row pass
// k (metrics of iteration k, constraint for iteration k+1).
void enqueue_loop(hg_plan p, int iters, cudaStream_t s) {
    ColArgs ca = col_args(p);
    RowArgs ra = row_args(p);
    ca.half = p->prow && p->prow->paired;  // the paired row pass rebuilds rows ny - ky
    ra.herm = herm_loop(p);
    const bool half_head = herm_ends(p);
    for (int k = 0; k + 1 < iters; ++k) {
        ca.half_in = ra.herm && (k > 0 || half_head);  // after a full head, column pass 0 reads every row
        if (ca.half_in && p->use_herm_col) launch_col_herm(p, ca, s);
        else launch_col_gs(p, col_role_gs(p), ca, s);
        ra.part = p->part + (size_t)k * p->batch * p->ppt_max * part_stride(p);
        lt_set(p, ra, k + 1);
        launch_row_iter(p, ra, s);
    }
}

hg_status run_loop(hg_plan p, int iters) {
    if (iters <= 1) return HG_OK;
    if (!p->use_graph || p->prof_on) {
        enqueue_loop(p, iters, p->stream);
        return map_err(cudaGetLastError());
    }
    if (!p->gexec || p->g_iters != iters || p->g_part != p->part) {
        if (p->gexec) cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
        cudaGraph_t g = nullptr;
        HG_CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int before = p->launches;
        enqueue_loop(p, iters, p->cap_stream);
        p->launches = before;
        cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
        if (e != cudaSuccess) return map_err(e);
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            return map_err(e);
        }
        p->g_iters = iters;
        p->g_part = p->part;
    }
    HG_CK(cudaGraphLaunch(p->gexec, p->stream));
    p->launches += 2 * (iters - 1);
    return HG_OK;
}

// The device-side work of one run (buffers already device-resident, partial
// and metric buffers already sized).  `capturing`: enqueued inside an outer
// stream capture, so the loop is enqueued pass by pass and WGS weights always
// restart at 1.
hg_status enqueue_run(hg_plan p, const float *d_t, const float *d_ph, int iters, uint8_t *d_ho,
                      double *d_mo, bool capturing) {
    hg_status st = HG_OK;
    HG_CK(cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream));
    enqueue_prep(p, d_t);

    RowArgs ra = row_args(p);
    ColArgs ca = col_args(p);
    if (p->algo == HG_ADOSPR) {
        HG_CK(cudaMemsetAsync(p->acc, 0, sizeof(float) * p->npx * p->batch, p->stream));
        ra.items = p->batch;
        ra.nsub = 1;  // the head draws subframe 0 of target `item`
        ra.phase = nullptr;
        ra.stream_id = 0;
        // Hermitian form: the running intensity sum is symmetric, rows ky <= ny/2 suffice
        const bool hm = adospr_pair(p);
        if (hm) launch_ospr_end(p, true, ra, p->stream);
        else launch_row(p, ROW_HEAD, ra, p->stream);
        ca.items = p->batch;
        ca.half_in = ca.half = hm;
        RowArgs rn = row_args(p);
        rn.acc = p->acc;
        rn.stream_id = 0;
        rn.nsub = p->nsub;
        for (int n = 0; n < p->nsub; ++n) {
            ca.holo = d_ho ? p->holo_tmp : nullptr;
            if (hm) launch_col_herm(p, ca, p->stream);
            else launch_col_gs(p, COL_GS_BIN, ca, p->stream);
            if (d_ho)  // subframe n of each target: [batch][subframes][ny][nx]
                HG_CK(cudaMemcpy2DAsync(d_ho + (size_t)n * p->npx, p->npx * p->nsub, p->holo_tmp, p->npx, p->npx,
                                        p->batch, cudaMemcpyDeviceToDevice, p->stream));
            rn.sub = n + 1;
            if (n + 1 < p->nsub) {
                if (hm) launch_adapt(p, rn, false, p->stream);
                else launch_row(p, ROW_ADAPT, rn, p->stream);
            } else {
                rn.part = p->part;
                if (hm) launch_adapt(p, rn, true, p->stream);
                else launch_row(p, ROW_ADFIN, rn, p->stream);
            }
        }
    } else if (p->algo == HG_OSPR) {
        ra.items = p->nchains;
        ra.nsub = p->nsub;
        ra.phase = nullptr;
        ra.stream_id = 0;
        ra.herm = p->ospr_herm;
        if (ospr_pair_ends(p)) launch_ospr_end(p, true, ra, p->stream);
        else launch_row(p, ROW_HEAD, ra, p->stream);
        ca.items = p->nchains;
        ca.holo = d_ho;
        if (p->ospr_herm) {
            ca.half_in = ca.half = 1;
            launch_col_herm(p, ca, p->stream);
        } else {
            launch_col_gs(p, COL_GS_BIN, ca, p->stream);
        }
        RowArgs rt = row_args(p);
        rt.nsub = p->nsub;
        rt.part = p->part;
        rt.herm = p->ospr_herm;
        if (ospr_pair_ends(p)) launch_ospr_end(p, false, rt, p->stream);
        else launch_row(p, ROW_AVG, rt, p->stream);
    } else if (is_search(p->algo)) {
        // initial guess: the quantised back-propagation of the target (head + column
        // pass), its replay field (tail), then the sweeps in one kernel
        ra.phase = d_ph;
        launch_row(p, ROW_HEAD, ra, p->stream);
        uint8_t *hb = d_ho ? d_ho : p->sholo;
        ca.holo = hb;
        launch_col(p, col_role_gs(p), ca, p->stream);
        RowArgs rt = row_args(p);
        rt.w = nullptr;
        rt.R_out = p->rbuf;
        launch_row(p, ROW_TAIL, rt, p->stream);
        SearchArgs sa{};
        sa.ny = p->ny;
        sa.nx = p->nx;
        sa.items = p->batch;
        sa.R0 = p->rbuf;
        sa.T = p->tf;
        sa.holo = hb;
        sa.lvl = p->lvl;
        sa.levels = p->levels;
        sa.binary = p->kind == HG_SLM_BINARY;
        sa.twx = p->twx;
        sa.twy = p->twy;
        sa.sweeps = iters;
        sa.tau0 = p->algo == HG_SA ? p->sa_temp : 0.0;
        sa.alpha = p->sa_cool;
        sa.seed_lo = (uint32_t)p->seed;
        sa.seed_hi = (uint32_t)(p->seed >> 32);
        sa.metrics = p->metrics;
        sa.mse_out = d_mo;
        sa.invN = (float)(1.0 / (double)p->npx);
        sa.invSqrtN = (float)(1.0 / std::sqrt((double)p->npx));
        sa.per_thread = p->slay.per_thread;
        sa.off_twy = (unsigned)p->slay.off_twy;
        sa.off_R = (unsigned)p->slay.off_R;
        sa.off_T = (unsigned)p->slay.off_T;
        sa.off_red = (unsigned)p->slay.off_red;
        sa.off_dred = (unsigned)p->slay.off_dred;
        sa.off_rnd = (unsigned)p->slay.off_rnd;
        sa.off_holo = (unsigned)p->slay.off_holo;
        HG_CK(search_launch(sa, p->slay, p->stream));
        p->launches++;
    } else {
        if (p->algo == HG_WGS && (!p->weights_preset || capturing)) {
            k_fill<<<ew_grid(p, p->npx * p->batch), 256, 0, p->stream>>>(p->w, p->npx * p->batch, 1.f);
            p->launches++;
        }
        ra.phase = d_ph;
        lt_set(p, ra, 0);
        const bool ends = herm_ends(p);
        if (ends) {
            ra.herm = 1;
            launch_pair_end(p, true, ra, p->stream);
        } else {
            launch_row(p, ROW_HEAD, ra, p->stream);
        }
        if (capturing) {
            enqueue_loop(p, iters, p->stream);
        } else if ((st = run_loop(p, iters)) != HG_OK) {
            return st;
        }
        ca.holo = d_ho;
        ca.half_in = herm_loop(p) && (iters >= 2 || ends);
        ca.half = ends;  // the Hermitian tail reads rows ky <= ny/2 only
        if (ca.half_in && p->use_herm_col) launch_col_herm(p, ca, p->stream);
        else launch_col_gs(p, col_role_gs(p), ca, p->stream);
        RowArgs rt = row_args(p);
        rt.part = p->part + (size_t)(iters - 1) * p->batch * p->ppt_max * part_stride(p);
        if (p->tc_prec) launch_row_tc(p, ROW_TAIL, rt, p->stream);
        else if (ends) launch_pair_end(p, false, rt, p->stream);
        else launch_row(p, ROW_TAIL, rt, p->stream);
    }
    const int panels_iter = p->tc_prec ? p->ppt_tc : p->prow ? p->ppt_pipe : p->ppt;
    int panels_last = (p->tc_prec && !is_ospr(p->algo)) ? p->ppt_tc : p->ppt;
    if (!is_ospr(p->algo) && !is_search(p->algo) && herm_ends(p)) panels_last = p->ppt_pipe;  // Hermitian tail
    if (p->ospr_herm) panels_last = (p->ny / 2 + p->rops->row_lines) / p->rops->row_lines;  // rows <= ny/2
    if (is_ospr(p->algo) && ospr_pair_ends(p)) panels_last = p->ny / 2 + 1;  // one panel per row
    if (is_search(p->algo)) {
        // the search kernel wrote the metrics and mse_out itself
    } else if (p->mod) {
        k_reduce_gen<<<(iters * p->batch * 32 + 127) / 128, 128, 0, p->stream>>>(
            p->part, iters, p->batch, p->ppt_max, panels_iter, panels_last, p->nroi, p->metrics, d_mo);
        p->launches++;
    } else {
        k_reduce<<<(iters * p->batch * 32 + 127) / 128, 128, 0, p->stream>>>(
            p->part, iters, p->batch, p->ppt_max, panels_iter, panels_last, 1.0 / (double)p->npx, p->metrics,
            d_mo);
        p->launches++;
    }
    HG_CK(cudaGetLastError());
    p->weights_preset = false;
    p->have_run = true;
    p->field_from_run = !is_ospr(p->algo) && !is_search(p->algo);
    p->last_iters = iters;
    return st;
}

hg_status check_err_flag(hg_plan p) {
    unsigned e = 0;
    HG_CK(cudaMemcpyAsync(&e, p->err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream));
    HG_CK(cudaStreamSynchronize(p->stream));
    if (e & ERR_BAD_VALUE) return HG_ERR_INVALID_ARG;
    if (e & ERR_ZERO_ENERGY) return HG_ERR_NUMERIC;
    if (e & ERR_TIMEOUT_BIT) return HG_ERR_TIMEOUT;
    return HG_OK;
}

bool make_cmap_box(hg_plan p, int cols, int boxr, CUtensorMap *m) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || cols < 1 || boxr < 1) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)2 * p->nx, (cuuint64_t)p->ny * p->nchains};
    const cuuint64_t gstride[1] = {(cuuint64_t)p->nx * 8};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * cols), (cuuint32_t)boxr};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->field, gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_cmap(hg_plan p, const PipeOps *pc, CUtensorMap *m) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)2 * p->nx, (cuuint64_t)p->ny * p->nchains};
    const cuuint64_t gstride[1] = {(cuuint64_t)p->nx * 8};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * pc->col_c), (cuuint32_t)pc->col_boxr};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->field, gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The column pass's tensor maps: the field, and for a modulated plan whose
// variant stages E in shared memory, the illumination with the same boxes
// (otherwise em repeats m, unused).
bool make_col_maps(hg_plan p, const PipeOps *pc, CUtensorMap *m, CUtensorMap *em) {
    if (!make_cmap(p, pc, m)) return false;
    *em = *m;
    if (!(p->mod && pc->col_emap)) return true;
    EncodeTiledFn enc = encode_tiled();
    if (!enc || !p->illum) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)2 * p->nx, (cuuint64_t)p->ny};
    const cuuint64_t gstride[1] = {(cuuint64_t)p->nx * 8};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * pc->col_c), (cuuint32_t)pc->col_boxr};
    const cuuint32_t estr[2] = {1, 1};
    return enc(em, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->illum, gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Best-of-3 launch time (ms, after one warm-up launch) of one pass variant on
// the plan's own zeroed buffers, on the private capture stream.
float time_variant(hg_plan p, const PipeOps *o, bool row, bool herm = false, bool herm_pairs = false) {
    if (!p->field || !p->tf || !p->twx || !p->twy || !p->lvl || !p->err) return 1e30f;
    cudaStream_t s = p->cap_stream;
    RowArgs ra = row_args(p);
    ra.w = nullptr;
    ra.part = nullptr;
    ra.herm = herm;
    ColArgs ca = col_args(p);
    CUtensorMap m, em;
    if (herm_pairs) {
        if (!o->col_herm || !make_cmap_box(p, o->herm_c, o->herm_boxr, &m)) return 1e30f;
    } else if (!row && !make_col_maps(p, o, &m, &em)) {
        return 1e30f;
    }
    const int role = p->mod ? COL_GS_MOD : p->kind == HG_SLM_BINARY ? COL_GS_BIN : COL_GS_LVL;
    if (!row && herm) ca.half = ca.half_in = 1;
    const int ppt = row ? row_panels(o, p->ny) : (p->nx + (herm_pairs ? o->herm_c : o->col_c) - 1) /
                                                     (herm_pairs ? o->herm_c : o->col_c);
    const int grid = grid_for(row ? o->row_blocks_per_sm
                                  : herm_pairs ? o->herm_blocks_per_sm : col_blocks(o, role),
                              p->nsm, (long)p->batch * ppt);
    PipeArgs pa = pipe_args(p);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 1e30f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 1e30f;
    }
    // 2 warm-up launches, then the median of 5 timed ones
    float t[5];
    int n = 0;
    for (int it = 0; it < 7; ++it) {
        cudaEventRecord(e0, s);
        if (row) o->row_iter(ra, pa, grid, s);
        else if (herm_pairs) o->col_herm(ca, pa, m, grid, s);
        else o->col_gs(role, ca, pa, m, em, grid, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (it >= 2) t[n++] = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || n < 5) return 1e30f;
    for (int i = 1; i < n; ++i)  // insertion sort of 5 values
        for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
            const float x = t[j];
            t[j] = t[j - 1];
            t[j - 1] = x;
        }
    return t[n / 2];
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Chunks of a run with host buffers: 1 (the whole batch at once) for OSPR,
// search, profiled plans and single targets; else opts.host_chunks, or (0)
// up to 4 while every chunk keeps at least 2^23 pixels, so that each pass
// still fills the GPU.
// Time of a chunk schedule under the plan's measured model: chunk k's inputs
// are copied after chunk k - 1's on one stream, its iterations start when
// both its inputs and chunk k - 1's iterations are done, and the last
// chunk's outputs are copied after its iterations.
double chunk_schedule_ms(hg_plan p, const std::vector<int> &st) {
    double copied = 0, done = 0;
    for (size_t k = 0; k + 1 < st.size(); ++k) {
        const int n = st[k + 1] - st[k];
        copied += n * p->x_in;
        done = std::max(done, copied) + n * p->x_it + p->x_fix;
    }
    return done + (st.size() > 1 ? (st[st.size() - 1] - st[st.size() - 2]) * p->x_out : 0.0);
}

// First target of each chunk of an hg_run with host buffers, then the batch
// size (one chunk: {0, batch}).  hg_opts.host_chunks = K > 0 splits the batch
// evenly.  The default (0), for batches of 2^24 pixels and more: the first
// call with a given iteration count runs a short lead chunk and one chunk for
// the rest.  Only the lead's input copy and the rest's output copy are then
// exposed, and the rest's input copy is hidden while the lead iterates if
//   lead * iters * c_iter >= (batch - lead) * c_in,
// where c_in / c_iter, one target's input copy over one of its iterations,
// is about 8 B/px at ~200 GB/s over 36 B/px at ~6 TB/s, i.e. r = 8 / iters.
// That call times its copies and its two chunks' iterations (per target, and
// the fixed cost of a chunk: launch tails of fewer targets, head and tail
// passes); later calls with the same iteration count take the schedule
// that this model says is fastest: a lead of n0 targets, then each next chunk
// either the rest (if waiting for its copy costs less than another chunk's
// fixed cost) or as many targets as are copied by the time the chunk before
// it finishes.  With fast host copies that is the two-chunk schedule; with
// slow ones a growing sequence of chunks.  (Measured at 1024^2 x 64 x 50
// iterations with pinned buffers, even chunks: 1 -> 21.92 ms, 2 -> 21.65,
// 4 -> 21.90, 8 -> 22.10; device buffers 19.02; lead of 9 then 55: 20.3.)
// Small batches (under 2^24 pixels) run as one chunk.
std::vector<int> host_chunk_starts(hg_plan p, int iters) {
    std::vector<int> st{0};
    const int B = p->batch;
    const bool one = is_ospr(p->algo) || is_search(p->algo) || p->prof_on || B < 2;
    if (!one && p->host_chunks > 0) {
        const int K = std::min(p->host_chunks, B), cs = (B + K - 1) / K;
        for (int b = cs; b < B; b += cs) st.push_back(b);
    } else if (!one && (long long)p->npx * B >= (1ll << 24)) {
        if (p->x_iters == iters && p->x_it > 0) {
            // chunks of at least 2^23 pixels, so that each still fills the GPU
            // (the model's cost per target holds for chunks of that size)
            const long long px_min = ((1ll << 23) + p->npx - 1) / p->npx;
            const int nmin = (int)std::min<long long>(B / 2, std::max<long long>(1, px_min));
            std::vector<int> best{0, B}, cand;
            double best_ms = chunk_schedule_ms(p, best);
            const int step = std::max(1, B / 256);
            for (int n0 = nmin; n0 <= B - nmin; n0 += step) {
                cand.assign({0, n0});
                double done = p->x_in * n0 + p->x_it * n0 + p->x_fix;
                int S = n0;
                while (S < B) {
                    int n = B - S;
                    if (p->x_in > 0 && B * p->x_in - done > p->x_fix)
                        n = std::min(n, std::max(nmin, (int)std::floor(done / p->x_in) - S));
                    if (B - S - n < nmin) n = B - S;
                    done = std::max(done, (S + n) * p->x_in) + n * p->x_it + p->x_fix;
                    S += n;
                    cand.push_back(S);
                }
                const double ms = chunk_schedule_ms(p, cand);
                if (ms < best_ms) best_ms = ms, best = cand;
            }
            return best;
        }
        const double r = 8.0 / std::max(iters, 1);
        const int lead = (int)std::ceil(B * r / (1.0 + r));
        if (lead < B) st.push_back(std::max(lead, 1));
    }
    st.push_back(B);
    return st;
}

// A view of targets [first, first + count) of p: p's passes, tensor-map boxes
// and settings on pointers into p's per-target buffers (field, prepared
// targets, weights, prep partials, scales).  Its metric partials and metrics
// are pointed into p's before each run; it owns only its loop graph.
hg_status make_view(hg_plan p, int first, int count, hg_plan *out) {
    hg_plan_s *v = new (std::nothrow) hg_plan_s(*p);
    if (!v) return HG_ERR_OOM;
    v->is_view = true;
    v->item0 = p->item0 + first;
    v->views.clear();
    v->chunk_ev.clear();
    v->x_ev.clear();
    v->prof_ev.clear();
    v->prof_kind.clear();
    v->prof_on = false;
    v->prof_used = 0;
    v->h2d_stream = v->d2h_stream = nullptr;
    v->batch = v->nchains = count;
    const size_t off = (size_t)first * p->npx;
    v->field = p->field + off;
    v->tf = p->tf + off;
    v->w = p->w ? p->w + off : nullptr;
    v->sum_part = p->sum_part + (size_t)first * PREP_BLOCKS;
    v->scale = p->scale + first;
    v->part = nullptr;
    v->part_iters = 0;
    v->metrics = nullptr;
    v->metrics_iters = 0;
    v->stage = nullptr;
    v->stage_bytes = 0;
    v->gexec = nullptr;
    v->g_iters = -1;
    v->g_part = nullptr;
    v->ev_part = nullptr;
    v->ev_buf = nullptr;
    v->rbuf = nullptr;
    v->sholo = nullptr;
    v->acc = nullptr;
    v->holo_tmp = nullptr;
    v->launches = 0;
    bool ok = true;
    if (v->pcol) ok = make_col_maps(v, v->pcol, &v->cmap, &v->emap);
    if (ok && v->use_herm_col && v->hops) ok = make_cmap_box(v, v->hops->herm_c, v->hops->herm_boxr, &v->cmap_herm);
    if (!ok) {
        delete v;
        return HG_ERR_CUDA;
    }
    *out = v;
    return HG_OK;
}

// hg_run with host buffers in K chunks: chunk c's inputs are copied on the
// H2D stream while chunk c - 1 iterates on the plan's stream, and its outputs
// are copied back on the D2H stream while chunk c + 1 iterates.  Every chunk
// runs the same kernels on its targets as a whole-batch run, so holograms,
// MSE and metrics are identical.  d_* point into the staging buffer (host
// sides) or at the caller's device buffers.
hg_status run_chunked(hg_plan p, const std::vector<int> &cst, const float *target, const float *d_t,
                      const float *init_phase, const float *d_ph, int iters, uint8_t *holo_out, uint8_t *d_ho,
                      double *mse_out, double *d_mo) {
    const int K = (int)cst.size() - 1;
    hg_status st;
    bool same = (int)p->views.size() == K;
    for (int c = 0; same && c < K; ++c)
        same = p->views[c]->item0 == p->item0 + cst[c] && p->views[c]->batch == cst[c + 1] - cst[c];
    if (!same) {
        for (hg_plan v : p->views) hg_plan_destroy(v);
        p->views.clear();
        for (int c = 0; c < K; ++c) {
            hg_plan v = nullptr;
            if ((st = make_view(p, cst[c], cst[c + 1] - cst[c], &v)) != HG_OK) return st;
            p->views.push_back(v);
        }
    }
    for (cudaStream_t *cs_ : {&p->h2d_stream, &p->d2h_stream})
        if (!*cs_) HG_CK(cudaStreamCreateWithFlags(cs_, cudaStreamNonBlocking));
    while ((int)p->chunk_ev.size() < 2 * K + 1) {
        cudaEvent_t e;
        HG_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->chunk_ev.push_back(e);
    }
    cudaEvent_t *ev_in = p->chunk_ev.data(), *ev_done = ev_in + K, ev_start = ev_in[2 * K];
    // the default schedule's first call with this iteration count times its
    // copies and chunks: input copies, then per chunk its iterations and its
    // output copies
    const bool measure = p->host_chunks == 0 && p->x_iters != iters;
    while (measure && (int)p->x_ev.size() < 2 + 4 * K) {
        cudaEvent_t e;
        HG_CK(cudaEventCreate(&e));
        p->x_ev.push_back(e);
    }
    cudaEvent_t *xe = measure ? p->x_ev.data() : nullptr;
    // the copies follow whatever the plan's stream already holds
    HG_CK(cudaEventRecord(ev_start, p->stream));
    HG_CK(cudaStreamWaitEvent(p->h2d_stream, ev_start, 0));
    HG_CK(cudaStreamWaitEvent(p->d2h_stream, ev_start, 0));
    if (measure) HG_CK(cudaEventRecord(xe[0], p->h2d_stream));
    const size_t npx = p->npx;
    for (int c = 0; c < K; ++c) {
        const size_t b0 = (size_t)cst[c], nb = p->views[c]->batch;
        if (d_t != target)
            HG_CK(cudaMemcpyAsync((void *)(d_t + b0 * npx), target + b0 * npx, sizeof(float) * nb * npx,
                                  cudaMemcpyHostToDevice, p->h2d_stream));
        if (d_ph && d_ph != init_phase)
            HG_CK(cudaMemcpyAsync((void *)(d_ph + b0 * npx), init_phase + b0 * npx, sizeof(float) * nb * npx,
                                  cudaMemcpyHostToDevice, p->h2d_stream));
        HG_CK(cudaEventRecord(ev_in[c], p->h2d_stream));
    }
    if (measure) HG_CK(cudaEventRecord(xe[1], p->h2d_stream));
    int launches = 0;
    for (int c = 0; c < K; ++c) {
        hg_plan v = p->views[c];
        const size_t b0 = (size_t)cst[c], nb = v->batch;
        v->part = p->part;  // the chunks run one after another on the plan's stream
        v->part_iters = p->part_iters;
        v->metrics = p->metrics + b0 * iters * NMET;
        v->metrics_iters = iters;
        v->weights_preset = p->weights_preset;
        v->wait_ns = p->wait_ns;
        v->drop_job = p->drop_job;
        HG_CK(cudaStreamWaitEvent(p->stream, ev_in[c], 0));
        if (measure) HG_CK(cudaEventRecord(xe[2 + 4 * c], p->stream));
        v->launches = 0;
        if ((st = enqueue_run(v, d_t + b0 * npx, d_ph ? d_ph + b0 * npx : nullptr, iters,
                              d_ho ? d_ho + b0 * npx : nullptr, d_mo ? d_mo + b0 * iters : nullptr, false)) != HG_OK)
            return st;
        launches += v->launches;
        HG_CK(cudaEventRecord(ev_done[c], p->stream));
        if (measure) HG_CK(cudaEventRecord(xe[3 + 4 * c], p->stream));
        HG_CK(cudaStreamWaitEvent(p->d2h_stream, ev_done[c], 0));
        if (measure) HG_CK(cudaEventRecord(xe[4 + 4 * c], p->d2h_stream));
        if (d_ho && d_ho != holo_out)
            HG_CK(cudaMemcpyAsync(holo_out + b0 * npx, d_ho + b0 * npx, nb * npx, cudaMemcpyDeviceToHost,
                                  p->d2h_stream));
        if (d_mo && d_mo != mse_out)
            HG_CK(cudaMemcpyAsync(mse_out + b0 * iters, d_mo + b0 * iters, sizeof(double) * nb * iters,
                                  cudaMemcpyDeviceToHost, p->d2h_stream));
        if (measure) HG_CK(cudaEventRecord(xe[5 + 4 * c], p->d2h_stream));
    }
    p->launches = launches;
    p->weights_preset = false;
    p->have_run = true;
    p->field_from_run = true;
    p->last_iters = iters;
    HG_CK(cudaStreamSynchronize(p->d2h_stream));
    hg_status sst = hg_sync(p);
    if (measure && sst == HG_OK) {
        // per-target copy and iteration times; the fixed cost of a chunk from
        // the two chunk sizes (iteration time = n x_it + x_fix)
        float ms = 0;
        double in_ms = 0, out_ms = 0, n[2] = {0, 0}, it_ms[2] = {0, 0};
        HG_CK(cudaEventElapsedTime(&ms, xe[0], xe[1]));
        in_ms = ms;
        for (int c = 0; c < K; ++c) {
            HG_CK(cudaEventElapsedTime(&ms, xe[2 + 4 * c], xe[3 + 4 * c]));
            const int i = c == 0 ? 0 : 1;
            n[i] += cst[c + 1] - cst[c];
            it_ms[i] += ms;
            HG_CK(cudaEventElapsedTime(&ms, xe[4 + 4 * c], xe[5 + 4 * c]));
            out_ms += ms;
        }
        const double B = p->batch;
        p->x_in = in_ms / B;
        p->x_out = out_ms / B;
        double it = (it_ms[0] + it_ms[1]) / B, fix = 0;
        if (K == 2 && n[0] != n[1]) {
            it = (it_ms[1] - it_ms[0]) / (n[1] - n[0]);
            fix = it_ms[0] - n[0] * it;
            if (it <= 0 || fix < 0) it = (it_ms[0] + it_ms[1]) / B, fix = 0;
        }
        p->x_it = it;
        p->x_fix = fix;
        p->x_iters = iters;
    }
    return sst;
}

}  // namespace

// ------------------------------------------------------------------- ABI

extern "C" {

void hg_opts_default(hg_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->subframes = 24;
    o->use_graph = 1;
    o->pipeline = -1;
    o->autotune = 1;
    o->lt_start = 0.25f;
    o->lt_grow = 10;
    o->modulated = 0;
    o->fresnel = 0.f;
    o->amp_clip = 2.f;
    o->sa_temp = 1e-3f;
    o->sa_cool = 0.9f;
    o->host_chunks = 0;
}

int hg_supported_length(int n) { return find_ops(n) != nullptr; }

const char *hg_status_string(hg_status st) {
    switch (st) {
        case HG_OK: return "ok";
        case HG_ERR_INVALID_ARG: return "invalid argument";
        case HG_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case HG_ERR_OOM: return "out of device memory";
        case HG_ERR_CUDA: return "CUDA error";
        case HG_ERR_TIMEOUT: return "device wait timed out";
        case HG_ERR_NUMERIC: return "target has zero energy";
        case HG_ERR_TOO_LARGE: return "side exceeds the fixed work memory of hg_run_noalloc";
        default: return "unknown status";
    }
}

void hg_plan_destroy(hg_plan p) {
    if (!p) return;
    DevGuard g(p->dev);
    if (p->stream || p->cap_stream) cudaStreamSynchronize(p->stream);
    if (p->is_view) {  // owns its loop graph only
        if (p->gexec) cudaGraphExecDestroy(p->gexec);
        delete p;
        return;
    }
    for (hg_plan v : p->views) hg_plan_destroy(v);
    for (cudaStream_t cs : {p->h2d_stream, p->d2h_stream})
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
    for (cudaEvent_t e : p->chunk_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : p->x_ev) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    void *bufs[] = {p->field, p->tf, p->w, p->part, p->metrics, p->sum_part, p->scale,
                    p->err, p->twx, p->twy, p->lvl, p->stage, p->tc_b, p->acc, p->holo_tmp,
                    p->illum, p->roi_rep, p->roi_dft, p->nroi, p->ev_part, p->ev_buf, p->rbuf, p->sholo};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p;
}

hg_status hg_plan_create(hg_plan *out, int ny, int nx, int batch, hg_slm slm, hg_algo algo,
                         const hg_opts *opts) {
    if (!out) return HG_ERR_INVALID_ARG;
    *out = nullptr;
    hg_opts o;
    hg_opts_default(&o);
    if (opts) o = *opts;
    if (batch < 1 || ny < 1 || nx < 1 || o.host_chunks < 0) return HG_ERR_INVALID_ARG;
    if (algo != HG_GS && algo != HG_WGS && algo != HG_OSPR && algo != HG_ADOSPR && algo != HG_LT &&
        algo != HG_DS && algo != HG_SA)
        return HG_ERR_INVALID_ARG;
    if (algo == HG_LT && (!(o.lt_start > 0.f) || o.lt_start > 1.f || o.lt_grow < 1)) return HG_ERR_INVALID_ARG;
    if (slm.kind != HG_SLM_BINARY && slm.kind != HG_SLM_LLEVEL && slm.kind != HG_SLM_AMPLITUDE)
        return HG_ERR_INVALID_ARG;
    if (slm.kind != HG_SLM_BINARY && (slm.levels < 2 || slm.levels > 256)) return HG_ERR_INVALID_ARG;
    const bool mod = o.modulated || slm.kind == HG_SLM_AMPLITUDE || o.fresnel != 0.f;
    if (mod && (algo != HG_GS || o.precision != 0 || !std::isfinite(o.fresnel) ||
                !(o.amp_clip > 0.f) || !std::isfinite(o.amp_clip)))
        return HG_ERR_INVALID_ARG;
    const bool search = algo == HG_DS || algo == HG_SA;
    SearchLayout slay{};
    if (search) {
        if (o.precision != 0 || o.pipeline == 1) return HG_ERR_INVALID_ARG;
        if (algo == HG_SA && (!(o.sa_temp > 0.f) || !std::isfinite(o.sa_temp) || !(o.sa_cool > 0.f) ||
                              o.sa_cool > 1.f))
            return HG_ERR_INVALID_ARG;
        if (!search_layout(ny, nx, &slay)) return HG_ERR_UNSUPPORTED_SIZE;
    }
    if (is_ospr(algo) && (slm.kind != HG_SLM_BINARY || o.subframes < 1)) return HG_ERR_INVALID_ARG;
    if (o.precision < 0 || o.precision > 4) return HG_ERR_INVALID_ARG;
    if (o.precision > 0 && ((nx != 1024 && nx != 2048) || ny % (nx == 1024 ? 4 : 2) != 0 || is_ospr(algo) || algo == HG_LT))
        return HG_ERR_UNSUPPORTED_SIZE;
    const LineOps *rops = find_ops(nx), *cops = find_ops(ny);
    if (!rops || !cops) return HG_ERR_UNSUPPORTED_SIZE;
    const size_t npx = (size_t)ny * nx;
    const int nsub = is_ospr(algo) ? o.subframes : 1;
    if ((double)npx * batch * nsub > 2.0e9 || (double)batch * nsub > 1e6)
        return HG_ERR_INVALID_ARG;

    hg_plan p = new (std::nothrow) hg_plan_s();
    if (!p) return HG_ERR_OOM;
    if (cudaGetDevice(&p->dev) != cudaSuccess) {
        delete p;
        return HG_ERR_CUDA;
    }
    p->ny = ny;
    p->nx = nx;
    p->batch = batch;
    p->algo = algo;
    p->kind = slm.kind;
    p->levels = slm.kind == HG_SLM_BINARY ? 2 : slm.levels;
    p->mod = mod;
    p->slay = slay;
    if (algo == HG_SA) {
        p->sa_temp = o.sa_temp;
        p->sa_cool = o.sa_cool;
    }
    p->fresnel = o.fresnel;
    p->host_chunks = o.host_chunks;
    p->amp_clip = o.amp_clip;

    p->nsub = nsub;
    p->nchains = batch * nsub;
    p->seed = o.seed;
    if (algo == HG_LT) {
        p->lt_start = o.lt_start;
        p->lt_grow = o.lt_grow;
    }
    p->stream = (cudaStream_t)o.stream;
    p->use_graph = o.use_graph ? 1 : 0;
    p->rops = rops;
    p->cops = cops;
    p->npx = npx;
    p->ppt = (ny + rops->row_lines - 1) / rops->row_lines;
    p->ppt_max = p->ppt;

    hg_status st = HG_OK;
    auto fail = [&](hg_status s) {
        hg_plan_destroy(p);
        return s;
    };
    cudaError_t ce = ensure_init(p->dev, rops);
    if (ce == cudaSuccess) ce = ensure_init(p->dev, cops);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return fail(map_err(ce));
    ce = cudaMalloc(&p->field, sizeof(float2) * npx * p->nchains);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->tf, sizeof(float) * npx * batch);
    if (ce != cudaSuccess) return fail(map_err(ce));

    if (ce == cudaSuccess && algo == HG_WGS) ce = cudaMalloc(&p->w, sizeof(float) * npx * batch);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->sum_part, sizeof(double) * PREP_BLOCKS * batch);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->scale, sizeof(double) * batch);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->err, sizeof(unsigned));
    if (ce == cudaSuccess) ce = cudaMemset(p->err, 0, sizeof(unsigned));
    if (ce != cudaSuccess) return fail(map_err(ce));
    if ((st = make_twiddles(nx, &p->twx)) != HG_OK) return fail(st);
    if ((st = make_twiddles(ny, &p->twy)) != HG_OK) return fail(st);
    {
        // SLM level phasors exp(2 pi i q / L), q < L; amplitude SLM: transmittance q / (L - 1)
        const int L = p->levels;
        float2 h[256];
        const long double two_pi = 6.283185307179586476925286766559005768L;
        for (int q = 0; q < L; ++q) {
            long double a = two_pi * (long double)q / (long double)L;
            h[q] = slm.kind == HG_SLM_AMPLITUDE ? make_float2((float)((double)q / (L - 1)), 0.f)
                                                : make_float2((float)cosl(a), (float)sinl(a));
        }
        ce = cudaMalloc(&p->lvl, sizeof(float2) * L);
        if (ce == cudaSuccess) ce = cudaMemcpy(p->lvl, h, sizeof(float2) * L, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) return fail(map_err(ce));
    }
    if (o.precision > 0) {  // tensor-core row pass: DFT-32 operands, per-device attributes
        p->tc_prec = o.precision;
        p->ppt_tc = ny / (nx == 1024 ? 4 : 2);  // CTA panels: 4 rows of 1024 or 2 rows of 2048
        if (p->ppt_tc > p->ppt_max) p->ppt_max = p->ppt_tc;
        ce = ensure_tc_init(p->dev, &p->tc_blocks);
        uint16_t *hb = (uint16_t *)malloc(4 * TC_B);
        if (!hb) return fail(HG_ERR_OOM);
        tc_make_bmats(o.precision, hb);
        if (ce == cudaSuccess) ce = cudaMalloc(&p->tc_b, 4 * TC_B);
        if (ce == cudaSuccess) ce = cudaMemcpy(p->tc_b, hb, 4 * TC_B, cudaMemcpyHostToDevice);
        free(hb);
        if (ce != cudaSuccess) return fail(map_err(ce));
    }
    if (mod) {  // uniform illumination with the Fresnel term and the whole field as the ROI until set
        const unsigned long long all = npx;
        ce = cudaMalloc(&p->illum, sizeof(float2) * npx);
        if (ce == cudaSuccess) ce = cudaMalloc(&p->roi_rep, npx);
        if (ce == cudaSuccess) ce = cudaMalloc(&p->roi_dft, npx);
        if (ce == cudaSuccess) ce = cudaMalloc(&p->nroi, sizeof(all));
        if (ce == cudaSuccess) ce = cudaMemset(p->roi_rep, 1, npx);
        if (ce == cudaSuccess) ce = cudaMemset(p->roi_dft, 1, npx);
        if (ce == cudaSuccess) ce = cudaMemcpy(p->nroi, &all, sizeof(all), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) return fail(map_err(ce));
        k_illum<<<ew_grid(p, npx), 256, 0, p->cap_stream>>>(nullptr, nullptr, ny, nx, (double)o.fresnel, p->illum,
                                                            p->err);
        ce = cudaStreamSynchronize(p->cap_stream);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(map_err(ce));
    }
    if (search) {
        ce = cudaMalloc(&p->rbuf, sizeof(float2) * npx * batch);
        if (ce == cudaSuccess) ce = cudaMalloc(&p->sholo, npx * batch);
        if (ce != cudaSuccess) return fail(map_err(ce));
    }
    // Pass variants are chosen (and timed) only once every buffer they touch exists;
    // search plans run the generic passes.  Modulated plans take unpaired TMA-fed rows (the
    // light leaving the SLM, E e^{iH}, is complex, so no Hermitian symmetry) and, among the
    // TMA-fed column passes, only those that stage E in shared memory (the others measured
    // slower than the generic column pass at 1024^2 x 64); pipeline 1 admits every
    // TMA-fed column pass.
    const bool mod_any_col = mod && o.pipeline == 1;
    if (o.pipeline != 0 && !search) {
        // TMA-fed passes: row panels need 16-byte aligned rows of T (nx % 4 == 0);
        // the column tiles need a 16-byte multiple row pitch (nx even).
        const PipeOps *rc[8], *cc[8];
        int nr = 0, nc = 0;
        {
            const PipeOps *all[8];
            const int k = pipe_candidates(nx, all, 8);
            for (int i = 0; i < k; ++i) {
                // paired rows need a binary SLM (real e^{iH}), an even column length and the
                // GS/WGS loop
                if (all[i]->paired && (slm.kind != HG_SLM_BINARY || ny % 2 || is_ospr(algo) || mod)) continue;
                if (all[i]->row_iter && nx % 4 == 0 && ensure_pipe_init(p->dev, all[i]) == cudaSuccess)
                    rc[nr++] = all[i];
            }
        }
        {
            const PipeOps *all[8];
            const int k = pipe_candidates(ny, all, 8);
            CUtensorMap m, em;
            for (int i = 0; i < k; ++i)
                if (!all[i]->paired && all[i]->col_gs && nx % 2 == 0 && (!mod || mod_any_col || all[i]->col_emap) &&
                    ensure_pipe_init(p->dev, all[i]) == cudaSuccess && make_col_maps(p, all[i], &m, &em))
                    cc[nc++] = all[i];
        }
        const PipeOps *row = nr ? rc[0] : nullptr, *col = nc ? cc[0] : nullptr;
        if (o.autotune >= 2) {  // forced candidate (tests, benchmarks of one variant)
            const int k = o.autotune - 2;
            if (k >= nr) return fail(HG_ERR_UNSUPPORTED_SIZE);
            row = rc[k];
            col = k < nc ? cc[k] : (nc ? cc[0] : nullptr);
        } else if (o.autotune == 1 && (nr > 1 || nc > 1)) {
            bool cached = false;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                for (const TuneEntry &t : g_tune)
                    if (t.dev == p->dev && t.ny == ny && t.nx == nx && t.items == p->nchains &&
                        t.kind == slm.kind + (mod ? (mod_any_col ? 8 : 24) : 0)) {
                        row = t.row;
                        col = t.col;
                        cached = true;
                    }
            }
            if (!cached) {
                // representative (non-zero) data: the epilogues branch on |R| and T
                k_fill_hash<<<ew_grid(p, 2 * npx * p->nchains), 256, 0, p->cap_stream>>>(
                    (float *)p->field, 2 * npx * p->nchains, -1.f, 2.f);
                k_fill_hash<<<ew_grid(p, npx * batch), 256, 0, p->cap_stream>>>(p->tf, npx * batch, 0.f, 1e-3f);
                ce = cudaStreamSynchronize(p->cap_stream);
                if (ce == cudaSuccess) ce = cudaGetLastError();
                if (ce != cudaSuccess) return fail(map_err(ce));
                // columns first; a row candidate is scored by its own time plus
                // the column pass it implies (in Hermitian form, the faster of the
                // per-column pass and its own column-pair pass)
                float best = 1e30f, best_col = 1e30f;
                for (int i = 0; i < nc; ++i) {
                    const float ms = nc > 1 || nr > 1 ? time_variant(p, cc[i], false) : 0.f;
                    if (i < 4) p->tune_ms[4 + i] = ms;
                    if (ms < best_col) best_col = ms, col = cc[i];
                }
                for (int i = 0; i < nr; ++i) {
                    // a paired row pass with a TMA-fed column pass runs in Hermitian form
                    const bool hm = rc[i]->paired && col && slm.kind == HG_SLM_BINARY;
                    float ms = time_variant(p, rc[i], true, hm);
                    if (i < 4) p->tune_ms[i] = ms;
                    float cm = nc ? best_col : 0.f;
                    if (hm) {
                        cm = time_variant(p, col, false, true);
                        if (rc[i]->col_herm && rc[i]->N == ny)
                            cm = fminf(cm, time_variant(p, rc[i], false, true, true));
                    }
                    ms += cm;
                    if (ms < best) best = ms, row = rc[i];
                }
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune.push_back({p->dev, ny, nx, p->nchains, slm.kind + (mod ? (mod_any_col ? 8 : 24) : 0), row,
                                  col});
            }
        }
        if (row && !p->tc_prec) {
            p->prow = row;
            p->ppt_pipe = row_panels(row, ny);
            if (p->ppt_pipe > p->ppt_max) p->ppt_max = p->ppt_pipe;
        }
        if (col && make_col_maps(p, col, &p->cmap, &p->emap)) p->pcol = col;
        if (o.pipeline == 1 && (!p->prow || !p->pcol)) return fail(HG_ERR_UNSUPPORTED_SIZE);
        // Hermitian loop: a column-pair pass of the column length, when it is at
        // least as fast as the per-column pass (a forced square candidate keeps
        // its own)
        if (herm_loop(p)) {
            const PipeOps *hc[8];
            int nh = 0;
            if (o.autotune >= 2 && p->prow->col_herm && p->prow->N == ny) {
                if (ensure_pipe_init(p->dev, p->prow) == cudaSuccess && p->prow->herm_blocks_per_sm > 0)
                    hc[nh++] = p->prow;
            } else {
                const PipeOps *all[8];
                const int k = pipe_candidates(ny, all, 8);
                for (int i = 0; i < k; ++i)
                    if (all[i]->col_herm && ensure_pipe_init(p->dev, all[i]) == cudaSuccess &&
                        all[i]->herm_blocks_per_sm > 0)
                        hc[nh++] = all[i];
            }
            const PipeOps *best = nullptr;
            float best_ms = 1e30f;
            // a forced candidate k of another column length takes that length's k-th
            // column-pair variant (the last one if it has fewer)
            if (o.autotune >= 2 && nh > 1 && p->prow->N != ny) {
                hc[0] = hc[std::min(o.autotune - 2, nh - 1)];
                nh = 1;
            }
            for (int i = 0; i < nh; ++i) {
                CUtensorMap m;
                if (!make_cmap_box(p, hc[i]->herm_c, hc[i]->herm_boxr, &m)) continue;
                const float ms = (o.autotune == 1 && nh > 0) ? time_variant(p, hc[i], false, true, true) : 0.f;
                if (!best || ms < best_ms) best = hc[i], best_ms = ms;
            }
            if (best) {
                bool take = true;
                if (o.autotune == 1) take = best_ms <= time_variant(p, p->pcol, false, true);
                if (take && make_cmap_box(p, best->herm_c, best->herm_boxr, &p->cmap_herm)) {
                    p->use_herm_col = true;
                    p->hops = best;
                }
            }
        }
        // Binary OSPR: one pass per subframe in Hermitian form with the column-pair
        // pass of any paired variant of this column length (square power-of-two fields)
        if (is_ospr(algo) && ny == nx && ny % 2 == 0) {
            // the fastest column-pair pass of the paired variants (the first when not tuning)
            const PipeOps *all[8];
            const int k = pipe_candidates(ny, all, 8);
            float best_ms = 1e30f;
            for (int i = 0; i < k; ++i) {
                CUtensorMap m;
                if (!(all[i]->paired && all[i]->col_herm && ensure_pipe_init(p->dev, all[i]) == cudaSuccess &&
                      all[i]->herm_blocks_per_sm > 0 && make_cmap_box(p, all[i]->herm_c, all[i]->herm_boxr, &m)))
                    continue;
                const float ms = o.autotune == 1 ? time_variant(p, all[i], false, true, true) : 0.f;
                if (!p->hops || ms < best_ms) {
                    p->hops = all[i];
                    p->cmap_herm = m;
                    best_ms = ms;
                }
                if (o.autotune != 1) break;
            }
            p->ospr_herm = p->hops != nullptr;
            // the Hermitian head and averages keep one metric panel per row ky <= ny/2
            if (p->ospr_herm && p->ppt_max < ny / 2 + 1) p->ppt_max = ny / 2 + 1;
        }
    }
    if ((st = ensure_part(p, is_ospr(algo) ? 1 : 8)) != HG_OK) return fail(st);
    if (algo == HG_ADOSPR) {
        ce = cudaMalloc(&p->acc, sizeof(float) * npx * batch);
        if (ce == cudaSuccess) ce = cudaMalloc(&p->holo_tmp, npx * batch);
        if (ce != cudaSuccess) return fail(map_err(ce));
    }
    if ((st = ensure_metrics(p, 1)) != HG_OK) return fail(st);
    *out = p;
    return HG_OK;
}

hg_status hg_sync(hg_plan p) {
    if (!p) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    HG_CK(cudaStreamSynchronize(p->stream));
    HG_CK(cudaGetLastError());
    return check_err_flag(p);
}

int hg_last_launch_count(hg_plan p) { return p ? p->launches : 0; }

hg_status hg_debug_inject(hg_plan p, int drop_job, uint64_t wait_ns) {
    if (!p || wait_ns == 0) return HG_ERR_INVALID_ARG;
    p->drop_job = drop_job;
    p->wait_ns = wait_ns;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);  // captured launches carry the old values
    p->gexec = nullptr;
    p->g_iters = -1;
    return HG_OK;
}

hg_status hg_profile_enable(hg_plan p, int max_passes) {
    if (!p || max_passes < 0) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    HG_CK(cudaStreamSynchronize(p->stream));
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    p->prof_kind.assign((size_t)max_passes, 0);
    p->prof_used = 0;
    p->prof_on = max_passes > 0;
    for (int i = 0; i < 2 * max_passes; ++i) {
        cudaEvent_t e;
        HG_CK(cudaEventCreate(&e));
        p->prof_ev.push_back(e);
    }
    return HG_OK;
}

hg_status hg_profile_read(hg_plan p, double *out4) {
    if (!p || !out4) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    HG_CK(cudaStreamSynchronize(p->stream));
    double acc[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < p->prof_used; ++i) {
        float ms = 0;
        HG_CK(cudaEventElapsedTime(&ms, p->prof_ev[2 * i], p->prof_ev[2 * i + 1]));
        acc[2 * p->prof_kind[i]] += ms;
        acc[2 * p->prof_kind[i] + 1] += 1;
    }
    memcpy(out4, acc, sizeof acc);
    p->prof_used = 0;
    return HG_OK;
}

const char *hg_plan_variant(hg_plan p, int pass) {
    if (!p) return "";
    if (pass == 1 && p->ospr_herm) {
        snprintf(p->vname[1], sizeof p->vname[1], "%s+herm-colpairs (OSPR)", p->hops->name);
        return p->vname[1];
    }
    if (pass == 0 && p->tc_prec) {
        static const char *names[2][5] = {
            {"", "1024:tc32x32-fp16hilo", "1024:tc32x32-fp16", "1024:tc32x32-bf16hilo", "1024:tc32x32-bf16"},
            {"", "2048:2x(tc32x32)-fp16hilo", "2048:2x(tc32x32)-fp16", "2048:2x(tc32x32)-bf16hilo",
             "2048:2x(tc32x32)-bf16"}};
        return names[p->nx == 2048][p->tc_prec];
    }
    const PipeOps *o = pass == 0 ? p->prow : p->pcol;
    if (o && herm_loop(p)) {  // Hermitian form of the binary loop
        // the column-pair pass may come from another variant than the per-column pass
        const bool pairs = pass == 1 && p->use_herm_col;
        snprintf(p->vname[pass], sizeof p->vname[pass], "%s+herm%s", pairs ? p->hops->name : o->name,
                 pairs ? "-colpairs" : "");
        return p->vname[pass];
    }
    return o ? o->name : "generic";
}

int hg_pipelined(hg_plan p) { return p ? (p->prow ? 1 : 0) | (p->pcol ? 2 : 0) : 0; }

hg_status hg_run(hg_plan p, const float *target, const float *init_phase, int iters,
                 uint8_t *holo_out, double *mse_out) {
    NvtxRange nv("hg_run");
    if (!p || !target) return HG_ERR_INVALID_ARG;
    if (is_ospr(p->algo)) {
        if (init_phase) return HG_ERR_INVALID_ARG;
        iters = 1;
    } else if (iters < 1) {
        return HG_ERR_INVALID_ARG;
    }
    DevGuard g(p->dev);
    p->launches = 0;
    const size_t fbytes = sizeof(float) * p->npx * p->batch;
    const size_t hbytes = p->npx * p->nchains;
    const size_t mbytes = sizeof(double) * p->batch * (is_ospr(p->algo) ? 1 : iters);
    const bool t_host = !is_device_ptr(target);
    const bool ph_host = init_phase && !is_device_ptr(init_phase);
    const bool ho_host = holo_out && !is_device_ptr(holo_out);
    const bool mo_host = mse_out && !is_device_ptr(mse_out);
    const bool any_host = t_host || ph_host || ho_host || mo_host;
    hg_status st;
    if (any_host) {
        // layout: [target][phase][holo][mse], 256-byte aligned pieces
        auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
        if ((st = ensure_stage(p, al(fbytes) * 2 + al(hbytes) + al(mbytes))) != HG_OK) return st;
    }
    char *sb = (char *)p->stage;
    auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const float *d_t = target, *d_ph = init_phase;
    uint8_t *d_ho = holo_out;
    double *d_mo = mse_out;
    const std::vector<int> cst = any_host ? host_chunk_starts(p, iters) : std::vector<int>{0, p->batch};
    const bool chunked = cst.size() > 2;  // copies by chunk, see run_chunked
    if (t_host) {
        if (!chunked) HG_CK(cudaMemcpyAsync(sb, target, fbytes, cudaMemcpyHostToDevice, p->stream));
        d_t = (const float *)sb;
    }
    if (ph_host) {
        if (!chunked)
            HG_CK(cudaMemcpyAsync(sb + al(fbytes), init_phase, fbytes, cudaMemcpyHostToDevice, p->stream));
        d_ph = (const float *)(sb + al(fbytes));
    }
    if (ho_host) d_ho = (uint8_t *)(sb + 2 * al(fbytes));
    if (mo_host) d_mo = (double *)(sb + 2 * al(fbytes) + al(hbytes));

    if ((st = ensure_part(p, iters)) != HG_OK) return st;
    if ((st = ensure_metrics(p, iters)) != HG_OK) return st;
    if (chunked) return run_chunked(p, cst, target, d_t, init_phase, d_ph, iters, holo_out, d_ho, mse_out, d_mo);
    if ((st = enqueue_run(p, d_t, d_ph, iters, d_ho, d_mo, false)) != HG_OK) return st;
    if (ho_host)
        HG_CK(cudaMemcpyAsync(holo_out, d_ho, hbytes, cudaMemcpyDeviceToHost, p->stream));
    if (mo_host) HG_CK(cudaMemcpyAsync(mse_out, d_mo, mbytes, cudaMemcpyDeviceToHost, p->stream));
    if (any_host) return hg_sync(p);
    return HG_OK;
}

hg_status hg_get_metrics(hg_plan p, double *out, size_t count) {
    if (!p || !out || !p->have_run) return HG_ERR_INVALID_ARG;
    const size_t n = (size_t)p->batch * p->last_iters * NMET;
    if (count < n) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    HG_CK(cudaMemcpyAsync(out, p->metrics, n * sizeof(double), cudaMemcpyDefault, p->stream));
    if (!is_device_ptr(out)) HG_CK(cudaStreamSynchronize(p->stream));
    return HG_OK;
}

hg_status hg_replay(hg_plan p, const uint8_t *holo, float *intensity_out) {
    NvtxRange nv("hg_replay");
    if (!p || !holo || !intensity_out) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    p->launches = 0;
    const size_t hbytes = p->npx * p->nchains, ibytes = sizeof(float) * p->npx * p->batch;
    const bool h_host = !is_device_ptr(holo), i_host = !is_device_ptr(intensity_out);
    hg_status st;
    if (h_host || i_host)
        if ((st = ensure_stage(p, hbytes + 256 + ibytes)) != HG_OK) return st;
    const uint8_t *d_h = holo;
    float *d_i = intensity_out;
    if (h_host) {
        HG_CK(cudaMemcpyAsync(p->stage, holo, hbytes, cudaMemcpyHostToDevice, p->stream));
        d_h = (const uint8_t *)p->stage;
    }
    if (i_host) d_i = (float *)((char *)p->stage + ((hbytes + 255) & ~(size_t)255));
    p->field_from_run = false;
    ColArgs ca = col_args(p);
    ca.items = p->nchains;
    ca.holo = const_cast<uint8_t *>(d_h);
    launch_col(p, col_role_holo(p), ca, p->stream);
    RowArgs ra = row_args(p);
    ra.nsub = p->nsub;
    ra.T = nullptr;
    ra.w = nullptr;
    ra.I_out = d_i;
    launch_row(p, ROW_AVG, ra, p->stream);
    if (p->mod) {  // the replay energy depends on the hologram: normalise by its sum
        if (!p->ev_part) HG_CK(cudaMalloc(&p->ev_part, sizeof(double) * (EV_S1 + EV_S2) * EV_BLOCKS * p->batch));
        const dim3 eg(EV_BLOCKS, p->batch);
        k_eval1<<<eg, EV_THREADS, 0, p->stream>>>(d_i, nullptr, nullptr, (int)p->npx, p->ev_part, p->err);
        k_eval2<<<eg, EV_THREADS, 0, p->stream>>>(d_i, nullptr, nullptr, (int)p->npx, p->ev_part, nullptr, d_i);
        p->launches += 2;
    }
    HG_CK(cudaGetLastError());
    if (i_host) {
        HG_CK(cudaMemcpyAsync(intensity_out, d_i, ibytes, cudaMemcpyDeviceToHost, p->stream));
        HG_CK(cudaStreamSynchronize(p->stream));
    }
    return HG_OK;
}

hg_status hg_get_phase(hg_plan p, float *phase_out) {
    if (!p || !phase_out || !p->field_from_run || is_ospr(p->algo)) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    p->launches = 0;
    // Recompute arg R of the last replay field (still in the field buffer
    // after the tail, which does not modify it) without touching metrics.
    const size_t bytes = sizeof(float) * p->npx * p->batch;
    const bool host = !is_device_ptr(phase_out);
    hg_status st;
    if (host && (st = ensure_stage(p, bytes)) != HG_OK) return st;
    float *d = host ? (float *)p->stage : phase_out;
    RowArgs ra = row_args(p);
    ra.w = nullptr;  // no weight update
    ra.phase_out = d;
    // after a run of the Hermitian loop the field holds rows ky <= ny/2 only
    if (herm_ends(p)) launch_pair_end(p, false, ra, p->stream);
    else launch_row(p, ROW_TAIL, ra, p->stream);
    HG_CK(cudaGetLastError());
    if (host) {
        HG_CK(cudaMemcpyAsync(phase_out, d, bytes, cudaMemcpyDeviceToHost, p->stream));
        HG_CK(cudaStreamSynchronize(p->stream));
    }
    return HG_OK;
}

hg_status hg_set_illumination(hg_plan p, const float *amp, const float *phase) {
    NvtxRange nv("hg_set_illumination");
    if (!p || !p->mod) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    const size_t bytes = sizeof(float) * p->npx, off = (bytes + 255) & ~(size_t)255;
    const bool ah = amp && !is_device_ptr(amp), fh = phase && !is_device_ptr(phase);
    hg_status st;
    if ((ah || fh) && (st = ensure_stage(p, 2 * off)) != HG_OK) return st;
    const float *da = amp, *df = phase;
    if (ah) {
        HG_CK(cudaMemcpyAsync(p->stage, amp, bytes, cudaMemcpyHostToDevice, p->stream));
        da = (const float *)p->stage;
    }
    if (fh) {
        float *d = (float *)((char *)p->stage + off);
        HG_CK(cudaMemcpyAsync(d, phase, bytes, cudaMemcpyHostToDevice, p->stream));
        df = d;
    }
    HG_CK(cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream));
    k_illum<<<ew_grid(p, p->npx), 256, 0, p->stream>>>(da, df, p->ny, p->nx, (double)p->fresnel, p->illum, p->err);
    HG_CK(cudaGetLastError());
    return check_err_flag(p);
}

hg_status hg_set_roi(hg_plan p, const uint8_t *roi) {
    NvtxRange nv("hg_set_roi");
    if (!p || !p->mod) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    if (!roi) {
        const unsigned long long all = p->npx;
        HG_CK(cudaMemsetAsync(p->roi_rep, 1, p->npx, p->stream));
        HG_CK(cudaMemsetAsync(p->roi_dft, 1, p->npx, p->stream));
        HG_CK(cudaMemcpyAsync(p->nroi, &all, sizeof(all), cudaMemcpyHostToDevice, p->stream));
    } else {
        HG_CK(cudaMemcpyAsync(p->roi_rep, roi, p->npx, cudaMemcpyDefault, p->stream));
        HG_CK(cudaMemsetAsync(p->nroi, 0, sizeof(unsigned long long), p->stream));
        k_roi_dft<<<ew_grid(p, p->npx), 256, 0, p->stream>>>(p->roi_rep, p->ny, p->nx, p->roi_dft, p->nroi);
        HG_CK(cudaGetLastError());
    }
    HG_CK(cudaStreamSynchronize(p->stream));  // the caller's buffer may be reused on return
    return HG_OK;
}

hg_status hg_evaluate(hg_plan p, const uint8_t *holo, const float *target, double *out) {
    NvtxRange nv("hg_evaluate");
    if (!p || !holo || !target || !out) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    p->launches = 0;
    const size_t hbytes = p->npx * p->nchains, tbytes = sizeof(float) * p->npx * p->batch,
                 obytes = sizeof(double) * 5 * p->batch;
    auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const bool h_host = !is_device_ptr(holo), t_host = !is_device_ptr(target), o_host = !is_device_ptr(out);
    hg_status st;
    if ((h_host || t_host || o_host) && (st = ensure_stage(p, al(hbytes) + al(tbytes) + obytes)) != HG_OK)
        return st;
    if (!p->ev_buf) HG_CK(cudaMalloc(&p->ev_buf, sizeof(float) * p->npx * p->batch));
    if (!p->ev_part) HG_CK(cudaMalloc(&p->ev_part, sizeof(double) * (EV_S1 + EV_S2) * EV_BLOCKS * p->batch));
    const uint8_t *d_h = holo;
    const float *d_t = target;
    double *d_o = out;
    if (h_host) {
        HG_CK(cudaMemcpyAsync(p->stage, holo, hbytes, cudaMemcpyHostToDevice, p->stream));
        d_h = (const uint8_t *)p->stage;
    }
    if (t_host) {
        float *d = (float *)((char *)p->stage + al(hbytes));
        HG_CK(cudaMemcpyAsync(d, target, tbytes, cudaMemcpyHostToDevice, p->stream));
        d_t = d;
    }
    if (o_host) d_o = (double *)((char *)p->stage + al(hbytes) + al(tbytes));
    HG_CK(cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream));
    p->field_from_run = false;
    ColArgs ca = col_args(p);
    ca.items = p->nchains;
    ca.holo = const_cast<uint8_t *>(d_h);
    launch_col(p, col_role_holo(p), ca, p->stream);
    RowArgs ra = row_args(p);
    ra.nsub = p->nsub;
    ra.T = nullptr;
    ra.w = nullptr;
    ra.I_out = p->ev_buf;
    launch_row(p, ROW_AVG, ra, p->stream);
    double *part1 = p->ev_part, *part2 = p->ev_part + (size_t)EV_S1 * EV_BLOCKS * p->batch;
    const dim3 eg(EV_BLOCKS, p->batch);
    k_eval1<<<eg, EV_THREADS, 0, p->stream>>>(p->ev_buf, d_t, p->roi_rep, (int)p->npx, part1, p->err);
    k_eval2<<<eg, EV_THREADS, 0, p->stream>>>(p->ev_buf, d_t, p->roi_rep, (int)p->npx, part1, part2, nullptr);
    k_eval_fin<<<(p->batch + 127) / 128, 128, 0, p->stream>>>(part1, part2, p->batch, p->nroi, (double)p->npx,
                                                               d_o, p->err);
    p->launches += 3;
    HG_CK(cudaGetLastError());
    if (o_host) HG_CK(cudaMemcpyAsync(out, d_o, obytes, cudaMemcpyDeviceToHost, p->stream));
    if (h_host || t_host || o_host) return hg_sync(p);
    return HG_OK;
}

hg_status hg_set_weights(hg_plan p, const float *w) {
    if (!p || !w || p->algo != HG_WGS) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    const size_t bytes = sizeof(float) * p->npx * p->batch;
    const float *src = w;
    hg_status st;
    if (!is_device_ptr(w)) {
        if ((st = ensure_stage(p, bytes)) != HG_OK) return st;
        HG_CK(cudaMemcpyAsync(p->stage, w, bytes, cudaMemcpyHostToDevice, p->stream));
        src = (const float *)p->stage;
    }
    k_reorder<<<ew_grid(p, p->npx * p->batch), 256, 0, p->stream>>>(src, p->w, p->ny, p->nx,
                                                                     p->batch, 1);
    HG_CK(cudaGetLastError());
    p->weights_preset = true;
    if (src != w) HG_CK(cudaStreamSynchronize(p->stream));
    return HG_OK;
}

hg_status hg_get_weights(hg_plan p, float *w_out) {
    if (!p || !w_out || p->algo != HG_WGS) return HG_ERR_INVALID_ARG;
    DevGuard g(p->dev);
    const size_t bytes = sizeof(float) * p->npx * p->batch;
    const bool host = !is_device_ptr(w_out);
    hg_status st;
    if (host && (st = ensure_stage(p, bytes)) != HG_OK) return st;
    float *d = host ? (float *)p->stage : w_out;
    k_reorder<<<ew_grid(p, p->npx * p->batch), 256, 0, p->stream>>>(p->w, d, p->ny, p->nx,
                                                                     p->batch, 0);
    HG_CK(cudaGetLastError());
    if (host) {
        HG_CK(cudaMemcpyAsync(w_out, d, bytes, cudaMemcpyDeviceToHost, p->stream));
        HG_CK(cudaStreamSynchronize(p->stream));
    }
    return HG_OK;
}

hg_status hg_debug_step(hg_plan p, const float *target, const float *phase_in, float *h_out,
                        uint8_t *holo_out, float *replay_out, double *metrics_out) {
    NvtxRange nv("hg_debug_step");
    if (!p || !target || !phase_in || is_ospr(p->algo) || is_search(p->algo) || p->mod) return HG_ERR_INVALID_ARG;
    for (const void *q : {(const void *)target, (const void *)phase_in, (const void *)h_out,
                          (const void *)holo_out, (const void *)replay_out,
                          (const void *)metrics_out})
        if (q && !is_device_ptr(q)) return HG_ERR_INVALID_ARG;  // device buffers only
    DevGuard g(p->dev);
    p->launches = 0;
    hg_status st;
    if ((st = ensure_part(p, 1)) != HG_OK) return st;
    if ((st = ensure_metrics(p, 1)) != HG_OK) return st;
    HG_CK(cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream));
    enqueue_prep(p, target);
    if (p->algo == HG_WGS && !p->weights_preset) {
        k_fill<<<ew_grid(p, p->npx * p->batch), 256, 0, p->stream>>>(p->w, p->npx * p->batch, 1.f);
        p->launches++;
    }
    RowArgs ra = row_args(p);
    ra.phase = phase_in;
    launch_row(p, ROW_HEAD, ra, p->stream);
    ColArgs ca = col_args(p);
    ca.holo = holo_out;
    ca.h_out = (float2 *)h_out;
    launch_col_gs(p, col_role_gs(p), ca, p->stream);
    RowArgs rt = row_args(p);
    rt.part = p->part;
    rt.R_out = (float2 *)replay_out;
    if (p->tc_prec) launch_row_tc(p, ROW_TAIL, rt, p->stream);
    else launch_row(p, ROW_TAIL, rt, p->stream);
    const int pl = p->tc_prec ? p->ppt_tc : p->ppt;
    k_reduce<<<(p->batch * 32 + 127) / 128, 128, 0, p->stream>>>(p->part, 1, p->batch, p->ppt_max, pl, pl,
                                                             1.0 / (double)p->npx, p->metrics, nullptr);
    p->launches++;
    if (metrics_out)
        HG_CK(cudaMemcpyAsync(metrics_out, p->metrics, sizeof(double) * NMET * p->batch,
                              cudaMemcpyDeviceToDevice, p->stream));
    HG_CK(cudaGetLastError());
    p->weights_preset = false;
    p->have_run = true;
    p->field_from_run = true;
    p->last_iters = 1;
    return HG_OK;
}

// One row pass and one column pass of the iteration loop, fed a hologram:
// the column spectra of the hologram's SLM field (generic HOLO role, all
// rows), then exactly the launches enqueue_loop makes for an iteration k >= 1
// (the plan's own row-pass and column-pass variants), then the metric
// reduction of the row pass's panels.
hg_status hg_debug_loop_step(hg_plan p, const float *target, const uint8_t *holo_in, int k, float *row_out,
                             uint8_t *holo_out, float *col_out, double *metrics_out) {
    NvtxRange nv("hg_debug_loop_step");
    if (!p || !target || !holo_in || k < 0 || is_ospr(p->algo) || is_search(p->algo)) return HG_ERR_INVALID_ARG;
    for (const void *q : {(const void *)target, (const void *)holo_in, (const void *)row_out,
                          (const void *)holo_out, (const void *)col_out, (const void *)metrics_out})
        if (q && !is_device_ptr(q)) return HG_ERR_INVALID_ARG;  // device buffers only
    DevGuard g(p->dev);
    p->launches = 0;
    hg_status st;
    if ((st = ensure_part(p, 1)) != HG_OK) return st;
    if ((st = ensure_metrics(p, 1)) != HG_OK) return st;
    const size_t fbytes = sizeof(float2) * p->npx * p->batch;
    HG_CK(cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream));
    enqueue_prep(p, target);
    if (p->algo == HG_WGS && !p->weights_preset) {
        k_fill<<<ew_grid(p, p->npx * p->batch), 256, 0, p->stream>>>(p->w, p->npx * p->batch, 1.f);
        p->launches++;
    }
    ColArgs ch = col_args(p);
    ch.holo = const_cast<uint8_t *>(holo_in);
    launch_col(p, col_role_holo(p), ch, p->stream);
    ColArgs ca = col_args(p);
    RowArgs ra = row_args(p);
    ca.half = p->prow && p->prow->paired;
    ra.herm = herm_loop(p);
    ca.half_in = ra.herm;
    ra.part = p->part;
    lt_set(p, ra, k + 1);
    launch_row_iter(p, ra, p->stream);
    if (row_out) HG_CK(cudaMemcpyAsync(row_out, p->field, fbytes, cudaMemcpyDeviceToDevice, p->stream));
    ca.holo = holo_out;
    if (ca.half_in && p->use_herm_col) launch_col_herm(p, ca, p->stream);
    else launch_col_gs(p, col_role_gs(p), ca, p->stream);
    if (col_out) HG_CK(cudaMemcpyAsync(col_out, p->field, fbytes, cudaMemcpyDeviceToDevice, p->stream));
    const int pl = p->tc_prec ? p->ppt_tc : p->prow ? p->ppt_pipe : p->ppt;
    if (p->mod)
        k_reduce_gen<<<(p->batch * 32 + 127) / 128, 128, 0, p->stream>>>(p->part, 1, p->batch, p->ppt_max, pl, pl,
                                                                     p->nroi, p->metrics, nullptr);
    else
        k_reduce<<<(p->batch * 32 + 127) / 128, 128, 0, p->stream>>>(p->part, 1, p->batch, p->ppt_max, pl, pl,
                                                                 1.0 / (double)p->npx, p->metrics, nullptr);
    p->launches++;
    if (metrics_out)
        HG_CK(cudaMemcpyAsync(metrics_out, p->metrics, sizeof(double) * NMET * p->batch,
                              cudaMemcpyDeviceToDevice, p->stream));
    HG_CK(cudaGetLastError());
    p->weights_preset = false;
    p->have_run = true;
    p->field_from_run = false;
    p->last_iters = 1;
    return HG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ groups
// Several plans (targets of different sizes) run as one CUDA graph: each
// plan's whole run is a branch forked from one capture, so the GPU executes
// the size buckets concurrently.

struct hg_group_s {
    int dev = 0, n = 0;
    hg_plan plans[HG_GROUP_MAX];
    cudaStream_t cap = nullptr;
    cudaStream_t branch[HG_GROUP_MAX] = {};
    cudaEvent_t fork = nullptr, join[HG_GROUP_MAX] = {};
    cudaGraphExec_t exec = nullptr;
    int iters = -1;
    const void *key[4 * HG_GROUP_MAX] = {};
    int launches = 0;
    int schedule = HG_GROUP_SERIAL;  // branches in sequence, or concurrent
};

extern "C" {

void hg_group_destroy(hg_group g) {
    if (!g) return;
    DevGuard dg(g->dev);
    if (g->cap) cudaStreamSynchronize(g->cap);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (int i = 0; i < g->n; ++i) {
        if (g->branch[i]) cudaStreamDestroy(g->branch[i]);
        if (g->join[i]) cudaEventDestroy(g->join[i]);
    }
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
}

hg_status hg_group_create(hg_group *out, int nplans, const hg_plan *plans) {
    if (!out || !plans || nplans < 1 || nplans > HG_GROUP_MAX) return HG_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < nplans; ++i)
        if (!plans[i] || plans[i]->dev != plans[0]->dev) return HG_ERR_INVALID_ARG;
    hg_group g = new (std::nothrow) hg_group_s();
    if (!g) return HG_ERR_OOM;
    g->dev = plans[0]->dev;
    g->n = nplans;
    DevGuard dg(g->dev);
    cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    for (int i = 0; i < nplans && e == cudaSuccess; ++i) {
        g->plans[i] = plans[i];
        e = cudaStreamCreateWithFlags(&g->branch[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        hg_group_destroy(g);
        return map_err(e);
    }
    *out = g;
    return HG_OK;
}

hg_status hg_group_run(hg_group g, const float *const *targets, const float *const *init_phases,
                       int iters, uint8_t *const *holo_out, double *const *mse_out, void *stream) {
    NvtxRange nv("hg_group_run");
    if (!g || !targets || iters < 1) return HG_ERR_INVALID_ARG;
    DevGuard dg(g->dev);
    const void *key[4 * HG_GROUP_MAX];
    for (int i = 0; i < g->n; ++i) {
        hg_plan p = g->plans[i];
        const void *q[4] = {targets[i], init_phases ? init_phases[i] : nullptr,
                            holo_out ? holo_out[i] : nullptr, mse_out ? mse_out[i] : nullptr};
        if (!q[0] || is_ospr(p->algo)) return HG_ERR_INVALID_ARG;
        for (int k = 0; k < 4; ++k) {
            if (q[k] && !is_device_ptr(q[k])) return HG_ERR_INVALID_ARG;  // device buffers only
            key[4 * i + k] = q[k];
        }
    }
    bool same = g->exec && g->iters == iters;
    for (int k = 0; same && k < 4 * g->n; ++k) same = key[k] == g->key[k];
    hg_status st;
    if (!same) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        for (int i = 0; i < g->n; ++i) {
            if ((st = ensure_part(g->plans[i], iters)) != HG_OK) return st;
            if ((st = ensure_metrics(g->plans[i], iters)) != HG_OK) return st;
        }
        HG_CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaEventRecord(g->fork, g->cap);
        g->launches = 0;
        const bool conc = g->schedule == HG_GROUP_CONCURRENT;
        for (int i = 0; i < g->n && e == cudaSuccess; ++i) {
            hg_plan p = g->plans[i];
            // serial: every plan's run on the capture stream, one after another;
            // concurrent: each run a branch forked from the capture stream
            if (conc) e = cudaStreamWaitEvent(g->branch[i], g->fork, 0);
            if (e != cudaSuccess) break;
            cudaStream_t keep = p->stream;
            const bool prof = p->prof_on;
            p->stream = conc ? g->branch[i] : g->cap;
            p->prof_on = false;
            p->launches = 0;
            st = enqueue_run(p, (const float *)key[4 * i], (const float *)key[4 * i + 1], iters,
                             (uint8_t *)key[4 * i + 2], (double *)key[4 * i + 3], true);
            g->launches += p->launches;
            p->stream = keep;
            p->prof_on = prof;
            if (st != HG_OK) e = cudaErrorUnknown;
            if (conc && e == cudaSuccess) e = cudaEventRecord(g->join[i], g->branch[i]);
            if (conc && e == cudaSuccess) e = cudaStreamWaitEvent(g->cap, g->join[i], 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(g->cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g->exec = nullptr;
            return map_err(e);
        }
        g->iters = iters;
        for (int k = 0; k < 4 * g->n; ++k) g->key[k] = key[k];
    }
    HG_CK(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    for (int i = 0; i < g->n; ++i) {
        hg_plan p = g->plans[i];
        p->have_run = true;
        p->field_from_run = true;
        p->last_iters = iters;
        p->weights_preset = false;
    }
    return HG_OK;
}

hg_status hg_group_sync(hg_group g, void *stream) {
    if (!g) return HG_ERR_INVALID_ARG;
    DevGuard dg(g->dev);
    HG_CK(cudaStreamSynchronize((cudaStream_t)stream));
    hg_status worst = HG_OK;
    for (int i = 0; i < g->n; ++i) {
        hg_status st = check_err_flag(g->plans[i]);
        if (st != HG_OK && worst == HG_OK) worst = st;
    }
    return worst;
}

int hg_group_launch_count(hg_group g) { return g ? g->launches : 0; }

hg_status hg_group_set_schedule(hg_group g, int schedule) {
    if (!g || (schedule != HG_GROUP_SERIAL && schedule != HG_GROUP_CONCURRENT)) return HG_ERR_INVALID_ARG;
    if (schedule != g->schedule) {
        g->schedule = schedule;
        if (g->exec) {  // captured with the other schedule: capture again at the next run
            DevGuard dg(g->dev);
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
    }
    return HG_OK;
}

}  // extern "C"

// ------------------------------------------------------- allocation-free run
// hg_run_noalloc: a single-target GS/WGS run whose work memory is one static
// device region instead of plan buffers.  It launches the same generic row
// and column kernels as a plan made with pipeline = 0; the one difference in
// the launch sequence is that each iteration's metric partials are reduced
// right after its row pass, so the region holds one iteration's partials
// rather than all of them and the iteration count is not bounded by it.

namespace {

constexpr int kNaSide = HG_NOALLOC_MAX_SIDE;
constexpr size_t kNaPx = (size_t)kNaSide * kNaSide;
constexpr size_t na_al(size_t n) { return (n + 255) & ~(size_t)255; }
// region layout (byte offsets, each piece 256-byte aligned)
constexpr size_t kNaField = 0;                                              // float2 [ny][nx]
constexpr size_t kNaTf = kNaField + na_al(sizeof(float2) * kNaPx);          // float [ny][nx]
constexpr size_t kNaW = kNaTf + na_al(sizeof(float) * kNaPx);               // float [ny][nx] (WGS)
constexpr size_t kNaPart = kNaW + na_al(sizeof(float) * kNaPx);             // double [panels <= ny][NMET]
constexpr size_t kNaMetrics = kNaPart + na_al(sizeof(double) * NMET * kNaSide);  // double [NMET]
constexpr size_t kNaSumPart = kNaMetrics + na_al(sizeof(double) * NMET);   // double [PREP_BLOCKS]
constexpr size_t kNaScale = kNaSumPart + na_al(sizeof(double) * PREP_BLOCKS);
constexpr size_t kNaErr = kNaScale + na_al(sizeof(double));
constexpr size_t kNaTwx = kNaErr + na_al(sizeof(unsigned));                 // float2 [nx]
constexpr size_t kNaTwy = kNaTwx + na_al(sizeof(float2) * kNaSide);         // float2 [ny]
constexpr size_t kNaLvl = kNaTwy + na_al(sizeof(float2) * kNaSide);         // float2 [256]
constexpr size_t kNaBytes = kNaLvl + na_al(sizeof(float2) * 256);
static_assert(kNaBytes == HG_NOALLOC_SCRATCH_BYTES, "header states the region's size");

// The region itself: static device memory of this library, one per device.
static __device__ __align__(256) unsigned char g_na_region[kNaBytes];

struct NaDevice {
    bool ready = false;
    char *base = nullptr;
    int nsm = 0;
};
std::mutex g_na_mu;
NaDevice g_na[kMaxDev];

// One-time per-device setup with `dev` current: the region's address, the SM
// count, and the kernel attributes of every compiled length up to the limit.
cudaError_t na_setup(int dev, NaDevice *out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    NaDevice &d = g_na[dev];
    if (!d.ready) {
        void *base = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&base, g_na_region);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        for (int n = 1; n <= kNaSide; ++n)
            if (const LineOps *o = find_ops(n))
                if ((e = ensure_init(dev, o)) != cudaSuccess) return e;
        d.base = (char *)base;
        d.ready = true;
    }
    *out = d;
    return cudaSuccess;
}

// Forward roots exp(-2 pi i e / n), e < n, as make_twiddles computes them,
// written into a caller array instead of a new device buffer.
void na_twiddles(int n, float2 *h) {
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int e = 0; e < n; ++e) {
        long double a = two_pi * (long double)e / (long double)n;
        h[e] = make_float2((float)cosl(a), (float)-sinl(a));
    }
}

}  // namespace

extern "C" hg_status hg_run_noalloc(int ny, int nx, hg_slm slm, hg_algo algo, const float *target,
                                    const float *init_phase, int iters, uint8_t *holo_out,
                                    double *mse_out, void *stream) {
    if (ny < 1 || nx < 1 || !target || iters < 1) return HG_ERR_INVALID_ARG;
    if (algo != HG_GS && algo != HG_WGS) return HG_ERR_INVALID_ARG;
    if (slm.kind != HG_SLM_BINARY && slm.kind != HG_SLM_LLEVEL) return HG_ERR_INVALID_ARG;
    if (slm.kind == HG_SLM_LLEVEL && (slm.levels < 2 || slm.levels > 256)) return HG_ERR_INVALID_ARG;
    if (ny > kNaSide || nx > kNaSide) return HG_ERR_TOO_LARGE;
    const LineOps *rops = find_ops(nx), *cops = find_ops(ny);
    if (!rops || !cops) return HG_ERR_UNSUPPORTED_SIZE;
    for (const void *ptr : {(const void *)target, (const void *)init_phase, (const void *)holo_out,
                            (const void *)mse_out})
        if (ptr && !is_device_ptr(ptr)) return HG_ERR_INVALID_ARG;

    int dev = 0;
    HG_CK(cudaGetDevice(&dev));
    NaDevice d;
    HG_CK(na_setup(dev, &d));
    const cudaStream_t s = (cudaStream_t)stream;

    // A plan record on the stack whose buffers all point into the region; it
    // owns nothing and is never destroyed through hg_plan_destroy.
    hg_plan_s q;
    q.dev = dev;
    q.ny = ny;
    q.nx = nx;
    q.batch = 1;
    q.algo = algo;
    q.kind = slm.kind;
    q.levels = slm.kind == HG_SLM_BINARY ? 2 : slm.levels;
    q.nchains = 1;
    q.stream = s;
    q.use_graph = 0;
    q.rops = rops;
    q.cops = cops;
    q.nsm = d.nsm;
    q.npx = (size_t)ny * nx;
    q.ppt = (ny + rops->row_lines - 1) / rops->row_lines;
    q.ppt_max = q.ppt;
    q.field = (float2 *)(d.base + kNaField);
    q.tf = (float *)(d.base + kNaTf);
    q.w = algo == HG_WGS ? (float *)(d.base + kNaW) : nullptr;
    q.part = (double *)(d.base + kNaPart);
    q.metrics = (double *)(d.base + kNaMetrics);
    q.sum_part = (double *)(d.base + kNaSumPart);
    q.scale = (double *)(d.base + kNaScale);
    q.err = (unsigned *)(d.base + kNaErr);
    q.twx = (float2 *)(d.base + kNaTwx);
    q.twy = (float2 *)(d.base + kNaTwy);
    q.lvl = (float2 *)(d.base + kNaLvl);

    // This call's tables, built on the host stack and copied into the region
    // in stream order (the copy has read the stack array when it returns).
    float2 hx[kNaSide], hy[kNaSide], hl[256];
    na_twiddles(nx, hx);
    na_twiddles(ny, hy);
    {
        const long double two_pi = 6.283185307179586476925286766559005768L;
        for (int l = 0; l < q.levels; ++l) {
            long double a = two_pi * (long double)l / (long double)q.levels;
            hl[l] = make_float2((float)cosl(a), (float)sinl(a));
        }
    }
    HG_CK(cudaMemcpyAsync(q.twx, hx, sizeof(float2) * nx, cudaMemcpyHostToDevice, s));
    HG_CK(cudaMemcpyAsync(q.twy, hy, sizeof(float2) * ny, cudaMemcpyHostToDevice, s));
    HG_CK(cudaMemcpyAsync(q.lvl, hl, sizeof(float2) * q.levels, cudaMemcpyHostToDevice, s));
    HG_CK(cudaMemsetAsync(q.err, 0, sizeof(unsigned), s));  // the one piece that starts at zero

    const double invN = 1.0 / (double)q.npx;
    auto reduce = [&](int k) {  // metrics of iteration k -> mse_out[k]
        k_reduce<<<1, 128, 0, s>>>(q.part, 1, 1, q.ppt_max, q.ppt, q.ppt, invN, q.metrics,
                                   mse_out ? mse_out + k : nullptr);
    };
    enqueue_prep(&q, target);
    if (q.w) k_fill<<<ew_grid(&q, q.npx), 256, 0, s>>>(q.w, q.npx, 1.f);
    RowArgs ra = row_args(&q);
    ra.phase = init_phase;
    launch_row(&q, ROW_HEAD, ra, s);
    ColArgs ca = col_args(&q);
    RowArgs ri = row_args(&q);
    ri.part = q.part;
    for (int k = 0; k + 1 < iters; ++k) {
        launch_col(&q, col_role_gs(&q), ca, s);
        launch_row(&q, ROW_ITER, ri, s);
        reduce(k);
    }
    ca.holo = holo_out;
    launch_col(&q, col_role_gs(&q), ca, s);
    launch_row(&q, ROW_TAIL, ri, s);
    reduce(iters - 1);
    HG_CK(cudaGetLastError());

    unsigned e = 0;
    HG_CK(cudaMemcpyAsync(&e, q.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HG_CK(cudaStreamSynchronize(s));
    if (e & ERR_BAD_VALUE) return HG_ERR_INVALID_ARG;
    if (e & ERR_ZERO_ENERGY) return HG_ERR_NUMERIC;
    return HG_OK;
}
