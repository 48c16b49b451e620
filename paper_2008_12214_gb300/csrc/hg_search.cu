// hg_search.cu -- direct search and simulated annealing (Section 3.3); see
// hg_search.cuh for the arithmetic and the shared-memory layout.
#include "hg_search.cuh"

namespace hg {
namespace {

// Sums four per-thread floats over the block (warps in double) and returns
// the totals to every thread.  All threads must call.
__device__ void search_sum4(float v0, float v1, float v2, float v3, double *dred, double out[4]) {
    double d[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
        for (int m = 0; m < 4; ++m) d[m] += __shfl_down_sync(0xffffffffu, d[m], off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < 4; ++m) dred[warp * 4 + m] = d[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        double s = 0;
        for (int w = 0; w < nw; ++w) s += dred[w * 4 + m];
        out[m] = s;
    }
    __syncthreads();
}

// KK trials per pass over the pixels: SEARCH_K for direct search, whose trials
// are mostly rejected, 1 for annealing, which accepts too many for speculation
// to pay.
template <int KK>
__global__ void __launch_bounds__(SEARCH_MAX_THREADS) k_search(const SearchArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int ny = a.ny, nx = a.nx, N = ny * nx, T = blockDim.x, tid = threadIdx.x, item = blockIdx.x;
    float2 *twx = reinterpret_cast<float2 *>(sm);
    float2 *twy = reinterpret_cast<float2 *>(sm + a.off_twy);
    float2 *R = reinterpret_cast<float2 *>(sm + a.off_R);
    float *G = reinterpret_cast<float *>(sm + a.off_T);  // 2 (I - T^2) per replay pixel
    float *red = reinterpret_cast<float *>(sm + a.off_red);
    double *dred = reinterpret_cast<double *>(sm + a.off_dred);
    uint8_t *hq = sm + a.off_holo;
    uint2 *rnd = reinterpret_cast<uint2 *>(sm + a.off_rnd);
    const size_t base = (size_t)item * N;
    for (int i = tid; i < nx; i += T) twx[i] = a.twx[i];
    for (int i = tid; i < ny; i += T) twy[i] = a.twy[i];
    for (int k = tid; k < N; k += T) {
        R[k] = a.R0[base + k];
        hq[k] = a.holo[base + k];
    }
    __syncthreads();
    // pixel j of this thread: k = tid + T j, replay column ix, row iy0 + rstep j
    const int ix = tid % nx, iy0 = tid / nx, rstep = T / nx;
    const int kx = (ix - nx / 2 + nx) % nx, ky0 = (iy0 - ny / 2 + ny) % ny, rstep_m = rstep % ny;
    const int J = a.per_thread, nw = T >> 5, lane = tid & 31, warp = tid >> 5;
    const bool full = J * T == N;  // every thread owns J pixels

    // metrics of the current R, and G = 2 (I - T^2) recomputed from it (which
    // also clears the rounding the in-place updates of G accumulate)
    auto metrics = [&](double out[4]) {
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
        for (int j = 0; j < J; ++j) {
            const int k = tid + T * j;
            if (k >= N) break;
            const int iy = k / nx, ixk = k - iy * nx;
            const int yc = (iy + ny - ny / 2) % ny, xc = (ixk + nx - nx / 2) % nx;  // DFT index
            const float t = __ldg(a.T + base + (size_t)yc * nx + xc);
            const float2 r = R[k];
            const float e2 = fmaf(r.x, r.x, r.y * r.y), I = e2 * a.invN;
            const float d = I - t * t, am = sqrtf(I) - t;
            G[k] = 2.f * d;
            m0 = fmaf(d, d, m0);
            m1 = fmaf(am, am, m1);
            if (t > 0.f) m2 += e2;
            m3 += e2;
        }
        search_sum4(m0, m1, m2, m3, dred, out);
    };
    const bool need_rand = !a.binary || a.tau0 > 0.0;
    double g[4];
    metrics(g);
    const double mse0 = g[0] / N;
    int buf = 0;
    for (int s = 0; s < a.sweeps; ++s) {
        const float tau = (float)(a.tau0 * mse0 * pow(a.alpha, (double)s));
        int accepted = 0;
        int eyb = 0, st = 0;  // (ky0 y) mod ny and (rstep y) mod ny
        for (int y = 0; y < ny; ++y) {
            int ex = 0;  // (kx x) mod nx
            if (need_rand) {
                // the row's random words, drawn once by the block; every thread read
                // the previous row's before the last trial's barrier
                for (int xx = tid; xx < nx; xx += T)
                    rnd[xx] = philox_words01((uint32_t)(y * nx + xx), (uint32_t)s, (uint32_t)item, 2u, a.seed_lo,
                                             a.seed_hi);
                __syncthreads();
            }
            // KK trials (pixels x0 .. x0 + kb - 1 of the row) are evaluated from the
            // same state in one pass; the first accepted one is applied and the search
            // resumes after it, so every decision is the sequential search's
            {
                for (int x0 = 0; x0 < nx;) {
                    const int kb = min(KK, nx - x0);
                    const float s2 = 2.f * a.invN;
                    float2 c2[KK];
                    float cc[KK], part[KK];
                    int exs[KK];        // x twiddle index of each trial
                    unsigned qpk = 0u;  // each trial's current level, one byte per trial
                    float2 c1 = make_float2(0.f, 0.f);  // KK == 1: the trial's dR coefficient
                    int qn[KK];
                    float u[KK];  // acceptance draws
                    int exk = ex;
#pragma unroll
                    for (int k = 0; k < KK; ++k) {
                        part[k] = 0.f;
                        c2[k] = make_float2(0.f, 0.f);
                        exs[k] = 0;
                        cc[k] = 0.f;
                        qn[k] = 0;
                        u[k] = 0.f;
                        if (k < kb) {
                            const uint2 r = need_rand ? rnd[x0 + k] : make_uint2(0u, 0u);
                            u[k] = (float)(r.x >> 8) * (1.0f / 16777216.0f);
                            const int q = hq[y * nx + x0 + k];
                            qpk |= (unsigned)q << (8 * k);
                            float2 ds;
                            if (a.binary) {
                                qn[k] = 1 - q;
                                ds = make_float2(q ? 2.f : -2.f, 0.f);
                            } else {
                                qn[k] = (q + 1 + (int)(r.y % (uint32_t)(a.levels - 1))) % a.levels;
                                const float2 l1 = __ldg(a.lvl + qn[k]), l0 = __ldg(a.lvl + q);
                                ds = make_float2(l1.x - l0.x, l1.y - l0.y);
                            }
                            // dR_i = c w_i with |w_i| = 1, so the intensity change is
                            // a_i = Re(R_i conj(w_i) conj(c)) 2 / N + |c|^2 / N
                            const float2 wx = twx[exk];
                            const float2 ck = make_float2((ds.x * wx.x - ds.y * wx.y) * a.invSqrtN,
                                                          (ds.x * wx.y + ds.y * wx.x) * a.invSqrtN);
                            c2[k] = make_float2(ck.x * s2, ck.y * s2);
                            cc[k] = fmaf(ck.x, ck.x, ck.y * ck.y) * a.invN;
                            exs[k] = exk;
                            if constexpr (KK == 1) c1 = ck;
                            exk += kx;
                            if (exk >= nx) exk -= nx;
                        }
                    }
                    int ey = eyb;
                    for (int j = 0; j < J; ++j) {
                        const int i = tid + T * j;
                        if (full || i < N) {
                            const float2 w = twy[ey];
                            const float2 rv = R[i];
                            const float g = G[i];
                            const float zx = fmaf(rv.x, w.x, rv.y * w.y), zy = fmaf(rv.y, w.x, -rv.x * w.y);
#pragma unroll
                            for (int k = 0; k < KK; ++k) {
                                const float aa = fmaf(zx, c2[k].x, fmaf(zy, c2[k].y, cc[k]));
                                part[k] = fmaf(aa, g + aa, part[k]);
                            }
                        }
                        ey += st;
                        if (ey >= ny) ey -= ny;
                    }
#pragma unroll
                    for (int k = 0; k < KK; ++k) {
#pragma unroll
                        for (int off = 16; off; off >>= 1) part[k] += __shfl_down_sync(0xffffffffu, part[k], off);
                        if (lane == 0) red[(buf * SEARCH_K + k) * 32 + warp] = part[k];
                    }
                    __syncthreads();
                    int jacc = -1;
                    for (int k = 0; k < kb; ++k) {
                        float dE = 0.f;
                        for (int w = 0; w < nw; ++w) dE += red[(buf * SEARCH_K + k) * 32 + w];
                        dE *= a.invN;
                        if (dE < 0.f || (tau > 0.f && u[k] < expf(-dE / tau))) {
                            jacc = k;
                            break;
                        }
                    }
                    buf ^= 1;
                    if (jacc >= 0) {
                        float2 c2j = c2[0];
                        float ccj = cc[0];
                        int qj = qn[0], exj = exs[0];
#pragma unroll
                        for (int k = 1; k < KK; ++k)
                            if (k == jacc) {
                                c2j = c2[k];
                                ccj = cc[k];
                                qj = qn[k];
                                exj = exs[k];
                            }
                        // the accepted trial's dR coefficient, as computed for its evaluation
                        // (its old level was read before the barrier: thread 0 rewrites it below)
                        float2 cj = c1;
                        if constexpr (KK > 1) {
                            const int q = (int)((qpk >> (8 * jacc)) & 0xffu);
                            float2 ds;
                            if (a.binary) {
                                ds = make_float2(q ? 2.f : -2.f, 0.f);
                            } else {
                                const float2 l1 = __ldg(a.lvl + qj), l0 = __ldg(a.lvl + q);
                                ds = make_float2(l1.x - l0.x, l1.y - l0.y);
                            }
                            const float2 wx = twx[exj];
                            cj = make_float2((ds.x * wx.x - ds.y * wx.y) * a.invSqrtN,
                                             (ds.x * wx.y + ds.y * wx.x) * a.invSqrtN);
                        }
                        ey = eyb;
                        for (int j = 0; j < J; ++j) {
                            const int i = tid + T * j;
                            if (full || i < N) {
                                const float2 w = twy[ey];
                                const float2 rv = R[i];
                                const float zx = fmaf(rv.x, w.x, rv.y * w.y), zy = fmaf(rv.y, w.x, -rv.x * w.y);
                                G[i] += 2.f * fmaf(zx, c2j.x, fmaf(zy, c2j.y, ccj));  // I gains a_i
                                R[i] = make_float2(rv.x + (cj.x * w.x - cj.y * w.y), rv.y + fmaf(cj.x, w.y, cj.y * w.x));
                            }
                            ey += st;
                            if (ey >= ny) ey -= ny;
                        }
                        if (tid == 0) hq[y * nx + x0 + jacc] = (uint8_t)qj;
                        ++accepted;
                    }
                    const int adv = jacc >= 0 ? jacc + 1 : kb;
                    for (int k = 0; k < adv; ++k) {
                        ex += kx;
                        if (ex >= nx) ex -= nx;
                    }
                    x0 += adv;
                }
            }
            eyb += ky0;
            if (eyb >= ny) eyb -= ny;
            st += rstep_m;
            if (st >= ny) st -= ny;
        }
        metrics(g);
        if (tid == 0) {
            double *o = a.metrics + ((size_t)item * a.sweeps + s) * 4;
            o[0] = g[0] / N;
            o[1] = g[1] / N;
            o[2] = g[3] > 0 ? g[2] / g[3] : 0.0;
            o[3] = accepted;
            if (a.mse_out) a.mse_out[(size_t)item * a.sweeps + s] = o[0];
        }
    }
    __syncthreads();
    for (int k = tid; k < N; k += T) a.holo[base + k] = hq[k];
}

bool g_search_attr[64][2];

}  // namespace

cudaError_t search_launch(const SearchArgs &a, const SearchLayout &L, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int spec = a.tau0 > 0.0 ? 0 : 1;
    const void *fn = spec ? (const void *)k_search<SEARCH_K> : (const void *)k_search<1>;
    if (!g_search_attr[dev][spec]) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEARCH_MAX_SMEM);
        if (e != cudaSuccess) return e;
        g_search_attr[dev][spec] = true;
    }
    if (spec) k_search<SEARCH_K><<<a.items, L.threads, L.bytes, s>>>(a);
    else k_search<1><<<a.items, L.threads, L.bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hg
