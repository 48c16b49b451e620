// Tensor-core row pass (1024- and 2048-sample rows): instantiations,
// launchers and the DFT-32 operand matrices.
#include <cmath>

#include "hg_pipe.cuh"
#include "hg_tc.cuh"

namespace hg {

namespace {
template <int PREC>
constexpr int tc_smem() {
    return TcLayout<TcPrec<PREC>::SPLIT>::SMEM;
}

template <int PREC, int NX>
cudaError_t set_attr_n() {
    cudaError_t e = cudaFuncSetAttribute((const void *)k_row_tc<PREC, ROW_ITER, NX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<PREC>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)k_row_tc<PREC, ROW_TAIL, NX>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<PREC>());
    return e;
}

// resident CTAs per SM of each precision's kernel for 1024- and 2048-sample
// rows, per device (set by tc_init)
int g_tc_occ[64][5][2];
int g_tc_nsm[64];

template <int PREC>
cudaError_t set_attr(int dev) {
    cudaError_t e = set_attr_n<PREC, 1024>();
    if (e == cudaSuccess) e = set_attr_n<PREC, 2048>();
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_tc_occ[dev][PREC][0], k_row_tc<PREC, ROW_ITER, 1024>,
                                                          128, tc_smem<PREC>());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_tc_occ[dev][PREC][1], k_row_tc<PREC, ROW_ITER, 2048>,
                                                          128, tc_smem<PREC>());
    return e;
}

// The grid fills the SMs with this precision's resident CTAs (the caller's
// grid assumes the hi+lo layout's occupancy).
template <int PREC>
void launch(int role, const RowArgs &a, const TcArgs &ta, int grid, cudaStream_t s) {
    int dev = 0;
    const int wide = a.nx == 2048;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && g_tc_occ[dev][PREC][wide] > 0 &&
        g_tc_nsm[dev] > 0) {
        const long work = (long)a.items * (a.ny / (wide ? 2 : 4));
        const long g = (long)g_tc_occ[dev][PREC][wide] * g_tc_nsm[dev];
        grid = (int)(g < work ? g : (work > 0 ? work : 1));
    }
    constexpr int SM = tc_smem<PREC>();
    if (a.nx == 2048) {
        if (role == ROW_ITER) k_row_tc<PREC, ROW_ITER, 2048><<<grid, 128, SM, s>>>(a, ta);
        else k_row_tc<PREC, ROW_TAIL, 2048><<<grid, 128, SM, s>>>(a, ta);
    } else {
        if (role == ROW_ITER) k_row_tc<PREC, ROW_ITER, 1024><<<grid, 128, SM, s>>>(a, ta);
        else k_row_tc<PREC, ROW_TAIL, 1024><<<grid, 128, SM, s>>>(a, ta);
    }
}

uint16_t bits_of(float x, int prec, float *back) {
    if (prec <= 2) {
        __half h = __float2half_rn(x);
        *back = __half2float(h);
        return *reinterpret_cast<uint16_t *>(&h);
    }
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    *back = __bfloat162float(b);
    return *reinterpret_cast<uint16_t *>(&b);
}
}  // namespace

cudaError_t tc_init(int *blocks_per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    e = cudaDeviceGetAttribute(&g_tc_nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = set_attr<1>(dev);
    if (e == cudaSuccess) e = set_attr<2>(dev);
    if (e == cudaSuccess) e = set_attr<3>(dev);
    if (e == cudaSuccess) e = set_attr<4>(dev);
    if (e == cudaSuccess) *blocks_per_sm = g_tc_occ[dev][1][0];
    return e;
}

void tc_launch_row(int prec, int role, const RowArgs &a, const TcArgs &ta, int grid, cudaStream_t s) {
    switch (prec) {
        case 1: launch<1>(role, a, ta, grid, s); break;
        case 2: launch<2>(role, a, ta, grid, s); break;
        case 3: launch<3>(role, a, ta, grid, s); break;
        default: launch<4>(role, a, ta, grid, s); break;
    }
}

// B[2k + c_out][2n + c_in] for W = exp(DIR 2 pi i n k / 32): the real form of
// y_k = sum_n W^{nk} x_n with interleaved (re, im).  Angles reduced as exact
// integers and evaluated in long double; hi = round(B), lo = round(B - hi).
void tc_make_bmats(int prec, uint16_t *out) {
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int d = 0; d < 2; ++d) {
        const int dir = d == 0 ? -1 : +1;
        uint16_t *hi = out + (2 * d) * 4096, *lo = out + (2 * d + 1) * 4096;
        for (int k = 0; k < 32; ++k)
            for (int n = 0; n < 32; ++n) {
                const long double ang = two_pi * (long double)((n * k) % 32) / 32.0L;
                const float re = (float)cosl(ang), im = (float)(dir * sinl(ang));
                const float vals[2][2] = {{re, -im}, {im, re}};  // [c_out][c_in]
                for (int co = 0; co < 2; ++co)
                    for (int ci = 0; ci < 2; ++ci) {
                        const int r = 2 * k + co, c = 2 * n + ci;
                        const int idx = ((r >> 3) * 1024 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2) / 2;
                        float back;
                        hi[idx] = bits_of(vals[co][ci], prec, &back);
                        float b2;
                        lo[idx] = bits_of(vals[co][ci] - back, prec, &b2);
                    }
            }
    }
}

}  // namespace hg
