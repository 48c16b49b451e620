// hg_search.cuh -- holographic search algorithms (Section 3.3): direct search
// and simulated annealing over single-pixel changes of a phase hologram.
//
// One CTA per target holds the replay field R (unitary, replay order), the
// target, the hologram and the twiddle tables in shared memory.  A sweep
// visits every SLM pixel (y, x) in raster order.  Changing that pixel's field
// by ds changes replay pixel (iy, ix), of frequency (ky, kx), by
// dR = ds W_ny^(ky y) W_nx^(kx x) / sqrt(N), and the intensity MSE by
// dE = mean(a (2 (I - T^2) + a)), a = (2 Re(R conj dR) + |dR|^2) / N,
// I = |R|^2 / N (a phase hologram keeps sum |R|^2 = N).  SEARCH_K
// consecutive trials are evaluated from the same state in one pass over the
// pixels; the first one accepted is applied and the next pass starts after
// it, so the decisions are those of the one-trial-at-a-time search.  Shared
// memory holds
// G = 2 (I - T^2) per replay pixel: an accepted change adds 2 a, and every
// sweep recomputes G from R and T.  Every thread sums
// its pixels' terms, warps reduce in float, and every thread adds the warp
// partials in the same order, so all threads take the same decision after
// one barrier per pass of SEARCH_K trials (the partials alternate between
// two buffers).
#pragma once
#include "hg_fft.cuh"

namespace hg {

constexpr int SEARCH_PX = 16;  // replay pixels per thread at most
constexpr int SEARCH_K = 4;    // trials evaluated per barrier
constexpr int SEARCH_MAX_THREADS = 1024;
constexpr size_t SEARCH_MAX_SMEM = 227 * 1024;

struct SearchArgs {
    int ny, nx, items;
    const float2 *R0;   // [items][ny][nx] replay of the initial hologram, replay order, unitary
    const float *T;     // prepared targets [items][ny][nx], DFT order, sum T^2 = 1
    uint8_t *holo;      // [items][ny][nx] SLM order: initial levels in, final levels out
                        // (T is read again at every sweep's metrics)
    const float2 *lvl;  // L-level phasors exp(2 pi i q / L)
    int levels, binary;
    const float2 *twx, *twy;  // W_n^e = exp(-2 pi i e / n)
    int sweeps;
    double tau0, alpha;  // tau_s = tau0 MSE(initial) alpha^s; tau0 = 0: direct search
    uint32_t seed_lo, seed_hi;
    double *metrics;  // [items][sweeps][4] {intensity MSE, amplitude MSE, efficiency, accepted}
    double *mse_out;  // [items][sweeps] or null
    float invN, invSqrtN;
    // shared-memory layout (search_layout)
    int per_thread;
    unsigned off_twy, off_R, off_T, off_red, off_dred, off_rnd, off_holo;
};

struct SearchLayout {
    int threads, per_thread;
    size_t off_twy, off_R, off_T, off_red, off_dred, off_rnd, off_holo, bytes;
};

// Thread t holds replay pixels t + threads j (j < per_thread), so `threads`
// must be a multiple of nx (every thread stays in one replay column and
// shares its x twiddle) and of 32.  False when no layout fits.
inline bool search_layout(int ny, int nx, SearchLayout *L) {
    int a = 32, b = nx;
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    const long unit = 32L / a * nx;  // lcm(32, nx)
    const long N = (long)ny * nx;
    if (unit > SEARCH_MAX_THREADS) return false;
    long t = (N + SEARCH_PX - 1) / SEARCH_PX;
    t = (t + unit - 1) / unit * unit;
    if (t > SEARCH_MAX_THREADS) return false;
    L->threads = (int)t;
    L->per_thread = (int)((N + t - 1) / t);
    size_t o = 8 * (size_t)nx;
    L->off_twy = o;
    o += 8 * (size_t)ny;
    L->off_R = o;
    o += 8 * (size_t)N;
    L->off_T = o;
    o += 4 * (size_t)N;
    o = (o + 7) & ~(size_t)7;
    L->off_red = o;
    o += 2 * SEARCH_K * 32 * sizeof(float);
    L->off_dred = o;
    o += 32 * 4 * sizeof(double);
    L->off_rnd = o;  // Philox words 0 and 1 of one SLM row's trials
    o += 8 * (size_t)nx;
    L->off_holo = o;
    o += (size_t)N;
    L->bytes = o;
    return o <= SEARCH_MAX_SMEM;
}

// Enqueues the search on `s` (one CTA per item); sets the kernel's shared
// memory limit on first use per device.
cudaError_t search_launch(const SearchArgs &a, const SearchLayout &L, cudaStream_t s);

}  // namespace hg
