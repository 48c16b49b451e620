// Transform plans for short lines (used by small fields and tests).
// Single-stage plans give each line to one thread (all samples in registers).
#include "hg_kernels.cuh"

namespace hg {
namespace {
template <int N>
using Single = Plan<N, 1, N, N>;

LineOps o4 = OpsImpl<Single<4>, 32, 32>::make();
LineOps o6 = OpsImpl<Single<6>, 32, 32>::make();
LineOps o8 = OpsImpl<Single<8>, 32, 32>::make();
LineOps o10 = OpsImpl<Single<10>, 32, 32>::make();
LineOps o12 = OpsImpl<Single<12>, 32, 32>::make();
LineOps o15 = OpsImpl<Single<15>, 32, 32>::make();
LineOps o16 = OpsImpl<Single<16>, 32, 32>::make();
LineOps o20 = OpsImpl<Single<20>, 32, 32>::make();
LineOps o30 = OpsImpl<Single<30>, 32, 32>::make();
LineOps o32 = OpsImpl<Single<32>, 32, 32>::make();
LineOps o60 = OpsImpl<Plan<60, 2, 30, 30, 2>, 16, 16>::make();
LineOps o64 = OpsImpl<Plan<64, 8, 8, 8, 8>, 8, 8>::make();
LineOps o96 = OpsImpl<Plan<96, 4, 24, 24, 4>, 8, 8>::make();
LineOps o128 = OpsImpl<Plan<128, 8, 16, 16, 8>, 8, 8>::make();
}  // namespace

const LineOps *ops_small(int n) {
    switch (n) {
        case 4: return &o4;
        case 6: return &o6;
        case 8: return &o8;
        case 10: return &o10;
        case 12: return &o12;
        case 15: return &o15;
        case 16: return &o16;
        case 20: return &o20;
        case 30: return &o30;
        case 32: return &o32;
        case 60: return &o60;
        case 64: return &o64;
        case 96: return &o96;
        case 128: return &o128;
        default: return nullptr;
    }
}
}  // namespace hg
