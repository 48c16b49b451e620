// Transform plans for 1024-sample lines.  Generic passes: 32 x 32, one warp
// per row, 32 samples per thread, 16 columns per CTA.  TMA-fed candidates
// (the autotuner picks per pass): unpaired 32 x 32 and 16 x 16 x 4 passes
// (L-level and modulated plans), and for the binary loop paired rows with a
// column-pair pass, on plans of 16 samples per thread (16 x 16 x 4, 64
// threads per line) or 8 (8 x 4 x 4 x 8, 128 threads per line).
#include "hg_pipe.cuh"

namespace hg {
namespace {
using P32 = Plan<1024, 32, 32, 32, 32>;
using P16 = Plan<1024, 64, 16, 16, 16, 4>;
using P8 = Plan<1024, 128, 8, 8, 4, 4, 8>;
LineOps o1024 = OpsImpl<P32, 8, 16, true>::make();
PipeOps p1024a = PipeImpl<P32, 1, 8, 2, 5, P32, 8, 1, 3, 5, 256>::make("1024:r32x32e32");
PipeOps p1024b = PipeImpl<P16, 1, 8, 2, 4, P16, 8, 1, 3, 4, 256>::make("1024:r16x16x4e16");
// paired rows (6 lines of 64 threads, 12 warps; 5 or 7 lines of 128 threads,
// 20 or 28 warps) with the column-pair pass of 16 columns x 32 samples (8
// warps), 16 columns x 16 samples (16 warps), 8 columns x 16 samples (two
// CTAs of 8 warps) or 8 columns x 8 samples (16 warps)
PipeOps p1024c = PairedOps<PairImpl<P16, 6, 2, 4>, &p1024a, NoPack, HermImpl<P32, 16, 3, 5, 256>>::make(
    "1024:pair16x16x4e16+c32x32e32/h32");
PipeOps p1024d =
    PairedOps<PairImpl<P8, 5, 2, 3>, &p1024a, NoPack, HermImpl<Reload<P16>, 16, 3, 4, 256>>::make(
        "1024:pair8x4x4x8e8w20+c32x32e32/h16c16");
PipeOps p1024e =
    PairedOps<PairImpl<P8, 7, 2, 3>, &p1024a, NoPack, HermImpl<Reload<P16>, 8, 3, 4, 256, 2>>::make(
        "1024:pair8x4x4x8e8w28+c32x32e32/h16c8x2");
PipeOps p1024f =
    PairedOps<PairImpl<Reload<P16>, 7, 2, 4>, &p1024a, NoPack, HermImpl<Reload<P8>, 8, 3, 3, 256>>::make(
        "1024:pair16x16x4e16w14+c32x32e32/h8c8");
}  // namespace

const LineOps *ops_1024(int n) { return n == 1024 ? &o1024 : nullptr; }

int pipe_ops_1024(int n, const PipeOps **out, int max) {
    if (n != 1024) return 0;
    const PipeOps *c[] = {&p1024a, &p1024b, &p1024c, &p1024d, &p1024e, &p1024f};
    int k = 0;
    for (const PipeOps *o : c)
        if (k < max) out[k++] = o;
    return k;
}
}  // namespace hg
