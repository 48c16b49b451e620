// Transform plans for 1024-sample lines.  Generic passes: 32 x 32, one warp
// per row, 32 samples per thread, 16 columns per CTA.  TMA-fed candidates
// (the autotuner picks per pass): unpaired 32 x 32 and 16 x 16 x 4 passes
// (L-level and modulated plans), and for the binary loop paired rows (6 lines
// of 64 threads, 16 x 16 x 4) with a column-pair pass of 8 columns x 16
// samples per thread (stage roots reloaded per line: 128 registers, two CTAs
// of 8 warps per SM, a ring of two slots: 0.187 ms per launch at 1024^2 x 64
// against 0.191 with three slots, 0.201-0.202 with the XOR swizzle over 8 or
// 32 addresses, 0.235 with four slots, which leave room for one CTA) or of 16
// columns x 32 samples (one CTA of 8 warps).
#include "hg_pipe.cuh"

namespace hg {
namespace {
using P32 = Plan<1024, 32, 32, 32, 32>;
using P16 = Plan<1024, 64, 16, 16, 16, 4>;
LineOps o1024 = OpsImpl<P32, 8, 16, true>::make();
PipeOps p1024a = PipeImpl<P32, 1, 8, 2, 5, P32, 8, 1, 3, 5, 256>::make("1024:r32x32e32");
PipeOps p1024b = PipeImpl<P16, 1, 8, 2, 4, P16, 8, 1, 3, 4, 256>::make("1024:r16x16x4e16");
PipeOps p1024c = PairedOps<PairImpl<P16, 6, 2, 4>, &p1024a, HermImpl<Reload<P16>, 8, 2, 4, 256, 2>>::make(
    "1024:pair16x16x4e16+c32x32e32/h16c8x2");
PipeOps p1024d = PairedOps<PairImpl<P16, 6, 2, 4>, &p1024a, HermImpl<P32, 16, 3, 5, 256>>::make(
    "1024:pair16x16x4e16+c32x32e32/h32c16");
}  // namespace

const LineOps *ops_1024(int n) { return n == 1024 ? &o1024 : nullptr; }

int pipe_ops_1024(int n, const PipeOps **out, int max) {
    if (n != 1024) return 0;
    const PipeOps *c[] = {&p1024a, &p1024b, &p1024c, &p1024d};
    int k = 0;
    for (const PipeOps *o : c)
        if (k < max) out[k++] = o;
    return k;
}
}  // namespace hg
