// Transform plans for 1024-sample lines.  Generic passes: 32 x 32, one warp
// per row, 32 samples per thread, 16 columns per CTA.  TMA-fed candidates
// (the autotuner picks per pass): unpaired 32 x 32 and 16 x 16 x 4 passes
// (L-level and modulated plans), and for the binary loop:
//  c: paired rows on 16 x 8 x 8 (64 threads per line) in 8 groups of one
//     ring slot each (16 warps per SM, stage roots reloaded per line: 128
//     registers), with column pairs of 8 columns x 16 samples (two CTAs of 8
//     warps per SM, two slots);
//  d: paired rows on 16 x 16 x 4 in 6 groups of two slots (12 warps, 168
//     registers) with column pairs of 16 columns x 32 samples.
//  f: the rows of e with a column pass for modulated plans: 4 columns per
//     group, two CTAs of 8 warps per SM, the group's illumination tile
//     staged in shared memory alongside the two-slot ring.
// Modulated Fresnel GS at 1024^2 x 64 (column ms): f 0.457; 4 columns in two
// groups per CTA 0.499, 8 columns 0.469; E read from global memory: generic
// 0.665, 4 columns in two groups 0.647, 8 columns 0.755.
// Measured at 1024^2 x 64 (row / column ms per launch): c 0.191 / 0.186,
// d 0.216 / 0.200; 16 x 8 x 8 rows in 6 groups of two slots 0.207, in 7 or
// 10 single-slot groups 0.215 and 0.222 (146 registers; 96 with spills);
// 16 x 16 x 4 rows in 8 single-slot groups 0.204; column pairs with three or
// four slots, or the XOR swizzle over 8 or 32 addresses, 0.191-0.235.
#include "hg_pipe.cuh"

namespace hg {
namespace {
using P32 = Plan<1024, 32, 32, 32, 32>;
using P16 = Plan<1024, 64, 16, 16, 16, 4>;
using P16b = Plan<1024, 64, 16, 16, 8, 8>;
LineOps o1024 = OpsImpl<P32, 8, 16, true>::make();
PipeOps p1024a = PipeImpl<P32, 1, 8, 2, 5, P32, 8, 1, 3, 5, 256>::make("1024:r32x32e32");
PipeOps p1024b = PipeImpl<P16, 1, 8, 2, 4, P16, 8, 1, 3, 4, 256>::make("1024:r16x16x4e16");
PipeOps p1024e = PipeImpl<Reload<P16b>, 1, 8, 1, 4, Reload<P16b>, 8, 1, 2, 4, 256>::make("1024:r16x8x8w16");
// modulated plans (complex fields): the rows of e, a column pass of 4 columns
// per group (two CTAs of 8 warps per SM) that stages E in shared memory
PipeOps p1024f = PipeImpl<Reload<P16b>, 1, 8, 1, 4, Reload<P16b>, 4, 1, 2, 4, 256, 2, true>::make("1024:r16x8x8w16+c4x2E");
PipeOps p1024c = PairedOps<PairImpl<Reload<P16b>, 8, 1, 4>, &p1024a, HermImpl<Reload<P16b>, 8, 2, 4, 256, 2>>::make(
    "1024:pair16x8x8w16+c32x32e32/h16c8x2");
PipeOps p1024d = PairedOps<PairImpl<P16, 6, 2, 4>, &p1024a, HermImpl<P32, 16, 3, 5, 256>>::make(
    "1024:pair16x16x4e16+c32x32e32/h32c16");
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
