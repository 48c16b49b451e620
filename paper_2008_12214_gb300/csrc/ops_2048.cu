// Transform plans for 2048-sample lines.  Generic passes: 32 x 8 x 8, 64
// threads per line.  TMA-fed candidates: unpaired 16 x 16 x 8 with 16 samples
// per thread and 32 x 8 x 8 with 32, and two paired variants for the binary
// loop.
#include "hg_pipe.cuh"

namespace hg {
namespace {
using Q16 = Plan<2048, 128, 16, 16, 16, 8>;
using Q16b = Plan<2048, 128, 16, 16, 8, 16>;
LineOps o2048 = OpsImpl<Plan<2048, 64, 32, 32, 8, 8>, 4, 8, true>::make();
PipeOps p2048a = PipeImpl<Q16, 1, 4, 2, 4, Q16, 4, 1, 3, 4, 256>::make("2048:r16x16x8e16");
PipeOps p2048b = PipeImpl<Plan<2048, 64, 32, 32, 8, 8>, 1, 4, 2, 5, Plan<2048, 64, 32, 32, 8, 8>, 4, 1, 3,
                          5, 256>::make("2048:r32x8x8e32");
// paired rows with the Hermitian column-pair pass (binary loop):
//  c: rows on 16 x 16 x 8 in 3 groups of two ring slots (12 warps, 168
//     registers), column pairs of 4 columns x 16 samples (one CTA of 8 warps);
//  d: rows on 16 x 8 x 16 in 4 single-slot groups (16 warps, stage roots
//     reloaded: 128 registers), column pairs of 4 columns at two CTAs per SM
//     (two slots, reloaded roots, 128 registers).
// Measured at 2048^2 x 16 (batched iterations/s, 50 per run): c 2098, d 2439;
// 16 x 16 x 8 rows in 4 single-slot groups with d's column pairs 2410, in 3
// groups of two slots 2293.
PipeOps p2048c = PairedOps<PairImpl<Q16, 3, 2, 4>, &p2048a, HermImpl<Q16, 4, 3, 4, 256>>::make(
    "2048:pair16x16x8e16+c16x16x8e16/h16c4");
PipeOps p2048d = PairedOps<PairImpl<Reload<Q16b>, 4, 1, 4>, &p2048a, HermImpl<Reload<Q16>, 4, 2, 4, 256, 2>>::make(
    "2048:pair16x8x16w16+c16x16x8e16/h16c4x2");
}  // namespace

const LineOps *ops_2048(int n) { return n == 2048 ? &o2048 : nullptr; }

int pipe_ops_2048(int n, const PipeOps **out, int max) {
    if (n != 2048) return 0;
    const PipeOps *c[] = {&p2048a, &p2048b, &p2048c, &p2048d};
    int k = 0;
    for (const PipeOps *o : c)
        if (k < max) out[k++] = o;
    return k;
}
}  // namespace hg
