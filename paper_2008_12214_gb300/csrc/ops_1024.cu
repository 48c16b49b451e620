// Transform plans for 1024-sample lines.  Generic passes: 32 x 32, one warp
// per row, 32 samples per thread, 16 columns per CTA.  TMA-fed candidates:
// 32 x 32 with 32 samples per thread (8 warps per SM), and 16 x 16 x 4 with 16
// samples per thread (16 warps per SM); the autotuner picks per pass.
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o1024 = OpsImpl<Plan<1024, 32, 32, 32, 32>, 8, 16, true>::make();
PipeOps p1024a = PipeImpl<Plan<1024, 32, 32, 32, 32>, 1, 8, 2, 5, Plan<1024, 32, 32, 32, 32>, 8, 1, 3, 5,
                          256>::make("1024:r32x32e32");
PipeOps p1024b = PipeImpl<Plan<1024, 64, 16, 16, 16, 4>, 1, 8, 2, 4, Plan<1024, 64, 16, 16, 16, 4>, 8, 1, 3,
                          4, 256>::make("1024:r16x16x4e16");
// paired rows with the Hermitian column-pair pass: 16 columns with 32
// samples per thread, or 8 columns with 16 samples per thread (256 threads)
using Herm1024a = HermImpl<Plan<1024, 32, 32, 32, 32>, 16, 3, 5, 256>;
using Herm1024b = HermImpl<Plan<1024, 64, 16, 16, 16, 4>, 8, 3, 4, 256>;
PipeOps p1024c = PairedOps<PairImpl<Plan<1024, 64, 16, 16, 16, 4>, 6, 2, 4>, &p1024a, NoPack, Herm1024b>::make(
    "1024:pair16x16x4e16+c32x32e32");
PipeOps p1024d = PairedOps<PairImpl<Plan<1024, 32, 32, 32, 32>, 6, 2, 5>, &p1024a, NoPack, Herm1024a>::make(
    "1024:pair32x32e32+c32x32e32");
PipeOps p1024f = PairedOps<PairImpl<Plan<1024, 64, 16, 16, 16, 4>, 6, 2, 4>, &p1024a, NoPack, Herm1024a>::make(
    "1024:pair16x16x4e16+c32x32e32/h16");
PipeOps p1024e =
    PairedOps<PairImpl<Plan<1024, 64, 16, 16, 16, 4>, 6, 2, 4>, &p1024a,
              PackImpl<Plan<1024, 32, 32, 32, 32>, Plan<1024, 64, 16, 16, 16, 4>, 8, 1, 3, 5, 4, 256>>::
        make("1024:pair16x16x4e16+pack32x32/16x16x4");
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
