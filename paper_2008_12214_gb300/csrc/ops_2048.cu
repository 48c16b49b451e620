// Transform plans for 2048-sample lines.  Generic passes: 32 x 8 x 8, 64
// threads per line.  TMA-fed candidates: 16 x 16 x 8 with 16 samples per
// thread, and 32 x 8 x 8 with 32 samples per thread.
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o2048 = OpsImpl<Plan<2048, 64, 32, 32, 8, 8>, 4, 8, true>::make();
PipeOps p2048a = PipeImpl<Plan<2048, 128, 16, 16, 16, 8>, 1, 4, 2, 4, Plan<2048, 128, 16, 16, 16, 8>, 4, 1,
                          3, 4, 256>::make("2048:r16x16x8e16");
PipeOps p2048b = PipeImpl<Plan<2048, 64, 32, 32, 8, 8>, 1, 4, 2, 5, Plan<2048, 64, 32, 32, 8, 8>, 4, 1, 3,
                          5, 256>::make("2048:r32x8x8e32");
// paired rows with the Hermitian column-pair pass (binary loop): 4 columns
// with 16 samples per thread, or 8 columns with 32 samples per thread
using Herm2048a = HermImpl<Plan<2048, 128, 16, 16, 16, 8>, 4, 3, 4, 256>;
using Herm2048b = HermImpl<Plan<2048, 64, 32, 32, 8, 8>, 8, 3, 5, 256>;
PipeOps p2048c = PairedOps<PairImpl<Plan<2048, 128, 16, 16, 16, 8>, 3, 2, 4>, &p2048a, Herm2048a>::make(
    "2048:pair16x16x8e16+c16x16x8e16");
PipeOps p2048d = PairedOps<PairImpl<Plan<2048, 128, 16, 16, 16, 8>, 3, 2, 4>, &p2048a, Herm2048b>::make(
    "2048:pair16x16x8e16+c16x16x8e16/h32");
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
