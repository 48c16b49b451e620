// Further TMA-fed candidates for 1024-sample lines (tile shapes): two column
// groups of 4 columns with 3-deep rings, and the paired row pass with 4 groups
// and 3-deep rings.  Kept in their own translation unit to keep builds parallel.
#include "hg_pipe.cuh"

namespace hg {
namespace {
PipeOps p1024f = PipeImpl<Plan<1024, 64, 16, 16, 16, 4>, 1, 8, 2, 4, Plan<1024, 32, 32, 32, 32>, 4, 2, 3, 5,
                          256>::make("1024:r16x16x4e16+c32x32e32x4col2grp");
PipeOps p1024g = PairedOps<PairImpl<Plan<1024, 64, 16, 16, 16, 4>, 4, 3, 4>, &p1024f>::make(
    "1024:pair16x16x4e16d3+c32x32e32x4col2grp");
}  // namespace

int pipe_ops_1024x(int n, const PipeOps **out, int max) {
    if (n != 1024) return 0;
    const PipeOps *c[] = {&p1024f, &p1024g};
    int k = 0;
    for (const PipeOps *o : c)
        if (k < max) out[k++] = o;
    return k;
}
}  // namespace hg
