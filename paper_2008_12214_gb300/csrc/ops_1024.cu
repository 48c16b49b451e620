// Transform plan for 1024-sample lines: 32 x 32, one warp per row, 32
// samples per thread; the column pass takes 16 columns per CTA.
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o1024 = OpsImpl<Plan<1024, 32, 32, 32, 32>, 8, 16>::make();
PipeOps p1024 = PipeImpl<Plan<1024, 32, 32, 32, 32>, 1, 8, 2, 5, Plan<1024, 32, 32, 32, 32>, 8, 1, 3, 5, 256>::make();
}  // namespace

const LineOps *ops_1024(int n) { return n == 1024 ? &o1024 : nullptr; }

const PipeOps *pipe_ops_1024(int n) { return n == 1024 ? &p1024 : nullptr; }
}  // namespace hg
