// Transform plan for 2048-sample lines: 32 x 8 x 8, 64 threads per line.
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o2048 = OpsImpl<Plan<2048, 64, 32, 32, 8, 8>, 4, 8>::make();
PipeOps p2048 = PipeImpl<Plan<2048, 128, 16, 16, 16, 8>, 1, 4, 2, 4, Plan<2048, 128, 16, 16, 16, 8>, 4, 1, 3, 4, 256>::make();
}  // namespace

const LineOps *ops_2048(int n) { return n == 2048 ? &o2048 : nullptr; }

const PipeOps *pipe_ops_2048(int n) { return n == 2048 ? &p2048 : nullptr; }
}  // namespace hg
