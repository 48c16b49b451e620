// Transform plan for 2048-sample lines: 32 x 8 x 8, 64 threads per line.
#include "hg_kernels.cuh"

namespace hg {
namespace {
LineOps o2048 = OpsImpl<Plan<2048, 64, 32, 32, 8, 8>, 4, 8>::make();
}  // namespace

const LineOps *ops_2048(int n) { return n == 2048 ? &o2048 : nullptr; }
}  // namespace hg
