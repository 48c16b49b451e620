// Transform plans for the 1080 x 1920 display format (radix 2/3/5):
// 1080 = 30 x 6 x 6 (36 threads per line), 1920 = 30 x 8 x 8 (64 threads per
// line; its last stage returns through shared memory).
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o1080 = OpsImpl<Plan<1080, 36, 30, 30, 6, 6>, 8, 16>::make();
LineOps o1920 = OpsImpl<Plan<1920, 64, 30, 30, 8, 8>, 4, 8>::make();
}  // namespace

const LineOps *ops_hd(int n) {
    switch (n) {
        case 1080: return &o1080;
        case 1920: return &o1920;
        default: return nullptr;
    }
}

// The display-format lengths use the generic passes only.
int pipe_ops_hd(int, const PipeOps **, int) { return 0; }
}  // namespace hg
