// Transform plans for 256- and 512-sample lines.
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o256 = OpsImpl<Plan<256, 16, 16, 16, 16>, 16, 16>::make();
LineOps o512 = OpsImpl<Plan<512, 16, 32, 32, 16>, 16, 16>::make();
PipeOps p256 = PipeImpl<Plan<256, 16, 16, 16, 16>, 2, 12, 3, 4, Plan<256, 16, 16, 16, 16>, 8, 3, 4, 4, 256>::make();
PipeOps p512 = PipeImpl<Plan<512, 16, 32, 32, 16>, 2, 8, 2, 5, Plan<512, 16, 32, 32, 16>, 8, 2, 3, 5, 256>::make();
}  // namespace

const LineOps *ops_mid(int n) {
    switch (n) {
        case 256: return &o256;
        case 512: return &o512;
        default: return nullptr;
    }
}

const PipeOps *pipe_ops_mid(int n) {
    switch (n) {
        case 256: return &p256;
        case 512: return &p512;
        default: return nullptr;
    }
}
}  // namespace hg
