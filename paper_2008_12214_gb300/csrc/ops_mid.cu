// Transform plans for 256- and 512-sample lines.
#include "hg_pipe.cuh"

namespace hg {
namespace {
LineOps o256 = OpsImpl<Plan<256, 16, 16, 16, 16>, 16, 16>::make();
LineOps o512 = OpsImpl<Plan<512, 16, 32, 32, 16>, 16, 16, true>::make();
PipeOps p256 = PipeImpl<Plan<256, 16, 16, 16, 16>, 2, 12, 3, 4, Plan<256, 16, 16, 16, 16>, 8, 3, 4, 4,
                         256>::make("256:r16x16e16");
PipeOps p512a = PipeImpl<Plan<512, 16, 32, 32, 16>, 2, 8, 2, 5, Plan<512, 16, 32, 32, 16>, 8, 2, 3, 5,
                          256>::make("512:r32x16e32");
PipeOps p512b = PipeImpl<Plan<512, 32, 16, 16, 16, 2>, 1, 16, 2, 4, Plan<512, 32, 16, 16, 16, 2>, 8, 2, 3,
                          4, 256>::make("512:r16x16x2e16");
// paired rows with the Hermitian column-pair pass (binary loop): 16 columns
// with 16 samples per thread, or 32 columns with 32 samples per thread
using Herm512a = HermImpl<Plan<512, 32, 16, 16, 16, 2>, 16, 3, 4, 256>;
using Herm512b = HermImpl<Plan<512, 16, 32, 32, 16>, 32, 3, 5, 256>;
PipeOps p512c = PairedOps<PairImpl<Plan<512, 32, 16, 16, 16, 2>, 12, 2, 4>, &p512a, Herm512a>::make(
    "512:pair16x16x2e16+c32x16e32");
PipeOps p512d = PairedOps<PairImpl<Plan<512, 32, 16, 16, 16, 2>, 12, 2, 4>, &p512a, Herm512b>::make(
    "512:pair16x16x2e16+c32x16e32/h32");
}  // namespace

const LineOps *ops_mid(int n) {
    switch (n) {
        case 256: return &o256;
        case 512: return &o512;
        default: return nullptr;
    }
}

int pipe_ops_mid(int n, const PipeOps **out, int max) {
    int k = 0;
    if (n == 256 && k < max) out[k++] = &p256;
    if (n == 512) {
        if (k < max) out[k++] = &p512a;
        if (k < max) out[k++] = &p512b;
        if (k < max) out[k++] = &p512c;
        if (k < max) out[k++] = &p512d;
    }
    return k;
}
}  // namespace hg
