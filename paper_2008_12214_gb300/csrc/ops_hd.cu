// Transform plans for the 1080 x 1920 display format (radix 2/3/5).
// Generic passes: 1080 = 30 x 6 x 6 (36 threads per line), 1920 = 30 x 8 x 8
// (64 threads per line; its last stage returns through shared memory).
// TMA-fed variants: 1080-sample columns (8 per CTA, 288 threads, boxes of 180
// rows) with column-pair passes of 8 columns on a 15 x 8 x 9 plan (72 threads
// per column pair, stage roots reloaded per line), one CTA per SM at 168
// registers or two at 96 (with spills), 1920-sample columns (4 per CTA, boxes
// of 240 rows), and the paired row pass on 1920-sample rows (3 single-slot
// lines of 128 threads, 15 x 16 x 8, reloaded roots: 168 registers; 0.146 ms
// per launch at 16 fields, against 0.161 for 2 lines of two slots).
// Measured at 16 fields of 1080 x 1920 (ms per launch): column pairs at two
// CTAs per SM 0.155 against 0.171 at one; 4 row lines at 128 registers (0.6 KB
// of spill per thread) and 2 lines at two CTAs per SM (128 registers, 0.9 KB
// of spill) lost to 3 lines, and 16-column pairs (96 registers) lost to the
// two-CTA 8-column pass.  The 30-samples-per-thread plans spill
// as TMA-fed paired or column-pair passes (255 and 168 registers plus 0.8-0.9
// KB per thread) and measured 1.6x (rows) and 1.2x (column pairs) slower.
#include "hg_pipe.cuh"

namespace hg {
namespace {
using P1080 = Plan<1080, 36, 30, 30, 6, 6>;
using P1080b = Plan<1080, 72, 16, 15, 8, 9>;
using P1920 = Plan<1920, 64, 30, 30, 8, 8>;
using P1920b = Plan<1920, 128, 16, 15, 16, 8>;
LineOps o1080 = OpsImpl<P1080, 8, 16>::make();
LineOps o1920 = OpsImpl<P1920, 4, 8>::make();
PipeOps p1080c = PipeImpl<P1080, 0, 1, 1, 3, P1080, 8, 1, 3, 3, 180>::make("1080:c30x6x6");
PipeOps p1080k = WithHerm<&p1080c, HermImpl<Reload<P1080b>, 8, 3, 0, 180>>::make("1080:c30x6x6/h15c8");
PipeOps p1080n = WithHerm<&p1080c, HermImpl<Reload<P1080b>, 8, 3, 0, 180, 2>>::make("1080:c30x6x6/h15c8x2");
PipeOps p1920c = PipeImpl<P1920, 0, 1, 1, 4, P1920, 4, 1, 3, 4, 240>::make("1920:c30x8x8");
PipeOps p1920r = PairedOps<PairImpl<Reload<P1920b>, 3, 1, 0>, &p1920c>::make("1920:pair15x16x8w12+c30x8x8");
}  // namespace

const LineOps *ops_hd(int n) {
    switch (n) {
        case 1080: return &o1080;
        case 1920: return &o1920;
        default: return nullptr;
    }
}

int pipe_ops_hd(int n, const PipeOps **out, int max) {
    int k = 0;
    if (n == 1080) {
        if (k < max) out[k++] = &p1080k;
        if (k < max) out[k++] = &p1080n;
    }
    if (n == 1920) {
        if (k < max) out[k++] = &p1920c;
        if (k < max) out[k++] = &p1920r;
    }
    return k;
}
}  // namespace hg
