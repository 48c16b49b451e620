"""The learned warm start end to end (labels from the engine's own GS,
training through the tensor-core kernels, time-to-MSE evaluation), at a
size that trains in seconds.  GS started from the network's phase must
still reach plain GS's quality (GS remains the yardstick and the fallback);
the gain itself is printed and is measured at full size by bench.py."""
import numpy as np
import pytest
import torch

from paper_2008_12214_gb300 import hologen as hg
from paper_2008_12214_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu


def test_warm_start_trains_and_gs_from_it_reaches_plain_gs_quality():
    H = 128
    kind, L = hg.HG_SLM_LLEVEL, 256
    net, losses, secs = ws.train(H, H, 2048, batch=16, lr=1e-3, chunk=64, label_iters=200, label_start="fixed",
                                 slm_kind=kind, levels=L)
    try:
        assert np.isfinite(losses).all() and len(losses) == 2048 // 16
        assert np.mean(losses[-16:]) < np.mean(losses[:4]), losses
        ev = ws.evaluate(net, H, H, 32, ref_iters=100, max_iters=100, chunk=16, slm_kind=kind, levels=L)
    finally:
        net.close()
    print("warm start: median speedup %.2f, reached %.2f, median iterations %s, curves (warm, random) at 1/10/100:"
          % (ev["median_speedup"], ev["reached"], ev["median_warm_iters"]),
          [round(ev["rel_warm_curve"][i], 3) for i in (0, 9, 99)], [round(ev["rel_rand_curve"][i], 3) for i in (0, 9, 99)])
    assert ev["n"] == 32
    assert ev["rel_rand_curve"][-1] == pytest.approx(1.0, abs=1e-9)
    assert ev["rel_warm_curve"][-1] <= 1.05, ev["rel_warm_curve"][-1]
    assert ev["ms_cnn_batch"] > 0 and ev["ms_per_gs_iter_batch"] > 0
