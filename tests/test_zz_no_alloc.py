"""hg_run_noalloc, the run that keeps its work memory in the library's fixed
device region, against hg_run on a plan of batch 1 with the generic passes
(pipeline = 0), which it is documented to match.  Two calls in a row per
case, with different targets, so that state left in the region by one call
cannot hide.  The file name sorts last, so the suite also runs it after every
other GPU test; it also passes on its own in a fresh process, where its first
call does the per-device setup."""
import numpy as np
import pytest
import torch

from paper_2008_12214_gb300 import hologen as hg
from paper_2008_12214_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# ny, nx, slm kind, levels, algorithm, iterations, explicit initial phase
CASES = [
    (64, 64, hg.HG_SLM_BINARY, 2, hg.HG_GS, 6, True),
    (96, 128, hg.HG_SLM_LLEVEL, 4, hg.HG_WGS, 5, False),
    (512, 512, hg.HG_SLM_BINARY, 2, hg.HG_GS, 4, True),
]


def plan_run(ny, nx, kind, levels, algo, iters, T, P):
    plan = hg.Plan(ny, nx, 1, kind, levels, algo, pipeline=0)
    holo = torch.empty((1, ny, nx), dtype=torch.uint8, device=DEV)
    mse = torch.empty((1, iters), dtype=torch.float64, device=DEV)
    plan.run(T, P, iters, holo, mse)
    plan.sync()
    plan.close()
    return holo.cpu().numpy()[0], mse.cpu().numpy()[0]


@pytest.mark.parametrize("ny,nx,kind,levels,algo,iters,explicit", CASES)
def test_noalloc_run_matches_plan_run_on_two_calls_in_a_row(ny, nx, kind, levels, algo, iters, explicit):
    for call in range(2):
        seed = 1000 + 7 * call + ny
        T = torch.from_numpy(synth.target(ny, nx, seed)).to(DEV)
        P = torch.from_numpy(synth.init_phase(ny, nx, seed)).to(DEV) if explicit else None
        holo = torch.full((ny, nx), 255, dtype=torch.uint8, device=DEV)
        mse = torch.full((iters,), -1.0, dtype=torch.float64, device=DEV)
        hg.hg_run_noalloc(ny, nx, T, P, iters, holo, mse, kind, levels, algo)
        ref_holo, ref_mse = plan_run(ny, nx, kind, levels, algo, iters, T.view(1, ny, nx),
                                     None if P is None else P.view(1, ny, nx))
        got_holo, got_mse = holo.cpu().numpy(), mse.cpu().numpy()
        assert np.all(got_mse > 0), (call, got_mse)
        # the same kernels on the same data in the same order, and every
        # panel's partial sums are combined in a fixed order whatever the grid
        # size: bit-identical holograms and MSE
        assert got_holo.max() < levels
        assert np.array_equal(got_holo, ref_holo), (call, int(np.sum(got_holo != ref_holo)))
        assert np.array_equal(got_mse, ref_mse), (call, got_mse, ref_mse)


def test_noalloc_rejects_sizes_beyond_its_region_and_host_pointers():
    n = hg.HG_NOALLOC_MAX_SIDE * 2
    T = torch.ones((n, n), dtype=torch.float32, device=DEV)
    with pytest.raises(hg.HgError) as e:
        hg.hg_run_noalloc(n, n, T, None, 2)
    assert e.value.status == 7
    with pytest.raises(hg.HgError) as e:
        hg.hg_run_noalloc(64, n, T, None, 2)
    assert e.value.status == 7
    with pytest.raises(hg.HgError) as e:
        hg.hg_run_noalloc(64, 64, torch.ones((64, 64), dtype=torch.float32), None, 2)
    assert e.value.status == 1
    # still usable after the rejections
    t = torch.from_numpy(synth.target(64, 64, 5)).to(DEV)
    mse = torch.empty(2, dtype=torch.float64, device=DEV)
    hg.hg_run_noalloc(64, 64, t, None, 2, None, mse)
    assert torch.all(mse > 0)
