"""Plans of the widened variants inside a group (one CUDA graph of
concurrent branches): a modulated plan with illumination, Fresnel term and
a region of interest, a direct-search plan and an annealing plan, next to a
plain GS plan.  The group run equals each plan run alone, bit for bit, and a
graph replay repeats it (marked gpu)."""
import numpy as np
import pytest
import torch

from paper_2008_12214_gb300 import hologen as hg
from paper_2008_12214_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_group_with_modulated_and_search_plans():
    n = 64
    y, x = np.mgrid[0:n, 0:n]
    amp = torch.from_numpy(np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * 20.0 ** 2)).astype(np.float32)).to(DEV)
    roi = torch.from_numpy((((y - n / 2) ** 2 + (x - n / 2) ** 2) <= 24 ** 2).astype(np.uint8)).to(DEV)
    mod = hg.Plan(n, n, 2, hg.HG_SLM_AMPLITUDE, 8, hg.HG_GS, fresnel=0.01)
    mod.set_illumination(amp, None)
    mod.set_roi(roi)
    plans = [hg.Plan(256, 256, 2), mod, hg.Plan(32, 32, 3, hg.HG_SLM_BINARY, 2, hg.HG_DS, seed=4),
             hg.Plan(32, 32, 2, hg.HG_SLM_LLEVEL, 4, hg.HG_SA, seed=5, sa_temp=1e-3, sa_cool=0.5)]
    iters = 3
    T, P, H, M = [], [], [], []
    for i, p in enumerate(plans):
        ny, nx, b = p.ny, p.nx, p.batch
        T.append(torch.from_numpy(synth.targets(b, ny, nx, 4000 + 10 * i)).to(DEV))
        P.append(torch.from_numpy(synth.init_phases(b, ny, nx, 4000 + 10 * i)).to(DEV))
        H.append(torch.empty((b, ny, nx), dtype=torch.uint8, device=DEV))
        M.append(torch.empty((b, iters), dtype=torch.float64, device=DEV))
    g = hg.hg_group_create([p for p in plans])
    try:
        hg.hg_group_run(g, T, P, iters, H, M)
        hg.hg_group_sync(g)
        first = [(h.cpu().numpy().copy(), m.cpu().numpy().copy()) for h, m in zip(H, M)]
        hg.hg_group_run(g, T, P, iters, H, M)  # graph replay
        hg.hg_group_sync(g)
        for i in range(len(plans)):
            assert np.array_equal(H[i].cpu().numpy(), first[i][0])
            assert np.array_equal(M[i].cpu().numpy(), first[i][1])
        for i, p in enumerate(plans):
            h2 = torch.empty_like(H[i])
            m2 = torch.empty_like(M[i])
            p.run(T[i], P[i], iters, h2, m2)
            p.sync()
            assert np.array_equal(h2.cpu().numpy(), first[i][0]), i
            assert np.array_equal(m2.cpu().numpy(), first[i][1]), i
    finally:
        hg.hg_group_destroy(g)
        for p in plans:
            p.close()
