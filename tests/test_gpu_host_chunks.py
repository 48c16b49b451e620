"""hg_run with host buffers runs the batch in chunks, each chunk's copies
overlapping another chunk's iterations (hg_opts.host_chunks).  Every chunk
runs the whole-batch run's kernels on its own targets, so the results must be
bit-identical to a run of the same plan on device buffers: holograms, MSE,
hg_get_metrics and hg_get_phase, for even and uneven chunks and the default
lead-chunk schedule, GS, WGS, LT and a modulated plan, and across repeated
calls with other iteration counts (which change the default's lead chunk)."""
import numpy as np
import pytest
import torch

from paper_2008_12214_gb300 import hologen as hg
from paper_2008_12214_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# ny, nx, batch, slm kind, levels, algorithm, host_chunks, plan options
CASES = [
    (1024, 1024, 8, hg.HG_SLM_BINARY, 2, hg.HG_GS, 4, {}),
    (512, 512, 6, hg.HG_SLM_LLEVEL, 16, hg.HG_WGS, 4, {}),
    (512, 512, 5, hg.HG_SLM_BINARY, 2, hg.HG_LT, 2, {}),
    (1024, 1024, 4, hg.HG_SLM_BINARY, 2, hg.HG_GS, 3, dict(modulated=True, fresnel=0.002)),
    (256, 512, 7, hg.HG_SLM_LLEVEL, 4, hg.HG_GS, 0, {}),
    # the default schedule on 2^24 pixels: a lead chunk whose size follows the
    # iteration count (10 targets at 5 iterations, 12 at 3), then the rest;
    # the repeated iteration count takes the schedule timed on its first call
    (1024, 1024, 16, hg.HG_SLM_BINARY, 2, hg.HG_GS, 0, {}),
]


def case_id(c):
    return "%dx%d-b%d-k%d-L%d-a%d-c%d%s" % (c[0], c[1], c[2], c[3], c[4], c[5], c[6], "-mod" if c[7] else "")


def run(plan, T, P, iters, batch, ny, nx, device):
    holo = torch.empty((batch, ny, nx), dtype=torch.uint8, device=device)
    mse = torch.empty((batch, iters), dtype=torch.float64, device=device)
    plan.run(T.to(device), None if P is None else P.to(device), iters, holo, mse)
    plan.sync()
    met = plan.metrics().cpu().numpy()
    ph = torch.empty((batch, ny, nx), dtype=torch.float32, device=DEV)
    hg.hg_get_phase(plan.h, ph)
    plan.sync()
    return holo.cpu().numpy(), mse.cpu().numpy(), met, ph.cpu().numpy(), hg.hg_last_launch_count(plan.h)


@pytest.mark.parametrize("c", CASES, ids=case_id)
def test_chunked_host_run_is_bit_identical_to_device_run(c):
    ny, nx, batch, kind, levels, algo, chunks, kw = c
    plan = hg.Plan(ny, nx, batch, kind, levels, algo, host_chunks=chunks, **kw)
    try:
        for iters, seed in ((5, 300), (5, 303), (3, 301), (5, 302)):
            T = torch.from_numpy(synth.targets(batch, ny, nx, seed))
            P = torch.from_numpy(synth.init_phases(batch, ny, nx, seed)) if seed != 301 else None
            h_host, m_host, met_host, ph_host, n_host = run(plan, T, P, iters, batch, ny, nx, "cpu")
            h_dev, m_dev, met_dev, ph_dev, n_dev = run(plan, T, P, iters, batch, ny, nx, DEV)
            assert n_host > 0 and n_dev > 0
            assert np.array_equal(h_host, h_dev), (iters, int(np.sum(h_host != h_dev)))
            assert np.array_equal(m_host, m_dev), iters
            assert np.array_equal(met_host, met_dev), iters
            assert np.array_equal(ph_host, ph_dev), iters
            assert np.all(m_host > 0)
    finally:
        plan.close()


def test_chunked_run_then_plain_run_and_ospr_unchunked():
    """A plan that ran chunked runs whole-batch on device buffers afterwards,
    and OSPR plans (one transform pass per subframe) never chunk."""
    ny = nx = 512
    batch = 4
    plan = hg.Plan(ny, nx, batch, host_chunks=4)
    T = torch.from_numpy(synth.targets(batch, ny, nx, 9))
    try:
        mse = torch.empty((batch, 4), dtype=torch.float64)
        plan.run(T, None, 4, None, mse)
        plan.sync()
        mse_d = torch.empty((batch, 4), dtype=torch.float64, device=DEV)
        plan.run(T.to(DEV), None, 4, None, mse_d)
        plan.sync()
        assert torch.equal(mse, mse_d.cpu())
    finally:
        plan.close()
    op = hg.Plan(ny, nx, 2, hg.HG_SLM_BINARY, 2, hg.HG_OSPR, subframes=4, host_chunks=2)
    try:
        m_host = torch.empty(2, dtype=torch.float64)
        op.run(T[:2], None, 1, None, m_host)
        op.sync()
        m_dev = torch.empty(2, dtype=torch.float64, device=DEV)
        op.run(T[:2].to(DEV), None, 1, None, m_dev)
        op.sync()
        assert torch.equal(m_host, m_dev.cpu())
    finally:
        op.close()
