#!/usr/bin/env python
"""Throughput of batched binary-phase Gerchberg-Saxton at 1024^2, batch 64.

One step = one hg_run of ITERS iterations over a batch of 64 seeded synthetic
targets (target preparation, head pass, ITERS-1 row/column pass pairs, tail
pass, metric reduction), inputs already resident in HBM.  value = batched GS
iterations per second over all ranks (weak scaling: every rank runs its own
batch).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--iters I] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GS iterations/s at 1024^2 batch 64, % HBM roofline; time-to-MSE vs plain GS"
UNIT = "batched GS iterations/s (64 targets of 1024x1024, binary phase)"
NY = NX = 1024
BATCH = 64
# Algorithmic HBM bytes per pixel and iteration.  Plain passes: row 20 (field
# read + write 16, target 4), column 16 (field read + write): 36 B/px.  With the
# paired-row pass (binary SLM: column spectra are Hermitian, so only rows
# ky <= ny/2 are stored and read back): row 16 (half field 4, target 4, field
# written 8), column 12 (field read 8, half written 4): 28 B/px.  In Hermitian
# form ("+herm": the row pass writes only rows ky <= ny/2 of the Hermitian part
# of F): row 12 (half read 4, target 4, half written 4), column 8 (half read 4,
# half written 4): 20 B/px.  The column pass after the head pass reads every
# row and the last one writes every row; column bytes are averaged over the
# passes of a run.
BYTES_ROW, BYTES_COL = 20, 16
BYTES_ROW_PAIRED, BYTES_COL_PAIRED = 16, 12
BYTES_ROW_HERM, BYTES_COL_HERM = 12, 8
BYTES_FUSED = 36
DATA = ("synthetic: seeded targets of 16 Gaussian blobs + 8 rectangles per 1024x1024 field "
        "(seeds 1000 + rank*64 + b), initial phase U[0, 2 pi)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pipeline", type=int, default=-1)
    ap.add_argument("--autotune", type=int, default=1, help="1 tune, 0 first variant, 2+k variant k")
    ap.add_argument("--precision", type=int, default=0,
                    help="0 FP32 engine; 1..4 tensor-core row pass (FP16 hi+lo, FP16, BF16 hi+lo, BF16); "
                         "fresnel workload: 0 binary phase SLM, 1 16-level amplitude SLM")
    ap.add_argument("--batch", type=int, default=None,
                    help="targets per rank (profiling runs; default: the workload's own, 64 for the headline; "
                         "mixed: targets per size)")
    ap.add_argument("--quick", action="store_true", help="skip the e2e and CPU-baseline legs")
    ap.add_argument("--pairs", type=int, default=2048, help="warmstart: training pairs")
    ap.add_argument("--search-waves", type=int, default=1, help="search: targets = waves x 4 x SMs")
    ap.add_argument("--heldout", type=int, default=64, help="warmstart: held-out targets")
    ap.add_argument("--residual", action="store_true",
                    help="warmstart: the shared start phase as the network's base phase (residual labels)")
    ap.add_argument("--warm-slm", choices=["both", "llevel256", "binary"], default="both",
                    help="warmstart: SLMs to train and evaluate")
    ap.add_argument("--workload", choices=["headline", "ospr", "adospr", "mixed", "warmstart", "gs2048", "wgs256", "fresnel", "lt", "search"],
                    default="headline",
                    help="headline: binary GS 1024^2 x 64 (the benchmark line); ospr: 8 targets x 24 "
                         "subframes of 1024^2; mixed: 16 targets each of 512^2, 1024^2, 2048^2, 1080x1920")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(
        os.environ.get("WORLD_SIZE", 1))


# Sources of the 1024-sample GS passes that the roofline and the committed
# DRAM traffic describe: the line engine, the passes, their 1024-sample
# instantiations and their launches.  A change to any of them makes the
# committed traffic stale.
GS_SOURCES = ("hg_fft.cuh", "hg_kernels.cuh", "hg_pipe.cuh", "hg_api.cu", "ops_1024.cu")


def src_hash():
    h = hashlib.sha256()
    files = set()
    for pat in GS_SOURCES:
        files.update(glob.glob(os.path.join(ROOT, "paper_2008_12214_gb300", "csrc", pat)))
    for f in sorted(files):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _oracle_worker(seed, steps, barrier, queue):
    """One host core: the oracle on its own 1024^2 target, single-threaded
    (OMP_NUM_THREADS = 1 before the oracle library loads), one warm-up GS
    iteration, then `steps` timed ones started together with the other
    workers.  Puts (start, end) wall times on `queue`."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    from paper_2008_12214_gb300 import synth
    t = synth.target(NY, NX, seed)
    ph = synth.init_phase(NY, NX, seed).astype(np.float64)
    T = oracle.prepare_target(t)
    ph = oracle.gs_step(T, ph)["phase"]
    barrier.wait()
    t0 = time.time()
    for _ in range(steps):
        ph = oracle.gs_step(T, ph)["phase"]
    queue.put((t0, time.time()))


def oracle_per_core(workers: int, steps: int, seed0: int = 1000):
    """The FP64 oracle as it stands, one target per host core: `workers`
    single-threaded processes (spawned, so no process is forked from one that
    holds a CUDA context) each run `steps` GS iterations of their own 1024^2
    binary target.  Returns target-iterations per second over the common
    timed span."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(seed0 + i, steps, barrier, queue)) for i in range(workers)]
    for pr in procs:
        pr.start()
    spans = [queue.get() for _ in procs]
    for pr in procs:
        pr.join()
    t0, t1 = min(a for a, _ in spans), max(b for _, b in spans)
    return workers * steps / (t1 - t0)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_sample(steps: int = 2):
    """CPU baseline: the oracle threaded one target per core on all host
    cores, and alone on one core, each core running `steps` whole GS
    iterations of a 1024^2 binary target (oracle.gs_step); scaled to the
    benchmark's unit, one batched iteration = 64 target-iterations."""
    cores = host_cores()
    all_rate = oracle_per_core(cores, steps)
    one_rate = oracle_per_core(1, steps)
    return dict(value=all_rate / BATCH, unit=UNIT, cores=cores, kind="oracle",
                single_core_value=one_rate / BATCH, single_core_s_per_target_iteration=1.0 / one_rate,
                sample="one target per core: %d single-threaded processes x %d GS iterations of their own "
                       "1024x1024 binary target (oracle.gs_step, FP64), %.2f target-iterations/s in all; "
                       "single core %.2f s per target-iteration; scaled to one batched iteration = %d "
                       "target-iterations" % (cores, steps, all_rate, 1.0 / one_rate, BATCH))


def run_reference(args):
    """The reference arm: the oracle, one target per host core.  Each step is
    one GS iteration on every core's own 1024^2 target (a bounded sample of
    the 64-target batch), scaled to batched iterations of 64 targets."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    if args.warmup:
        oracle_per_core(cores, 1)
    rate = oracle_per_core(cores, args.steps)
    B = args.batch or BATCH
    value = rate / B
    per = cores / rate  # wall seconds per step (one iteration on every core)
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=per * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data=DATA,
                config=dict(workload="gs_binary_1024x1024_batch%d" % B, ny=NY, nx=NX, batch=B,
                            step="one GS iteration of one 1024x1024 target on each of %d host cores "
                                 "(bounded sample), scaled to %d targets" % (cores, B)),
                cpu_baseline=dict(kind="oracle", cores=cores, value=value, unit=UNIT,
                                  sample="%d steps x %d single-threaded processes, one 1024x1024 target "
                                         "each" % (args.steps, cores)),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(", ") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


def traffic_for(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel_key)
        if e and e.get("src_hash") == src_hash():
            return e.get("bytes_per_launch")
    except Exception:
        pass
    return None


def run_warmstart(args, dev, s0):
    """The learned warm start at 1024^2: training throughput of the tensor-core
    network on the engine's own GS-200 phases, the tensor-core convolution
    against the measured BF16 peak, and GS iterations / wall time from the
    network's phase to the plain random-phase GS-100 MSE on held-out targets,
    for the 256-level and the binary SLM."""
    import torch
    from paper_2008_12214_gb300 import hologen as hg
    from paper_2008_12214_gb300 import warmstart as ws
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = json.load(f).get("bf16_tflops_sustained")
    except Exception:
        pass
    # tensor-core convolutions of the 1024^2 net, batch 4: level-2 decoder input
    # (384 -> 128 channels at 256^2) and the bottleneck (256 -> 256 at 128^2)
    convs = []
    for (Bc, Hc, cin, cout) in ((4, 256, 384, 128), (4, 128, 256, 256), (4, 1024, 96, 32)):
        x = torch.randn(Bc, Hc, Hc, cin, device=dev).to(torch.bfloat16)
        w = (torch.randn(9, cout, cin, device=dev) * 0.03).to(torch.bfloat16)
        y = torch.empty(Bc, Hc, Hc, cout, device=dev, dtype=torch.bfloat16)
        for _ in range(3):
            hg.hg_conv3x3_forward(x, Bc, Hc, Hc, cin, w, cout, None, 1, None, y)
        e0.record(s0)
        for _ in range(20):
            hg.hg_conv3x3_forward(x, Bc, Hc, Hc, cin, w, cout, None, 1, None, y)
        e1.record(s0)
        hg.hg_conv_status()
        ms = e0.elapsed_time(e1) / 20
        tf = 2.0 * 9 * cin * cout * Bc * Hc * Hc / (ms / 1e3) / 1e12
        convs.append(dict(layer="%dx%d %d->%d batch %d" % (Hc, Hc, cin, cout, Bc), ms=ms, tflops=tf,
                          frac_of_sustained_bf16=tf / peak if peak else None))
        del x, w, y
    res = dict(workload="warmstart_cnn_1024x1024", pairs=args.pairs, heldout=args.heldout, label_iters=200,
               residual=args.residual, conv_kernel_k_conv_fwd=convs, peak_bf16_tflops_sustained=peak)
    for name, kind, L in (("llevel256", hg.HG_SLM_LLEVEL, 256), ("binary", hg.HG_SLM_BINARY, 2)):
        if args.warm_slm not in ("both", name):
            continue
        net, losses, secs = ws.train(NY, NX, args.pairs, batch=4, lr=1e-3, chunk=64, label_iters=200,
                                     label_start="fixed", slm_kind=kind, levels=L, residual=args.residual)
        ev = ws.evaluate(net, NY, NX, args.heldout, ref_iters=100, max_iters=100, chunk=4, slm_kind=kind, levels=L)
        net.close()
        pick = (0, 9, 49, 99)
        res[name] = dict(train_seconds=secs, pairs_per_s=args.pairs / secs, loss_first=losses[0],
                         loss_last20=float(sum(losses[-20:]) / 20), reached=ev["reached"],
                         median_warm_iters=ev["median_warm_iters"], median_speedup=ev["median_speedup"],
                         ms_cnn_per_batch=ev["ms_cnn_batch"], ms_gs_iter_per_batch=ev["ms_per_gs_iter_batch"],
                         eval_batch=ev["batch"],
                         rel_mse_random_at_1_10_50_100=[ev["rel_rand_curve"][i] for i in pick],
                         rel_mse_warm_at_1_10_50_100=[ev["rel_warm_curve"][i] for i in pick])
    return res


def run_side_workload(args):
    """Throughput of the other configurations (reported in DESIGN, not the
    benchmark line): OSPR subframes/s, and batched iterations/s of the mixed
    batch run as one CUDA graph."""
    import torch
    import __graft_entry__
    from paper_2008_12214_gb300 import hologen as hg
    from paper_2008_12214_gb300 import synth
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    s0 = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.workload in ("ospr", "adospr"):
        B, NS = args.batch or 8, 24
        T = torch.from_numpy(synth.targets(B, NY, NX)).to(dev)
        holo = torch.empty((B, NS, NY, NX), dtype=torch.uint8, device=dev)
        mse = torch.empty(B, dtype=torch.float64, device=dev)
        algo = hg.HG_OSPR if args.workload == "ospr" else hg.HG_ADOSPR
        plan = hg.Plan(NY, NX, B, hg.HG_SLM_BINARY, 2, algo, subframes=NS, seed=7)
        for _ in range(args.warmup):
            plan.run(T, None, 1, holo, mse)
        plan.sync()
        e0.record(s0)
        for _ in range(args.steps):
            plan.run(T, None, 1, holo, mse)
        e1.record(s0)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        out = dict(workload="%s_%dx24_1024x1024" % (args.workload, B), ms_per_step=ms, subframes_per_s=B * NS / (ms / 1e3),
                   algorithmic_gbs=36.0 * B * NS * NY * NX / (ms / 1e3) / 1e9,
                   mse=mse.cpu().numpy().tolist(), column_variant=hg.hg_plan_variant(plan.h, 1))
        plan.close()
    elif args.workload == "warmstart":
        out = run_warmstart(args, dev, s0)
    elif args.workload == "wgs256":
        # weighted GS, one 1024^2 target, 256-level SLM, 100 iterations
        n, iters = 1024, 100
        T = torch.from_numpy(synth.targets(1, n, n, 6000)).to(dev)
        P = torch.from_numpy(synth.init_phases(1, n, n, 6000)).to(dev)
        mse = torch.empty((1, iters), dtype=torch.float64, device=dev)
        holo = torch.empty((1, n, n), dtype=torch.uint8, device=dev)
        plan = hg.Plan(n, n, 1, hg.HG_SLM_LLEVEL, 256, hg.HG_WGS)
        for _ in range(args.warmup):
            plan.run(T, P, iters, holo, mse)
        plan.sync()
        e0.record(s0)
        for _ in range(args.steps):
            plan.run(T, P, iters, holo, mse)
        e1.record(s0)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        met = plan.metrics().cpu().numpy()[0]
        out = dict(workload="wgs_llevel256_1024x1024_batch1", ms_per_run=ms, iterations_per_s=iters / (ms / 1e3),
                   final_mse=float(met[-1, 0]), final_amplitude_mse=float(met[-1, 1]),
                   diffraction_efficiency=float(met[-1, 2]), mse_iter_1_10_100=[float(met[i, 0]) for i in (0, 9, 99)],
                   row_variant=hg.hg_plan_variant(plan.h, 0), column_variant=hg.hg_plan_variant(plan.h, 1))
        plan.close()
    elif args.workload == "search":
        # direct search (--precision 0) / simulated annealing (--precision 1): 64x64 binary holograms,
        # one per CTA, 4 CTAs per SM resident (52 KB of shared memory each), 2 sweeps
        n, sweeps = 64, 2
        B = 4 * torch.cuda.get_device_properties(dev).multi_processor_count * args.search_waves
        algo = hg.HG_SA if args.precision == 1 else hg.HG_DS
        T = torch.from_numpy(synth.targets(B, n, n, 9000)).to(dev)
        P = torch.from_numpy(synth.init_phases(B, n, n, 9000)).to(dev)
        mse = torch.empty((B, sweeps), dtype=torch.float64, device=dev)
        plan = hg.Plan(n, n, B, hg.HG_SLM_BINARY, 2, algo, seed=5, sa_temp=1e-3, sa_cool=0.5)
        for _ in range(args.warmup):
            plan.run(T, P, sweeps, None, mse)
        plan.sync()
        e0.record(s0)
        for _ in range(args.steps):
            plan.run(T, P, sweeps, None, mse)
        e1.record(s0)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        met = plan.metrics().cpu().numpy()
        trials = B * sweeps * n * n
        px_evals = trials * n * n
        # FP32 work per replay pixel per trial: dR = c w (6 flops), |R|^2 / N (4), the
        # intensity change a (7), a (2 (I - T^2) + a) accumulated (6): 23 flops with FMA = 2
        flops = 23.0 * px_evals
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x FMA x maximum SM clock
        achieved = flops / (ms / 1e3) / 1e12
        out = dict(workload="%s_binary_64x64_batch%d" % ("sa" if algo == hg.HG_SA else "ds", B), ms_per_step=ms,
                   sweeps=sweeps, trials_per_s=trials / (ms / 1e3), pixel_evaluations_per_s=px_evals / (ms / 1e3),
                   roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                                 flops_per_pixel_evaluation=23),
                   mse_initial_to_final_mean=float((met[:, -1, 0]).mean()),
                   accepted_per_sweep_mean=[float(met[:, k, 3].mean()) for k in range(sweeps)])
        plan.close()
    elif args.workload == "lt":
        # Liu-Taghizadeh GS, 64 binary holograms of 1024^2, window 0.25 -> 1 over 10 constraints
        B, n = args.batch or 64, 1024
        T = torch.from_numpy(synth.targets(B, n, n, 7100)).to(dev)
        P = torch.from_numpy(synth.init_phases(B, n, n, 7100)).to(dev)
        mse = torch.empty((B, args.iters), dtype=torch.float64, device=dev)
        plan = hg.Plan(n, n, B, hg.HG_SLM_BINARY, 2, hg.HG_LT, lt_start=0.25, lt_grow=10)
        for _ in range(args.warmup):
            plan.run(T, P, args.iters, None, mse)
        plan.sync()
        e0.record(s0)
        for _ in range(args.steps):
            plan.run(T, P, args.iters, None, mse)
        e1.record(s0)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        it_ms = ms / args.iters
        out = dict(workload="lt_binary_1024x1024_batch%d" % B, ms_per_step=ms, iters_per_step=args.iters,
                   batched_iterations_per_s=1e3 / it_ms, gbs_at_36=36.0 * B * n * n / (it_ms / 1e3) / 1e9,
                   final_mse_mean=float(mse[:, -1].mean().item()),
                   row_variant=hg.hg_plan_variant(plan.h, 0), column_variant=hg.hg_plan_variant(plan.h, 1))
        plan.close()
    elif args.workload == "fresnel":
        # modulated GS: 64 Fresnel holograms of 1024^2 (quadratic phase pi dx^2 / (lambda z) for
        # 8 um pixels, 532 nm, 0.5 m), Gaussian illumination, disc region of interest, binary
        # phase or 16-level amplitude SLM (--precision 0 / 1 selects), 50 iterations
        B, n = args.batch or 64, 1024
        c = float(np.pi * (8e-6) ** 2 / (532e-9 * 0.5))
        amp_slm = args.precision == 1
        kind, levels = (hg.HG_SLM_AMPLITUDE, 16) if amp_slm else (hg.HG_SLM_BINARY, 2)
        y, x = np.mgrid[0:n, 0:n]
        A = np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * (0.3 * n) ** 2)).astype(np.float32)
        roi = (((y - n / 2) ** 2 + (x - n / 2) ** 2) <= (0.35 * n) ** 2).astype(np.uint8)
        T = torch.from_numpy(synth.targets(B, n, n, 7000)).to(dev)
        P = torch.from_numpy(synth.init_phases(B, n, n, 7000)).to(dev)
        mse = torch.empty((B, args.iters), dtype=torch.float64, device=dev)
        holo = torch.empty((B, n, n), dtype=torch.uint8, device=dev)
        plan = hg.Plan(n, n, B, kind, levels, hg.HG_GS, fresnel=c, modulated=True, pipeline=args.pipeline,
                       autotune=args.autotune)
        plan.set_illumination(torch.from_numpy(A).to(dev), None)
        plan.set_roi(torch.from_numpy(roi).to(dev))
        for _ in range(args.warmup):
            plan.run(T, P, args.iters, holo, mse)
        plan.sync()
        e0.record(s0)
        for _ in range(args.steps):
            plan.run(T, P, args.iters, holo, mse)
        e1.record(s0)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        hg.hg_profile_enable(plan.h, 2 * args.iters + 8)
        plan.run(T, P, args.iters, holo, mse)
        prof = hg.hg_profile_read(plan.h)
        hg.hg_profile_enable(plan.h, 0)
        ev = plan.evaluate(holo, T).cpu().numpy()
        it_ms = ms / args.iters
        px = B * n * n
        # generic passes: row 8 + 8 (field) + 4 (T) + 1 (ROI); column 8 + 8 (field) + 8 (illumination)
        out = dict(workload="fresnel_%s_1024x1024_batch%d" % ("amplitude16" if amp_slm else "binary", B),
                   ms_per_step=ms, iters_per_step=args.iters, batched_iterations_per_s=1e3 / it_ms,
                   algorithmic_gbs_at_45=45.0 * px / (it_ms / 1e3) / 1e9,
                   final_roi_mse_mean=float(mse[:, -1].mean().item()), roi_ssim_mean=float(ev[:, 3].mean()),
                   efficiency_mean=float(ev[:, 2].mean()), fresnel_rad_per_px2=c,
                   row_ms=prof[0] / max(prof[1], 1), column_ms=prof[2] / max(prof[3], 1),
                   row_variant=hg.hg_plan_variant(plan.h, 0), column_variant=hg.hg_plan_variant(plan.h, 1))
        plan.close()
    elif args.workload == "gs2048":
        B, n = args.batch or 16, 2048
        T = torch.from_numpy(synth.targets(B, n, n, 5000)).to(dev)
        P = torch.from_numpy(synth.init_phases(B, n, n, 5000)).to(dev)
        mse = torch.empty((B, args.iters), dtype=torch.float64, device=dev)
        plan = hg.Plan(n, n, B, hg.HG_SLM_BINARY, 2, hg.HG_GS, precision=args.precision, autotune=args.autotune)
        for _ in range(args.warmup):
            plan.run(T, P, args.iters, None, mse)
        plan.sync()
        e0.record(s0)
        for _ in range(args.steps):
            plan.run(T, P, args.iters, None, mse)
        e1.record(s0)
        plan.sync()
        ms = e0.elapsed_time(e1) / args.steps
        px = B * n * n
        it_ms = ms / args.iters
        out = dict(workload="gs_binary_2048x2048_batch%d" % B, precision=args.precision, ms_per_step=ms,
                   iters_per_step=args.iters, final_mse_mean=float(mse[:, -1].mean().item()),
                   batched_iterations_per_s=1e3 / it_ms, gbs_at_36=36.0 * px / (it_ms / 1e3) / 1e9,
                   row_variant=hg.hg_plan_variant(plan.h, 0), column_variant=hg.hg_plan_variant(plan.h, 1))
        plan.close()
    else:
        shapes = [(512, 512), (1024, 1024), (2048, 2048), (1080, 1920)]
        nb = args.batch or 16
        plans, Ts, Ps, Ms = [], [], [], []
        for i, (ny, nx) in enumerate(shapes):
            plans.append(hg.Plan(ny, nx, nb))
            Ts.append(torch.from_numpy(synth.targets(nb, ny, nx, 3000 + 16 * i)).to(dev))
            Ps.append(torch.from_numpy(synth.init_phases(nb, ny, nx, 3000 + 16 * i)).to(dev))
            Ms.append(torch.empty((nb, args.iters), dtype=torch.float64, device=dev))
        g = hg.hg_group_create(plans)
        sched_ms = {}
        for name, sched in (("concurrent", hg.HG_GROUP_CONCURRENT), ("serial", hg.HG_GROUP_SERIAL)):
            hg.hg_group_set_schedule(g, sched)
            for _ in range(args.warmup):
                hg.hg_group_run(g, Ts, Ps, args.iters, None, Ms)
            hg.hg_group_sync(g)
            e0.record(s0)
            for _ in range(args.steps):
                hg.hg_group_run(g, Ts, Ps, args.iters, None, Ms)
            e1.record(s0)
            hg.hg_group_sync(g)
            sched_ms[name] = e0.elapsed_time(e1) / args.steps
        ms = sched_ms["serial"]  # the default schedule
        px = nb * sum(a * b for a, b in shapes)
        # each size alone (its plan's own hg_run), and its loop passes one by one
        alone = []
        for i, p in enumerate(plans):
            for _ in range(2):
                p.run(Ts[i], Ps[i], args.iters, None, Ms[i])
            p.sync()
            e0.record(s0)
            for _ in range(args.steps):
                p.run(Ts[i], Ps[i], args.iters, None, Ms[i])
            e1.record(s0)
            p.sync()
            ms_i = e0.elapsed_time(e1) / args.steps
            hg.hg_profile_enable(p.h, 2 * args.iters + 8)
            p.run(Ts[i], Ps[i], args.iters, None, Ms[i])
            prof = hg.hg_profile_read(p.h)
            hg.hg_profile_enable(p.h, 0)
            alone.append(dict(shape="%dx%d" % shapes[i], ms_per_run=ms_i,
                              row_ms=prof[0] / max(prof[1], 1), column_ms=prof[2] / max(prof[3], 1),
                              gbs_at_36=36.0 * nb * shapes[i][0] * shapes[i][1] * args.iters / (ms_i / 1e3) / 1e9))
        out = dict(workload="mixed_%d_targets_one_graph" % (4 * nb), ms_per_step=ms, iters_per_step=args.iters,
                   batched_iterations_per_s=args.iters / (ms / 1e3),
                   algorithmic_gbs_at_36=36.0 * px * args.iters / (ms / 1e3) / 1e9,
                   ms_per_step_by_schedule=sched_ms,
                   sum_of_sizes_alone_ms=sum(a["ms_per_run"] for a in alone), sizes_alone=alone,
                   variants=[(hg.hg_plan_variant(p.h, 0), hg.hg_plan_variant(p.h, 1)) for p in plans],
                   launches_per_step=hg.hg_group_launch_count(g))
        hg.hg_group_destroy(g)
        for p in plans:
            p.close()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "headline":
        run_side_workload(args)
        return
    import torch
    import __graft_entry__
    from paper_2008_12214_gb300 import hologen as hg
    from paper_2008_12214_gb300 import shard
    from paper_2008_12214_gb300 import synth

    rank, local, world = dist_env()
    clocks = ClockSampler(local) if rank == 0 else None  # running through warm-up and timed steps
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()

    B = args.batch or BATCH
    base = shard.target_seeds(rank, B)[0]
    t_host = synth.targets(B, NY, NX, base)
    p_host = synth.init_phases(B, NY, NX, base)
    T = torch.from_numpy(t_host).to(dev)
    P = torch.from_numpy(p_host).to(dev)
    holo = torch.empty((B, NY, NX), dtype=torch.uint8, device=dev)
    mse = torch.empty((B, args.iters), dtype=torch.float64, device=dev)
    plan = hg.Plan(NY, NX, B, hg.HG_SLM_BINARY, 2, hg.HG_GS, pipeline=args.pipeline,
                   autotune=args.autotune, precision=args.precision)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan.run(T, P, args.iters, holo, mse)
    plan.sync()

    # timed region: K steps as the library runs them (the iteration loop
    # replayed as one CUDA graph), bracketed by CUDA events on the plan's stream
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        plan.run(T, P, args.iters, holo, mse)
        launches += hg.hg_last_launch_count(plan.h)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    plan.sync()
    el_ms = e0.elapsed_time(e1)
    # per-pass durations for the roofline: the same K steps again with an event
    # pair around every row and column pass (the loop is then launched pass by
    # pass instead of as the graph)
    hg.hg_profile_enable(plan.h, 2 * args.steps * args.iters + 8)
    for _ in range(args.steps):
        plan.run(T, P, args.iters, holo, mse)
    prof = hg.hg_profile_read(plan.h)
    hg.hg_profile_enable(plan.h, 0)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    el_ms = shard.max_over_ranks(el_ms, dev)
    value = shard.weak_scaling_rate(world, args.steps * args.iters, el_ms / 1e3)

    # end to end through the C ABI with pinned host buffers (copies inside)
    e2e = None
    if not args.quick:
        tp = torch.from_numpy(t_host).pin_memory()
        pp = torch.from_numpy(p_host).pin_memory()
        hp = torch.empty((B, NY, NX), dtype=torch.uint8).pin_memory()
        mp = torch.empty((B, args.iters), dtype=torch.float64).pin_memory()
        for _ in range(2):  # the first call times the copies, the second takes its chunk sizes
            plan.run(tp, pp, args.iters, hp, mp)
        e2e_steps = max(2, min(args.steps, 5))
        if world > 1:
            dist.barrier()
        w0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.run(tp, pp, args.iters, hp, mp)
        e2e_s = time.perf_counter() - w0
        e2e_s = shard.max_over_ranks(e2e_s, dev)
        e2e = dict(value=shard.weak_scaling_rate(world, e2e_steps * args.iters, e2e_s), unit=UNIT,
                   h2d_bytes_per_step=int(tp.numel() * 4 + pp.numel() * 4),
                   d2h_bytes_per_step=int(hp.numel() + mp.numel() * 8))
    variants = (hg.hg_plan_variant(plan.h, 0), hg.hg_plan_variant(plan.h, 1))
    plan.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    npx = NY * NX * B
    row_ms = prof[0] / max(prof[1], 1)
    col_ms = prof[2] / max(prof[3], 1)
    paired = "pair" in variants[0]
    herm = "+herm" in variants[0]
    it = args.iters
    if herm:
        b_row = BYTES_ROW_HERM
        b_col = (2 * 12 + max(it - 2, 0) * BYTES_COL_HERM) / it  # first: full read; last: full write
    elif paired:
        b_row = BYTES_ROW_PAIRED
        b_col = ((it - 1) * BYTES_COL_PAIRED + 16) / it  # last column pass writes every row
    else:
        b_row, b_col = BYTES_ROW, BYTES_COL
    # "bytes": the algorithmic bytes of the fused schedule's pass (row 20, column 16 B/px),
    # the per-unit figure of the roofline; "moved": what the running variant reads and writes
    passes = {
        "row": dict(bytes=BYTES_ROW * npx, moved=b_row * npx, ms=row_ms, launches=int(prof[1]), variant=variants[0]),
        "column": dict(bytes=BYTES_COL * npx, moved=b_col * npx, ms=col_ms, launches=int(prof[3]),
                       variant=variants[1]),
    }
    for v in passes.values():
        v["gbs"] = v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else None
        v["gbs_moved"] = v["moved"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else None
    dom = max(passes, key=lambda k: passes[k]["ms"] * passes[k]["launches"])
    d = passes[dom]
    kernel_key = d["variant"] + (" row" if dom == "row" else " column")
    traffic = traffic_for(kernel_key)
    roofline = dict(bound="hbm", achieved=d["gbs"], peak=peak, unit="GB/s",
                    frac=(d["gbs"] / peak) if d["gbs"] else None, traffic=traffic,
                    kernel="%s pass (%s)" % (dom, kernel_key), peak_source=peak_src,
                    frac_basis="equivalent bandwidth: the fused schedule's algorithmic bytes (%d B/px for the "
                               "%s pass) over the launch time; frac_moved uses the bytes this variant reads "
                               "and writes" % (BYTES_ROW if dom == "row" else BYTES_COL, dom),
                    algorithmic_bytes_per_launch=d["bytes"], avg_launch_ms=d["ms"],
                    variant_bytes_per_launch=d["moved"],
                    frac_moved=(d["gbs_moved"] / peak) if d["gbs_moved"] else None,
                    timing="per-pass CUDA events on the plan's stream over a second K-step region")
    iter_ms = el_ms / (args.steps * args.iters)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=el_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32" if args.precision == 0 else ["", "f16x2", "f16", "bf16x2", "bf16"][args.precision],
        data=DATA,
        config=dict(workload="gs_binary_1024x1024_batch%d" % B, ny=NY, nx=NX, batch=B,
                    iters_per_step=args.iters, slm="binary", parallelism="dp%d" % world,
                    row_variant=variants[0], column_variant=variants[1],
                    l2="inputs larger than L2: field 512 MiB + prepared targets 256 MiB per rank"),
        holograms_per_s=value * B / args.iters,
        whole_iteration=dict(
            ms=iter_ms, loop_row_plus_column_ms=row_ms + col_ms,
            bytes_per_px_moved=b_row + b_col,
            gbs_moved=(b_row + b_col) * npx / (iter_ms / 1e3) / 1e9,
            bytes_per_px_36=BYTES_FUSED,
            gbs_at_36=BYTES_FUSED * npx / (iter_ms / 1e3) / 1e9,
            frac_at_36=BYTES_FUSED * npx / (iter_ms / 1e3) / 1e9 / peak),
        roofline=roofline,
        passes={k: dict(avg_ms=v["ms"], gbs=v["gbs"], frac=(v["gbs"] / peak if v["gbs"] else None),
                        launches=v["launches"], bytes_per_px=v["bytes"] / npx, variant=v["variant"],
                        bytes_per_px_moved=v["moved"] / npx, gbs_moved=v["gbs_moved"],
                        frac_moved=(v["gbs_moved"] / peak if v["gbs_moved"] else None))
                for k, v in passes.items()},
        cpu_baseline=None if args.quick else cpu_oracle_sample(),
        e2e=e2e,
        clocks=clk,
        gpu_launches=launches,
        src_hash=src_hash(),
    )
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
