"""Benchmark: primal-dual iterations of the sparse imaging hot path on one GB300 (or N replicas).

Workload (FP32 bulk, FP64 norms): 1024^2 sky (50 points + 20 blobs), 2048^2 grid,
Kaiser-Bessel J = 4 with a 2^12-per-cell table, M = 1e7 visibilities (Gaussian core
plus 20 % uniform-disk outliers, weights U[0.5, 1], 30 dB noise), SARA Dirac +
db1..db8 over 4 levels.  One step = one primal-dual iteration: Psi^dagger with the
l1-dual update, Phi (pad/correct, FFT, degrid with the l2-ball dual update), the
FP64 ball scalar, Phi^dagger (grid, inverse FFT), Psi, and the primal update with
the FP64 convergence norms.  Metric: visibilities per second through Phi and
Phi^dagger (M per iteration) and ms per iteration.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbri|reference]
Under torchrun each rank solves its own problem (seed + rank): replicas, weak scaling.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L2_BYTES = 129 * 1024 * 1024

# DRAM bytes (read + write) per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the current kernels at the 1024^2 / M = 1e7 workload; set to None
# whenever a kernel changes after its capture.
KERNEL_TRAFFIC = {"degrid": None, "grid": 195.45e6, "degrid_grid": 361.91e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gbri", choices=["gbri", "reference"])
    ap.add_argument("--config", default="large", choices=["large", "small", "huge"],
                    help="huge: the precision study (4096^2, J = 6, M = 2e9), mixed vs FP64 paths")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=10.0, help="Poisson job arrivals per second")
    ap.add_argument("--serve-rates", default="",
                    help="comma-separated arrival rates for several serving runs (overrides --serve-rate)")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0, help="HBM admission budget of the serving leg")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="arrival window of the serving leg (0: skip)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the Phi / Phi^dagger sweep over image sizes")
    ap.add_argument("--batch-problems", type=int, default=64,
                    help="independent problems of the batching leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=20, help="timed iterations of the batching leg")
    ap.add_argument("--fp64-steps", type=int, default=50,
                    help="timed iterations of the plain FP64 path (0: skip the precision leg)")
    ap.add_argument("--algo-steps", type=int, default=100,
                    help="timed iterations per solver of the algorithms leg (0: skip)")
    ap.add_argument("--interp-steps", type=int, default=200,
                    help="timed iterations of the first-order interpolation leg (0: skip)")
    ap.add_argument("--wstack-planes", default="8,32",
                    help="comma-separated w-plane counts of the w-stacking leg (empty: skip)")
    ap.add_argument("--quick", action="store_true",
                    help="profiling run: short power method, no end-to-end, operator or CPU legs")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(cfg_name, rank=0):
    cfg = dict(synth.CONFIGS[cfg_name])
    seed = cfg["seed"] + rank
    x_true = synth.sky(cfg["n_side"], cfg["n_points"], cfg["n_blobs"], seed=seed)
    uvw = synth.uv_coverage(cfg["M"], seed=seed + 1, outlier_frac=cfg["outlier_frac"], weights=cfg["weights"])
    return cfg, seed, x_true, uvw


def aggregate_replicas(ms_local, units_local, steps):
    """Weak-scaling aggregate over ranks: the slowest rank's time and the sum of the units all
    ranks processed (whole-job throughput).  Works with any initialised process group."""
    import torch
    import torch.distributed as dist
    ms, units = float(ms_local), float(units_local)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units], dtype=torch.float64, device=dev)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), float(u.item())
    return ms, units * steps / (ms / 1e3)


def per_kernel_roofline(kern, cfg, K, M, peak):
    """Every kernel of one primal-dual iteration against the HBM roofline: algorithmic bytes per
    iteration (what the step must move at least: its inputs read once, its outputs written once)
    over the kernel's device time per iteration (launch-averaged CUDA events on the launching
    stream, times its launches per iteration).
      pad: x read, the n x n block of the padded image written (8 B per pixel);
      fft_fwd: real K x K in, half spectrum K (K/2 + 1) complex out; fft_inv: the K x K complex
      grid read, its real inverse transform (K x K real) written;
      degrid_grid: 32 B per visibility (metadata, u, y read, u written), half spectrum read and
      grid written once;
      psi_adjoint: x read once, the dual z1 of every basis read and written (8 B per
      coefficient), the LL carries of levels 1 .. L-1 written and read back;
      psi: z1 of every basis read, x written;
      update: the real inverse transform at every pixel, psi z1 and x read, x and xhat written."""
    n = cfg["n_side"]
    N = n * n
    nw = len(cfg["db_orders"])
    nb = nw - (1 if 0 in cfg["db_orders"] else 0)
    L = cfg["levels"]
    carry = sum(4.0 ** -l for l in range(1, L))
    alg = {"pad": 8 * N, "fft_fwd": 4 * K * K + 8 * K * (K // 2 + 1), "fft_inv": 12 * K * K,
           "degrid_grid": 32 * M + 8 * K * (K // 2 + 1) + 8 * K * K,
           "psi_adjoint": 4 * N + 8 * nw * N + 8 * N * nb * carry, "psi": 4 * nw * N + 4 * N, "update": 20 * N}
    launches = {"pad": 1, "fft_fwd": 1, "fft_inv": 1, "degrid_grid": 1, "update": 1,
                "psi_adjoint": (1 if 0 in cfg["db_orders"] else 0) + (L if nb else 0),
                "psi": (L + 1) if nb else 1}
    out = {}
    for k, b in alg.items():
        if k not in kern:
            continue
        t = kern[k]["ms_avg"] * launches[k] * 1e-3
        a = b / t / 1e9
        out[k] = {"us_per_iteration": t * 1e6, "launches_per_iteration": launches[k], "algorithmic_bytes": int(b),
                  "achieved": a, "frac": a / peak}
    return out


def describe(cfg):
    return ("%d^2 sky, %d^2 grid, J=%d, S=%d, M=%.0e, SARA %s over %d levels, primal-dual iteration"
            % (cfg["n_side"], cfg["n_side"] * cfg["oversample"], cfg["J"], cfg["S"], cfg["M"],
               "Dirac+db1-%d" % max(cfg["db_orders"]), cfg["levels"]))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(cfg, x_true, uvw, sample, iters=2):
    """The oracle as it stands: primal-dual iterations on a bounded sample of the visibilities
    (full image and dictionary), on this host's cores."""
    from oracle import measurement as me, solvers as so, wavelets as wv
    idx = np.random.default_rng(0).choice(len(uvw), min(sample, len(uvw)), replace=False)
    sub = uvw[np.sort(idx)]
    n, orders, L = cfg["n_side"], cfg["db_orders"], cfg["levels"]
    geo = me.Geometry(sub, n, cfg["oversample"], cfg["J"], cfg["S"])
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y = ops[0](x_true)
    wv.psi_adjoint(x_true, orders, L)  # build the cached analysis matrices outside the timing
    p = so.PDParams(gamma=1e-3, op_norm_sq=float(len(sub)), eps=1e-3 * np.linalg.norm(y), max_iter=iters)
    t0 = time.perf_counter()
    so.primal_dual(y, *ops, p)
    dt = (time.perf_counter() - t0) / iters
    cores = len(os.sched_getaffinity(0))
    return {"value": len(sub) / dt, "unit": "vis/s", "cores": cores, "kind": "oracle",
            "sample": "%d of the M visibilities (uniform subsample), full %d^2 image and dictionary, "
                      "%d primal-dual iterations, FP64; %.2f s per iteration" % (len(sub), n, iters, dt)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.config == "huge":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle is not run at the precision-study size"}))
        return 0
    cfg, seed, x_true, uvw = workload(args.config, 0)
    steps, warm = max(1, args.steps), max(0, args.warmup)
    # each step: one oracle primal-dual iteration on the bounded sample; keep the run to minutes
    steps = min(steps, 3)
    warm = min(warm, 1)
    from oracle import measurement as me, solvers as so, wavelets as wv
    idx = np.random.default_rng(0).choice(len(uvw), min(args.cpu_sample, len(uvw)), replace=False)
    sub = uvw[np.sort(idx)]
    n, orders, L = cfg["n_side"], cfg["db_orders"], cfg["levels"]
    geo = me.Geometry(sub, n, cfg["oversample"], cfg["J"], cfg["S"])
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y = ops[0](x_true)
    p = so.PDParams(gamma=1e-3, op_norm_sq=float(len(sub)), eps=1e-3 * np.linalg.norm(y), max_iter=1)
    for _ in range(warm):
        so.primal_dual(y, *ops, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        so.primal_dual(y, *ops, p)
    dt = (time.perf_counter() - t0) / steps
    v = len(sub) / dt
    cores = len(os.sched_getaffinity(0))
    line = {"metric": "Phi+Phi-dagger visibilities/s per primal-dual iteration", "value": v, "unit": "vis/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": describe(cfg) + " (oracle on a %d-visibility sample)" % len(sub)},
            "cpu_baseline": {"value": v, "unit": "vis/s", "cores": cores, "kind": "oracle",
                             "sample": "%d visibilities of the workload, one oracle primal-dual iteration per step"
                                       % len(sub)},
            "e2e": {"value": v, "unit": "vis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def serving_leg(args, dev, seed=1000, rate=None, budget_gb=None):
    """Request loop under Poisson arrivals with the job mix of the serving workload: image side
    uniform in {256, 512, 1024, 2048}, M log-uniform in [1e5, 5e7], J in {4, 6}, SARA Dirac +
    db1..db8 over 4 levels, at most 300 primal-dual iterations or relative change < 1e-3, 150 GB
    admission budget.  Coverage drawn on the device (``synth.uv_coverage_device``), data
    y = Phi x + noise kept on the device; ||Phi||^2 by 50 power iterations to 1e-4 as the server
    does.  Reports job latency p50 / p99 and throughput, and the same jobs run one at a time
    (plan, power method, solve, image to the host, back to back)."""
    import torch
    import paper_1903_04502_gb300 as g
    from paper_1903_04502_gb300 import serve
    rng = np.random.default_rng(seed)
    rate = args.serve_rate if rate is None else rate
    budget_gb = args.serve_budget_gb if budget_gb is None else budget_gb
    n_jobs = max(1, int(round(rate * args.serve_seconds)))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    jobs = []
    t_gen = time.perf_counter()
    for i in range(n_jobs):
        n = int(rng.choice([256, 512, 1024, 2048]))
        M = int(np.exp(rng.uniform(np.log(1e5), np.log(5e7))))
        J = int(rng.choice([4, 6]))
        uvw = synth.uv_coverage_device(M, seed + 17 * i + 1, dev)
        x = torch.from_numpy(synth.sky(n, 10, 4, seed=seed + i).astype(np.float32)).to(dev)
        plan = g.Plan(uvw, n, J=J)
        y0 = g.phi(plan, x)
        plan.close()
        sigma = 10 ** (-30 / 20) * float(torch.linalg.vector_norm(y0.to(torch.complex128))) / np.sqrt(M)
        y = y0 + sigma * torch.randn(M, dtype=torch.complex64, device=dev, generator=gen)
        del y0, x
        jobs.append(serve.Job(uvw=uvw, y=y, n_side=n, eps=sigma * np.sqrt(M + 2 * np.sqrt(M)), J=J,
                              db_orders=tuple(range(9)), levels=4, max_iter=300, rel_tol=1e-3,
                              arrival=float(arrivals[i])))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    eng = serve.GpuEngine(dev.index or 0)
    srv = serve.Server(eng, hbm_budget=budget_gb * 1e9, check_every=10)
    t0 = time.perf_counter()
    srv.run(jobs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    eng.close()
    st = srv.stats()
    # the same jobs, one at a time, back to back (no arrivals: device throughput with set-up)
    t1 = time.perf_counter()
    seq_vis = 0
    for j in jobs:
        plan = g.Plan(j.uvw, j.n_side, J=j.J)
        wav = g.Wavelet(j.n_side, j.levels, j.db_orders)
        opn, _ = g.op_norm(plan, 50, 1e-4, seed=j.job_id)  # as the request loop does
        s = g.Solver(plan, wav, j.y, eps=j.eps, op_norm_sq=opn)
        s.step(j.iters)
        s.x().cpu()
        seq_vis += j.iters * j.M
        s.close(); wav.close(); plan.close()
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    t_first = min(j.arrival for j in jobs)
    t_last = max(j.done_at for j in srv.done) if srv.done else t_first
    span = max(1e-9, t_last - t_first)
    return {"rate_jobs_per_s": rate, "jobs": st["jobs"], "failed": st["failed"],
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_resident": st["max_resident"],
            "iterations_per_s": srv.iterations / span, "vis_per_s": srv.vis_iterations / span,
            "span_s": span, "wall_s": wall, "one_at_a_time_vis_per_s": seq_vis / seq, "one_at_a_time_s": seq,
            "served_over_one_at_a_time": (srv.vis_iterations / span) / (seq_vis / seq),
            "budget_gb": budget_gb, "generation_s": t_gen,
            "jobs_mix": "n in {256,512,1024,2048}, M log-uniform [1e5, 5e7], J in {4,6}, inputs on the device",
            "note": "served vis/s over the span from the first arrival to the last result (includes waiting "
                    "for arrivals and the set-up of each job); one at a time includes each job's set-up"}


def wstack_leg(args, dev, cfg, seed=9000, reps=10):
    """Non-coplanar operator by w-stacking on the FP32 workload's coverage size: 1024^2 image,
    M = 1e7, J = 4, w tied to baseline length (``synth.uvw_noncoplanar``, w_frac 0.5, pixel
    size 0.5 / n_side: a 0.5 rad field), for each plane count: ms per application of Phi and
    Phi^dagger (caller order) and visibilities per second; CUDA events on the launching stream."""
    import torch
    import paper_1903_04502_gb300 as g
    n, M = cfg["n_side"], cfg["M"]
    delta = 0.5 / n
    uvw = torch.from_numpy(synth.uvw_noncoplanar(M, seed=seed, delta=delta, w_frac=0.5)).to(dev)
    x = torch.from_numpy(synth.sky(n, 10, 4, seed=seed).astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream()
    out = []
    for planes in [int(p) for p in args.wstack_planes.split(",") if p]:
        w = g.WStack(uvw, n, planes, delta, J=cfg["J"], S=cfg["S"])
        y = w.phi(x)
        xa = w.phi_adjoint(y)
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        for _ in range(reps):
            w.phi(x, y)
        b.record(stream)
        for _ in range(reps):
            w.phi_adjoint(y, xa)
        c.record(stream)
        torch.cuda.synchronize()
        t_phi, t_adj = a.elapsed_time(b) / reps, b.elapsed_time(c) / reps
        counts, _ = w.info()
        out.append({"planes": planes, "non_empty_planes": int((counts > 0).sum()), "phi_ms": t_phi,
                    "phi_adjoint_ms": t_adj, "phi_vis_per_s": M / (t_phi * 1e-3),
                    "phi_adjoint_vis_per_s": M / (t_adj * 1e-3)})
        w.close()
    return {"n_side": n, "M": M, "pixel_size": delta, "w_frac": 0.5, "runs": out,
            "note": "two coplanar applications per plane (the screened image's real and imaginary parts)"}


def sweep_leg(dev, seed=7000, M=5_000_000, reps=20):
    """The shape of the paper's CPU/GPU operator benchmark: M = 5e6 visibilities, J = 4, image
    side 256 ... 2048 (grid 512^2 ... 4096^2).  ms per application of Phi and Phi^dagger (plan
    order, with pad / crop and the FFTs), CUDA events on the launching stream, inputs resident."""
    import torch
    import paper_1903_04502_gb300 as g
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    stream = torch.cuda.current_stream()
    out = []
    for n in (256, 512, 1024, 2048):
        plan = g.Plan(synth.uv_coverage_device(M, seed + n, dev), n, J=4)
        x = torch.rand((n, n), device=dev, generator=gen)
        y = torch.empty(M, dtype=torch.complex64, device=dev)
        xo = torch.empty_like(x)
        for _ in range(3):
            g.phi(plan, x, y, plan_order=True)
            g.phi_adjoint(plan, y, xo, plan_order=True)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        for _ in range(reps):
            g.phi(plan, x, y, plan_order=True)
        b.record(stream)
        for _ in range(reps):
            g.phi_adjoint(plan, y, xo, plan_order=True)
        c.record(stream)
        torch.cuda.synchronize()
        out.append({"n_side": n, "grid": 2 * n, "M": M, "phi_ms": a.elapsed_time(b) / reps,
                    "phi_adjoint_ms": b.elapsed_time(c) / reps})
        plan.close()
    return out


def batch_leg(args, dev, seed=5000):
    """Many independent problems at once: image side uniform in {256, 512, 1024, 2048}, M
    log-uniform in [1e5, 5e7], J in {4, 6}, SARA Dirac + db1..db8 over 4 levels, FP32 with
    FP64 norms, autotuned plans.  Times the batch (one CUDA-graph launch per iteration: the
    primal-dual members on J = 4 step-layout plans share one fused degridding + gridding
    launch, the others are branches holding their own iterations), the batch without the
    shared pass, and the same problems stepped one after the other (one graph launch per
    problem and iteration)."""
    import torch
    import paper_1903_04502_gb300 as g
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    objs, Ms, tune = [], [], {}
    t_setup = time.perf_counter()
    for i in range(args.batch_problems):
        n = int(rng.choice([256, 512, 1024, 2048]))
        M = int(np.exp(rng.uniform(np.log(1e5), np.log(5e7))))
        J = int(rng.choice([4, 6]))
        uvw = synth.uv_coverage_device(M, seed + 100 + i, dev)
        plan = g.Plan(uvw, n, J=J, autotune=True)
        del uvw
        run, dg, gr = plan.launch_config()
        key = "n%d_J%d" % (n, J)
        tune.setdefault(key, []).append([M, run, dg, gr])
        x = torch.from_numpy(synth.sky(n, 10, 4, seed=seed + i).astype(np.float32)).to(dev)
        y0 = g.phi(plan, x)
        sigma = 10 ** (-30 / 20) * float(torch.linalg.vector_norm(y0.to(torch.complex128))) / np.sqrt(M)
        y = y0 + sigma * torch.randn(M, dtype=torch.complex64, device=dev, generator=gen)
        del y0, x
        opn, _ = g.op_norm(plan, 20, 1e-4, seed=i)
        wav = g.Wavelet(n, 4, tuple(range(9)))
        s = g.Solver(plan, wav, y, eps=sigma * np.sqrt(M + 2 * np.sqrt(M)), op_norm_sq=opn)
        del y
        objs.append((plan, wav, s))
        Ms.append(M)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_batch(shared):
        batch = g.Batch()
        batch.set_shared_pass(shared)
        for _, _, s in objs:
            batch.add(s)
        batch.step(3)
        torch.cuda.synchronize()
        a.record(stream)
        batch.step(args.batch_steps)
        b.record(stream)
        torch.cuda.synchronize()
        n_shared = batch.shared_members()
        batch.close()
        return a.elapsed_time(b) * 1e-3, n_shared

    # the primal-dual members on FP32 step-layout plans share one fused pass per iteration
    # (gbri_batch_set_shared_pass), and without it every member keeps its own launches
    t_batch, n_shared = time_batch(True)
    t_sep, _ = time_batch(False)
    for _, _, s in objs:
        s.step(3)
    torch.cuda.synchronize()
    a.record(stream)
    for _, _, s in objs:
        s.step(args.batch_steps)
    b.record(stream)
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b) * 1e-3
    for plan, wav, s in objs:
        s.close()
        wav.close()
        plan.close()
    vis = float(sum(Ms)) * args.batch_steps
    its = len(Ms) * args.batch_steps
    return {"problems": len(Ms), "total_visibilities": int(sum(Ms)), "steps": args.batch_steps,
            "batch_vis_per_s": vis / t_batch, "batch_iterations_per_s": its / t_batch,
            "one_by_one_vis_per_s": vis / t_seq, "one_by_one_iterations_per_s": its / t_seq,
            "speedup": t_seq / t_batch, "setup_s": t_setup, "shared_pass_members": n_shared,
            "batch_without_shared_pass_vis_per_s": vis / t_sep,
            "autotune": {k: v for k, v in sorted(tune.items())},
            "mix": "n in {256,512,1024,2048}, M log-uniform [1e5, 5e7], J in {4,6}, uv drawn on the device"}


def precision_leg(args, g, cfg, uvw_dev, y, eps, opn, gamma, ms_mixed, stream):
    """The plain FP64 path on the same workload: ms per primal-dual iteration (graph replays,
    CUDA events) and, after the workload's iteration count from x = 0 on both paths, the
    relative L2 distance of the mixed-precision image from the FP64 image."""
    import torch
    n, M = cfg["n_side"], cfg["M"]
    kw = dict(oversample=cfg["oversample"], J=cfg["J"], S=cfg["S"])
    p64 = g.Plan(uvw_dev, n, precision=g.F64, **kw)
    w64 = g.Wavelet(n, cfg["levels"], cfg["db_orders"], precision=g.F64)
    y64 = y.to(torch.complex128)
    s64 = g.Solver(p64, w64, y64, eps=eps, op_norm_sq=opn, gamma=gamma)
    s64.step(3)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s64.step(args.fp64_steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b) / args.fp64_steps
    # per-kernel breakdown of the FP64 iteration (kernel by kernel, events on the stream)
    from paper_1903_04502_gb300 import _lib
    k = min(args.fp64_steps, 20)
    g.profile_enable(k + 8)
    s64.step(k)
    torch.cuda.synchronize()
    kern64 = {}
    for i, name in enumerate(_lib.K_NAMES):
        tot, cnt = g.profile_read(i)
        if cnt:
            kern64[name] = {"ms_avg": tot / cnt, "launches": cnt}
    g.profile_enable(0)
    s64.close()
    iters = cfg["iters"]
    s64 = g.Solver(p64, w64, y64, eps=eps, op_norm_sq=opn, gamma=gamma)
    s64.step(iters)
    p32 = g.Plan(uvw_dev, n, **kw)
    w32 = g.Wavelet(n, cfg["levels"], cfg["db_orders"])
    s32 = g.Solver(p32, w32, y, eps=eps, op_norm_sq=opn, gamma=gamma)
    s32.step(iters)
    x64 = s64.x()
    x32 = s32.x().to(torch.float64)
    err = float(torch.linalg.vector_norm(x32 - x64) / torch.linalg.vector_norm(x64))
    for o in (s32, w32, p32, s64, w64, p64):
        o.close()
    return {"fp64_ms_per_step": ms64, "fp64_value": M / (ms64 * 1e-3), "mixed_ms_per_step": ms_mixed,
            "speedup_mixed_over_fp64": ms64 / ms_mixed, "iterations_compared": iters,
            "final_image_rel_err_mixed_vs_fp64": err, "fp64_steps": args.fp64_steps, "fp64_kernels": kern64,
            "note": "both paths from x = 0 with the same data, ||Phi||^2, gamma and eps; CUDA-graph replays"}


def interp_leg(args, g, cfg, uvw_dev, y, eps, opn, gamma, ms_zeroth, stream):
    """The same workload on a first-order plan (kernel taps interpolated linearly between
    table samples, coordinates quantised 256 times finer): ms per primal-dual iteration
    (graph replays, CUDA events) and its visibility kernels kernel by kernel."""
    import torch
    from paper_1903_04502_gb300 import _lib
    n, M = cfg["n_side"], cfg["M"]
    p1 = g.Plan(uvw_dev, n, oversample=cfg["oversample"], J=cfg["J"], S=cfg["S"], interp_order=1)
    w1 = g.Wavelet(n, cfg["levels"], cfg["db_orders"])
    s1 = g.Solver(p1, w1, y, eps=eps, op_norm_sq=opn, gamma=gamma)
    s1.step(3)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s1.step(args.interp_steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms1 = a.elapsed_time(b) / args.interp_steps
    k = min(args.interp_steps, 50)
    g.profile_enable(k + 8)
    s1.step(k)
    torch.cuda.synchronize()
    kern = {}
    for i, name in enumerate(_lib.K_NAMES):
        tot, cnt = g.profile_read(i)
        if cnt and name in ("degrid", "grid", "degrid_grid"):
            kern[name] = {"ms_avg": tot / cnt, "launches": cnt}
    g.profile_enable(0)
    for o in (s1, w1, p1):
        o.close()
    return {"first_order_ms_per_step": ms1, "first_order_value": M / (ms1 * 1e-3), "zeroth_order_ms_per_step": ms_zeroth,
            "first_order_kernels": kern, "steps": args.interp_steps,
            "note": "same data, ||Phi||^2, gamma and eps; FP32 path; CUDA-graph replays"}


def algorithms_leg(args, g, plan, wav, y, eps, opn, gamma, stream, nw, uvw_dev=None, cfg=None):
    """The other solvers and options on the same plan and data (graph replays, CUDA events):
    ms per iteration of Dual-FB ADMM, FISTA (default gamma), primal-dual with 8 local l2
    balls, primal-dual after one reweighting and primal-dual on a deterministic plan (its
    cost: bitwise-reproducible gridding); and the proximal operators on the workload's
    vectors (the coefficient stack and the visibilities), us per call."""
    import torch
    n, M = plan.n_side, plan.M
    steps = args.algo_steps

    def per_iter(s):
        s.step(3)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    out = {"steps": steps}
    for name, kw in (("admm", dict(algo=g.ALGO_ADMM, gamma=gamma)), ("fista", dict(algo=g.ALGO_FISTA)),
                     ("pd_local_balls_8", dict(gamma=gamma, n_balls=8)), ("pd_reweighted", dict(gamma=gamma))):
        s = g.Solver(plan, wav, y, eps=eps, op_norm_sq=opn, **kw)
        if name == "pd_reweighted":
            s.step(10)
            s.reweight(1e-3)
        out[name + "_ms_per_iter"] = per_iter(s)
        s.close()
    if uvw_dev is not None:
        pdet = g.Plan(uvw_dev, n, oversample=cfg["oversample"], J=cfg["J"], S=cfg["S"], deterministic=True)
        s = g.Solver(pdet, wav, y, eps=eps, op_norm_sq=opn, gamma=gamma)
        out["pd_deterministic_ms_per_iter"] = per_iter(s)
        s.close()
        pdet.close()

    def per_call(fn, reps=200):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e3

    gen = torch.Generator(device=y.device)
    gen.manual_seed(3)
    z = torch.randn(nw * n * n, device=y.device, generator=gen)
    w = torch.rand(nw * n * n, device=y.device, generator=gen)
    zo = torch.empty_like(z)
    yo = torch.empty_like(y)
    c0 = torch.zeros_like(y)
    out["prox_l1_us"] = per_call(lambda: g.prox_l1(z, 0.1, out=zo))
    out["prox_l1_weighted_us"] = per_call(lambda: g.prox_l1_weighted(z, w, 0.1, out=zo))
    out["proj_l2ball_us"] = per_call(lambda: g.proj_l2ball(y, c0, eps, out=yo))
    out["sizes"] = {"coefficients": nw * n * n, "visibilities": M}
    return out


def run_huge(args):
    """Precision study at full size (4096^2 image, 8192^2 grid, J = 6, M = 2e9, uv drawn on
    the device): primal-dual iterations of the mixed-precision path and of the plain FP64
    path (CUDA-graph replays, CUDA events), and the relative L2 distance of the two images
    after the same number of iterations from x = 0 with the same data and parameters."""
    import torch
    import paper_1903_04502_gb300 as g
    cfg = dict(synth.CONFIGS["huge"])
    n, M, J = cfg["n_side"], cfg["M"], cfg["J"]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    iters = args.steps
    x_true = torch.from_numpy(synth.sky(n, cfg["n_points"], cfg["n_blobs"], seed=cfg["seed"]).astype(np.float32)).to(dev)

    def timed(solver, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solver.step(k)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    out = {}
    t0 = time.perf_counter()
    plan = g.Plan(synth.uv_coverage_device(M, cfg["seed"] + 1, dev), n, J=J, S=cfg["S"])
    torch.cuda.synchronize()
    out["plan_s"] = time.perf_counter() - t0
    y = g.phi(plan, x_true)
    sigma = 10 ** (-cfg["snr_db"] / 20) * float(torch.linalg.vector_norm(y)) / np.sqrt(M)
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg["seed"] + 3)
    for a in range(0, M, 1 << 27):
        k = min(1 << 27, M - a)
        y[a:a + k] += sigma * torch.randn(k, dtype=torch.complex64, device=dev, generator=gen)
    eps = sigma * np.sqrt(M + 2 * np.sqrt(M))
    opn, _ = g.op_norm(plan, 20, 1e-4, seed=cfg["seed"])
    wav = g.Wavelet(n, cfg["levels"], cfg["db_orders"])
    s = g.Solver(plan, wav, y, eps=eps, op_norm_sq=opn)
    gamma = s.report()["gamma"]
    s.step(args.warmup)
    torch.cuda.synchronize()
    ms32 = timed(s, iters)
    x32 = s.x().cpu()
    y_host = y.cpu()
    s.close(); wav.close(); plan.close()
    del y
    torch.cuda.empty_cache()
    # plain FP64 path on the same data (the coverage is drawn again from the same seed)
    p64 = g.Plan(synth.uv_coverage_device(M, cfg["seed"] + 1, dev), n, J=J, S=cfg["S"], precision=g.F64)
    w64 = g.Wavelet(n, cfg["levels"], cfg["db_orders"], precision=g.F64)
    y64 = torch.empty(M, dtype=torch.complex128, device=dev)
    for a in range(0, M, 1 << 27):
        y64[a:a + (1 << 27)] = y_host[a:a + (1 << 27)].to(dev).to(torch.complex128)
    s64 = g.Solver(p64, w64, y64, eps=eps, op_norm_sq=opn, gamma=gamma)
    del y64
    s64.step(args.warmup)  # both paths: warmup + steps iterations from x = 0
    ms64 = timed(s64, iters)
    x64 = s64.x().cpu()
    s64.close(); w64.close(); p64.close()
    err = float(torch.linalg.vector_norm(x32.double() - x64) / torch.linalg.vector_norm(x64))
    line = {"metric": "Phi+Phi-dagger visibilities/s per primal-dual iteration (precision study)",
            "value": M / (ms32 * 1e-3), "unit": "vis/s", "n_gpus": 1, "steps": iters, "warmup": args.warmup,
            "ms_per_step": ms32, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "precision study: 4096^2 sky, 8192^2 grid, J = 6, M = 2e9, uv drawn on the device",
                       "n_side": n, "M": M, "J": J, "op_norm_sq": opn, "gamma": gamma, "plan_s": out["plan_s"]},
            "fp64_ms_per_step": ms64, "fp64_value": M / (ms64 * 1e-3), "speedup_mixed_over_fp64": ms64 / ms32,
            "final_image_rel_err_mixed_vs_fp64": err, "impl": "gbri"}
    print(json.dumps(line))
    return 0


def run_gbri(args):
    import torch
    import paper_1903_04502_gb300 as g
    from paper_1903_04502_gb300 import _lib

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    cfg, seed, x_true, uvw = workload(args.config, rank)
    n, M = cfg["n_side"], cfg["M"]
    stream = torch.cuda.current_stream()

    t_plan = time.perf_counter()
    plan = g.Plan(torch.from_numpy(uvw).to(dev), n, oversample=cfg["oversample"], J=cfg["J"], S=cfg["S"])
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    wav = g.Wavelet(n, cfg["levels"], cfg["db_orders"])
    xt = torch.from_numpy(x_true.astype(np.float32)).to(dev)
    y0 = g.phi(plan, xt)
    sigma = 10 ** (-cfg["snr_db"] / 20) * float(torch.linalg.vector_norm(y0.to(torch.complex128))) / np.sqrt(M)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 3)
    noise = torch.randn(M, dtype=torch.complex64, device=dev, generator=gen)
    y = y0 + sigma * noise
    eps = sigma * np.sqrt(M + 2 * np.sqrt(M))
    opn, _ = g.op_norm(plan, 3 if args.quick else 100, 1e-6, seed=seed)
    solver = g.Solver(plan, wav, y, eps=eps, op_norm_sq=opn)
    gamma = solver.report()["gamma"]

    # warm-up
    solver.step(args.warmup)
    torch.cuda.synchronize()
    # timed region: K iterations (each a CUDA-graph replay of one iteration)
    clocks = Clocks(dev.index if dev.index is not None else 0)
    if rank == 0:
        clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n0 = g.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = g.launch_count() - n0
    ms, value = aggregate_replicas(e0.elapsed_time(e1), M, args.steps)
    clk = clocks.stop() if rank == 0 else None
    # profiled timed region: the same iterations launched kernel by kernel, each kernel
    # bracketed by CUDA events on its launching stream (graph replay is off while timing)
    k_prof = min(args.steps, 400)
    g.profile_enable(k_prof + 8)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    solver.step(k_prof)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1) / k_prof
    kern = {}
    for k, name in enumerate(_lib.K_NAMES):
        tot, cnt = g.profile_read(k)
        if cnt:
            kern[name] = {"ms_total": tot, "launches": cnt, "ms_avg": tot / cnt}
    g.profile_enable(0)
    ms_per = ms / args.steps

    # roofline of the dominant visibility kernel (algorithmic bytes per launch)
    K = plan.K
    alg = {"degrid": 32 * M + 8 * K * (K // 2 + 1),  # meta 8 + u 8 + y 8 read, u 8 written; half spectrum once
           "grid": 16 * M + 8 * K * K,    # meta 8 + u 8 read; grid written once
           # fused degrid + grid of the updated dual: meta 8 + u 8 + y 8 read, u 8 written;
           # half spectrum read once, grid written once
           "degrid_grid": 32 * M + 8 * K * (K // 2 + 1) + 8 * K * K}
    dom = max(("degrid", "grid", "degrid_grid"), key=lambda k: kern.get(k, {}).get("ms_total", 0.0))
    peak, peak_kind = measured_peak()
    achieved = alg[dom] / (kern[dom]["ms_avg"] * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": KERNEL_TRAFFIC.get(dom) if args.config == "large" else None, "kernel": dom,
            "algorithmic_bytes": alg[dom],
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
            else "fallback 6.8 TB/s"}
    other = {"degrid": "grid", "grid": "degrid"}.get(dom)
    if other in kern:
        a2 = alg[other] / (kern[other]["ms_avg"] * 1e-3) / 1e9
        roof["other"] = {"kernel": other, "achieved": a2, "frac": a2 / peak}
    roof["per_kernel"] = per_kernel_roofline(kern, cfg, K, M, peak)

    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": ms_per, "value": value, "kernels": kern,
                              "gpu_launches": launches, "ms_per_step_profiled": ms_prof, "roofline": roof}))
        return 0
    # end to end through the public API with host buffers: pinned y in, full solve, x out
    y_host = y.cpu().pin_memory()
    x_host = torch.empty((n, n), dtype=torch.float32).pin_memory()
    iters_e2e = cfg["iters"]
    y_dev = torch.empty_like(y)
    torch.cuda.synchronize()
    e2e_steps = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        y_dev.copy_(y_host, non_blocking=True)
        x_dev, rep = g.solve(plan, wav, y_dev, eps=eps, op_norm_sq=opn, gamma=gamma, max_iter=iters_e2e)
        x_host.copy_(x_dev, non_blocking=True)
        torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": ws * M * iters_e2e / dt, "unit": "vis/s", "h2d_bytes_per_step": M * 8,
           "d2h_bytes_per_step": n * n * 4, "iterations_per_step": iters_e2e, "ms_per_step": dt * 1e3}

    # operator-level throughput (context): Phi and Phi^dagger alone, caller order, events
    xd = xt
    yd = torch.empty(M, dtype=torch.complex64, device=dev)
    for _ in range(3):
        g.phi(plan, xd, yd)
        g.phi_adjoint(plan, yd, xd.clone())
    reps = 20
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    xo = torch.empty_like(xd)
    a.record(stream)
    for _ in range(reps):
        g.phi(plan, xd, yd, plan_order=True)
    b.record(stream)
    for _ in range(reps):
        g.phi_adjoint(plan, yd, xo, plan_order=True)
    c.record(stream)
    torch.cuda.synchronize()
    ops = {"phi_vis_per_s": M * reps / (a.elapsed_time(b) * 1e-3),
           "phi_adjoint_vis_per_s": M * reps / (b.elapsed_time(c) * 1e-3)}
    # the standalone degridding and gridding kernels (Phi, Phi^dagger, the power method and
    # the solvers the fused pass does not cover), kernel by kernel with events; in Phi the
    # degridding reads the metadata and writes y (16 B per visibility), in Phi^dagger the
    # gridding reads the metadata and y (16 B)
    alg_ops = {"degrid": 16 * M + 8 * K * (K // 2 + 1), "grid": 16 * M + 8 * K * K}
    def time_standalone(pl):
        for _ in range(3):
            g.phi(pl, xd, yd, plan_order=True)
            g.phi_adjoint(pl, yd, xo, plan_order=True)
        g.profile_enable(reps + 8)
        for _ in range(reps):
            g.phi(pl, xd, yd, plan_order=True)
            g.phi_adjoint(pl, yd, xo, plan_order=True)
        torch.cuda.synchronize()
        out = {}
        for i, name in enumerate(_lib.K_NAMES):
            if name in ("degrid", "grid"):
                tot, cnt = g.profile_read(i)
                if cnt:
                    t = tot / cnt
                    a2 = alg_ops[name] / (t * 1e-3) / 1e9
                    out[name] = {"call": "phi" if name == "degrid" else "phi_adjoint", "us": t * 1e3,
                                 "achieved": a2, "frac": a2 / peak, "algorithmic_bytes": alg_ops[name]}
        g.profile_enable(0)
        return out
    # the solver's plan (step layout: the fused primal-dual pass) and the same problem on the
    # run layout (gbri_plan_desc.layout = 1), the faster layout for Phi and Phi^dagger alone
    roof["standalone"] = time_standalone(plan)
    plan_runs = g.Plan(torch.from_numpy(uvw).to(dev), n, oversample=cfg["oversample"], J=cfg["J"], S=cfg["S"],
                       layout=1)
    roof["standalone_run_layout"] = time_standalone(plan_runs)
    plan_runs.close()
    precision = None
    if args.fp64_steps > 0:
        precision = precision_leg(args, g, cfg, torch.from_numpy(uvw).to(dev), y, eps, opn, gamma, ms_per, stream)
    algorithms = None
    if args.algo_steps > 0:
        algorithms = algorithms_leg(args, g, plan, wav, y, eps, opn, gamma, stream, len(cfg["db_orders"]),
                                    torch.from_numpy(uvw).to(dev), cfg)
    wstacking = None
    if args.wstack_planes and ws == 1:
        wstacking = wstack_leg(args, dev, cfg)
    interpolation = None
    if args.interp_steps > 0:
        interpolation = interp_leg(args, g, cfg, torch.from_numpy(uvw).to(dev), y, eps, opn, gamma, ms_per, stream)

    if ws > 1:
        torch.distributed.barrier()
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(cfg, x_true, uvw, args.cpu_sample)
    sweep = None
    if not args.no_sweep and ws == 1:
        sweep = sweep_leg(dev)
    batching = None
    if args.batch_problems > 0 and ws == 1:
        batching = batch_leg(args, dev)
    serving = None
    if args.serve_seconds > 0 and ws == 1:
        solver.close()
        if args.serve_rates:
            serving = [serving_leg(args, dev, seed=1000 + 17 * i, rate=float(r))
                       for i, r in enumerate(args.serve_rates.split(","))]
        else:
            serving = serving_leg(args, dev)
    ws_bytes = plan.device_bytes + 2 * M * 8 + cfg["n_side"] ** 2 * 4 * (len(cfg["db_orders"]) + 8)
    line = {
        "metric": "Phi+Phi-dagger visibilities/s per primal-dual iteration", "value": value, "unit": "vis/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(cfg), "n_side": n, "M": M, "J": cfg["J"], "grid": K,
                   "bases": len(cfg["db_orders"]), "levels": cfg["levels"], "parallelism": "replicas" if ws > 1
                   else "single", "l2": "inputs larger than L2: per-iteration working set %.2f GB > 129 MB"
                   % (ws_bytes / 1e9), "plan_s": t_plan, "op_norm_sq": opn, "gamma": gamma},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "profiled_region": {"steps": k_prof, "ms_per_step": ms_prof, "launch": "kernel by kernel with events"},
        "clocks": clk, "kernels": kern, "operators": ops, "operator_sweep": sweep, "precision": precision,
        "interpolation": interpolation, "algorithms": algorithms, "wstacking": wstacking,
        "batching": batching,
        "serving": serving,
        "impl": "gbri",
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "huge":
        return run_huge(args)
    return run_gbri(args)


if __name__ == "__main__":
    sys.exit(main())
