"""Benchmark of one SMC^2 iteration of the CRN particle filter on synthetic data.

A step is one pass of the whole hot path: the outer proposal (Langevin), one CRN
particle filter per sample with its reverse-time adjoint, the L-kernel weights,
normalisation, ESS, estimate, recycling statistic and resampling.  The default
workload is the differentiable batched linear-Gaussian filter (d_x=4, d_y=2,
D=10, T=250, N=1024 samples, M=1024 particles).

Metric: fwd+grad CRN-PF particle-steps/s = N*M*T per step / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload lg4]

--impl reference times the FP64 CPU oracle (the plain reference implementation
of the same method) on the host cores on a bounded sample of the same workload.
Prints one JSON line on rank 0.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+grad CRN-PF particle-steps/s"
UNIT = "particle-steps/s"

# Algorithmic lane-operations per particle-step (forward + adjoint, every step stored so
# no recomputation), per model shape, in the per-item convention of the method's op
# accounting: a Philox4x32-10 call is 90 operations (10 rounds of two 32x32->64-bit
# multiplies at two operations each, two three-way XORs at two each and the key bump), a
# Box-Muller pair 9 (four transcendental + five FP32), propagation 2 d_x, observation
# d_y d_x + 3 d_y (d_y + 3 d_y with H = I), the log-sum-exp 5, resampling log2 M + 10, and
# the adjoint twice the forward's non-random FP32/INT32 arithmetic plus its exponentials.  The normals a
# particle-step needs are drawn four per Philox call, so 1-d states use a quarter call.
ALG_OPS = {"lg1": 55 + 55, "lg4": 155 + 93, "sv": 61 + 66, "lg16": 553 + 241}
# The same work counted strictly (each wide multiply, three-way XOR and transcendental one
# operation; the key schedule is precomputed): the lower bound reported beside it.
ALG_OPS_STRICT = {"lg1": 33 + 14, "lg4": 94 + 47, "sv": 36 + 15, "lg16": 333 + 154}

# DRAM bytes per filter of the forward + adjoint pair: dram__bytes_read.sum +
# dram__bytes_write.sum from ncu (one pass, no replay) over the four filter launches of the
# second SMC2 iteration of the benchmark command itself (two halves, each a forward and an
# adjoint launch) for the 4-d workload (N = 1024, M = 1024, T = 250; forward 8 particles a
# thread at 128 registers, adjoint 4 at 128; with the adjoint at 80 registers the same
# iteration moves 11.145 GB, the same bytes) and the 16-d workload (N = 2048, M = 1024,
# T = 200; 8 at 128 both), divided by N; for SV (M = 2048, T = 500; forward 8 at 64, adjoint 8
# at 128) from a capture of 304 filters.  Every step's slice is stored and read back once;
# the log-weights, tape and first-offspring rows of resampling steps add to it, so the bytes
# per filter follow the resampling rate of the sampler's population.
TRAFFIC_PER_FILTER = {("lg4", 1024, 250): (2755.332e6 + 1.253e6 + 2815.374e6 + 0.304e6 +
                                           2752.610e6 + 1.293e6 + 2815.872e6 + 0.166e6) / 1024,
                      ("sv", 2048, 500): (1.823e6 + 1552.773e6 + 1612.209e6 + 0.372e6) / 304,
                      ("lg16", 1024, 200): (14705.495e6 + 6.959e6 + 14755.096e6 + 19.128e6 +
                                            14702.515e6 + 5.834e6 + 14756.709e6 + 19.663e6) / 2048}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="lg4")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    p.add_argument("--cpu-procs", type=int, default=0, help="oracle processes (0: all host cores)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true", help="skip the short serving comparison of the line")
    p.add_argument("--mode", default="auto", choices=["auto", "sharded", "replicas"],
                   help="several GPUs: one job whose rows are split over the ranks (sharded: N rows a rank, "
                        "one all-gather of the filter outputs per iteration) or independent jobs (replicas); "
                        "auto = sharded when the job's N x ranks fits a handle")
    p.add_argument("--N", type=int, default=0, help="override the number of samples (profiling runs)")
    p.add_argument("--no-autotune", action="store_true", help="use the default launch configuration")
    p.add_argument("--hmc-steps", type=int, default=0,
                   help="run the workload with the HMC proposal of this many leapfrog steps "
                        "(step gamma / sqrt(L); every step runs the N filters)")
    p.add_argument("--nuts-depth", type=int, default=0,
                   help="run the workload with the NUTS proposal of this maximum depth J (2^J - 1 "
                        "trajectory points an iteration, each running the N filters; step "
                        "gamma / sqrt(2^J - 1))")
    p.add_argument("--resample", default="systematic", choices=["systematic", "multinomial"],
                   help="the filters' resampling scheme (multinomial is the paper's, Sec. II-B)")
    p.add_argument("--launch", default=None,
                   help="pin the launch instead of tuning: fwd_ppt,fwd_regs,adj_ppt,adj_regs,ckpt")
    p.add_argument("--experiment", default=None, choices=["lgssm"],
                   help="re-run the paper's LGSSM parameter-estimation experiment (Table II setting)")
    p.add_argument("--runs", type=int, default=5, help="independent runs per proposal (--experiment)")
    p.add_argument("--serve", action="store_true",
                   help="serving workload: Poisson-arriving jobs, batched server vs one job at a time")
    p.add_argument("--serve-jobs", type=int, default=256)
    p.add_argument("--serve-iters", type=int, default=2, help="SMC2 iterations per served job")
    p.add_argument("--serve-load", type=float, default=0.7, help="arrival rate as a fraction of capacity")
    return p.parse_args()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)

def _oracle_filter(args):
    import oracle
    fam, dx, dy, H, theta, y, M, seed, it, row, scheme = args
    r = oracle.pf(fam, dx, dy, H, theta, y, M, seed, it, row, scheme=scheme, want_tape=False)
    return r["loglik"]


def cpu_oracle_rate(w, budget_s, procs=None, pool=None):
    """Time the oracle's filter forward + forward-mode gradient on a bounded sample of the
    workload's filters: procs = 1 in this process, else a spawn pool over procs host cores (or
    the given pool of that size); returns (rate, threads, info)."""
    import multiprocessing as mp

    import numpy as np
    from paper_2407_17296_gb300 import workloads
    procs = procs or os.cpu_count() or 1
    theta = workloads.thetas_near(w, w.N, 0.05, seed=99)
    H = None if w.H is None else np.asarray(w.H, dtype=np.float64)
    # calibrate on one filter, then size the sample to the budget
    t0 = time.perf_counter()
    scheme = 1 if getattr(w, "resample", "systematic") == "multinomial" else 0
    _oracle_filter((w.family, w.dx, w.dy, H, theta[0], w.y, w.M, w.seed, 2, 0, scheme))
    one = time.perf_counter() - t0
    # enough filter runs for the budget, cycling over the iteration's filters when they
    # are fewer (small workloads would otherwise time milliseconds of pool overhead)
    n = int(max(procs, min(500000, budget_s * procs / max(one, 1e-6))))
    n = max(procs, (n // procs) * procs)
    jobs = [(w.family, w.dx, w.dy, H, theta[i % w.N], w.y, w.M, w.seed, 2, i % w.N, scheme) for i in range(n)]
    if procs == 1:
        t0 = time.perf_counter()
        for j in jobs:
            _oracle_filter(j)
        dt = time.perf_counter() - t0
    else:
        own = pool is None
        if own:
            pool = mp.get_context("spawn").Pool(procs)
        try:
            pool.map(_oracle_filter, jobs[:procs])  # start-up outside the timing
            t0 = time.perf_counter()
            pool.map(_oracle_filter, jobs, chunksize=1)
            dt = time.perf_counter() - t0
        finally:
            if own:
                pool.close()
                pool.join()
    rate = n * w.M * w.T / dt
    info = {"filters": n, "of": w.N, "seconds": dt, "single_filter_s": one}
    return rate, procs, info


def cpu_baseline_line(w, budget_s, procs=None):
    """The oracle on the host: one thread, then all cores (a third and two thirds of the budget)."""
    r1, _, i1 = cpu_oracle_rate(w, budget_s / 3.0, 1)
    rn, cores, info = cpu_oracle_rate(w, 2.0 * budget_s / 3.0, procs)
    return {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{info['filters']} filter runs over the {info['of']} filters of one iteration "
                      f"(forward + forward-mode gradient, FP64), spawn pool of {cores} processes, "
                      f"{info['seconds']:.1f} s; one thread: {i1['filters']} filter runs, {i1['seconds']:.1f} s",
            "threads_all": {"value": rn, "threads": cores},
            "threads_1": {"value": r1, "threads": 1}}


def make_workload(a):
    """The workload of the command line (both arms)."""
    from paper_2407_17296_gb300 import workloads
    w = workloads.ALL[a.workload]()
    if a.N:
        w = w.with_sizes(N=a.N)
    if a.hmc_steps:
        # leapfrog step gamma / sqrt(L): Langevin-sized steps over several points leave the
        # outer weights degenerate on these workloads
        from dataclasses import replace
        w = replace(w, proposal="hmc", hmc_steps=a.hmc_steps, gamma=w.gamma / math.sqrt(a.hmc_steps))
    if a.nuts_depth:
        from dataclasses import replace
        pts = 2 ** a.nuts_depth - 1
        w = replace(w, proposal="nuts", nuts_depth=a.nuts_depth, gamma=w.gamma / math.sqrt(pts))
    w.resample = a.resample
    return w


def points_per_step(w):
    """Filter launches (leapfrog points) of one SMC2 iteration after the first."""
    if w.proposal == "hmc":
        return w.hmc_steps
    if w.proposal == "nuts":
        return 2 ** w.nuts_depth - 1
    return 1


def workload_config(w):
    """The workload part of the JSON line's config, the same for both arms."""
    return {"workload": f"{w.name}: LG-diag d_x={w.dx} d_y={w.dy}" if w.family == 0 else f"{w.name}: SV",
            "N": w.N, "M": w.M, "T": w.T, "D": w.D, "proposal": w.proposal, "gamma": w.gamma,
            "resample": getattr(w, "resample", "systematic")}


# ------------------------------------------------------------------ GPU arm

def run_gpu(a, rank, world, local):
    import numpy as np
    import torch
    from paper_2407_17296_gb300 import binding, workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = make_workload(a)
    mode = a.mode
    if mode == "auto":
        mode = "sharded" if world > 1 and w.N * world <= 16384 and w.proposal not in ("hmc", "nuts") else "replicas"
    if mode == "sharded":
        # weak scaling of one job: N rows a rank of a job with N x ranks samples, the ranks
        # exchanging the filter outputs (one all-gather) before every outer update
        from dataclasses import replace
        w = replace(w, N=w.N * world)
        w.resample = a.resample
    else:
        # weak scaling: every rank runs its own independent job (own seed), no data-path collective
        w.seed = w.seed + 1000 * rank
    binding.load()
    stream = torch.cuda.Stream(device=dev)
    cfg = binding.config_for(w, stream=stream.cuda_stream,
                             pf_resample=binding.MULTINOMIAL if w.resample == "multinomial" else binding.SYSTEMATIC)
    if a.launch:
        binding.set_launch(cfg, [int(v) for v in a.launch.split(",")])
    elif not a.no_autotune:
        # tune on parameters near the data-generating ones: the steady state of the sampler
        binding.autotune(cfg, workloads.thetas_near(w, w.N, 0.05, seed=5))
    h = binding.Handle(cfg)
    launch = h.launch()
    if mode == "sharded":
        return run_sharded(a, rank, world, dev, w, h, stream, launch)
    ps_launch = w.N * w.M * w.T  # particle-steps of one filter launch (one leapfrog point)
    ps_per_step = ps_launch * points_per_step(w)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(a.warmup):
        h.step(want_means=False)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    launches0 = binding.kernel_launches()
    # steps replay the captured step graph with event-record nodes around the filter passes
    # (the production launch path, timed on the device)
    h.set_step_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    fwd_t, adj_t = [], []
    left = a.steps
    while left > 0:
        n = min(left, 512)
        h.run(n, want_means=False)  # n iterations back to back, one host round trip
        # the dominant kernels' mean device time over those iterations (events on the
        # handle's stream around the forward and adjoint passes of every iteration)
        f_ms, b_ms = h.step_timing()
        fwd_t += [f_ms] * n
        adj_t += [b_ms] * n
        left -= n
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = binding.kernel_launches() - launches0
    ms_total = ev0.elapsed_time(ev1)
    clocks = clk.stop()
    fwd_ms = statistics.fmean(fwd_t)
    overlapped = min(adj_t) < 0  # two halves of the filters, passes overlapped on two streams
    pf_ms = fwd_ms if overlapped else fwd_ms + statistics.fmean(adj_t)
    ll_state, _ = h.state()
    dead = int(np.sum(~np.isfinite(ll_state)))  # filters that ended early (weights vanished)
    h.set_step_timing(False)  # the end-to-end loop runs the replayed step graph

    # end to end through the C ABI with host buffers: observations in, stats + samples out
    y_host = torch.tensor(w.y, dtype=torch.float32).pin_memory().numpy()
    th_host = np.zeros((w.N, w.D))
    lw_host = np.zeros(w.N)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        h.set_observations(y_host)
        h.step(want_means=True)
        binding.check(binding.load().smc2_get_samples(h.h, binding._ptr(th_host), binding._ptr(lw_host)),
                      "smc2_get_samples")
    e2e_s = time.perf_counter() - t0

    times = torch.tensor([ms_total, e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(times, op=dist.ReduceOp.MAX)
    ms_total, e2e_s = float(times[0]), float(times[1])
    ms_step = ms_total / a.steps
    value = world * ps_per_step * a.steps / (ms_total / 1e3)
    e2e_value = world * ps_per_step * a.steps / e2e_s
    h.close()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    peak_tops = sm_count * 128 * max_mhz * 1e6 / 1e12
    achieved_tops = ALG_OPS.get(w.name, 0) * ps_launch / (pf_ms / 1e3) / 1e12
    strict_tops = ALG_OPS_STRICT.get(w.name, 0) * ps_launch / (pf_ms / 1e3) / 1e12
    per_filter = TRAFFIC_PER_FILTER.get((w.name, w.M, w.T))
    traffic = per_filter * w.N if per_filter else None
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded simulation of the model; no dataset)",
        "config": {**workload_config(w),
                   "launch": {"forward_ppt": launch[0], "forward_regs": launch[1], "adjoint_ppt": launch[2],
                              "adjoint_regs": launch[3], "ckpt_every": launch[4]},
                   "step": ("one SMC2 iteration: propose, N filters fwd+adjoint, L-kernel weights, resample"
                            if w.proposal not in ("hmc", "nuts") else
                            f"one SMC2 iteration: HMC move of {w.hmc_steps} leapfrog steps (N filters "
                            f"fwd+adjoint at each point), L-kernel weights, resample" if w.proposal == "hmc" else
                            f"one SMC2 iteration: NUTS move of depth {w.nuts_depth} ({2 ** w.nuts_depth - 1} "
                            f"lockstep trajectory points, N filters fwd+adjoint at each), weights, resample"),
                   "dead_samples": dead,
                   "l2": "inputs larger than L2 (particle trajectory of several GB written and read per step)",
                   "parallelism": f"replicas x{world} (independent jobs)" if world > 1 else "one job, one GPU"},
        "smc2_iters_per_s": 1e3 / ms_step,
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved_tops / peak_tops if peak_tops else None, "traffic": traffic,
                     "kernel": "pf_forward_kernel + pf_backward_kernel",
                     "kernel_ms": pf_ms,
                     "forward_ms": None if overlapped else fwd_ms,
                     "adjoint_ms": None if overlapped else pf_ms - fwd_ms,
                     "passes": ("two halves of the filters on two streams, forward of one overlapping "
                                "the adjoint of the other; kernel_ms spans both passes")
                               if overlapped else "forward, then adjoint",
                     "ops_per_particle_step": ALG_OPS.get(w.name),
                     "ops_per_particle_step_strict": ALG_OPS_STRICT.get(w.name),
                     "frac_strict": strict_tops / peak_tops if peak_tops else None,
                     "peak_basis": f"{sm_count} SMs x 128 FP32/INT32 lanes x {max_mhz:.0f} MHz"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(w.T * w.dy * 4),
                "d2h_bytes_per_step": int(w.N * w.D * 8 + w.N * 8 + 8 * (6 + 2 * w.D))},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if not a.no_serving and world == 1:
        out["serving"] = serving_leg()
    if not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_line(w, a.cpu_seconds, a.cpu_procs or None)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def run_sharded(a, rank, world, dev, w, h, stream, launch):
    """One SMC^2 job whose N x ranks filters are split over the ranks (sharded.py): each rank
    filters its N rows, one NCCL all-gather of the filter outputs, the outer update everywhere.
    value = filter particle-steps of the whole job per second (the max over ranks of the time)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2407_17296_gb300 import binding, sharded
    if world == 1 and not dist.is_initialized():
        import socket
        with socket.socket() as s_:
            s_.bind(("127.0.0.1", 0))
            port = s_.getsockname()[1]
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                                device_id=dev)
    eng = sharded.HandleEngine(h, stream)
    drv = sharded.ShardedSMC2(eng, w.N, w.D)
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            drv.step()
    torch.cuda.synchronize()
    clk = ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
    clk.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    launches0 = binding.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for k in range(a.steps):
            evs[k][0].record(stream)
            ll, g = eng.step_filters(drv.row0, drv.n)
            evs[k][1].record(stream)
            ll_all, g_all = drv._exchange(ll, g)
            eng.step_update(ll_all, g_all)
        ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    launches = binding.kernel_launches() - launches0
    clocks = clk.stop()
    ms_total = ev0.elapsed_time(ev1)
    pf_ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))
    # end to end: observations in, statistics and the samples out, every step
    y_host = torch.tensor(w.y, dtype=torch.float32).pin_memory().numpy()
    dist.barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(a.steps):
            h.set_observations(y_host)
            drv.step()
            h.samples()
    e2e_s = time.perf_counter() - t0
    times = torch.tensor([ms_total, e2e_s, pf_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(times, op=dist.ReduceOp.MAX)
    ms_total, e2e_s, pf_ms = float(times[0]), float(times[1]), float(times[2])
    h.close()
    if rank != 0:
        dist.destroy_process_group()
        return None
    ps_step = w.N * w.M * w.T
    props = torch.cuda.get_device_properties(dev)
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak_tops = world * props.multi_processor_count * 128 * max_mhz * 1e6 / 1e12
    achieved = ALG_OPS.get(w.name, 0) * ps_step / (pf_ms / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": ps_step * a.steps / (ms_total / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_total / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded simulation of the model; no dataset)",
        "config": {**workload_config(w),
                   "launch": {"forward_ppt": launch[0], "forward_regs": launch[1], "adjoint_ppt": launch[2],
                              "adjoint_regs": launch[3], "ckpt_every": launch[4]},
                   "step": "one SMC2 iteration of one job: propose, each rank's N/ranks filters fwd+adjoint, "
                           "all-gather of the filter outputs, L-kernel weights, resample",
                   "l2": "inputs larger than L2 (particle trajectory of several GB written and read per step)",
                   "parallelism": f"sharded x{world} (rows of one job split over the ranks, one NCCL "
                                  f"all-gather of N x (1 + D) FP64 values per iteration)"},
        "smc2_iters_per_s": 1e3 * a.steps / ms_total,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved / peak_tops, "traffic": None,
                     "kernel": "pf_forward_kernel + pf_backward_kernel (each rank's rows, max over ranks)",
                     "kernel_ms": pf_ms, "ops_per_particle_step": ALG_OPS.get(w.name),
                     "peak_basis": f"{world} x {props.multi_processor_count} SMs x 128 lanes x {max_mhz:.0f} MHz"},
        "e2e": {"value": ps_step * a.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(w.T * w.dy * 4),
                "d2h_bytes_per_step": int(w.N * w.D * 8 + w.N * 8 + 8 * (6 + 2 * w.D))},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    dist.destroy_process_group()
    return out


def run_reference(a, rank, world):
    """The CPU oracle as the reference arm: each step a bounded sample of the workload's filters
    on all host cores (one spawn pool for the whole run)."""
    if rank != 0:
        return None
    import multiprocessing as mp
    w = make_workload(a)
    procs = a.cpu_procs or os.cpu_count() or 1
    per = max(1.0, a.cpu_seconds / max(1, a.steps + a.warmup))
    rates, infos, walls = [], [], []
    with mp.get_context("spawn").Pool(procs) as pool:
        for _ in range(a.warmup):
            cpu_oracle_rate(w, per / 4, procs, pool)
        t0 = time.perf_counter()
        for _ in range(a.steps):
            s0 = time.perf_counter()
            r, cores, info = cpu_oracle_rate(w, per, procs, pool)
            walls.append(time.perf_counter() - s0)
            rates.append(r)
            infos.append(info)
        wall = time.perf_counter() - t0
    value = statistics.mean(rates)
    # what one whole iteration of the GPU arm's step (N filters at each of the move's leapfrog
    # points) would take at this rate: extrapolated, not timed
    ms_iter = 1e3 * w.N * w.M * w.T * points_per_step(w) / value
    r1, _, i1 = cpu_oracle_rate(w, max(2.0, per), 1)
    return {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * wall / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded simulation of the model; no dataset)",
        "config": {**workload_config(w),
                   "step": "a bounded sample of the workload's filters (forward + forward-mode gradient) "
                           "on the host cores; ms_per_step is its measured wall time, value the rate "
                           "in particle-steps/s",
                   "extrapolated_ms_per_iteration": ms_iter,
                   "runs_on": "host CPU cores (rank 0 only); no GPU work"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step {infos[0]['filters']} filter runs cycling over the {w.N} filters "
                                   f"of one iteration (forward + gradient), {wall:.1f} s over {a.steps} steps; "
                                   f"one thread: {i1['filters']} filter runs, {i1['seconds']:.1f} s",
                         "threads_all": {"value": value, "threads": cores},
                         "threads_1": {"value": r1, "threads": 1}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _serve_jobs(jobs, arrivals, mode, budget, max_active=16):
    """Submit the jobs at the given arrival times (seconds from the start) to a server in one
    mode: 'fused' (ready jobs step together, filter passes of jobs of one kernel variant in one
    persistent launch), 'streams' (every job on its own stream) or 'serial' (one job at a time).
    Returns (latencies [s], makespan [s])."""
    import numpy as np
    from paper_2407_17296_gb300 import binding
    lat = np.zeros(len(jobs))
    with binding.Server(budget, 1 if mode == "serial" else max_active) as srv:
        srv.set_fused(mode == "fused")
        ids = [None] * len(jobs)
        done = 0
        nxt = 0
        t0 = time.perf_counter()
        while done < len(jobs):
            now = time.perf_counter() - t0
            while nxt < len(jobs) and arrivals[nxt] <= now:
                ids[nxt] = srv.submit(binding.config_for(jobs[nxt]))
                nxt += 1
            for j in range(nxt):
                if ids[j] is not None:
                    r = srv.poll(ids[j])
                    if r is not None:
                        if r["status"] != 0:
                            raise RuntimeError(f"served job {j} failed: {r['status']}")
                        lat[j] = r["latency_s"]
                        ids[j] = None
                        done += 1
            time.sleep(0.0005)
        makespan = time.perf_counter() - t0
    return lat, makespan


def _mode_line(jobs, lat, span):
    import numpy as np
    work = float(sum(w.N * w.M * w.T * w.K for w in jobs))
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "particle_steps_per_s": work / span, "makespan_s": span}


def serving_leg(n_jobs=48, iters=2, ensemble=32):
    """Short serving comparison for the benchmark line, all jobs submitted at once (capacity):
    (1) the first n_jobs of the served mix (families lg1/lg4/sv/lg16, T ~ U[50, 1000],
    N in {256, 1024, 4096}, M in {128, 512, 2048}); (2) `ensemble` replicate runs of the small
    linear-Gaussian job (N=64, M=128, T=100, 10 iterations, own seeds), the case one job alone
    leaves most of the GPU idle; each in the three server modes."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_2407_17296_gb300 import workloads
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    mix = [replace(wl, K=iters) for _, wl in workloads.serving_stream(n_jobs=n_jobs, rate_hz=1.0)]
    ens = [replace(workloads.lg1(), seed=5000 + r) for r in range(ensemble)]
    out = {"workload": f"{n_jobs} jobs of the served mix, {iters} SMC2 iterations each, all submitted at once; "
                       f"{ensemble} replicate runs of lg1 (N=64, M=128, T=100, 10 iterations)",
           "max_active": 16}
    for name, jobs, mx in (("mix", mix, 16), ("ensemble", ens, ensemble)):
        res = {}
        for mode in ("fused", "streams", "serial"):
            lat, span = _serve_jobs(jobs, np.zeros(len(jobs)), mode, budget, mx)
            res[mode] = _mode_line(jobs, lat, span)
        res["fused_over_serial_throughput"] = res["fused"]["particle_steps_per_s"] / res["serial"]["particle_steps_per_s"]
        res["fused_over_streams_throughput"] = res["fused"]["particle_steps_per_s"] / res["streams"]["particle_steps_per_s"]
        out[name] = res
    return out


def run_serve(a):
    """256 jobs of the four model families with T ~ U[50, 1000], N in {256, 1024, 4096},
    M in {128, 512, 2048}, Poisson arrivals.
    1. capacity: all jobs submitted at once to the batched server;
    2. arrivals at serve_load x capacity and at 100% of capacity, batched (up to 16 jobs in
       flight) and serial (one job at a time, the same arrival times): p50/p99 job latency
       and throughput."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_2407_17296_gb300 import binding, workloads

    torch.cuda.set_device(0)
    binding.load()
    stream = workloads.serving_stream(n_jobs=a.serve_jobs, rate_hz=1.0)
    jobs = []
    for t, wl in stream:
        jobs.append((t, replace(wl, K=a.serve_iters)))
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)

    wls = [wl for _, wl in jobs]
    sat = {m: _serve_jobs(wls, np.zeros(len(jobs)), m, budget) for m in ("fused", "streams", "serial")}
    sat_span = sat["fused"][1]
    capacity = len(jobs) / sat_span
    base = np.array([t for t, _ in jobs])

    def at_load(load):
        lam = load * capacity
        arrivals = base * (1.0 / lam) / (base[-1] / len(jobs))  # same Poisson pattern at rate lam
        res = {"load": load, "arrival_rate_jobs_per_s": lam}
        for mode in ("fused", "streams", "serial"):
            lat, span = _serve_jobs(wls, arrivals, mode, budget)
            res[mode] = {**_mode_line(wls, lat, span), "max_active": 1 if mode == "serial" else 16}
        return res

    loads = [at_load(a.serve_load)] + ([at_load(1.0)] if a.serve_load != 1.0 else [])
    out = {
        "metric": "served-job latency p50/p99 and particle-steps/s: fused batching, per-job streams, serial",
        "workload": f"{len(jobs)} jobs, families lg1/lg4/sv/lg16, T~U[50,1000], N in {{256,1024,4096}}, "
                    f"M in {{128,512,2048}}, {a.serve_iters} SMC2 iterations per job, Poisson arrivals",
        "capacity_jobs_per_s": capacity,
        "saturated": {m: _mode_line(wls, *sat[m]) for m in sat},
        "hbm_budget_bytes": budget,
        "loads": loads,
    }
    return out


def run_lgssm_experiment(a):
    """Sec. IV-A: the linear-Gaussian model with the optimal proposal, uniform priors, T=500,
    N_x=250 particles, N=64 samples, K=15 iterations, random walk (step 0.175) and first-order
    Langevin (step 0.085) proposals, `runs` independent runs each.  Reports the recycled
    estimates averaged over runs, their mean squared error from theta* and the mean
    normalised ESS over iterations, as in Table II (whose numbers came from the paper's own
    data set; these inputs are a seeded synthetic series from the same theta*)."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_2407_17296_gb300 import binding, workloads

    torch.cuda.set_device(0)
    binding.load()
    out = {"experiment": "lgssm parameter estimation (Sec. IV-A, Table II setting)",
           "theta_star": [0.75, 1.0, 1.0], "runs": a.runs}
    for proposal in ("rw", "langevin"):
        base = workloads.lgssm(proposal=proposal)
        ws = [replace(base, seed=base.seed + 1000 * r) for r in range(a.runs)]
        # the independent runs step together: their 64 filters each (too few to fill the GPU
        # alone) run in one fused launch per pass (smc2_batch_step)
        t0 = time.perf_counter()
        hs = [binding.Handle(binding.config_for(w)) for w in ws]
        runs_stats = [[] for _ in ws]
        with binding.Batch(len(hs)) as b:
            for _ in range(base.K):
                for r, st in enumerate(b.step(hs)):
                    runs_stats[r].append(st)
        for h in hs:
            h.close()
        batched_s = time.perf_counter() - t0
        # the same runs one after the other (timing reference; identical results)
        t0 = time.perf_counter()
        for w in ws[:min(len(ws), 5)]:
            with binding.Handle(binding.config_for(w)) as h:
                for _ in range(w.K):
                    h.step()
        serial_per_run = (time.perf_counter() - t0) / min(len(ws), 5)
        means, finals, ess = [], [], []
        for stats in runs_stats:
            means.append(stats[-1]["recycled_mean"])
            finals.append(stats[-1]["mean"])
            ess.append(float(np.mean([st["ess"] for st in stats])) / base.N)
        secs = [batched_s / len(ws)]
        m = np.mean(means, axis=0)
        f = np.mean(finals, axis=0)
        out[proposal] = {"step_size": base.gamma, "E_mu": float(m[0]), "E_phi": float(m[1]),
                         "E_sigma": float(m[2]),
                         "mse": float(np.mean((m - base.theta_star) ** 2)),
                         "ess_over_N": float(np.mean(ess)),
                         "final_iteration_mean": list(map(float, f)),
                         "final_iteration_mse": float(np.mean((f - base.theta_star) ** 2)),
                         "per_run_estimates": [list(map(float, v)) for v in means],
                         "seconds_per_run": float(np.mean(secs)),
                         "seconds_per_run_one_at_a_time": serial_per_run,
                         "runs_batched": "all runs stepped together with fused filter passes"}
    return out


def main():
    a = _args()
    rank, world, local = _dist_env()
    if a.experiment == "lgssm":
        if rank == 0:
            print(json.dumps(run_lgssm_experiment(a)), flush=True)
        return
    if a.serve:
        if rank == 0:
            print(json.dumps(run_serve(a)), flush=True)
        return
    if a.impl == "reference":
        out = run_reference(a, rank, world)
    else:
        out = run_gpu(a, rank, world, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
