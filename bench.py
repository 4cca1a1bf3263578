#!/usr/bin/env python
"""Benchmark of the batched Brinkmanlet forward model inside transitional MCMC on GB300.

Workload (one "step" = one TMCMC stage of Algorithm 1 over a batch of synthetic input):
  1024 samples per stage, N = 128 points, theta = (alpha ~ U[0,10], log10 K_C ~ U[-1,1],
  a ~ U[0.05,0.2]), observations = head (x, y) every 100 Euler steps, 2e4 steps per forward
  run, synthetic data from theta* = (1, 0, 0.1) plus 5 % Gaussian noise.  Forward Euler is
  stable only for dt below 2/lambda_max (lambda_max ~ K_C / ds^3 for the 3-point curvature
  stencil); dt = 1e-4/64 keeps dt * lambda_max <= 1 at the true K_C, so the 2e4 steps span
  2e4 * dt time units.  A stage whose annealing exponent reaches 1 is followed by a fresh
  prior draw and its log-likelihood (Algorithm 1 "Generate"), counted in the next step.

Metric: Brinkmanlet pair evaluations per second executed by the forward kernel over the
timed stages (one pair-eval = one (target, source) term, self term included), summed over
ranks, plus TMCMC samples per second.  `--impl reference` times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Brinkmanlet pair-evals/s & TMCMC samples/s, surrogate vs plain at fixed error"
N_PTS, B_STAGE, STEPS, OBS_EVERY = 128, 1024, 20000, 100
DT = 1e-4 / 64
THETA_TRUE = (1.0, 0.0, 0.1)
PRIOR_LO = (0.0, -1.0, 0.05)
PRIOR_HI = (10.0, 1.0, 0.2)
NOISE = 0.05
# FP32 flops of one unordered pair {i, j} in the symmetric pair sum (separations in units of
# delta): difference 2, u = 1 + |e|^2 4, quadratic table 8, the symmetric 2x2 mobility 7 (all
# shared by both directions), then per direction M F 8
FLOPS_PER_UNORDERED_PAIR = 37


def pair_sum_flops(ordered_pairs, unordered_per_ordered):
    """FP32 flops of the pair sum for `ordered_pairs` pair evaluations (n^2 per sample and
    step, self terms included) of which `unordered_per_ordered` are distinct unordered pairs
    (n (n - 1) / 2 per n^2)."""
    return FLOPS_PER_UNORDERED_PAIR * ordered_pairs * unordered_per_ordered


def workload_config(precision_name):
    return {
        "workload": "TMCMC stage: 1024 samples, N=128 flagellum points, 3 unknowns, head x,y every "
                    "100 steps, 2e4 Euler steps per forward run (dt=1e-4/64), 5% noise",
        "samples_per_stage": B_STAGE, "n_points": N_PTS, "steps_per_run": STEPS, "dt": DT,
        "obs_every": OBS_EVERY, "precision": precision_name,
        "l2": "256 MiB buffer written between timed steps (inputs are < L2)",
    }


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
                "samples": len(sms)}


def kernel_traffic():
    """DRAM bytes per forward run (sample) of the forward kernel from the committed ncu
    summary, if it was captured on the current kernel source (else None).  The kernel's DRAM
    traffic is the per-sample table plus the observation rows: it scales with the samples a
    launch processes, not with the time steps."""
    src = os.path.join(ROOT, "paper_1910_12007_gb300", "csrc", "forward.cu")
    path = os.path.join(ROOT, "profiles", "forward_kernel_traffic.json")
    try:
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
        with open(path) as f:
            rec = json.load(f)
        if rec.get("forward_cu_sha256") != digest:
            return None
        return rec["dram_bytes_per_sample"]
    except Exception:
        return None


# -------------------------------------------------------------------------------------
# oracle (CPU) legs
# -------------------------------------------------------------------------------------
def host_cores():
    """Host CPUs this process may run on: (count, affinity list as ranges)."""
    try:
        cpus = sorted(os.sched_getaffinity(0))
    except AttributeError:
        cpus = list(range(os.cpu_count() or 1))
    ranges, start = [], None
    for i, c in enumerate(cpus):
        if start is None:
            start = c
        if i + 1 == len(cpus) or cpus[i + 1] != c + 1:
            ranges.append(f"{start}-{c}" if c > start else f"{c}")
            start = None
    return len(cpus), ",".join(ranges)


class OracleSample:
    """The FP64 C oracle on a bounded sample of the workload: `samples` forward runs of the
    workload's swimmer (prior draws with K_C in the stable range) of `steps` Euler steps, one
    run per host core (OpenMP over runs).  The per-run kernel tables are built once, untimed,
    as the GPU path builds its tables once per run outside its per-step loop; `time()` runs
    the time loops."""

    def __init__(self, samples=None, steps=5000):
        import numpy as np

        import synthetic
        from oracle import swimmer as sw

        self.sw = sw
        self.cores, self.affinity = host_cores()
        self.samples = samples or self.cores
        self.steps = steps
        base = sw.SwimmerParams(n=N_PTS, dt=DT, steps=steps, obs_every=OBS_EVERY)
        thetas = synthetic.prior_samples(99, PRIOR_LO, PRIOR_HI, self.samples)
        thetas[:, 1] = np.minimum(thetas[:, 1], 0.2)  # stay in the stable K_C range
        self.ps = [base.with_theta(t) for t in thetas]
        self.tables = [sw.kernel_table(p) for p in self.ps]

    def time(self):
        t0 = time.perf_counter()
        self.sw.run_c_batch(self.ps, self.tables, threads=min(self.cores, self.samples))
        return time.perf_counter() - t0

    @property
    def pairs(self):
        return self.samples * N_PTS * N_PTS * self.steps

    def describe(self):
        return (f"{self.samples} forward runs x {self.steps} Euler steps of the N={N_PTS} workload swimmer (FP64 C "
                f"oracle, OpenMP over runs on {min(self.cores, self.samples)} threads, host CPUs {self.affinity}; "
                f"kernel tables built once, untimed)")


def reference_arm(args, rank):
    if rank != 0:
        return 0
    W, K = args.warmup, args.steps
    o = OracleSample()
    times = []
    for i in range(W + K):
        t = o.time()
        if i >= W:
            times.append(t)
    tot = sum(times)
    value = o.pairs * K / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * tot / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config("fp64-oracle"),
        "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": min(o.cores, o.samples),
                         "affinity": o.affinity, "kind": "oracle", "sample": "per step: " + o.describe()},
        "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------------------------
# GPU leg
# -------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave out the side-by-side leg of the plain FP64, batched FP32 and surrogate forms")
    ap.add_argument("--horizon", default="short", choices=["short", "full"],
                    help="--workload posterior: the benchmark's 2e4-step horizon, or the configured two beats "
                         "(1.28e6 steps at the stable dt)")
    ap.add_argument("--seeds", type=int, default=4, help="--workload posterior: TMCMC runs per precision")
    ap.add_argument("--shard-stage", action="store_true",
                    help="N > 1: one TMCMC population sharded over the ranks (strong scaling, one SUM "
                         "all-reduce per stage) instead of an independent TMCMC per rank (weak scaling)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one forward batch of the workload (1024 samples, 200 steps; with --workload large: "
                         "256 samples x N=1024, 50 steps) twice, for ncu, and exit")
    ap.add_argument("--batch", type=int, default=0,
                    help="--profile-case (TMCMC workload): samples in the launch (default 1024; 152 puts one on "
                         "each SM, as in a stage's last pre-fetch round)")
    ap.add_argument("--shape", default=None,
                    help="--profile-case launch shape: threads per sample, suffix w (q) for two- (four-) target "
                         "pair units (e.g. 128w); default: the untuned heuristic")
    ap.add_argument("--workload", default="tmcmc",
                    choices=["tmcmc", "uneven", "large", "surrogate", "shapes", "sperm", "sperm-tmcmc", "two-sperm",
                             "flow", "posterior"],
                    help="tmcmc (default): TMCMC stages, 1024 samples, N=128; uneven: 4096 samples with "
                         "N in {64,128,256,512} in one graph-captured persistent launch; large: 256 samples "
                         "x N=1024 x 4e4 steps; surrogate: delayed-acceptance vs plain TMCMC, 4096 samples/stage; "
                         "shapes: forward-kernel time per step vs samples per SM and threads per sample; sperm: "
                         "1024 full sperm models (flagellum 50 + head 24 points, Table Tab:param) x one beat; "
                         "sperm-tmcmc: a whole TMCMC run on the full sperm model, head-centre velocities; "
                         "two-sperm: 1024 pairs of sperm models 0.5 apart (148 points) x one beat, distances; "
                         "flow: velocity and pressure of a sperm model on a 1024 x 1024 grid; posterior: whole "
                         "TMCMC runs to q = 1 on the TMCMC workload, FP32 vs FP64 kernel, posterior moments")
    args = ap.parse_args()

    from paper_1910_12007_gb300 import ranks

    rank, world, local_rank = ranks.rank_env()
    if args.impl == "reference":
        return reference_arm(args, rank)

    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic

    if args.profile_case and args.workload == "surrogate":
        return profile_case_mlp(args, local_rank)
    if args.profile_case and args.workload == "large":
        return profile_case_large(args, local_rank)
    if args.workload in ("uneven", "large", "sperm", "two-sperm"):
        return forward_workload(args, rank, world, local_rank)
    if args.workload == "surrogate":
        return surrogate_workload(args, rank, world, local_rank)
    if args.workload == "shapes":
        return shapes_workload(args, rank, local_rank)
    if args.workload == "sperm-tmcmc":
        return sperm_tmcmc_workload(args, rank, local_rank)
    if args.workload == "flow":
        return flow_workload(args, rank, local_rank)
    if args.workload == "posterior":
        return posterior_workload(args, rank, local_rank)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    prec = g.FP64 if args.precision == "fp64" else g.FP32C
    cfg = g.SwimmerConfig(n_max=N_PTS, b_max=B_STAGE, length=1.0, dt=DT, steps=STEPS, obs_every=OBS_EVERY,
                          precision=prec)
    if args.profile_case:
        cfg.steps = 200
        h = g.swimmer_init(cfg)
        if args.shape:
            g.swimmer_tuning(h, prec, [shape_arg(g, args.shape)] * 17)
        nb = args.batch if args.batch > 0 else B_STAGE
        th = torch.tensor(synthetic.prior_samples(5, PRIOR_LO, (10.0, 0.2, 0.2), nb), device=dev)
        for rep in range(2):
            g.swimmer_profile(h, 1)
            g.forward_batch(h, th, want_traj=False)
            k2_ms, _, _, pairs, _ = g.swimmer_profile(h, 2)
        g.swimmer_profile(h, 0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": f"{nb} samples x N={N_PTS} x {cfg.steps} steps",
                          "shape": args.shape or "heuristic",
                          "k2_ms": k2_ms, "us_per_step": 1e3 * k2_ms / cfg.steps,
                          "pair_evals_per_s": pairs / (k2_ms * 1e-3),
                          "tflops": pair_sum_flops(pairs, (N_PTS - 1) / (2.0 * N_PTS)) / (k2_ms * 1e-3) / 1e12}))
        h.close()
        return 0
    h = g.swimmer_init(cfg)
    # launch shape per bucket of samples per SM (untimed), on draws of the stage-0 sampler:
    # runs that diverge early make batches uneven, which the shape choice must see
    th_tune = torch.tensor(synthetic.prior_samples(4242, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
    tuned = g.swimmer_autotune(h, steps=2000, theta=th_tune)
    shard = args.shard_stage and world > 1
    seed0 = 1000 if shard else ranks.rank_seed(1000, rank)  # one shared population, or one per rank

    # synthetic observations: forward model at theta*, plus 5 % noise (untimed set-up)
    th_true = torch.tensor([THETA_TRUE], dtype=torch.float64, device=dev)
    traj, _, st_true = g.forward_batch(h, th_true)
    xi = traj[0].cpu().numpy()
    sigma = NOISE * float(np.mean(np.abs(xi)))
    D = xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    obs = torch.tensor(D, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB

    class Job:
        """Algorithm 1 over and over: stage after stage, a fresh prior draw after q = 1."""

        def __init__(self):
            self.seed = seed0
            self.stage = 0
            self.state = None
            self.stages_done = 0

        def generate(self):
            th0 = torch.tensor(synthetic.prior_samples(self.seed, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
            if shard:  # each rank evaluates its block of the prior draws, one SUM assembles them
                a, z = ranks.shard(B_STAGE, world, rank)
                ll = torch.zeros(B_STAGE, dtype=torch.float64, device=dev)
                if z > a:
                    ll[a:z] = g.loglik_batch(h, th0[a:z].contiguous(), obs, sigma)[0]
                dist.all_reduce(ll, op=dist.ReduceOp.SUM)
            else:
                ll, _ = g.loglik_batch(h, th0, obs, sigma)
            self.state = g.TmcmcState(th0, ll, obs, sigma, PRIOR_LO, PRIOR_HI)
            self.stage = 0

        def randoms(self):
            u_res, u_acc, z = synthetic.stage_randoms(self.seed, self.stage, B_STAGE, 3)
            return np.concatenate([u_res[None], u_acc]), z

        def step(self, host_io=None):
            if self.state is None or self.state.q >= 1.0:
                self.seed += 1
                self.generate()
            U, Z = self.randoms()
            if host_io is None:
                Ud = torch.tensor(U, device=dev)
                Zd = torch.tensor(Z, device=dev)
            else:
                Ud, Zd = host_io(U, Z)
            if shard:
                g.tmcmc_stage(h, self.state, Ud, Zd, rank=rank, world=world)
                ranks.assemble_stage(dist, self.state)
            else:
                g.tmcmc_stage(h, self.state, Ud, Zd)
            self.stage += 1
            self.stages_done += 1

    job = Job()
    for _ in range(args.warmup):
        job.step()
        flush.zero_()
    torch.cuda.synchronize()

    # ---- device-timed region: inputs of each stage are made on the device side of the
    #      API (H2D of the random numbers is part of the e2e leg below)
    clocks = ClockSampler(local_rank)
    g.swimmer_profile(h, 1)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    stages0 = job.stages_done
    t0 = time.perf_counter()
    for _ in range(args.steps):
        job.step()
        flush.zero_()
    e1.record()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    barrier()
    clk = clocks.stop()
    k2_ms, k2_launches, launches, pairs_exec, pairs = g.swimmer_profile(h, 2)
    g.swimmer_profile(h, 0)
    ms_total = e0.elapsed_time(e1)
    stages = job.stages_done - stages0

    # ---- end-to-end: host buffers in, results out, per stage
    pin_u = torch.empty((3, B_STAGE), dtype=torch.float64).pin_memory()
    pin_z = torch.empty((B_STAGE, 3), dtype=torch.float64).pin_memory()
    out_th = torch.empty((B_STAGE, 3), dtype=torch.float64).pin_memory()
    out_ll = torch.empty(B_STAGE, dtype=torch.float64).pin_memory()
    dev_u = torch.empty((3, B_STAGE), dtype=torch.float64, device=dev)
    dev_z = torch.empty((B_STAGE, 3), dtype=torch.float64, device=dev)

    def host_io(U, Z):
        pin_u.copy_(torch.from_numpy(U))
        pin_z.copy_(torch.from_numpy(Z))
        dev_u.copy_(pin_u, non_blocking=True)
        dev_z.copy_(pin_z, non_blocking=True)
        return dev_u, dev_z

    g.swimmer_profile(h, 1)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for _ in range(args.steps):
        job.step(host_io)
        out_th.copy_(job.state.theta, non_blocking=True)
        out_ll.copy_(job.state.loglik, non_blocking=True)
        torch.cuda.synchronize()
    t3 = time.perf_counter()
    _, _, _, _, pairs_e2e = g.swimmer_profile(h, 2)
    g.swimmer_profile(h, 0)

    # ---- aggregate over ranks (max time, summed work)
    # a shared population counts its samples once (each rank adds its share)
    samples_mine = stages * B_STAGE / (world if shard else 1)
    (pairs_all, samples_all, pairs_e2e_all, pairs_exec_all), (ms_all, e2e_s) = ranks.totals(
        dist, [pairs, samples_mine, pairs_e2e, pairs_exec], [ms_total, t3 - t2], device=dev)

    if rank == 0:
        peaks, peak_src = load_peaks()
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        fp32_peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s
        k2_avg_ms = k2_ms / max(k2_launches, 1)
        # the kernel's rate counts every pair it executes (pre-fetched runs included)
        upo = (N_PTS - 1) / (2.0 * N_PTS)
        achieved = pair_sum_flops(pairs_exec, upo) / (k2_ms * 1e-3) / 1e12 if k2_ms > 0 else 0.0
        traffic_pp = kernel_traffic()
        value = pairs_all / (ms_all * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None,
            "dtype": "f32" if prec == g.FP32C else "f64", "data": "synthetic",
            "config": dict(workload_config(args.precision),
                           parallelism=(f"dp{world} (one TMCMC population, chains sharded over ranks, one SUM "
                                        f"all-reduce of theta/loglik per stage)") if shard
                           else f"dp{world} (independent TMCMC per GPU)"),
            "tmcmc_samples_per_s": samples_all / (ms_all * 1e-3),
            "value_counts": "pair evaluations a one-step-at-a-time TMCMC performs (pre-fetched runs off the "
                            "realized chain paths excluded)",
            "executed_pair_evals_per_s": pairs_exec_all / (ms_all * 1e-3),
            "autotuned_threads_per_sample": {f"{k}_per_sm": v for k, v in tuned.items()},
            "clocks": clk,
            "e2e": {"value": pairs_e2e_all / e2e_s, "unit": "pair-evals/s",
                    "h2d_bytes_per_step": int(6 * B_STAGE * 8),
                    "d2h_bytes_per_step": int(4 * B_STAGE * 8)},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak,
                         "traffic": (traffic_pp * pairs_exec / (N_PTS * N_PTS * STEPS) / max(k2_launches, 1))
                         if traffic_pp else None,
                         "kernel": "forward_kernel<fp32c>" if prec == g.FP32C else "forward_kernel<fp64>",
                         "launches": int(k2_launches), "avg_launch_ms": k2_avg_ms,
                         "peak_note": f"FP32 {sm_count} SMs x 128 lanes x 2 x {max_mhz:.0f} MHz ({peak_src} max clock)"},
        }
        if world == 1 and not args.no_forms:
            line["forms"] = forms_leg(dev)
        if world == 1 and not args.no_cpu_baseline:
            o = OracleSample()
            secs = o.time()
            line["cpu_baseline"] = {"value": o.pairs / secs, "unit": "pair-evals/s",
                                    "cores": min(o.cores, o.samples), "affinity": o.affinity, "kind": "oracle",
                                    "sample": o.describe()}
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


FORMS_SEEDS = 8


def forms_leg(dev, seed=700):
    """The three forms side by side on one inference problem: whole TMCMC runs to q = 1 with the
    plain FP64 kernel, the batched FP32 kernel and the FP32 kernel behind the learned surrogate
    (delayed acceptance), sharing every random number.  The TMCMC workload's swimmer (1024
    samples per stage, N = 128, dt = 1e-4/64) over a 2000-step horizon, head x, y every 50
    steps (the 40 times the surrogate predicts), noise 5 % of the head's mean displacement
    (several stages).  The surrogate is trained
    on 50k forward runs of the prior sampler by the library's MLP kernels first (timed apart).
    Samples/s count every stage's population; the posterior gaps are against the FP64 run.  The
    two FP32 forms then run again over FORMS_SEEDS further seeds, for the surrogate's posterior
    against the plain one in units of their Monte Carlo standard errors."""
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic
    from paper_1910_12007_gb300 import surrogate as sg

    steps, obs_every = 2000, 50
    cfgs = {name: g.SwimmerConfig(n_max=N_PTS, b_max=B_STAGE, length=1.0, dt=DT, steps=steps, obs_every=obs_every,
                                  precision=prec) for name, prec in (("fp64", g.FP64), ("fp32c", g.FP32C))}
    hs = {name: g.swimmer_init(c) for name, c in cfgs.items()}
    th_tune = torch.tensor(synthetic.prior_samples(4242, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
    for h in hs.values():
        g.swimmer_autotune(h, steps=200, theta=th_tune)
    xi = g.forward_batch(hs["fp64"], torch.tensor([THETA_TRUE], dtype=torch.float64, device=dev))[0][0].cpu().numpy()
    sigma = 0.05 * float(np.mean(np.abs(xi - [1.0, 0.0])))
    obs = torch.tensor(xi + sigma * synthetic.normals(1236, synthetic.NOISE, 0, xi.size).reshape(xi.shape),
                       device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th_train = torch.tensor(synthetic.prior_samples(seed + 77, PRIOR_LO, PRIOR_HI, 50000), device=dev)
    traj, status = sg.generate_training_set(hs["fp32c"], th_train)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur = sg.train(hs["fp32c"], th_train, PRIOR_LO, PRIOR_HI, epochs=40, batch=2048, lr=2e-3, seed=1, traj=traj,
                   status=status)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    th_val = torch.tensor(synthetic.prior_samples(seed + 78, PRIOR_LO, PRIOR_HI, 2048), device=dev)
    tv, sv = sg.generate_training_set(hs["fp32c"], th_val)
    val_err = sg.validation_error(sur, tv, th_val, sv)
    out = {}
    for form, name, da in (("plain_fp64", "fp64", False), ("batched_fp32", "fp32c", False),
                           ("surrogate_fp32", "fp32c", True)):
        h = hs[name]
        if da:
            sur.attach(h)
        th0 = torch.tensor(synthetic.prior_samples(seed, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
        log = []
        g.swimmer_profile(h, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.tmcmc_run(h, th0, obs, sigma, PRIOR_LO, PRIOR_HI, lambda j: synthetic.stage_randoms(seed, j, B_STAGE, 3),
                         use_surrogate=da, log=log)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        _, _, _, pairs_exec, pairs = g.swimmer_profile(h, 2)
        g.swimmer_profile(h, 0)
        th = st.theta.cpu().numpy()
        out[form] = {"tmcmc_samples_per_s": B_STAGE * (len(log) + 1) / el, "seconds": el, "stages": len(log),
                     "pair_evals_per_s": pairs / el, "executed_pair_evals_per_s": pairs_exec / el,
                     "exact_forward_runs": int(sum(s["n_exact_path"] for s in log) + B_STAGE),
                     "posterior_mean": th.mean(0).tolist(), "posterior_sd": th.std(0).tolist(),
                     "accepts": [s["n_accept"] for s in log]}
        if da:
            out[form]["screened"] = int(sum(s["n_screened"] for s in log))
            out[form]["stages_screened"] = [int(s["surrogate_used"]) for s in log]
            out[form]["surrogate_error_nats"] = [s["surrogate_error"] for s in log]
    # the two FP32 forms over more seeds: across-seed averages of the posterior moments with their
    # standard errors, so that the surrogate's gap reads against the Monte Carlo error of a run
    per = {"batched_fp32": [], "surrogate_fp32": []}
    for k in range(FORMS_SEEDS):
        sk = seed + 1 + k
        th0 = torch.tensor(synthetic.prior_samples(sk, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
        for form, da in (("batched_fp32", False), ("surrogate_fp32", True)):
            st = g.tmcmc_run(hs["fp32c"], th0, obs, sigma, PRIOR_LO, PRIOR_HI,
                             lambda j, sk=sk: synthetic.stage_randoms(sk, j, B_STAGE, 3), use_surrogate=da)
            th = st.theta.cpu().numpy()
            per[form].append((th.mean(0), th.std(0)))
    seeds = {"seeds": FORMS_SEEDS, "first_seed": seed + 1}
    for form, runs in per.items():
        mu, sd = np.array([r[0] for r in runs]), np.array([r[1] for r in runs])
        seeds[form] = {"mean": mu.mean(0).tolist(), "mean_se": (mu.std(0, ddof=1) / np.sqrt(len(runs))).tolist(),
                       "sd": sd.mean(0).tolist(), "sd_se": (sd.std(0, ddof=1) / np.sqrt(len(runs))).tolist()}
    a, b = seeds["batched_fp32"], seeds["surrogate_fp32"]
    for key in ("mean", "sd"):
        se = np.hypot(a[key + "_se"], b[key + "_se"])
        seeds[key + "_gap_in_se"] = ((np.array(b[key]) - np.array(a[key])) / se).tolist()
    seeds["sd_gap_rel"] = ((np.array(b["sd"]) - np.array(a["sd"])) / np.array(a["sd"])).tolist()
    out["surrogate_vs_plain_over_seeds"] = seeds
    for h in hs.values():
        h.close()
    m64, s64 = np.array(out["plain_fp64"]["posterior_mean"]), np.array(out["plain_fp64"]["posterior_sd"])
    for form in ("batched_fp32", "surrogate_fp32"):
        m, sd = np.array(out[form]["posterior_mean"]), np.array(out[form]["posterior_sd"])
        out[form]["mean_gap_rel_vs_fp64"] = (np.abs(m - m64) / np.maximum(np.abs(m64), s64)).tolist()
        out[form]["sd_gap_rel_vs_fp64"] = (np.abs(sd - s64) / s64).tolist()
        out[form]["same_decisions_as_fp64"] = out[form]["accepts"] == out["plain_fp64"]["accepts"]
    out["surrogate_fp32"]["training"] = {"runs": 50000, "generate_s": t_gen, "train_s": t_train,
                                         "val_rel_rmse": val_err}
    out["workload"] = ("TMCMC to q = 1, 1024 samples/stage, N=128, dt=1e-4/64, 2000 steps per run, head x,y every "
                       "50 steps, noise 5% of the head's mean displacement; shared random streams")
    out["gap_scale"] = "mean gaps relative to max(|mean|, sd) of the FP64 posterior; sd gaps relative to its sd"
    return out


def shape_arg(g, s):
    """--shape value: threads per sample, suffix w (q) for two- (four-) target pair units."""
    return int(s.rstrip("wq")) | {"w": g.SHAPE_WIDE, "q": g.SHAPE_QUAD}.get(s[-1], 0)


def profile_case_mlp(args, local_rank):
    """The surrogate MLP's forward and backward passes on 4096 samples (the delayed-acceptance
    workload's stage size), twice each: the second launches are the ones to capture."""
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    from paper_1910_12007_gb300 import api
    from paper_1910_12007_gb300 import surrogate as sg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = 4096
    params = sg.init_params(1, dev)
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.uniform(-1, 1, (n, api.MLP_IN)), dtype=torch.float32, device=dev)
    t = torch.tensor(rng.normal(0, 1, (n, api.MLP_OUT)), dtype=torch.float32, device=dev)
    ws = g.mlp_workspace(n, dev)
    times = []
    for _ in range(2):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        y = g.mlp_forward(params, x, workspace=ws)
        e1.record()
        grad, loss = g.mlp_backward(params, x, t, workspace=ws)
        e2.record()
        torch.cuda.synchronize()
        times.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    flops_fwd = 2.0 * n * (5 * 256 + 256 * 256 * 2 + 256 * 80)
    print(json.dumps({"profile_case": f"MLP 5-256-256-256-80, {n} samples", "forward_ms": times[-1][0],
                      "backward_ms": times[-1][1], "forward_tflops": flops_fwd / (times[-1][0] * 1e-3) / 1e12,
                      "finite": bool(torch.isfinite(y).all() and torch.isfinite(grad).all())}))
    return 0


def profile_case_large(args, local_rank):
    """One forward batch of the large sweep's swimmer (256 samples x N=1024, 50 steps) at the
    autotuned (or --shape) launch shape, run twice: the second launch is the one to capture."""
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B, n, steps = 256, 1024, 50
    cfg = g.SwimmerConfig(n_max=n, b_max=B, dt=1e-4 / 2 ** 15, steps=steps, obs_every=steps, precision=g.FP32C)
    h = g.swimmer_init(cfg)
    th = torch.tensor(synthetic.prior_samples(3000, (0.0, -1.0, 0.05), (50.0, 0.0, 0.2), B), device=dev)
    if args.shape:
        g.swimmer_tuning(h, g.FP32C, [shape_arg(g, args.shape)] * 17)
    else:
        g.swimmer_autotune(h, steps=steps, theta=th)
    for _ in range(2):
        g.swimmer_profile(h, 1)
        _, _, st = g.forward_batch(h, th, want_traj=False)
        k2_ms, *_ = g.swimmer_profile(h, 2)
        g.swimmer_profile(h, 0)
    torch.cuda.synchronize()
    pairs = B * n * n * steps
    print(json.dumps({"profile_case": f"{B} samples x N={n} x {steps} steps", "shape": g.swimmer_tuning(h, g.FP32C)[0],
                      "k2_ms": k2_ms, "pair_evals_per_s": pairs / (k2_ms * 1e-3),
                      "tflops": pair_sum_flops(pairs, (n - 1) / (2.0 * n)) / (k2_ms * 1e-3) / 1e12,
                      "status_ok": bool((st == 0).all())}))
    h.close()
    return 0


# -------------------------------------------------------------------------------------
# forward-only workloads: uneven N in one launch (graph-captured), large N sweep
# -------------------------------------------------------------------------------------
def forward_workload(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic

    from paper_1910_12007_gb300 import ranks

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    prec = g.FP64 if args.precision == "fp64" else g.FP32C
    if args.workload == "uneven":
        B, steps, ds = 4096, 10000, 1.0 / 255
        n_choices = [64, 128, 256, 512]
        dt = 1e-4 / 512  # dt * lambda_max <= 1 at ds = 1/255, K_C = 1
        cfg = g.SwimmerConfig(n_max=512, b_max=B, ds_fixed=ds, dt=dt, steps=steps, obs_every=steps, precision=prec)
        ns = synthetic.choice_n(ranks.rank_seed(2000, rank), n_choices, B).astype(np.int32)
        lo, hi = PRIOR_LO, (10.0, 0.0, 0.2)
        desc = ("4096 samples, N uniform in {64,128,256,512} at fixed ds=1/255 (L=(N-1)ds), 1e4 steps, "
                "dt=1e-4/512, one graph-captured persistent launch, longest first")
    elif args.workload == "two-sperm":
        # Sec. 4.2: two Table Tab:param swimmers 0.5 apart, coupled by the fluid; tail and
        # head distances observed, two noise levels
        B, steps = 1024, 40000
        dt = 1e-4 / 8
        cfg = g.SwimmerConfig(n_max=148, b_max=B, length=1.0, delta_over_ds=0.045 * 49, dt=dt, k_t=1e4,
                              omega=4 * math.pi, steps=steps, obs_every=4000, precision=prec, n_head=24,
                              k_head_tens=1e4, k_head_c=0.8, k_neck_tens=500.0, k_neck_ang=1e4,
                              obs_kind=g.OBS_PAIR_DISTANCES, n_swimmers=2, swimmer_distance=0.5, sigma_ratio=2.0)
        ns = None
        lo, hi = (0.0, 0.6, 0.08), (5.0, 0.95, 0.12)
        desc = ("1024 pairs of full sperm models (2 x (50 + 24) points) 0.5 apart, Table Tab:param stiffnesses, "
                "alpha in [0,5], K_C in [4,9], one beat (4e4 steps, dt=1e-4/8), tail and head distances every 4000 "
                "steps")
    elif args.workload == "sperm":
        # Table Tab:param: flagellum 50 points, head 24, epsilon 0.045, K_tens 1e4, K_C ~ 8,
        # K_H,tens 1e4, K_H,C 0.8, K_N,tens 500, K_N,ang 1e4, omega 4 pi, a ~ 0.1; the printed
        # dt = 1e-4 is beyond the forward-Euler bound, dt / 8 is stable; one beat (T = 0.5)
        B, steps = 1024, 40000
        dt = 1e-4 / 8
        cfg = g.SwimmerConfig(n_max=74, b_max=B, length=1.0, delta_over_ds=0.045 * 49, dt=dt, k_t=1e4,
                              omega=4 * math.pi, steps=steps, obs_every=4000, precision=prec, n_head=24,
                              k_head_tens=1e4, k_head_c=0.8, k_neck_tens=500.0, k_neck_ang=1e4,
                              obs_kind=g.OBS_HEAD_VELOCITY)
        ns = None
        lo, hi = (0.0, 0.6, 0.08), (5.0, 0.95, 0.12)
        desc = ("1024 full sperm models (flagellum 50 + head 24 points, Table Tab:param stiffnesses), alpha in "
                "[0,5], K_C in [4,9], one beat (4e4 steps, dt=1e-4/8), head-centre velocities every 4000 steps")
    else:
        B, steps = 256, 40000
        dt = 1e-4 / 2 ** 15  # dt * lambda_max <= 1 for N = 1024, K_C = 1
        cfg = g.SwimmerConfig(n_max=1024, b_max=B, dt=dt, steps=steps, obs_every=steps, precision=prec)
        ns = None
        lo, hi = (0.0, -1.0, 0.05), (50.0, 0.0, 0.2)
        desc = "256 samples x N=1024 x 4e4 steps, alpha in [0,50], dt=1e-4/2^15"
    h = g.swimmer_init(cfg)
    tuned = g.swimmer_autotune(h, steps=50)
    th = torch.tensor(synthetic.prior_samples(ranks.rank_seed(3000, rank), lo, hi, B), device=dev)
    nsd = torch.tensor(ns, device=dev) if ns is not None else None
    graph = g.ForwardGraph(h, th, nsd)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    g.swimmer_profile(h, 1)
    clocks = ClockSampler(local_rank)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    k2_ms, k2_launches, launches, pairs, _ = g.swimmer_profile(h, 2)
    # the forward kernel counts the pair evaluations each run executed (n^2 x the steps it
    # ran, so a run that stopped early counts only its steps), graph replays included
    if pairs <= 0:
        raise RuntimeError("the forward kernel's work counters read zero")
    n_tot = cfg.n_max
    status = graph.out[2].cpu().numpy()
    (pairs, ok_all, samples_all), (ms,) = ranks.totals(dist, [pairs, float(np.sum(status == 0)), B], [ms], device=dev)
    peaks, _ = load_peaks()
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sm * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    if ns is not None:
        nn = ns.astype(np.float64)
        upo = float((nn * (nn - 1) / 2).sum() / (nn ** 2).sum())
    else:
        upo = (n_tot - 1) / (2.0 * n_tot)
    achieved = pair_sum_flops(pairs, upo) / (ms * 1e-3) / 1e12
    line = {"metric": METRIC, "value": pairs / (ms * 1e-3), "unit": "pair-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == g.FP32C else "f64",
            "data": "synthetic", "config": {"workload": desc, "precision": args.precision},
            "clocks": clk, "status_ok_fraction": ok_all / samples_all,
            "autotuned_threads_per_sample": {f"{k}_per_sm": v for k, v in tuned.items()},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak,
                         "note": "whole graph (table build + forward kernel) per step"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# -------------------------------------------------------------------------------------
# launch-shape study: forward-kernel time per step vs samples per SM and threads per sample
# -------------------------------------------------------------------------------------
def shapes_workload(args, rank, local_rank):
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic

    if rank != 0:
        return 0
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    steps = 2000
    cfg = g.SwimmerConfig(n_max=N_PTS, b_max=B_STAGE, length=1.0, dt=DT, steps=steps, obs_every=OBS_EVERY,
                          precision=g.FP32C)
    h = g.swimmer_init(cfg)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # posterior-like samples (every run finishes), so the time is the kernel's, not divergence's
    lo, hi = (0.5, -0.3, 0.08), (5.0, 0.3, 0.12)
    rows = []
    for per in [0] + list(range(1, 8)):
        B = 1 if per == 0 else min(per * sms, B_STAGE)
        th = torch.tensor(synthetic.prior_samples(77, lo, hi, B), device=dev)
        row = {}
        for T in (128, 256, 512, 1024, 128 | g.SHAPE_WIDE, 256 | g.SHAPE_WIDE, 512 | g.SHAPE_WIDE, 128 | g.SHAPE_QUAD,
                  256 | g.SHAPE_QUAD, 512 | g.SHAPE_QUAD):
            try:
                g.swimmer_tuning(h, g.FP32C, [T] * 17)
            except RuntimeError:
                continue
            g.forward_batch(h, th, want_traj=False)
            torch.cuda.synchronize()
            g.swimmer_profile(h, 1)
            _, _, st = g.forward_batch(h, th, want_traj=False)
            ms, *_ = g.swimmer_profile(h, 2)
            g.swimmer_profile(h, 0)
            if bool((st == 0).all()):
                row[f"{T & 0xFFFF}{'w' if T & g.SHAPE_WIDE else 'q' if T & g.SHAPE_QUAD else ''}"] = round(ms * 1e3 / steps, 3)
        rows.append({"samples": B, "samples_per_sm": B / sms, "us_per_step_by_threads": row})
    print(json.dumps({"workload": f"forward kernel, N={N_PTS}, {steps} steps, FP32C: microseconds per time step",
                      "sms": sms, "shapes": "threads per sample, w/q: two-/four-target pair units", "rows": rows}), flush=True)
    h.close()
    return 0


# -------------------------------------------------------------------------------------
# flow and pressure fields (Eqs. BrP, BrV on a grid) of the full sperm model
# -------------------------------------------------------------------------------------
def flow_workload(args, rank, local_rank):
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g

    if rank != 0:
        return 0
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = g.SwimmerConfig(n_max=74, b_max=1, length=1.0, delta_over_ds=0.045 * 49, dt=1e-4 / 8, k_t=1e4,
                          omega=4 * math.pi, steps=40000, obs_every=4000, precision=g.FP64, n_head=24,
                          k_head_tens=1e4, k_head_c=0.8, k_neck_tens=500.0, k_neck_ang=1e4,
                          obs_kind=g.OBS_HEAD_VELOCITY)
    h = g.swimmer_init(cfg)
    _, _, status, state = g.forward_batch_state(h, torch.tensor([[1.0, math.log10(8.0), 0.1]],
                                                                dtype=torch.float64, device=dev))
    st0 = state[0].contiguous()
    n_grid = 1024
    xs = torch.linspace(-0.5, 2.0, n_grid, dtype=torch.float64, device=dev)
    ys = torch.linspace(-1.25, 1.25, n_grid, dtype=torch.float64, device=dev)
    grid = torch.stack(torch.meshgrid(xs, ys, indexing="ij"), dim=-1).reshape(-1, 2).contiguous()
    delta = 0.045
    for _ in range(max(args.warmup, 1)):
        g.swimmer_flow_field(h, 1.0, delta, 4.0, st0, grid)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        vel, pres = g.swimmer_flow_field(h, 1.0, delta, 4.0, st0, grid)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    evals = grid.shape[0] * 74
    line = {"metric": METRIC, "value": evals / (ms * 1e-3), "unit": "target-source evaluations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "velocity and pressure (Eqs. BrP, BrV) on a 1024 x 1024 grid from the final "
                                   "state of one full sperm model (74 points) after one beat, FP64, table "
                                   "build included"},
            "status": int(status[0].item()), "max_speed": float(vel.norm(dim=1).max().item()),
            "pressure_range": [float(pres.min().item()), float(pres.max().item())]}
    print(json.dumps(line), flush=True)
    h.close()
    return 0


# -------------------------------------------------------------------------------------
# a whole TMCMC run on the full sperm model (the paper's single-swimmer experiments)
# -------------------------------------------------------------------------------------
def sperm_tmcmc_workload(args, rank, local_rank):
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic

    if rank != 0:
        return 0
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # Table Tab:param swimmer, 2000 samples per stage (Sec. 4), head-centre velocities at 50
    # observation times; the horizon is T = 2 (4 beats) instead of T = 20, at the stable
    # dt = 1e-4 / 8 (1.6e5 steps per run)
    B, steps, obs_every = 2000, 160000, 3200
    cfg = g.SwimmerConfig(n_max=74, b_max=B, length=1.0, delta_over_ds=0.045 * 49, dt=1e-4 / 8, k_t=1e4,
                          omega=4 * math.pi, steps=steps, obs_every=obs_every, precision=g.FP32C, n_head=24,
                          k_head_tens=1e4, k_head_c=0.8, k_neck_tens=500.0, k_neck_ang=1e4,
                          obs_kind=g.OBS_HEAD_VELOCITY)
    h = g.swimmer_init(cfg)
    lo, hi = (0.0, 0.6, 0.08), (5.0, 0.95, 0.12)
    th_tune = torch.tensor(synthetic.prior_samples(4243, lo, hi, B), device=dev)
    g.swimmer_autotune(h, steps=2000, theta=th_tune)
    truth = (1.0, math.log10(8.0), 0.1)
    xi = g.forward_batch(h, torch.tensor([truth], dtype=torch.float64, device=dev))[0][0].cpu().numpy()
    sigma = 0.1 * float(np.mean(np.abs(xi)))  # 10 % noise
    obs = torch.tensor(xi + sigma * synthetic.normals(1235, synthetic.NOISE, 0, xi.size).reshape(xi.shape),
                       device=dev)
    th0 = torch.tensor(synthetic.prior_samples(601, lo, hi, B), device=dev)
    log = []
    g.swimmer_profile(h, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = g.tmcmc_run(h, th0, obs, sigma, lo, hi, lambda j: synthetic.stage_randoms(601, j, B, 3), log=log)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    _, _, _, pairs_exec, pairs = g.swimmer_profile(h, 2)
    g.swimmer_profile(h, 0)
    th = st.theta.cpu().numpy()
    samples = B * (len(log) + 1)  # the prior draw and every stage's population
    line = {"metric": METRIC, "value": samples / secs, "unit": "TMCMC samples/s", "n_gpus": 1, "steps": len(log),
            "warmup": 0, "ms_per_step": 1e3 * secs / max(len(log), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "TMCMC on the full sperm model (flagellum 50 + head 24 points, Table Tab:param), "
                                   "2000 samples per stage, theta = (alpha, log10 K_C, a), head-centre velocities "
                                   "at 50 times over T = 2 (1.6e5 steps per run, dt = 1e-4/8), 10 % noise"},
            "stages": len(log), "seconds": secs, "pair_evals_per_s": pairs / secs,
            "executed_pair_evals_per_s": pairs_exec / secs,
            "posterior_mean": th.mean(0).tolist(), "posterior_sd": th.std(0).tolist(), "truth": list(truth),
            "q": [s["q"] for s in log]}
    print(json.dumps(line), flush=True)
    h.close()
    return 0


# -------------------------------------------------------------------------------------
# whole TMCMC runs to q = 1 at the TMCMC workload's full size, FP32 kernel vs FP64 kernel
# -------------------------------------------------------------------------------------
def posterior_workload(args, rank, local_rank):
    """Posterior moments of the FP32 kernel against the FP64 kernel (which equals the FP64
    oracle to 1e-8 sample by sample in the tests), on the TMCMC workload: 1024 samples per
    stage, N = 128, dt = 1e-4/64, head x, y observed, 5 % noise.

    --horizon short: 2e4 Euler steps, observations every 100 (the benchmark's horizon).  Per
    seed, one FP64 and one FP32 TMCMC run sharing every random number; then the FP64
    log-likelihood at the FP32 run's final samples.
    --horizon full: the configured two beats, 1.28e6 steps, the same 200 observation times
    (every 6400 steps).  FP32 TMCMC runs; the FP64 log-likelihood at a subsample of 152 of
    their final samples (a whole FP64 TMCMC run at this horizon takes hours).

    A target posterior whose log-likelihood differs by at most eps has every moment within a
    factor exp(2 eps) of the other's; the FP64 moments follow from the FP32 samples by
    reweighting with exp(l64 - l32).  The Monte-Carlo standard error of one run's moments is the
    spread over the seeds."""
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic

    if rank != 0:
        return 0  # a comparison of two precisions on one GPU: rank 0 alone runs it
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    full = args.horizon == "full"
    steps, obs_every = (1280000, 6400) if full else (STEPS, OBS_EVERY)
    seeds = [600 + i for i in range(args.seeds)]
    hs = {}
    for name, prec in (("fp64", g.FP64), ("fp32c", g.FP32C)):
        cfg = g.SwimmerConfig(n_max=N_PTS, b_max=B_STAGE, length=1.0, dt=DT, steps=steps, obs_every=obs_every,
                              precision=prec)
        hs[name] = g.swimmer_init(cfg)
    th_tune = torch.tensor(synthetic.prior_samples(4242, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
    g.swimmer_autotune(hs["fp32c"], steps=200, theta=th_tune)
    if not full:
        g.swimmer_autotune(hs["fp64"], steps=200, theta=th_tune)
    # one data set for all runs: the FP64 model at theta* plus 5 % noise
    xi = g.forward_batch(hs["fp64"], torch.tensor([THETA_TRUE], dtype=torch.float64, device=dev))[0][0].cpu().numpy()
    sigma = NOISE * float(np.mean(np.abs(xi)))
    D = xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    obs = torch.tensor(D, dtype=torch.float64, device=dev)

    def run(name, seed):
        th0 = torch.tensor(synthetic.prior_samples(seed, PRIOR_LO, PRIOR_HI, B_STAGE), device=dev)
        log = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.tmcmc_run(hs[name], th0, obs, sigma, PRIOR_LO, PRIOR_HI,
                         lambda j: synthetic.stage_randoms(seed, j, B_STAGE, 3), log=log)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        th = st.theta.cpu().numpy()
        return th, st.loglik.cpu().numpy(), log, el

    per_seed = []
    m32s, s32s = [], []
    for seed in seeds:
        th32, ll32, log32, t32 = run("fp32c", seed)
        rec = {"seed": seed, "fp32c": {"seconds": t32, "stages": len(log32),
                                       "samples_per_s": B_STAGE * len(log32) / t32,
                                       "q": [s["q"] for s in log32], "mean": th32.mean(0).tolist(),
                                       "sd": th32.std(0).tolist(), "log_evidence": log32[-1]["log_evidence"]}}
        m32s.append(th32.mean(0))
        s32s.append(th32.std(0))
        # the FP64 log-likelihood at the FP32 run's final samples (all, or 152 of them)
        rows = np.arange(B_STAGE) if not full else np.sort(
            np.argsort(synthetic.uniforms(seed, synthetic.PRIOR, 9, B_STAGE))[:152])
        sub = torch.tensor(th32[rows], device=dev)
        ll64_at, st64 = g.loglik_batch(hs["fp64"], sub.contiguous(), obs, sigma)
        torch.cuda.synchronize()
        a, b = ll32[rows], ll64_at.cpu().numpy()
        ok = st64.cpu().numpy() == 0
        eps = float(np.max(np.abs(a - b)[ok]))
        w = np.exp(b[ok] - a[ok])
        w /= w.sum()
        t = th32[rows][ok]
        m_plain, s_plain = t.mean(0), t.std(0)
        m_rw = w @ t
        s_rw = np.sqrt(w @ (t - m_rw) ** 2)
        rec["reweighted"] = {"samples": int(ok.sum()), "max_abs_dloglik": eps,
                             "moment_bound_rel": float(np.expm1(2 * eps)),
                             "mean_gap_rel_sd": (np.abs(m_rw - m_plain) / s_plain).tolist(),
                             "sd_gap_rel": (np.abs(s_rw - s_plain) / s_plain).tolist()}
        if not full:
            th64, _, log64, t64 = run("fp64", seed)
            m64, s64 = th64.mean(0), th64.std(0)
            rec["fp64"] = {"seconds": t64, "stages": len(log64), "samples_per_s": B_STAGE * len(log64) / t64,
                           "q": [s["q"] for s in log64], "mean": m64.tolist(), "sd": s64.tolist()}
            rec["coupled"] = {"same_decisions": [s["n_accept"] for s in log32] == [s["n_accept"] for s in log64],
                              "mean_gap_rel": (np.abs(m32s[-1] - m64) / np.maximum(np.abs(m64), s64)).tolist(),
                              "sd_gap_rel": (np.abs(s32s[-1] - s64) / s64).tolist()}
        per_seed.append(rec)
        print(json.dumps({"progress": rec}), flush=True)
    for h in hs.values():
        h.close()
    m32s, s32s = np.array(m32s), np.array(s32s)
    mc_se_mean = (m32s.std(0, ddof=1) if len(seeds) > 1 else np.full(3, np.nan)).tolist()
    mc_se_sd = (s32s.std(0, ddof=1) if len(seeds) > 1 else np.full(3, np.nan)).tolist()
    worst_bound = max(r["reweighted"]["moment_bound_rel"] for r in per_seed)
    rw_mean = max(max(r["reweighted"]["mean_gap_rel_sd"]) for r in per_seed)
    rw_sd = max(max(r["reweighted"]["sd_gap_rel"]) for r in per_seed)
    secs = sum(r["fp32c"]["seconds"] for r in per_seed)
    stages = sum(r["fp32c"]["stages"] for r in per_seed)
    line = {"metric": METRIC, "value": B_STAGE * stages / secs, "unit": "TMCMC samples/s", "n_gpus": 1,
            "steps": len(seeds), "warmup": 0, "ms_per_step": 1e3 * secs / len(seeds), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"whole TMCMC runs to q = 1 on the TMCMC workload (1024 samples/stage, N=128, "
                                   f"dt=1e-4/64, {steps} steps per run, head x,y every {obs_every} steps, 5% noise), "
                                   f"FP32 kernel against the FP64 kernel, {len(seeds)} seeds",
                       "horizon": args.horizon},
            "posterior_mean_fp32": m32s.mean(0).tolist(), "posterior_sd_fp32": s32s.mean(0).tolist(),
            "mc_standard_error_of_one_run": {"mean": mc_se_mean, "sd": mc_se_sd},
            "fp32_vs_fp64_target": {"max_abs_dloglik": max(r["reweighted"]["max_abs_dloglik"] for r in per_seed),
                                    "moment_bound_rel": worst_bound, "reweighted_mean_gap_rel_sd": rw_mean,
                                    "reweighted_sd_gap_rel": rw_sd,
                                    "within_2pct": bool(rw_mean < 0.02 and rw_sd < 0.02),
                                    "note": "the FP64 posterior's moments estimated from the FP32 samples by "
                                            "weights exp(l64 - l32) (the Monte-Carlo error of the two estimates is "
                                            "shared); moment_bound_rel = exp(2 max|dl|) - 1 bounds every moment "
                                            "gap but is loose when few samples carry the largest |dl|"},
            "per_seed": per_seed}
    if not full:
        line["coupled_runs"] = {
            "same_decisions": [r["coupled"]["same_decisions"] for r in per_seed],
            "max_mean_gap_rel": max(max(r["coupled"]["mean_gap_rel"]) for r in per_seed),
            "max_sd_gap_rel": max(max(r["coupled"]["sd_gap_rel"]) for r in per_seed),
            "speedup_fp32_over_fp64": (sum(B_STAGE * r["fp32c"]["stages"] for r in per_seed) / secs) /
                                      (sum(B_STAGE * r["fp64"]["stages"] for r in per_seed) /
                                       sum(r["fp64"]["seconds"] for r in per_seed))}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------------------------
# delayed acceptance through the learned surrogate vs plain TMCMC
# -------------------------------------------------------------------------------------
def surrogate_workload(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1910_12007_gb300 as g
    import synthetic
    from paper_1910_12007_gb300 import surrogate as sg

    if rank != 0:
        return 0  # a comparison of two methods on one GPU: rank 0 alone runs it
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B = 4096
    cfg = g.SwimmerConfig(n_max=N_PTS, b_max=B, dt=DT, steps=STEPS, obs_every=OBS_EVERY, precision=g.FP32C)
    h = g.swimmer_init(cfg)
    g.swimmer_autotune(h, steps=200)
    # training set: 50k forward runs from the prior sampler of the TMCMC workload
    t0 = time.perf_counter()
    th_train = torch.tensor(synthetic.prior_samples(77 + rank, PRIOR_LO, PRIOR_HI, 50000), device=dev)
    traj, status = sg.generate_training_set(h, th_train)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur = sg.train(h, th_train, PRIOR_LO, PRIOR_HI, epochs=40, batch=2048, lr=2e-3, seed=1, traj=traj, status=status)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    th_val = torch.tensor(synthetic.prior_samples(78 + rank, PRIOR_LO, PRIOR_HI, 2048), device=dev)
    tv, sv = sg.generate_training_set(h, th_val)
    val_err = sg.validation_error(sur, tv, th_val, sv)
    th_true = torch.tensor([THETA_TRUE], dtype=torch.float64, device=dev)
    xi = g.forward_batch(h, th_true)[0][0].cpu().numpy()
    sigma = NOISE * float(np.mean(np.abs(xi)))
    obs = torch.tensor(xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape), device=dev)
    results = {}
    for mode in ("plain", "surrogate"):
        if mode == "surrogate":
            sur.attach(h)
        seed = 500 + rank
        th0 = torch.tensor(synthetic.prior_samples(seed, PRIOR_LO, PRIOR_HI, B), device=dev)
        log = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.tmcmc_run(h, th0, obs, sigma, PRIOR_LO, PRIOR_HI, lambda j: synthetic.stage_randoms(seed, j, B, 3),
                         use_surrogate=(mode == "surrogate"), log=log)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        th = st.theta.cpu().numpy()
        results[mode] = {"seconds": el, "stages": len(log), "samples_per_s": B * len(log) / el,
                         "exact_forward_runs": int(sum(s["n_exact_path"] for s in log) + B),
                         "forward_runs_executed": int(sum(s["n_exact"] for s in log) + B),
                         "screened": int(sum(s["n_screened"] for s in log)),
                         "posterior_mean": th.mean(0).tolist(), "posterior_sd": th.std(0).tolist()}
    p, d = results["plain"], results["surrogate"]
    rel_mean = [abs(a - b) / max(abs(b), 1e-12) for a, b in zip(d["posterior_mean"], p["posterior_mean"])]
    line = {"metric": METRIC, "value": d["samples_per_s"], "unit": "TMCMC samples/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * d["seconds"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "delayed-acceptance TMCMC with the MLP surrogate (trained on 50k forward runs of "
                                   "the TMCMC workload's prior sampler) vs plain TMCMC, 4096 samples/stage, N=128, "
                                   "2e4 steps per run"},
            "plain": p, "surrogate": d, "training": {"generate_s": t_gen, "train_s": t_train, "val_rel_rmse": val_err,
                                                     "final_loss": sur.losses[-1]},
            "posterior_mean_rel_diff": rel_mean,
            "speedup_samples_per_s": d["samples_per_s"] / p["samples_per_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
