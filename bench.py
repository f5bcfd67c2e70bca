"""Benchmark: Metropolis updates/s of GPU population annealing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one GPU): the large-population run — 3D +-1 Edwards-Anderson spin
glass, L = 10 (1000 sites), R = 10^6 replicas, temperature steps chosen to hold
the culling fraction at 0.272 up to beta = 5, 10 sweeps per step.  A "step" is
one temperature step of the whole hot path: reweight, copy numbers + scan +
parents, parent gather + 10 Metropolis sweeps + energy levels/histogram, family
statistics.  The 2 GB double-buffered population is far larger than L2, so no
flush is needed between steps.

value   = Metropolis site updates (sum over timed steps of S N R~_t) / device time
e2e     = the same metric through the public C ABI with a host read of every
          step's observables (pa_step + pa_observables), transfers counted by the
          library
roofline: the sweep kernel (dominant), integer-ALU bound, see the design notes
cpu_baseline: the CPU oracle (OpenMP over replicas) on a bounded sample.

Under torchrun (N > 1) every rank runs an independent replica of the workload
(weak scaling, no collective on the data path); rank 0 prints the line.
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
import tempfile
import time

import numpy as np

# Hardware work queues for the many-stream batched and served runs (read by CUDA
# when it creates the context; the default is 8).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Metropolis updates/s (L=10,R=1e6)"
UNIT = "updates/s"
# Rooflines of the sweep kernels: integer instruction issue.  Their instructions
# are logic (LOP3, ISETP, SHF, ...) and integer multiplies (IMAD, the 32x32->64
# IMAD.WIDE of Philox), which share 16 lanes per clock per SM sub-partition, 64
# thread-operations per clock per SM: LOP3 alone, IMAD alone and 64-bit multiply
# + LOP3 pairs all reach 2.0e13/s on 152 SMs at 2.07 GHz, and logic added to a
# multiply-bound Philox loop adds its own time (probes of include/pa_bench.h).
# The work of one update (integer instructions per update, ncu) and the rate are
# read from each kernel's committed profile summary.
# HBM bytes per update of the sweep kernel: the tile is read (gather) and
# written once per step, i.e. 2 bytes per site and replica every S sweeps, plus
# 8 bytes of parent index and energy level per replica.

PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "sweep_L10_R1e6_adaptive.txt")
GAUSS_PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "sweep_gauss_L10_R1e6_linear101.txt")
SWEEP_SOURCE = os.path.join(ROOT, "paper_1711_02146_gb300", "csrc", "pa_sweep.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default sweep launch shapes (no autotuner launches before the timed steps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--R", type=int, default=0, help="override the population size (profiling runs)")
    ap.add_argument("--probe", action="store_true", help="also run the integer-throughput probes")
    ap.add_argument("--batched-runs", type=int, default=256,
                    help="runs of the batched mix (256 in the full workload; 0 = skip)")
    ap.add_argument("--gaussian-steps", type=int, default=6,
                    help="timed steps of the Gaussian-coupling workload (0 = skip)")
    ap.add_argument("--gaussian-R", type=int, default=0, help="override its population size (profiling runs)")
    ap.add_argument("--gaussian-only", action="store_true",
                    help="time only the Gaussian-coupling workload (profiling runs; prints its object)")
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="requests of the serving stream (2000 in the full workload; 0 = skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.skip = 0

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first sample so
        # that the samples fall inside the timed region that follows
        t_end = time.perf_counter() + 3.0
        while time.perf_counter() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.01)
        self.skip = 1 if os.path.getsize(self.path) > 0 else 0  # that first sample precedes the timed region
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        lines = open(self.path).read().splitlines()
        if len(lines) > self.skip:
            lines = lines[self.skip:]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle

def oracle_updates_per_s(w, R_sample: int, min_seconds: float, max_steps: int, n_threads: int):
    """Times the oracle as it stands on the first temperature steps of workload w
    with R reduced to R_sample; returns (updates/s, steps, seconds)."""
    import oracle
    oracle.build()
    run = oracle.Run(oracle.RunConfig(L=w.L, R=R_sample, disorder_seed=w.disorder_seed, run_seed=w.run_seed,
                                      betas=w.betas, n_temps=w.n_temps, beta_max=w.beta_max,
                                      eps_target=w.eps_target, n_sweeps=w.n_sweeps, n_pop=w.n_pop,
                                      n_threads=n_threads))
    updates, steps = 0, 0
    t0 = time.perf_counter()
    while steps < max_steps:
        if run.step() != 0:
            break
        steps += 1
        updates += w.n_sweeps * w.N * run.obs(run.t)["R_tilde"] * w.n_pop
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    return updates / dt, steps, dt


def small_config_full_run(pa, cores: int):
    """The small workload (L = 4, R = 1000, 51 linear temperatures, 10 sweeps) run
    to its end on the GPU (pa_run, creation included) and by the oracle on the host
    cores, with the two runs' final free energies side by side."""
    import torch
    import oracle
    from paper_1711_02146_gb300.workloads import C1
    oracle.build()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = pa.Run.from_workload(C1)
    r.run()
    r.sync()
    gpu_s = time.perf_counter() - t0
    g = r.obs(r.t)
    r.close()
    t0 = time.perf_counter()
    o = oracle.Run(oracle.RunConfig(L=C1.L, R=C1.R, disorder_seed=C1.disorder_seed, run_seed=C1.run_seed,
                                    betas=C1.betas, n_temps=C1.n_temps, beta_max=C1.beta_max,
                                    eps_target=C1.eps_target, n_sweeps=C1.n_sweeps, n_pop=C1.n_pop,
                                    n_threads=cores))
    while o.step() == 0:
        pass
    oracle_s = time.perf_counter() - t0
    upd = total_updates(C1)
    return {"workload": f"{C1.name}: L=4, R=1000, 51 linear temperatures to beta=5, 10 sweeps, full run",
            "gpu_seconds": gpu_s, "oracle_seconds": oracle_s, "oracle_cores": cores, "updates_approx": upd,
            "gpu_updates_per_s": upd / gpu_s, "oracle_updates_per_s": upd / oracle_s,
            "final_minus_beta_F_gpu": g["minus_beta_F"], "final_minus_beta_F_oracle": o.obs(o.t)["minus_beta_F"]}


def two_population_full_run(pa, cpu: bool, cores: int):
    """The overlap workload (L = 8, R = 1e5 per population, two populations, 201 linear
    temperatures to beta = 5, 10 sweeps) run to its end on the GPU (creation included),
    and, with cpu, the oracle timed on its first temperature steps with R = 5000."""
    import torch
    from paper_1711_02146_gb300.workloads import C2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = pa.Run.from_workload(C2)
    run.run()
    run.sync()
    dt = time.perf_counter() - t0
    st = run.stats()
    o = run.obs(run.t)
    run.close()
    out = {"workload": f"{C2.name}: L=8, R=1e5 x 2 populations, 201 linear temperatures to beta=5, 10 sweeps",
           "seconds": dt, "updates_per_s": st["updates"] / dt, "I02_final": o["I02"], "rho_t_final": o["rho_t"],
           "timing": "host clock around creation and the whole run (pa_run), one synchronisation"}
    if cpu:
        import oracle
        oracle.build()
        ref = oracle.Run(oracle.RunConfig(L=C2.L, R=5000, disorder_seed=C2.disorder_seed, run_seed=C2.run_seed,
                                          betas=C2.betas, n_sweeps=C2.n_sweeps, n_pop=2, q_bins=C2.q_bins,
                                          n_threads=cores))
        updates, n, t0 = 0, 0, time.perf_counter()
        while n < 20 and time.perf_counter() - t0 < 5.0:
            ref.step()
            n += 1
            updates += C2.n_sweeps * C2.N * (ref.obs(ref.t, 0)["R_tilde"] + ref.obs(ref.t, 1)["R_tilde"])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": updates / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first {n} temperature steps of the same run with R=5000 ({dt:.1f} s)"}
    return out


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1711_02146_gb300.workloads import C3
    cores = os.cpu_count() or 1
    R_sample = 4000
    import oracle
    oracle.build()
    run = oracle.Run(oracle.RunConfig(L=C3.L, R=R_sample, disorder_seed=C3.disorder_seed, run_seed=C3.run_seed,
                                      n_temps=C3.n_temps, beta_max=C3.beta_max, eps_target=C3.eps_target,
                                      n_sweeps=C3.n_sweeps, n_threads=cores))
    for _ in range(args.warmup):
        run.step()
    updates = 0
    t0 = time.perf_counter()
    steps = 0
    for _ in range(args.steps):
        if run.step() != 0:
            break
        steps += 1
        updates += C3.n_sweeps * C3.N * run.obs(run.t)["R_tilde"]
    dt = time.perf_counter() - t0
    value = updates / dt
    sample = (f"oracle, first {args.warmup}+{steps} temperature steps of the L=10 adaptive (eps=0.272) run "
              f"with R reduced to {R_sample}; {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": C3.name, "L": C3.L, "R": R_sample, "eps_target": C3.eps_target,
                       "n_sweeps": C3.n_sweeps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def profile_lines(path: str):
    """The machine-read `key: value` lines of a committed profile summary."""
    vals = {}
    if os.path.exists(path):
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    return vals


def source_digest() -> str:
    return hashlib.sha256(open(SWEEP_SOURCE, "rb").read()).hexdigest()[:16]


def tail_kernel(L: int, tail):
    """Name of the second sweep launch (the last wave's smaller tiles), or None."""
    if tail is None:
        return None
    return f"k_sweep<{L},{tail['words']},{tail['threads']},{tail['ctas_per_sm']}>"


def profile_traffic(kernel: str = "k_sweep<10,32,640,1>", tail=None):
    """DRAM bytes per step's sweep from the committed ncu summary, if it was taken on
    the current sweep kernel source and the launch shapes in use (else None)."""
    vals = profile_lines(PROFILE_SUMMARY)
    if vals.get("sweep_source_sha256_16") != source_digest():
        return None
    if vals.get("sweep_kernel", "k_sweep<10,32,640,1>") != kernel:
        return None
    if vals.get("sweep_tail_kernel", "none") != (tail or "none"):
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def ops_per_update(path: str):
    """(instructions per update, instructions per clock per SM, their kind, whether they
    were profiled on the current source) from a committed profile summary."""
    vals = profile_lines(path)
    try:
        return (float(vals["ops_per_update"]), float(vals["ops_per_clk_per_sm"]), vals.get("ops_kind", ""),
                vals.get("sweep_source_sha256_16") == source_digest())
    except (KeyError, ValueError):
        return None, None, "", False


def issue_peak(n_sm: int, sm_mhz: float, path: str):
    """Issue roofline in Gupdates/s and its basis, for the kernel profiled in path."""
    ops, per_clk, kind, current = ops_per_update(path)
    if ops is None:
        return None, "no instruction count profiled"
    peak = n_sm * per_clk * sm_mhz * 1e6 / ops / 1e9
    return peak, (f"{n_sm} SMs x {per_clk:.0f} thread instructions/clk x {sm_mhz:.0f} MHz / {ops:.3f} {kind} "
                  f"per update (ncu, {'this source' if current else 'an earlier source of the kernel'})")


def reduce_over_ranks(ms: float, updates: float, dist=None, device: str = "cpu"):
    """Whole-job timing of independent replicas: the slowest rank's time and the
    updates of all ranks (identity without a process group)."""
    if dist is None:
        return float(ms), float(updates)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def total_updates(w) -> int:
    """Metropolis updates of a run with an explicit schedule, counting the target R
    per step (the realised sizes fluctuate by O(sqrt R) around it)."""
    return int(w.n_sweeps * w.N * w.R * (len(w.betas) - 1) * w.n_pop)


def batched_vs_serial(pa, n_runs: int):
    """The batched mix: all runs advanced together (pa_batch: in fused rounds, one
    CUDA graph launch per temperature step for the whole batch, and, for comparison,
    each run on its own stream) vs one at a time (pa_create + pa_run + pa_destroy),
    same GPU, creation included in all three."""
    import torch
    from paper_1711_02146_gb300.workloads import batched_mix
    ws = batched_mix(256)[:n_runs]
    times, launches = {}, {}
    for mode in ("fused", "streams"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = pa.Batch(ws, mode=mode)
        b.run()
        times[mode] = time.perf_counter() - t0
        launches[mode] = b.launches()
        b.close()
    t_batch = times["fused"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for w in ws:
        r = pa.Run.from_workload(w)
        r.run()
        r.close()
    t_serial = time.perf_counter() - t0
    upd = sum(total_updates(w) for w in ws)
    return {"runs": len(ws), "workload": "L in {4,6,8,10}, R log-uniform [1e4,1e5], 101 linear temperatures, "
                                        "10 sweeps (first %d of 256 disorder seeds 100..355)" % len(ws),
            "mode": "fused: per temperature step one CUDA graph launch holding one reweighting, one resampling, "
                    "one sweep launch per L and one round-counter launch for all runs",
            "runs_per_s": len(ws) / t_batch, "serial_runs_per_s": len(ws) / t_serial,
            "speedup_vs_serial": t_serial / t_batch, "updates_per_s": upd / t_batch,
            "serial_updates_per_s": upd / t_serial, "seconds": t_batch, "serial_seconds": t_serial,
            "launches": launches["fused"],
            "streams_mode": {"runs_per_s": len(ws) / times["streams"], "seconds": times["streams"],
                             "speedup_vs_serial": t_serial / times["streams"], "launches": launches["streams"]}}


def served_vs_serial(pa, n_req: int, mem_budget: int):
    """Continuous batching: requests arrive as a Poisson stream at 0.8 x the
    served capacity (calibrated on the same mix) and are admitted by memory
    footprint; latency = finish - arrival.  Serial: each request run alone, its
    measured service time queued FIFO with the same arrivals."""
    import torch
    from paper_1711_02146_gb300.workloads import serving_stream
    reqs = serving_stream(n_req)
    ws = [w for w, _ in reqs]
    # serial service times (one request at a time on the GPU)
    service = []
    for w in ws:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pa.Run.from_workload(w)
        r.run()
        r.close()
        service.append(time.perf_counter() - t0)
    # capacity: everything submitted at once
    srv = pa.Server(mem_budget, max_active=256, steps_per_poll=4)
    t0 = time.perf_counter()
    ids = [srv.submit(w) for w in ws]
    pending = set(ids)
    while pending:
        for rid in srv.poll():
            pending.discard(rid)
    capacity = len(ws) / (time.perf_counter() - t0)
    srv.close()
    # the stream at 0.8 x capacity
    gap = 1.0 / (0.8 * capacity)
    arrivals = [a * gap for _, a in reqs]
    lat, span = serve_stream(pa, ws, arrivals, mem_budget)
    # a lighter load, 0.5 x capacity, on the first half of the stream
    n_light = max(1, len(ws) // 2)
    light_arrivals = [a / (0.5 * capacity) for _, a in reqs[:n_light]]
    light_lat, light_span = serve_stream(pa, ws[:n_light], light_arrivals, mem_budget)
    # serial FIFO queue with the same arrivals
    f_prev, slat = 0.0, []
    for a, sv in zip(arrivals, service):
        f_prev = max(a, f_prev) + sv
        slat.append(f_prev - a)
    slat = np.array(slat)
    upd = sum(total_updates(w) for w in ws)
    return {"requests": len(ws), "workload": "L in {4,6,8,10,12}, R log-uniform [1e3,2e5], 51/101/201 linear "
                                             "temperatures, 10 sweeps, Poisson arrivals (first %d of 2000)" % len(ws),
            "offered_load_runs_per_s": 0.8 * capacity, "capacity_runs_per_s": capacity,
            "runs_per_s": len(ws) / span, "updates_per_s": upd / span,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "serial_runs_per_s": len(ws) / sum(service),
            "serial_p50_latency_s": float(np.percentile(slat, 50)),
            "serial_p99_latency_s": float(np.percentile(slat, 99)),
            "throughput_vs_serial": (len(ws) / span) / (len(ws) / sum(service)),
            "capacity_vs_serial": capacity / (len(ws) / sum(service)),
            "p50_latency_serial_over_served": float(np.percentile(slat, 50) / np.percentile(lat, 50)),
            "light_load": {"requests": n_light, "offered_load_runs_per_s": 0.5 * capacity,
                           "runs_per_s": n_light / light_span,
                           "p50_latency_s": float(np.percentile(light_lat, 50)),
                           "p99_latency_s": float(np.percentile(light_lat, 99))},
            "mem_budget_bytes": mem_budget}


def serve_stream(pa, ws, arrivals, mem_budget):
    """Submits request i at arrivals[i] seconds after the start (the host polls in
    between); returns the latencies (finish - arrival) and the span from the first
    arrival to the last finish."""
    srv = pa.Server(mem_budget, max_active=256, steps_per_poll=4)
    t0 = time.perf_counter()
    finish, arrive_of = {}, {}
    nxt = 0
    while len(finish) < len(ws):
        now = time.perf_counter() - t0
        while nxt < len(ws) and arrivals[nxt] <= now:
            rid = srv.submit(ws[nxt])
            arrive_of[rid] = arrivals[nxt]
            nxt += 1
        for rid in srv.poll():
            finish[rid] = time.perf_counter() - t0
    srv.close()
    lat = np.array([finish[r] - arrive_of[r] for r in finish])
    return lat, max(finish.values()) - arrivals[0]


def autotune_shapes(pa, sizes):
    """Selects the sweep kernel's launch shape for every lattice size the bench
    runs (pa_sweep_autotune on a scratch population of about 6e8 spins: some four
    waves of the largest tiles at L = 10)."""
    out = {}
    for L in sorted(sizes):
        R = max(4096, int(6e8 // L ** 3))
        best, ms = pa.sweep_autotune(L, R, launches=3)
        shapes = pa.sweep_shapes(L)
        name = lambda sh: f"W{sh['words']}/T{sh['threads']}/x{sh['ctas_per_sm']}"
        out[str(L)] = {"selected": name(shapes[best]), "scratch_R": R,
                       "ms_per_launch": {name(sh): round(m, 4) for sh, m in zip(shapes, ms)}}
    return out


def gaussian_workload():
    """The paper's model (Gaussian couplings) at the headline size: L = 10,
    R = 1e6, 101 linear temperatures to beta = 5, 10 sweeps per step."""
    from paper_1711_02146_gb300.workloads import Workload, linear_betas
    return Workload("L10_R1e6_gauss_linear101", L=10, R=1_000_000, disorder_seed=3, run_seed=1003,
                    betas=linear_betas(101, 5.0), n_sweeps=10, model=1)


def gaussian_measurement(pa, steps: int, warmup: int, n_sm: int, cpu: bool, R: int = 0):
    """Whole-step and sweep-kernel updates/s of the Gaussian-coupling model, and
    the Gaussian oracle timed on a sample of the same run."""
    import torch
    w = gaussian_workload()
    if R:
        w = w.with_(R=R, name=f"{w.name}_R{R}")
    stream = torch.cuda.Stream()
    run = pa.Run.from_workload(w, stream=stream)
    for _ in range(warmup):
        run.step()
    run.sync()
    run.stats_reset(timing=True)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    done = 0
    for _ in range(steps):
        if run.step() != 0:
            break
        done += 1
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    st = run.stats()
    o = run.gobs(run.t)
    run.close()
    sweep_ms = st["phase_ms"]["sweep"] / max(st["phase_count"]["sweep"], 1)
    per_launch = st["updates"] / max(st["phase_count"]["sweep"], 1)
    achieved = per_launch / (sweep_ms / 1e3) / 1e9
    peak, peak_basis = issue_peak(n_sm, 2070.0, GAUSS_PROFILE_SUMMARY)
    out = {"workload": w.name, "steps_timed": f"temperature steps {warmup + 1}..{warmup + done}",
           "value": st["updates"] / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / max(done, 1),
           "sweep": {"achieved": achieved, "peak": peak, "unit": "Gupdates/s", "frac": achieved / peak if peak else None,
                     "peak_basis": peak_basis, "launch_ms": sweep_ms, "kernel": "k_sweep_g<10,32,640,1>"},
           "phase_share": {k: v / max(ms, 1e-9) for k, v in st["phase_ms"].items()},
           "last_step": {"beta": o["beta"], "R_tilde": o["R_tilde"], "mean_E_per_spin": o["mean_E"] / w.N,
                         "rho_t": o["rho_t"]}}
    # the same model with the adaptive schedule (constant culling fraction 0.272 to beta = 5),
    # whose steps include the on-device bisection of dbeta
    wa = w.with_(betas=None, n_temps=4096, beta_max=5.0, eps_target=0.272, name=w.name.replace("linear101", "adaptive"))
    run = pa.Run.from_workload(wa, stream=stream)
    for _ in range(warmup):
        run.step()
    run.sync()
    run.stats_reset(timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_ad = 0
    for _ in range(steps):
        if run.step() != 0:
            break
        n_ad += 1
    run.sync()
    dt = time.perf_counter() - t0
    sta = run.stats()
    out["adaptive"] = {"workload": wa.name, "steps_timed": n_ad, "ms_per_step": 1e3 * dt / max(n_ad, 1),
                       "updates_per_s": sta["updates"] / dt, "beta_reached": run.beta(run.t),
                       "timing": "host clock around the steps (each step waits for the device's bisection)"}
    run.close()
    if cpu:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        ref = oracle.GRun(oracle.RunConfig(L=w.L, R=20000, disorder_seed=w.disorder_seed, run_seed=w.run_seed,
                                           betas=w.betas, n_sweeps=w.n_sweeps, n_threads=cores))
        updates, n, t0 = 0, 0, time.perf_counter()
        while n < 5 and time.perf_counter() - t0 < 10.0:
            ref.step()
            n += 1
            updates += w.n_sweeps * w.N * ref.obs(ref.t)["R_tilde"]
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": updates / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first {n} temperature steps of the same run with R=2e4 ({dt:.1f} s)"}
    return out


def measured_hbm_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure of an earlier GB300 measurement


def ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1711_02146_gb300 import build, pa
    from paper_1711_02146_gb300.workloads import C3
    build.build()
    if args.gaussian_only:
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        print(json.dumps(gaussian_measurement(pa, args.gaussian_steps, args.warmup, n_sm, cpu=False,
                                              R=args.gaussian_R)), flush=True)
        return
    w = C3.with_(run_seed=C3.run_seed + 7919 * rank)
    if args.R:
        w = w.with_(R=args.R, name=f"{C3.name}_R{args.R}")
    stream = torch.cuda.Stream()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    sizes = {w.L}
    if rank == 0 and world == 1 and args.batched_runs > 0:
        sizes |= {4, 6, 8, 10}
    if rank == 0 and world == 1 and args.served_requests > 0:
        sizes |= {4, 6, 8, 10, 12}
    tuned = None if args.no_autotune else autotune_shapes(pa, sizes)

    run = pa.Run.from_workload(w, stream=stream)
    plan = run.sweep_plan()
    shapes = pa.sweep_shapes(w.L)
    shape = shapes[plan["shape"]]
    tail = shapes[plan["tail_shape"]] if plan["tail_shape"] >= 0 else None
    for _ in range(args.warmup):
        run.step()
    run.sync()
    run.stats_reset(timing=True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        done = 0
        for _ in range(args.steps):
            if run.step() != 0:
                break
            done += 1
        end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = start.elapsed_time(end)
    st = run.stats()
    ms, updates = reduce_over_ranks(ms, st["updates"], dist, "cuda")
    value = updates / (ms / 1e3)
    # resampling traffic of the timed steps (k_resample): level read, copy number
    # written and label read per old slot, parent and label written per new slot; the
    # replica copy itself is the sweep's gather
    sizes = [run.obs(u)["R_tilde"] for u in range(run.t - done, run.t + 1)]
    resample_bytes = sum(12 * r_old + 8 * r_new for r_old, r_new in zip(sizes[:-1], sizes[1:]))
    resample_ms = st["phase_ms"]["resample"]

    # e2e: the same steps through the public API, reading every step's observables back
    e2e = None
    if not args.no_e2e and not run.t >= run.n_temps - 1:
        run.stats_reset(timing=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e, prev = 0, None
        for _ in range(args.steps):
            if run.step() != 0:
                break
            if prev is not None:
                run.obs(prev)   # the previous step's observables, read while this step runs
            prev = run.t
            n_e2e += 1
        if prev is not None:
            run.obs(prev)
        dt = time.perf_counter() - t0
        s2 = run.stats()
        if n_e2e:
            e2e = {"value": s2["updates"] / dt, "unit": UNIT,
                   "h2d_bytes_per_step": s2["h2d_bytes"] // n_e2e, "d2h_bytes_per_step": s2["d2h_bytes"] // n_e2e,
                   "steps": n_e2e, "api": "pa_step of step t + 1, then pa_observables of step t (it waits for step t "
                                                 "only), every step read inside the timed region"}

    clk = clocks.summary()
    sweep_ms = st["phase_ms"]["sweep"] / max(st["phase_count"]["sweep"], 1)
    updates_per_launch = st["updates"] / max(st["phase_count"]["sweep"], 1)
    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    peak, peak_basis = issue_peak(n_sm, sm_mhz, PROFILE_SUMMARY)   # Gupdates/s
    achieved = updates_per_launch / (sweep_ms / 1e3) / 1e9
    kernel = f"k_sweep<{w.L},{shape['words']},{shape['threads']},{shape['ctas_per_sm']}>"
    traffic = profile_traffic(kernel, tail_kernel(w.L, tail))
    if traffic is not None:
        traffic = traffic * updates_per_launch / (w.n_sweeps * w.N * w.R)
    replicas = updates_per_launch / (w.n_sweeps * w.N)
    hbm_bytes = 2.0 * w.N * replicas + 8.0 * replicas
    hbm_peak = measured_hbm_gbs()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gupdates/s",
                "frac": achieved / peak if peak else None, "traffic": traffic,
                "kernel": kernel if tail is None else f"{kernel} + {tail_kernel(w.L, tail)} from slot "
                                                      f"{plan['tail_from']}",
                "launch_ms": sweep_ms, "updates_per_launch": updates_per_launch,
                "launch_note": "one step's sweep: its CUDA events bracket the tile launch and, when the last "
                               "wave of tiles runs as smaller tiles, that second launch (the kernel field names "
                               "both, and the first slot of the second)",
                "peak_basis": peak_basis + (" (median SM clock sampled during the timed region)" if clk
                                            else " (max clock, no samples)"),
                "algorithmic_bytes_per_launch": hbm_bytes,
                "hbm_GBps_achieved": hbm_bytes / (sweep_ms / 1e3) / 1e9, "hbm_GBps_peak_measured": hbm_peak,
                "hbm_frac": (hbm_bytes / (sweep_ms / 1e3) / 1e9) / hbm_peak if hbm_peak else None,
                "basis_note": "peak = the measured integer-issue budget divided by the kernel's own integer "
                              "instructions per update (ncu); a Philox-count estimate of about 19 integer "
                              "operations per update (15 for Philox, 4 for the test) would give a lower peak "
                              "than achieved, because the bit-column test draws about 2.1 Philox blocks per 32 "
                              "replicas; hbm_frac is the same launch against its algorithmic HBM bytes"}
    phase_share = {k: v / max(ms, 1e-9) for k, v in st["phase_ms"].items()}
    resample_gbs = resample_bytes / (resample_ms / 1e3) / 1e9 if resample_ms > 0 else None
    resample = {"GBps": resample_gbs, "peak_GBps": hbm_peak, "unit": "GB/s",
                "frac": resample_gbs / hbm_peak if resample_gbs and hbm_peak else None,
                "bytes_per_step": resample_bytes / max(done, 1), "ms_per_step": resample_ms / max(done, 1),
                "kernels": "k_resample (CUDA events around its launch)",
                "bytes_basis": "12 B per old slot + 8 B per new slot (algorithmic; spins move in the sweep's gather)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": done,
            "warmup": args.warmup, "ms_per_step": ms / max(done, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": w.name, "L": w.L, "R": w.R, "eps_target": w.eps_target, "beta_max": w.beta_max,
                       "n_sweeps": w.n_sweeps, "steps_timed": f"temperature steps {args.warmup + 1}.."
                                                              f"{args.warmup + done}",
                       "l2": "inputs larger than L2 (2 GB double-buffered int8 population)",
                       "sweep_shapes": tuned},
            "roofline": roofline, "resample": resample, "e2e": e2e, "gpu_launches": st["kernel_launches"],
            "phase_share": phase_share, "clocks": clk}
    run.close()
    # the many-run workloads and the Gaussian model are single-GPU measurements
    if rank == 0 and world == 1 and args.batched_runs > 0:
        line["batched"] = batched_vs_serial(pa, args.batched_runs)
    if rank == 0 and world == 1 and args.served_requests > 0:
        free, _ = torch.cuda.mem_get_info()
        line["served"] = served_vs_serial(pa, args.served_requests, int(0.5 * free))
    if rank == 0 and world == 1 and args.batched_runs > 0:   # the overlap workload, one full run
        line["two_populations"] = two_population_full_run(pa, cpu=not args.no_cpu_baseline, cores=os.cpu_count() or 1)
    if rank == 0 and world == 1 and args.gaussian_steps > 0:
        line["gaussian"] = gaussian_measurement(pa, args.gaussian_steps, args.warmup, n_sm,
                                                cpu=world == 1 and not args.no_cpu_baseline, R=args.gaussian_R)
    if args.probe:
        line["int_probes_per_s"] = {k: pa.int_throughput(k) for k in pa.PROBES}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v, steps, dt = oracle_updates_per_s(C3, R_sample=20000, min_seconds=10.0, max_steps=5, n_threads=cores)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {steps} temperature steps of the same run with R=2e4 "
                                          f"({dt:.1f} s, {cpu_model()})"}
        line["small_config"] = small_config_full_run(pa, cores)
        # the many-run workloads on the CPU, estimated from the oracle's measured rate (a
        # full pass of the oracle over them would take hours)
        for key in ("batched", "served"):
            sec = line.get(key)
            if sec and sec.get("updates_per_s"):
                n = sec.get("runs", sec.get("requests"))
                upd = sec["updates_per_s"] * (sec["seconds"] if key == "batched" else n / sec["runs_per_s"])
                sec["oracle_runs_per_s_estimate"] = n / (upd / v)
                sec["oracle_estimate_basis"] = ("the runs' updates divided by the oracle's updates/s on the "
                                                "L=10 sample above (its rate varies with L)")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
