#!/usr/bin/env python
"""Benchmark of the heated simulated bifurcation hot path on GB300.

One benchmark step is one whole run of the library's hot path over one batch
of synthetic input: seeded initial state, `sb_steps` heated discrete SB time
steps of R replicas (force J sgn(X) on the tensor cores, fused update, walls,
heating, pump schedule), energy evaluation every 100 steps with best tracking,
and the final evaluation.  Workload: one +/-1 Sherrington-Kirkpatrick instance
with N = 2000 spins (seeded stand-in for K2000), R = 1024 replicas, 2000 steps,
the paper's tuned HdSB parameters (dt = 1.1, c1 = 0.7, gamma = 0.06).

Metric: replica-spin-steps/s = N * R * sb_steps / time.

Output: one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (the reference arm of this pipeline).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "replica-spin-steps/s and % of dense tensor roofline at N=2000, R=1024 vs plain FP32 GPU"
UNIT = "replica-spin-steps/s"
WORKLOAD = dict(name="HdSB SK +/-1 N=2000 R=1024 2000 steps FP8", N=2000, J_seed=1, R=1024,
                sb_steps=2000, form="discrete", prec="fp8", c1=0.7, dt=1.1, gamma=0.06,
                init_half_width=1.0, eval_every=100, a0=1.0)
L2_FLUSH_BYTES = 256 << 20
# every source compiled into the loop kernel (its DRAM record is void once any changes)
TC_SOURCES = [os.path.join(ROOT, "paper_2203_08361_gb300", "csrc", f)
              for f in ("hsb_persist.cu", "hsb_ptx.cuh", "hsb_device.cuh", "hsb_internal.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---- one process per GPU, replicas only: no data-path collective.  Each rank
# runs R independent replicas of its own seed; the host-side collectives are
# the barriers around the timed region and the max of the ranks' times.

def rank_seed(rank: int) -> int:
    """Seed of a rank's replicas (distinct per rank: independent trials)."""
    return 1000 + rank


def max_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    """The largest of the ranks' values (the job's time is its slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank's time."""
    return world * units_per_rank / seconds


def _config(extra=None):
    w = WORKLOAD
    cfg = {"workload": w["name"], "N": w["N"], "R": w["R"], "sb_steps": w["sb_steps"],
           "form": w["form"], "prec": w["prec"], "dt": w["dt"], "c1": w["c1"],
           "gamma": w["gamma"], "eval_every": w["eval_every"], "J": f"sk_pm1(seed={w['J_seed']})"}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------- CPU oracle ---

def oracle_sample(reps: int, sb_steps: int, nthreads: int):
    """Runs the binary32 oracle (as it stands) on a sample of the workload and
    returns (replica-spin-steps/s, seconds)."""
    import oracle
    import synth
    w = WORKLOAD
    J = synth.sk_pm1(w["N"], w["J_seed"])
    op = oracle.make_params(1, oracle.c0_from_c1(J, w["c1"]), w["dt"], w["gamma"],
                            a0=w["a0"], init_half_width=w["init_half_width"],
                            eval_every=w["eval_every"])
    t0 = time.perf_counter()
    oracle.run(J, op, sb_steps, 1, range(reps), "f32", nthreads=nthreads)
    dt = time.perf_counter() - t0
    return w["N"] * reps * sb_steps / dt, dt


def cpu_baseline(target_s: float = 20.0):
    cores = os.cpu_count() or 1
    reps = max(cores, 8)
    rate, t = oracle_sample(reps, 10, cores)  # calibration
    # the whole step count of the workload on as many replicas (a multiple of
    # the thread count) as fill about target_s seconds
    steps = WORKLOAD["sb_steps"]
    want = target_s * rate / (WORKLOAD["N"] * steps)
    reps = int(min(WORKLOAD["R"], max(cores, round(want / cores) * cores)))
    rate, t = oracle_sample(reps, steps, cores)
    # the same oracle on one thread (one replica, steps for about 3 s): the
    # per-core rate, beside the all-cores figure
    r1, _ = oracle_sample(1, 10, 1)
    s1 = int(max(10, min(steps, 3.0 * r1 / WORKLOAD["N"])))
    r1, t1 = oracle_sample(1, s1, 1)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} replicas x {steps} of the {WORKLOAD['sb_steps']} steps "
                      f"(N={WORKLOAD['N']}), binary32 oracle, {cores} threads, {t:.1f} s",
            "single_thread": {"value": r1, "unit": UNIT, "cores": 1,
                              "sample": f"1 replica x {s1} steps, {t1:.1f} s"}}


def run_reference(args):
    world, rank, _ = _dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    reps = max(cores, 8)
    sb = 100
    for _ in range(args.warmup):
        oracle_sample(reps, sb, cores)
    times = []
    for _ in range(args.steps):
        _, t = oracle_sample(reps, sb, cores)
        times.append(t)
    total = sum(times)
    value = WORKLOAD["N"] * reps * sb * args.steps / total
    sample = f"{reps} replicas x {sb} steps of the workload per step (binary32 oracle, {cores} threads)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config({"sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- clocks ---

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock under load, the maximum clock, and every throttle
        reason seen active, from the sampler's CSV lines (index, clocks.sm,
        clocks.max.sm, power, active mask, then the four reason columns)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ GPU arm ----

def _traffic_for_current_kernel():
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in TC_SOURCES:
            with open(f, "rb") as fh:
                h.update(fh.read())
        sha = h.hexdigest()[:16]
        if rec.get("source_sha256_16") == sha:
            return rec.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mp = json.load(fh)
        return mp, "measured"
    except (OSError, ValueError):
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}, \
            "fallback"


FP8_PEAK_FILE = os.path.join(ROOT, "profiles", "fp8_peak.json")


def fp8_denominator(mp, src):
    """Dense FP8 denominator of a kernel timed alone at full clock: the larger
    of 2 x the BF16 burst peak (nominal FP8/BF16 ratio 4.5/2.25) and the FP8
    burst rate measured with `bench.py --fp8-peak` (profiles/fp8_peak.json)."""
    bf16 = float(mp.get("bf16_tflops", mp.get("bf16_tflops_sustained")))
    peak, how = 2.0 * bf16, f"2 x bf16 burst of {src} peaks ({2.0 * bf16:.1f})"
    try:
        with open(FP8_PEAK_FILE) as fh:
            fp8 = float(json.load(fh)["fp8_tflops"])
        how += f"; cuBLAS FP8 burst measured {fp8:.1f}"
        if fp8 > peak:
            peak, how = fp8, how + " (taken)"
    except (OSError, ValueError, KeyError):
        pass
    return peak, how


def fp8_dense_peak(n: int = 8192, seconds: float = 4.0):
    """Dense FP8 e4m3 tensor rate of this GPU through the vendor library:
    torch._scaled_mm at n^3 (2 n^3 flops per call, unit scales, FP32
    accumulation, bf16 output), timed with CUDA events on one stream.  Returns
    the best of 10 single calls (burst) and a back-to-back loop of `seconds`
    (sustained), each with the SM clocks sampled meanwhile."""
    import torch
    torch.cuda.set_device(0)
    gen = torch.Generator(device="cuda").manual_seed(0)
    a = torch.randn(n, n, device="cuda", generator=gen).to(torch.float8_e4m3fn)
    b = torch.randn(n, n, device="cuda", generator=gen).to(torch.float8_e4m3fn)
    one = torch.ones((), dtype=torch.float32, device="cuda")

    def mm():
        return torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)

    for _ in range(5):
        mm()
    torch.cuda.synchronize()
    flops = 2.0 * n ** 3
    clocks = ClockSampler(0)
    clocks.start()
    best = float("inf")
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mm()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1000.0)
    burst_clocks = clocks.stop()
    clocks = ClockSampler(0)
    clocks.start()
    calls = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for _ in range(20):
            mm()
        calls += 20
        torch.cuda.synchronize()
    e1.record()
    e1.synchronize()
    sus_clocks = clocks.stop()
    sustained = flops * calls / (e0.elapsed_time(e1) / 1000.0)
    return {"fp8_tflops": flops / best / 1e12, "fp8_tflops_sustained": sustained / 1e12,
            "n": n, "calls_sustained": calls, "burst_clocks": burst_clocks,
            "sustained_clocks": sus_clocks,
            "how": f"torch._scaled_mm e4m3 x e4m3 -> bf16 at {n}^3 (2 n^3 flops), unit "
                   f"scales; best of 10 (burst) and back to back for {seconds:.0f} s "
                   "(sustained), CUDA events",
            "torch": torch.__version__, "gpu": torch.cuda.get_device_name(0)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2203_08361_gb300 as hsb
    import synth

    world, rank, local = _dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    w = WORKLOAD
    N, R, S = w["N"], w["R"], w["sb_steps"]
    J = synth.sk_pm1(N, w["J_seed"])
    p = hsb.params(w["form"], w["prec"], a0=w["a0"], c1=w["c1"], dt=w["dt"], gamma=w["gamma"],
                   init_half_width=w["init_half_width"], eval_every=w["eval_every"])
    seed = rank_seed(rank)  # independent replicas on every rank
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    spins = torch.empty((R, N), dtype=torch.int8, device="cuda")
    energy = torch.empty(R, dtype=torch.float64, device="cuda")

    solver = hsb.Solver(J)
    solver.set_stream(stream.cuda_stream)

    def one_run():
        solver.run_device(p, R, S, seed, spins.data_ptr(), energy.data_ptr())

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            one_run()
        solver.synchronize()
        launches_per_run = solver.run_stats()

        # ---- device-resident timed region: K runs, L2 flushed between runs
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(torch.cuda.current_device())
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
            one_run()
            ends[i].record(stream)
        solver.synchronize()
        torch.cuda.synchronize()
        clock_rec = clocks.stop()
        if world > 1:
            dist.barrier()
        elapsed_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))

        # ---- step-loop kernel timing: the S updates of one run without the
        # evaluations, queued as in a run (one persistent launch), CUDA events
        # on the launching stream
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        reps_k = 3
        solver.advance_device(p, R, S, 0, S)  # warm
        solver.synchronize()
        launches_adv = solver.run_stats()
        k0.record(stream)
        for _ in range(reps_k):
            solver.advance_device(p, R, S, 0, S)
        k1.record(stream)
        solver.synchronize()
        loop_ms = k0.elapsed_time(k1) / reps_k

    # ---- the plain FP32 GPU form on the same workload (CUDA cores, fused
    # multiply-add force): its trajectories are identical to the FP8 path's,
    # so the speedup compares runs of equal final-energy accuracy
    def fp32_comparison():
        p32 = hsb.params(w["form"], "fp32", a0=w["a0"], c1=w["c1"], dt=w["dt"],
                         gamma=w["gamma"], init_half_width=w["init_half_width"],
                         eval_every=w["eval_every"])
        spins32 = torch.empty_like(spins)
        energy32 = torch.empty_like(energy)
        with torch.cuda.stream(stream):
            solver.run_device(p32, R, S, seed, spins32.data_ptr(), energy32.data_ptr())
            solver.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            fp32_runs = 2
            f0.record(stream)
            for _ in range(fp32_runs):
                solver.run_device(p32, R, S, seed, spins32.data_ptr(), energy32.data_ptr())
            f1.record(stream)
            solver.synchronize()
            ms = f0.elapsed_time(f1) / fp32_runs
            one_run()
            solver.synchronize()
        same = bool(torch.equal(spins, spins32) and torch.equal(energy, energy32))
        return ms, same

    fp32_ms, identical = (None, None) if args.no_fp32_baseline else fp32_comparison()

    t_max = max_over_ranks(elapsed_ms, world, "cuda")
    value = whole_job_rate(world, N * R * S * args.steps, t_max / 1000.0)

    # ---- end to end through the C ABI with host buffers (rank-local)
    pin_J = torch.from_numpy(J).pin_memory()
    out_s = torch.empty((R, N), dtype=torch.int8).pin_memory()
    out_e = torch.empty(R, dtype=torch.float64).pin_memory()
    import ctypes as C
    lib = hsb.load()

    def e2e_step():
        st = lib.hsb_set_couplings(C.c_void_p(solver.h), C.c_void_p(pin_J.data_ptr()))
        if st != 0:
            raise hsb.HsbError(st, lib.hsb_last_error().decode())
        st = lib.hsb_run(C.c_void_p(solver.h), C.byref(p), R, S, C.c_uint64(seed),
                         C.c_void_p(out_s.data_ptr()), C.c_void_p(out_e.data_ptr()))
        if st != 0:
            raise hsb.HsbError(st, lib.hsb_last_error().decode())

    e2e_step()
    e2e_iters = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_iters
    e2e_value = whole_job_rate(world, N * R * S, max_over_ranks(e2e_s, world, "cuda"))
    solver.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # algorithmic work of the loop: 2 N^2 R flops per step (unpadded N)
    flops_loop = 2.0 * N * N * R * S
    launch_ms = loop_ms / max(launches_adv, 1)
    flops_per_launch = flops_loop / max(launches_adv, 1)
    achieved = flops_loop / (loop_ms / 1000.0) / 1e12
    mp, src = _peaks()
    peak, peak_how = fp8_denominator(mp, src)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": _traffic_for_current_kernel(),
                "kernel": ("tc_fp8_persistent_kernel" if launches_adv == 1
                           else "tc_step_kernel<0> (FP8, one launch per step)"),
                "launches_per_loop": launches_adv, "launch_ms": launch_ms,
                "peak_source": "FP8 dense, burst (the loop kernel runs alone at full clock): "
                               + peak_how,
                "flops_per_launch": flops_per_launch}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp8", "data": "synthetic",
            "config": _config({"l2": "256 MiB buffer written between timed runs (outside the "
                                     "per-run CUDA-event intervals)",
                               "parallelism": f"replicas only: {world} x {R} independent "
                                              "replicas"}),
            "roofline": roofline, "clocks": clock_rec,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(N * N * 4),
                    "d2h_bytes_per_step": int(R * N + R * 8)},
            "gpu_launches": int(launches_per_run * args.steps),
            "fp32_gpu_baseline": None if fp32_ms is None else {
                "value": N * R * S / (fp32_ms / 1000.0), "unit": UNIT, "ms_per_run": fp32_ms,
                "speedup_fp8": (t_max / args.steps) and fp32_ms / (t_max / args.steps),
                "identical_results": identical,
                "kernel": "simt_step_kernel (plain FP32, CUDA cores)"}}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------- the other configurations ---
# The same measurement for the other workloads of the library's configuration
# list (not the headline line): the Gaussian-coupling BF16x3 run, the batch of
# uneven instances, and the large streamed instance.  `--workload NAME`.

OTHER = {
    "gauss2000": dict(name="HbSB Gaussian SK N=2000 R=1024 5000 steps BF16x3", kind="single",
                      N=2000, J="gauss", J_seed=2, R=1024, sb_steps=5000, form="ballistic",
                      prec="bf16x3", c1=0.9, dt=1.1, gamma=0.5, eval_every=100, trace_every=0,
                      peak="bf16", dtype="bf16x3"),
    "sk16384": dict(name="HdSB SK +/-1 N=16384 R=4096 10000 steps FP8 with per-step trace",
                    kind="single", N=16384, J="pm1", J_seed=3, R=4096, sb_steps=10000,
                    form="discrete", prec="fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=100,
                    trace_every=1, peak="fp8", dtype="fp8"),
    "sk2000_fp4": dict(name="HdSB SK +/-1 N=2000 R=1024 2000 steps FP4 e2m1 (persistent)",
                       kind="single", N=2000, J="pm1", J_seed=1, R=1024, sb_steps=2000,
                       form="discrete", prec="fp4", c1=0.7, dt=1.1, gamma=0.06, eval_every=100,
                       trace_every=0, peak="fp4", dtype="fp4"),
    "sk16384_fp4": dict(name="HdSB SK +/-1 N=16384 R=4096 10000 steps FP4 e2m1 with per-step "
                             "trace", kind="single", N=16384, J="pm1", J_seed=3, R=4096,
                        sb_steps=10000, form="discrete", prec="fp4", c1=0.7, dt=1.1, gamma=0.06,
                        eval_every=100, trace_every=1, peak="fp4", dtype="fp4"),
    "trace2000": dict(name="HdSB SK +/-1 N=2000 R=1024 2000 steps FP8 with per-step trace "
                           "(min / mean E, mean T_inst)", kind="single", N=2000, J="pm1",
                      J_seed=1, R=1024, sb_steps=2000, form="discrete", prec="fp8", c1=0.7,
                      dt=1.1, gamma=0.06, eval_every=100, trace_every=1, peak="fp8",
                      dtype="fp8"),
    "nh2000": dict(name="Nose-Hoover dSB SK +/-1 N=2000 R=1024 2000 steps FP8 "
                        "(T=0.3, M=40000, xi0=-0.05)", kind="single", N=2000, J="pm1", J_seed=1,
                   R=1024, sb_steps=2000, form="discrete", prec="fp8", c1=0.7, dt=1.1,
                   gamma=0.0, eval_every=100, trace_every=0, peak="fp8", dtype="fp8",
                   nh=dict(thermostat="nose_hoover", nh_T=0.3, nh_M=40000.0, nh_xi0=-0.05)),
    "batch256": dict(name="HdSB 256 SK +/-1 instances, N uniform in [100, 2000], R=64, 2000 "
                          "steps, FP8, one batched launch", kind="batch", count=256, sizes_seed=4,
                     R=64, sb_steps=2000, form="discrete", prec="fp8", c1=0.7, dt=1.1,
                     gamma=0.06, eval_every=100, trace_every=0, peak="fp8", dtype="fp8"),
    "batch256_fp4": dict(name="HdSB 256 SK +/-1 instances, N uniform in [100, 2000], R=64, "
                              "2000 steps, FP4 e2m1, one batched launch", kind="batch",
                         count=256, sizes_seed=4, R=64, sb_steps=2000, form="discrete",
                         prec="fp4", c1=0.7, dt=1.1, gamma=0.06, eval_every=100, trace_every=0,
                         peak="fp4", dtype="fp4"),
}


def _other_couplings(w):
    import synth
    if w["kind"] == "batch":
        sizes = [int(v) for v in synth.batch_sizes(w["count"], w["sizes_seed"])]
        return [synth.sk_pm1(n, 500 + b) for b, n in enumerate(sizes)]
    gen = synth.sk_gauss if w["J"] == "gauss" else synth.sk_pm1
    return [gen(w["N"], w["J_seed"])]


def _other_cpu_baseline(w, Js, target_s=10.0):
    """The binary32 oracle on a bounded sample: the first instance, one
    replica per thread, steps calibrated to about target_s seconds."""
    import oracle
    cores = os.cpu_count() or 1
    J = Js[0]
    nh = w.get("nh")
    op = oracle.make_params(0 if w["form"] == "ballistic" else 1,
                            oracle.c0_from_c1(J, w["c1"]), w["dt"], w["gamma"],
                            eval_every=w["eval_every"], nose_hoover=nh is not None,
                            **({k: v for k, v in nh.items() if k != "thermostat"} if nh else {}))
    t0 = time.perf_counter()
    oracle.run(J, op, 4, 1, range(cores), "f32", nthreads=cores)
    rate = J.shape[0] * cores * 4 / (time.perf_counter() - t0)
    steps = int(max(4, min(w["sb_steps"], target_s * rate / (J.shape[0] * cores))))
    t0 = time.perf_counter()
    oracle.run(J, op, steps, 1, range(cores), "f32", nthreads=cores)
    t = time.perf_counter() - t0
    return {"value": J.shape[0] * cores * steps / t, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} replicas x {steps} steps of instance 0 (N={J.shape[0]}), "
                      f"binary32 oracle, {cores} threads, {t:.1f} s"}


def run_other(args, w):
    import torch
    import paper_2203_08361_gb300 as hsb

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    world, rank, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    R, S = w["R"], w["sb_steps"]
    Js = _other_couplings(w)
    p = hsb.params(w["form"], w["prec"], c1=w["c1"], dt=w["dt"], gamma=w["gamma"],
                   eval_every=w["eval_every"], trace_every=w["trace_every"],
                   schedule=args.schedule, **w.get("nh", {}))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    units = sum(J.shape[0] for J in Js) * R * S            # replica-spin-steps per run
    flops = sum(2.0 * J.shape[0] ** 2 for J in Js) * R * S  # algorithmic
    seed = rank_seed(rank)
    clocks = ClockSampler(torch.cuda.current_device())
    if w["kind"] == "batch":
        solvers = [hsb.Solver(J) for J in Js]
        hs = [s.h for s in solvers]
        for _ in range(max(args.warmup, 3)):
            hsb.run_batch(hs, p, R, S, seed)  # the first call also tunes the launch
        times = []
        if world > 1:
            dist.barrier()
        clocks.start()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hsb.run_batch(hs, p, R, S, seed)  # host outputs: the whole call
            times.append(time.perf_counter() - t0)
        clock_rec = clocks.stop()
        t_run = sum(times) / len(times)
        e2e_t, launches = t_run, 1
        for s in solvers:
            s.close()
        timing = "host wall clock around hsb_run_batch (one launch plus output copies)"
    else:
        stream = torch.cuda.Stream()
        solver = hsb.Solver(Js[0])
        solver.set_stream(stream.cuda_stream)
        N = Js[0].shape[0]
        spins = torch.empty((R, N), dtype=torch.int8, device="cuda")
        energy = torch.empty(R, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(max(args.warmup, 3)):
                solver.run_device(p, R, S, seed, spins.data_ptr(), energy.data_ptr())
            solver.synchronize()
            launches = solver.run_stats()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            clocks.start()
            for i in range(args.steps):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
                solver.run_device(p, R, S, seed, spins.data_ptr(), energy.data_ptr())
                ev[i][1].record(stream)
            solver.synchronize()
            torch.cuda.synchronize()
            clock_rec = clocks.stop()
        t_run = sum(a.elapsed_time(b) for a, b in ev) / args.steps / 1000.0
        pin_J = torch.from_numpy(Js[0]).pin_memory()
        import ctypes as C
        lib = hsb.load()
        out_s = torch.empty((R, N), dtype=torch.int8).pin_memory()
        out_e = torch.empty(R, dtype=torch.float64).pin_memory()
        t0 = time.perf_counter()
        st = lib.hsb_set_couplings(C.c_void_p(solver.h), C.c_void_p(pin_J.data_ptr()))
        if st == 0:
            st = lib.hsb_run(C.c_void_p(solver.h), C.byref(p), R, S, C.c_uint64(seed),
                             C.c_void_p(out_s.data_ptr()), C.c_void_p(out_e.data_ptr()))
        if st != 0:
            raise hsb.HsbError(st, lib.hsb_last_error().decode())
        e2e_t = time.perf_counter() - t0
        solver.close()
        timing = "CUDA events on the solver's stream around each whole run"
    if world > 1:
        dist.barrier()
    # the job's time is its slowest rank's; every rank ran `units` of its own
    t_run = max_over_ranks(t_run, world, "cuda")
    e2e_t = max_over_ranks(e2e_t, world, "cuda")
    units_job = world * units
    mp, src = _peaks()
    bf16 = float(mp.get("bf16_tflops", mp.get("bf16_tflops_sustained")))
    if w["peak"] == "fp8":
        peak, peak_how = fp8_denominator(mp, src)
        peak_how = "FP8 dense, burst: " + peak_how
    elif w["peak"] == "fp4":
        # no FP4 library GEMM is timed: the measured bf16 burst times the
        # nominal dense FP4 / bf16 ratio (13.5 / 2.25 PFLOP/s)
        peak = 6.0 * bf16
        peak_how = f"FP4 dense: 6 x bf16 burst of {src} peaks (nominal 13.5 / 2.25 ratio)"
    else:
        peak, peak_how = bf16, f"bf16 burst of {src} peaks"
    achieved = world * flops / t_run / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": peak_how,
                "scope": "whole run (force, update, evaluations, final energies); "
                         "algorithmic 2 N^2 R per step"}
    if w["kind"] == "batch":
        # The batch streams every instance's couplings each step (their sum
        # exceeds L2) and keeps x, y in global memory: per step and instance
        # N^2 bytes of FP8 J (N^2 / 2 packed e2m1), 16 N R bytes of x, y read
        # and written, 2 N R bytes of the sign operand written and read back
        # (N R in e2m1).  That traffic, not the tensor rate, bounds it.
        jb, sb = (0.5, 1) if w["prec"] == "fp4" else (1.0, 2)
        nbytes = world * sum(jb * J.shape[0] ** 2 + (16 + sb) * J.shape[0] * R for J in Js) * S
        hbm = float(mp.get("hbm_gbs", 6800.0))
        gbs = nbytes / t_run / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                    "frac": gbs / hbm, "traffic": None,
                    "peak_source": f"hbm_gbs of {src} peaks",
                    "scope": "whole batched launch; algorithmic bytes per step and instance "
                             + ("N^2/2 (J, e2m1) + 17 N R" if w["prec"] == "fp4" else
                                "N^2 (J, FP8) + 18 N R")
                             + " (x, y read and written, sign operand)",
                    "tensor_frac": achieved / peak}
    if w["prec"] == "bf16x3":
        roofline["executed_tflops"] = 3.0 * achieved
    line = {"metric": f"replica-spin-steps/s ({w['name']})", "value": units_job / t_run,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": 1000.0 * t_run, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic",
            "config": {"workload": w["name"], "R": R, "sb_steps": S,
                       "l2": "256 MiB buffer written between timed runs", "timing": timing},
            "roofline": roofline, "clocks": clock_rec,
            "e2e": {"value": units_job / e2e_t, "unit": UNIT,
                    "h2d_bytes_per_step": 0 if w["kind"] == "batch" else int(Js[0].size * 4),
                    "d2h_bytes_per_step": int(sum(J.shape[0] for J in Js) * R + 8 * R * len(Js))},
            "gpu_launches": int(launches * args.steps)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _other_cpu_baseline(w, Js)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hsb", "reference"], default="hsb")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-baseline", action="store_true",
                    help="skip the plain FP32 GPU comparison (e.g. for launch-list captures)")
    ap.add_argument("--workload", choices=["sk2000"] + sorted(OTHER), default="sk2000",
                    help="sk2000 (default): the headline line; the others measure the "
                         "remaining configurations the same way")
    ap.add_argument("--schedule", choices=["auto", "persistent", "per_step"], default="auto",
                    help="FP8 step loop of the --workload runs (profiling of the "
                         "one-launch-per-step path)")
    ap.add_argument("--sb-steps", type=int, default=None,
                    help="override the SB steps per run (profiling of small cases only; "
                         "the headline workload is 2000)")
    ap.add_argument("--fp8-peak", action="store_true",
                    help="measure the dense FP8 tensor rate of this GPU (torch._scaled_mm "
                         "at 8192^3) and print it as one JSON line")
    args = ap.parse_args()
    if args.fp8_peak:
        print(json.dumps(fp8_dense_peak()), flush=True)
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.sb_steps:
        WORKLOAD["sb_steps"] = int(args.sb_steps)
        WORKLOAD["name"] = WORKLOAD["name"].replace("2000 steps", f"{args.sb_steps} steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "sk2000":
        w = dict(OTHER[args.workload])
        if args.sb_steps:
            w["sb_steps"] = int(args.sb_steps)
        if args.schedule != "auto":
            w["name"] += f", {args.schedule.replace('_', '-')} schedule"
        return run_other(args, w)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
