"""Benchmark of the parallel multicanonical hot path on GB300.

One step = the whole path on the periodic 64x64 Ising workload with p = 1024 chains:
infinite-temperature start, 40 weight iterations of 1000 sweeps per chain (sweeps,
histogram merge, recursion + boundary correction, thresholds), a production run of
10^4 sweeps per chain recording (E, M), and FP64 reweighting to 512 betas in
[0.3, 0.6].  Metric: MUCA spin-flip attempts per nanosecond.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the plain restatement of the method) on the
host cores, each step a bounded sample of the same workload.  Under torchrun with
N > 1 each rank runs an independent replica (its own seed): weak scaling, no
collective on the data path.

The JSON line carries, besides the contract keys: `roofline` of the dominant kernel
(the weight-iteration sweeps) with the p-sweep of the same kernel, `cpu_baseline`,
`reweight` (the bench workload's reweighting rates and errors), `other_workloads`
(8-Potts 32x32 and the large lattices), `batched`, `statistical_study`,
`interface_tension`, and last a short `summary` of the headline figures.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

import workloads

ROOT = os.path.dirname(os.path.abspath(__file__))
WORKLOAD = "ising_L64_p1024"
METRIC = "MUCA spin-flip attempts/ns on 1 GB300, plain vs batched; reweighted betas/s at 1e-6"
L2_BYTES = 129 * 1024 * 1024

REASON_BITS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
    0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting",
}

# Counters of the sweep kernels measured with ncu (summaries in profiles/), each with
# the hash of the kernel sources it was measured on; a counter whose hash differs from
# the current sources is reported as stale (and the fractions built on it as null).
SWEEP_SOURCES = ["paper_1212_3975_gb300/csrc/ws_bodies.cuh", "paper_1212_3975_gb300/csrc/sweep_ws.cu",
                 "paper_1212_3975_gb300/csrc/sweep_kernels.cu"]
COUNTERS = {
    # Ising 64x64, p = 1024: 147 blocks of 7 chains, one per SM (the idle lanes of each
    # warp issue too, so these counts are per attempt of a real chain):
    # profiles/ising_ws_sweep_L64_p1024.md
    "ising_L64": {"source": "8c638c33e6db10d8", "inst_per_attempt": 8.508,
                  "shared_wavefronts_per_attempt": 1.013, "traffic_bytes_per_launch": 2565120,
                  "chains_per_block": 7},
    # Ising 64x64, compact staging, two blocks per SM (p = 9728):
    # profiles/ising_ws_compact_L64_p9728.md
    "ising_L64_compact": {"source": "8c638c33e6db10d8", "inst_per_attempt": 1.904,
                          "shared_wavefronts_per_attempt": 0.365, "traffic_bytes_per_launch": 5169920},
    # Ising 64x64, compact staging with the 16-bit table, three blocks per SM
    # (p = 14592): profiles/ising_ws_t16_L64_p14592.md
    "ising_L64_t16": {"source": "8c638c33e6db10d8", "inst_per_attempt": 1.989,
                      "shared_wavefronts_per_attempt": 0.356, "traffic_bytes_per_launch": 7665664},
    # 8-Potts 32x32 (p = 4096: 152 blocks of 27 chains): profiles/potts_ws_sweep_L32_p4096.md
    "potts_L32": {"source": "8c638c33e6db10d8", "inst_per_attempt": 3.158, "shared_wavefronts_per_attempt": 0.582,
                  "traffic_bytes_per_launch": 5122048},
}
# cycles per site of the Ising stream decider's loop run alone on one warp
# (tests/gpu_decider_loop.cu, profiles/ising_decider_loop_replica.md)
DECIDER_CYCLES_PER_ATTEMPT_ALONE = 36.6
# the same for the 8-Potts slot decider (tests/gpu_potts_decider_loop.cu,
# profiles/potts_decider_loop_replica.md)
POTTS_DECIDER_CYCLES_PER_ATTEMPT_ALONE = 43.4
# MUFU ex2 results per clock per SM (the special-function units: 4 per sub-partition
# per clock); the FP32 reweighting evaluates one ex2 per contributing (beta, bin)
MUFU_EX2_PER_CLK_PER_SM = 16


def sweep_source_sha16():
    """Hash of the sweep kernels' code: comments and whitespace are left out, so that
    only a change of the code itself makes the measured counters stale."""
    import re
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def chains_per_block(p, n_sm):
    """Chains per block of a warp-specialised sweep launch with the lattices staged in
    shared memory: 32, or, while groups of 32 leave SMs idle, ceil(p / SMs)."""
    return 32 if (p + 31) // 32 >= n_sm else (p + n_sm - 1) // n_sm


def sweep_blocks(p, n_sm):
    cpg = chains_per_block(p, n_sm)
    return (p + cpg - 1) // cpg


def counters(name):
    """The counters of one kernel configuration and whether they match the sources."""
    c = dict(COUNTERS[name])
    c["matches_source"] = c["source"] == sweep_source_sha16()
    return c


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_attempts(w):
    V = w["L"] * w["L"]
    return w["p"] * V * (w["iterations"] * w["sweeps"] + w["production"])


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the time)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def whole_job_rate(attempts_per_rank, world, seconds):
    """Attempts per nanosecond of the whole job: every rank ran its own replica."""
    return attempts_per_rank * world / (seconds * 1e9)


def rnd(x, n=4):
    """Round for the JSON line (None and non-finite values pass as None)."""
    if x is None:
        return None
    x = float(x)
    if not math.isfinite(x):
        return None
    return float("%.*g" % (n, x))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: MUCA_CLOCKS_CSV if set (kept), else a temporary file
        self.path = os.environ.get("MUCA_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "muca_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        with open(self.path) as fh:
            lines = fh.readlines()
        if not os.environ.get("MUCA_CLOCKS_CSV"):
            os.remove(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[3], 16)
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cuda_timer(torch, stream):
    """Device time (s) of fn() on `stream` by CUDA events, synchronised on both sides."""
    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3
    return timed


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build as b

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    b.build()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    w = workloads.WORKLOADS[WORKLOAD]
    stream = torch.cuda.Stream()
    seed0 = w["seed"] + (rank << 20)
    g = m.Muca(w["model"], w["L"], w["q"], w["p"], seed0, stream=stream.cuda_stream)
    betas_h = workloads.beta_grid(w["betas"])
    n_beta = len(betas_h)
    betas_d = torch.tensor(betas_h, dtype=torch.float64, device="cuda")
    out_d = torch.empty((4, n_beta), dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    sweep_events = []

    def step(seed, timed):
        """One full pass of the hot path, inputs and outputs resident on the device."""
        g.reset(seed)
        for _ in range(w["iterations"]):
            if timed:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            m.check(m.lib().muca_iterate(g.handle, w["sweeps"], None))
            if timed:
                e1.record(stream)
                sweep_events.append((e0, e1))
            m.check(m.lib().muca_update_weights(g.handle, None))
        m.check(m.lib().muca_produce(g.handle, w["production"], None, None))
        g.reweight(betas_d, m.MUCA_FP64, out=out_d)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(seed0 + 1000 + i, False)
        barrier()
        clocks = ClockSampler(local)
        clocks.start()
        launches0 = m.kernel_launches()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        barrier()
        t0.record(stream)
        for i in range(args.steps):
            flush.zero_()                      # evict the small working set from L2
            step(seed0 + i, True)
        t1.record(stream)
        barrier()
        launches = m.kernel_launches() - launches0
        clk = clocks.stop()
        elapsed_ms = t0.elapsed_time(t1)
        sweep_ms = [a.elapsed_time(z) for a, z in sweep_events]

    # end to end through the C ABI with pinned host buffers: the betas go in, every
    # iteration's histogram, all (E, M) records and the observables come out; the same
    # steps and the same L2 flush as the device-timed value
    E_h = torch.empty((w["production"], w["p"]), dtype=torch.int32, pin_memory=True)
    M_h = torch.empty((w["production"], w["p"]), dtype=torch.int32, pin_memory=True)
    H_h = torch.empty(g.n_bins, dtype=torch.int64, pin_memory=True)
    betas_pin = torch.tensor(betas_h, dtype=torch.float64).pin_memory()
    obs_h = torch.empty((4, n_beta), dtype=torch.float64, pin_memory=True)

    def step_host(seed):
        g.reset(seed)
        for _ in range(w["iterations"]):
            m.check(m.lib().muca_iterate(g.handle, w["sweeps"], m._ptr(H_h)))
            m.check(m.lib().muca_update_weights(g.handle, None))
        m.check(m.lib().muca_produce(g.handle, w["production"], m._ptr(E_h), m._ptr(M_h)))
        m.check(m.lib().muca_reweight(g.handle, m._ptr(betas_pin), n_beta, m.MUCA_FP64,
                                      m._ptr(obs_h[0]), m._ptr(obs_h[1]), m._ptr(obs_h[2]),
                                      m._ptr(obs_h[3])))

    with torch.cuda.stream(stream):
        step_host(seed0 + 5000)
        barrier()
        h0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            step_host(seed0 + 6000 + i)
        barrier()
        e2e_s = time.perf_counter() - h0

    total_ms, e2e_s = max_over_ranks([elapsed_ms, e2e_s], world, "cuda")
    attempts = workload_attempts(w)
    value = whole_job_rate(attempts * args.steps, world, total_ms * 1e-3)
    e2e_value = whole_job_rate(attempts * args.steps, world, e2e_s)

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    roofline = sweep_roofline(w, float(np.mean(sweep_ms)), n_sm, sm_max)
    result = {
        "metric": METRIC, "value": value, "unit": "attempts/ns", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "model": "ising", "L": w["L"], "p": w["p"],
                   "iterations": w["iterations"], "sweeps": w["sweeps"],
                   "production": w["production"], "n_beta": n_beta, "reweight": "fp64",
                   "weights": "f64", "attempts_per_step": attempts,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas%d" % world},
        "e2e": {"value": e2e_value, "unit": "attempts/ns",
                "h2d_bytes_per_step": int(n_beta * 8),
                "d2h_bytes_per_step": int(w["iterations"] * g.n_bins * 8
                                          + 2 * w["production"] * w["p"] * 4
                                          + 4 * n_beta * 8),
                "steps": args.steps, "l2": "flushed between steps"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    summary = {"value": rnd(value), "e2e": rnd(e2e_value),
               "sweep_attempts_per_ns": rnd(roofline["attempts_per_ns"]), "sweep_issue_frac": rnd(roofline["frac"], 3)}
    if rank == 0 and not args.no_extras:
        with torch.cuda.stream(stream):
            roofline["p_sweep"] = p_sweep(m, torch, stream, n_sm, sm_max)
    result["roofline"] = roofline
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w)
    if rank == 0 and not args.no_extras:
        with torch.cuda.stream(stream):
            result["reweight"] = reweight_rates(m, torch, stream, n_sm, sm_max, g, betas_h, betas_d)
        g.close()
        result["other_workloads"] = other_workloads(m, torch, stream, n_sm, sm_max)
        result["batched"] = batched_comparison(m, torch)
        result["statistical_study"] = statistical_study()
        result["interface_tension"] = interface_tension()
        summary.update(make_summary(result))
    else:
        g.close()
    result["summary"] = summary
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def sweep_roofline(w, sweep_avg_ms, n_sm, sm_max):
    """Issue roofline of the weight-iteration sweeps of the bench workload."""
    c = counters("ising_L64")
    att_per_launch = w["p"] * w["L"] * w["L"] * w["sweeps"]
    rate = att_per_launch / (sweep_avg_ms * 1e6)           # attempts/ns
    peak = n_sm * 4 * sm_max * 1e6 / 1e9                   # Gwarp-inst/s
    inst = c["inst_per_attempt"]
    achieved = inst * rate                                   # Gwarp-inst/s
    ok = c["matches_source"]
    occupied = min(4 * n_sm, 4 * sweep_blocks(w["p"], n_sm))
    latency = w["p"] * sm_max * 1e6 / DECIDER_CYCLES_PER_ATTEMPT_ALONE / 1e9
    return {
        "bound": "alu", "achieved": achieved if ok else None, "peak": peak, "unit": "Gwarp-inst/s",
        "frac": achieved / peak if ok else None,
        "traffic": c["traffic_bytes_per_launch"] if ok else None,
        "kernel": "ising_ws_kernel (weight-iteration sweeps, warp-specialised)",
        "launch_ms": sweep_avg_ms, "attempts_per_ns": rate,
        "warp_inst_per_attempt": inst, "counters_match_source": ok,
        "peak_note": "%d SMs x 4 schedulers x 1 warp-instruction/clock at %.0f MHz, of measured max clock"
                     % (n_sm, sm_max),
        "occupied_schedulers": occupied,
        "frac_of_occupied_schedulers": achieved / (peak * occupied / (4 * n_sm)) if ok else None,
        # the three bounds on attempts/ns of the sweeps at the measured max clock: issue
        # (every scheduler busy at this instruction count), shared-memory LSU (one
        # wavefront per clock per SM) and chain latency (p chains at the decider loop's
        # cycles per attempt)
        "bounds_attempts_per_ns": {
            "issue": 4 * n_sm * sm_max * 1e6 / inst / 1e9,
            "lsu": n_sm * sm_max * 1e6 / c["shared_wavefronts_per_attempt"] / 1e9,
            "latency": latency,
        },
        "frac_of_latency_bound": rate / latency,
    }


def p_sweep(m, torch, stream, n_sm, sm_max):
    """Ising 64x64 weight-iteration launches at growing p: where the issue roofline
    saturates.  One block of 32 chains per SM up to p = 32 x SMs; beyond, the compact
    staging runs two blocks per SM, and three (the table of 16-bit threshold halves)
    where that takes fewer waves: at 96 and 192 x SMs."""
    timed = cuda_timer(torch, stream)
    peak = n_sm * 4 * sm_max * 1e6 / 1e9
    out = []
    for p in (1024, 2048, 32 * n_sm, 64 * n_sm, 96 * n_sm, 128 * n_sm, 192 * n_sm):
        sweeps = 100 if p <= 96 * n_sm else 50
        g = m.Muca(m.MUCA_ISING, 64, 2, p, 1, stream=stream.cuda_stream)
        g.iterate(2)
        g.update_weights()
        g.iterate(10)
        g.update_weights()
        plan = g.plan()
        t = min(timed(lambda: m.check(m.lib().muca_iterate(g.handle, sweeps, None))) for _ in range(2))
        g.close()
        rate = p * 4096 * sweeps / t / 1e9
        c = counters("ising_L64_t16" if plan & m.MUCA_PLAN_TABLE16 else
                     "ising_L64_compact" if plan & m.MUCA_PLAN_COMPACT else "ising_L64")
        ok = c["matches_source"]
        if "chains_per_block" in c:
            # a warp issues for all 32 lanes: per attempt of a chain the counts scale
            # with 1 / (chains per block) from the captured launch's
            scale = c["chains_per_block"] / chains_per_block(p, n_sm)
            c["inst_per_attempt"] *= scale
            c["shared_wavefronts_per_attempt"] *= scale
        out.append({"p": p, "attempts_per_ns": rnd(rate), "compact": bool(plan & m.MUCA_PLAN_COMPACT),
                    "blocks_per_sm": 3 if plan & m.MUCA_PLAN_TABLE16 else 2 if plan & m.MUCA_PLAN_COMPACT else 1,
                    "issue_frac": rnd(rate * c["inst_per_attempt"] / peak, 3) if ok else None,
                    "lsu_frac": rnd(rate * c["shared_wavefronts_per_attempt"] / (n_sm * sm_max * 1e-3), 3)
                    if ok else None,
                    "latency_frac": rnd(rate / (p * sm_max * 1e-3 / DECIDER_CYCLES_PER_ATTEMPT_ALONE), 3)})
    return out


def reweight_rates(m, torch, stream, n_sm, sm_max, g, betas_h, betas_d):
    """Reweighting of the bench workload's production sums (the last step's) to its 512
    betas: betas/s of muca_reweight per precision, the error of FP32 and BF16 against
    FP64 per observable, and the roofline of the FP32 form (one MUFU ex2 per (beta,
    bin) whose weight reaches e^-100 of the largest)."""
    timed = cuda_timer(torch, stream)
    n_beta = len(betas_h)
    out = {"workload": WORKLOAD, "n_beta": n_beta, "n_bins": g.n_bins}
    res = {}
    for name, prec in (("fp64", m.MUCA_FP64), ("fp32", m.MUCA_FP32), ("bf16", m.MUCA_BF16)):
        o = torch.empty((4, n_beta), dtype=torch.float64, device="cuda")
        g.reweight(betas_d, prec, out=o)          # warm-up (and scratch)
        reps = 20
        t = timed(lambda: [g.reweight(betas_d, prec, out=o) for _ in range(reps)]) / reps
        out[name + "_betas_per_s"] = rnd(n_beta / t)
        out[name + "_us"] = rnd(t * 1e6)
        res[name] = o.cpu().numpy()
    for name in ("fp32", "bf16"):
        err = np.abs(res[name] - res["fp64"]) / np.maximum(np.abs(res["fp64"]), 1e-300)
        out[name + "_max_rel_err"] = {k: rnd(err[i].max(), 3) for i, k in enumerate(("e", "C", "absm", "chi"))}
        out[name + "_within_1e-6"] = bool(err.max() <= 1e-6)
    n, _, _ = g.get_samples()
    exps = contributing_terms(g.model, g.L, n, g.get_lnw(), betas_h)  # weights unchanged since production
    t32 = out["fp32_us"] * 1e-6
    peak = n_sm * MUFU_EX2_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
    out["roofline_fp32"] = {"bound": "alu", "unit": "Tex2/s", "exps_per_call": exps,
                            "achieved": rnd(exps / t32 / 1e12), "peak": rnd(peak),
                            "frac": rnd(exps / t32 / 1e12 / peak, 3),
                            "peak_note": "%d SMs x %d MUFU ex2/clock at %.0f MHz"
                                         % (n_sm, MUFU_EX2_PER_CLK_PER_SM, sm_max)}
    return out


def contributing_terms(model, L, n, lnw, betas):
    """(beta, bin) pairs whose weight reaches e^-100 of the largest at that beta."""
    V = L * L
    b = np.nonzero(n)[0]
    E = 4.0 * b - 2.0 * V if model == 0 else b - 2.0 * V
    lo = np.log(n[b].astype(np.float64)) - lnw[b]
    total = 0
    for beta in betas:
        a = lo - beta * E
        total += int(np.count_nonzero(a >= a.max() - 100.0))
    return total


def other_workloads(m, torch, stream, n_sm, sm_max):
    """Rates of the other configurations on a bounded part of their schedules (each line
    says which): 8-Potts 32x32 (one 500-sweep weight iteration from ln W = 0, then
    2000 production sweeps at the fixed canonical weights of beta_0 after 200
    thermalisation sweeps, reweighted to its 1024 betas) and the large lattices at
    fixed ln W = -beta_0 E (100 production sweeps, 4096 betas).  Device time by CUDA
    events on the context's stream; FP32 and BF16 reweighting errors against FP64."""
    timed = cuda_timer(torch, stream)
    peak = n_sm * 4 * sm_max * 1e6 / 1e9
    out = {}
    cases = (("potts8_L32_p4096", 500, 2000), ("ising_L256_p8192", 0, 100), ("potts8_L128_p4096", 0, 100))
    for name, it_sweeps, prod in cases:
        w = workloads.WORKLOADS[name]
        g = m.Muca(w["model"], w["L"], w["q"], w["p"], w["seed"], stream=stream.cuda_stream)
        V = w["L"] * w["L"]
        rec = {"sample": "%s%d production sweeps, %d betas"
               % ("one %d-sweep iteration, " % it_sweeps if it_sweeps else "", prod, w["betas"][2])}
        with torch.cuda.stream(stream):
            if it_sweeps:
                g.iterate(2)
                g.update_weights()
                t = timed(lambda: m.check(m.lib().muca_iterate(g.handle, it_sweeps, None)))
                rate = w["p"] * V * it_sweeps / t / 1e9
                rec["iterate_attempts_per_ns"] = rnd(rate)
                c = counters("potts_L32")
                rec["roofline"] = {"bound": "alu", "unit": "Gwarp-inst/s",
                                   "warp_inst_per_attempt": c["inst_per_attempt"],
                                   "frac": rnd(rate * c["inst_per_attempt"] / peak, 3) if c["matches_source"]
                                   else None,
                                   "counters_match_source": c["matches_source"],
                                   "occupied_sms": min(n_sm, sweep_blocks(w["p"], n_sm)),
                                   # p chains at the slot decider's cycles per attempt alone
                                   "latency_bound_attempts_per_ns": rnd(
                                       w["p"] * sm_max * 1e-3 / POTTS_DECIDER_CYCLES_PER_ATTEMPT_ALONE),
                                   "frac_of_latency_bound": rnd(
                                       rate / (w["p"] * sm_max * 1e-3 / POTTS_DECIDER_CYCLES_PER_ATTEMPT_ALONE), 3)}
            beta0 = workloads.ISING_BETA0 if w["model"] == workloads.ISING else workloads.POTTS8_BETA0
            lnw = workloads.canonical_lnw(w["model"], w["L"], w.get("fixed_beta", beta0))
            g.set_lnw(lnw - lnw.max())
            g.thermalize(200 if it_sweeps else 20)
            g.reset_samples()
            t = timed(lambda: m.check(m.lib().muca_produce(g.handle, prod, None, None)))
            rec["produce_attempts_per_ns"] = rnd(w["p"] * V * prod / t / 1e9)
            betas_h = workloads.beta_grid(w["betas"])
            betas_d = torch.tensor(betas_h, dtype=torch.float64, device="cuda")
            n_beta = len(betas_h)
            res = {}
            for prec_name, prec in (("fp64", m.MUCA_FP64), ("fp32", m.MUCA_FP32), ("bf16", m.MUCA_BF16)):
                o = torch.empty((4, n_beta), dtype=torch.float64, device="cuda")
                g.reweight(betas_d, prec, out=o)
                reps = 5
                t = timed(lambda: [g.reweight(betas_d, prec, out=o) for _ in range(reps)]) / reps
                rec[prec_name + "_betas_per_s"] = rnd(n_beta / t)
                res[prec_name] = o.cpu().numpy()
            for prec_name in ("fp32", "bf16"):
                err = np.abs(res[prec_name] - res["fp64"]) / np.maximum(np.abs(res["fp64"]), 1e-300)
                rec[prec_name + "_max_rel_err"] = rnd(err.max(), 3)
                rec[prec_name + "_within_1e-6"] = bool(err.max() <= 1e-6)
        g.close()
        out[name] = rec
    return out


def statistical_study():
    """The performance study of Sec. 4, bounded: 8x8 Ising, p = 1..32 chains, 10 seeds,
    M on a geometric grid around Eq. 7's M_opt(8, p), runs capped at 400 iterations.
    M_opt(p) is the minimum of N_iter M p; S*_p comes from the same minima."""
    from paper_1212_3975_gb300 import study
    fin = lambda x: None if not math.isfinite(x) else round(float(x), 3)  # noqa: E731
    ps = [1, 2, 4, 8, 16, 32]
    factors = [0.5, 0.7, 1.0, 1.4, 2.0, 2.8, 4.0]
    t0 = time.perf_counter()
    scan = study.m_scan(study.ISING, 8, ps, factors, 10, 400)
    m_opt, per_chain, S = study.speedup_from_scan(scan)
    m1 = study.fit_m1(ps, [m_opt[p] for p in ps])
    # intermediate thermalisation between iterations (Sec. 4): 8-Potts 8x8, p = 16 chains,
    # M = Eq. 7's M_opt(8, 16), 16 seeds, at most 200 iterations
    therm = {}
    p = 16
    M = int(round(study.eq7_m_opt(study.POTTS, 8, p)))
    for T in (0, M // 4, M):
        runs = study.n_iter_runs(study.POTTS, 8, [p], M, 16, 200, seed0=11, therm_sweeps=T)[p]
        ok = runs[runs > 0]
        therm["T%d" % T] = {
            "converged": "%d/%d" % (len(ok), len(runs)),
            "median_n_iter": fin(float(np.median(ok))) if len(ok) else None,
            "median_sweeps_per_chain": fin(float(np.median(ok * M + (ok - 1) * T))) if len(ok) else None}
    # multimagnetic Ising at beta = (3/2) beta_0 (Sec. 4, Fig. 6): the same scan, with
    # the weights in M; one context per run
    beta_mm = 1.5 * math.log(1.0 + math.sqrt(2.0)) / 2.0
    # (a single chain rarely converges within the cap here, so the speedup is quoted
    # relative to p = 4: S*_p / S*_4 = [N_iter M]_4 / [N_iter M]_p)
    ps_mm = [4, 16, 64]
    scan_mm = study.m_scan(study.ISING, 8, ps_mm, [0.5, 1.0, 2.0, 4.0], 3, 200,
                           M_center=lambda p: 1000.0 / p, muma_beta=beta_mm)
    m_mm, per_chain_mm, _ = study.speedup_from_scan(scan_mm)
    muma = {
        "workload": "multimagnetic 8x8 Ising at beta = (3/2) beta_0, p in {4, 16, 64}, 3 seeds per (p, M), "
                    "M grid x{0.5..4} around 1000/p, <= 200 iterations",
        "M_opt": {str(p): fin(m_mm[p]) for p in ps_mm},
        "sweeps_per_chain_to_convergence": {str(p): fin(per_chain_mm[p]) for p in ps_mm},
        "S_star_relative_to_p4": {str(p): fin(per_chain_mm[4] / per_chain_mm[p])
                                  if math.isfinite(per_chain_mm[p]) and math.isfinite(per_chain_mm[4]) else None
                                  for p in ps_mm},
    }
    return {
        "workload": "8x8 Ising, p in 1..32, 10 seeds per (p, M), M grid x{0.5..4} around Eq. 7, <= 400 iterations",
        "M_opt": {str(p): fin(m_opt[p]) for p in ps},
        "M1_fit": round(m1, 1), "M1_eq7": round(study.eq7_m_opt(study.ISING, 8, 1), 1),
        "sweeps_per_chain_to_convergence": {str(p): fin(per_chain[p]) for p in ps},
        "S_star": {str(p): fin(S[p]) for p in ps},
        "multimagnetic": muma,
        "intermediate_thermalization": {"workload": "8-Potts 8x8, p = 16, M = Eq. 7 M_opt(8, 16) = %d, T sweeps "
                                                    "after every unconverged update, 16 seeds, <= 200 iterations" % M,
                                        **therm},
        "seconds": round(time.perf_counter() - t0, 2),
    }


def interface_tension():
    """sigma_od of the 8-state Potts model (Sec. 5), bounded: L = 8, 12, 16, four
    independent runs of 16 chains each per L iterated to convergence together, 4000
    production sweeps per converged run, equal-height analysis; sigma_inf from
    sigma_od(L) = sigma_inf + c/L (small L: large finite-size corrections)."""
    from paper_1212_3975_gb300 import study
    t0 = time.perf_counter()
    res, (s_inf, c) = study.sigma_od_scan([8, 12, 16])
    fin = lambda x: None if not (isinstance(x, float) and math.isfinite(x)) else round(float(x), 6)  # noqa: E731
    return {
        "workload": "8-Potts L = 8, 12, 16, 4 runs x 16 chains, M = Eq. 7 M_opt(L, 16), <= 300 iterations, "
                    "200 thermalisation + 4000 production sweeps per converged run, beta in [1.25, 1.45]",
        "per_L": {str(L): {k: (fin(v) if isinstance(v, float) else v) for k, v in r.items()} for L, r in res.items()},
        "sigma_inf_fit": fin(s_inf), "fit_c": fin(c),
        "paper_sigma_inf": 0.045,
        "seconds": round(time.perf_counter() - t0, 2),
    }


def batched_comparison(m, torch):
    """Mixed workload (Ising L = 16..128 and 8-Potts L = 16..48, 256 chains each,
    20 x 200 sweeps): one persistent launch per iteration under a CUDA graph,
    autotuned, against one launch sequence per lattice."""
    wb = workloads.BATCHED_MIXED
    jobs, iters, sweeps = wb["jobs"], wb["iterations"], wb["sweeps"]
    att = sum(p * L * L for (_, L, _, p, _) in jobs) * iters * sweeps

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    ctxs = [m.Muca(*j) for j in jobs]

    def per_lattice():
        for c in ctxs:
            for _ in range(iters):
                m.check(m.lib().muca_iterate(c.handle, sweeps, None))
                m.check(m.lib().muca_update_weights(c.handle, None))

    t_seq = timed(per_lattice)
    for c in ctxs:
        c.close()
    b = m.MucaBatch(jobs)
    choice = b.autotune(sweeps)
    b.iterate(1, sweeps, graph=True)        # builds the 1-iteration graph (warm-up)
    t_bat = timed(lambda: b.iterate(iters, sweeps, graph=True))
    b.close()
    return {"workload": "mixed: Ising L=16..128 + 8-Potts L=16..48, 256 chains each, %d x %d sweeps"
                        % (iters, sweeps),
            "per_lattice_attempts_per_ns": rnd(att / t_seq / 1e9),
            "batched_attempts_per_ns": rnd(att / t_bat / 1e9),
            "speedup": rnd(t_seq / t_bat), "per_lattice_s": rnd(t_seq), "batched_s": rnd(t_bat),
            "autotuned": {"grid": choice[0], "staging": choice[1], "launches_per_iteration": choice[2]}}


def make_summary(r):
    """The headline figures of the extras, short enough to stay at the end of the line."""
    s = {}
    ps = r["roofline"].get("p_sweep") or []
    if ps:
        best = max(ps, key=lambda x: x["attempts_per_ns"] or 0)
        s["p_sweep_best"] = {k: best[k] for k in ("p", "attempts_per_ns", "issue_frac")}
    rw = r.get("reweight", {})
    s["reweight_c2_betas_per_s"] = {k: rw.get(k + "_betas_per_s") for k in ("fp64", "fp32", "bf16")}
    s["reweight_c2_within_1e-6"] = {k: rw.get(k + "_within_1e-6") for k in ("fp32", "bf16")}
    s["reweight_c2_fp32_ex2_frac"] = rw.get("roofline_fp32", {}).get("frac")
    ow = r.get("other_workloads", {})
    c3 = ow.get("potts8_L32_p4096", {})
    s["c3_iterate_attempts_per_ns"] = c3.get("iterate_attempts_per_ns")
    s["c3_issue_frac"] = c3.get("roofline", {}).get("frac")
    s["c3_latency_frac"] = c3.get("roofline", {}).get("frac_of_latency_bound")
    s["c3_reweight_betas_per_s"] = {k: c3.get(k + "_betas_per_s") for k in ("fp64", "fp32", "bf16")}
    for name in ("ising_L256_p8192", "potts8_L128_p4096"):
        c5 = ow.get(name, {})
        key = "c5_" + name.split("_")[0]
        s[key + "_produce_attempts_per_ns"] = c5.get("produce_attempts_per_ns")
        s[key + "_fp32_max_rel_err"] = c5.get("fp32_max_rel_err")
    bt = r.get("batched", {})
    s["batched_speedup"] = bt.get("speedup")
    s["batched_attempts_per_ns"] = bt.get("batched_attempts_per_ns")
    cb = r.get("cpu_baseline", {})
    if cb:
        s["cpu_attempts_per_ns"] = {"all_cores": rnd(cb.get("value")), "one_core_iterate": cb["one_core"]["iterate"]}
    return s


def run_probe(args):
    """One small launch of a workload's sweeps, for profiler captures: start, a 2-sweep
    iteration and update (the launch skipped by -s 1), then one iteration of
    --probe-sweeps sweeps (the captured launch); with --probe-phase produce, a 2-sweep
    thermalisation (skipped) and production sweeps at the workload's weights."""
    import torch
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build as b
    b.build()
    w = dict(workloads.WORKLOADS[args.probe])
    if args.probe_p:
        w["p"] = args.probe_p
    g = m.Muca(w["model"], w["L"], w["q"], w["p"], w["seed"])
    if w.get("fixed_beta"):
        lnw = workloads.canonical_lnw(w["model"], w["L"], w["fixed_beta"])
        g.set_lnw(lnw - lnw.max())
    if args.probe_phase == "produce":
        g.thermalize(2)          # at the workload's weights
    else:
        g.iterate(2)
        g.update_weights()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.probe_phase == "produce":
        g.produce(args.probe_sweeps, None, None)
    else:
        g.iterate(args.probe_sweeps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"probe": args.probe, "phase": args.probe_phase, "p": w["p"], "plan": g.plan(),
                      "sweeps": args.probe_sweeps,
                      "attempts_per_ns": w["p"] * w["L"] * w["L"] * args.probe_sweeps / dt / 1e9}))
    g.close()


# ----------------------------------------------------------------------------- CPU oracle
def cpu_phases(w, n_chains, it_sweeps, prod_sweeps, threads):
    """The oracle as it stands on `threads` host cores: one weight iteration of
    `it_sweeps` sweeps of `n_chains` chains, the update, `prod_sweeps` production sweeps,
    and the FP64 reweighting to every beta; seconds of each phase."""
    from oracle import MucaOracle, reweight, sampler
    sampler.set_threads(threads)
    betas = workloads.beta_grid(w["betas"])
    o = MucaOracle(w["model"], w["L"], w["q"], n_chains, w["seed"])
    t0 = time.perf_counter()
    o.iterate(it_sweeps)
    t1 = time.perf_counter()
    o.update_weights()
    t2 = time.perf_counter()
    E, M = o.produce(prod_sweeps)
    t3 = time.perf_counter()
    reweight.reweight_binned(w["model"], w["L"], w["q"], o.lnw, *reweight.bin_series(w["model"], w["L"], E, M),
                             betas)
    t4 = time.perf_counter()
    return {"iterate": t1 - t0, "update": t2 - t1, "produce": t3 - t2, "reweight": t4 - t3,
            "n_beta": len(betas)}


def cpu_baseline(w):
    """The oracle on the host cores, bounded: all 1024 chains on every core, 64 chains on
    one core; attempts/ns of the iteration and production phases separately and FP64
    reweighting betas/s; `value` is the whole all-core sample."""
    from oracle import sampler
    cores = sampler.max_threads()
    V = w["L"] * w["L"]
    it_s, pr_s = 400, 400
    allc = cpu_phases(w, w["p"], it_s, pr_s, cores)
    one = cpu_phases(w, 64, 100, 100, 1)
    sampler.set_threads(cores)
    att_all = w["p"] * V * (it_s + pr_s)
    secs = allc["iterate"] + allc["update"] + allc["produce"] + allc["reweight"]
    return {"value": att_all / (secs * 1e9), "unit": "attempts/ns", "cores": cores, "kind": "oracle",
            "seconds": rnd(secs + one["iterate"] + one["update"] + one["produce"] + one["reweight"]),
            "all_cores": {"iterate": rnd(w["p"] * V * it_s / allc["iterate"] / 1e9),
                          "produce": rnd(w["p"] * V * pr_s / allc["produce"] / 1e9),
                          "reweight_fp64_betas_per_s": rnd(allc["n_beta"] / allc["reweight"])},
            "one_core": {"iterate": rnd(64 * V * 100 / one["iterate"] / 1e9),
                         "produce": rnd(64 * V * 100 / one["produce"] / 1e9),
                         "reweight_fp64_betas_per_s": rnd(one["n_beta"] / one["reweight"])},
            "sample": "%s: all %d chains x (1 iteration of %d sweeps + update + %d production sweeps) + FP64 "
                      "reweighting to %d betas on %d cores; 64 chains x (100 + 100 sweeps) on 1 core"
                      % (WORKLOAD, w["p"], it_s, pr_s, allc["n_beta"], cores)}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import sampler
    w = workloads.WORKLOADS[WORKLOAD]
    cores = sampler.max_threads()
    V = w["L"] * w["L"]
    it_s, pr_s = 100, 20
    secs = []
    for i in range(args.warmup + args.steps):
        ph = cpu_phases(w, w["p"], it_s, pr_s, cores)
        if i >= args.warmup:
            secs.append(ph["iterate"] + ph["update"] + ph["produce"] + ph["reweight"])
    att = w["p"] * V * (it_s + pr_s) * len(secs)
    value = att / (sum(secs) * 1e9)
    sample = ("%s: all %d chains, 1 iteration x %d sweeps + update + %d production sweeps + FP64 reweight "
              "to %d betas per step" % (WORKLOAD, w["p"], it_s, pr_s, len(workloads.beta_grid(w["betas"]))))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/ns",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(secs) * 1e3 / len(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64/int", "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": w["L"], "p": w["p"], "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "attempts/ns", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "attempts/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the reweighting and batched lines")
    ap.add_argument("--probe", default=None, choices=sorted(workloads.WORKLOADS),
                    help="run one small sweep launch of a workload (for profiler captures)")
    ap.add_argument("--probe-sweeps", type=int, default=10)
    ap.add_argument("--probe-p", type=int, default=0, help="number of chains of the probe (default: the workload's)")
    ap.add_argument("--probe-phase", default="iterate", choices=["iterate", "produce"],
                    help="the captured launch: a weight iteration or production sweeps")
    args = ap.parse_args()
    if args.probe:
        run_probe(args)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
