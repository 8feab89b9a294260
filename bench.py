#!/usr/bin/env python3
"""Benchmark of the batched dense simplex (Gurung & Ray, arXiv 1802.08557).

One step = one lp_batch_solve over the whole batch: every LP's tableau is
built on the device from A, b, c and Steps 1-3 run until each LP halts.

Default workload: 1e5 random dense LPs of 50 x 50 (A~U[-1,1], c~U[-1,1],
80% with b~U[1,10], 20% with b~U[-5,10] needing phase I, ~5% infeasible or
unbounded by construction), FP64.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
on the host cores instead (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LPs solved/s on 1 GB300 vs plain FP64 GPU simplex at <=1e-9 rel obj err; % roofline"
DEFAULT_WORKLOAD = "dense50x50_phase1_100k"
# Nominal unit throughputs (used only if the library's own microbenchmarks,
# lpb_measure_peaks, cannot run): FP64 FMA pipe 152 SMs x 2 FMA/clk x 2 flop x
# 2.07 GHz (the GB300's nominal 1.25 TFLOP/s FP64); FP32 FMA pipe 152 x 128 x 2
# x 2.07 GHz; shared memory 152 SMs x 128 bytes/clk x 2.07 GHz.
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.070
FP32_NOMINAL_GFLOPS = 152 * 128 * 2 * 2.070
SMEM_NOMINAL_GBS = 152 * 128 * 2.070
def _measured_peaks():
    """HBM copy bandwidth and BF16 tensor throughput measured on this machine's
    GB300s (MEASURED_PEAKS.json beside this file), else the earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "MEASURED_PEAKS.json"
    except Exception:  # noqa: BLE001
        return 6784.5, 1958.9, "earlier measurement (MEASURED_PEAKS.json absent)"


# HBM bandwidth (STREAM-style copy, read + write bytes) and dense BF16 tensor
# throughput (cuBLAS GEMM, burst) of a GB300
HBM_PEAK_GBS, BF16_PEAK_TFLOPS, PEAKS_SOURCE = _measured_peaks()
# DRAM bytes per LP (read + write) from ncu captures of the kernels as they are
# now, for the roofline's `traffic` (scaled to a launch by the LPs it solves):
# profiles/mixed_warp_kernel__dense50x50_20k__ncu.md (k = 0 group, 15629 LPs:
# 350.7 MB + 12.6 MB) and profiles/hyperbox_tile_kernel__dirs1M_dim28__ncu.md
# (2^20 LPs in R^28: 234.9 MB + 7.6 MB).
MIXED_DRAM_BYTES_PER_LP = (350.654208e6 + 12.641024e6) / 15629
HYPERBOX_DRAM_BYTES_PER_LP_DIM28 = (234.9e6 + 7.6e6) / (1 << 20)
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--num-lps", type=int, default=None, help="override the workload's batch size")
    p.add_argument("--cpu-sample", type=int, default=20000, help="LPs timed for the CPU oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--per-lp-file", default=None,
                   help="write the headline's per-LP errors against the oracle (npz) to this path")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-chunks", type=int, default=0,
                   help="chunks of lp_solve_host in the end-to-end measurement (0: the library's choice)")
    p.add_argument("--no-hyperbox", action="store_true", help="skip the hyperbox LP (Eq. 7) measurement")
    p.add_argument("--no-warm", action="store_true", help="skip the learned warm-start measurement")
    p.add_argument("--no-uneven", action="store_true", help="skip the uneven-batch measurement")
    p.add_argument("--no-support", action="store_true", help="skip the support-function measurement")
    p.add_argument("--no-c1", action="store_true", help="skip the 1000 LPs of 5 x 5 measurement")
    p.add_argument("--oracle-sample", type=int, default=2000,
                   help="LPs of each secondary workload compared with the oracle (uneven: a fifth of it)")
    p.add_argument("--support-dirs", type=int, default=100_000, help="directions of the support-function measurement")
    p.add_argument("--uneven-lps", type=int, default=20_000, help="LPs of the uneven-batch measurement")
    p.add_argument("--warm-train", type=int, default=1_000_000, help="self-solved LPs the network is trained on")
    p.add_argument("--warm-test", type=int, default=100_000, help="test LPs of the warm-start measurement")
    p.add_argument("--hyperbox-dirs", type=int, default=1 << 22, help="directions of the hyperbox measurement")
    p.add_argument("--profile-case", default=None, choices=["gemm_tc_layer1", "fp64_streamed_uneven"],
                   help="run one workload a few times for a profiler and exit (no JSON line): the warm-start "
                        "network's first-layer product on the tcgen05 kernel (1e5 x 320 -> 512, bias + ReLU), or "
                        "the uneven workload's LPs above one CTA on the streamed FP64 kernel")
    p.add_argument("--precision", default="fp32r", choices=["fp32r", "fp64"],
                   help="headline path: FP32 tableau + FP64 certificate (default) or plain FP64")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_batch(name, num, rank):
    """The named workload; rank r of a weak-scaling run solves LPs r*N .. (r+1)*N-1."""
    import inspect
    from paper_1802_08557_gb300 import workloads as W
    fn = W.WORKLOADS[name]
    count = num if num is not None else inspect.signature(fn).parameters["num"].default
    return fn(num=count, start=rank * count)


def algorithmic_fmas(batch, iters):
    """Algorithmic FMA count: every pivot updates the (m+1) x (n+1) condensed
    tableau (lower bound: phase I's wider tableau is not counted)."""
    m = batch.m.astype(np.float64)
    n = batch.n.astype(np.float64)
    return float(np.sum(iters.astype(np.float64) * (m + 1.0) * (n + 1.0)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


def sample_indices(num_lps: int, sample: int) -> np.ndarray:
    """`sample` evenly spaced LP indices of a batch."""
    k = min(sample, num_lps)
    return np.linspace(0, num_lps - 1, k).astype(np.int64)


def cpu_oracle_run(batch, idx, threads: int):
    """The oracle as it stands on LPs idx of the batch, on `threads` host
    threads.  Returns (LPs/s, wall seconds, oracle results)."""
    import oracle
    lps = [batch.lp(int(i)) for i in idx]
    oracle.lib()
    t0 = time.perf_counter()
    res = oracle.solve_batch(lps, threads=threads)
    dt = time.perf_counter() - t0
    return len(idx) / dt, dt, res


def cpu_oracle_rate(batch, sample: int, threads: int):
    """Oracle LPs/s on `sample` evenly spaced LPs (rate, wall time, count)."""
    idx = sample_indices(batch.num_lps, sample)
    rate, dt, _ = cpu_oracle_run(batch, idx, threads)
    return rate, dt, len(idx)


def oracle_rate_note(rate: float, seconds: float, count: int) -> dict:
    """The oracle's own rate on the LPs it was compared on (all host threads)."""
    return {"all_threads": rate, "cores": os.cpu_count() or 1, "unit": "LPs/s",
            "sample": f"{count} evenly spaced LPs, {seconds:.2f} s wall"}


def vs_oracle(status, obj, idx, ores) -> dict:
    """Per-LP agreement of GPU results (status, obj over the whole batch) with
    the oracle's on LPs idx: status mismatches and the distribution of the
    relative objective error |obj - obj*| / max(1, |obj*|) over the LPs the
    oracle finds optimal."""
    st = np.asarray(status)[idx]
    so = np.asarray(ores["status"])
    opt = so == 0
    rel = np.abs(np.asarray(obj)[idx][opt] - np.asarray(ores["obj"])[opt]) / np.maximum(1.0, np.abs(ores["obj"][opt]))
    out = {"lps_compared": int(len(idx)), "status_mismatches": int(np.sum(st != so)),
           "optimal_lps": int(opt.sum())}
    if rel.size:
        out["rel_obj_err"] = {"max": float(rel.max()), "p99": float(np.quantile(rel, 0.99)),
                              "median": float(np.median(rel)), "count_above_1e-9": int(np.sum(rel > 1e-9))}
    return out


def bench_config(workload: str, batch) -> dict:
    """The workload description shared by both arms' JSON lines."""
    in_bytes = (batch.A.size + batch.b.size + batch.c.size) * 8
    return {"workload": workload, "num_lps_per_gpu": int(batch.num_lps),
            "l2": f"inputs larger than L2 ({in_bytes / 1e9:.2f} GB of A,b,c per step vs 0.13 GB L2)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    batch = make_batch(args.workload, args.num_lps, 0)
    threads = os.cpu_count() or 1
    sample = max(100, min(args.cpu_sample, batch.num_lps))
    for _ in range(args.warmup):
        cpu_oracle_rate(batch, max(10, sample // 20), threads)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt, k = cpu_oracle_rate(batch, sample, threads)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "LPs/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(args.workload, batch),
        "cpu_baseline": {"value": value, "unit": "LPs/s", "cores": threads, "kind": "oracle",
                         "sample": f"{sample} of {batch.num_lps} LPs per step, evenly spaced indices"},
        "e2e": {"value": value, "unit": "LPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1802_08557_gb300 import build, lpbatch as lpb
    from paper_1802_08557_gb300 import workloads as W
    build.build()
    lpb.load()

    # roofline denominators of the FP64 / FP32 / shared-memory bound kernels,
    # measured on this device by the library's microbenchmarks
    try:
        peaks = lpb.lpb_measure_peaks(torch.cuda.current_stream(dev))
        peaks["source"] = "measured (lpb_measure_peaks: FMA chains and 16-byte shared-memory loads+stores, all SMs)"
    except Exception as ex:  # noqa: BLE001
        peaks = {"fp64_gflops": FP64_NOMINAL_GFLOPS, "fp32_gflops": FP32_NOMINAL_GFLOPS,
                 "smem_gbs": SMEM_NOMINAL_GBS, "source": f"nominal (measurement failed: {ex})"}
    FP64_PEAK_GFLOPS = peaks["fp64_gflops"]
    FP32_PEAK_GFLOPS = peaks["fp32_gflops"]
    SMEM_PEAK_GBS = peaks["smem_gbs"]

    batch = make_batch(args.workload, args.num_lps, rank)
    N = batch.num_lps
    A = torch.from_numpy(batch.A).to(dev)
    b = torch.from_numpy(batch.b).to(dev)
    c = torch.from_numpy(batch.c).to(dev)
    stream = torch.cuda.current_stream(dev)
    in_bytes = (A.numel() + b.numel() + c.numel()) * 8
    head_prec = lpb.LP_PREC_FP32_REFINE if args.precision == "fp32r" else lpb.LP_PREC_FP64

    def create(prec, host=None):
        opts = lpb.lpb_default_opts(precision=prec)
        if host is None:
            return lpb.lp_batch_create(batch.m, batch.n, batch.a_off, A, batch.b_off, b, batch.c_off, c,
                                       lpb.LPB_DEVICE, opts, stream)
        return lpb.lp_batch_create(batch.m, batch.n, batch.a_off, host["A"], batch.b_off, host["b"],
                                   batch.c_off, host["c"], lpb.LPB_HOST, opts, stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(v):
        if ws > 1:
            import torch.distributed as dist
            t = torch.tensor([v], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        return v

    def timed(h, steps, warmup, clocks=False):
        for _ in range(max(3, warmup)):
            lpb.lp_batch_solve(h, stream)
        torch.cuda.synchronize()
        lpb.lp_batch_set_timing(h, True)  # per-stage CUDA events on the solve's stream
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index) if clocks else None
        if sampler:
            sampler.__enter__()
            time.sleep(0.25)
        start.record(stream)
        for s in range(steps):
            ev[s][0].record(stream)
            lpb.lp_batch_solve(h, stream)
            ev[s][1].record(stream)
        stop.record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__()
        barrier()
        elapsed = max_over_ranks(start.elapsed_time(stop))
        stages = lpb.lp_batch_stage_times(h)
        lpb.lp_batch_set_timing(h, False)
        return elapsed, [e[0].elapsed_time(e[1]) for e in ev], (sampler.summary() if sampler else None), stages

    def results(h):
        r = dict(status=np.zeros(N, np.int32), iters=np.zeros(N, np.int32), obj=np.zeros(N))
        lpb.lp_batch_results(h, r["status"], r["iters"], r["obj"], None, None, lpb.LPB_HOST)
        return r

    # ---- headline path ----------------------------------------------------
    h = create(head_prec)
    info = lpb.lp_batch_plan_info(h)
    elapsed_ms, step_ms, clocks, stages = timed(h, args.steps, args.warmup, clocks=True)
    res = results(h)
    info = lpb.lp_batch_plan_info(h)  # fallback count of the last solve
    value = N * ws * args.steps / (elapsed_ms * 1e-3)

    # ---- plain FP64 GPU simplex on the same data (the comparison) ----------
    fp64 = None
    r64 = None
    if head_prec != lpb.LP_PREC_FP64:
        h64 = create(lpb.LP_PREC_FP64)
        e64, s64, _, stages64 = timed(h64, args.steps, args.warmup)
        r64 = results(h64)
        lpb.lp_batch_destroy(h64)
        opt = r64["status"] == 0
        rel = np.abs(res["obj"][opt] - r64["obj"][opt]) / np.maximum(1.0, np.abs(r64["obj"][opt]))
        fp64 = {"value": N * ws * args.steps / (e64 * 1e-3), "unit": "LPs/s", "ms_per_step": e64 / args.steps,
                "speedup_of_headline": value / (N * ws * args.steps / (e64 * 1e-3)),
                "headline_vs_fp64_gpu": {"lps_compared": N,
                                         "status_mismatches": int(np.sum(res["status"] != r64["status"])),
                                         "max_rel_obj_err_on_optimal": float(rel.max()) if rel.size else 0.0}}
        fp64_fmas = algorithmic_fmas(batch, r64["iters"])
        fp64_kernel_ms = stages64[0]
        fp64["roofline"] = {"bound": "alu", "kernel": "fp64_resident_kernel",
                            "achieved": 2.0 * fp64_fmas / (fp64_kernel_ms * 1e-3) / 1e9, "peak": FP64_PEAK_GFLOPS,
                            "unit": "GFLOP/s",
                            "frac": 2.0 * fp64_fmas / (fp64_kernel_ms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                            "kernel_ms": fp64_kernel_ms,
                            "timing": "CUDA events around the solve's launch groups, mean of the timed steps"}

    # stage 0 = every launch group of a solve (CUDA events, fork to join);
    # stage 1 = FP64 re-solve of uncertified LPs (mixed precision only)
    kernel_ms, fallback_ms, _ = stages
    fmas = algorithmic_fmas(batch, res["iters"])
    if head_prec == lpb.LP_PREC_FP64:
        achieved = 2.0 * fmas / (kernel_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "kernel": "fp64_resident_kernel", "achieved": achieved,
                    "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
                    "traffic": None, "kernel_ms": kernel_ms,
                    "peak_source": peaks["source"],
                    "work": "sum over LPs of pivots x (m+1)(n+1) FMAs"}
    else:
        # FP32 tableau pivots in shared memory: each pivot reads and writes the
        # (m+1)(n+1) FP32 tableau once (algorithmic bytes), and does (m+1)(n+1)
        # FMAs on the FP32 pipe
        smem_bytes = 2.0 * 4.0 * fmas
        achieved = smem_bytes / (kernel_ms * 1e-3) / 1e9
        flops = 2.0 * fmas / (kernel_ms * 1e-3) / 1e9
        mixed_threads = {g["threads"] for g in lpb.lp_batch_groups(h) if g["kind"] == 0}
        mixed_name = "mixed_warp_kernel" if mixed_threads == {32} else "mixed_kernel"
        roofline = {"bound": "smem", "kernel": mixed_name, "achieved": achieved,
                    "peak": SMEM_PEAK_GBS, "unit": "GB/s", "frac": achieved / SMEM_PEAK_GBS,
                    "peak_source": peaks["source"],
                    "traffic": MIXED_DRAM_BYTES_PER_LP * N if mixed_name == "mixed_warp_kernel" else None,
                    "traffic_note": "DRAM bytes per step: the ncu capture's read+write per LP (A, b, c once, "
                                    "outputs) x the step's LPs; the tableau itself never leaves shared memory; "
                                    f"algorithmic DRAM bytes of the inputs alone: {in_bytes:.4g}",
                    "kernel_ms": kernel_ms, "fallback_ms": fallback_ms,
                    "work": "shared-memory bytes: sum over LPs of reported pivots x 2 x (m+1)(n+1) x 4 (the FP32 "
                            "tableau read and written once per pivot; FP32 pivots of certified LPs, the FP64 "
                            "re-solve's pivots for uncertified ones; build and FP64 certificate not counted)",
                    "fp32_pipe": {"achieved_gflops": flops, "peak_gflops": FP32_PEAK_GFLOPS,
                                  "frac": flops / FP32_PEAK_GFLOPS},
                    "timing": f"CUDA events around the solve's launch groups (all {mixed_name} launches, "
                              "fork to join), mean of the timed steps"}

    # ---- hyperbox LPs (Section 4.4, Eq. 7): support function of one box ----
    hyperbox = None
    if not args.no_hyperbox:
        hb_num, hb_dim = args.hyperbox_dirs, 28
        Lh, loh, hih = W.hyperbox_directions(hb_num, hb_dim, start=rank * hb_num)
        dL = torch.from_numpy(Lh).to(dev)
        dlo, dhi = torch.from_numpy(loh).to(dev), torch.from_numpy(hih).to(dev)
        dobj = torch.empty(hb_num, dtype=torch.float64, device=dev)
        del Lh
        for _ in range(max(3, args.warmup)):
            lpb.lp_hyperbox_solve(dL, dlo, dhi, dobj, None, ptr_kind=lpb.LPB_DEVICE, stream=stream)
        torch.cuda.synchronize()
        hb_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        barrier()
        for s_ in range(args.steps):
            hb_ev[s_][0].record(stream)
            lpb.lp_hyperbox_solve(dL, dlo, dhi, dobj, None, ptr_kind=lpb.LPB_DEVICE, stream=stream)
            hb_ev[s_][1].record(stream)
        torch.cuda.synchronize()
        hb_ms = max_over_ranks(statistics.mean(e0.elapsed_time(e1) for e0, e1 in hb_ev))
        flops = 2.0 * hb_num * hb_dim
        bytes_ = 8.0 * hb_num * (hb_dim + 1)
        hyperbox = {
            "workload": f"hyperbox{hb_dim}_dirs{hb_num}", "value": hb_num * ws / (hb_ms * 1e-3), "unit": "LPs/s",
            "ms_per_step": hb_ms,
            "roofline": {"bound": "alu", "kernel": "hyperbox_tile_kernel",
                         "achieved": flops / (hb_ms * 1e-3) / 1e9, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": flops / (hb_ms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                         "traffic": HYPERBOX_DRAM_BYTES_PER_LP_DIM28 * hb_num if hb_dim == 28 else None,
                         "hbm_gbs": bytes_ / (hb_ms * 1e-3) / 1e9, "hbm_peak_gbs": HBM_PEAK_GBS,
                         "hbm_frac": bytes_ / (hb_ms * 1e-3) / 1e9 / HBM_PEAK_GBS,
                         "work": "one FP64 FMA per direction coordinate (the FP64 pipe binds before HBM: "
                                 "1 FMA per 8 bytes read)"},
            "timing": "CUDA events around each call on the launching stream, mean of the timed steps; "
                      "inputs (0.94 GB) larger than L2",
        }
        del dL, dlo, dhi, dobj

    def ev_time(fn):
        """Mean ms of K calls of fn between CUDA events on the solve's stream (after W warm-ups)."""
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a0.record(stream)
        for _ in range(args.steps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(a0.elapsed_time(a1)) / args.steps

    # ---- support function of one polytope: 40 halfspaces in R^10, 1e5 directions
    support = None
    if not args.no_support:
        sb = W.support_function(args.support_dirs, start=rank * args.support_dirs)
        support = {"workload": f"support40x10_dirs{sb.num_lps}", "unit": "LPs/s"}
        res_s = {}
        for label, prec in (("fp64", lpb.LP_PREC_FP64), ("fp32r", lpb.LP_PREC_FP32_REFINE)):
            hs = lpb.BatchSolver(sb, opts=lpb.lpb_default_opts(precision=prec), stream=stream)
            ms = ev_time(lambda: lpb.lp_batch_solve(hs.h, stream))
            res_s[label] = hs.results()
            info_s = hs.plan_info()
            hs.close()
            support[label] = {"value": sb.num_lps * ws / (ms * 1e-3), "ms_per_step": ms,
                              "fp64_fallback_lps": int(info_s["num_fallback"]) if prec != lpb.LP_PREC_FP64 else 0}
            # roofline of the whole solve, from the solver's own pivot counts:
            # FP64, FMAs on the FP64 pipe; mixed, the FP32 tableau's shared-
            # memory bytes (read and written once per pivot), as for the headline
            fm_s = algorithmic_fmas(sb, res_s[label]["iters"])
            if prec == lpb.LP_PREC_FP64:
                ach_s = 2.0 * fm_s / (ms * 1e-3) / 1e9
                support[label]["roofline"] = {
                    "bound": "alu", "achieved": ach_s, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": ach_s / FP64_PEAK_GFLOPS, "work": "sum over LPs of pivots x (m+1)(n+1) FMAs",
                    "timing": "whole solve (every launch)"}
            else:
                ach_s = 8.0 * fm_s / (ms * 1e-3) / 1e9
                support[label]["roofline"] = {
                    "bound": "smem", "achieved": ach_s, "peak": SMEM_PEAK_GBS, "unit": "GB/s",
                    "frac": ach_s / SMEM_PEAK_GBS,
                    "work": "sum over LPs of pivots x 2 x (m+1)(n+1) x 4 bytes (FP32 tableau read and written "
                            "once per pivot; certificate not counted)",
                    "timing": "whole solve (every launch, FP64 re-solve included)"}
        r64s, r32s = res_s["fp64"], res_s["fp32r"]
        opt = r64s["status"] == 0
        rel = np.abs(r32s["obj"][opt] - r64s["obj"][opt]) / np.maximum(1.0, np.abs(r64s["obj"][opt]))
        support["value"] = support["fp32r"]["value"]
        support["speedup_over_fp64"] = support["fp32r"]["value"] / support["fp64"]["value"]
        support["fp32r_vs_fp64_gpu"] = {"lps_compared": int(sb.num_lps),
                                        "status_mismatches": int(np.sum(r32s["status"] != r64s["status"])),
                                        "max_rel_obj_err_on_optimal": float(rel.max()) if rel.size else 0.0}
        if rank == 0:
            idx_s = sample_indices(sb.num_lps, args.oracle_sample)
            r_s, dt_s, o_s = cpu_oracle_run(sb, idx_s, os.cpu_count() or 1)
            support["vs_oracle"] = {lab: vs_oracle(res_s[lab]["status"], res_s[lab]["obj"], idx_s, o_s)
                                    for lab in ("fp64", "fp32r")}
            support["cpu_oracle"] = oracle_rate_note(r_s, dt_s, len(idx_s))
        support["timing"] = "CUDA events on the solve's stream around K whole solves"
        del sb, res_s

    # ---- 1000 LPs of 5 x 5 (positive data, slack basis feasible) -----------
    c1 = None
    if not args.no_c1:
        b1 = make_batch("dense5x5_1k", None, rank)
        c1 = {"workload": f"dense5x5_{b1.num_lps}", "unit": "LPs/s"}
        for label, prec in (("fp64", lpb.LP_PREC_FP64), ("fp32r", lpb.LP_PREC_FP32_REFINE)):
            h1_ = lpb.BatchSolver(b1, opts=lpb.lpb_default_opts(precision=prec), stream=stream)
            ms_plain = ev_time(lambda: lpb.lp_batch_solve(h1_.h, stream))
            r1 = h1_.results()
            # the same solve captured once and replayed as a CUDA graph: one
            # launch instead of the counter resets, events and kernel launches
            ms_graph = ev_time(lambda: lpb.lp_batch_solve_graph(h1_.h, stream))
            rg = h1_.results()
            h1_.close()
            ms = min(ms_plain, ms_graph)
            fl1 = 2.0 * algorithmic_fmas(b1, r1["iters"])
            c1[label] = {"value": b1.num_lps * ws / (ms * 1e-3), "ms_per_step": ms, "ms_plain": ms_plain,
                         "ms_graph": ms_graph, "result": r1,
                         "graph_results_identical": bool(all(np.array_equal(r1[k], rg[k])
                                                             for k in ("status", "iters", "obj", "x"))),
                         "fp64_pipe_frac": fl1 / (ms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS}
        c1["value"] = c1["fp64"]["value"]
        c1["timing"] = ("CUDA events on the solve's stream around K whole solves, plain and as a CUDA-graph replay "
                        "(the faster is the value); one launch of 1000 tiny CTAs, so the time is launch and "
                        "latency, not throughput")
        if rank == 0:
            idx1 = np.arange(b1.num_lps)
            r_one, dt_one, o1 = cpu_oracle_run(b1, idx1, 1)
            r_all, dt_all, _ = cpu_oracle_run(b1, idx1, os.cpu_count() or 1)
            c1["cpu_oracle"] = {"one_thread": r_one, "all_threads": r_all, "cores": os.cpu_count() or 1,
                                "unit": "LPs/s", "sample": f"all {b1.num_lps} LPs"}
            for label in ("fp64", "fp32r"):
                c1[label]["vs_oracle"] = vs_oracle(c1[label]["result"]["status"], c1[label]["result"]["obj"],
                                                   idx1, o1)
        for label in ("fp64", "fp32r"):
            del c1[label]["result"]
        del b1

    # ---- uneven batch: m, n log-uniform in [10, 500], 2e4 LPs ----------------
    uneven = None
    if not args.no_uneven:
        ub = W.uneven_dense(args.uneven_lps, start=rank * args.uneven_lps)
        um, un = ub.m.astype(np.float64), ub.n.astype(np.float64)

        uneven = {"workload": f"uneven10to500_{ub.num_lps}", "unit": "LPs/s"}
        res_u = {}
        for label, prec in (("fp64", lpb.LP_PREC_FP64), ("fp32r", lpb.LP_PREC_FP32_REFINE)):
            hu = lpb.BatchSolver(ub, opts=lpb.lpb_default_opts(precision=prec), stream=stream)
            ms_default = ev_time(lambda: lpb.lp_batch_solve(hu.h, stream))
            ru = hu.results()
            lpb.lp_batch_autotune(hu.h, rounds=1, stream=stream)
            ms_tuned = ev_time(lambda: lpb.lp_batch_solve(hu.h, stream))
            ms_graph = ev_time(lambda: lpb.lp_batch_solve_graph(hu.h, stream))
            rt = hu.results()
            res_u[label] = rt
            groups = lpb.lp_batch_groups(hu.h)
            hu.close()
            best = min(ms_tuned, ms_graph)
            fl = 2.0 * float(np.sum(rt["iters"] * (um + 1.0) * (un + 1.0)))
            uneven[label] = {
                "value": ub.num_lps * ws / (best * 1e-3), "ms_default_plan": ms_default, "ms_autotuned": ms_tuned,
                "ms_graph": ms_graph, "groups": len(groups),
                "persistent_groups": sum(1 for g in groups if g["persistent"] and g["kind"] != 2),
                "streamed_lps": sum(g["count"] for g in groups if g["kind"] in (2, 4)),
                "results_unchanged_by_tuning": bool(all(np.array_equal(ru[k], rt[k]) for k in ("status", "obj", "x"))),
                "achieved_gflops": fl / (best * 1e-3) / 1e9, "fp64_peak_gflops": FP64_PEAK_GFLOPS,
            }
        # FP64 in one persistent launch (LPB_SCHED_SINGLE: one work queue,
        # longest work first, shared memory or a global slot per LP)
        hs1 = lpb.BatchSolver(ub, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64,
                                                             schedule=lpb.LPB_SCHED_SINGLE), stream=stream)
        ms_single = ev_time(lambda: lpb.lp_batch_solve(hs1.h, stream))
        ms_single_graph = ev_time(lambda: lpb.lp_batch_solve_graph(hs1.h, stream))
        r1 = hs1.results()
        uneven["fp64_single_launch"] = {
            "ms": ms_single, "ms_graph": ms_single_graph, "launches_per_solve": hs1.plan_info()["num_groups"],
            "default_plan_launches_per_solve": uneven["fp64"]["groups"],
            "value": ub.num_lps * ws / (min(ms_single, ms_single_graph) * 1e-3),
            "results_identical_to_default_plan": bool(all(np.array_equal(r1[k], res_u["fp64"][k])
                                                          for k in ("status", "iters", "obj", "x", "y")))}
        hs1.close()
        # the same for mixed precision: one persistent launch of the mixed
        # per-LP code, then the FP64 re-solves of the uncertified LPs
        hs2 = lpb.BatchSolver(ub, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP32_REFINE,
                                                             schedule=lpb.LPB_SCHED_SINGLE), stream=stream)
        ms_single2 = ev_time(lambda: lpb.lp_batch_solve(hs2.h, stream))
        ms_single2_graph = ev_time(lambda: lpb.lp_batch_solve_graph(hs2.h, stream))
        r2 = hs2.results()
        uneven["fp32r_single_launch"] = {
            "ms": ms_single2, "ms_graph": ms_single2_graph,
            "launches_per_solve": hs2.plan_info()["num_groups"],
            "what": "one launch of the mixed per-LP code plus the FP64 re-solve launches",
            "default_plan_launches_per_solve": uneven["fp32r"]["groups"],
            "value": ub.num_lps * ws / (min(ms_single2, ms_single2_graph) * 1e-3),
            "results_identical_to_default_plan": bool(all(np.array_equal(r2[k], res_u["fp32r"][k])
                                                          for k in ("status", "iters", "obj", "x", "y")))}
        hs2.close()
        uneven["value"] = max(uneven["fp64"]["value"], uneven["fp32r"]["value"])
        opt_u = res_u["fp64"]["status"] == 0
        rel_u = (np.abs(res_u["fp32r"]["obj"][opt_u] - res_u["fp64"]["obj"][opt_u])
                 / np.maximum(1.0, np.abs(res_u["fp64"]["obj"][opt_u])))
        uneven["fp32r_vs_fp64_gpu"] = {
            "lps_compared": int(ub.num_lps),
            "status_mismatches": int(np.sum(res_u["fp32r"]["status"] != res_u["fp64"]["status"])),
            "max_rel_obj_err_on_optimal": float(rel_u.max()) if rel_u.size else 0.0}
        # the LPs above one CTA's shared memory alone: through the streamed FP64
        # kernel (tableau in a global workspace slot, 16-byte rank-1 updates; the
        # default for them) and on thread-block clusters (tableau split over the
        # cluster's shared memory): the same bits.  The streamed kernel is HBM/L2
        # bound: its roofline is the algorithmic bytes 2 (m+1)(n+1) 8 per pivot
        big_lp = np.nonzero((um + 2.0) * (un + 1.0) * 8.0 > 227 * 1024)[0]
        if big_lp.size:
            bsub = ub.subset(big_lp)
            big = {}
            for lab, sch in (("streamed", lpb.LPB_SCHED_STREAMED), ("cluster", lpb.LPB_SCHED_CLUSTER)):
                hs = lpb.BatchSolver(bsub, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64, schedule=sch),
                                     stream=stream)
                big[lab] = (ev_time(lambda: lpb.lp_batch_solve(hs.h, stream)), hs.results())
                hs.close()
            ms_s, rs = big["streamed"]
            bm, bn = bsub.m.astype(np.float64), bsub.n.astype(np.float64)
            sbytes = 2.0 * 8.0 * float(np.sum(rs["iters"] * (bm + 1.0) * (bn + 1.0)))
            same = all(np.array_equal(rs[k], big["cluster"][1][k]) and np.array_equal(rs[k], res_u["fp64"][k][big_lp])
                       for k in ("status", "iters", "obj"))
            uneven["fp64_large_lps"] = {
                "lps": int(big_lp.size), "what": "the LPs whose FP64 tableau exceeds one CTA (~227 KB)",
                "streamed_ms": ms_s, "cluster_ms": big["cluster"][0],
                "streamed_roofline": {"bound": "hbm", "achieved": sbytes / (ms_s * 1e-3) / 1e9, "peak": HBM_PEAK_GBS,
                                      "unit": "GB/s", "frac": sbytes / (ms_s * 1e-3) / 1e9 / HBM_PEAK_GBS,
                                      "work": "sum over LPs of pivots x 2 (m+1)(n+1) x 8 bytes (the condensed "
                                              "tableau read and written once per pivot; part of it from L2)"},
                "same_status_iters_obj_streamed_cluster_default": bool(same)}
            del bsub, big
        if rank == 0:
            idx_u = sample_indices(ub.num_lps, max(50, args.oracle_sample // 5))
            r_u, dt_u, o_u = cpu_oracle_run(ub, idx_u, os.cpu_count() or 1)
            uneven["vs_oracle"] = {lab: vs_oracle(res_u[lab]["status"], res_u[lab]["obj"], idx_u, o_u)
                                   for lab in ("fp64", "fp32r")}
            uneven["vs_oracle"]["sample"] = f"{len(idx_u)} evenly spaced LPs (oracle {dt_u:.2f} s)"
            uneven["cpu_oracle"] = oracle_rate_note(r_u, dt_u, len(idx_u))
        uneven["timing"] = "CUDA events on the solve's stream around K whole solves (default plan, autotuned plan, graph replay)"
        del ub

    # ---- learned warm start on the shared-A family (200 x 100) ----------------
    warm = None
    if not args.no_warm:
        from paper_1802_08557_gb300 import warmstart as WS
        t0 = time.perf_counter()
        train_set = W.shared_matrix_family_blocks(args.warm_train, start=rank * args.warm_train)
        net, tinfo = WS.train(train_set, epochs=2.0, batch_size=1024, seed=0)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del train_set
        test_set = W.shared_matrix_family(args.warm_test, start=rank * args.warm_test)
        hw = lpb.BatchSolver(test_set, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64), stream=stream)
        # cold FP64
        e_cold, _, _, st_cold = timed(hw.h, args.steps, args.warmup)
        rc = hw.results()
        # warm: network + restricted solves + cold FP64 for the rest, every step
        for _ in range(max(3, args.warmup)):
            lpb.lp_batch_solve_warm(hw.h, net, 0.2, stream)
        torch.cuda.synchronize()
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        w0.record(stream)
        for _ in range(args.steps):
            lpb.lp_batch_solve_warm(hw.h, net, 0.2, stream)
        w1.record(stream)
        torch.cuda.synchronize()
        e_warm = max_over_ranks(w0.elapsed_time(w1))
        rw = hw.results()
        pw = hw.plan_info()
        # the network alone: forward over the test set's features
        feats = torch.empty((test_set.num_lps, 300), dtype=torch.float32, device=dev)
        logits = torch.empty((test_set.num_lps, 200), dtype=torch.float32, device=dev)
        lpb.lp_batch_features(hw.h, feats, stream)
        net.forward(feats, logits, stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            net.forward(feats, logits, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = f0.elapsed_time(f1) / args.steps
        mlp_flops = 2.0 * test_set.num_lps * (300 * 512 + 512 * 512 + 512 * 200)
        # the first layer's product alone (1e5 x 320 . 512 x 320^T, bias + ReLU
        # into BF16 activations) through the same kernel, on operands of its shape
        nl = test_set.num_lps
        a1_in = torch.randn((nl, 320), device=dev).to(torch.bfloat16)
        w1 = (torch.rand((512, 320), device=dev) * 0.2 - 0.1).to(torch.bfloat16)
        b1 = torch.zeros(512, dtype=torch.float32, device=dev)
        h1 = torch.empty((nl, 512), dtype=torch.bfloat16, device=dev)

        def layer1_call():
            lpb.lp_mlp_gemm_bf16(lpb.LPB_EPI_BIAS_RELU, lpb.LPB_GEMM_TC, nl, 512, 320, a1_in, 320, w1, 320, None, 0,
                                 b1, None, h1, 512, None, 0, stream)

        l1_ms = ev_time(layer1_call)
        l1_flops = 2.0 * nl * 512 * 320
        l1_bytes = 2.0 * nl * (320 + 512) + 2.0 * 512 * 320
        layer1 = {"shape": f"{nl} x 320 . 512 x 320^T, bias + ReLU -> BF16", "ms": l1_ms,
                  "achieved_tflops": l1_flops / (l1_ms * 1e-3) / 1e12, "peak_tflops": BF16_PEAK_TFLOPS,
                  "frac": l1_flops / (l1_ms * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                  "hbm_gbs": l1_bytes / (l1_ms * 1e-3) / 1e9, "hbm_frac": l1_bytes / (l1_ms * 1e-3) / 1e9 / HBM_PEAK_GBS,
                  "tc_faults": lpb.lp_mlp_tc_faults()}
        del a1_in, w1, b1, h1
        hw.close()
        net.close()
        opt = rc["status"] == 0
        rel = np.abs(rw["obj"][opt] - rc["obj"][opt]) / np.maximum(1.0, np.abs(rc["obj"][opt]))
        nt_ = test_set.num_lps
        warm_oracle = None
        if rank == 0:
            idx_w = sample_indices(nt_, args.oracle_sample)
            r_w, dt_w, o_w = cpu_oracle_run(test_set, idx_w, os.cpu_count() or 1)
            warm_oracle = {"warm": vs_oracle(rw["status"], rw["obj"], idx_w, o_w),
                           "cold_fp64": vs_oracle(rc["status"], rc["obj"], idx_w, o_w),
                           "cpu_oracle": oracle_rate_note(r_w, dt_w, len(idx_w))}
        warm = {
            "workload": f"shared200x100_test{nt_}",
            "value": nt_ * ws * args.steps / (e_warm * 1e-3), "unit": "LPs/s", "ms_per_step": e_warm / args.steps,
            "cold_fp64": {"value": nt_ * ws * args.steps / (e_cold * 1e-3), "ms_per_step": e_cold / args.steps},
            "speedup_over_cold_fp64": e_cold / e_warm,
            "certified_fraction": pw["num_warm_certified"] / nt_,
            "restricted_solves_per_lp": pw["num_warm_rounds"] / nt_,
            "warm_vs_cold_fp64_gpu": {"lps_compared": int(nt_),
                                      "status_mismatches": int(np.sum(rw["status"] != rc["status"])),
                                      "max_rel_obj_err_on_optimal": float(rel.max()) if rel.size else 0.0},
            "vs_oracle": warm_oracle,
            "training": {"lps": tinfo["train_lps"], "steps": tinfo["steps"], "seconds": train_s,
                         "first_loss": tinfo["first_loss"], "last_loss": tinfo["last_loss"],
                         "what": "cold FP64 solve of the training LPs + features/labels + Adam steps, all on the GPU"},
            "network_forward": {"ms": fwd_ms, "achieved_tflops": mlp_flops / (fwd_ms * 1e-3) / 1e12,
                                "peak_tflops": BF16_PEAK_TFLOPS, "peak_source": PEAKS_SOURCE,
                                "frac": mlp_flops / (fwd_ms * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                                "note": "tcgen05 GEMMs (TMA tiles, TMEM accumulators) with fused bias/ReLU/BF16 "
                                        "epilogues; 300->512->512->200 over the test set, one chunk"},
            "layer1_product": layer1,
            "timing": "CUDA events on the solve's stream around K whole warm solves "
                      "(features, network, restricted solves, cold FP64 re-solve)",
        }
        del feats, logits

    # ---- end to end through the C ABI with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(getattr(batch, k)).pin_memory() for k in ("A", "b", "c")}
        out = dict(status=torch.empty(N, dtype=torch.int32).pin_memory(),
                   iters=torch.empty(N, dtype=torch.int32).pin_memory(),
                   obj=torch.empty(N, dtype=torch.float64).pin_memory(),
                   x=torch.empty(int(batch.n.astype(np.int64).sum()), dtype=torch.float64).pin_memory())
        meta_bytes = N * (4 + 4 + 8 + 8 + 8)
        h2d = sum(v.numel() * 8 for v in pinned.values()) + meta_bytes
        d2h = sum(v.numel() * v.element_size() for v in out.values())
        e2e_opts = lpb.lpb_default_opts(precision=head_prec)

        def e2e_step():
            # one C-ABI call: pinned host inputs -> host results, the input
            # copies of each chunk overlapped with the previous chunk's solve
            lpb.lp_solve_host(batch.m, batch.n, batch.a_off, pinned["A"], batch.b_off, pinned["b"], batch.c_off,
                              pinned["c"], out["status"], out["iters"], out["obj"], out["x"], None,
                              opts=e2e_opts, chunks=args.e2e_chunks)

        e2e_step()
        torch.cuda.synchronize()
        e2e_steps = max(10, args.steps)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": N * ws * e2e_steps / dt, "unit": "LPs/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * dt / e2e_steps,
               "api": "lp_solve_host (pinned host inputs, host results; copies overlapped with the solve "
                      f"in {'the library default' if args.e2e_chunks == 0 else args.e2e_chunks} chunks)"}

    cpu = None
    headline_vs_oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        idx_h = sample_indices(N, args.cpu_sample)
        rate, dt, o_h = cpu_oracle_run(batch, idx_h, threads)
        idx_1 = sample_indices(N, max(100, args.cpu_sample // 10))
        rate_1, dt_1, _ = cpu_oracle_run(batch, idx_1, 1)
        cpu = {"value": rate, "unit": "LPs/s", "cores": threads, "kind": "oracle",
               "sample": f"{len(idx_h)} of {N} LPs (evenly spaced indices), {dt:.1f} s wall",
               "one_thread": {"value": rate_1, "unit": "LPs/s", "cores": 1,
                              "sample": f"{len(idx_1)} of {N} LPs (evenly spaced), {dt_1:.1f} s wall"}}
        # per-LP accuracy of both GPU paths against the oracle on the same LPs
        headline_vs_oracle = vs_oracle(res["status"], res["obj"], idx_h, o_h)
        if fp64 is not None:
            fp64["vs_oracle"] = vs_oracle(r64["status"], r64["obj"], idx_h, o_h)
        if args.per_lp_file:
            st_h = res["status"][idx_h]
            rel_h = np.where(o_h["status"] == 0,
                             np.abs(res["obj"][idx_h] - o_h["obj"]) / np.maximum(1.0, np.abs(o_h["obj"])), np.nan)
            np.savez_compressed(args.per_lp_file, lp_index=idx_h, oracle_status=o_h["status"], gpu_status=st_h,
                                oracle_obj=o_h["obj"], gpu_obj=res["obj"][idx_h], rel_obj_err=rel_h)

    lpb.lp_batch_destroy(h)
    if rank == 0:
        counts = np.bincount(res["status"], minlength=5)
        launches = info["num_groups"]
        line = {
            "metric": METRIC, "value": value, "unit": "LPs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head_prec == lpb.LP_PREC_FP64 else "f32+f64",
            "data": "synthetic",
            "config": bench_config(args.workload, batch),
            "run": {"precision": "fp64" if head_prec == lpb.LP_PREC_FP64 else
                    "fp32 tableau + fp64 certificate (fp64 re-solve of uncertified LPs)",
                       "launch_groups": launches, "phase1_lps": info["num_phase1"],
                       "fp64_fallback_lps": info["num_fallback"],
                       "kernel_self_check_failures": info["internal_errors"],
                       "status_counts": {"optimal": int(counts[0]), "infeasible": int(counts[1]),
                                         "unbounded": int(counts[2]), "iter_limit": int(counts[3]),
                                         "numerical": int(counts[4])},
                       "mean_pivots": float(res["iters"].mean())},
            "roofline": roofline,
            "vs_oracle": headline_vs_oracle,
            "peaks": peaks,
            "fp64_plain": fp64,
            "dense5x5": c1,
            "hyperbox": hyperbox,
            "warm_start": warm,
            "support_function": support,
            "uneven": uneven,
            "clocks": clocks,
            "gpu_launches": args.steps * launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """One workload, a few launches, for ncu (see --profile-case)."""
    import torch
    from paper_1802_08557_gb300 import build, lpbatch as lpb
    from paper_1802_08557_gb300 import workloads as W
    build.build()
    lpb.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    if args.profile_case == "gemm_tc_layer1":
        nl = args.warm_test
        g = torch.Generator(device=dev).manual_seed(0)
        a = torch.randn((nl, 320), device=dev, generator=g).to(torch.bfloat16)
        w = (torch.rand((512, 320), device=dev, generator=g) * 0.2 - 0.1).to(torch.bfloat16)
        bias = torch.zeros(512, dtype=torch.float32, device=dev)
        h = torch.empty((nl, 512), dtype=torch.bfloat16, device=dev)
        for _ in range(4):
            lpb.lp_mlp_gemm_bf16(lpb.LPB_EPI_BIAS_RELU, lpb.LPB_GEMM_TC, nl, 512, 320, a, 320, w, 320, None, 0, bias,
                                 None, h, 512, None, 0, stream)
        torch.cuda.synchronize()
        print(f"gemm_tc_layer1: 4 launches of {nl} x 320 -> 512, faults {lpb.lp_mlp_tc_faults()}")
    else:
        ub = W.uneven_dense(args.uneven_lps)
        um, un = ub.m.astype(np.float64), ub.n.astype(np.float64)
        big = ub.subset(np.nonzero((um + 2.0) * (un + 1.0) * 8.0 > 227 * 1024)[0])
        hs = lpb.BatchSolver(big, opts=lpb.lpb_default_opts(precision=lpb.LP_PREC_FP64,
                                                            schedule=lpb.LPB_SCHED_STREAMED), stream=stream)
        for _ in range(3):
            lpb.lp_batch_solve(hs.h, stream)
        r = hs.results()
        hs.close()
        print(f"fp64_streamed_uneven: 3 solves of {big.num_lps} LPs, mean pivots {r['iters'].mean():.1f}")
    return 0


def main():
    args = parse()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
