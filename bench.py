#!/usr/bin/env python3
"""Throughput of the HMM recognition hot path on GB300 (one JSON line).

Default workload: the large-state configuration -- K=4 activity HMMs, N=128
states, M=256 symbols, Dirichlet(0.3) rows, 16384 ragged sequences with
T ~ U{100..2000} -- synthetic and seeded (the paper's UCF teamwork
recordings are not available). It is the largest configuration that fits
one GPU.

One step = the BF16 tensor-core forward of every (sequence, model) pair with
the argmax over models (recognition) and the BF16 tensor-core
forward-backward adjoint of every sequence against its labelled model (the
Baum-Welch E-step's expected counts, which are the log-likelihood gradient),
the two on two streams. Throughput unit: observations x models per second
(sum_s T_s * (K + 1) per step). `value` is timed with CUDA events around
eager steps on device-resident inputs, with an L2 flush (a 256 MB write)
between steps outside the timed events; `e2e` repeats the step through the
public API with the inputs copied from pinned host memory and every result
copied back inside the timed region. The line also carries the TF32 forward
and the Viterbi decoding of the same batch, the error of each precision
against the FP64 oracle on a sample, the measured peaks (BF16 from the pool's
file, FP32 from the library's FMA probe, TF32 from a GEMM), the oracle's
CPU throughput (all host threads and one), and short summaries of the
batched-recognition and training configurations.

Other workloads (--workload): batched (K=10, N=16: forward, Viterbi, adjoint,
gradient and Adam in one CUDA graph), gradient / training (the learning step),
teamwork (per-role recognition, N=5), cuhmm (512 states), longseq (few very
long sequences).

Multi-GPU: every rank runs its own shard (its own batch, seed + rank) with no
collective on the data path ("weak" scaling); the barrier and the max over
ranks use torch.distributed. `--impl reference` times the FP64 CPU oracle on
the host cores instead (rank 0 only), on a bounded sample of the same
configuration per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "large"
METRIC = "HMM obs·models/s (forward, Viterbi, fwd+adjoint)"
UNIT = "obs*models/s"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# setup x3, softmax, forward, v-scores, v-paths, adjoint, reduce x2, grad, adam x2
# (the adjoint is two kernels when its segments are split into ranges)
KERNELS_PER_STEP = 13
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-graph", action="store_true", help="time eager steps instead of replays")
    ap.add_argument("--scan-chunk", type=int, default=0,
                    help="longseq: steps per chunk of the parallel-in-time forward (0 = auto)")
    ap.add_argument("--teamwork-calls", default="sets", choices=["sets", "roles"],
                    help="teamwork recognition as one call per op over per-role model sets, "
                         "or one call per role on its own stream")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--skip-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--n-seqs", type=int, default=None, help="smaller batch (profiling only)")
    ap.add_argument("--lanes", default=None,
                    help="fixed lanes per pair 'fwd,viterbi,paths,adjoint' instead of autotuning")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["large", "batched", "gradient", "training", "teamwork", "cuhmm",
                             "longseq"],
                    help="large: tensor-core forward and adjoint (default); batched: the "
                         "full N=16 step; gradient/training: the learning step (and a "
                         "Baum-Welch iteration); teamwork: per-role recognition, N=5; "
                         "cuhmm: the 512-state forward")
    ap.add_argument("--skip-others", action="store_true",
                    help="large: skip the batched and training summaries")
    ap.add_argument("--quick", action="store_true",
                    help="large: the timed step and per-kernel times only (profiling runs)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def units_of(w) -> int:
    return int(w.lengths.astype(np.int64).sum()) * w.K


# ---------------------------------------------------------------------------
# CPU oracle leg (shared by the cpu_baseline key and --impl reference)
# ---------------------------------------------------------------------------
def oracle_step(w, idx, nthreads):
    """The step's arithmetic on the FP64 CPU oracle for sequences idx."""
    import oracle
    P = oracle.params(w.pi, w.A, w.B)
    sub = (w.symbols, w.offsets[idx], w.lengths[idx])
    oracle.forward(P, *sub, nthreads=nthreads)
    oracle.viterbi(P, *sub, nthreads=nthreads)
    _, cpi, cA, cB, _ = oracle.forward_backward(P, *sub, w.labels[idx], nthreads=nthreads)
    oracle.softmax_grad(P, cpi, cA, cB)


def cpu_sample(w, n):
    return np.random.default_rng(12345).choice(w.S, size=min(n, w.S), replace=False)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_1310_3322_gb300 import synth
    cores = os.cpu_count() or 1
    if args.workload == "large":
        w = synth.make_workload("large")
        # 8 sequences per step (a fresh seeded draw each step): a few seconds
        # of FP64 work on the host cores, so the whole run ends in minutes
        draws = [large_sample(w, 8, 0, 100 + i) for i in range(args.warmup + args.steps)]
        per_unit = w.K + 1
        work = oracle_large_step
        cfg = (f"large K={w.K} N={w.N} M={w.M} S={w.S} T~U{{100..2000}} (forward of all K "
               "models + argmax, forward-backward adjoint against the labelled model)")
        what = ("forward over all K models + labelled forward-backward counts, FP64 "
                "log-space, a fresh seeded draw of 8 sequences per step")
    else:
        w = synth.make_workload("batched")
        draws = [cpu_sample(w, 512)] * (args.warmup + args.steps)
        per_unit = w.K
        work = oracle_step
        cfg = "batched-recognition K=10 N=16 M=32 S=4096 T~U{30..300}"
        what = ("forward+Viterbi over all K models, labelled adjoint + logit gradient, FP64, "
                "512 sequences per step")
    for i in range(args.warmup):
        work(w, draws[i], cores)
    times, units = [], []
    for i in range(args.steps):
        idx = draws[args.warmup + i]
        t0 = time.perf_counter()
        work(w, idx, cores)
        times.append(time.perf_counter() - t0)
        units.append(int(w.lengths[idx].astype(np.int64).sum()) * per_unit)
    ms = 1e3 * float(np.mean(times))
    value = float(np.sum(units)) / float(np.sum(times))
    sample = f"{what}: {int(np.mean(units))} obs*models per step on average"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg, "sample_sequences": int(len(draws[-1])), "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"hmm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def setup_launches(S: int, ordered: bool = True) -> int:
    """Kernel launches of one call's setup: one block up to 4096 sequences;
    above, validation blocks plus (when the call needs the length order or
    prefix sums) the offsets block and the placement blocks."""
    return 1 if (S <= 4096 or not ordered) else 3


def traffic_for(kernel: str, n_seqs=None):
    """Per-launch DRAM bytes of `kernel` (for the adjoint: its two launches)
    from a committed ncu capture of the full workload, or None when a source
    changed since or the batch is not the full one (n_seqs set)."""
    if n_seqs is not None:
        return None
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    srcs = rec.get("sources") or [rec["source"]]
    want = rec["source_sha"] if isinstance(rec["source_sha"], list) else [rec["source_sha"]]
    for name, sha_want in zip(srcs, want):
        with open(os.path.join(ROOT, "paper_1310_3322_gb300", "csrc", name), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != sha_want:
                return None
    return rec["bytes_per_launch_full_workload"]


def run_gpu(args, emit=True):
    import torch
    import torch.distributed as dist
    from paper_1310_3322_gb300 import hmm, synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = synth.make_workload("batched", n_seqs=args.n_seqs, seed=synth.SEEDS["batched"] + rank)
    K, N, M = w.K, w.N, w.M
    units = units_of(w)
    sumT = int(w.lengths.astype(np.int64).sum())

    # ---- device-resident state --------------------------------------------
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device=dev)
    labels = torch.from_numpy(w.labels).to(dev)
    lab = seqs.labelled(labels)
    sizes = [K * N, K * N * N, K * N * M]
    logits = torch.from_numpy(np.concatenate([np.log(w.pi).ravel(), np.log(w.A).ravel(),
                                              np.log(w.B).ravel()]).astype(np.float32)).to(dev)
    grads = torch.zeros_like(logits)
    adam_m, adam_v = torch.zeros_like(logits), torch.zeros_like(logits)
    counter = torch.zeros(1, dtype=torch.int32, device=dev)
    shapes = [(K, N), (K, N, N), (K, N, M)]

    def views(flat):
        out, o = [], 0
        for n, sh in zip(sizes, shapes):
            out.append(flat[o:o + n].view(*sh))
            o += n
        return out

    lg, gr = views(logits), views(grads)
    probs = [torch.empty(sh, device=dev) for sh in shapes]
    ll = torch.empty((w.S, K), device=dev)
    am = torch.empty(w.S, dtype=torch.int32, device=dev)
    vs = torch.empty((w.S, K), device=dev)
    vbest = torch.empty(w.S, dtype=torch.int32, device=dev)
    vpath = torch.empty(max(w.total_obs, 1), dtype=torch.int32, device=dev)
    fll = torch.empty(w.S, device=dev)
    cnts = [torch.empty(sh, device=dev) for sh in shapes]
    ws = [hmm.Workspace(dev) for _ in range(3)]
    lr, gscale = 1e-3, -1.0 / float(sumT)

    # recognition (forward + argmax, Viterbi) and learning (adjoint, gradient,
    # Adam) only share the softmax output: the three latency-bound recursions
    # run on three streams (fork after the softmax, join before the step ends)
    rec_streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]

    def step(sq=seqs, lb=lab, concurrent=True, copy_out=None):
        cur = torch.cuda.current_stream()
        hmm.hmm_softmax_rows(*lg, out=probs)
        if concurrent:
            for x in rec_streams:
                x.wait_stream(cur)
        # the longest chain (the adjoint) is launched first
        hmm.hmm_forward_backward(*probs, lb, loglik=fll, counts=cnts, workspace=ws[2])
        # recognition results go to the host from their own streams, beside the
        # adjoint (copy_out = pinned host (argmax, path))
        with torch.cuda.stream(rec_streams[0] if concurrent else cur):
            hmm.hmm_viterbi(*probs, sq, score=vs, best_model=vbest, path=vpath, workspace=ws[1])
            if copy_out is not None:
                copy_out[1].copy_(vpath, non_blocking=True)
        with torch.cuda.stream(rec_streams[1] if concurrent else cur):
            hmm.hmm_forward(*probs, sq, loglik=ll, argmax=am, workspace=ws[0])
            if copy_out is not None:
                copy_out[0].copy_(am, non_blocking=True)
        hmm.hmm_softmax_grad(*probs, *cnts, out=gr)
        if concurrent:  # the next softmax overwrites probs: recognition must be done
            for x in rec_streams:
                cur.wait_stream(x)
        hmm.hmm_adam_step(logits, grads, adam_m, adam_v, lr, grad_scale=gscale,
                          step_counter=counter)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up (with the lanes-per-pair autotuner), then capture --------
    step()
    torch.cuda.synchronize()
    from paper_1310_3322_gb300 import tune
    if args.lanes:
        # fixed lanes per pair (forward, viterbi scores, viterbi paths, adjoint)
        npad = tune.n_pad(N)
        tuning = {}
        for op, g in zip((hmm.HMM_OP_FORWARD, hmm.HMM_OP_VITERBI, hmm.HMM_TUNE_VITERBI_PATHS,
                          hmm.HMM_OP_FORWARD_BACKWARD), (int(x) for x in args.lanes.split(","))):
            hmm.hmm_set_tuning(op, npad, g)
            tuning[tune.KERNEL_OF[op]] = {"lanes": g, "ms": {}}
    else:
        tuning = tune.autotune(*probs, seqs, lab, repeats=3, cache=None)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    status = hmm.hmm_get_device_status(ws[0]) | hmm.hmm_get_device_status(ws[1]) | \
        hmm.hmm_get_device_status(ws[2])
    if status:
        raise RuntimeError(f"device status {status:#x}")
    graph = None
    if not args.no_graph:
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                step()
        torch.cuda.current_stream().wait_stream(side)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()

    # ---- timed region ------------------------------------------------------
    clocks = Clocks(local)
    cur = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    clocks.start()
    time.sleep(0.3)  # let the sampler start
    for i in range(args.steps):
        flush.fill_(i & 0xff)          # L2 flush, outside the timed events
        evs[i][0].record(cur)
        if graph is not None:
            graph.replay()
        else:
            step()
        evs[i][1].record(cur)
    barrier()
    clk = clocks.stop()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    t_max = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms_max = float(t_max.item())
    value = units * world / (ms_max / 1e3)

    # ---- per-kernel breakdown (library CUDA events, eager steps with the
    # kernels serialised, so each launch is timed alone) --------------------
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        step(concurrent=False)
    torch.cuda.synchronize()
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    per_launch = {k: (v[1] / v[0] if v[0] else 0.0) for k, v in kt.items()}
    totals = {k: v[1] for k, v in kt.items()}
    step_kernel_ms = sum(totals.values()) / max(args.steps, 1)
    if kt["adjoint_pass"][0]:  # segment ranges: the adjoint is its passes + ranges
        per_launch["adjoint_ranges"] = per_launch["adjoint"]
        per_launch["adjoint"] += per_launch["adjoint_pass"]
        totals["adjoint"] += totals["adjoint_pass"]
    flops = {
        "forward": (2 * N * N + 3 * N) * sumT * K,
        "viterbi_scores": 2 * N * N * sumT * K,
        "viterbi_paths": 2 * N * N * sumT,
        "adjoint": (8 * N * N + 10 * N) * sumT,
    }
    dom = max(flops, key=lambda k: totals.get(k, 0.0))
    peak, peak_basis, nominal = fp32_peak(torch, dev)
    achieved = flops[dom] / (per_launch[dom] / 1e3) / 1e12
    roofline = {
        "bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": achieved / peak, "traffic": traffic_for(dom, args.n_seqs),
        "peak_basis": peak_basis, "frac_of_nominal": achieved / nominal,
        "launch_ms": per_launch[dom],
    }
    phases = {}
    for name, n_units in (("forward", units), ("viterbi_scores", units), ("viterbi_paths", sumT),
                          ("adjoint", sumT)):
        if per_launch.get(name):
            phases[name] = {"ms": per_launch[name],
                            "obs_models_per_s": n_units / (per_launch[name] / 1e3),
                            "tflops": flops[name] / (per_launch[name] / 1e3) / 1e12}
    for name in ("setup", "count_reduce", "softmax_rows", "softmax_grad", "adam"):
        phases[name] = {"ms": totals[name] / max(args.steps, 1)}

    # ---- end to end through the public API ---------------------------------
    e2e = None
    if not args.skip_e2e:
        h_sym = torch.from_numpy(w.symbols).pin_memory()
        h_off = torch.from_numpy(w.offsets).pin_memory()
        h_len = torch.from_numpy(w.lengths).pin_memory()
        h_lab = torch.from_numpy(w.labels).pin_memory()
        d_sym, d_off = torch.empty_like(seqs.symbols), torch.empty_like(seqs.offsets)
        d_len, d_lab = torch.empty_like(seqs.lengths), torch.empty_like(labels)
        sq2 = hmm.Sequences(d_sym, d_off, d_len, seqs.max_len)
        lb2 = sq2.labelled(d_lab)
        o_am = torch.empty(w.S, dtype=torch.int32).pin_memory()
        o_path = torch.empty(max(w.total_obs, 1), dtype=torch.int32).pin_memory()
        o_nll = torch.empty(1, dtype=torch.float32).pin_memory()
        bi = sum(t.numel() * t.element_size() for t in (h_sym, h_off, h_len, h_lab))
        bo = sum(t.numel() * t.element_size() for t in (o_am, o_path, o_nll))
        times = []
        barrier()
        for i in range(max(args.warmup, 3) + args.steps):
            flush.fill_(i & 0xff)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_sym.copy_(h_sym, non_blocking=True)
            d_off.copy_(h_off, non_blocking=True)
            d_len.copy_(h_len, non_blocking=True)
            d_lab.copy_(h_lab, non_blocking=True)
            step(sq2, lb2, copy_out=(o_am, o_path))
            o_nll.copy_(fll.sum().neg().view(1), non_blocking=True)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        barrier()
        times = times[max(args.warmup, 3):]   # the first iterations load lazy kernels
        e_ms = float(np.mean(times)) * 1e3
        t_e = torch.tensor([e_ms], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
        e2e = {"value": units * world / (float(t_e.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "ms_per_step": float(t_e.item())}

    # ---- CPU oracle baseline (rank 0, N = 1 only) --------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cores = os.cpu_count() or 1
        idx = np.arange(w.S)
        t0 = time.perf_counter()
        oracle_step(w, idx, cores)
        dt = time.perf_counter() - t0
        cpu = {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the whole batch ({w.S} sequences, {units} obs*models), one step: "
                         "FP64 log-space forward+Viterbi over all K models, labelled "
                         "forward-backward counts and logit gradient",
               "seconds": dt}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batched-recognition K={K} N={N} M={M} S={w.S} "
                                   "T~U{30..300} (all K models per sequence + labelled adjoint)",
                       "units_per_step": units, "sum_T": sumT,
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "timing": "CUDA-graph replay of the whole step" if graph is not None
                       else "eager step", "parallelism": f"replicas x{world}",
                       "tuning": {k: v["lanes"] for k, v in tuning.items()}},
            "autotune_ms": {k: v["ms"] for k, v in tuning.items()},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": (KERNELS_PER_STEP + (1 if hmm.hmm_get_tuning(
                hmm.HMM_TUNE_FB_RANGES, tune.n_pad(N)) > 1 else 0)) * args.steps,
            "clocks": clk,
            "phases": phases,
            "kernel_ms_per_step": step_kernel_ms,
        }
        if emit:
            print(json.dumps(line), flush=True)
        return line
    return None


def measured_peak_bf16():
    """Dense BF16 TFLOP/s measured on this machine (burst), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def plan_launches(K: int, labelled: bool) -> int:
    """Kernel launches of the tensor-core adjoint's tile plan: row compaction
    (count, scan, place), 3 launches per 8-bit radix pass over (model,
    length) keys (an even number of passes), the tile stage and the work
    lists of its two kernels."""
    bits = 10
    if labelled:
        while bits < 32 and ((K - 1) >> (bits - 10)) != 0:
            bits += 1
    passes = (bits + 7) // 8
    passes += passes & 1
    return 3 + 3 * passes + 2


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def fma_peak(torch, dev):
    """Measured FP32 FMA throughput (TFLOP/s) from the library's probe kernel:
    best of 5 launches per mode (scalar FFMA, packed FFMA2), CUDA events."""
    from paper_1310_3322_gb300 import hmm
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = sms * 4, 256, 20000
    out = torch.empty(blocks, device=dev)
    res = {}
    for mode, name in ((0, "ffma"), (1, "ffma2")):
        hmm.hmm_fma_probe(blocks, threads, 100, mode, out)
        best = float("inf")
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fl = hmm.hmm_fma_probe(blocks, threads, iters, mode, out)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        res[name] = fl / (best / 1e3) / 1e12
    assert bool(torch.isfinite(out).all())
    return max(res.values()), res


def fp32_peak(torch, dev):
    """The FP32 roofline denominator of the SIMT kernels: the measured FFMA
    rate (fma_peak) with its basis, and the nominal SMs x 128 lanes x 2 flop x
    maximum clock beside it."""
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal = sm_count * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    measured, modes = fma_peak(torch, dev)
    basis = (f"measured: hmm_fma_probe, best of scalar FFMA {modes['ffma']:.1f} and packed "
             f"FFMA2 {modes['ffma2']:.1f} TFLOP/s (nominal {sm_count} SMs x 128 lanes x 2 flop x "
             f"{SM_MAX_MHZ:.0f} MHz = {nominal:.1f})")
    return measured, basis, nominal


def tf32_peak(torch, dev):
    """Dense TF32 GEMM throughput (TFLOP/s): torch.matmul of 8192^3 FP32
    operands with TF32 tensor cores allowed, best of 5 (the TF32 forward's
    roofline denominator, measured as the BF16 one was)."""
    n = 8192
    a = torch.randn(n, n, device=dev)
    b = torch.randn(n, n, device=dev)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        torch.matmul(a, b)
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def large_sample(w, n, longest, seed):
    """n sequences of the batch: its `longest` longest and a seeded draw."""
    order = np.argsort(-w.lengths, kind="stable")
    rest = np.random.default_rng(seed).choice(order[longest:], size=n - longest, replace=False)
    return np.sort(np.concatenate([order[:longest], rest]))


def oracle_large_step(w, idx, nthreads):
    """The large step's arithmetic on the FP64 CPU oracle for sequences idx:
    forward of every model (the argmax is its by-product) and the labelled
    forward-backward counts."""
    import oracle
    P = oracle.params(w.pi, w.A, w.B)
    sub = (w.symbols, w.offsets[idx], w.lengths[idx])
    oracle.forward(P, *sub, nthreads=nthreads)
    oracle.forward_backward(P, *sub, w.labels[idx], nthreads=nthreads)


def error_stats(ll, ref, lengths):
    """max and mean |delta log P| / T over the compared pairs."""
    T = np.maximum(np.asarray(lengths, np.float64), 1.0)
    if ll.ndim == 2:
        T = T[:, None]
    e = np.abs(np.asarray(ll, np.float64) - ref) / T
    return {"max_abs_per_obs": float(e.max()), "mean_abs_per_obs": float(e.mean())}


def run_large(args, emit=True):
    """The large-state configuration (K=4, N=128, M=256, 16384 sequences,
    T ~ U{100..2000}) on the tensor cores. One step = the BF16 forward of
    every sequence against all K models with the argmax (recognition) and the
    BF16 forward-backward adjoint of every sequence against its labelled model
    (the E-step's expected counts, i.e. the log-likelihood gradient); units =
    sum_s T_s (K + 1). The TF32 forward and the Viterbi decoding of the same
    batch are timed beside it, with the error of each precision against the
    FP64 oracle on a sample."""
    import torch
    import torch.distributed as dist
    from paper_1310_3322_gb300 import hmm, synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.make_workload("large", n_seqs=args.n_seqs, seed=synth.SEEDS["large"] + rank)
    K, N, M = w.K, w.N, w.M
    sumT = int(w.lengths.astype(np.int64).sum())
    units = sumT * (K + 1)
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device=dev)
    labels = torch.from_numpy(w.labels).to(dev)
    lab = seqs.labelled(labels)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    ll = torch.empty((w.S, K), device=dev)
    am = torch.empty(w.S, dtype=torch.int32, device=dev)
    fll = torch.empty(w.S, device=dev)
    cnts = [torch.empty(sh, device=dev) for sh in ((K, N), (K, N, N), (K, N, M))]
    ws = [hmm.Workspace(dev), hmm.Workspace(dev)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    prec = hmm.HMM_BF16_MMA
    # the recognition forward runs beside the adjoint on a second stream
    rec = torch.cuda.Stream(device=dev)

    def step(sq=seqs, lb=lab, concurrent=True):
        cur = torch.cuda.current_stream()
        if concurrent:
            rec.wait_stream(cur)
        # the adjoint (the longer chain) is launched first
        hmm.hmm_forward_backward(pi, A, B, lb, precision=prec, loglik=fll, counts=cnts,
                                 workspace=ws[1])
        with torch.cuda.stream(rec if concurrent else cur):
            hmm.hmm_forward(pi, A, B, sq, precision=prec, loglik=ll, argmax=am, workspace=ws[0])
        if concurrent:
            cur.wait_stream(rec)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws[0]) == 0 and hmm.hmm_get_device_status(ws[1]) == 0

    # ---- timed region: CUDA events on the launching stream, L2 flushed ----
    clocks = Clocks(local)
    cur = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(i & 0xff)          # L2 flush, outside the timed events
        evs[i][0].record(cur)
        step()
        evs[i][1].record(cur)
    barrier()
    clk = clocks.stop()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    t_max = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms_max = float(t_max.item())
    value = units * world / (ms_max / 1e3)
    ll_bf16 = ll.cpu().numpy()
    am_bf16 = am.cpu().numpy()
    fll_bf16 = fll.cpu().numpy()

    # ---- per-kernel times: each launch timed alone (serialised eager step)
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, lambda: step(concurrent=False), args.steps, flush)
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    kms = {k: v[1] / max(v[0], 1) for k, v in kt.items() if v[0]}
    # the adjoint is two kernels: the forward/backward passes and the segment
    # ranges; its algorithmic work is counted against the pair
    kms["adjoint_ranges"] = kms["adjoint"]
    kms["adjoint"] = kms["adjoint_ranges"] + kms.get("adjoint_pass", 0.0)
    # forward: setup + kernel; adjoint: setup (validation only), plan, the two
    # kernels, two-level count reduction
    launches_per_step = (setup_launches(w.S) + 1) + (setup_launches(w.S, ordered=False)
                                                     + plan_launches(K, True) + 2 + 2)

    if args.quick:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_max,
                "config": {"workload": f"large K={K} N={N} M={M} S={w.S} (quick)"},
                "kernel_ms": kms, "clocks": clk, "gpu_launches": launches_per_step * args.steps}
        if emit and rank == 0:
            print(json.dumps(line), flush=True)
        return line

    # ---- the TF32 forward on the same data ----------------------------------
    ll32 = torch.empty_like(ll)

    def fwd_tf32():
        hmm.hmm_forward(pi, A, B, seqs, precision=hmm.HMM_TF32_MMA, loglik=ll32, argmax=am,
                        workspace=ws[0])
    fwd_tf32()
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, fwd_tf32, args.steps, flush)
    kt32 = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    tf32_ms = kt32["forward"][1] / max(kt32["forward"][0], 1)
    ll_tf32 = ll32.cpu().numpy()

    # ---- the TF32 adjoint on the same data (every step's rows kept) ---------
    fll32 = torch.empty_like(fll)
    cnts32 = [torch.empty_like(c) for c in cnts]
    ws32 = hmm.Workspace(dev)

    def adj_tf32():
        hmm.hmm_forward_backward(pi, A, B, lab, precision=hmm.HMM_TF32_MMA, loglik=fll32,
                                 counts=cnts32, workspace=ws32)
    adj_tf32()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws32) == 0
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, adj_tf32, max(2, args.steps // 2), flush)
    kta = {k2: v[1] / v[0] for k2, v in hmm.hmm_timing_read().items() if v[0]}
    hmm.hmm_timing_enable(False)
    fll_tf32 = fll32.cpu().numpy()
    cnt_diff = [float(torch.linalg.vector_norm(a32 - a16) / torch.linalg.vector_norm(a16))
                for a32, a16 in zip(cnts32, cnts)]
    ws32 = None
    torch.cuda.empty_cache()

    # ---- Viterbi of every sequence against all K models (FP32 SIMT) --------
    vsc = torch.empty((w.S, K), device=dev)
    vbest = torch.empty(w.S, dtype=torch.int32, device=dev)
    vpath = torch.empty(max(w.total_obs, 1), dtype=torch.int32, device=dev)

    def vit():
        hmm.hmm_viterbi(pi, A, B, seqs, score=vsc, best_model=vbest, path=vpath,
                        workspace=ws[0])
    vit()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws[0]) == 0
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    vit_ms = _time_steps(torch, vit, 2, flush)
    ktv = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    vkms = {k2: v[1] / v[0] for k2, v in ktv.items() if v[0]}

    # ---- peaks: measured BF16 (pool file), FP32 FMA probe, TF32 GEMM -------
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_nominal = sm_count * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fp32_peak, fp32_modes = fma_peak(torch, dev)
    tf32_tflops = tf32_peak(torch, dev)
    peak, basis = measured_peak_bf16()
    vs_tf = 2.0 * N * N * sumT * K / (vkms["viterbi_scores"] / 1e3) / 1e12
    f_tf = 2.0 * N * N * sumT * K / (kms["forward"] / 1e3) / 1e12
    f32_tf = 2.0 * N * N * sumT * K / (tf32_ms / 1e3) / 1e12
    a_flop = (8.0 * N * N + 10 * N) * sumT
    a_tf = a_flop / (kms["adjoint"] / 1e3) / 1e12
    tf32_adj_ms = kta.get("adjoint_pass", 0.0) + kta.get("adjoint", 0.0)
    dom = "adjoint" if kms["adjoint"] >= kms["forward"] else "forward"
    achieved = a_tf if dom == "adjoint" else f_tf

    # ---- error of each precision against the FP64 oracle (a sample) --------
    import oracle
    cores = os.cpu_count() or 1
    eidx = large_sample(w, min(32, w.S), min(8, w.S), 21)
    P = oracle.params(w.pi, w.A, w.B)
    ref, ref_am, _ = oracle.forward(P, w.symbols, w.offsets[eidx], w.lengths[eidx],
                                    nthreads=cores)
    lab_ref = ref[np.arange(eidx.size), w.labels[eidx]]
    err = {"sample": f"{eidx.size} sequences (the {min(8, w.S)} longest and a seeded draw), "
                     f"all {K} models, FP64 oracle",
           "bf16_forward": error_stats(ll_bf16[eidx], ref, w.lengths[eidx]),
           "tf32_forward": error_stats(ll_tf32[eidx], ref, w.lengths[eidx]),
           "bf16_adjoint_loglik": error_stats(fll_bf16[eidx], lab_ref, w.lengths[eidx]),
           "tf32_adjoint_loglik": error_stats(fll_tf32[eidx], lab_ref, w.lengths[eidx]),
           "adjoint_counts_rel_l2_tf32_vs_bf16": cnt_diff,
           "argmax_agreement_bf16": float(np.mean(am_bf16[eidx] == ref_am))}

    # ---- end to end through the public API (host buffers) ------------------
    e2e = None
    if not args.skip_e2e:
        h_in = [torch.from_numpy(x).pin_memory() for x in (w.symbols, w.offsets, w.lengths,
                                                            w.labels)]
        d_in = [torch.empty_like(x, device=dev) for x in h_in]
        sq2 = hmm.Sequences(d_in[0], d_in[1], d_in[2], seqs.max_len)
        lb2 = sq2.labelled(d_in[3])
        outs = [ll, am, fll] + cnts
        h_out = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in outs]
        bi = sum(t.numel() * t.element_size() for t in h_in)
        bo = sum(t.numel() * t.element_size() for t in h_out)
        times = []
        barrier()
        for i in range(max(args.warmup, 3) + args.steps):
            flush.fill_(i & 0xff)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for d, h in zip(d_in, h_in):
                d.copy_(h, non_blocking=True)
            step(sq2, lb2)
            for h, d in zip(h_out, outs):
                h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        barrier()
        e_ms = float(np.mean(times[max(args.warmup, 3):])) * 1e3
        t_e = torch.tensor([e_ms], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
        e2e = {"value": units * world / (float(t_e.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "ms_per_step": float(t_e.item()),
               "copies": "H2D symbols, offsets, lengths, labels (pinned); D2H log-likelihoods "
                         "[S][K], argmax [S], labelled log-likelihoods [S], counts"}

    # ---- CPU oracle baseline (rank 0, N = 1): a sample, extrapolated -------
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cidx = large_sample(w, min(48, w.S), min(4, w.S), 22)
        c_units = int(w.lengths[cidx].astype(np.int64).sum()) * (K + 1)
        t0 = time.perf_counter()
        oracle_large_step(w, cidx, cores)
        dt = time.perf_counter() - t0
        c1idx = large_sample(w, min(4, w.S), 0, 23)
        c1_units = int(w.lengths[c1idx].astype(np.int64).sum()) * (K + 1)
        t0 = time.perf_counter()
        oracle_large_step(w, c1idx, 1)
        dt1 = time.perf_counter() - t0
        cpu = {"value": c_units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cidx.size} of {w.S} sequences ({c_units} obs*models): FP64 "
                         f"log-space forward over all {K} models + labelled forward-backward "
                         f"counts, {cores} threads, {dt:.1f} s; the full step extrapolated "
                         "linearly in sum T*K*N^2",
               "full_step_seconds_extrapolated": dt * units / c_units,
               "value_1thread": c1_units / dt1,
               "sample_1thread": f"{c1idx.size} sequences ({c1_units} obs*models), 1 thread, "
                                 f"{dt1:.1f} s",
               "cpu_model": cpu_model()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"large K={K} N={N} M={M} S={w.S} T~U{{100..2000}} "
                               "(BF16 forward of all K models + argmax, and the BF16 "
                               "forward-backward adjoint against the labelled model)",
                   "precision": "BF16 tensor-core operands (tcgen05 kind::f16), FP32 "
                                "accumulation, FP64 final log",
                   "units_per_step": units, "sum_T": sumT,
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "timing": "eager step (adjoint and forward on two streams), CUDA events; "
                             "per-kernel times from an eager pass with the kernels "
                             "serialised", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "tensor", "kernel": dom + "_mma", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "launch_ms": kms[dom], "peak_basis": f"dense BF16, {basis} (burst)",
                     "algorithmic": "adjoint 8N^2+10N flop per obs (forward, recompute, "
                                    "backward, xi) over its two launches (passes + segment "
                                    "ranges); forward 2N^2 per obs*model",
                     "traffic": traffic_for("adjoint_mma" if dom == "adjoint" else
                                            "forward_mma", args.n_seqs)},
        "error_vs_oracle": err,
        "phases": {"forward": {"ms": kms["forward"], "tflops": f_tf, "frac_bf16": f_tf / peak,
                               "obs_models_per_s": sumT * K / (kms["forward"] / 1e3)},
                   "adjoint": {"ms": kms["adjoint"], "tflops": a_tf, "frac_bf16": a_tf / peak,
                               "obs_per_s": sumT / (kms["adjoint"] / 1e3),
                               "pass_ms": kms.get("adjoint_pass"),
                               "ranges_ms": kms["adjoint_ranges"]},
                   "forward_tf32": {"ms": tf32_ms, "tflops": f32_tf,
                                    "frac_tf32": f32_tf / tf32_tflops,
                                    "obs_models_per_s": sumT * K / (tf32_ms / 1e3)},
                   "adjoint_tf32": {"ms": tf32_adj_ms, "pass_ms": kta.get("adjoint_pass", 0.0),
                                    "counts_ms": kta.get("adjoint", 0.0),
                                    "setup_plan_ms": kta.get("setup", 0.0),
                                    "tflops": a_flop / (tf32_adj_ms / 1e3) / 1e12,
                                    "frac_tf32": a_flop / (tf32_adj_ms / 1e3) / 1e12 / tf32_tflops,
                                    "obs_per_s": sumT / (tf32_adj_ms / 1e3),
                                    "note": "forward and backward passes (TF32 tcgen05) keeping "
                                            "every step's rows, then gamma / xi (TF32 "
                                            "contraction) / emission counts from the rows"},
                   "viterbi": {"ms": vit_ms, "kernel_ms": vkms,
                               "obs_models_per_s": sumT * K / (vit_ms / 1e3),
                               "scores_tflops": vs_tf, "scores_frac_fp32": vs_tf / fp32_peak,
                               "note": "FP32 SIMT max-plus (2N^2 ops per obs*model), all K "
                                       "models + decoded model + best path"},
                   **{k: {"ms": v} for k, v in kms.items()
                      if k not in ("forward", "adjoint", "adjoint_pass", "adjoint_ranges")}},
        "peaks": {"bf16_tflops": peak, "bf16_basis": basis, "tf32_tflops_measured": tf32_tflops,
                  "fp32_tflops_measured": fp32_peak, "fp32_probe": fp32_modes,
                  "fp32_tflops_nominal_max_clock": fp32_nominal},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
    }
    if emit and rank == 0:
        print(json.dumps(line), flush=True)
    return line


def _time_steps(torch, step, steps, flush):
    """Mean ms of `steps` calls of step() with an L2 flush before each."""
    evs = []
    for i in range(steps):
        flush.fill_(i & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([x.elapsed_time(y) for x, y in evs]))


def run_learning(args, emit=True):
    """One learning step on the gradient / training configurations: softmax
    rows -> forward + adjoint of every sequence against its labelled model ->
    logit gradient -> Adam, captured in a CUDA graph; units = sum_s T_s. The
    plain all-models forward kernels on the same data are reported beside it."""
    import torch
    from paper_1310_3322_gb300 import hmm, synth, tune

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.make_workload(args.workload, n_seqs=args.n_seqs,
                            seed=synth.SEEDS[args.workload] + rank)
    K, N, M = w.K, w.N, w.M
    # the library's choice: FP32 SIMT adjoint up to N = 32, tensor cores above
    mma = N > 32
    prec = hmm.HMM_AUTO
    sumT = int(w.lengths.astype(np.int64).sum())
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device=dev)
    lab = seqs.labelled(torch.from_numpy(w.labels).to(dev))
    sizes = [K * N, K * N * N, K * N * M]
    shapes = [(K, N), (K, N, N), (K, N, M)]
    logits = torch.from_numpy(np.concatenate([x.ravel() for x in w.logits]).astype(np.float32)).to(dev)
    grads = torch.zeros_like(logits)
    m_, v_ = torch.zeros_like(logits), torch.zeros_like(logits)
    counter = torch.zeros(1, dtype=torch.int32, device=dev)

    def views(flat):
        out, o = [], 0
        for n, sh in zip(sizes, shapes):
            out.append(flat[o:o + n].view(*sh))
            o += n
        return out

    lg, gr = views(logits), views(grads)
    probs = [torch.empty(sh, device=dev) for sh in shapes]
    fll = torch.empty(w.S, device=dev)
    cnts = [torch.empty(sh, device=dev) for sh in shapes]
    ws = hmm.Workspace(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        hmm.hmm_softmax_rows(*lg, out=probs)
        hmm.hmm_forward_backward(*probs, lab, precision=prec, loglik=fll, counts=cnts,
                                 workspace=ws)
        hmm.hmm_softmax_grad(*probs, *cnts, out=gr)
        hmm.hmm_adam_step(logits, grads, m_, v_, 1e-3, grad_scale=-1.0 / sumT,
                          step_counter=counter)

    step()
    torch.cuda.synchronize()
    tuning = {} if mma else tune.autotune(*probs, seqs, lab,
                                          ops=[hmm.HMM_OP_FORWARD_BACKWARD, hmm.HMM_TUNE_FB_RANGES],
                                          cache=None)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws) == 0
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms = _time_steps(torch, graph.replay, args.steps, flush)
    clk = clocks.stop()
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, step, args.steps, flush)
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    adj_ms = kt["adjoint"][1] / max(kt["adjoint"][0], 1)
    if kt.get("adjoint_pass", (0, 0.0))[0]:  # tensor cores: passes + segment ranges
        adj_ms += kt["adjoint_pass"][1] / kt["adjoint_pass"][0]
    flops = (8 * N * N + 10 * N) * sumT
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    if mma:
        peak, basis = measured_peak_bf16()
        peak_basis = f"dense BF16, {basis} (burst)"
    else:
        peak, peak_basis, _ = fp32_peak(torch, dev)
    achieved = flops / (adj_ms / 1e3) / 1e12

    # the plain per-sequence forward kernels on the same data (all K models)
    fwd = {}
    ll = torch.empty((w.S, K), device=dev)
    am = torch.empty(w.S, dtype=torch.int32, device=dev)
    for name, prec in (("fp32_simt", hmm.HMM_FP32), ("bf16_mma", hmm.HMM_BF16_MMA)):
        if N > hmm.hmm_max_states(hmm.HMM_OP_FORWARD, prec) or (prec == hmm.HMM_BF16_MMA and N <= 32):
            continue
        def fstep(prec=prec):
            hmm.hmm_forward(*probs, seqs, precision=prec, loglik=ll, argmax=am, workspace=ws)
        fstep()
        fms = _time_steps(torch, fstep, args.steps, flush)
        fwd[name] = {"ms": fms, "obs_models_per_s": sumT * K / (fms / 1e3),
                     "tflops": 2.0 * N * N * sumT * K / (fms / 1e3) / 1e12}
    # Baum-Welch re-estimation (E-step + M-step) on the same data: one
    # iteration captured in a CUDA graph and timed like the learning step, and
    # the library's graph-replayed loop run for a few iterations from the
    # current parameters (the log-likelihood it reports must not fall)
    from paper_1310_3322_gb300 import baum_welch
    bw_p = [x.clone() for x in probs]
    bw_ll = torch.empty(w.S, device=dev)

    def bw_iter():
        hmm.hmm_forward_backward(*bw_p, lab, precision=hmm.HMM_AUTO, loglik=bw_ll, counts=cnts,
                                 workspace=ws)
        hmm.hmm_mstep(*bw_p, *cnts, out=bw_p)

    bw_iter()
    torch.cuda.synchronize()
    bw_graph = torch.cuda.CUDAGraph()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(bw_graph, stream=side):
            bw_iter()
    torch.cuda.current_stream().wait_stream(side)
    bw_ms = _time_steps(torch, bw_graph.replay, args.steps, flush)
    bw_hist = baum_welch.baum_welch(*bw_p, lab, max_iters=6, tol=0.0, chunk=3, workspace=ws)
    assert hmm.hmm_get_device_status(ws) == 0
    bw = {"ms_per_iter": bw_ms, "obs_per_s": sumT / (bw_ms / 1e3),
          "loglik_per_obs_first_last": [bw_hist[0] / sumT, bw_hist[-1] / sumT],
          "timing": "CUDA-graph replay of forward-backward + M-step, L2 flushed"}
    line = {
        "metric": METRIC, "value": sumT / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if mma else "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} K={K} N={N} M={M} S={w.S} (softmax rows, "
                               "forward+adjoint against the labelled model, logit gradient, "
                               "Adam; CUDA graph)", "units_per_step": sumT,
                   "adjoint": "tcgen05 BF16" if mma else "FP32 SIMT",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "tuning": {k: v["lanes"] for k, v in tuning.items()}},
        "roofline": {"bound": "tensor" if mma else "alu", "kernel": "adjoint",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "launch_ms": adj_ms,
                     "peak_basis": peak_basis, "traffic": None},
        "clocks": clk,
        "kernel_ms": {k: v[1] / max(v[0], 1) for k, v in kt.items() if v[0]},
        "forward_all_models": fwd,
        "baum_welch": bw,
        # softmax, setup, (tensor cores: tile plan), adjoint (the SIMT one with
        # segment ranges: two kernels), two-level count reduction, gradient, Adam
        "gpu_launches": (1 + setup_launches(w.S, ordered=not mma)
                         + (plan_launches(K, True) if mma else 0)
                         + (2 if mma or hmm.hmm_get_tuning(hmm.HMM_TUNE_FB_RANGES,
                                                           tune.n_pad(N)) > 1 else 1)
                         + 2 + 1 + 1) * args.steps,
    }
    if emit and rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_teamwork(args):
    """Paper-shaped recognition (Sec. 5.7): four roles with one set of six
    action HMMs each (N = 5, M = 64), many short sequences; one step = for
    every role, the forward of its sequences against its six models with the
    argmax and the Viterbi scores, decoded action and best path, in one CUDA
    graph. ``sets``: one forward and one Viterbi call over all sequences, each
    scored against its role's model set; ``roles``: one call pair per role, the
    four roles on four streams. Units = sum_s T_s * 6."""
    import torch
    from paper_1310_3322_gb300 import hmm, synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.make_workload("teamwork", n_seqs=args.n_seqs, seed=synth.SEEDS["teamwork"] + rank)
    R = w.meta["roles"]
    Kr, N, M = w.K // R, w.N, w.M
    sumT = int(w.lengths.astype(np.int64).sum())
    units = sumT * Kr
    sym = torch.from_numpy(w.symbols).to(dev)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    path = torch.empty(max(w.total_obs, 1), dtype=torch.int32, device=dev)
    roles = []
    for r in (range(R) if args.teamwork_calls == "roles" else []):
        idx = np.nonzero(w.labels // Kr == r)[0]
        sq = hmm.Sequences(symbols=sym, offsets=torch.from_numpy(w.offsets[idx]).to(dev),
                           lengths=torch.from_numpy(w.lengths[idx]).to(dev),
                           max_len=int(w.lengths[idx].max()))
        sl = slice(r * Kr, (r + 1) * Kr)
        roles.append(dict(seqs=sq, p=(pi[sl], A[sl], B[sl]),
                          ll=torch.empty((idx.size, Kr), device=dev),
                          am=torch.empty(idx.size, dtype=torch.int32, device=dev),
                          vs=torch.empty((idx.size, Kr), device=dev),
                          vb=torch.empty(idx.size, dtype=torch.int32, device=dev),
                          ws=(hmm.Workspace(dev), hmm.Workspace(dev)),
                          streams=(torch.cuda.Stream(device=dev),)))
    if args.teamwork_calls == "sets":
        sq = hmm.Sequences(symbols=sym, offsets=torch.from_numpy(w.offsets).to(dev),
                           lengths=torch.from_numpy(w.lengths).to(dev), max_len=w.max_len)
        base = torch.from_numpy((w.labels // Kr * Kr).astype(np.int32)).to(dev)
        roles.append(dict(seqs=sq.model_sets(base, Kr), p=(pi, A, B),
                          ll=torch.empty((w.S, Kr), device=dev),
                          am=torch.empty(w.S, dtype=torch.int32, device=dev),
                          vs=torch.empty((w.S, Kr), device=dev),
                          vb=torch.empty(w.S, dtype=torch.int32, device=dev),
                          ws=(hmm.Workspace(dev), hmm.Workspace(dev)),
                          streams=(torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(serial=False):
        # forward and Viterbi of a role (or of the model-set call) on the
        # role's stream(s): with two, the two ops run side by side; serial =
        # everything on the current stream (per-kernel timing)
        cur = torch.cuda.current_stream()
        for x in roles:
            sf, sv = (cur, cur) if serial else (x["streams"][0], x["streams"][-1])
            for st in x["streams"]:
                st.wait_stream(cur)
            with torch.cuda.stream(sf):
                hmm.hmm_forward(*x["p"], x["seqs"], loglik=x["ll"], argmax=x["am"],
                                workspace=x["ws"][0])
            with torch.cuda.stream(sv):
                hmm.hmm_viterbi(*x["p"], x["seqs"], score=x["vs"], best_model=x["vb"],
                                path=path, workspace=x["ws"][1])
        for x in roles:
            for st in x["streams"]:
                cur.wait_stream(st)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    for x in roles:
        st = hmm.hmm_get_device_status(x["ws"][0]) | hmm.hmm_get_device_status(x["ws"][1])
        if st:
            raise RuntimeError(f"device status {st:#x}")
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms = _time_steps(torch, graph.replay, args.steps, flush)
    clk = clocks.stop()
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, lambda: step(serial=True), args.steps, flush)
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    per_launch = {k: v[1] / v[0] for k, v in kt.items() if v[0]}
    # algorithmic work per launch (one role, or all of them with model sets):
    # 2N^2 + N flop per obs*model (forward: alpha A, emission; Viterbi scores:
    # the same count in max-plus)
    flop_launch = (2.0 * N * N + N) * units / len(roles)
    dom = max(("forward", "viterbi_scores"), key=lambda k: per_launch.get(k, 0.0))
    achieved = flop_launch / (per_launch[dom] / 1e3) / 1e12
    peak, peak_basis, _ = fp32_peak(torch, dev)
    line = {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"teamwork {R} roles x {Kr} actions, N={N} M={M} S={w.S} "
                               "T~U{20..120} (per role: forward of its models + argmax, "
                               "Viterbi scores + decoded action + path; "
                               + ("one call per op over per-role model sets, forward and "
                                  "Viterbi on two streams"
                                  if args.teamwork_calls == "sets" else "one call per role, "
                                  "4 streams") + ", CUDA graph)",
                   "units_per_step": units,
                   "l2": "flushed between steps (256 MB write outside the timed events)"},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "launch_ms": per_launch[dom],
                     "peak_basis": peak_basis, "traffic": None},
        "clocks": clk,
        "kernel_ms_per_launch": per_launch,
        "gpu_launches": sum(v[0] for v in kt.values())
                        + (setup_launches(w.S if args.teamwork_calls == "sets" else w.S // R) - 1)
                        * kt["setup"][0],
    }
    print(json.dumps(line), flush=True)


def run_wide(args):
    """The 512-state x 512-sequence shape Sec. 5.6 quotes for the cited forward
    kernel: the forward of every sequence on the tensor cores (each 128-row
    tile on a cluster of N/64 CTAs, every CTA with its 64-column slice of A
    resident, the rows exchanged through distributed shared memory every
    step); units = sum_s T_s * K."""
    import torch
    from paper_1310_3322_gb300 import hmm, synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.make_workload("cuhmm", n_seqs=args.n_seqs, seed=synth.SEEDS["cuhmm"] + rank)
    K, N, M = w.K, w.N, w.M
    sumT = int(w.lengths.astype(np.int64).sum())
    units = sumT * K
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device=dev)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    ll = torch.empty((w.S, K), device=dev)
    am = torch.empty(w.S, dtype=torch.int32, device=dev)
    ws = hmm.Workspace(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        hmm.hmm_forward(pi, A, B, seqs, precision=hmm.HMM_BF16_MMA, loglik=ll, argmax=am,
                        workspace=ws)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws) == 0
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms = _time_steps(torch, step, args.steps, flush)
    clk = clocks.stop()
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, step, args.steps, flush)
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    kms = {k: v[1] / v[0] for k, v in kt.items() if v[0]}
    achieved = 2.0 * N * N * units / (kms["forward"] / 1e3) / 1e12
    peak, basis = measured_peak_bf16()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    cl = 4 if N <= 256 else 8  # CTAs per cluster: N_pad / 64
    # rows per tile: the fewest of 32, 64, 128 whose clusters fit one wave
    rows = next((r for r in (32, 64) if -(-w.S // r) * K * cl <= sm_count), 128)
    busy = min(-(-w.S // rows) * K * cl, sm_count)
    # one Baum-Welch iteration of the same shape (Sec. 5.6 quotes forward and
    # Baum-Welch): tensor-core forward + backward passes keeping their rows,
    # count contraction, M-step (in place on copies of the parameters)
    bw_pi, bw_A, bw_B = pi.clone(), A.clone(), B.clone()
    cnt = (torch.empty_like(pi), torch.empty_like(A), torch.empty_like(B))
    bll = torch.empty((w.S, K), device=dev)
    wsb = hmm.Workspace(dev)

    def bw_step():
        hmm.hmm_forward_backward(bw_pi, bw_A, bw_B, seqs, precision=hmm.HMM_BF16_MMA, loglik=bll,
                                 counts=cnt, workspace=wsb)
        hmm.hmm_mstep(bw_pi, bw_A, bw_B, *cnt, out=(bw_pi, bw_A, bw_B))

    bw_step()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(wsb) == 0
    ll0 = float(bll.sum())
    bw_ms = _time_steps(torch, bw_step, max(2, args.steps // 2), flush)
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, bw_step, 2, flush)
    bkt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    bkms = {k2: v[1] / v[0] for k2, v in bkt.items() if v[0]}
    ll1 = float(bll.sum())
    line = {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"cuhmm K={K} N={N} M={M} S={w.S} T~U{{100..500}} (forward of "
                               "every sequence, tcgen05 BF16, one cluster of "
                               f"{cl} CTAs per {rows}-row tile)",
                   "units_per_step": units, "tiles": -(-w.S // rows) * K,
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "timing": "eager step, CUDA events"},
        "roofline": {"bound": "tensor", "kernel": "forward_cluster", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "launch_ms": kms["forward"], "peak_basis": f"dense BF16, {basis} (burst)",
                     "busy_sms": busy,
                     "frac_of_busy_sms": achieved / (peak * busy / sm_count),
                     "traffic": traffic_for("forward_cluster", args.n_seqs)},
        "kernel_ms": kms,
        "baum_welch": {"ms_per_iteration": bw_ms, "value": units / (bw_ms / 1e3), "unit": UNIT,
                       "kernel_ms": bkms, "loglik_sum_first_last": [ll0, ll1],
                       "note": "forward + backward passes (BF16 tcgen05) keeping per-step "
                               "rows, count contraction, M-step"},
        "clocks": clk,
        "gpu_launches": 2 * args.steps,  # setup, forward
    }
    print(json.dumps(line), flush=True)


def run_longseq(args):
    """Few very long sequences (8 x T ~ U{2^19..2^20}, K=4, N=32): every
    sequence against every model by the parallel-in-time forward (chunk
    products, then the ordered per-pair combine), with the sequential FP32
    forward on the same batch timed beside it. Units = sum_s T_s * K."""
    import torch
    from paper_1310_3322_gb300 import hmm, synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.make_workload("longseq", n_seqs=args.n_seqs, seed=synth.SEEDS["longseq"] + rank)
    K, N, M = w.K, w.N, w.M
    NP = 1 << max(2, (N - 1).bit_length())
    sumT = int(w.lengths.astype(np.int64).sum())
    units = sumT * K
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device=dev)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    ll = torch.empty((w.S, K), device=dev)
    am = torch.empty(w.S, dtype=torch.int32, device=dev)
    ws = hmm.Workspace(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        hmm.hmm_forward_scan(pi, A, B, seqs, chunk=args.scan_chunk, loglik=ll, argmax=am,
                             workspace=ws)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws) == 0
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms = _time_steps(torch, step, args.steps, flush)
    clk = clocks.stop()
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    _time_steps(torch, step, args.steps, flush)
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    kms = {k: v[1] / v[0] for k, v in kt.items() if v[0]}
    # the sequential recursion on the same batch (one chain of T steps per pair)
    sl = torch.empty_like(ll)
    hmm.hmm_forward(pi, A, B, seqs, loglik=sl, argmax=am, workspace=ws)
    torch.cuda.synchronize()
    seq_ms = _time_steps(torch, lambda: hmm.hmm_forward(pi, A, B, seqs, loglik=sl, argmax=am,
                                                        workspace=ws), 2, flush)
    diff = float((ll - sl).abs().max())
    # chunk products: 2 NP^3 flop per step and pair (row i of a product is the
    # recursion started from state i); the sequential recursion does 2 N^2
    steps = int((np.maximum(w.lengths.astype(np.int64), 1) - 1).sum()) * K
    achieved = 2.0 * NP ** 3 * steps / (kms["scan_chunks"] / 1e3) / 1e12
    peak, peak_basis, _ = fp32_peak(torch, dev)
    L = args.scan_chunk or min(65536, -(-int(np.ceil(np.sqrt(2.0 * w.max_len))) // 16) * 16)
    line = {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"longseq K={K} N={N} M={M} S={w.S} T~U{{2^19..2^20}} "
                               f"(parallel-in-time forward, {L} steps per chunk, every "
                               "sequence against every model + argmax)",
                   "units_per_step": units, "chunk": L,
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "timing": "eager step, CUDA events"},
        "roofline": {"bound": "alu", "kernel": "scan_chunks", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "launch_ms": kms["scan_chunks"],
                     "peak_basis": peak_basis, "traffic": None},
        "kernel_ms": kms,
        "sequential_forward": {"ms": seq_ms, "value": units / (seq_ms / 1e3),
                               "max_abs_diff_nats": diff},
        "clocks": clk,
        "gpu_launches": 3 * args.steps,  # setup, chunk products, combine
    }
    print(json.dumps(line), flush=True)


def summary(line):
    """The headline numbers of another configuration's line."""
    if not line:
        return None
    keep = ("metric", "value", "unit", "ms_per_step", "dtype")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line["config"]["workload"]
    r = line.get("roofline") or {}
    out["roofline"] = {k: r.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit",
                                             "frac", "launch_ms")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__
    __graft_entry__.build()
    rank, local, world = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        dispatch(args, rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def dispatch(args, rank):
    if args.workload == "large":
        line = run_large(args, emit=False)
        if not args.skip_others and not args.quick and args.n_seqs is None:
            # the batched-recognition and training configurations, shortly:
            # their headline numbers beside the large one (own full lines with
            # --workload batched / training)
            import copy
            import torch
            others = {}
            for name, fn in (("batched", run_gpu), ("training", run_learning)):
                a2 = copy.copy(args)
                a2.workload, a2.steps, a2.skip_cpu, a2.skip_e2e = name, min(args.steps, 10), True, True
                torch.cuda.empty_cache()
                others[name] = summary(fn(a2, emit=False))
            line["other_configs"] = others
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload in ("gradient", "training"):
        run_learning(args)
        return
    if args.workload == "teamwork":
        run_teamwork(args)
        return
    if args.workload == "cuhmm":
        run_wide(args)
        return
    if args.workload == "longseq":
        run_longseq(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
