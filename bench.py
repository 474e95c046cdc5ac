"""Throughput of the block-matching step on one GB300 (or N, one rank per GPU).

Workload (default): a 31 x 31 grid of 256 x 256 windows at stride 128 on a pair
of 4096 x 4096 uint8 EM-like sections (the second warped by a small random
affine plus a smooth displacement field), whitening exponent 0.65, Hann taper,
SNR exclusion radius 3 px: 961 window pairs per step.  Synthetic stand-ins for
the paper's ssEM sections (generated by ``synth``).

Timing: W warm-up steps, then K timed steps; L2 is flushed (256 MiB write)
before every timed step, outside the CUDA events that time the step itself.
Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (the reference arm; there is no upstream code).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "match windows/sec (256² whitened FFT correlations) & % roofline vs plain FP32"
N_WIN = 256
STRIDE = 128
SECTION = 4096
W_EXP = 0.65
RADIUS = 3.0
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def flops_per_pair(n: int) -> float:
    """Algorithmic FP32 work of one window pair: three real 2D FFTs counted as
    2.5 * M * log2(M) each (M = n^2 points; 5 M log2 M per complex transform,
    half for real data) plus ~30 flops per pixel for taper, mean, whitening
    (two transcendental ops per bin) and the reductions."""
    m = n * n
    return 7.5 * m * math.log2(m) + 30.0 * m


def fp32_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def workload_description():
    return (f"{(SECTION - N_WIN) // STRIDE + 1}x{(SECTION - N_WIN) // STRIDE + 1} grid of {N_WIN}x{N_WIN} "
            f"windows (stride {STRIDE}) on a {SECTION}x{SECTION} uint8 EM-like section pair")


def make_inputs(pairs: int = 1):
    import synth
    secs = []
    for p in range(pairs):
        a, b = synth.em_section_pair(SECTION, seed_content=0 + 10 * p, seed_warp=1 + 10 * p,
                                     seed_noise=(2 + 10 * p, 3 + 10 * p))
        secs.append((a, b))
    org = synth.grid_origins(SECTION, N_WIN, STRIDE)
    return secs, org


# --------------------------------------------------------------------------- #
# clocks sampled during the timed region
# --------------------------------------------------------------------------- #
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- #
# ncu-derived traffic for the dominant kernel (valid only for unchanged sources)
# --------------------------------------------------------------------------- #
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1612_04787_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel_key)
    except (ValueError, OSError):
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- #
# oracle timing on the host cores (reference arm and cpu_baseline)
# --------------------------------------------------------------------------- #
def _oracle_chunk(args):
    mov, ref = args
    from oracle import swim
    lv = swim.Level(N_WIN, W_EXP, swim.APOD_HANN, 1.0, RADIUS)
    return [swim.match_pair(m, r, lv)["status"] for m, r in zip(mov, ref)]


def oracle_throughput(secs, org, sample: int):
    """Windows/s of the FP64 oracle over the first ``sample`` windows, one
    single-threaded worker process per host core (spawned)."""
    a, b = secs[0]
    idx = np.arange(min(sample, len(org)))
    movs = [b[o[0]:o[0] + N_WIN, o[1]:o[1] + N_WIN].astype(np.float64) for o in org[idx]]
    refs = [a[o[0]:o[0] + N_WIN, o[1]:o[1] + N_WIN].astype(np.float64) for o in org[idx]]
    cores = len(os.sched_getaffinity(0))
    chunks = [(movs[i::cores], refs[i::cores]) for i in range(cores)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_chunk, [([m], [r]) for m, r in zip(movs[:cores], refs[:cores])])  # warm
            t0 = time.perf_counter()
            pool.map(_oracle_chunk, chunks)
            dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return len(idx) / dt, cores, dt


# --------------------------------------------------------------------------- #
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pairs", type=int, default=1, help="section pairs per step (961 windows each)")
    ap.add_argument("--oracle-sample", type=int, default=961)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--windows", type=int, default=0,
                    help="use only the first K windows of the grid (small profiling cases)")
    args = ap.parse_args()
    world, rank, local = dist_setup()

    if args.impl == "reference":
        if rank != 0:
            return
        secs, org = make_inputs(1)
        sample = min(args.oracle_sample, len(org))
        vals = []
        cores = 0
        for _ in range(args.warmup):
            oracle_throughput(secs, org, min(sample, 64))
        for _ in range(args.steps):
            v, cores, _dt = oracle_throughput(secs, org, sample)
            vals.append(v)
        value = statistics.median(vals)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_description(), "windows_per_step": sample},
            "cpu_baseline": {"value": value, "unit": "windows/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {sample} windows of the workload per step"},
            "e2e": {"value": value, "unit": "windows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_1612_04787_gb300 as swift

    secs, org = make_inputs(args.pairs)
    if args.windows > 0:
        org = org[: args.windows]
    B1 = len(org)
    plan = swift.Plan([swift.Level(N_WIN, W_EXP, "hann", 1.0, RADIUS)], dtype="u8", max_windows=B1)
    d_secs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in secs]
    d_org = torch.from_numpy(org).to(dev)
    outs = [torch.empty((B1, 8), dtype=torch.int32, device=dev) for _ in secs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        for (a, b), o in zip(d_secs, outs):
            plan.match(a, b, d_org, d_org, out=o, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    res = swift.decode(outs[0])
    ok_frac = float((res["status"] == 0).mean())

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    durs = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    total_ms = sum(durs)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    windows_per_step = B1 * len(secs)
    value = world * windows_per_step * args.steps / (total_ms / 1e3)
    print(f"[bench] rank {rank}: {args.steps} steps, {total_ms / args.steps:.4f} ms/step, "
          f"{value:.1f} windows/s", file=sys.stderr, flush=True)

    # e2e: pinned host sections -> device, match, results -> host, every step
    h_secs = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in secs]
    h_org = torch.from_numpy(org).pin_memory()
    h_out = [torch.empty((B1, 8), dtype=torch.int32).pin_memory() for _ in secs]
    e2e_steps = max(3, min(args.steps, 50))

    def e2e_step():
        d_o = d_org.copy_(h_org, non_blocking=True)
        for (ha, hb), (da, db), o, ho in zip(h_secs, d_secs, outs, h_out):
            da.copy_(ha, non_blocking=True)
            db.copy_(hb, non_blocking=True)
            plan.match(da, db, d_o, d_o, out=o, stream=stream)
            ho.copy_(o, non_blocking=True)
        torch.cuda.synchronize(dev)

    e2e_step()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * windows_per_step * e2e_steps / e2e_s
    h2d = sum(a.nbytes + b.nbytes for a, b in secs) + org.nbytes
    d2h = windows_per_step * 32

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, dt = oracle_throughput(secs, org, args.oracle_sample)
        cpu = {"value": v, "unit": "windows/s", "cores": cores, "kind": "oracle",
               "sample": f"first {min(args.oracle_sample, B1)} of the {B1} windows, FP64 direct-DFT oracle, "
                         f"one single-threaded process per core ({dt:.1f} s)"}

    kernel_ms = total_ms / (args.steps * len(secs))  # one launch per section pair per step
    achieved = flops_per_pair(N_WIN) * B1 / (kernel_ms / 1e3) / 1e12
    peak = fp32_peak_tflops()
    traffic = recorded_traffic("swim_forward_kernel<256,4,u8>")
    line = {
        "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_description(), "window": N_WIN, "windows_per_step": windows_per_step,
                   "section_pairs_per_step": len(secs), "whiten_exponent": W_EXP, "apod": "hann",
                   "snr_exclusion_radius": RADIUS, "input": "uint8",
                   "l2": "flushed before every timed step (256 MiB write, outside the step's events)",
                   "status_ok_fraction": ok_frac},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "swim_forward_kernel<256,4,u8>",
                     "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (max SM clock), derived",
                     "flops_per_window": flops_per_pair(N_WIN)},
        "e2e": {"value": e2e_value, "unit": "windows/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": args.steps * len(secs),
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
