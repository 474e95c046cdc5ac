"""Throughput of the block-matching step on one GB300 (or N, one rank per GPU).

Default workload (the headline metric): a 31 x 31 grid of 256 x 256 windows at
stride 128 on a pair of 4096 x 4096 uint8 EM-like sections (the second warped
by a small random affine plus a smooth displacement field), whitening exponent
0.65, Hann taper, SNR exclusion radius 3 px: 961 window pairs per step.
Other workloads (``--workload``):

  noise64     the 64 x 64 worked example (blurred noise shifted by (-3, +5)), one pair
  pyramid     the same section pair at 1024^2 / 2048^2 / 4096^2 with 64 / 128 / 256
              windows at stride n/4 (11,163 windows), w = 0.5 / 0.65 / 0.8, schedules
              picked by the autotuner, every step one CUDA-graph replay
  patches128  8192 float32 128 x 128 patch pairs with known subpixel shifts (1 GiB)
  patches256  8192 float32 256 x 256 patch pairs (4 GiB)
  warp        2048 windows of 128 x 128 on a 9-section stack: reference = mean of the
              8 neighbours, moving = resampled under per-window affine warps; a step is
              the forward and the backward of loss = -sum snr * peak
  mir         the rendering step: per-triangle affine fit to the SNR-weighted swim
              correspondences of the headline grid and texture mapping of the 4096^2
              moving section (metric: output pixels/s)
  remod       the model and pyramid steps: Z-averaged model of every section of a
              9-section 4096^2 stack and its 2x / 4x box-mean levels (metric: sections/s)
  align       the registration loop: 8 sections of 1024^2 at known offsets, 3 iterations
              of model / match / fit / render (metric: section-iterations/s)

All inputs are seeded synthetic stand-ins for the paper's ssEM sections
(``synth``).  Timing: W warm-up steps, then K timed steps; L2 is flushed (256 MiB
write) before every timed step, outside the CUDA events that time the step.
Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the host
cores instead (the reference arm: there is no upstream code to run).
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "match windows/sec (256² whitened FFT correlations) & % roofline vs plain FP32"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def flops_per_pair(n: int) -> float:
    """Algorithmic FP32 work of one window pair: three real 2D FFTs counted as
    2.5 * M * log2(M) each (M = n^2; 5 M log2 M per complex transform, half for
    real data) plus ~30 flops per pixel for taper, mean, whitening (two
    transcendental ops per bin) and the reductions."""
    m = n * n
    return 7.5 * m * math.log2(m) + 30.0 * m


def stream_slices(count: int, max_windows: int, lanes: int) -> int:
    """Streaming slices of a level's `count` windows in a plan for
    `max_windows`: one lane takes slices of min(max_windows, 2048); two lanes
    split the level into halves of at least 256 windows (at most the lane's
    slice of min(max_windows, 2048), or half of it when that slice passes
    2 GiB of workspace, which no bench plan does)."""
    work = min(max_windows, 2048)
    if lanes <= 1:
        cap = work
    else:
        cap = min(max(-(-count // lanes), 256), work)
    return -(-count // max(cap, 1))


def kernel_flops(n: int) -> dict:
    """The same work split over the streaming kernels: rows = the row transforms
    of z = m' + i r' (one complex 2D half), cols = the forward column transforms
    plus the inverse columns for kx <= n/2 plus unpack and whitening, irows =
    the paired inverse rows, stats and final = the statistics and reductions."""
    m = n * n
    half = 5.0 * m * math.log2(n)  # n complex FFTs of length n
    return {"stats": 2.5 * m, "rows": half + 5.0 * m, "cols": 1.5 * half + 15.0 * m,
            "irows": 0.5 * half + 5.0 * m, "final": 2.5 * m, "fused": flops_per_pair(n),
            "persistent": flops_per_pair(n)}


def fp32_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def tensor_flops(n: int) -> dict:
    """Executed tensor-core work of the BF16X2 / FP16X2 kernels per window: a
    warp's n-point DFT issues 16 (n = 256) or 6 (n = 128) m16n8k16 products per
    hi/lo term, three terms; rows transform n lines, columns 3 per kx pair
    (n/2 pairs), inverse rows n/2 packed lines."""
    per_dft = 2 * 16 * 8 * 16 * (48 if n == 256 else 18)
    return {"rows": n * per_dft, "cols": (3 * n // 2) * per_dft, "irows": (n // 2) * per_dft,
            "stats": 0.0, "final": 0.0}


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------------------- #
# library comparisons: the same match on cuFFT (torch.fft) and on host FFTs
# --------------------------------------------------------------------------- #
def fft_match_torch(torch, mov, ref, A, w):
    """Apodise, rfft2, C = M conj(R), whitening, irfft2, argmax: the transform
    part of the match with library FFTs (no SNR or subpixel fit)."""
    n = mov.shape[-1]
    sa = A.sum()
    mp = A * (mov - (A * mov).sum((-2, -1), keepdim=True) / sa)
    rp = A * (ref - (A * ref).sum((-2, -1), keepdim=True) / sa)
    c = torch.fft.rfft2(mp) * torch.fft.rfft2(rp).conj()
    mag2 = c.real * c.real + c.imag * c.imag
    g = c * (torch.where(mag2 > 0, mag2.pow(-0.5 * w), torch.zeros_like(mag2)) / (n * n))
    g[:, 0, 0] = 0
    return torch.fft.irfft2(g, s=(n, n)).flatten(1).argmax(1)


def cufft_throughput(torch, W, stream, steps, flush):
    """Windows/s of the library-FFT match (cuFFT through torch.fft), window
    gather included, with the same L2 flush between steps."""
    get = W.torch_windows(torch)
    A = torch.outer(*(2 * [0.5 - 0.5 * torch.cos(2 * math.pi * torch.arange(W.n, device=flush.device,
                                                                         dtype=torch.float32) / W.n)]))
    for _ in range(3):
        for m, r in get():
            fft_match_torch(torch, m, r, A, W.w)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        for m, r in get():
            fft_match_torch(torch, m, r, A, W.w)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    return W.windows / (ms / 1e3), ms


def cpu_fft_throughput(movs, refs, n, w):
    """Windows/s of the same library-FFT match in float32 on the host cores
    (scipy.fft, all cores): the like-for-like counterpart of single-precision
    FFTW on CPU cores."""
    import scipy.fft as sf
    cores = len(os.sched_getaffinity(0))
    a = (0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n) / n)).astype(np.float32)
    A = np.outer(a, a)
    m = np.stack(movs).astype(np.float32)
    r = np.stack(refs).astype(np.float32)

    def run():
        sa = A.sum()
        mp = A * (m - (A * m).sum((1, 2), keepdims=True) / sa)
        rp = A * (r - (A * r).sum((1, 2), keepdims=True) / sa)
        c = sf.rfft2(mp, workers=cores) * np.conj(sf.rfft2(rp, workers=cores))
        mag2 = (c.real * c.real + c.imag * c.imag).astype(np.float32)
        with np.errstate(divide="ignore"):
            g = c * (np.where(mag2 > 0, mag2 ** np.float32(-0.5 * w), 0).astype(np.float32) / (n * n))
        g[:, 0, 0] = 0
        return sf.irfft2(g, s=(n, n), workers=cores).reshape(len(m), -1).argmax(1)

    run()
    t0 = time.perf_counter()
    run()
    dt = time.perf_counter() - t0
    return len(m) / dt, cores, dt


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
        # raw samples: SWIFT_CLOCKS_DIR if set (kept for inspection), else a temporary directory
        d = os.environ.get("SWIFT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"swift_clocks_rank{gpu_index}.csv")

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
def kernel_source_hash(files=None) -> str:
    """SHA-256 (16 hex digits) over the given csrc files (all .cu / .cuh / .h
    files when None), in sorted order."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1612_04787_gb300", "csrc")
    names = files if files is not None else [f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h"))]
    for f in sorted(names):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str, windows_per_launch: int):
    """DRAM bytes per launch from a committed ncu capture, scaled to this
    launch's windows (traffic grows in proportion), or None when a source file
    of that kernel (the record's "sources") changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel_key)
    except (ValueError, OSError):
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash(rec.get("sources")):
        return None
    return rec["dram_bytes_per_window"] * windows_per_launch


# --------------------------------------------------------------------------- #
# oracle timing on the host cores (reference arm and cpu_baseline)
# --------------------------------------------------------------------------- #
def _oracle_chunk(args):
    mov, ref, n, w, r = args
    from oracle import swim
    lv = swim.Level(n, w, swim.APOD_HANN, 1.0, r)
    return [swim.match_pair(m, rr, lv)["status"] for m, rr in zip(mov, ref)]


def oracle_throughput(movs, refs, n, w, r):
    """Windows/s of the FP64 oracle over the given windows, one single-threaded
    worker process per host core (spawned)."""
    cores = len(os.sched_getaffinity(0))
    chunks = [(movs[i::cores], refs[i::cores], n, w, r) for i in range(cores)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_chunk, [([m], [rr], n, w, r) for m, rr in zip(movs[:cores], refs[:cores])])
            t0 = time.perf_counter()
            pool.map(_oracle_chunk, chunks)
            dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return len(movs) / dt, cores, dt


# --------------------------------------------------------------------------- #
# workloads
# --------------------------------------------------------------------------- #
class Sections:
    name = "sections"
    dominant_n = 256

    def __init__(self, torch, swift, dev, pairs=1, windows=0, precision="fp32", rank=0, lanes=0, mov_shift=0,
                 row_tma=-1):
        import synth
        self.n, self.w, self.r, self.size, self.stride = 256, 0.65, 3.0, 4096, 128
        # the job is world x pairs section pairs: rank r matches pairs r*pairs .. r*pairs + pairs - 1
        # (its own shard; no collective on the data path)
        first = rank * pairs
        self.secs = [synth.em_section_pair(self.size, seed_content=10 * p, seed_warp=1 + 10 * p,
                                           seed_noise=(2 + 10 * p, 3 + 10 * p)) for p in range(first, first + pairs)]
        org = synth.grid_origins(self.size, self.n, self.stride)
        self.org = org[:windows] if windows > 0 else org
        # moving windows mov_shift px right of the reference windows (left where
        # that would leave the section): rows off 16-byte boundaries
        self.morg = self.org.copy()
        if mov_shift:
            x = self.morg[:, 1]
            self.morg[:, 1] = np.where(x + mov_shift <= self.size - self.n, x + mov_shift, x - mov_shift)
        g = (self.size - self.n) // self.stride + 1
        self.description = (f"{g}x{g} grid of {self.n}x{self.n} windows (stride {self.stride}) on a "
                            f"{self.size}x{self.size} uint8 EM-like section pair")
        if mov_shift:
            self.description += f", moving windows shifted {mov_shift} px in x"
        self.B1 = len(self.org)
        self.windows = self.B1 * pairs
        self.plan = swift.Plan([swift.Level(self.n, self.w, "hann", 1.0, self.r)], dtype="u8",
                               precision=precision, max_windows=self.B1)
        if lanes:
            self.plan.set_lanes(lanes)
        if row_tma >= 0:
            self.plan.set_row_tma(row_tma)
        self.d = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in self.secs]
        self.dorg = torch.from_numpy(self.org).to(dev)
        self.shifted = mov_shift != 0  # else the moving windows use the reference origins' buffers
        self.dmorg = torch.from_numpy(self.morg).to(dev) if self.shifted else self.dorg
        self.outs = [torch.empty((self.B1, 8), dtype=torch.int32, device=dev) for _ in self.secs]
        self.h = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in self.secs]
        self.horg = torch.from_numpy(self.org).pin_memory()
        self.hmorg = torch.from_numpy(self.morg).pin_memory() if self.shifted else self.horg
        self.hout = [torch.empty((self.B1, 8), dtype=torch.int32).pin_memory() for _ in self.secs]
        self.flops = flops_per_pair(self.n) * self.windows
        self.launches_per_step = 3 * self.plan.lanes * len(self.secs)
        self.config = {"window": self.n, "windows_per_step": self.windows, "section_pairs_per_step": pairs,
                       "whiten_exponent": self.w, "apod": "hann", "snr_exclusion_radius": self.r, "input": "uint8",
                       "lanes": self.plan.lanes, "row_tma": self.plan.row_tma}
        if mov_shift:
            self.config["mov_shift_x"] = mov_shift

    def step(self, stream):
        for (a, b), o in zip(self.d, self.outs):
            self.plan.match(a, b, self.dorg, self.dmorg, out=o, stream=stream)

    def e2e_step(self, torch, stream):
        self.dorg.copy_(self.horg, non_blocking=True)
        if self.shifted:
            self.dmorg.copy_(self.hmorg, non_blocking=True)
        for (ha, hb), (da, db), o, ho in zip(self.h, self.d, self.outs, self.hout):
            da.copy_(ha, non_blocking=True)
            db.copy_(hb, non_blocking=True)
            self.plan.match(da, db, self.dorg, self.dmorg, out=o, stream=stream)
            ho.copy_(o, non_blocking=True)
        stream.synchronize()

    def e2e_run(self, torch, stream, steps):
        """Steps through the public API with host buffers, double-buffered: the
        host-to-device copy of step k's sections (a copy stream) overlaps the
        match of step k - 1; every step copies its inputs in and its results
        out.  Returns the seconds from the first copy to the last result."""
        if not hasattr(self, "d2"):
            self.d2 = [(torch.empty_like(a), torch.empty_like(b)) for a, b in self.d]
            self.org2 = torch.empty_like(self.dorg)
            self.morg2 = torch.empty_like(self.dmorg) if self.shifted else self.org2
            self.outs2 = [torch.empty_like(o) for o in self.outs]
            self.copy_stream = torch.cuda.Stream(device=self.dorg.device)
        sets = [(self.d, self.dorg, self.dmorg, self.outs), (self.d2, self.org2, self.morg2, self.outs2)]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            d, org, morg, outs = sets[k % 2]
            if k >= 2:
                self.copy_stream.wait_event(done[k % 2])  # step k - 2 no longer reads these buffers
            with torch.cuda.stream(self.copy_stream):
                org.copy_(self.horg, non_blocking=True)
                if self.shifted:
                    morg.copy_(self.hmorg, non_blocking=True)
                for (ha, hb), (da, db) in zip(self.h, d):
                    da.copy_(ha, non_blocking=True)
                    db.copy_(hb, non_blocking=True)
                copied[k % 2].record(self.copy_stream)
            stream.wait_event(copied[k % 2])
            for (da, db), o, ho in zip(d, outs, self.hout):
                self.plan.match(da, db, org, morg, out=o, stream=stream)
                ho.copy_(o, non_blocking=True)
            done[k % 2].record(stream)
        stream.synchronize()
        return time.perf_counter() - t0

    def io_bytes(self):
        return sum(a.nbytes + b.nbytes for a, b in self.secs) + self.org.nbytes * (2 if self.shifted else 1), self.windows * 32

    def ok_fraction(self, swift):
        return float((swift.decode(self.outs[0])["status"] == 0).mean())

    def torch_windows(self, torch):
        n, st = self.n, self.stride

        def get():
            for a, b in self.d:
                mw = b.unfold(0, n, st).unfold(1, n, st).reshape(-1, n, n)[:self.B1].float()
                rw = a.unfold(0, n, st).unfold(1, n, st).reshape(-1, n, n)[:self.B1].float()
                yield mw, rw
        return get

    def oracle_windows(self, k):
        a, b = self.secs[0]
        n = self.n
        return ([b[y:y + n, x:x + n].astype(np.float64) for y, x in self.morg[:k]],
                [a[y:y + n, x:x + n].astype(np.float64) for y, x in self.org[:k]], n, self.w, self.r)


class Noise64:
    name = "noise64"
    dominant_n = 64

    def __init__(self, torch, swift, dev, **_):
        import synth
        self.n, self.w, self.r = 64, 0.65, 3.0
        ref, mov = synth.noise_pair(64, (-3, 5))
        self.ref, self.mov = ref.astype(np.float32)[None], mov.astype(np.float32)[None]
        self.description = "64x64 worked example: blurred seed-0 noise and its (-3, +5) shift plus noise, one pair"
        self.windows = 1
        self.plan = swift.Plan([swift.Level(64, self.w, "hann", 1.0, self.r)], dtype="f32", max_windows=1)
        self.dr, self.dm = torch.from_numpy(self.ref).to(dev), torch.from_numpy(self.mov).to(dev)
        self.out = torch.empty((1, 8), dtype=torch.int32, device=dev)
        self.hr, self.hm = torch.from_numpy(self.ref).pin_memory(), torch.from_numpy(self.mov).pin_memory()
        self.hout = torch.empty((1, 8), dtype=torch.int32).pin_memory()
        self.flops = flops_per_pair(64)
        self.launches_per_step = 1
        # one call is a single small launch: the device step is the captured
        # call replayed as one graph launch (the host's per-call argument
        # checks and driver launch path stay out of the device time); the
        # e2e figure keeps the plain call with its copies
        self.cap_stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(self.cap_stream):
            self.plan.capture(self.dr, self.dm, out=self.out, stream=self.cap_stream)
        self.cap_stream.synchronize()
        self.config = {"window": 64, "windows_per_step": 1, "whiten_exponent": self.w, "input": "float32",
                       "graph": "one cudaGraphLaunch per step (e2e: the plain call)"}

    def step(self, stream):
        self.plan.replay(stream=stream)

    def e2e_step(self, torch, stream):
        self.dr.copy_(self.hr, non_blocking=True)
        self.dm.copy_(self.hm, non_blocking=True)
        self.plan.match(self.dr, self.dm, out=self.out, stream=stream)
        self.hout.copy_(self.out, non_blocking=True)
        stream.synchronize()

    def io_bytes(self):
        return self.ref.nbytes + self.mov.nbytes, 32

    def ok_fraction(self, swift):
        return float((swift.decode(self.out)["status"] == 0).mean())

    def oracle_windows(self, k):
        # the one pair, k times: a single window would time the worker pool, not the oracle
        self.oracle_note = "copies of the workload's one pair"
        m, r = self.mov[0].astype(np.float64), self.ref[0].astype(np.float64)
        return [m] * k, [r] * k, 64, self.w, self.r


class Pyramid:
    name = "pyramid"
    dominant_n = 256

    def __init__(self, torch, swift, dev, schedule="default", lanes=0, **_):
        import synth
        a, b = synth.em_section_pair(4096)
        self.imgs = [(synth.box_downsample(a, 4), synth.box_downsample(b, 4)),
                     (synth.box_downsample(a, 2), synth.box_downsample(b, 2)), (a, b)]
        self.levels = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8)]
        orgs, lvls = [], []
        for k, ((ia, _), lv) in enumerate(zip(self.imgs, self.levels)):
            o = synth.grid_origins(ia.shape[0], lv.n, lv.n // 4)
            orgs.append(o)
            lvls.append(np.full(len(o), k, np.int32))
        self.org = np.concatenate(orgs).astype(np.int32)  # sorted by level
        self.lvl = np.concatenate(lvls)
        self.offs = [0] + list(np.cumsum([len(o) for o in orgs]))
        self.windows = len(self.org)
        self.description = (f"pyramid of one section pair at 1024^2 / 2048^2 / 4096^2 with 64 / 128 / 256 windows "
                            f"at stride n/4 ({self.windows} windows, sorted by level), w = 0.5 / 0.65 / 0.8, "
                            f"one CUDA-graph replay per step")
        self.plan = swift.Plan(self.levels, dtype="u8", max_windows=self.windows)
        T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)  # noqa: E731
        self.da = [T(x[0]) for x in self.imgs]
        self.db = [T(x[1]) for x in self.imgs]
        self.dorg, self.dlvl = T(self.org), T(self.lvl)
        if schedule == "default":
            self.chosen, _ = self.plan.autotune(self.da, self.db, self.dorg, self.dorg, level=self.dlvl,
                                                level_offsets=self.offs)
        else:  # one schedule for every level, no autotuning
            for l in range(len(self.levels)):
                self.plan.set_schedule(l, schedule)
            self.chosen = [schedule] * len(self.levels)
        if lanes:
            self.plan.set_lanes(lanes)
        self.cap_stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(self.cap_stream):
            self.out = self.plan.capture(self.da, self.db, self.dorg, self.dorg, level=self.dlvl,
                                         stream=self.cap_stream, level_offsets=self.offs)
        self.cap_stream.synchronize()
        self.flops = sum(flops_per_pair(lv.n) * int((self.lvl == k).sum()) for k, lv in enumerate(self.levels))
        # the streaming schedule walks each level's range in slices (three
        # kernels a slice up to 256 x 256: the statistics folded into the rows
        # and the column pairs, the finalize into the inverse rows for
        # exclusion radii below 8 px)
        counts = [self.offs[k + 1] - self.offs[k] for k in range(len(self.levels))]
        self.lanes = self.plan.lanes
        self.launches_per_step = int(sum(1 if c == "fused" else 3 * stream_slices(int(n), self.windows, self.lanes)
                                      for c, n in zip(self.chosen, counts) if c != "persistent")
                                  + (1 if "persistent" in self.chosen else 0))
        self.h = [(torch.from_numpy(x[0]).pin_memory(), torch.from_numpy(x[1]).pin_memory()) for x in self.imgs]
        self.hout = torch.empty((self.windows, 8), dtype=torch.int32).pin_memory()
        self.config = {"windows_per_step": self.windows, "levels": [64, 128, 256],
                       "whiten_exponent": [0.5, 0.65, 0.8], "schedules": self.chosen, "lanes": self.lanes,
                       "input": "uint8", "graph": "one cudaGraphLaunch per step"}

    def step(self, stream):
        self.plan.replay(stream=stream)

    def e2e_step(self, torch, stream):
        for (ha, hb), da, db in zip(self.h, self.da, self.db):
            da.copy_(ha, non_blocking=True)
            db.copy_(hb, non_blocking=True)
        self.plan.replay(stream=stream)
        self.hout.copy_(self.out, non_blocking=True)
        stream.synchronize()

    def io_bytes(self):
        return sum(a.nbytes + b.nbytes for a, b in self.imgs), self.windows * 32

    def ok_fraction(self, swift):
        return float((swift.decode(self.out)["status"] == 0).mean())

    def oracle_windows(self, k):
        movs, refs = [], []
        a, b = self.imgs[2]
        for i in np.nonzero(self.lvl == 2)[0][:k]:
            y, x = self.org[i]
            movs.append(b[y:y + 256, x:x + 256].astype(np.float64))
            refs.append(a[y:y + 256, x:x + 256].astype(np.float64))
        return movs, refs, 256, 0.8, 3.0


class Patches:
    def __init__(self, torch, swift, dev, n=128, count=8192, precision="fp32", lanes=0, **_):
        import synth
        self.name = f"patches{n}"
        self.dominant_n = n
        self.n, self.w, self.r = n, 0.65, 3.0
        a, _ = synth.em_section_pair(4096, seed_content=60, seed_warp=61, seed_noise=(62, 63))
        self.ref, self.mov = self._make(torch, dev, a, n, count, seed=10 if n == 128 else 11)
        self.windows = count
        self.description = (f"{count} float32 {n}x{n} patch pairs cut from an EM-like section; moving = the 2n x 2n "
                            f"tile shifted by U(+-20 px)^2 through a Fourier phase ramp, centre-cropped")
        self.plan = swift.Plan([swift.Level(n, self.w, "hann", 1.0, self.r)], dtype="f32", precision=precision,
                               max_windows=count)
        if lanes:
            self.plan.set_lanes(lanes)
        self.out = torch.empty((count, 8), dtype=torch.int32, device=dev)
        self.flops = flops_per_pair(n) * count
        # used only when no timing events count them: FP32 three kernels a
        # slice, the tensor-core forms five
        slices = stream_slices(count, count, self.plan.lanes)
        self.launches_per_step = (3 if precision == "fp32" else 5) * slices
        self.hout = torch.empty((count, 8), dtype=torch.int32).pin_memory()
        self.config = {"window": n, "windows_per_step": count, "input": "float32", "precision": precision,
                       "whiten_exponent": self.w}

    @staticmethod
    def _make(torch, dev, section, n, count, seed):
        """Reference = centre of a 2n tile; moving = the tile shifted by a known
        subpixel d (phase ramp), centre-cropped (input generation, on the GPU)."""
        rng = np.random.default_rng(seed)
        m = 2 * n
        oy = rng.integers(0, section.shape[0] - m + 1, count)
        ox = rng.integers(0, section.shape[1] - m + 1, count)
        d = rng.uniform(-20.0, 20.0, (count, 2))
        sec = torch.from_numpy(section.astype(np.float32)).to(dev)
        k = torch.fft.fftfreq(m, device=dev, dtype=torch.float64)
        ref = torch.empty((count, n, n), dtype=torch.float32, device=dev)
        mov = torch.empty((count, n, n), dtype=torch.float32, device=dev)
        c0 = n // 2
        for s in range(0, count, 512):
            e = min(count, s + 512)
            tiles = torch.stack([sec[oy[i]:oy[i] + m, ox[i]:ox[i] + m] for i in range(s, e)]).double()
            dd = torch.from_numpy(d[s:e]).to(dev)
            ramp = torch.exp(-2j * math.pi * (k[None, :, None] * dd[:, 0, None, None]
                                               + k[None, None, :] * dd[:, 1, None, None]))
            shifted = torch.fft.ifft2(torch.fft.fft2(tiles) * ramp).real
            ref[s:e] = tiles[:, c0:c0 + n, c0:c0 + n].float()
            mov[s:e] = shifted[:, c0:c0 + n, c0:c0 + n].float()
        return ref.contiguous(), mov.contiguous()

    def step(self, stream):
        self.plan.match(self.ref, self.mov, out=self.out, stream=stream)

    def e2e_step(self, torch, stream):
        if not hasattr(self, "href"):
            self.href, self.hmov = self.ref.cpu().pin_memory(), self.mov.cpu().pin_memory()
        self.ref.copy_(self.href, non_blocking=True)
        self.mov.copy_(self.hmov, non_blocking=True)
        self.plan.match(self.ref, self.mov, out=self.out, stream=stream)
        self.hout.copy_(self.out, non_blocking=True)
        stream.synchronize()

    def io_bytes(self):
        return 2 * self.ref.numel() * 4, self.windows * 32

    def ok_fraction(self, swift):
        return float((swift.decode(self.out)["status"] == 0).mean())

    def torch_windows(self, torch):
        def get():
            yield self.mov, self.ref
        return get

    def oracle_windows(self, k):
        r = self.ref[:k].double().cpu().numpy()
        m = self.mov[:k].double().cpu().numpy()
        return list(m), list(r), self.n, self.w, self.r


class Warp:
    name = "warp"
    dominant_n = 128

    def __init__(self, torch, swift, dev, count=2048, **_):
        import synth
        self.n, self.w, self.r = 128, 0.65, 3.0
        size = 2048
        stack = synth.section_stack(size, depth=9, seed=20)
        self.model = np.ascontiguousarray(stack[[0, 1, 2, 3, 5, 6, 7, 8]])
        self.movsec = np.ascontiguousarray(stack[4])
        self.org = synth.random_origins(count, size, size, self.n, seed=21, margin=8)
        self.theta = synth.affine_params(count, seed=22)
        self.windows = count
        self.description = (f"{count} windows of 128x128 on a 9-section {size}^2 stack: reference = mean of the 8 "
                            f"neighbours of section 4, moving = section 4 resampled under per-window affine warps "
                            f"(offset +-2 px, rotation +-0.5 deg); step = forward + backward of -sum snr*peak")
        self.plan = swift.Plan([swift.Level(self.n, self.w, "hann", 1.0, self.r)], dtype="u8", max_windows=count)
        T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)  # noqa: E731
        self.dm, self.ds = T(self.model), T(self.movsec)
        self.dorg, self.dth = T(self.org), T(self.theta)
        self.out = torch.empty((count, 8), dtype=torch.int32, device=dev)
        self.flops = 3.0 * flops_per_pair(self.n) * count  # forward + (recomputed forward + adjoint)
        slices = -(-count // 1024)  # warp / backward slices of 1024 windows
        self.launches_per_step = slices * (1 + 5) + slices * (1 + 10) + 1
        self.config = {"window": 128, "windows_per_step": count, "model_sections": 8, "input": "uint8",
                       "step": "forward + backward"}

    def step(self, stream):
        import torch
        self.plan.match(self.dm, self.ds, self.dorg, self.dorg, out=self.out, stream=stream, affine=self.dth)
        f = self.out.view(torch.float32)
        self.plan.backward(self.dm, self.ds, self.dorg, self.dorg, -f[:, 4], -f[:, 5], affine=self.dth,
                           stream=stream)

    def e2e_step(self, torch, stream):
        if not hasattr(self, "hth"):
            self.hth = torch.from_numpy(self.theta).pin_memory()
            self.hg = torch.empty((self.windows, 6), dtype=torch.float32).pin_memory()
        self.dth.copy_(self.hth, non_blocking=True)
        self.plan.match(self.dm, self.ds, self.dorg, self.dorg, out=self.out, stream=stream, affine=self.dth)
        f = self.out.view(torch.float32)
        g, _ = self.plan.backward(self.dm, self.ds, self.dorg, self.dorg, -f[:, 4], -f[:, 5], affine=self.dth,
                                  stream=stream)
        self.hg.copy_(g, non_blocking=True)
        stream.synchronize()

    def io_bytes(self):
        return self.theta.nbytes, self.windows * 6 * 4

    def ok_fraction(self, swift):
        return float((swift.decode(self.out)["status"] == 0).mean())

    def oracle_windows(self, k):
        from oracle import swim
        movs, refs = [], []
        for i in range(k):
            movs.append(swim.resample(self.movsec, self.org[i], self.n, self.theta[i].astype(np.float64)))
            refs.append(swim.project(list(self.model), self.org[i], self.n))
        return movs, refs, self.n, self.w, self.r


class Whitening:
    """The whitening-exponent study (Sec. III, Fig. 2) as a batched workload:
    damaged 256 x 256 pairs matched at 11 exponents in one call."""
    name = "whitening"
    dominant_n = 256

    def __init__(self, torch, swift, dev, count=256, lanes=0, **_):
        import synth
        self.n, self.w, self.r = 256, 0.6, 3.0
        self.exps = [round(0.1 * k, 1) for k in range(11)]
        ref, mov, self.shifts = synth.damaged_pairs(self.n, count, seed=90)
        self.ref_np, self.mov_np = ref, mov
        E = len(self.exps)
        self.windows = count * E
        self.description = (f"{count} damaged 256x256 uint8 pairs (illumination gradient, dark fold, smeared half "
                            f"plane, shot noise; known integer shifts) matched at {E} whitening exponents "
                            f"0, 0.1, ..., 1 in one call ({self.windows} windows)")
        self.plan = swift.Plan([swift.Level(self.n, w, "hann", 1.0, self.r) for w in self.exps], dtype="u8",
                               max_windows=self.windows)
        if lanes:
            self.plan.set_lanes(lanes)
        T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)  # noqa: E731
        self.dref = T(np.tile(ref, (E, 1, 1)))
        self.dmov = T(np.tile(mov, (E, 1, 1)))
        self.lvl = T(np.repeat(np.arange(E, dtype=np.int32), count))
        self.out = torch.empty((self.windows, 8), dtype=torch.int32, device=dev)
        self.hout = torch.empty((self.windows, 8), dtype=torch.int32).pin_memory()
        self.flops = flops_per_pair(self.n) * self.windows
        # each exponent's range in its slices, three kernels a slice
        self.launches_per_step = 3 * E * stream_slices(count, self.windows, self.plan.lanes)
        self.count = count
        self.config = {"window": 256, "windows_per_step": self.windows, "pairs": count, "exponents": self.exps,
                       "input": "uint8"}

    def step(self, stream):
        E = len(self.exps)
        self.plan.match([self.dref] * E, [self.dmov] * E, level=self.lvl, out=self.out, stream=stream,
                        level_offsets=[self.count * e for e in range(E + 1)])

    def e2e_step(self, torch, stream):
        if not hasattr(self, "href"):
            self.href, self.hmov = self.dref.cpu().pin_memory(), self.dmov.cpu().pin_memory()
        self.dref.copy_(self.href, non_blocking=True)
        self.dmov.copy_(self.hmov, non_blocking=True)
        self.step(stream)
        self.hout.copy_(self.out, non_blocking=True)
        stream.synchronize()

    def io_bytes(self):
        return 2 * self.dref.numel(), self.windows * 32

    def ok_fraction(self, swift):
        g = swift.decode(self.out)
        E, P = len(self.exps), self.count
        curve = []
        for e, w in enumerate(self.exps):
            sl = slice(e * P, (e + 1) * P)
            hit = (np.abs(g["sy"][sl] - self.shifts[:, 0]) <= 1.5) & (np.abs(g["sx"][sl] - self.shifts[:, 1]) <= 1.5)
            curve.append({"w": w, "median_snr": round(float(np.median(g["snr"][sl])), 3),
                          "located_within_1.5px": round(float(hit.mean()), 4)})
        self.config["snr_curve"] = curve
        return float((g["status"] == 0).mean())

    def oracle_windows(self, k):
        k = min(k, self.count)
        lvl = self.exps.index(self.w)
        return ([m.astype(np.float64) for m in self.mov_np[:k]], [r.astype(np.float64) for r in self.ref_np[:k]],
                self.n, self.exps[lvl], self.r)


def make_workload(name, torch, swift, dev, args):
    if name == "sections":
        return Sections(torch, swift, dev, pairs=args.pairs, windows=args.windows, precision=args.precision,
                        rank=int(os.environ.get("RANK", "0")), lanes=args.lanes, mov_shift=args.mov_shift,
                        row_tma=args.row_tma)
    if name == "noise64":
        return Noise64(torch, swift, dev)
    if name == "pyramid":
        return Pyramid(torch, swift, dev, schedule=args.schedule, lanes=args.lanes)
    if name in ("patches128", "patches256"):
        return Patches(torch, swift, dev, n=int(name[7:]), count=args.windows or 8192, precision=args.precision,
                       lanes=args.lanes)
    if name == "warp":
        return Warp(torch, swift, dev, count=args.windows or 2048)
    if name == "whitening":
        return Whitening(torch, swift, dev, count=args.windows or 256, lanes=args.lanes)
    raise ValueError(name)


# --------------------------------------------------------------------------- #
# the rendering step (mir): mesh fit + texture mapping of a whole section
# --------------------------------------------------------------------------- #
MIR_METRIC = "rendered output pixels/sec (mir: per-triangle SNR-weighted affine fit + texture mapping)"


def mir_main(args, torch, swift, dev, world, rank):
    """Workload: the headline section pair's swim grid (31 x 31 windows of
    256^2, computed once) gives SNR-weighted correspondences; a step fits one
    affine per triangle of a 16 x 16-cell mesh (cell 256 px, band 256 px) and
    renders the moving section (uint8, 4096^2) into the reference frame as
    float32.  Metric: output pixels per second."""
    import synth
    size, n, stride, cell = 4096, 256, 128, 256
    a, b = synth.em_section_pair(size)
    org = synth.grid_origins(size, n, stride)
    da, db = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    dorg = torch.from_numpy(org).to(dev)
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=len(org))
    res = plan.match(da, db, dorg, dorg)
    q, p, w = swift.correspondences(res, dorg, dorg, n, min_snr=5.0)
    mesh = swift.Mesh(0, 0, cell, size // cell, size // cell)
    band = cell
    out = torch.empty((size, size), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    recs = torch.empty((mesh.n_triangles, 8), dtype=torch.float32, device=dev)

    def step():
        th, st = swift.mesh_fit(q, p, w, mesh, band, stream=stream)
        swift.render_records(th, mesh, records=recs, stream=stream)
        swift.render(db, th, mesh, size, size, fill=0.0, out=out, records=recs, stream=stream)
        return th, st

    warm = max(args.warmup, 3)
    for _ in range(warm):
        th, st = step()
    torch.cuda.synchronize(dev)
    ok_frac = float((st == swift.FIT_OK).float().mean())
    sampler = ClockSampler(local_rank())
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        th, _ = swift.mesh_fit(q, p, w, mesh, band, stream=stream)
        swift.render_records(th, mesh, records=recs, stream=stream)
        mids[k].record(stream)
        swift.render(db, th, mesh, size, size, fill=0.0, out=out, records=recs, stream=stream)
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    fit_ms = sum(s_.elapsed_time(m_) for s_, m_ in zip(starts, mids)) / args.steps
    render_ms = sum(m_.elapsed_time(e_) for m_, e_ in zip(mids, ends)) / args.steps
    px = size * size
    total_ms, value = aggregate_over_ranks(total_ms, px, args.steps, world, dev)
    print(f"[bench] mir rank {rank}: {args.steps} steps, {total_ms / args.steps:.4f} ms/step "
          f"(fit {fit_ms:.4f}, render {render_ms:.4f}), {value / 1e9:.3f} Gpx/s", file=sys.stderr, flush=True)

    # e2e: section and correspondences in from pinned host memory, image out
    hb = b.copy()
    hb_t = torch.from_numpy(hb).pin_memory()
    hq, hp, hw = q.cpu().pin_memory(), p.cpu().pin_memory(), w.cpu().pin_memory()
    hout = torch.empty((size, size), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        db.copy_(hb_t, non_blocking=True)
        q.copy_(hq, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        w.copy_(hw, non_blocking=True)
        step()
        hout.copy_(out, non_blocking=True)
        stream.synchronize()
    e2e_value = world * px * e2e_steps / (time.perf_counter() - t0)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    algo_bytes = px * (1 + 4)  # uint8 source read once, float32 written
    achieved = algo_bytes / (render_ms / 1e3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import mir as omir
        qn, pn, wn = q.cpu().numpy(), p.cpu().numpy(), w.cpu().numpy()
        rows = np.arange(0, size, 16)  # every 16th output row
        t0 = time.perf_counter()
        oth, _ = omir.mesh_fit(qn, pn, wn, omir.Mesh(0, 0, cell, size // cell, size // cell), band)
        omir.render(b, oth, omir.Mesh(0, 0, cell, size // cell, size // cell), size, size, 0.0, rows=rows)
        dt = time.perf_counter() - t0
        cpu = {"value": len(rows) * size / dt, "unit": "pixels/s", "cores": 1, "kind": "oracle",
               "sample": f"mesh fit of all {mesh.n_triangles} triangles + {len(rows)} of {size} output rows "
                         f"(every 16th), FP64 numpy, one process ({dt:.1f} s)"}
    line = {
        "metric": MIR_METRIC, "value": value, "unit": "pixels/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 fits)", "data": "synthetic",
        "config": {"workload": f"mir: {mesh.n_triangles}-triangle mesh (cell {cell}, band {band}) fitted to the "
                               f"SNR-weighted swim correspondences of the {len(org)}-window 256^2 grid, "
                               f"{size}x{size} uint8 moving section rendered as float32",
                   "name": "mir", "fit_ok_fraction": ok_frac, "fit_ms": fit_ms, "render_ms": render_ms,
                   "l2": "flushed before every timed step (256 MiB write, outside the step's events)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "render_run_kernel<u8>",
                     "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json); algorithmic bytes = 1 B "
                                  "source + 4 B output per pixel"},
        "e2e": {"value": e2e_value, "unit": "pixels/s", "h2d_bytes_per_step": int(hb.nbytes + 5 * 4 * len(org)),
                "d2h_bytes_per_step": int(px * 4)},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))


REMOD_METRIC = "sections/sec (remod: Z-averaged model of every section + iscale 2x/4x pyramid)"


def remod_main(args, torch, swift, dev, world, rank):
    """Workload: a 9-section stack of 4096^2 uint8 EM-like sections (the
    headline section drifting by one pixel per section, independent noise);
    a step computes the Z model of every section (k = 4, section 6 marked
    damaged) and the 2x and 4x box-mean pyramid levels of every section.
    Metric: sections per second."""
    import synth
    size, Z, k = 4096, 9, 4
    a, _ = synth.em_section_pair(size)
    rng = np.random.default_rng(90)
    stack = np.stack([np.clip(np.roll(a, (z, -z), (0, 1)).astype(np.int16)
                              + rng.integers(-6, 7, a.shape, dtype=np.int16), 0, 255).astype(np.uint8)
                      for z in range(Z)])
    ts = torch.from_numpy(stack).to(dev)
    valid = torch.ones(Z, dtype=torch.uint8, device=dev)
    valid[6] = 0
    model = torch.empty((Z, size, size), dtype=torch.float32, device=dev)
    p2 = torch.empty((Z, size // 2, size // 2), dtype=torch.uint8, device=dev)
    p4 = torch.empty((Z, size // 4, size // 4), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        swift.zmodel(ts, k, valid=valid, out=model, stream=stream)
        swift.downsample(ts, 2, out=p2, stream=stream)
        swift.downsample(ts, 4, out=p4, stream=stream)

    warm = max(args.warmup, 3)
    for _ in range(warm):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local_rank())
    sampler.start()
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    for e0, e1, e2 in ev:
        flush.zero_()
        e0.record(stream)
        swift.zmodel(ts, k, valid=valid, out=model, stream=stream)
        e1.record(stream)
        swift.downsample(ts, 2, out=p2, stream=stream)
        swift.downsample(ts, 4, out=p4, stream=stream)
        e2.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = sum(e0.elapsed_time(e2) for e0, _, e2 in ev)
    zm_ms = sum(e0.elapsed_time(e1) for e0, e1, _ in ev) / args.steps
    ds_ms = sum(e1.elapsed_time(e2) for _, e1, e2 in ev) / args.steps
    total_ms, value = aggregate_over_ranks(total_ms, Z, args.steps, world, dev)
    print(f"[bench] remod rank {rank}: {args.steps} steps, {total_ms / args.steps:.4f} ms/step "
          f"(zmodel {zm_ms:.4f}, pyramid {ds_ms:.4f}), {value:.1f} sections/s", file=sys.stderr, flush=True)

    hs = torch.from_numpy(stack).pin_memory()
    hm = torch.empty((Z, size, size), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ts.copy_(hs, non_blocking=True)
        step()
        hm.copy_(model, non_blocking=True)
        stream.synchronize()
    e2e_value = world * Z * e2e_steps / (time.perf_counter() - t0)

    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    px = size * size
    algo_bytes = Z * px * (1 + 4)  # each section read once, each model written (float32)
    achieved = algo_bytes / (zm_ms / 1e3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import remod as orm
        rows = 256  # a band of rows of every section
        t0 = time.perf_counter()
        orm.zmodel(stack[:, :rows], k, valid.cpu().numpy().astype(bool))
        for z in range(Z):
            orm.downsample(stack[z, :rows // 4 * 4, :256], 4)
        dt = time.perf_counter() - t0
        cpu = {"value": Z * rows / size / dt, "unit": "sections/s", "cores": 1, "kind": "oracle",
               "sample": f"Z models of the first {rows} of {size} rows of all {Z} sections plus a 4x pyramid "
                         f"block, numpy, one process ({dt:.2f} s), scaled to whole sections"}
    line = {
        "metric": REMOD_METRIC, "value": value, "unit": "sections/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8 in, f32 model", "data": "synthetic",
        "config": {"workload": f"{Z}-section {size}x{size} uint8 stack; Z model (k = {k}, one damaged section) "
                               f"and 2x / 4x pyramid levels of every section",
                   "name": "remod", "zmodel_ms": zm_ms, "pyramid_ms": ds_ms,
                   "l2": "flushed before every timed step (256 MiB write, outside the step's events)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "zmodel_kernel<16>",
                     "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json); algorithmic bytes = 1 B "
                                  "read + 4 B written per section pixel"},
        "e2e": {"value": e2e_value, "unit": "sections/s", "h2d_bytes_per_step": int(stack.nbytes),
                "d2h_bytes_per_step": int(Z * px * 4)},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))


ALIGN_METRIC = "section-iterations/sec (registration loop: Z model, grid match, SNR-weighted affine, render)"


def align_main(args, torch, swift, dev, world, rank):
    """Workload: 8 crops (1024^2, uint8) of the headline EM-like section at
    known offsets of up to +-6 px, independent noise; a step is one call of
    the registration loop with 3 iterations (128^2 windows at stride 64, 225
    per section, k = 3), through one reusable StackAligner (every iteration
    a replay of its captured CUDA graph).  Timed by the host clock around each
    call (the loop reads the window results back once per iteration).
    Metric: section-iterations per second."""
    import synth
    from paper_1612_04787_gb300 import align
    size, Z, n, stride, k, iters = 1024, 8, 128, 64, 3, 3
    a, _ = synth.em_section_pair(2048)
    rng = np.random.default_rng(95)
    offs = rng.integers(-6, 7, (Z, 2))
    raw = np.stack([np.clip(a[512 + dy:512 + dy + size, 512 + dx:512 + dx + size].astype(np.int16)
                            + rng.integers(-6, 7, (size, size), dtype=np.int16), 0, 255).astype(np.uint8)
                    for dy, dx in offs])
    traw = torch.from_numpy(raw).to(dev)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    aligner = align.StackAligner(Z, size, size, lv, stride, k, device=dev)  # plan, buffers and graph reused
    warm = max(args.warmup, 3)
    for _ in range(warm):
        aligned, theta, hist = aligner.run(traw, iters)
    torch.cuda.synchronize(dev)
    # displacement of the section centre (the translation at q = 0 trades off against A over 1024 px)
    th = theta.cpu().numpy()
    c = size / 2.0
    disp = np.stack([th[:, 0] * c + th[:, 1] * c + th[:, 2] - c, th[:, 3] * c + th[:, 4] * c + th[:, 5] - c], 1)
    resid = float(np.abs((disp - disp.mean(0)) + (offs - offs.mean(0))).max())
    sampler = ClockSampler(local_rank())
    sampler.start()
    time.sleep(0.3)
    steps = max(1, min(args.steps, 20))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        aligner.run(traw, iters)
    torch.cuda.synchronize(dev)
    total_ms = (time.perf_counter() - t0) * 1e3
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms, value = aggregate_over_ranks(total_ms, Z * iters, steps, world, dev)
    B = len(align.window_grid(size, size, n, stride))
    match_flops = flops_per_pair(n) * B * Z * iters
    achieved = match_flops / (total_ms / steps / 1e3) / 1e12
    peak = fp32_peak_tflops()
    print(f"[bench] align rank {rank}: {steps} steps, {total_ms / steps:.3f} ms/step, {value:.1f} "
          f"section-iterations/s, offset residual {resid:.3f} px", file=sys.stderr, flush=True)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import driver as odrv, swim as osw
        small = raw[:3, :256, :256]
        t1 = time.perf_counter()
        odrv.align_stack(small, osw.Level(64, 0.65, osw.APOD_HANN, 1.0, 3.0), 48, 2, 1)
        dt = time.perf_counter() - t1
        cpu = {"value": 3 / dt, "unit": "section-iterations/s", "cores": 1, "kind": "oracle",
               "sample": f"one iteration on 3 sections of 256^2 with 64^2 windows (16 per section), FP64 oracle, "
                         f"one process ({dt:.1f} s); a far smaller problem than the GPU step"}
    line = {
        "metric": ALIGN_METRIC, "value": value, "unit": "section-iterations/s", "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8 images, f32 match, f64 fits", "data": "synthetic",
        "config": {"workload": f"{Z} sections of {size}x{size} uint8 at known offsets (+-6 px), {iters} iterations, "
                               f"{B} windows of {n}^2 per section, k = {k}",
                   "name": "align", "centre_offset_residual_px": resid, "median_snr_per_iteration": hist,
                   "timing": "host clock around each call (one graph replay and one result read-back per iteration)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole loop (match flops only)",
                     "peak_note": "derived FP32 FMA peak; achieved counts only the matches' algorithmic flops over "
                                  "the whole loop's time"},
        "e2e": {"value": value, "unit": "section-iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(Z * iters * (B * 32 + 4))},
        "gpu_launches": steps * iters * (3 + 7 * Z),  # per iteration: models, 5 per match, correspondences, fit, 2 per render
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))


def local_rank() -> int:
    return int(os.environ.get("LOCAL_RANK", "0"))


# --------------------------------------------------------------------------- #
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_over_ranks(total_ms, windows, steps, world, device=None):
    """Weak scaling: every rank matches its own shard of the job (its own
    section pairs, the same count per rank) on its own GPU; the job time is
    the slowest rank's (all-reduce MAX), and the value counts the windows of
    all ranks.  Returns (job ms, windows/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * windows * steps / (total_ms / 1e3)


def reference_arm(args):
    """The FP64 oracle timed on the host cores (no GPU)."""
    import synth
    n, w, r = 256, 0.65, 3.0
    a, b = synth.em_section_pair(4096)
    org = synth.grid_origins(4096, 256, 128)[: args.oracle_sample]
    movs = [b[y:y + n, x:x + n].astype(np.float64) for y, x in org]
    refs = [a[y:y + n, x:x + n].astype(np.float64) for y, x in org]
    for _ in range(args.warmup):
        oracle_throughput(movs[:64], refs[:64], n, w, r)
    vals, cores = [], 0
    for _ in range(args.steps):
        v, cores, _dt = oracle_throughput(movs, refs, n, w, r)
        vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * len(org) / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "31x31 grid of 256x256 windows (stride 128) on a 4096x4096 uint8 EM-like "
                               "section pair", "windows_per_step": len(org)},
        "cpu_baseline": {"value": value, "unit": "windows/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {len(org)} windows of the workload per step, FP64 direct-DFT oracle, "
                                   f"one single-threaded process per core"},
        "e2e": {"value": value, "unit": "windows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def kernel_names(n: int) -> dict:
    """Kernel of each streaming slot of the FP32 schedule at window size n
    (column pairs up to 256, per-column kernel at 512)."""
    return {"stats": "stream_stats_kernel", "rows": "stream_rows_kernel",
            "cols": "stream_cpair_kernel" if n <= 256 else "stream_cols_kernel",
            "irows": "stream_irows_kernel", "final": "stream_peak_kernel", "fused": "swim_forward_kernel",
            "persistent": "swim_persistent_kernel"}
TC_KERNEL_NAMES = {"stats": "stream_stats_kernel", "rows": "tcf_rows_kernel", "cols": "tcf_cols_kernel",
                   "irows": "tcf_irows_kernel", "final": "stream_final_kernel"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sections",
                    choices=["sections", "noise64", "pyramid", "patches128", "patches256", "warp", "whitening", "mir", "remod",
                             "align"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x2", "fp16x2"])
    ap.add_argument("--schedule", default="default", choices=["default", "fused", "stream", "persistent"],
                    help="forward schedule of every level (FP32 workloads without their own choice)")
    ap.add_argument("--pairs", type=int, default=1, help="section pairs per step (sections workload)")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2],
                    help="streams an FP32 call spreads over (0: the plan's default / the autotuner's pick)")
    ap.add_argument("--windows", type=int, default=0, help="limit the windows per step (small profiling cases)")
    ap.add_argument("--mov-shift", type=int, default=0,
                    help="sections: moving windows shifted this many px in x (rows off 16-byte boundaries)")
    ap.add_argument("--row-tma", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="sections: uint8 row loads (0 plain, 1 tile copies for unaligned rows, 2 tile copies; "
                         "-1 the plan's default)")
    ap.add_argument("--oracle-sample", type=int, default=961)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the cuFFT and host-FFT comparisons")
    args = ap.parse_args()
    world, rank, local = dist_setup()

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_1612_04787_gb300 as swift

    if args.workload in ("mir", "remod", "align"):
        {"mir": mir_main, "remod": remod_main, "align": align_main}[args.workload](args, torch, swift, dev, world,
                                                                                   rank)
        if world > 1:
            dist.destroy_process_group()
        return
    W = make_workload(args.workload, torch, swift, dev, args)
    if args.schedule != "default" and args.workload not in ("pyramid", "warp"):
        for l in range(len(W.plan.levels)):
            W.plan.set_schedule(l, args.schedule)
        W.config["schedule"] = args.schedule
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    warm = max(args.warmup, 3)
    for _ in range(warm):
        W.step(stream)
    torch.cuda.synchronize(dev)
    ok_frac = W.ok_fraction(swift)

    # per-kernel CUDA events around the library's launches (not under graph
    # replay).  With two lanes a launch shares the GPU with the other lane's
    # launches, so its event duration is not the kernel's own: the per-kernel
    # figures then come from a second timed region of the same steps with one
    # lane, and the headline value stays the two-lane region's
    timing = args.workload not in ("pyramid", "warp", "noise64")
    lanes = W.plan.lanes if timing else 1
    separate = timing and lanes > 1

    def count_launches():
        # one untimed step counts each kernel's launches per step; a timed
        # region's event ring may keep only its most recent launches, so the
        # windows per launch come from this count, not from the ring's size
        W.plan.set_timing(True)
        W.plan.timings()
        W.step(stream)
        torch.cuda.synchronize(dev)
        return {k: v[1] for k, v in W.plan.timings().items()}
    launches_per_step = count_launches() if timing else {}
    launches_kernel = launches_per_step
    if separate:
        W.plan.set_timing(False)
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
        W.step(stream)
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    kt = W.plan.timings() if timing and not separate else {}
    if timing:
        W.plan.set_timing(False)
    if separate:
        W.plan.set_lanes(1)
        for _ in range(3):
            W.step(stream)
        launches_kernel = count_launches()
        for _ in range(args.steps):
            flush.zero_()
            W.step(stream)
        torch.cuda.synchronize(dev)
        kt = W.plan.timings()
        W.plan.set_timing(False)
        W.plan.set_lanes(lanes)
    durs = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    total_ms, value = aggregate_over_ranks(sum(durs), W.windows, args.steps, world, dev)
    print(f"[bench] {W.name} rank {rank}: {args.steps} steps, {total_ms / args.steps:.4f} ms/step, "
          f"{value:.1f} windows/s", file=sys.stderr, flush=True)

    # e2e through the public API with host buffers
    e2e_steps = max(3, min(args.steps, 30))
    W.e2e_step(torch, stream)
    if hasattr(W, "e2e_run"):
        W.e2e_run(torch, stream, 2)
        e2e_s = W.e2e_run(torch, stream, e2e_steps)
    else:
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            W.e2e_step(torch, stream)
        e2e_s = time.perf_counter() - t0
    e2e_value = world * W.windows * e2e_steps / e2e_s
    h2d, d2h = W.io_bytes()

    cufft = None
    if hasattr(W, "torch_windows") and not args.no_compare:
        v, ms = cufft_throughput(torch, W, stream, min(args.steps, 20), flush)
        cufft = {"value": v, "unit": "windows/s", "ms_per_step": ms,
                 "kind": "cuFFT through torch.fft: apodise, rfft2, C = M conj(R), whitening, irfft2, argmax "
                         "(window gather included; no SNR or subpixel fit); a library comparison, not the product"}

    cpu = cpu_fft = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        movs, refs, n, w, r = W.oracle_windows(args.oracle_sample)
        v, cores, dt = oracle_throughput(movs, refs, n, w, r)
        what = getattr(W, "oracle_note", "windows of the workload")
        cpu = {"value": v, "unit": "windows/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(movs)} {what} ({n}x{n}), FP64 direct-DFT oracle, forward only, "
                         f"one single-threaded process per core ({dt:.1f} s)"}
        if not args.no_compare:
            v, cores, dt = cpu_fft_throughput(movs, refs, n, w)
            cpu_fft = {"value": v, "unit": "windows/s", "cores": cores,
                       "kind": "scipy.fft float32 (pocketfft), all host cores: apodise, rfft2, C = M conj(R), "
                               "whitening, irfft2, argmax (no SNR or subpixel fit)",
                       "sample": f"{len(movs)} {what} ({n}x{n}), {dt:.2f} s"}

    tensor = args.precision != "fp32"
    peak = fp32_peak_tflops()
    step_tflops = W.flops / (total_ms / args.steps / 1e3) / 1e12
    if kt:
        dom = max(kt, key=lambda k: kt[k][0])
        launches = kt[dom][1]
        dom_ms = kt[dom][0] / launches
        windows_per_launch = W.windows / launches_kernel[dom]
        per_window = tensor_flops(W.dominant_n)[dom] if tensor else kernel_flops(W.dominant_n)[dom]
        achieved = per_window * windows_per_launch / (dom_ms / 1e3) / 1e12
        tot = sum(x[0] for x in kt.values())
        shares = {k: round(v[0] / tot, 4) for k, v in kt.items()}
        dom_name = (TC_KERNEL_NAMES if tensor else kernel_names(W.dominant_n))[dom]
    else:
        # no per-kernel events: graph replays, or a step with the backward's kernels
        label = "pipeline (graph replay)" if "graph" in W.config else "pipeline (whole step)"
        dom_name, achieved, shares, windows_per_launch = label, step_tflops, None, W.windows
    # traffic records are per kernel, window size and input type (a row kernel
    # reads 1-byte or 4-byte pixels)
    in_key = "u8" if W.config.get("input") == "uint8" else "f32"
    traffic = recorded_traffic(f"{dom_name}<{W.dominant_n},{in_key}>", windows_per_launch)
    if tensor:
        pk = measured_peaks().get("bf16_tflops_sustained") or 1700.0
        roofline = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                    "traffic": traffic, "kernel": f"{dom_name}<{W.dominant_n}>",
                    "peak_note": "measured dense BF16 cuBLAS GEMM, sustained (MEASURED_PEAKS.json); FP16 has the "
                                 "same nominal rate; achieved counts the executed m16n8k16 products (three hi/lo "
                                 "terms), not algorithmic FFT work; mma.sync m16n8k16 itself measured ~600 TFLOP/s "
                                 "on this GPU",
                    "kernel_share_of_step": shares,
                    "algorithmic_fp32_tflops": step_tflops, "algorithmic_fp32_frac": step_tflops / peak}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": f"{dom_name}<{W.dominant_n}>",
                    "peak_note": "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz (max SM clock)",
                    "kernel_share_of_step": shares,
                    "pipeline_tflops": step_tflops, "pipeline_frac": step_tflops / peak}
    if separate:
        roofline["kernel_timing"] = (f"per-kernel durations and shares from a second timed region of the same "
                                     f"{args.steps} steps with one lane (the value's region ran {lanes} lanes, "
                                     f"whose launches overlap)")
    line = {
        "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": total_ms / args.steps,
        "ms_per_step_best": min(durs), "ms_per_step_median": statistics.median(durs),  # this rank's steps
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x2": "bf16x2 (f32 accumulate)",
                                                         "fp16x2": "f16x2 (f32 accumulate)"}[args.precision],
        "data": "synthetic",
        "config": dict({"workload": W.description, "name": W.name,
                        "l2": "flushed before every timed step (256 MiB write, outside the step's events)",
                        "status_ok_fraction": ok_frac}, **W.config),
        "roofline": roofline,
        "e2e": dict({"value": e2e_value, "unit": "windows/s", "h2d_bytes_per_step": int(h2d),
                     "d2h_bytes_per_step": int(d2h)},
                    **({"pipelining": "double-buffered: step k's host-to-device copy (copy stream) overlaps step "
                                      "k-1's match; every step copies its sections in and its results out"}
                       if hasattr(W, "e2e_run") else {})),
        "gpu_launches": args.steps * (sum(launches_per_step.values()) if launches_per_step else W.launches_per_step),
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if cpu_fft is not None:
        line["cpu_fft_baseline"] = cpu_fft
    if cufft is not None:
        line["cufft_comparison"] = cufft
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
