"""The registration loop of Sec. IV on the device: align a section stack at
one resolution by matching, rendering and remodelling until the swim SNR
settles (``align_stack``), and coarse to fine over a box-downsampled pyramid,
expanding each level's affines to the next higher resolution
(``align_pyramid``).

Every image step is a library kernel: uint8 Z models (``swift_zmodel``),
the grid match of each raw section against its model (``swift_match_batch``),
SNR-weighted correspondences and the least-squares affine, which keeps a
section's previous affine when its fit is degenerate
(``swift_correspondences``, ``swift_fit_affine_update``), and the render of
the raw section through that affine (``swift_render_prepare`` /
``swift_render``, uint8).  The host only sequences the calls (or replays
them as one CUDA graph) and applies the convergence rule on the median SNR
of each iteration (read back from the results), as the paper's own driver
scripts did around its modules.

Readings (the same as the oracle's): a section whose fit is degenerate keeps
its previous affine; the loop stops when the median SNR of the OK windows
changes by at most ``tol`` (relative), or after ``iters`` iterations.  The
models need neighbours on both sides: with large initial offsets, k = 1
(nearest neighbours only) can oscillate, k >= 2 converges.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Level, Mesh, Plan, correspondences, decode, downsample, fit_affine, render, render_records,
               zmodel)


def window_grid(h: int, w: int, n: int, stride: int, margin: int = 0) -> np.ndarray:
    """(y, x) origins of the n x n windows at the given stride, at least
    ``margin`` px inside every border, int32 [B, 2]."""
    ys = np.arange(margin, h - n - margin + 1, stride)
    xs = np.arange(margin, w - n - margin + 1, stride)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([Y.ravel(), X.ravel()], 1).astype(np.int32)


class StackAligner:
    """The registration loop for stacks of one shape, reusable: it owns the
    plan, the buffers and (with ``graph``) one captured CUDA graph of an
    iteration.  An iteration: the Z models, every section's grid match (one
    call per section), one correspondence call and one grouped affine update
    over all sections (a degenerate fit keeps the section's previous affine on
    the device), and the renders; then one read-back of the match results for
    the convergence rule.  The very first iteration runs call by call, the
    second is captured, and every later iteration (of this run or of later
    runs) is one replay of that graph: a run copies its stack into the
    aligner's own buffer, so the graph's pointers stay valid.  Runs on the
    current CUDA stream."""

    def __init__(self, Z: int, H: int, W: int, level: Level, stride: int, k: int, min_snr: float = 0.0,
                 device=None, graph: bool = True, margin: int = 0):
        dev = torch.device(device if device is not None else "cuda")
        self.Z, self.H, self.W, self.k, self.min_snr, self.graph = Z, H, W, k, min_snr, graph
        self.n = level.n
        org = torch.from_numpy(window_grid(H, W, level.n, stride, margin)).to(dev)
        self.B = B = int(org.shape[0])
        self.org, self.org_all = org, org.repeat(Z, 1)  # the same grid in every section
        self.offsets = torch.arange(0, (Z + 1) * B, B, dtype=torch.int64, device=dev)
        self.plan = Plan([level], dtype="u8", max_windows=B)
        self.raw = torch.empty((Z, H, W), dtype=torch.uint8, device=dev)
        self.aligned = torch.empty_like(self.raw)
        self.model = torch.empty_like(self.raw)
        self.identity = torch.tensor([1.0, 0.0, 0.0, 0.0, 1.0, 0.0], dtype=torch.float64, device=dev).repeat(Z, 1)
        self.theta = self.identity.clone()
        self.status = torch.empty((Z,), dtype=torch.int32, device=dev)
        self.mesh = Mesh(0, 0, max(H, W), 1, 1)
        nt = self.mesh.n_triangles
        self.tri = torch.empty((Z, nt, 6), dtype=torch.float64, device=dev)  # both triangles: the section's affine
        self.recs = torch.empty((Z, nt, 8), dtype=torch.float32, device=dev)
        self.res = torch.empty((Z, B, 8), dtype=torch.int32, device=dev)
        self.g = None
        self.iterations_done = 0

    def _render_all(self):
        """Render every raw section through its current affine (both mesh
        triangles carry the section's affine)."""
        Z, nt = self.Z, self.mesh.n_triangles
        self.tri.copy_(self.theta[:, None, :].expand(Z, nt, 6))
        for z in range(Z):
            render_records(self.tri[z], self.mesh, records=self.recs[z])
            render(self.raw[z], self.tri[z], self.mesh, self.H, self.W, fill=0.0, out=self.aligned[z],
                   records=self.recs[z])

    def _iteration(self):
        Z, B, n = self.Z, self.B, self.n
        zmodel(self.aligned, self.k, out=self.model)
        for z in range(Z):
            self.plan.match(self.model[z], self.raw[z], self.org, self.org, out=self.res[z])
        q, p, w = correspondences(self.res.view(Z * B, 8), self.org_all, self.org_all, n, self.min_snr)
        fit_affine(q, p, w, offsets=self.offsets, update=self.theta, status=self.status)
        self._render_all()

    def _step(self):
        dev = self.raw.device
        if self.g is not None:
            self.g.replay()
        elif self.graph and self.iterations_done >= 1:
            self.g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.graph(self.g, stream=side):
                self._iteration()
            torch.cuda.current_stream(dev).wait_stream(side)
            self.g.replay()
        else:
            self._iteration()
        self.iterations_done += 1

    def run(self, raw: torch.Tensor, iters: int, tol: float = 0.0, theta0: torch.Tensor = None):
        """Align ``raw`` (uint8 [Z, H, W] on the aligner's device).  Returns
        (aligned uint8 [Z, H, W], theta float64 [Z, 6] (model frame -> raw
        section: p = A q + t), list of the median SNR of every iteration).
        ``theta0`` (float64 [Z, 6]): start from these affines -- the raw
        sections are rendered through them before the first models -- instead
        of the identity."""
        if raw.dtype != torch.uint8 or tuple(raw.shape) != (self.Z, self.H, self.W) or raw.device != self.raw.device:
            raise TypeError("raw must be a uint8 [Z, H, W] tensor of this aligner's shape and device")
        self.raw.copy_(raw)
        if theta0 is None:
            self.aligned.copy_(raw)
            self.theta.copy_(self.identity)
        else:
            self.theta.copy_(theta0.reshape(self.Z, 6))
            self._render_all()
        hist = []
        for _ in range(iters):
            self._step()
            d = decode(self.res.view(self.Z * self.B, 8))
            good = (d["status"] == 0) & np.isfinite(d["snr"])
            hist.append(float(np.median(d["snr"][good])) if good.any() else 0.0)
            if len(hist) > 1 and abs(hist[-1] - hist[-2]) <= tol * abs(hist[-2]):
                break
        return self.aligned.clone(), self.theta.clone(), hist


def align_stack(raw: torch.Tensor, level: Level, stride: int, k: int, iters: int, tol: float = 0.0,
                min_snr: float = 0.0, graph: bool = True, theta0: torch.Tensor = None, margin: int = 0):
    """Align a uint8 [Z, H, W] CUDA stack once (a StackAligner made for it).
    Returns (aligned uint8 [Z, H, W], theta float64 [Z, 6], list of the median
    SNR of every iteration)."""
    if raw.dtype != torch.uint8 or raw.dim() != 3 or not raw.is_cuda or not raw.is_contiguous():
        raise TypeError("raw must be a contiguous uint8 [Z, H, W] CUDA tensor")
    Z, H, W = raw.shape
    return StackAligner(Z, H, W, level, stride, k, min_snr, raw.device, graph, margin).run(raw, iters, tol, theta0)


def expand_affine(theta: torch.Tensor, r: int) -> torch.Tensor:
    """Affines [Z, 6] of a level r times coarser in the finer level's pixels:
    a coarse pixel centre u is the centre of an r x r box, fine coordinate
    r u + (r - 1) / 2, so t becomes r t + (r - 1) / 2 (1 - A 1); A is kept."""
    th = theta.clone()
    c = (r - 1) / 2.0
    th[:, 2] = r * theta[:, 2] + c * (1.0 - theta[:, 0] - theta[:, 1])
    th[:, 5] = r * theta[:, 5] + c * (1.0 - theta[:, 3] - theta[:, 4])
    return th


def align_pyramid(raw: torch.Tensor, factors, levels, strides, k: int, iters, tol=0.0, min_snr: float = 0.0,
                  margins=0, graph: bool = True):
    """Coarse-to-fine registration (Sec. IV: align at a working resolution until
    the SNR settles, then expand the model to the next higher resolution).

    ``factors`` decrease to 1, each a multiple of the next; level i works on
    the raw stack box-downsampled by factors[i] (``downsample``, uint8) with
    matching level ``levels[i]``, window stride ``strides[i]``, iteration cap
    ``iters[i]``, tolerance ``tol[i]`` and grid margin ``margins[i]`` (single
    numbers apply to every level).  Between levels the stack's common
    translation (mean t) is removed and the affines are expanded to the finer
    pixels (``expand_affine``); the finer level renders its raw sections
    through them before its first models.  Returns (aligned uint8 [Z, H, W] at
    full resolution, theta float64 [Z, 6] in full-resolution pixels, list of
    the per-level median-SNR histories)."""
    if raw.dtype != torch.uint8 or raw.dim() != 3 or not raw.is_cuda or not raw.is_contiguous():
        raise TypeError("raw must be a contiguous uint8 [Z, H, W] CUDA tensor")
    factors = [int(f) for f in factors]
    if factors[-1] != 1 or any(factors[i] % factors[i + 1] for i in range(len(factors) - 1)):
        raise ValueError("factors must decrease to 1, each a multiple of the next")
    L = len(factors)
    per = lambda v, cast: [cast(x) for x in v] if np.ndim(v) else [cast(v)] * L  # noqa: E731
    iters, tol, margins = per(iters, int), per(tol, float), per(margins, int)
    theta, hists, aligned = None, [], None
    for i, f in enumerate(factors):
        stack = raw if f == 1 else downsample(raw, f)
        if theta is not None:
            theta = theta.clone()
            theta[:, [2, 5]] -= theta[:, [2, 5]].mean(0)
            theta = expand_affine(theta, factors[i - 1] // f)
        aligned, theta, hist = align_stack(stack.contiguous(), levels[i], strides[i], k, iters[i], tol[i], min_snr,
                                           graph, theta, margins[i])
        hists.append(hist)
    return aligned, theta, hists
