"""The registration loop of Sec. IV on the device: align a section stack at
one resolution by matching, rendering and remodelling until the swim SNR
settles.

Every image step is a library kernel: uint8 Z models (``swift_zmodel``),
the grid match of each raw section against its model (``swift_match_batch``),
SNR-weighted correspondences and the least-squares affine
(``swift_correspondences``, ``swift_fit_affine``), and the render of the raw
section through that affine (``swift_render_prepare`` / ``swift_render``,
uint8).  The host only sequences the calls, keeps a section's previous
affine when its fit is degenerate, and applies the convergence rule on the
median SNR of each iteration (read back from the results), as the paper's
own driver scripts did around its modules.

Readings (the same as the oracle's): a section whose fit is degenerate keeps
its previous affine; the loop stops when the median SNR of the OK windows
changes by at most ``tol`` (relative), or after ``iters`` iterations.  The
models need neighbours on both sides: with large initial offsets, k = 1
(nearest neighbours only) can oscillate, k >= 2 converges.
"""
from __future__ import annotations

import numpy as np
import torch

from . import FIT_OK, Level, Mesh, Plan, correspondences, decode, fit_affine, render, render_records, zmodel


def window_grid(h: int, w: int, n: int, stride: int) -> np.ndarray:
    """(y, x) origins of the n x n windows at the given stride, int32 [B, 2]."""
    ys = np.arange(0, h - n + 1, stride)
    xs = np.arange(0, w - n + 1, stride)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([Y.ravel(), X.ravel()], 1).astype(np.int32)


def align_stack(raw: torch.Tensor, level: Level, stride: int, k: int, iters: int, tol: float = 0.0,
                min_snr: float = 0.0, stream=None):
    """Align a uint8 [Z, H, W] CUDA stack.  Returns (aligned uint8 [Z, H, W],
    theta float64 [Z, 6] (model frame -> raw section: p = A q + t), list of
    the median SNR of every iteration).

    Per iteration: the Z models, then every section's grid match (one call per
    section), then one correspondence call and one grouped fit over all
    sections, one read-back of the fit statuses and the match results, and
    the renders.  A section's match and fit depend only on the models built at
    the start of the iteration, so queueing them all before the read-back
    gives the same affines as handling the sections one by one."""
    if raw.dtype != torch.uint8 or raw.dim() != 3 or not raw.is_cuda or not raw.is_contiguous():
        raise TypeError("raw must be a contiguous uint8 [Z, H, W] CUDA tensor")
    Z, H, W = raw.shape
    dev = raw.device
    n = level.n
    org = torch.from_numpy(window_grid(H, W, n, stride)).to(dev)
    B = int(org.shape[0])
    org_all = org.repeat(Z, 1)  # the same grid in every section
    offsets = torch.arange(0, (Z + 1) * B, B, dtype=torch.int64, device=dev)
    plan = Plan([level], dtype="u8", max_windows=B)
    aligned = raw.clone()
    model = torch.empty_like(raw)
    theta = torch.tensor([1.0, 0.0, 0.0, 0.0, 1.0, 0.0], dtype=torch.float64, device=dev).repeat(Z, 1)
    mesh = Mesh(0, 0, max(H, W), 1, 1)
    recs = torch.empty((mesh.n_triangles, 8), dtype=torch.float32, device=dev)
    res = torch.empty((Z, B, 8), dtype=torch.int32, device=dev)
    hist = []
    for _ in range(iters):
        zmodel(aligned, k, out=model, stream=stream)
        for z in range(Z):
            plan.match(model[z], raw[z], org, org, out=res[z], stream=stream)
        q, p, w = correspondences(res.view(Z * B, 8), org_all, org_all, n, min_snr, stream=stream)
        th, st = fit_affine(q, p, w, offsets=offsets, stream=stream)
        if stream is not None:
            stream.synchronize()
        ok = st.cpu().numpy() == FIT_OK  # a degenerate fit keeps the section's previous affine
        d = decode(res.view(Z * B, 8))
        for z in range(Z):
            if ok[z]:
                theta[z] = th[z]
            tri = theta[z].repeat(mesh.n_triangles, 1)
            render_records(tri, mesh, records=recs, stream=stream)
            render(raw[z], tri, mesh, H, W, fill=0.0, out=aligned[z], records=recs, stream=stream)
        good = (d["status"] == 0) & np.isfinite(d["snr"])
        hist.append(float(np.median(d["snr"][good])) if good.any() else 0.0)
        if len(hist) > 1 and abs(hist[-1] - hist[-2]) <= tol * abs(hist[-2]):
            break
    return aligned, theta, hist
