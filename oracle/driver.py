"""FP64 oracle of SWiFT-IR's outer registration loop (Sec. IV): match,
render and remodel at one resolution until the swim SNR stops changing.

TEST INFRASTRUCTURE ONLY (see ``oracle.swim``): it composes the oracle's own
steps, ``remod.zmodel`` -> ``swim.match_pair`` per window -> ``mir`` fit and
render, and shares no code with the CUDA path.

The paper's description: the main workflow aligns iteratively at the current
working resolution until the SNR scores stabilise, the model being the local
Z average of the aligned sections; at low resolution one affine per section
suffices (Sec. IV).

Readings where the paper is silent (also listed with the design notes):

* one iteration: uint8 models of the current aligned stack (k neighbours
  each way, the section itself excluded, the exact mean rounded half to
  even); every raw section is matched against its
  model on a regular grid of windows (reference = model, moving = raw);
  the SNR-weighted least-squares affine maps the model frame to the raw
  section; the raw section is rendered through it (uint8, fill 0);
* a section whose fit is degenerate keeps its previous affine;
* convergence: the median SNR of the OK windows of the iteration changes by
  at most ``tol`` (relative) from the previous iteration, or ``iters``
  iterations have run.

The paper then advances to the next higher resolution "by first expanding
the current model" (Sec. IV).  Readings for ``align_pyramid``:

* the pyramid is the box-mean (iscale) downsampling of the raw stack by
  factors f_0 > f_1 > ... > 1, each a multiple of the next;
* a coarse pixel centre u stands for the fine coordinate r u + (r - 1) / 2
  (r = f_coarse / f_fine: the centre of its r x r box), so an affine
  p = A q + t found at the coarse level becomes A q + (r t + (r - 1)/2 (1 - A 1))
  at the finer one (same A, 1 = (1, 1));
* "expanding the model": the finer level starts from the expanded affines --
  its raw sections are rendered through them before its first models are
  made -- and then iterates as at one resolution;
* before the expansion the stack's common translation (the mean of the
  sections' t) is removed: the alignment is relative, and a common drift would
  only widen the fill borders that the finer level's models carry (border
  windows then lock onto the fill edge instead of the content).
"""
from __future__ import annotations

import numpy as np

from . import mir, remod, swim


def grid(h: int, w: int, n: int, stride: int, margin: int = 0) -> np.ndarray:
    """(y, x) origins of the n x n windows at the given stride, at least
    ``margin`` px inside every border."""
    ys = np.arange(margin, h - n - margin + 1, stride)
    xs = np.arange(margin, w - n - margin + 1, stride)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([Y.ravel(), X.ravel()], 1).astype(np.int32)


def expand_affine(theta: np.ndarray, r: int) -> np.ndarray:
    """Affines [Z, 6] (a_yy, a_yx, t_y, a_xy, a_xx, t_x) of a level r times
    coarser, in the finer level's pixel coordinates (coarse centre u = fine
    r u + (r - 1) / 2)."""
    th = np.array(theta, dtype=np.float64, copy=True).reshape(-1, 6)
    c = (r - 1) / 2.0
    ty = r * th[:, 2] + c * (1.0 - th[:, 0] - th[:, 1])
    tx = r * th[:, 5] + c * (1.0 - th[:, 3] - th[:, 4])
    th[:, 2], th[:, 5] = ty, tx
    return th


def align_stack(raw: np.ndarray, level: swim.Level, stride: int, k: int, iters: int, tol: float = 0.0,
                min_snr: float = 0.0, theta0=None, margin: int = 0):
    """Returns (aligned uint8 [Z, H, W], theta [Z, 6], median SNR per iteration).
    ``theta0`` ([Z, 6]): start from these affines (the raw sections rendered
    through them) instead of the identity; ``margin``: the window grid keeps
    that many px from every border."""
    Z, H, W = raw.shape
    n = level.n
    org = grid(H, W, n, stride, margin)
    mesh = mir.Mesh(0, 0, max(H, W), 1, 1)
    if theta0 is None:
        aligned = raw.copy()
        theta = np.broadcast_to(mir.identity(), (Z, 6)).copy()
    else:
        theta = np.array(theta0, dtype=np.float64).reshape(Z, 6).copy()
        aligned = np.stack([mir.to_u8(mir.render(raw[z], np.stack([theta[z], theta[z]]), mesh, H, W, 0.0))
                            for z in range(Z)])
    hist = []
    for _ in range(iters):
        model = remod.zmodel(aligned, k, dtype=np.uint8)
        snrs = []
        for z in range(Z):
            res = [swim.match_pair(swim.gather(raw[z], o, n), swim.gather(model[z], o, n), level) for o in org]
            q, p, w = mir.correspondences(res, org, org, n, min_snr)
            th, st = mir.fit_affine(q, p, w)
            if st == mir.OK:
                theta[z] = th
            aligned[z] = mir.to_u8(mir.render(raw[z], np.stack([theta[z], theta[z]]), mesh, H, W, 0.0))
            snrs.extend(r["snr"] for r in res if r["status"] == swim.OK and np.isfinite(r["snr"]))
        hist.append(float(np.median(snrs)) if snrs else 0.0)
        if len(hist) > 1 and abs(hist[-1] - hist[-2]) <= tol * abs(hist[-2]):
            break
    return aligned, theta, hist


def align_pyramid(raw: np.ndarray, factors, levels, strides, k: int, iters, tol=0.0, min_snr: float = 0.0,
                  margins=0):
    """Coarse-to-fine registration: ``factors`` decreasing to 1 (each a
    multiple of the next), one matching level, window stride, iteration cap,
    tolerance and grid margin per factor (``iters`` / ``tol`` / ``margins`` may
    be single numbers).
    Returns (aligned uint8 [Z, H, W] at full resolution, theta [Z, 6] in full-
    resolution pixels, list of the per-level median-SNR histories)."""
    factors = list(factors)
    if factors[-1] != 1 or any(factors[i] % factors[i + 1] for i in range(len(factors) - 1)):
        raise ValueError("factors must decrease to 1, each a multiple of the next")
    L = len(factors)
    iters = list(iters) if np.ndim(iters) else [int(iters)] * L
    tol = list(tol) if np.ndim(tol) else [float(tol)] * L
    margins = list(margins) if np.ndim(margins) else [int(margins)] * L
    theta, hists, aligned = None, [], None
    for i, (f, lv, st) in enumerate(zip(factors, levels, strides)):
        stack = raw if f == 1 else np.stack([remod.downsample(s, f) for s in raw])
        if theta is not None:
            theta = theta.copy()
            theta[:, [2, 5]] -= theta[:, [2, 5]].mean(0)
            theta = expand_affine(theta, factors[i - 1] // f)
        aligned, theta, hist = align_stack(stack, lv, st, k, iters[i], tol[i], min_snr, theta0=theta,
                                           margin=margins[i])
        hists.append(hist)
    return aligned, theta, hists
