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
"""
from __future__ import annotations

import numpy as np

from . import mir, remod, swim


def grid(h: int, w: int, n: int, stride: int) -> np.ndarray:
    ys = np.arange(0, h - n + 1, stride)
    xs = np.arange(0, w - n + 1, stride)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([Y.ravel(), X.ravel()], 1).astype(np.int32)


def align_stack(raw: np.ndarray, level: swim.Level, stride: int, k: int, iters: int, tol: float = 0.0,
                min_snr: float = 0.0):
    """Returns (aligned uint8 [Z, H, W], theta [Z, 6], median SNR per iteration)."""
    Z, H, W = raw.shape
    n = level.n
    org = grid(H, W, n, stride)
    aligned = raw.copy()
    theta = np.broadcast_to(mir.identity(), (Z, 6)).copy()
    mesh = mir.Mesh(0, 0, max(H, W), 1, 1)
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
