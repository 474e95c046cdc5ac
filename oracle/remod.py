"""FP64 / exact-integer oracle of SWiFT-IR's pyramid and model steps ("iscale"
and "remod", Sec. III module list and model averaging).

TEST INFRASTRUCTURE ONLY.  Like the other oracle modules it is the slow,
plainly written reference the CUDA library is checked against; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` may
use it, and it shares no code with the CUDA path.

The paper's description:

* iscale produces the hierarchical source pyramid, usually by powers of 2,
  with factors 3 and 5 also useful (Sec. III, module list);
* remod generates locally Z-averaged models (Sec. III, module list): the
  reference for a section is the average of its aligned neighbours, which
  reduces noise as 1/sqrt(N) and smooths geometry along Z; the current
  section and damaged sections are left out (Sec. III, model averaging).

Readings where the paper is silent (also listed with the design notes):

* iscale: output (y, x) is the mean of the f x f input block at
  (f y, f x); the partial blocks at the right and bottom edges are dropped
  (output floor(H/f) x floor(W/f)); uint8 output rounds the exact mean half
  to even (integer arithmetic), float32 output is the float32 sum of the
  block divided by f^2 in float32;
* remod: the model of section z is the mean of the valid sections
  j in [z - k, z + k], j != z, clipped to the stack; float32 output is
  float32(integer sum) / float32(count) (one correctly rounded division),
  uint8 output the exact mean rounded half to even; with no valid neighbour
  the model is the section itself.
"""
from __future__ import annotations

import numpy as np


def downsample(img: np.ndarray, f: int) -> np.ndarray:
    """f x f box mean (uint8: exact, rounded half to even; float32: float32)."""
    h, w = img.shape
    H, W = h // f, w // f
    if img.dtype == np.uint8:
        out = np.zeros((H, W), np.uint8)
        d = f * f
        for y in range(H):
            for x in range(W):
                s = int(img[f * y:f * y + f, f * x:f * x + f].astype(np.int64).sum())
                q, r = divmod(s, d)
                if 2 * r > d or (2 * r == d and q % 2 == 1):
                    q += 1
                out[y, x] = q
        return out
    v = img[:H * f, :W * f].astype(np.float32).reshape(H, f, W, f)
    s = np.zeros((H, W), np.float32)
    for i in range(f):  # float32 sum in row-major order within the block
        for j in range(f):
            s = s + v[:, i, :, j]
    return (s / np.float32(f * f)).astype(np.float32)


def zmodel(stack: np.ndarray, k: int, valid=None, dtype=np.float32) -> np.ndarray:
    """Model of every section of a uint8 [Z, H, W] stack: float32 [Z, H, W],
    or uint8 (the exact mean rounded half to even) with dtype=np.uint8."""
    Z = stack.shape[0]
    valid = np.ones(Z, bool) if valid is None else np.asarray(valid, bool)
    out = np.zeros(stack.shape, dtype)
    for z in range(Z):
        js = [j for j in range(max(0, z - k), min(Z, z + k + 1)) if j != z and valid[j]]
        if not js:
            out[z] = stack[z]
            continue
        s = sum(stack[j].astype(np.int64) for j in js)
        if dtype == np.uint8:
            c = len(js)
            q, r = np.divmod(s, c)
            q = q + ((2 * r > c) | ((2 * r == c) & (q % 2 == 1)))
            out[z] = q.astype(np.uint8)
        else:
            out[z] = s.astype(np.float32) / np.float32(len(js))
    return out
