"""Shared helpers for the GPU-vs-oracle parity tests.

Tolerances (the block-matching targets): integer peak bit-exact, subpixel
shift within 0.02 px, SNR within 1e-3 relative.  A window is "ambiguous" when
the oracle's best value at any other pixel is within 1e-4 * std_bg of its
peak: FP32 and FP64 rounding may then legitimately pick different maxima, so
the GPU's peak must only be one of those near-tied pixels, and its other
outputs are not compared.
"""
from __future__ import annotations

import numpy as np

from oracle import swim

SUBPIXEL_TOL = 0.02
SNR_RTOL = 1e-3
PEAK_RTOL = 1e-3
AMBIGUITY = 1e-4


def oracle_window(mov_w, ref_w, level):
    res, s = swim.match_pair(mov_w, ref_w, level, return_surface=True)
    tied = None
    if s is not None:
        py, px = swim.peak_index(s)
        _, _, sd = swim.snr(s, py, px, level.snr_exclusion_radius)
        thr = s[py, px] - AMBIGUITY * sd
        ys, xs = np.nonzero(s >= thr)
        tied = {(int(y), int(x)) for y, x in zip(ys, xs)}
    return res, tied


def compare(gpu: dict, i: int, ref: dict, tied, n: int, where: str = ""):
    """Assert GPU window i agrees with the oracle's result dict; returns 'ambiguous' or 'exact'."""
    g = {k: gpu[k][i] for k in gpu}
    assert int(g["status"]) == ref["status"], f"{where} window {i}: status {g['status']} vs {ref['status']}"
    if ref["status"] != swim.OK:
        return "status"
    gp = (int(g["dy"]) % n, int(g["dx"]) % n)
    rp = (ref["dy"] % n, ref["dx"] % n)
    if tied is not None and len(tied) > 1:
        assert gp in tied, f"{where} window {i}: peak {gp} not among near-tied oracle maxima {sorted(tied)[:8]}"
        return "ambiguous"
    assert gp == rp, f"{where} window {i}: integer peak {gp} vs oracle {rp}"
    assert abs(float(g["sy"]) - ref["sy"]) <= SUBPIXEL_TOL, f"{where} window {i}: sy {g['sy']} vs {ref['sy']}"
    assert abs(float(g["sx"]) - ref["sx"]) <= SUBPIXEL_TOL, f"{where} window {i}: sx {g['sx']} vs {ref['sx']}"
    if np.isfinite(ref["snr"]):
        assert abs(float(g["snr"]) - ref["snr"]) <= SNR_RTOL * abs(ref["snr"]), \
            f"{where} window {i}: snr {g['snr']} vs {ref['snr']}"
    assert abs(float(g["peak"]) - ref["peak"]) <= PEAK_RTOL * abs(ref["peak"]) + 1e-6, \
        f"{where} window {i}: peak {g['peak']} vs {ref['peak']}"
    return "exact"
