"""The oracle's analytic adjoint against central finite differences (FP64).

The argmax is held fixed (the objective is the envelope the adjoint
differentiates); sample coordinates stay at least 0.05 px away from integers,
where bilinear resampling is not differentiable.
"""
import math

import numpy as np
import pytest

import synth
from oracle import swim


def _case(n, seed, w, apod=swim.APOD_HANN):
    stack = synth.section_stack(160, depth=3, seed=seed)
    sec = stack[1].astype(np.float64)
    ref = stack[0].astype(np.float64)[40:40 + n, 40:40 + n]
    th = synth.affine_params(1, seed=seed + 7, max_offset=1.5, max_rot_deg=0.5)[0].astype(np.float64)
    return sec, (40, 40), th, ref, swim.Level(n, w, apod, 1.0, 2.0)


@pytest.mark.parametrize("w", [0.0, 0.5, 0.9])
@pytest.mark.parametrize("gp,gs", [(1.0, 0.0), (0.0, 1.0), (-0.7, 0.3)])
def test_adjoint_matches_finite_differences(w, gp, gs):
    n = 32
    sec, org, th, ref, lv = _case(n, 3, w)
    fwd, gth, gw = swim.match_backward(sec, org, th, ref, lv, gp, gs)
    pk = (fwd["dy"] % n, fwd["dx"] % n)
    f = lambda t, lvl=lv: swim.affine_objective(sec, org, t, ref, lvl, gp, gs, peak_at=pk)  # noqa: E731
    h = 1e-6
    for k in range(6):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (f(tp) - f(tm)) / (2 * h)
        assert abs(gth[k] - fd) <= 1e-5 * max(1.0, abs(fd)), (k, gth[k], fd)
    lp = swim.Level(n, w + h, lv.apod, lv.tukey_alpha, lv.snr_exclusion_radius)
    lm = swim.Level(n, w - h, lv.apod, lv.tukey_alpha, lv.snr_exclusion_radius)
    fdw = (f(th, lp) - f(th, lm)) / (2 * h)
    assert abs(gw - fdw) <= 1e-5 * max(1.0, abs(fdw)), (gw, fdw)


def test_adjoint_forward_agrees_with_match_pair():
    n = 32
    sec, org, th, ref, lv = _case(n, 5, 0.65)
    fwd, _, _ = swim.match_backward(sec, org, th, ref, lv, 1.0, 1.0)
    res = swim.match_pair(swim.resample(sec, org, n, th), ref, lv)
    assert (fwd["dy"], fwd["dx"]) == (res["dy"], res["dx"])
    assert math.isclose(fwd["snr"], res["snr"], rel_tol=1e-12)
    assert math.isclose(fwd["peak"], res["peak"], rel_tol=1e-12)


def test_translation_gradient_points_toward_the_match():
    """Moving a pure translation toward the true offset raises the peak."""
    n = 32
    stack = synth.section_stack(160, depth=2, seed=11)
    sec = stack[0].astype(np.float64)
    ref = sec[50:50 + n, 50:50 + n]
    lv = swim.Level(n, 0.5, swim.APOD_HANN, 1.0, 2.0)
    th = np.array([1.0, 0.0, 0.35, 0.0, 1.0, -0.3])  # true offset is (0, 0)
    _, g, _ = swim.match_backward(sec, (50, 50), th, ref, lv, 1.0, 0.0)
    assert g[2] < 0 and g[5] > 0  # d(peak)/dt_y < 0 at t_y > 0; > 0 at t_x < 0
