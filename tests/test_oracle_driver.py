"""Pin of the registration-loop oracle against physical truth: identical
sections (independent noise) displaced by known integer offsets are brought
into one frame; the recovered translations equal the offsets up to one
common translation, and the median SNR rises and settles."""
import numpy as np

import synth
from oracle import driver, swim


def test_known_offsets_are_recovered_up_to_a_common_translation():
    base = synth.section_stack(320, depth=4, seed=12, drift=0.0, radius_jitter=0.0)
    offs = np.array([[0, 0], [4, -3], [-2, 5], [3, 2]])
    # section z shows the content of base position P at P - 32 - offs[z] (crops, no wrap)
    raw = np.stack([base[z, 32 + dy:288 + dy, 32 + dx:288 + dx] for z, (dy, dx) in enumerate(offs)])
    lv = swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0)
    aligned, theta, hist = driver.align_stack(raw, lv, stride=48, k=3, iters=6)
    t = theta[:, [2, 5]]  # raw position of model position q: q + t, so t = -offs + common
    rel = (t - t.mean(0)) + (offs - offs.mean(0))
    assert np.abs(rel).max() < 0.3, rel
    np.testing.assert_allclose(theta[:, [0, 1, 3, 4]], np.broadcast_to([1, 0, 0, 1], (4, 4)), atol=3e-3)
    assert hist[-1] > 2 * hist[0]  # the model sharpens as the sections come into register
    assert abs(hist[-1] - hist[-2]) < 0.05 * hist[-1]  # and the SNR settles


def test_convergence_rule_stops_early():
    base = synth.section_stack(128, depth=3, seed=13, drift=0.0, radius_jitter=0.0)
    lv = swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0)
    _, _, hist = driver.align_stack(base, lv, stride=32, k=2, iters=8, tol=0.5)
    assert len(hist) == 2  # already aligned: the second iteration changes the SNR by less than 50 %
