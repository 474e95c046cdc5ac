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


def test_expand_affine_maps_box_centres():
    """A coarse pixel centre u is the centre of an r x r box of fine pixels,
    fine coordinate r u + (r - 1) / 2.  The expanded affine must send the fine
    image of every coarse point q to the fine image of A q + t (brute force
    over random affines and points, r = 2, 3, 4)."""
    rng = np.random.default_rng(4)
    for r in (2, 3, 4):
        th = rng.normal(0, 1, (5, 6))
        th[:, [0, 4]] += 1.0
        ex = driver.expand_affine(th, r)
        c = (r - 1) / 2.0
        for z in range(5):
            q = rng.uniform(-50, 50, (20, 2))
            p = np.stack([th[z, 0] * q[:, 0] + th[z, 1] * q[:, 1] + th[z, 2],
                          th[z, 3] * q[:, 0] + th[z, 4] * q[:, 1] + th[z, 5]], 1)
            qf, pf = r * q + c, r * p + c
            got = np.stack([ex[z, 0] * qf[:, 0] + ex[z, 1] * qf[:, 1] + ex[z, 2],
                            ex[z, 3] * qf[:, 0] + ex[z, 4] * qf[:, 1] + ex[z, 5]], 1)
            np.testing.assert_allclose(got, pf, atol=1e-9)
        assert np.array_equal(ex[:, [0, 1, 3, 4]], th[:, [0, 1, 3, 4]])


def pyramid_stack(size, depth, offs, seed):
    """Identical EM-like sections (independent noise) cropped at known offsets."""
    base = synth.section_stack(size + 128, depth=depth, seed=seed, drift=0.0, radius_jitter=0.0)
    return np.stack([base[z, 64 + dy:64 + dy + size, 64 + dx:64 + dx + size] for z, (dy, dx) in enumerate(offs)])


# factors, matching levels, strides, iteration caps, tolerances and margins of a three-level run
PYRAMID = dict(factors=[4, 2, 1], sizes=[64, 64, 128], strides=[16, 32, 64], iters=[8, 3, 3], tol=[0.0, 0.01, 0.01],
               margins=[0, 8, 24], k=2)


def test_pyramid_recovers_offsets_beyond_one_level():
    """Offsets up to 40 px at full resolution: the 4x level brings them within
    a few px, the 2x and full levels refine them; the translations come back
    within 0.3 px of the offsets (up to one common translation)."""
    offs = np.random.default_rng(3).integers(-40, 41, (4, 2))
    raw = pyramid_stack(512, 4, offs, seed=31)
    P = PYRAMID
    lvs = [swim.Level(n, 0.65, swim.APOD_HANN, 1.0, 3.0) for n in P["sizes"]]
    aligned, theta, hists = driver.align_pyramid(raw, P["factors"], lvs, P["strides"], P["k"], P["iters"], P["tol"],
                                                 margins=P["margins"])
    t = theta[:, [2, 5]]
    assert np.abs((t - t.mean(0)) + (offs - offs.mean(0))).max() < 0.3
    assert len(hists) == 3 and len(hists[0]) == 8
    assert hists[0][-1] > 1.5 * hists[0][0]  # the coarse level pulls the stack into register
    assert aligned.shape == raw.shape and aligned.dtype == np.uint8
