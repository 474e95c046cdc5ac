"""The damaged-pair workload reproduces the shape of the paper's Fig. 2 on the
FP64 oracle (Sec. III): matching a damaged patch against its undamaged
reference gives its strongest SNR at an intermediate whitening exponent,
weaker at both ordinary correlation (w = 0) and phase-only correlation
(w = 1), and ordinary correlation mislocates more often.  The paper's own
numbers (SNR 2.0 / 13.5 / 8.5 at w = 0 / 0.7 / 1) come from an image that is
not available and are not reproduced: this checks the stand-in workload, not
the oracle's arithmetic (its pins are in test_oracle_pins.py)."""
import numpy as np

import synth
from oracle import swim


def test_damaged_pairs_are_reproducible_and_shaped():
    r1, m1, d1 = synth.damaged_pairs(64, 3, 5)
    r2, m2, d2 = synth.damaged_pairs(64, 3, 5)
    assert r1.dtype == np.uint8 and m1.shape == (3, 64, 64) and d1.shape == (3, 2)
    assert (r1 == r2).all() and (m1 == m2).all() and (d1 == d2).all()
    assert (np.abs(d1) <= 24).all()


def test_snr_peaks_at_an_intermediate_exponent():
    n, count = 128, 10
    ref, mov, d = synth.damaged_pairs(n, count, 7)
    med, located = {}, {}
    for w in (0.0, 0.6, 1.0):
        lv = swim.Level(n, w, swim.APOD_HANN, 1.0, 3.0)
        snrs, hits = [], 0
        for i in range(count):
            o = swim.match_pair(mov[i].astype(np.float64), ref[i].astype(np.float64), lv)
            snrs.append(o["snr"])
            hits += abs(o["sy"] - d[i, 0]) <= 1.5 and abs(o["sx"] - d[i, 1]) <= 1.5
        med[w], located[w] = float(np.median(snrs)), hits
    assert med[0.6] > 1.5 * med[0.0] and med[0.6] > 1.3 * med[1.0], med
    assert located[0.6] >= located[0.0] + 2 and located[0.6] >= count - 1, located
