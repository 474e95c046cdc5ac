"""Pins for the FP64 oracle: facts the paper and the mathematics fix.

None of these re-types an oracle formula.  Each one checks the oracle against
something independent of it: a library routine (numpy's FFT, scipy's window
functions), a closed form (the phase-only surface of an exact shift, Parseval),
brute force (spatial circular correlation by explicit sums), or a hand-worked
example stored under ``tests/golden/``.  A dropped term, a sign error, a
swapped axis or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.signal import windows

import synth
from oracle import swim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- #
# transforms
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("n", [8, 16, 64])
def test_dft_equals_library_fft(n):
    x = np.random.default_rng(n).standard_normal((n, n)) + 1j * np.random.default_rng(n + 1).standard_normal((n, n))
    np.testing.assert_allclose(swim.dft2(x), np.fft.fft2(x), rtol=0, atol=1e-9 * n * n)
    np.testing.assert_allclose(swim.idft2(x), np.fft.ifft2(x), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [16, 32])
def test_parseval_and_inverse(n):
    x = np.random.default_rng(3).standard_normal((n, n))
    X = swim.dft2(x)
    assert abs((np.abs(x) ** 2).sum() - (np.abs(X) ** 2).sum() / n ** 2) < 1e-12 * (x ** 2).sum()
    np.testing.assert_allclose(swim.idft2(X).real, x, atol=1e-12)
    np.testing.assert_allclose(swim.idft2(X).imag, 0, atol=1e-12)


def test_single_frequency_is_a_delta():
    n, a, b = 16, 3, 11
    y, x = np.mgrid[0:n, 0:n]
    # e^{+2 pi i (a y + b x)/n} transforms to n^2 at (a, b) under e^{-2 pi i ...}
    X = swim.dft2(np.exp(2j * np.pi * (a * y + b * x) / n))
    expect = np.zeros((n, n), complex)
    expect[a, b] = n * n
    np.testing.assert_allclose(X, expect, atol=1e-9)


# --------------------------------------------------------------------------- #
# apodisation (Sec. III: cosine taper)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("n", [8, 64, 256])
def test_hann_matches_scipy_periodic(n):
    np.testing.assert_allclose(swim.taper_1d(n, swim.APOD_HANN), windows.hann(n, sym=False), atol=1e-15)
    a = swim.taper_1d(n, swim.APOD_HANN)
    assert a[0] == 0.0 and a[n // 2] == 1.0 and abs(a[n // 4] - 0.5) < 1e-15


@pytest.mark.parametrize("alpha", [0.25, 0.5, 1.0])
def test_tukey_matches_scipy_periodic(alpha):
    n = 64
    np.testing.assert_allclose(swim.taper_1d(n, swim.APOD_TUKEY, alpha),
                               windows.tukey(n, alpha, sym=False), atol=1e-14)


def test_apodise_zero_mean_and_affine_equivariance():
    n = 32
    A = swim.taper_2d(n, swim.APOD_HANN)
    x = np.random.default_rng(5).uniform(0, 255, (n, n))
    xp = swim.apodise(x, A)
    assert abs(xp.sum()) < 1e-9
    np.testing.assert_allclose(swim.apodise(3.0 * x + 17.0, A), 3.0 * xp, atol=1e-9)
    # inside the taper's support the window is A * (x - mu): spot value by hand
    mu = (A * x).sum() / A.sum()
    assert abs(xp[7, 9] - A[7, 9] * (x[7, 9] - mu)) < 1e-12


# --------------------------------------------------------------------------- #
# whitening (Sec. III: amplitude power function, phases untouched)
# --------------------------------------------------------------------------- #
def test_whitening_magnitude_and_phase_by_hand():
    C = np.zeros((2, 2), complex)
    C[0, 1] = 4.0 * np.exp(1j * 0.7)
    C[1, 0] = 0.25 * np.exp(-1j * 2.0)
    C[1, 1] = 0.0
    C[0, 0] = 5.0
    G = swim.whiten(C, 0.5)
    assert G[0, 0] == 0  # DC dropped
    assert abs(G[0, 1] - 2.0 * np.exp(1j * 0.7)) < 1e-15   # 4^(1-0.5) = 2
    assert abs(G[1, 0] - 0.5 * np.exp(-1j * 2.0)) < 1e-15  # 0.25^(0.5) = 0.5
    assert G[1, 1] == 0
    G1 = swim.whiten(C, 1.0)
    assert abs(abs(G1[0, 1]) - 1.0) < 1e-15 and abs(abs(G1[1, 0]) - 1.0) < 1e-15
    G0 = swim.whiten(C, 0.0)
    assert G0[0, 1] == C[0, 1] and G0[1, 0] == C[1, 0]


@pytest.mark.parametrize("w", [0.0, 0.35, 0.65, 1.0])
def test_whitening_before_or_after_product_is_equivalent(w):
    """Sec. III: amplitudes may be adjusted before or after the product."""
    n = 32
    ref, mov = synth.noise_pair(n, (2, -5), seed=11)
    A = swim.taper_2d(n, swim.APOD_HANN)
    M = np.fft.fft2(swim.apodise(mov, A))
    R = np.fft.fft2(swim.apodise(ref, A))
    # per-spectrum scaling |F|^-w on each input, DC removed
    before = (M * np.abs(M) ** (-w)) * np.conj(R * np.abs(R) ** (-w))
    before[0, 0] = 0
    after = swim.whiten(M * np.conj(R), w)
    np.testing.assert_allclose(after, before, rtol=1e-12, atol=0)
    # and the whole surface, direct DFT against library FFT of the "before" form
    surf = swim.match_surface(mov, ref, swim.Level(n, w, swim.APOD_HANN))
    np.testing.assert_allclose(surf, np.fft.ifft2(before).real, rtol=0,
                               atol=1e-8 * np.abs(surf).max())


# --------------------------------------------------------------------------- #
# correlation (w = 0) and phase-only (w = 1) special cases
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("n", [8, 16, 32])
def test_w0_equals_bruteforce_circular_correlation(n):
    rng = np.random.default_rng(n)
    mov, ref = rng.uniform(0, 255, (n, n)), rng.uniform(0, 255, (n, n))
    A = swim.taper_2d(n, swim.APOD_HANN)
    m, r = swim.apodise(mov, A), swim.apodise(ref, A)
    brute = np.zeros((n, n))
    for ty in range(n):
        for tx in range(n):
            acc = 0.0
            for by in range(n):
                for bx in range(n):
                    acc += m[(by + ty) % n, (bx + tx) % n] * r[by, bx]
            brute[ty, tx] = acc
    s = swim.match_surface(mov, ref, swim.Level(n, 0.0, swim.APOD_HANN))
    np.testing.assert_allclose(s, brute, atol=1e-12 * np.abs(brute).max())


@pytest.mark.parametrize("d", [(0, 1), (-3, 5), (7, -8), (-16, 15)])
def test_phase_only_of_exact_shift_is_a_delta(d):
    """Sec. III: identical images, one shifted -> a single Dirac pulse at the shift."""
    n = 32
    ref = np.random.default_rng(7).standard_normal((n, n))
    mov = np.roll(ref, d, axis=(0, 1))
    s = swim.match_surface(mov, ref, swim.Level(n, 1.0, swim.APOD_NONE))
    expect = np.full((n, n), -1.0 / n ** 2)
    expect[d[0] % n, d[1] % n] += 1.0
    np.testing.assert_allclose(s, expect, atol=1e-12)


@pytest.mark.parametrize("w", [0.0, 0.35, 0.65, 1.0])
def test_exact_integer_shift_recovered(w):
    n = 64
    rng = np.random.default_rng(int(w * 100) + 1)
    ref = rng.standard_normal((n, n))
    for _ in range(4):
        d = tuple(int(v) for v in rng.integers(-n // 2, n // 2, 2))
        mov = np.roll(ref, d, axis=(0, 1))
        res = swim.match_pair(mov, ref, swim.Level(n, w, swim.APOD_NONE, 1.0, 3.0))
        assert (res["dy"], res["dx"]) == d


def test_noise_pair_worked_example():
    ref, mov = synth.noise_pair(64, (-3, 5))
    res = swim.match_pair(mov, ref, swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0))
    assert (res["dy"], res["dx"]) == (-3, 5)
    assert res["status"] == swim.OK and res["snr"] > 10
    assert abs(res["sy"] + 3) < 0.1 and abs(res["sx"] - 5) < 0.1
    with open(os.path.join(GOLDEN, "noise_pair_64.json")) as f:
        g = json.load(f)
    for k in ("dy", "dx", "status"):
        assert res[k] == g["result"][k]
    for k in ("sy", "sx", "snr", "peak"):
        assert abs(res[k] - g["result"][k]) <= 1e-9 * max(1.0, abs(g["result"][k]))


def test_swap_inputs_negates_shift():
    ref, mov = synth.noise_pair(64, (-3, 5), seed=4)
    lv = swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0)
    a = swim.match_pair(mov, ref, lv)
    b = swim.match_pair(ref, mov, lv)
    assert (b["dy"], b["dx"]) == (-a["dy"], -a["dx"])
    assert abs(a["snr"] - b["snr"]) < 1e-9 * a["snr"]


def test_peak_and_snr_invariant_to_affine_intensity():
    ref, mov = synth.noise_pair(64, (6, -2), seed=9)
    lv = swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0)
    a = swim.match_pair(mov, ref, lv)
    b = swim.match_pair(2.5 * mov + 40.0, 0.3 * ref - 7.0, lv)
    assert (a["dy"], a["dx"]) == (b["dy"], b["dx"])
    assert abs(a["snr"] - b["snr"]) < 1e-9 * a["snr"]
    assert abs(a["sy"] - b["sy"]) < 1e-9 and abs(a["sx"] - b["sx"]) < 1e-9


# --------------------------------------------------------------------------- #
# peak, SNR, subpixel by hand
# --------------------------------------------------------------------------- #
def test_snr_hand_worked():
    with open(os.path.join(GOLDEN, "snr_hand.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        s = np.array(c["surface"], dtype=np.float64)
        py, px = swim.peak_index(s)
        assert [py, px] == c["peak"]
        z, mu, sd = swim.snr(s, py, px, c["radius"])
        assert abs(mu - c["mean_bg"]) < 1e-12
        assert abs(sd - c["std_bg"]) < 1e-12
        assert abs(z - c["snr"]) < 1e-12


def test_background_disc_is_wrapped():
    m = swim.background_mask(5, 0, 0, 1.0)
    excluded = {(int(y), int(x)) for y, x in zip(*np.nonzero(~m))}
    assert excluded == {(0, 0), (0, 1), (1, 0), (0, 4), (4, 0)}


def test_peak_tie_goes_to_first_row_major():
    s = np.zeros((4, 4))
    s[2, 1] = s[1, 3] = s[3, 0] = 1.0
    assert swim.peak_index(s) == (1, 3)
    assert swim.signed_shift(1, 4) == 1 and swim.signed_shift(2, 4) == -2 and swim.signed_shift(3, 4) == -1


@pytest.mark.parametrize("fy,fx", [(0.2, -0.4), (-0.49, 0.0), (0.0, 0.31)])
def test_subpixel_exact_on_sampled_parabola(fy, fx):
    n = 16
    py, px = 5, 15  # px at the right edge exercises the wrap
    y, x = np.mgrid[0:n, 0:n].astype(float)
    dy = (y - py + n / 2) % n - n / 2
    dx = (x - px + n / 2) % n - n / 2
    s = 10.0 - (dy - fy) ** 2 - 2.0 * (dx - fx) ** 2
    assert swim.peak_index(s) == (py, px)
    gy, gx = swim.subpixel(s, py, px)
    assert abs(gy - fy) < 1e-12 and abs(gx - fx) < 1e-12


def test_snr_falls_as_noise_is_added():
    """The SNR is a Z score of the peak against the background (Sec. II), so
    independent noise added to the moving window lowers it in expectation:
    the mean over six seeds falls strictly across noise levels 0.05 to 3 (the
    signal has unit variance)."""
    lv = swim.Level(32, 0.65, swim.APOD_HANN, 1.0, 2.0)
    means = []
    for sigma in (0.05, 0.3, 1.0, 3.0):
        snr = [swim.match_pair(*reversed(synth.noise_pair(32, (2, -3), noise=sigma, seed=s)), lv)["snr"]
               for s in range(6)]
        means.append(float(np.mean(snr)))
    assert all(a > b for a, b in zip(means, means[1:])), means


@pytest.mark.parametrize("w", [0.0, 0.65, 1.0])
def test_band_limited_subpixel_shift_within_parabola_bias(w):
    """Ground truth, not the oracle's own formula: a periodic texture shifted
    by an exact band-limited subpixel amount (a Fourier phase ramp) is found
    at that shift up to the 3-point parabola's bias.  Measured worst cases are
    0.08 / 0.05 / 0.13 px for w = 0 / 0.65 / 1 over these twelve shifts; 0.2 px
    is the bar, far below the ~1 px that a wrong sign or wrap would give."""
    n = 32
    rng = np.random.default_rng(5)
    k = np.fft.fftfreq(n)
    lv = swim.Level(n, w, swim.APOD_NONE, 1.0, 2.0)
    for i in range(12):
        ref, _ = synth.noise_pair(n, (0, 0), noise=0.0, seed=100 + i)
        d = rng.uniform(-4, 4, 2)
        ramp = np.exp(-2j * np.pi * (k[:, None] * d[0] + k[None, :] * d[1]))
        mov = np.fft.ifft2(np.fft.fft2(ref) * ramp).real
        r = swim.match_pair(mov, ref, lv)
        assert abs(r["sy"] - d[0]) < 0.2 and abs(r["sx"] - d[1]) < 0.2, (w, d, r["sy"], r["sx"])


# --------------------------------------------------------------------------- #
# window sources
# --------------------------------------------------------------------------- #
def test_projection_and_resampling_special_cases():
    rng = np.random.default_rng(2)
    secs = rng.integers(0, 256, (3, 40, 50)).astype(np.uint8)
    o = (5, 7)
    n = 16
    np.testing.assert_array_equal(swim.project(secs[:1], o, n), secs[0, 5:21, 7:23])
    np.testing.assert_allclose(swim.project(secs, o, n),
                               secs[:, 5:21, 7:23].astype(float).sum(0) / 3.0)
    ident = (1, 0, 0, 0, 1, 0)
    np.testing.assert_allclose(swim.resample(secs[1], o, n, ident), secs[1, 5:21, 7:23])
    shifted = (1, 0, 2, 0, 1, -3)
    np.testing.assert_allclose(swim.resample(secs[1], o, n, shifted), secs[1, 7:23, 4:20])
    # bilinear interpolation reproduces a linear ramp exactly
    yy, xx = np.mgrid[0:40, 0:50]
    ramp = 3.0 * yy - 2.0 * xx + 1.0
    th = (math.cos(0.1), -math.sin(0.1), 0.37, math.sin(0.1), math.cos(0.1), -0.61)
    Y, X = swim.affine_sample_points(o, n, th)
    np.testing.assert_allclose(swim.bilinear(ramp, Y, X), 3.0 * Y - 2.0 * X + 1.0, atol=1e-9)
    assert swim.resample(secs[1], (30, 40), n, ident) is None


def test_status_codes():
    lv = swim.Level(16, 0.65, swim.APOD_HANN)
    flat = np.full((16, 16), 7.0)
    rnd = np.random.default_rng(0).standard_normal((16, 16))
    assert swim.match_pair(flat, rnd, lv)["status"] == swim.FLAT
    assert swim.match_pair(rnd, flat, lv)["status"] == swim.FLAT
    bad = rnd.copy()
    bad[3, 3] = np.nan
    assert swim.match_pair(bad, rnd, lv)["status"] == swim.NONFINITE
    sec = np.zeros((20, 20), np.uint8)
    r = swim.match_batch([sec], [sec], np.array([[10, 0]]), np.array([[0, 0]]), [lv])
    assert r[0]["status"] == swim.OUT_OF_BOUNDS
