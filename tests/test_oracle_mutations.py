"""Planted mistakes in the oracle must be caught by its pins.

Each case swaps one oracle function for a plausibly wrong version (on the CPU,
inside this process only) and checks that at least one pin in
``test_oracle_pins`` then fails.  This is evidence that the pins constrain the
oracle rather than restate it.
"""
import numpy as np
import pytest

from oracle import swim
import test_oracle_pins as pins


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _whiten_wrong_sign(C, w):
    mag = np.abs(C)
    G = np.zeros_like(C)
    nz = mag > 0
    G[nz] = C[nz] * mag[nz] ** (+w)
    G[0, 0] = 0
    return G


def _whiten_keeps_dc(C, w):
    mag = np.abs(C)
    G = np.zeros_like(C)
    nz = mag > 0
    G[nz] = C[nz] * mag[nz] ** (-w)
    return G


def _surface_conj_wrong_operand(mov_w, ref_w, level):
    A = swim.taper_2d(level.n, level.apod, level.tukey_alpha)
    C = np.conj(swim.dft2(swim.apodise(mov_w, A))) * swim.dft2(swim.apodise(ref_w, A))
    return swim.idft2(swim.whiten(C, level.whiten_exponent)).real


def _apodise_no_mean(x, A):
    return A * np.asarray(x, dtype=np.float64)


def _dft2_transposed(x):
    F = swim.dft_matrix(x.shape[0])
    return F @ x.T @ F.T


def _idft2_unnormalised(X):
    Fi = np.conj(swim.dft_matrix(X.shape[0]))
    return Fi @ X @ Fi.T


def _snr_sample_std(s, py, px, radius):
    bg = s[swim.background_mask(s.shape[0], py, px, radius)]
    mu = float(bg.mean())
    sd = float(bg.std(ddof=1))
    return (float(s[py, px]) - mu) / sd, mu, sd


def _mask_unwrapped(n, py, px, radius):
    d = np.arange(n)
    dy = np.abs(d - py).astype(float)
    dx = np.abs(d - px).astype(float)
    return (dy[:, None] ** 2 + dx[None, :] ** 2) > radius * radius


def _parabola_wrong_sign(sm, s0, sp):
    den = sm - 2.0 * s0 + sp
    if not den < 0.0:
        return 0.0
    return min(0.5, max(-0.5, 0.5 * (sp - sm) / den))


def _taper_symmetric(n, apod, alpha=1.0):
    k = np.arange(n, dtype=np.float64)
    if apod == swim.APOD_NONE:
        return np.ones(n)
    return 0.5 * (1.0 - np.cos(2.0 * np.pi * k / (n - 1)))


def _peak_last_tie(s):
    flat = s.ravel()
    i = len(flat) - 1 - int(np.argmax(flat[::-1]))
    return divmod(i, s.shape[1])


MUTATIONS = [
    ("whiten", _whiten_wrong_sign, [(pins.test_phase_only_of_exact_shift_is_a_delta, (0, 1))]),
    ("whiten", _whiten_keeps_dc, [(pins.test_whitening_magnitude_and_phase_by_hand, None)]),
    ("match_surface", _surface_conj_wrong_operand, [(pins.test_noise_pair_worked_example, None)]),
    ("apodise", _apodise_no_mean, [(pins.test_apodise_zero_mean_and_affine_equivariance, None)]),
    ("dft2", _dft2_transposed, [(pins.test_dft_equals_library_fft, 8)]),
    ("idft2", _idft2_unnormalised, [(pins.test_dft_equals_library_fft, 8)]),
    ("snr", _snr_sample_std, [(pins.test_snr_hand_worked, None)]),
    ("background_mask", _mask_unwrapped, [(pins.test_background_disc_is_wrapped, None)]),
    ("parabola_offset", _parabola_wrong_sign, [(pins.test_subpixel_exact_on_sampled_parabola, (0.2, -0.4))]),
    ("taper_1d", _taper_symmetric, [(pins.test_hann_matches_scipy_periodic, 64)]),
    ("peak_index", _peak_last_tie, [(pins.test_peak_tie_goes_to_first_row_major, None)]),
]


@pytest.mark.parametrize("name,bad,checks", MUTATIONS, ids=[f"{m[0]}:{m[1].__name__}" for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, bad, checks):
    # the pins must pass on the real oracle first
    for fn, arg in checks:
        args = () if arg is None else (arg if isinstance(arg, tuple) and fn.__code__.co_argcount == len(arg) else (arg,))
        fn(*args)
    monkeypatch.setattr(swim, name, bad)
    caught = False
    for fn, arg in checks:
        args = () if arg is None else (arg if isinstance(arg, tuple) and fn.__code__.co_argcount == len(arg) else (arg,))
        caught |= _fails(fn, *args)
    assert caught, f"planted mistake in {name} not caught"
