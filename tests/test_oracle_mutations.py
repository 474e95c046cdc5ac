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


# --------------------------------------------------------------------------- #
# the rendering step (mir)
# --------------------------------------------------------------------------- #
from oracle import mir  # noqa: E402
import test_oracle_mir as mir_pins  # noqa: E402


def _fit_unweighted_means(q, p, w):
    q = np.asarray(q, dtype=np.float64).reshape(-1, 2)
    p = np.asarray(p, dtype=np.float64).reshape(-1, 2)
    w = np.asarray(w, dtype=np.float64).reshape(-1)
    if not w.sum() > 0:
        return mir.identity(), mir.DEGENERATE
    qb, pb = q.mean(0), p.mean(0)  # plain means instead of weighted ones
    dq, dp = q - qb, p - pb
    Sqq = (w[:, None, None] * dq[:, :, None] * dq[:, None, :]).sum(0)
    Cpq = (w[:, None, None] * dp[:, :, None] * dq[:, None, :]).sum(0)
    det = np.linalg.det(Sqq)
    if not det > mir.DET_EPS * (0.5 * np.trace(Sqq)) ** 2:
        return mir.identity(), mir.DEGENERATE
    A = Cpq @ np.linalg.inv(Sqq)
    t = pb - A @ qb
    return np.array([A[0, 0], A[0, 1], t[0], A[1, 0], A[1, 1], t[1]]), mir.OK


def _fit_transposed(q, p, w):
    th, st = _REAL_FIT(q, p, w)
    return th[[0, 3, 2, 1, 4, 5]], st  # A^T instead of A


_REAL_FIT = mir.fit_affine


class _MeshFlippedDiagonal(mir.Mesh):
    def locate(self, y, x):
        t = super().locate(y, x)
        return t ^ 1


class _MeshEuclideanBand(mir.Mesh):
    def supports(self, t, q, band):
        q = np.asarray(q, dtype=np.float64)
        _, _, half, y0, x0 = self.triangle(t)
        c = self.cell
        dy, dx = q[:, 0] - y0, q[:, 1] - x0
        box = (dy >= -band) & (dy <= c + band) & (dx >= -band) & (dx <= c + band)
        diag = (dx - dy >= -band) if half == 0 else (dy - dx >= -band)  # grows the diagonal by b, not 2b
        return box & diag


def _bilinear_swapped(src, Y, X, fill):
    h, w = src.shape
    inside = (Y >= 0) & (X >= 0) & (Y <= h - 1) & (X <= w - 1)
    Yc, Xc = np.where(inside, Y, 0.0), np.where(inside, X, 0.0)
    y0 = np.minimum(np.floor(Yc).astype(np.int64), h - 2)
    x0 = np.minimum(np.floor(Xc).astype(np.int64), w - 2)
    fx, fy = Yc - y0, Xc - x0  # fractions swapped between the axes
    S = src.astype(np.float64)
    v = ((1 - fy) * (1 - fx) * S[y0, x0] + (1 - fy) * fx * S[y0, x0 + 1]
         + fy * (1 - fx) * S[y0 + 1, x0] + fy * fx * S[y0 + 1, x0 + 1])
    return np.where(inside, v, fill)


MIR_MUTATIONS = [
    ("fit_affine", _fit_unweighted_means, [mir_pins.test_fit_matches_weighted_lstsq]),
    ("fit_affine", _fit_transposed, [mir_pins.test_fit_recovers_a_known_affine_exactly]),
    ("Mesh", _MeshFlippedDiagonal, [mir_pins.test_locate_puts_every_pixel_in_its_triangle]),
    ("Mesh", _MeshEuclideanBand, [mir_pins.test_supports_equal_brute_force_chebyshev_distance]),
    ("bilinear_fill", _bilinear_swapped, [mir_pins.test_render_identity_translation_and_linear_images]),
]


@pytest.mark.parametrize("name,bad,checks", MIR_MUTATIONS, ids=[f"{m[0]}:{m[1].__name__}" for m in MIR_MUTATIONS])
def test_planted_mir_mistake_is_caught(monkeypatch, name, bad, checks):
    for fn in checks:
        fn()
    monkeypatch.setattr(mir, name, bad)
    assert any(_fails(fn) for fn in checks), f"planted mistake in mir.{name} not caught"
