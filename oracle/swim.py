"""FP64 oracle of the SWiFT-IR block-matching step ("swim", Sec. III).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plainly written reference
that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library itself never calls it and has no CPU fallback.  It shares no
code with the CUDA path: its inputs come from the ``synth`` generators or from
the tests, never from the GPU.

Every step follows the paper's description of the matching step in order:

* tiling into local windows                            (Sec. III, FFT size)
* cosine-taper apodisation against wrap-around          (Sec. III, apodization)
* forward 2D transforms of both windows                 (Sec. III, FFT correlation; Sec. II)
* frequency-domain product with amplitude whitening by
  a 0..1 power-law exponent, phases untouched           (Sec. III, Javidi power scaling)
* inverse transform to the pixel-level match response   (Sec. III, Fig. 2)
* peak position = relative shift                        (Sec. III, Dirac pulse of POC)
* SNR = Z score of the peak against the background      (Sec. III, Fig. 2 discussion)
* subpixel peak position (the paper does not say how; a separable 3-point
  parabola is this library's reading)
* the reference may be a mean "model" of K neighbouring sections (Sec. III)
* the moving window may be resampled under an affine warp (Sec. III, mir's
  locally affine triangles; used here as a differentiable window transform)

Transforms are direct DFTs, X = F x F^T with F[k, n] = exp(-2 pi i k n / N)
built in FP64, not FFTs: the definition written out.  ``numpy`` matrix
products are the only library step.

Readings where the paper is silent (all also listed with the project's design
notes):
  * whitening: G = C |C|^(-w) with C = M conj(R); w = 0 is plain correlation,
    w = 1 phase-only.  G[0,0] = 0 and G = 0 where |C| = 0.
  * mean: weighted mean removal before the taper, x' = A (x - sum(A x)/sum(A)),
    so the DC term of every apodised window is exactly zero.
  * taper: Tukey(alpha) built from a periodic cosine; Hann = Tukey(1).
  * correlation is circular; the inverse transform carries 1/N^2, so an exact
    circular shift under phase-only matching gives delta(tau - d) - 1/N^2.
  * peak ties: smallest row-major index.  Shift range [-N/2, N/2).
  * SNR background: pixels whose wrapped Euclidean distance to the peak is
    greater than the exclusion radius; population standard deviation.
  * subpixel: separable 3-point parabola on the wrapped neighbours; offset 0
    when the parabola is not concave; clamped to [-1/2, 1/2].
  * flat window (all pixels equal in either input): status FLAT, outputs 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# per-window status codes (same meaning as the library's result status)
OK = 0
OUT_OF_BOUNDS = 1
FLAT = 2
NONFINITE = 3

APOD_NONE = 0
APOD_HANN = 1
APOD_TUKEY = 2


@dataclass
class Level:
    """One matching configuration: window side, whitening, taper, SNR radius."""
    n: int
    whiten_exponent: float = 0.65
    apod: int = APOD_HANN
    tukey_alpha: float = 1.0
    snr_exclusion_radius: float = 3.0


# --------------------------------------------------------------------------- #
# apodisation (Sec. III: a cosine taper, keeps more interior than Blackman)
# --------------------------------------------------------------------------- #
def taper_1d(n: int, apod: int, alpha: float = 1.0) -> np.ndarray:
    """1D taper a[0..n-1] in FP64.

    NONE: all ones.  TUKEY(alpha): flat top with raised-cosine ramps of
    alpha*n/2 samples at each side, periodic convention (a[0] = 0 for
    alpha > 0).  HANN is TUKEY(1): a[k] = (1 - cos(2 pi k / n)) / 2.
    """
    k = np.arange(n, dtype=np.float64)
    if apod == APOD_NONE:
        return np.ones(n)
    if apod == APOD_HANN:
        alpha = 1.0
    if not (0.0 < alpha <= 1.0):
        raise ValueError("tukey alpha must be in (0, 1]")
    ramp = alpha * n / 2.0
    a = np.ones(n)
    lo = k < ramp
    hi = k > n - ramp
    a[lo] = 0.5 * (1.0 - np.cos(np.pi * k[lo] / ramp))
    a[hi] = 0.5 * (1.0 - np.cos(np.pi * (n - k[hi]) / ramp))
    return a


def taper_2d(n: int, apod: int, alpha: float = 1.0) -> np.ndarray:
    """Separable 2D taper A[y, x] = a[y] a[x]."""
    a = taper_1d(n, apod, alpha)
    return np.outer(a, a)


def apodise(x: np.ndarray, A: np.ndarray) -> np.ndarray:
    """x' = A * (x - mu_A), mu_A = sum(A x) / sum(A): zero-DC tapered window."""
    x = np.asarray(x, dtype=np.float64)
    mu = float((A * x).sum() / A.sum())
    return A * (x - mu)


# --------------------------------------------------------------------------- #
# direct 2D DFT (the definition; no FFT)
# --------------------------------------------------------------------------- #
_F_CACHE: dict[int, np.ndarray] = {}


def dft_matrix(n: int) -> np.ndarray:
    """F[k, m] = exp(-2 pi i k m / n) in complex128 (k m reduced mod n first)."""
    F = _F_CACHE.get(n)
    if F is None:
        km = np.mod(np.outer(np.arange(n), np.arange(n)), n).astype(np.float64)
        F = np.exp(-2j * np.pi * km / n)
        _F_CACHE[n] = F
    return F


def dft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2D DFT: X[ky, kx] = sum x[y, x] e^{-2pi i (ky y + kx x)/N}."""
    F = dft_matrix(x.shape[0])
    return F @ x @ F.T


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse 2D DFT with the 1/N^2 factor."""
    n = X.shape[0]
    Fi = np.conj(dft_matrix(n))
    return (Fi @ X @ Fi.T) / (n * n)


# --------------------------------------------------------------------------- #
# whitened cross-power spectrum (Sec. III, power scaling of the amplitudes)
# --------------------------------------------------------------------------- #
def whiten(C: np.ndarray, w: float) -> np.ndarray:
    """G = C |C|^(-w): magnitudes raised to 1 - w, phases kept; G[0,0] = 0."""
    mag = np.abs(C)
    G = np.zeros_like(C)
    nz = mag > 0
    G[nz] = C[nz] * mag[nz] ** (-w)
    G[0, 0] = 0.0
    return G


def match_surface(mov_w: np.ndarray, ref_w: np.ndarray, level: Level) -> np.ndarray:
    """Pixel-level match response s[tau] of a window pair.

    s = Re( IDFT2( whiten( DFT2(m') conj(DFT2(r')) ) ) ), m', r' apodised.
    With the moving window a circular shift of the reference by d, s peaks at
    tau = d.
    """
    A = taper_2d(level.n, level.apod, level.tukey_alpha)
    m = apodise(mov_w, A)
    r = apodise(ref_w, A)
    C = dft2(m) * np.conj(dft2(r))
    return idft2(whiten(C, level.whiten_exponent)).real


# --------------------------------------------------------------------------- #
# peak, SNR, subpixel
# --------------------------------------------------------------------------- #
def peak_index(s: np.ndarray):
    """(py, px) of the maximum; ties go to the smallest row-major index."""
    i = int(np.argmax(s))  # numpy returns the first occurrence
    return divmod(i, s.shape[1])


def signed_shift(k: int, n: int) -> int:
    """Index 0..n-1 to a shift in [-n/2, n/2)."""
    return k if k < n // 2 else k - n


def background_mask(n: int, py: int, px: int, radius: float) -> np.ndarray:
    """True where the wrapped Euclidean distance to (py, px) exceeds radius."""
    d = np.arange(n)
    dy = np.minimum(np.abs(d - py), n - np.abs(d - py)).astype(np.float64)
    dx = np.minimum(np.abs(d - px), n - np.abs(d - px)).astype(np.float64)
    return (dy[:, None] ** 2 + dx[None, :] ** 2) > radius * radius


def snr(s: np.ndarray, py: int, px: int, radius: float):
    """Z score of the peak: (s_peak - mean_bg) / std_bg (population std).

    Returns (snr, mean_bg, std_bg).  std_bg == 0 gives +inf when the peak lies
    above the background mean, else 0.
    """
    bg = s[background_mask(s.shape[0], py, px, radius)]
    mu = float(bg.mean())
    sd = float(np.sqrt(((bg - mu) ** 2).mean()))
    peak = float(s[py, px])
    if sd == 0.0:
        return (math.inf if peak > mu else 0.0), mu, sd
    return (peak - mu) / sd, mu, sd


def parabola_offset(sm: float, s0: float, sp: float) -> float:
    """Vertex offset of the parabola through (-1, sm), (0, s0), (+1, sp)."""
    den = sm - 2.0 * s0 + sp
    if not den < 0.0:
        return 0.0
    d = 0.5 * (sm - sp) / den
    return min(0.5, max(-0.5, d))


def subpixel(s: np.ndarray, py: int, px: int):
    """Separable 3-point parabola fit on the wrapped neighbours -> (dy, dx)."""
    n = s.shape[0]
    fy = parabola_offset(s[(py - 1) % n, px], s[py, px], s[(py + 1) % n, px])
    fx = parabola_offset(s[py, (px - 1) % n], s[py, px], s[py, (px + 1) % n])
    return fy, fx


# --------------------------------------------------------------------------- #
# one window pair -> result record
# --------------------------------------------------------------------------- #
RESULT_FIELDS = ("dy", "dx", "sy", "sx", "snr", "peak", "status")


def empty_result(status: int) -> dict:
    return dict(dy=0, dx=0, sy=0.0, sx=0.0, snr=0.0, peak=0.0, status=status)


def match_pair(mov_w: np.ndarray, ref_w: np.ndarray, level: Level,
               return_surface: bool = False):
    """Match one moving window against one reference window.

    Returns a dict with dy, dx (integer peak as a signed shift), sy, sx
    (subpixel shift), snr, peak (surface value at the peak) and status.
    """
    mov_w = np.asarray(mov_w, dtype=np.float64)
    ref_w = np.asarray(ref_w, dtype=np.float64)
    n = level.n
    if mov_w.shape != (n, n) or ref_w.shape != (n, n):
        raise ValueError("window shape mismatch")
    if not (np.isfinite(mov_w).all() and np.isfinite(ref_w).all()):
        res = empty_result(NONFINITE)
        return (res, None) if return_surface else res
    if mov_w.max() == mov_w.min() or ref_w.max() == ref_w.min():
        res = empty_result(FLAT)
        return (res, None) if return_surface else res
    s = match_surface(mov_w, ref_w, level)
    py, px = peak_index(s)
    z, _, _ = snr(s, py, px, level.snr_exclusion_radius)
    fy, fx = subpixel(s, py, px)
    dy, dx = signed_shift(py, n), signed_shift(px, n)
    res = dict(dy=dy, dx=dx, sy=dy + fy, sx=dx + fx, snr=z, peak=float(s[py, px]),
               status=OK)
    return (res, s) if return_surface else res


# --------------------------------------------------------------------------- #
# window sources: gather, model projection, affine resampling
# --------------------------------------------------------------------------- #
def gather(section: np.ndarray, origin, n: int):
    """n x n window at (y, x) origin, FP64; None when it leaves the section."""
    y, x = int(origin[0]), int(origin[1])
    h, w = section.shape
    if y < 0 or x < 0 or y + n > h or x + n > w:
        return None
    return section[y:y + n, x:x + n].astype(np.float64)


def project(sections, origin, n: int):
    """Model window: mean of the n x n windows of K sections (Sec. III, remod)."""
    wins = [gather(s, origin, n) for s in sections]
    if any(w is None for w in wins):
        return None
    return sum(wins) / float(len(wins))


def affine_sample_points(origin, n: int, theta):
    """Section coordinates sampled for window pixel (i, j) under ``theta``.

    theta = (a_yy, a_yx, t_y, a_xy, a_xx, t_x) acts about the window centre
    c = (n/2, n/2): p = origin + c + [[a_yy, a_yx], [a_xy, a_xx]] ((i,j) - c) + t.
    Returns (Y, X) float64 arrays [n, n].
    """
    c = n / 2.0
    i, j = np.meshgrid(np.arange(n, dtype=np.float64) - c,
                       np.arange(n, dtype=np.float64) - c, indexing="ij")
    a_yy, a_yx, t_y, a_xy, a_xx, t_x = (float(v) for v in theta)
    Y = origin[0] + c + a_yy * i + a_yx * j + t_y
    X = origin[1] + c + a_xy * i + a_xx * j + t_x
    return Y, X


def bilinear(section: np.ndarray, Y: np.ndarray, X: np.ndarray):
    """Bilinear samples of ``section`` at (Y, X); None if any leaves [0, h-1]x[0, w-1]."""
    h, w = section.shape
    if Y.min() < 0 or X.min() < 0 or Y.max() > h - 1 or X.max() > w - 1:
        return None
    y0 = np.minimum(np.floor(Y).astype(np.int64), h - 2)
    x0 = np.minimum(np.floor(X).astype(np.int64), w - 2)
    fy, fx = Y - y0, X - x0
    S = section.astype(np.float64)
    return ((1 - fy) * (1 - fx) * S[y0, x0] + (1 - fy) * fx * S[y0, x0 + 1]
            + fy * (1 - fx) * S[y0 + 1, x0] + fy * fx * S[y0 + 1, x0 + 1])


def resample(section: np.ndarray, origin, n: int, theta):
    """Moving window resampled bilinearly under the affine ``theta``."""
    Y, X = affine_sample_points(origin, n, theta)
    return bilinear(section, Y, X)


# --------------------------------------------------------------------------- #
# batch driver
# --------------------------------------------------------------------------- #
def match_batch(ref_sections, mov_sections, ref_origins, mov_origins, levels,
                level_index=None, affine=None):
    """Match every window of a batch; returns a list of result dicts.

    ``ref_sections[l]`` / ``mov_sections[l]`` are the images of level l.  A
    reference entry may be a list of K sections, in which case the model
    window is their mean.  ``affine`` [B, 6] resamples the moving windows.
    """
    out = []
    B = len(ref_origins)
    for b in range(B):
        l = 0 if level_index is None else int(level_index[b])
        lv = levels[l]
        rs = ref_sections[l]
        if isinstance(rs, (list, tuple)) or (isinstance(rs, np.ndarray) and rs.ndim == 3):
            r = project(rs, ref_origins[b], lv.n)
        else:
            r = gather(rs, ref_origins[b], lv.n)
        if affine is None:
            m = gather(mov_sections[l], mov_origins[b], lv.n)
        else:
            m = resample(mov_sections[l], mov_origins[b], lv.n, affine[b])
        if r is None or m is None:
            out.append(empty_result(OUT_OF_BOUNDS))
            continue
        out.append(match_pair(m, r, lv))
    return out


def match_patches(ref, mov, level: Level):
    """Match [B, n, n] patch pairs (no gather)."""
    return [match_pair(mov[b], ref[b], level) for b in range(len(ref))]


# --------------------------------------------------------------------------- #
# adjoint (gradients of peak height and SNR)
# --------------------------------------------------------------------------- #
def bilinear_grad(section: np.ndarray, Y: np.ndarray, X: np.ndarray):
    """d(bilinear sample)/dY and d/dX at (Y, X) (inside the section)."""
    h, w = section.shape
    y0 = np.minimum(np.floor(Y).astype(np.int64), h - 2)
    x0 = np.minimum(np.floor(X).astype(np.int64), w - 2)
    fy, fx = Y - y0, X - x0
    S = section.astype(np.float64)
    s00, s01, s10, s11 = S[y0, x0], S[y0, x0 + 1], S[y0 + 1, x0], S[y0 + 1, x0 + 1]
    dY = (1 - fx) * (s10 - s00) + fx * (s11 - s01)
    dX = (1 - fy) * (s01 - s00) + fy * (s11 - s10)
    return dY, dX


def match_backward(mov_section, origin, theta, ref_w, level: Level, grad_peak: float,
                   grad_snr: float):
    """Gradient of L = grad_peak * peak + grad_snr * snr of one window pair.

    The moving window is the section resampled under ``theta`` (see
    ``resample``); the reference window is fixed.  The peak index and hence
    the background set are held fixed (the argmax has no derivative).  Returns
    (forward result dict, dL/dtheta [6], dL/dw).

    Chain, in the order of the forward step it undoes:
      dL/ds      peak term: delta at the peak; SNR term:
                 (delta_peak - [bg]/n_bg - snr [bg] (s - mu_bg)/(n_bg sigma_bg)) / sigma_bg
      dL/dG      = DFT2(dL/ds)          (s = Re IDFT2(G); complex gradient
                                          convention g = dL/dRe + i dL/dIm)
      dL/dC      = e^{i phi} rho^-w [(1 - w) Re(u) - i Im(u)] / n^2 with
                   u = conj(dL/dG) e^{i phi}, C = rho e^{i phi}
      dL/dw      = -sum_k ln(rho_k) Re(conj(dL/dG_k) G_k)
      dL/dM      = dL/dC * R            (C = M conj(R))
      dL/dm'     = Re( n^2 IDFT2(dL/dM) ) (M = DFT2(m'), m' real)
      dL/dm      = A dL/dm' - A sum(A dL/dm') / sum(A)   (m' = A (m - mu_A))
      dL/dtheta  = sum_ij dL/dm_ij d(bilinear)/d(Y, X) d(Y, X)/dtheta
    """
    n = level.n
    theta = np.asarray(theta, dtype=np.float64)
    Y, X = affine_sample_points(origin, n, theta)
    mov_w = bilinear(mov_section, Y, X)
    if mov_w is None:
        raise ValueError("resampled window leaves the section")
    A = taper_2d(n, level.apod, level.tukey_alpha)
    mp = apodise(mov_w, A)
    rp = apodise(np.asarray(ref_w, dtype=np.float64), A)
    M = dft2(mp)
    R = dft2(rp)
    C = M * np.conj(R)
    w = level.whiten_exponent
    G = whiten(C, w) / (n * n)
    s = (idft2(G) * (n * n)).real  # G already carries 1/n^2
    py, px = peak_index(s)
    z, mu, sd = snr(s, py, px, level.snr_exclusion_radius)
    bg = background_mask(n, py, px, level.snr_exclusion_radius)
    nbg = float(bg.sum())
    peak = float(s[py, px])
    # dL/ds
    gs = np.zeros((n, n))
    gs[py, px] += grad_peak + grad_snr / sd
    gs[bg] += grad_snr * (-1.0 / (nbg * sd) - z * (s[bg] - mu) / (nbg * sd * sd))
    # dL/dG (complex-gradient convention)
    gG = dft2(gs)
    rho = np.abs(C)
    valid = rho > 0
    valid[0, 0] = False
    e = np.zeros_like(C)
    e[valid] = C[valid] / rho[valid]
    u = np.conj(gG) * e
    gC = np.zeros_like(C)
    gC[valid] = (e[valid] * rho[valid] ** (-w) / (n * n)
                 * ((1.0 - w) * u[valid].real - 1j * u[valid].imag))
    gw = -float(np.sum(np.log(rho[valid]) * (np.conj(gG[valid]) * G[valid]).real))
    gM = gC * R
    gmp = (idft2(gM) * (n * n)).real
    gm = A * gmp - A * float((A * gmp).sum()) / float(A.sum())
    dY, dX = bilinear_grad(mov_section, Y, X)
    c = n / 2.0
    ii, jj = np.meshgrid(np.arange(n, dtype=np.float64) - c, np.arange(n, dtype=np.float64) - c,
                         indexing="ij")
    gy, gx = gm * dY, gm * dX
    gtheta = np.array([(gy * ii).sum(), (gy * jj).sum(), gy.sum(),
                       (gx * ii).sum(), (gx * jj).sum(), gx.sum()])
    fwd = dict(dy=signed_shift(py, n), dx=signed_shift(px, n), snr=z, peak=peak, status=OK)
    return fwd, gtheta, gw


def affine_objective(mov_section, origin, theta, ref_w, level: Level, grad_peak: float,
                     grad_snr: float, peak_at=None):
    """L = grad_peak * peak + grad_snr * snr with the peak optionally held at
    ``peak_at`` = (py, px) (the envelope the adjoint differentiates)."""
    n = level.n
    mov_w = resample(mov_section, origin, n, theta)
    s = match_surface(mov_w, ref_w, level)
    py, px = peak_at if peak_at is not None else peak_index(s)
    z, _, _ = snr(s, py, px, level.snr_exclusion_radius)
    return grad_peak * float(s[py, px]) + grad_snr * z
