"""Seeded synthetic inputs for the SWiFT-IR block-matching step.

This module only makes input images, window origins and warp parameters.  It
holds none of the matching arithmetic (no apodisation, transform, whitening,
peak or SNR code), so both the FP64 oracle and the CUDA library can be fed from
it without sharing any of the method.

The paper's data (mouse LGN and zebrafish ssEM stacks, Sec. IV) are not
available, so every workload is a stand-in with the same structure: 8-bit
sections of densely packed cell profiles (dark membranes around bright
interiors) with shot noise, a second section that is an affinely and smoothly
warped copy of the first, and a pyramid of box-downsampled levels (Sec. III,
"iscale" produces powers-of-two pyramids).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

__all__ = [
    "noise_pair",
    "em_clean",
    "shot_noise",
    "warp_section",
    "em_section_pair",
    "box_downsample",
    "grid_origins",
    "random_origins",
    "shifted_patches",
    "section_stack",
    "affine_params",
    "damaged_pairs",
]


# --------------------------------------------------------------------------- #
# small Gaussian-noise pair (64 x 64 worked example)
# --------------------------------------------------------------------------- #
def noise_pair(n: int = 64, shift=(-3, 5), sigma: float = 1.5,
               noise: float = 0.1, seed: int = 0):
    """Blurred white-noise reference and its circular shift plus noise.

    reference = Gaussian blur (sigma px, circular boundary) of
    ``default_rng(seed).standard_normal((n, n))``, normalised to zero mean and
    unit standard deviation; moving = ``np.roll(reference, shift, (0, 1))``
    plus N(0, noise^2) drawn from ``default_rng(seed + 1)``.  ``shift`` is
    (dy, dx).  Returns float64 arrays (reference, moving).
    """
    rng = np.random.default_rng(seed)
    ref = ndimage.gaussian_filter(rng.standard_normal((n, n)), sigma, mode="wrap")
    ref = (ref - ref.mean()) / ref.std()
    mov = np.roll(ref, shift, axis=(0, 1))
    mov = mov + np.random.default_rng(seed + 1).normal(0.0, noise, (n, n))
    return ref, mov


# --------------------------------------------------------------------------- #
# EM-like sections
# --------------------------------------------------------------------------- #
def em_clean(size: int, seed: int = 0, coverage: float = 0.9,
             semi_axes=(6.0, 40.0), rim=(2.0, 4.0), rim_level=(40.0, 70.0),
             interior=(150.0, 190.0), blur: float = 1.0) -> np.ndarray:
    """Noise-free EM-like section (float64, 0..255).

    Mid-grey canvas painted with random ellipses (semi-axes uniform in
    ``semi_axes`` px, random orientation) until ``coverage`` of the canvas is
    covered; each ellipse has a dark rim ``rim`` px wide at a grey level drawn
    from ``rim_level`` around a bright interior drawn from ``interior``.  Later
    ellipses paint over earlier ones, which leaves membrane-like boundaries
    everywhere.  A Gaussian blur of ``blur`` px finishes it.
    """
    rng = np.random.default_rng(seed)
    img = np.full((size, size), rng.uniform(*interior), dtype=np.float32)
    covered = np.zeros((size, size), dtype=bool)
    amax = semi_axes[1] + 1
    batch = 256
    while covered.mean() < coverage:
        for _ in range(batch):
            cy, cx = rng.uniform(-amax, size + amax, 2)
            a, b = rng.uniform(*semi_axes, 2)
            th = rng.uniform(0.0, np.pi)
            rw = rng.uniform(*rim)
            vr = rng.uniform(*rim_level)
            vi = rng.uniform(*interior)
            r = int(np.ceil(max(a, b))) + 1
            y0, y1 = max(int(cy) - r, 0), min(int(cy) + r + 1, size)
            x0, x1 = max(int(cx) - r, 0), min(int(cx) + r + 1, size)
            if y0 >= y1 or x0 >= x1:
                continue
            yy, xx = np.mgrid[y0:y1, x0:x1]
            dy, dx = yy - cy, xx - cx
            c, s = np.cos(th), np.sin(th)
            u = (c * dx + s * dy) / a
            v = (-s * dx + c * dy) / b
            rho = np.sqrt(u * u + v * v)
            inside = rho <= 1.0
            # distance to the boundary, approximately (1 - rho) * mean radius
            in_rim = inside & ((1.0 - rho) * 0.5 * (a + b) < rw)
            patch = img[y0:y1, x0:x1]
            patch[inside] = vi
            patch[in_rim] = vr
            covered[y0:y1, x0:x1] |= inside
    if blur > 0:
        img = ndimage.gaussian_filter(img, blur, mode="reflect")
    return img.astype(np.float64)


def shot_noise(img: np.ndarray, seed: int, snr: float = 8.0) -> np.ndarray:
    """Poisson shot noise, clipped and rounded to uint8.

    value = Poisson(I / g) * g with the gain g chosen so that a pixel at the
    image's median intensity has signal-to-noise ``snr`` (sqrt(I/g) = snr).
    """
    rng = np.random.default_rng(seed)
    g = float(np.median(img)) / (snr * snr)
    out = rng.poisson(np.maximum(img, 0.0) / g).astype(np.float64) * g
    return np.clip(np.rint(out), 0, 255).astype(np.uint8)


def warp_section(img: np.ndarray, seed: int, max_rot_deg: float = 1.0,
                 max_scale: float = 0.01, disp_amp: float = 8.0,
                 disp_spacing: int = 512) -> np.ndarray:
    """Affine + smooth displacement warp of ``img`` (backward mapping).

    out(p) = img(c + S R (p - c) + u(p)): rotation uniform in
    +-``max_rot_deg``, isotropic scale 1 + U(+-``max_scale``) about the image
    centre c, and a displacement field u given on a control grid of spacing
    ``disp_spacing`` px with entries U(+-``disp_amp``), cubic-spline
    interpolated and clipped to |u| <= ``disp_amp``.  Bilinear sampling,
    nearest-edge extension.
    """
    rng = np.random.default_rng(seed)
    h, w = img.shape
    th = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg))
    sc = 1.0 + rng.uniform(-max_scale, max_scale)
    ng = max(h, w) // disp_spacing + 1
    grid = rng.uniform(-disp_amp, disp_amp, (2, ng, ng))
    # cubic spline through the control grid, evaluated on a 16-px coarse grid
    step = 16
    cy = np.arange(0, h + step, step) / disp_spacing
    cx = np.arange(0, w + step, step) / disp_spacing
    gy, gx = np.meshgrid(cy, cx, indexing="ij")
    coarse = np.stack([ndimage.map_coordinates(grid[k], [gy, gx], order=3, mode="nearest")
                       for k in range(2)])
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    u = np.stack([ndimage.map_coordinates(coarse[k], [yy / step, xx / step], order=1,
                                          mode="nearest") for k in range(2)])
    u = np.clip(u, -disp_amp, disp_amp)
    c0y, c0x = (h - 1) / 2.0, (w - 1) / 2.0
    py, px = yy - c0y, xx - c0x
    cs, sn = np.cos(th), np.sin(th)
    sy = c0y + sc * (cs * py - sn * px) + u[0]
    sx = c0x + sc * (sn * py + cs * px) + u[1]
    return ndimage.map_coordinates(img, [sy, sx], order=1, mode="nearest")


def em_section_pair(size: int = 4096, seed_content: int = 0, seed_warp: int = 1,
                    seed_noise=(2, 3)):
    """Two uint8 EM-like sections: A and an affinely + smoothly warped A.

    Both get independent shot noise.  Returns (A, B) as C-contiguous uint8.
    """
    clean = em_clean(size, seed_content)
    a = shot_noise(clean, seed_noise[0])
    b = shot_noise(warp_section(clean, seed_warp), seed_noise[1])
    return np.ascontiguousarray(a), np.ascontiguousarray(b)


def box_downsample(img: np.ndarray, f: int) -> np.ndarray:
    """f x f box average, rounded back to uint8 (a pyramid level)."""
    h, w = img.shape
    v = img[: h - h % f, : w - w % f].astype(np.float64)
    v = v.reshape(h // f, f, w // f, f).mean(axis=(1, 3))
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


# --------------------------------------------------------------------------- #
# window placement and patch sets
# --------------------------------------------------------------------------- #
def grid_origins(size: int, n: int, stride: int) -> np.ndarray:
    """(y, x) origins of an evenly strided grid of n x n windows, int32 [B, 2]."""
    k = (size - n) // stride + 1
    i, j = np.meshgrid(np.arange(k) * stride, np.arange(k) * stride, indexing="ij")
    return np.stack([i.ravel(), j.ravel()], axis=1).astype(np.int32)


def random_origins(count: int, height: int, width: int, n: int, seed: int,
                   margin: int = 0) -> np.ndarray:
    """Uniform random in-bounds (y, x) origins, int32 [count, 2]."""
    rng = np.random.default_rng(seed)
    y = rng.integers(margin, height - n - margin + 1, count)
    x = rng.integers(margin, width - n - margin + 1, count)
    return np.stack([y, x], axis=1).astype(np.int32)


def shifted_patches(section: np.ndarray, n: int, count: int, seed: int,
                    max_shift: float = 20.0):
    """Float32 patch pairs with known, exactly band-limited subpixel shifts.

    For each pair a 2n x 2n tile is cut from ``section`` at a random origin;
    the reference is its centre n x n; the moving patch is the centre n x n of
    the tile circularly shifted by d ~ U(+-max_shift)^2 through a Fourier phase
    ramp (an exact band-limited shift of the periodic tile).  Returns
    (ref [count,n,n] f32, mov [count,n,n] f32, d [count,2] f64 as (dy, dx)).
    """
    rng = np.random.default_rng(seed)
    m = 2 * n
    h, w = section.shape
    oy = rng.integers(0, h - m + 1, count)
    ox = rng.integers(0, w - m + 1, count)
    d = rng.uniform(-max_shift, max_shift, (count, 2))
    k = np.fft.fftfreq(m)
    ref = np.empty((count, n, n), np.float32)
    mov = np.empty((count, n, n), np.float32)
    c0 = n // 2
    for i in range(count):
        tile = section[oy[i]:oy[i] + m, ox[i]:ox[i] + m].astype(np.float64)
        ramp = np.exp(-2j * np.pi * (k[:, None] * d[i, 0] + k[None, :] * d[i, 1]))
        shifted = np.fft.ifft2(np.fft.fft2(tile) * ramp).real
        ref[i] = tile[c0:c0 + n, c0:c0 + n]
        mov[i] = shifted[c0:c0 + n, c0:c0 + n]
    return ref, mov, d


def section_stack(size: int, depth: int = 9, seed: int = 20, drift: float = 1.0,
                  radius_jitter: float = 0.03, coverage: float = 0.9):
    """``depth`` uint8 EM-like sections whose cell profiles drift slowly in z.

    Ellipse centres move by U(+-drift) px and semi-axes by U(+-radius_jitter)
    (relative) from one section to the next, as cell profiles do through
    consecutive ssEM sections; each section gets its own shot noise.
    """
    rng = np.random.default_rng(seed)
    # draw one persistent set of ellipses, then re-render it per section
    amax = 41.0
    n_ell = int(4.0 * size * size / (np.pi * 23.0 * 23.0)) + 64
    cy = rng.uniform(-amax, size + amax, n_ell)
    cx = rng.uniform(-amax, size + amax, n_ell)
    a = rng.uniform(6.0, 40.0, n_ell)
    b = rng.uniform(6.0, 40.0, n_ell)
    th = rng.uniform(0.0, np.pi, n_ell)
    rw = rng.uniform(2.0, 4.0, n_ell)
    vr = rng.uniform(40.0, 70.0, n_ell)
    vi = rng.uniform(150.0, 190.0, n_ell)
    bg = rng.uniform(150.0, 190.0)
    out = []
    for z in range(depth):
        img = np.full((size, size), bg, dtype=np.float32)
        for e in range(n_ell):
            r = int(np.ceil(max(a[e], b[e]))) + 1
            y0, y1 = max(int(cy[e]) - r, 0), min(int(cy[e]) + r + 1, size)
            x0, x1 = max(int(cx[e]) - r, 0), min(int(cx[e]) + r + 1, size)
            if y0 >= y1 or x0 >= x1:
                continue
            yy, xx = np.mgrid[y0:y1, x0:x1]
            dy, dx = yy - cy[e], xx - cx[e]
            c, s = np.cos(th[e]), np.sin(th[e])
            u = (c * dx + s * dy) / a[e]
            v = (-s * dx + c * dy) / b[e]
            rho = np.sqrt(u * u + v * v)
            inside = rho <= 1.0
            in_rim = inside & ((1.0 - rho) * 0.5 * (a[e] + b[e]) < rw[e])
            patch = img[y0:y1, x0:x1]
            patch[inside] = vi[e]
            patch[in_rim] = vr[e]
        img = ndimage.gaussian_filter(img, 1.0, mode="reflect")
        out.append(shot_noise(img.astype(np.float64), seed + 100 + z))
        cy += rng.uniform(-drift, drift, n_ell)
        cx += rng.uniform(-drift, drift, n_ell)
        a *= 1.0 + rng.uniform(-radius_jitter, radius_jitter, n_ell)
        b *= 1.0 + rng.uniform(-radius_jitter, radius_jitter, n_ell)
    return np.stack(out)


def affine_params(count: int, seed: int, max_offset: float = 2.0,
                  max_rot_deg: float = 0.5) -> np.ndarray:
    """Per-window 2x3 affine warps, float32 [count, 6].

    Row-major (a_yy, a_yx, t_y, a_xy, a_xx, t_x): a rotation uniform in
    +-``max_rot_deg`` and a translation uniform in +-``max_offset`` px.  The
    translation's fractional parts are kept at least 0.05 px away from
    integers so that bilinear sampling is differentiable at every sample.
    """
    rng = np.random.default_rng(seed)
    th = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, count))
    t = rng.uniform(-max_offset, max_offset, (count, 2))
    frac = t - np.floor(t)
    t = np.where(frac < 0.05, t + 0.05, t)
    t = np.where(frac > 0.95, t - 0.05, t)
    c, s = np.cos(th), np.sin(th)
    return np.stack([c, -s, t[:, 0], s, c, t[:, 1]], axis=1).astype(np.float32)


# --------------------------------------------------------------------------- #
# damaged pairs (whitening-exponent study, the Fig. 2 setting)
# --------------------------------------------------------------------------- #
def damaged_pairs(n: int, count: int, seed: int, size: int | None = None, max_shift: int = 24):
    """Reference patches and damaged, shifted copies of them (uint8).

    The paper's Fig. 2 locates a damaged region B inside an undamaged area A at
    several whitening exponents.  Stand-in: from one clean EM-like section
    (``em_clean``, content seed ``seed + 1``) the reference is the n x n tile
    at a random origin; the moving patch is the tile shifted by an integer
    d ~ U{-max_shift..max_shift}^2 (moving(y) = clean(y0 - d + y), so the
    match finds +d) and damaged by
      * a smooth illumination gradient (x 1 +- 0.25 across the patch),
      * a dark fold: a band 4-10 px wide at a random angle, x 0.25,
      * a smeared half plane (Gaussian blur, sigma 2.5 px),
    then shot noise at SNR 3 (reference: SNR 6).  Returns
    (ref [count,n,n] uint8, mov [count,n,n] uint8, d [count,2] int64 as (dy, dx)).
    """
    rng = np.random.default_rng(seed)
    size = size or max(1024, 4 * n)
    clean = em_clean(size, seed=seed + 1)
    ref = np.empty((count, n, n), np.uint8)
    mov = np.empty((count, n, n), np.uint8)
    shifts = np.empty((count, 2), np.int64)
    yy, xx = np.mgrid[0:n, 0:n] / n
    margin = max_shift + 16
    for i in range(count):
        y0, x0 = rng.integers(margin, size - n - margin, 2)
        d = rng.integers(-max_shift, max_shift + 1, 2)
        a = clean[y0:y0 + n, x0:x0 + n]
        b = clean[y0 - d[0]:y0 - d[0] + n, x0 - d[1]:x0 - d[1] + n].copy()
        phi = rng.uniform(0.0, 2.0 * np.pi, 2)
        b = b * (1.0 + 0.5 * ((yy - 0.5) * np.cos(phi[0]) + (xx - 0.5) * np.sin(phi[1])))
        th, c, half_width = rng.uniform(0.0, np.pi), rng.uniform(0.3, 0.7), rng.uniform(4.0, 10.0)
        band = np.abs((yy - c) * np.cos(th) + (xx - 0.5) * np.sin(th)) < half_width / n
        b[band] *= 0.25
        side = ((yy - 0.5) * np.sin(th) - (xx - 0.5) * np.cos(th)) > rng.uniform(-0.2, 0.2)
        b = np.where(side, ndimage.gaussian_filter(b, 2.5), b)
        ref[i] = shot_noise(np.clip(a, 0, 255), seed=seed * 1000 + 2 * i, snr=6.0)
        mov[i] = shot_noise(np.clip(b, 0, 255), seed=seed * 1000 + 2 * i + 1, snr=3.0)
        shifts[i] = d
    return ref, mov, shifts
