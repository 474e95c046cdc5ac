"""FP64 oracle of SWiFT-IR's rendering step ("mir", Sec. III module list and
Sec. IV): least-squares affines from swim correspondence points, a locally
affine triangle mesh, and rendering by texture mapping of the triangles.

TEST INFRASTRUCTURE ONLY.  Like ``oracle.swim`` this module is the slow,
plainly written reference the CUDA library is checked against; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` may
use it, and it shares no code with the CUDA path.

The paper's description, step by step:

* mir renders aligned output images from the linear least-squares solution
  of the correspondence points found by swim (Sec. III, module list);
* at low resolution one affine for the whole section suffices (Sec. IV);
* later, a locally affine triangulated mesh: each triangle's affine is the
  least-squares solution of the match points inside the triangle and inside
  an external band that takes in the surrounding triangles (Sec. IV);
* rendering is software texture mapping of the triangles (Sec. III).

Readings where the paper is silent (also listed with the design notes):

* a correspondence is (q, p, w): q the point in the output (reference)
  frame, p the matching point in the source (moving) section, w >= 0 its
  weight (the library's Python layer uses the swim SNR of OK windows and 0
  otherwise: the SNR-weighted least squares);
* the affine maps output to source, p = A q + t, stored as
  (a_yy, a_yx, t_y, a_xy, a_xx, t_x) with (y, x) coordinates;
* least squares: minimise sum_i w_i |A q_i + t - p_i|^2; solved in centred
  form, A = Cpq Sqq^-1, t = p_bar - A q_bar (weighted means and centred
  second moments); DEGENERATE when sum w = 0 or det(Sqq) <= 1e-9 (tr Sqq / 2)^2
  (fewer than three non-collinear weighted points);
* mesh: square cells of side c from integer origin (oy, ox), ny x nx cells,
  each split by its main diagonal: triangle 2 (cy nx + cx) + 0 holds the
  points with (x - x0) >= (y - y0) ("upper"), + 1 those with (x - x0) <=
  (y - y0) ("lower");
* band: a point supports a triangle when its Chebyshev distance to the
  (closed) triangle is at most b, i.e. it lies in the triangle grown by the
  square [-b, b]^2; with b = c this takes in the neighbouring triangles;
* a triangle whose support is degenerate takes the whole-section affine
  (status FALLBACK); if that is degenerate too, the identity (status
  DEGENERATE);
* rendering: output pixel (y, x) (integer coordinates) belongs to the
  triangle of its cell (cells clamped to the mesh, then the diagonal rule);
  its value is the bilinear sample of the source at p = A q + t, or the fill
  value when p leaves [0, h-1] x [0, w-1].
"""
from __future__ import annotations

import numpy as np

OK = 0
FALLBACK = 1
DEGENERATE = 2

DET_EPS = 1e-9


def fit_affine(q, p, w):
    """Weighted least-squares affine p ~ A q + t.  Returns (theta[6], status)."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 2)
    p = np.asarray(p, dtype=np.float64).reshape(-1, 2)
    w = np.asarray(w, dtype=np.float64).reshape(-1)
    W = w.sum()
    if not W > 0:
        return identity(), DEGENERATE
    qb = (w[:, None] * q).sum(0) / W
    pb = (w[:, None] * p).sum(0) / W
    dq = q - qb
    dp = p - pb
    Sqq = (w[:, None, None] * dq[:, :, None] * dq[:, None, :]).sum(0)  # [2, 2]
    Cpq = (w[:, None, None] * dp[:, :, None] * dq[:, None, :]).sum(0)  # [2, 2]
    det = Sqq[0, 0] * Sqq[1, 1] - Sqq[0, 1] * Sqq[1, 0]
    tr = Sqq[0, 0] + Sqq[1, 1]
    if not det > DET_EPS * (0.5 * tr) ** 2:
        return identity(), DEGENERATE
    inv = np.array([[Sqq[1, 1], -Sqq[0, 1]], [-Sqq[1, 0], Sqq[0, 0]]]) / det
    A = Cpq @ inv
    t = pb - A @ qb
    return np.array([A[0, 0], A[0, 1], t[0], A[1, 0], A[1, 1], t[1]]), OK


def identity():
    return np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0])


def apply(theta, q):
    """p = A q + t for points q [..., 2] (y, x)."""
    q = np.asarray(q, dtype=np.float64)
    a_yy, a_yx, t_y, a_xy, a_xx, t_x = theta
    return np.stack([a_yy * q[..., 0] + a_yx * q[..., 1] + t_y,
                     a_xy * q[..., 0] + a_xx * q[..., 1] + t_x], axis=-1)


class Mesh:
    """Regular triangle mesh: ny x nx square cells of side ``cell`` from the
    integer origin (oy, ox), two triangles per cell."""

    def __init__(self, oy: int, ox: int, cell: int, ny: int, nx: int):
        self.oy, self.ox, self.cell, self.ny, self.nx = int(oy), int(ox), int(cell), int(ny), int(nx)

    @property
    def n_triangles(self):
        return 2 * self.ny * self.nx

    def triangle(self, t: int):
        """(cy, cx, half, y0, x0) of triangle t."""
        c = t // 2
        cy, cx = divmod(c, self.nx)
        return cy, cx, t % 2, self.oy + cy * self.cell, self.ox + cx * self.cell

    def supports(self, t: int, q, band: int):
        """Mask of the points q [P, 2] within Chebyshev distance ``band`` of triangle t."""
        q = np.asarray(q, dtype=np.float64)
        _, _, half, y0, x0 = self.triangle(t)
        c, b = self.cell, band
        dy = q[:, 0] - y0
        dx = q[:, 1] - x0
        box = (dy >= -b) & (dy <= c + b) & (dx >= -b) & (dx <= c + b)
        diag = (dx - dy >= -2 * b) if half == 0 else (dy - dx >= -2 * b)
        return box & diag

    def locate(self, y, x):
        """Triangle index of integer output pixels (y, x) (arrays)."""
        y = np.asarray(y, dtype=np.int64)
        x = np.asarray(x, dtype=np.int64)
        cy = np.clip(np.floor_divide(y - self.oy, self.cell), 0, self.ny - 1)
        cx = np.clip(np.floor_divide(x - self.ox, self.cell), 0, self.nx - 1)
        dy = y - (self.oy + cy * self.cell)
        dx = x - (self.ox + cx * self.cell)
        half = np.where(dx >= dy, 0, 1)
        return 2 * (cy * self.nx + cx) + half


def mesh_fit(q, p, w, mesh: Mesh, band: int):
    """Per-triangle affines [T, 6] and statuses [T] (Sec. IV: each triangle's
    least squares over its own area plus the surrounding band)."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 2)
    p = np.asarray(p, dtype=np.float64).reshape(-1, 2)
    w = np.asarray(w, dtype=np.float64).reshape(-1)
    g, gst = fit_affine(q, p, w)
    thetas = np.zeros((mesh.n_triangles, 6))
    status = np.zeros(mesh.n_triangles, dtype=np.int32)
    for t in range(mesh.n_triangles):
        m = mesh.supports(t, q, band)
        th, st = fit_affine(q[m], p[m], w[m])
        if st != OK:
            th, st = (g, FALLBACK) if gst == OK else (identity(), DEGENERATE)
        thetas[t] = th
        status[t] = st
    return thetas, status


def bilinear_fill(src: np.ndarray, Y: np.ndarray, X: np.ndarray, fill: float):
    """Bilinear samples of ``src`` at (Y, X); ``fill`` outside [0, h-1] x [0, w-1]."""
    h, w = src.shape
    inside = (Y >= 0) & (X >= 0) & (Y <= h - 1) & (X <= w - 1)
    Yc = np.where(inside, Y, 0.0)
    Xc = np.where(inside, X, 0.0)
    y0 = np.minimum(np.floor(Yc).astype(np.int64), h - 2)
    x0 = np.minimum(np.floor(Xc).astype(np.int64), w - 2)
    fy, fx = Yc - y0, Xc - x0
    S = src.astype(np.float64)
    v = ((1 - fy) * (1 - fx) * S[y0, x0] + (1 - fy) * fx * S[y0, x0 + 1]
         + fy * (1 - fx) * S[y0 + 1, x0] + fy * fx * S[y0 + 1, x0 + 1])
    return np.where(inside, v, fill)


def render(src: np.ndarray, thetas, mesh: Mesh, out_h: int, out_w: int, fill: float = 0.0,
           rows=None):
    """Texture-map ``src`` through the mesh into an out_h x out_w image (FP64).
    ``rows`` restricts the output to the given row indices (for sampling)."""
    ys = np.arange(out_h) if rows is None else np.asarray(rows)
    Y, X = np.meshgrid(ys, np.arange(out_w), indexing="ij")
    tri = mesh.locate(Y, X)
    th = np.asarray(thetas, dtype=np.float64)[tri]  # [H, W, 6]
    py = th[..., 0] * Y + th[..., 1] * X + th[..., 2]
    px = th[..., 3] * Y + th[..., 4] * X + th[..., 5]
    return bilinear_fill(src, py, px, fill)


def correspondences(results, ref_origins, mov_origins, n: int, min_snr: float = 0.0):
    """(q, p, w) from swim results (list of dicts): q = reference window
    centre, p = moving window centre + subpixel shift (where the reference
    content sits in the moving section), w = SNR of OK windows with a finite
    SNR >= min_snr, else 0 (p then the moving centre)."""
    B = len(results)
    q = np.zeros((B, 2))
    p = np.zeros((B, 2))
    w = np.zeros(B)
    c = n / 2.0
    for b, r in enumerate(results):
        q[b] = (ref_origins[b][0] + c, ref_origins[b][1] + c)
        ok = r["status"] == 0 and np.isfinite(r["snr"]) and r["snr"] >= min_snr
        p[b] = (mov_origins[b][0] + c + (r["sy"] if ok else 0.0), mov_origins[b][1] + c + (r["sx"] if ok else 0.0))
        w[b] = r["snr"] if ok else 0.0
    return q, p, w


def to_u8(v):
    """Rendered values stored as uint8: rounded half to even, clamped to [0, 255]."""
    v = np.nan_to_num(np.asarray(v, dtype=np.float64), nan=0.0)
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)
