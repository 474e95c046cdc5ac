"""Pins of the mir oracle (least-squares affines, triangle mesh, rendering)
against what the mathematics fixes, independent of the oracle's own formulas:
numpy's least-squares solver on the weighted design matrix, exact recovery of
known affines, brute-force geometry on integer points, and exactness of
bilinear resampling on linear images."""
import numpy as np
import pytest

from oracle import mir


def _affine(rng):
    A = np.eye(2) + rng.uniform(-0.05, 0.05, (2, 2))
    t = rng.uniform(-20, 20, 2)
    return np.array([A[0, 0], A[0, 1], t[0], A[1, 0], A[1, 1], t[1]])


def test_fit_matches_weighted_lstsq():
    rng = np.random.default_rng(0)
    q = rng.uniform(0, 4096, (200, 2))
    p = q + rng.normal(0, 3, (200, 2))
    w = rng.uniform(0, 10, 200)
    th, st = mir.fit_affine(q, p, w)
    assert st == mir.OK
    D = np.column_stack([q[:, 0], q[:, 1], np.ones(len(q))]) * np.sqrt(w)[:, None]
    ay = np.linalg.lstsq(D, p[:, 0] * np.sqrt(w), rcond=None)[0]
    ax = np.linalg.lstsq(D, p[:, 1] * np.sqrt(w), rcond=None)[0]
    np.testing.assert_allclose(th, [ay[0], ay[1], ay[2], ax[0], ax[1], ax[2]], rtol=1e-9, atol=1e-7)


def test_fit_recovers_a_known_affine_exactly():
    rng = np.random.default_rng(1)
    th0 = _affine(rng)
    q = rng.uniform(0, 2048, (50, 2))
    p = mir.apply(th0, q)
    th, st = mir.fit_affine(q, p, rng.uniform(0.5, 2.0, 50))
    assert st == mir.OK
    np.testing.assert_allclose(th, th0, rtol=1e-10, atol=1e-8)


def test_zero_weight_points_do_not_count_and_weights_are_scale_free():
    rng = np.random.default_rng(2)
    q = rng.uniform(0, 1000, (40, 2))
    p = q + rng.normal(0, 1, (40, 2))
    w = rng.uniform(0.1, 1, 40)
    th, _ = mir.fit_affine(q, p, w)
    q2 = np.vstack([q, rng.uniform(0, 1000, (10, 2))])
    p2 = np.vstack([p, rng.uniform(-5000, 5000, (10, 2))])  # wild outliers with weight 0
    w2 = np.concatenate([w, np.zeros(10)])
    np.testing.assert_allclose(mir.fit_affine(q2, p2, w2)[0], th, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(mir.fit_affine(q, p, 7.0 * w)[0], th, rtol=1e-12, atol=1e-10)


def test_degenerate_point_sets():
    assert mir.fit_affine([[0, 0], [10, 10]], [[1, 1], [11, 11]], [1, 1])[1] == mir.DEGENERATE
    q = np.array([[0, 0], [10, 10], [20, 20], [35, 35]], float)  # collinear
    assert mir.fit_affine(q, q + 1, np.ones(4))[1] == mir.DEGENERATE
    assert mir.fit_affine(q[:3], q[:3], np.zeros(3))[1] == mir.DEGENERATE
    th, st = mir.fit_affine([[0, 0], [0, 10], [10, 0]], [[1, 2], [1, 12], [11, 2]], [1, 1, 1])
    assert st == mir.OK
    np.testing.assert_allclose(th, [1, 0, 1, 0, 1, 2], atol=1e-12)


def _inside(tri_half, y0, x0, c, y, x):
    dy, dx = y - y0, x - x0
    if not (0 <= dy <= c and 0 <= dx <= c):
        return False
    return dx >= dy if tri_half == 0 else dx <= dy


def test_locate_puts_every_pixel_in_its_triangle():
    m = mir.Mesh(3, -5, 16, 4, 5)
    Y, X = np.meshgrid(np.arange(3, 3 + 64), np.arange(-5, -5 + 80), indexing="ij")
    tri = m.locate(Y, X)
    counts = np.bincount(tri.ravel(), minlength=m.n_triangles)
    for t in range(m.n_triangles):
        _, _, half, y0, x0 = m.triangle(t)
        ys, xs = np.nonzero(tri == t)
        assert all(_inside(half, y0, x0, 16, Y[a, b], X[a, b]) for a, b in zip(ys, xs))
        # half-open cells: the upper triangle keeps the diagonal, c (c + 1) / 2 pixels
        assert counts[t] == (16 * 17 // 2 if half == 0 else 16 * 15 // 2)


def test_supports_equal_brute_force_chebyshev_distance():
    m = mir.Mesh(0, 0, 8, 3, 3)
    q = np.array([[y, x] for y in range(-12, 37, 3) for x in range(-12, 37, 2)], float)
    for band in (0, 4, 8):
        for t in range(m.n_triangles):
            _, _, half, y0, x0 = m.triangle(t)
            pts = [(y, x) for y in range(y0, y0 + 9) for x in range(x0, x0 + 9) if _inside(half, y0, x0, 8, y, x)]
            want = np.array([min(max(abs(a - y), abs(b - x)) for y, x in pts) <= band for a, b in q])
            np.testing.assert_array_equal(m.supports(t, q, band), want)


def test_mesh_fit_on_a_global_affine_and_fallback():
    rng = np.random.default_rng(3)
    th0 = _affine(rng)
    gy, gx = np.meshgrid(np.arange(16, 512, 32), np.arange(16, 512, 32), indexing="ij")
    q = np.column_stack([gy.ravel(), gx.ravel()]).astype(float)
    p = mir.apply(th0, q)
    w = np.ones(len(q))
    m = mir.Mesh(0, 0, 64, 8, 9)  # the last column of cells has no points
    th, st = mir.mesh_fit(q, p, w, m, band=0)
    np.testing.assert_allclose(th, np.broadcast_to(th0, th.shape), rtol=1e-9, atol=1e-7)
    last = [t for t in range(m.n_triangles) if m.triangle(t)[1] == 8]
    assert (st[last] == mir.FALLBACK).all()
    assert (np.delete(st, last) == mir.OK).all()


def test_render_identity_translation_and_linear_images():
    rng = np.random.default_rng(4)
    src = rng.integers(0, 256, (40, 50)).astype(np.uint8)
    m = mir.Mesh(0, 0, 8, 5, 7)
    ident = np.broadcast_to(mir.identity(), (m.n_triangles, 6))
    np.testing.assert_array_equal(mir.render(src, ident, m, 40, 50), src.astype(float))
    shift = np.broadcast_to([1, 0, 3, 0, 1, -2], (m.n_triangles, 6))
    out = mir.render(src, shift, m, 40, 50, fill=-1)
    np.testing.assert_array_equal(out[:37, 2:], src[3:, :48].astype(float))
    assert (out[37:] == -1).all() and (out[:, :2] == -1).all()
    # bilinear reproduces a linear image exactly under any affine
    lin = (0.7 * np.arange(60)[:, None] + 1.3 * np.arange(70)[None, :] + 5.0)
    th = np.array([_affine(rng) for _ in range(m.n_triangles)])
    th[:, [2, 5]] = rng.uniform(5, 15, (m.n_triangles, 2))
    out = mir.render(lin, th, m, 40, 50, fill=np.nan)
    Y, X = np.meshgrid(np.arange(40), np.arange(50), indexing="ij")
    P = np.array([mir.apply(th[t], [y, x]) for y, x, t in zip(Y.ravel(), X.ravel(), m.locate(Y, X).ravel())])
    want = 0.7 * P[:, 0] + 1.3 * P[:, 1] + 5.0
    ok = ~np.isnan(out.ravel())
    assert ok.mean() > 0.5
    np.testing.assert_allclose(out.ravel()[ok], want[ok], rtol=1e-12, atol=1e-9)


def test_correspondences_follow_a_physical_translation():
    """Content shifted by (+3, -5) in the moving section: swim's shift and the
    correspondence point p = q + shift must point to where it went."""
    import synth
    from oracle import swim
    a, _ = synth.em_section_pair(512, seed_content=31, seed_warp=32, seed_noise=(33, 34))
    b = np.roll(a, (3, -5), axis=(0, 1))
    lv = swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0)
    org = [(100, 120), (300, 260), (220, 380)]
    res = [swim.match_pair(swim.gather(b, o, 64), swim.gather(a, o, 64), lv) for o in org]
    q, p, w = mir.correspondences(res, org, org, 64)
    np.testing.assert_allclose(p - q, np.broadcast_to([3.0, -5.0], (3, 2)), atol=0.05)
    np.testing.assert_allclose(q, np.array(org) + 32.0)
    assert (w > 5).all()
    bad = dict(res[0], status=1)
    assert mir.correspondences([bad], org[:1], org[:1], 64)[2][0] == 0.0
