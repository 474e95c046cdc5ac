"""The rendering step (mir) on the GPU against the FP64 oracle, through the C ABI.

Inputs are synthetic: correspondences on a regular grid of window centres
under a smooth warp plus noise (some weights 0, one region without points),
EM-like sections for rendering, and triangle affines near the identity with
translations of up to +-20 px.

Tolerances: fits are FP64 on both sides (1e-9 relative); statuses exact.
Rendering computes each sample point as an integer base plus an FP32 fraction
of magnitude below ~2 x (mesh extent), so |dp| <= ~1e-4 px and a sample moves
by at most 1e-4 x 255 grey levels: 0.05 is the bar.  Pixels whose oracle
sample point lies within 1e-3 px of the source border are ambiguous
(inside/outside may legitimately differ) and are not compared.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import mir

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402

DEV = "cuda:0"
RENDER_TOL = 0.05


def T(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return (t.to(dtype) if dtype is not None else t).to(DEV)


def _grid_points(rng, gy, gx, spacing, origin, warp_amp=6.0, noise=0.3):
    yy, xx = np.meshgrid(origin + spacing * np.arange(gy), origin + spacing * np.arange(gx), indexing="ij")
    q = np.column_stack([yy.ravel(), xx.ravel()]).astype(np.float32)
    ext = spacing * max(gy, gx)
    d = np.column_stack([warp_amp * np.sin(2 * np.pi * q[:, 1] / ext) + 3.0,
                         warp_amp * np.cos(2 * np.pi * q[:, 0] / ext) - 2.0])
    p = (q + d + rng.normal(0, noise, q.shape)).astype(np.float32)
    w = rng.uniform(1, 30, len(q)).astype(np.float32)
    return q, p, w


def test_fit_affine_groups_match_oracle():
    rng = np.random.default_rng(7)
    groups, qs, ps, ws = [0], [], [], []
    for g in range(12):
        n = [0, 2, 3, 40, 200, 5][g % 6]
        q = rng.uniform(0, 4096, (n, 2)).astype(np.float32)
        p = (q + rng.normal(0, 2, (n, 2)) + rng.uniform(-30, 30, 2)).astype(np.float32)
        w = rng.uniform(0, 5, n).astype(np.float32)
        if g == 5:  # collinear: degenerate
            q[:, 1] = q[:, 0]
        qs.append(q), ps.append(p), ws.append(w)
        groups.append(groups[-1] + n)
    q, p, w = np.concatenate(qs), np.concatenate(ps), np.concatenate(ws)
    th, st = swift.fit_affine(T(q), T(p), T(w), offsets=T(np.array(groups, np.int64)))
    th, st = th.cpu().numpy(), st.cpu().numpy()
    for g in range(12):
        a, b = groups[g], groups[g + 1]
        ot, os_ = mir.fit_affine(q[a:b], p[a:b], w[a:b])
        assert st[g] == os_, (g, st[g], os_)
        np.testing.assert_allclose(th[g], ot, rtol=1e-9, atol=1e-7 * (1 + np.abs(ot).max()))


def test_fit_affine_update_keeps_previous_affines_of_degenerate_groups():
    """The update form: an OK group is overwritten by its fit (the oracle's),
    a degenerate group (all weights 0, or collinear points) keeps what theta
    held."""
    rng = np.random.default_rng(17)
    q = rng.uniform(0, 2000, (60, 2)).astype(np.float32)
    p = (q + rng.normal(0, 1, (60, 2)) + 5).astype(np.float32)
    w = rng.uniform(0.5, 3, 60).astype(np.float32)
    w[20:40] = 0.0                    # group 1: no weight
    q[40:60, 1] = q[40:60, 0]         # group 2: collinear
    offsets = np.array([0, 20, 40, 60], np.int64)
    prev = rng.normal(0, 1, (3, 6))
    theta = T(prev.copy())
    th, st = swift.fit_affine(T(q), T(p), T(w), offsets=T(offsets), update=theta)
    assert th.data_ptr() == theta.data_ptr()
    th, st = th.cpu().numpy(), st.cpu().numpy()
    ot, os_ = mir.fit_affine(q[:20], p[:20], w[:20])
    assert st[0] == os_ == swift.FIT_OK
    np.testing.assert_allclose(th[0], ot, rtol=1e-9, atol=1e-7)
    assert (st[1:] == mir.DEGENERATE).all()
    np.testing.assert_array_equal(th[1:], prev[1:])


@pytest.mark.parametrize("band", [0, 64, 128])
def test_mesh_fit_matches_oracle(band):
    rng = np.random.default_rng(11 + band)
    q, p, w = _grid_points(rng, 24, 24, 64.0, 32.0)
    w[rng.random(len(w)) < 0.15] = 0.0  # failed windows
    keep = ~((q[:, 0] > 900) & (q[:, 1] > 900))  # a corner without points -> fallbacks
    q, p, w = q[keep], p[keep], w[keep]
    mesh = swift.Mesh(0, 0, 128, 12, 13)
    th, st = swift.mesh_fit(T(q), T(p), T(w), mesh, band)
    th, st = th.cpu().numpy(), st.cpu().numpy()
    ot, ost = mir.mesh_fit(q, p, w, mir.Mesh(0, 0, 128, 12, 13), band)
    np.testing.assert_array_equal(st, ost)
    assert (ost == mir.FALLBACK).any() and (ost == mir.OK).any()
    np.testing.assert_allclose(th, ot, rtol=1e-9, atol=1e-7)


def _random_thetas(rng, mesh):
    th = np.zeros((mesh.n_triangles, 6))
    for t in range(mesh.n_triangles):
        A = np.eye(2) + rng.uniform(-0.02, 0.02, (2, 2))
        th[t] = [A[0, 0], A[0, 1], rng.uniform(-20, 20), A[1, 0], A[1, 1], rng.uniform(-20, 20)]
    return th


def _compare_render(src, th, mesh_o, out, out_h, out_w, fill, where):
    ref = mir.render(src, th, mesh_o, out_h, out_w, fill)
    Y, X = np.meshgrid(np.arange(out_h), np.arange(out_w), indexing="ij")
    tri = mesh_o.locate(Y, X)
    t6 = th[tri]
    py = t6[..., 0] * Y + t6[..., 1] * X + t6[..., 2]
    px = t6[..., 3] * Y + t6[..., 4] * X + t6[..., 5]
    h, w = src.shape
    eps = 1e-3
    amb = ((np.abs(py) < eps) | (np.abs(px) < eps) | (np.abs(py - (h - 1)) < eps) | (np.abs(px - (w - 1)) < eps))
    ok = ~amb
    assert ok.mean() > 0.99
    diff = np.abs(out - ref)[ok]
    assert diff.max() <= RENDER_TOL, f"{where}: max |diff| {diff.max()}"
    inside = (py >= 0) & (px >= 0) & (py <= h - 1) & (px <= w - 1)
    assert (out[ok & ~inside] == fill).all(), f"{where}: fill pixels differ"
    return inside[ok].mean()


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_render_matches_oracle(dtype):
    rng = np.random.default_rng(21)
    a, _ = synth.em_section_pair(512, seed_content=41, seed_warp=42, seed_noise=(43, 44))
    src = a[:300, :420]
    if dtype == "f32":
        src = src.astype(np.float32) * 0.37 - 11.0
    mesh = swift.Mesh(-8, 5, 40, 8, 10)  # pixels outside the mesh use the border cells
    mesh_o = mir.Mesh(-8, 5, 40, 8, 10)
    th = _random_thetas(rng, mesh)
    out_h, out_w = 330, 430
    out = swift.render(T(src), T(th), mesh, out_h, out_w, fill=-7.0).cpu().numpy()
    frac = _compare_render(src, th, mesh_o, out, out_h, out_w, -7.0, dtype)
    assert 0.5 < frac < 1.0  # both inside and fill pixels are exercised


def test_render_identity_is_exact_and_large_coordinates_keep_precision():
    rng = np.random.default_rng(5)
    src = rng.integers(0, 256, (2500, 4200)).astype(np.uint8)
    mesh = swift.Mesh(0, 0, 256, 10, 17)
    ident = np.broadcast_to(mir.identity(), (mesh.n_triangles, 6)).copy()
    out = swift.render(T(src), T(ident), mesh, 2500, 4200).cpu().numpy()
    np.testing.assert_array_equal(out, src.astype(np.float32))
    # a sub-pixel translation far from the origin: precision does not decay with the coordinate
    th = ident.copy()
    th[:, 2], th[:, 5] = 0.25, 0.5
    out = swift.render(T(src), T(th), mesh, 2500, 4200, fill=0.0).cpu().numpy()
    rows = np.array([0, 1, 1200, 2497])
    ref = mir.render(src, th, mir.Mesh(0, 0, 256, 10, 17), 2500, 4200, 0.0, rows=rows)
    np.testing.assert_allclose(out[rows][:, :4198], ref[:, :4198], atol=1e-3)


def test_correspondences_kernel_matches_oracle():
    rng = np.random.default_rng(9)
    B, n = 50, 128
    res = np.zeros((B, 8), np.int32)
    f = res.view(np.float32)
    res[:, 0] = rng.integers(-10, 10, B)
    res[:, 1] = rng.integers(-10, 10, B)
    f[:, 2] = res[:, 0] + rng.uniform(-0.5, 0.5, B)
    f[:, 3] = res[:, 1] + rng.uniform(-0.5, 0.5, B)
    f[:, 4] = rng.uniform(0, 40, B)
    f[:, 5] = rng.uniform(0, 1, B)
    res[:, 6] = np.where(rng.random(B) < 0.2, 1, 0)
    f[3, 4] = np.inf
    ro = rng.integers(0, 4000, (B, 2)).astype(np.int32)
    mo = (ro + rng.integers(-20, 20, (B, 2))).astype(np.int32)
    q, p, w = swift.correspondences(T(res), T(ro), T(mo), n, min_snr=5.0)
    d = swift.decode(res)
    results = [{k: d[k][b] for k in ("sy", "sx", "snr", "status")} for b in range(B)]
    oq, op, ow = mir.correspondences(results, ro, mo, n, min_snr=5.0)
    np.testing.assert_allclose(q.cpu().numpy(), oq, rtol=0, atol=1e-3)
    np.testing.assert_allclose(p.cpu().numpy(), op, rtol=0, atol=1e-3)
    np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=1e-7)
    assert w[3].item() == 0.0


def test_swim_then_mir_recovers_a_known_affine():
    """End to end on the device: a section and its affinely warped copy, swim
    on a grid, SNR-weighted fit: the recovered affine moves no grid point by
    more than 0.25 px from the known one (shifts reach ~16 px; the
    parabola fit's subpixel bias is the main error)."""
    rng = np.random.default_rng(3)
    a, _ = synth.em_section_pair(1536, seed_content=51, seed_warp=52, seed_noise=(53, 54))
    th0 = np.array([1.004, 0.006, -7.3, -0.005, 0.997, 4.6])  # reference frame -> moving section
    # moving section b(p) = a(q) with p = A q + t, i.e. b = a sampled at the inverse map
    A = np.array([[th0[0], th0[1]], [th0[3], th0[4]]])
    Ai = np.linalg.inv(A)
    Y, X = np.meshgrid(np.arange(1536.0), np.arange(1536.0), indexing="ij")
    P = np.stack([Y - th0[2], X - th0[5]], -1) @ Ai.T
    b = mir.bilinear_fill(a, P[..., 0], P[..., 1], 0.0).round().clip(0, 255).astype(np.uint8)
    n = 128
    org = synth.grid_origins(1536, n, 96)
    org = org[(org.min(1) >= 64) & (org.max(1) <= 1536 - n - 64)]
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=len(org))
    torg = T(org.astype(np.int32))
    res = plan.match(T(a), T(b), torg, torg)
    q, p, w = swift.correspondences(res, torg, torg, n, min_snr=8.0)
    assert (w > 0).float().mean().item() > 0.9
    th, st = swift.fit_affine(q, p, w)
    assert st.item() == swift.FIT_OK
    th = th.cpu().numpy()[0]
    qn = q.cpu().numpy()
    err = np.abs(mir.apply(th, qn) - mir.apply(th0, qn)).max()
    assert err < 0.25, err
