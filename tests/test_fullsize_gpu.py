"""The configured workloads at full size, in the launch configuration the
benchmark times, checked on sampled windows the oracle computes one by one
and on properties that hold at any size.

- Pyramid: one section pair at 1024^2 / 2048^2 / 4096^2 with 64 / 128 / 256
  windows at stride n/4 (11,163 windows), autotuned schedules, one captured
  CUDA graph replayed.
- Differentiation: 2048 windows of 128^2 on a 9-section 2048^2 stack
  (reference = mean of the 8 neighbours, moving = section 4 under per-window
  affine warps), forward and backward of -sum snr * peak.
- Precision: 8192 window pairs per call at 256^2 (BF16X2) and 128^2 (FP16X2),
  64 distinct shifted-patch pairs repeated 128 times: every repetition must
  give the same result, and samples from every workspace slice match the
  oracle.
- Models and pyramid: a 9-section 4096^2 uint8 stack (one section marked
  damaged), Z models (k = 4) bit-exact in full, 2x / 4x levels of the batch
  bit-exact on two sections.
- Rendering: the 512-triangle mesh (cell 256, band 256) fitted to the SNR-
  weighted correspondences of the 961-window grid, and the 4096^2 render of
  the moving section: the fits against the FP64 oracle, 16 sampled rows of
  the render against the oracle's.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import mir, remod, swim
from parity import compare, oracle_window

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402

DEV = "cuda:0"


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _olv(lv):
    return swim.Level(lv.n, lv.whiten_exponent, swim.APOD_HANN, 1.0, lv.snr_exclusion_radius)


def test_pyramid_full_size_graph_replay():
    a, b = synth.em_section_pair(4096)
    imgs = [(synth.box_downsample(a, 4), synth.box_downsample(b, 4)),
            (synth.box_downsample(a, 2), synth.box_downsample(b, 2)), (a, b)]
    levels = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8)]
    orgs, lvls = [], []
    for k, ((ia, _), lv) in enumerate(zip(imgs, levels)):
        o = synth.grid_origins(ia.shape[0], lv.n, lv.n // 4)
        orgs.append(o)
        lvls.append(np.full(len(o), k, np.int32))
    org, lvl = np.concatenate(orgs).astype(np.int32), np.concatenate(lvls)
    assert len(org) == 11163
    plan = swift.Plan(levels, dtype="u8", max_windows=len(org))
    da, db = [T(x[0]) for x in imgs], [T(x[1]) for x in imgs]
    dorg, dlvl = T(org), T(lvl)
    plan.autotune(da, db, dorg, dorg, level=dlvl)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out = plan.capture(da, db, dorg, dorg, level=dlvl, stream=stream)
        out.fill_(-1)
        plan.replay(stream)
    stream.synchronize()
    g = swift.decode(out)
    assert (g["status"] == 0).all()
    half = np.array([lv.n // 2 for lv in levels])[lvl]
    assert ((g["dy"] >= -half) & (g["dy"] < half) & (g["dx"] >= -half) & (g["dx"] < half)).all()
    assert np.isfinite(g["snr"]).all() and (g["snr"] > 0).all()
    rng = np.random.default_rng(11163)
    for k, lv in enumerate(levels):
        for i in rng.choice(np.nonzero(lvl == k)[0], 24, replace=False):
            ia, ib = imgs[k]
            o, tied = oracle_window(swim.gather(ib, org[i], lv.n), swim.gather(ia, org[i], lv.n), _olv(lv))
            compare(g, int(i), o, tied, lv.n, f"full-size pyramid level {k}")


def test_differentiation_full_size_forward_and_backward():
    n, count, size = 128, 2048, 2048
    stack = synth.section_stack(size, depth=9, seed=20)
    model = np.ascontiguousarray(stack[[0, 1, 2, 3, 5, 6, 7, 8]])
    movsec = np.ascontiguousarray(stack[4])
    org = synth.random_origins(count, size, size, n, seed=21, margin=8)
    theta = synth.affine_params(count, seed=22)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=count)
    dm, ds, dorg, dth = T(model), T(movsec), T(org), T(theta)
    res = plan.match(dm, ds, dorg, dorg, affine=dth)
    f = res.view(torch.float32)
    gp, gs = -f[:, 4].clone(), -f[:, 5].clone()  # d(-sum snr * peak): grad_peak = -snr, grad_snr = -peak
    g_aff, g_w = plan.backward(dm, ds, dorg, dorg, gp, gs, affine=dth)
    torch.cuda.synchronize()
    g = swift.decode(res)
    assert (g["status"] == 0).all()
    g_aff, gp, gs = g_aff.cpu().numpy(), gp.cpu().numpy(), gs.cpu().numpy()
    assert np.isfinite(g_aff).all() and np.isfinite(g_w.cpu().numpy()).all()
    olv = _olv(lv)
    rng = np.random.default_rng(2048)
    for i in rng.choice(count, 8, replace=False):
        m = swim.resample(movsec, org[i], n, theta[i].astype(np.float64))
        r = swim.project(list(model), org[i], n).astype(np.float32).astype(np.float64)
        o, tied = oracle_window(m.astype(np.float32).astype(np.float64), r, olv)
        compare(g, int(i), o, tied, n, "full-size warped forward")
        _, gth, _ = swim.match_backward(movsec.astype(np.float64), org[i], theta[i].astype(np.float64), r, olv,
                                        float(gp[i]), float(gs[i]))
        scale = max(np.abs(gth).max(), 1e-30)
        assert np.abs(g_aff[i] - gth).max() <= 2e-3 * scale, (int(i), g_aff[i], gth)


@pytest.mark.parametrize("n,precision", [(256, "bf16x2"), (128, "fp16x2")])
def test_precision_full_size_tiled(n, precision):
    section, _ = synth.em_section_pair(1024, seed_content=30, seed_warp=31, seed_noise=(32, 33))
    ref64, mov64, _ = synth.shifted_patches(section, n, 64, seed=10 + n)
    ref, mov = np.tile(ref64, (128, 1, 1)), np.tile(mov64, (128, 1, 1))
    count = ref.shape[0]
    assert count == 8192
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", precision=precision, max_windows=count)
    g = swift.decode(plan.match(T(ref), T(mov)))
    assert (g["status"] == 0).all()
    for key in g:  # the same inputs in every repetition (and every workspace slice): the same outputs
        v = g[key].reshape(128, 64)
        assert (v == v[0]).all(), key
    olv = _olv(lv)
    for i in [5, 2048 + 17, 4096 + 40, 6144 + 63]:  # one sample in each slice of 2048
        o, tied = oracle_window(mov[i].astype(np.float64), ref[i].astype(np.float64), olv)
        compare(g, i, o, tied, n, f"full-size {precision} n={n}")


def test_models_and_pyramid_full_size():
    size, Z, k = 4096, 9, 4
    a, _ = synth.em_section_pair(size)
    rng = np.random.default_rng(90)
    stack = np.stack([np.clip(np.roll(a, (z, -z), (0, 1)).astype(np.int16)
                              + rng.integers(-6, 7, a.shape, dtype=np.int16), 0, 255).astype(np.uint8)
                      for z in range(Z)])
    valid = np.ones(Z, bool)
    valid[6] = False
    ts = T(stack)
    model = swift.zmodel(ts, k, valid=T(valid.astype(np.uint8))).cpu().numpy()
    np.testing.assert_array_equal(model, remod.zmodel(stack, k, valid))
    for f in (2, 4):
        got = swift.downsample(ts, f).cpu().numpy()
        assert got.shape == (Z, size // f, size // f)
        for z in (0, 6):
            np.testing.assert_array_equal(got[z], remod.downsample(stack[z], f))


def test_rendering_full_size():
    size, n, stride, cell = 4096, 256, 128, 256
    a, b = synth.em_section_pair(size)
    org = synth.grid_origins(size, n, stride)
    da, db, dorg = T(a), T(b), T(org)
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=len(org))
    res = plan.match(da, db, dorg, dorg)
    q, p, w = swift.correspondences(res, dorg, dorg, n, min_snr=5.0)
    mesh = swift.Mesh(0, 0, cell, size // cell, size // cell)
    mesh_o = mir.Mesh(0, 0, cell, size // cell, size // cell)
    th, st = swift.mesh_fit(q, p, w, mesh, cell)
    out = swift.render(db, th, mesh, size, size, fill=0.0).cpu().numpy()
    th, st = th.cpu().numpy(), st.cpu().numpy()
    qn, pn, wn = q.cpu().numpy(), p.cpu().numpy(), w.cpu().numpy()
    ot, ost = mir.mesh_fit(qn, pn, wn, mesh_o, cell)
    np.testing.assert_array_equal(st, ost)
    np.testing.assert_allclose(th, ot, rtol=1e-9, atol=1e-7)
    rows = np.sort(np.random.default_rng(4096).choice(size, 16, replace=False))
    ref = mir.render(b, th, mesh_o, size, size, 0.0, rows=rows)
    Y, X = np.meshgrid(rows, np.arange(size), indexing="ij")
    t6 = th[mesh_o.locate(Y, X)]
    py = t6[..., 0] * Y + t6[..., 1] * X + t6[..., 2]
    px = t6[..., 3] * Y + t6[..., 4] * X + t6[..., 5]
    eps = 1e-3  # sample points this close to the source border may fall on either side
    amb = (np.abs(py) < eps) | (np.abs(px) < eps) | (np.abs(py - (size - 1)) < eps) | (np.abs(px - (size - 1)) < eps)
    assert (~amb).mean() > 0.99
    assert np.abs(out[rows] - ref)[~amb].max() <= 0.05
