"""The registration loop on the device against the oracle's loop (same
readings), through the library's kernels: one stack of identical EM-like
sections (independent noise) cut at known offsets.

Tolerances: each step has its own parity test; composed over iterations the
device and the oracle may differ where a rendered value rounds differently to
uint8 (FP32 vs FP64 sample), so the bar is on the outputs of the loop: every
section's affine moves the section corners by at most 0.05 px from the
oracle's, median SNRs agree within 2 %, and at least 99.5 % of the aligned
pixels agree within one grey level."""
import numpy as np
import pytest
import torch

import synth
from oracle import driver, swim

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402
from paper_1612_04787_gb300 import align  # noqa: E402

DEV = "cuda:0"


def _stack(size, depth, offs, seed):
    base = synth.section_stack(size + 64, depth=depth, seed=seed, drift=0.0, radius_jitter=0.0)
    return np.stack([base[z, 32 + dy:32 + dy + size, 32 + dx:32 + dx + size] for z, (dy, dx) in enumerate(offs)])


def _corners(th, h, w):
    q = np.array([[0, 0], [0, w - 1], [h - 1, 0], [h - 1, w - 1]], float)
    return np.stack([th[0] * q[:, 0] + th[1] * q[:, 1] + th[2], th[3] * q[:, 0] + th[4] * q[:, 1] + th[5]], 1)


def test_loop_matches_the_oracle_loop():
    offs = np.array([[0, 0], [4, -3], [-2, 5], [3, 2]])
    raw = _stack(256, 4, offs, seed=12)
    lv = swift.Level(64, 0.65, "hann", 1.0, 3.0)
    aligned, theta, hist = align.align_stack(torch.from_numpy(raw).to(DEV), lv, stride=48, k=3, iters=3)
    oa, ot, oh = driver.align_stack(raw, swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0), stride=48, k=3, iters=3)
    theta = theta.cpu().numpy()
    assert len(hist) == len(oh)
    np.testing.assert_allclose(hist, oh, rtol=2e-2)
    for z in range(4):
        assert np.abs(_corners(theta[z], 256, 256) - _corners(ot[z], 256, 256)).max() <= 0.05, z
    diff = np.abs(aligned.cpu().numpy().astype(int) - oa.astype(int))
    assert (diff <= 1).mean() >= 0.995


def test_graph_replay_gives_the_call_by_call_results():
    """Iterations 2.. replayed from one captured CUDA graph give exactly what
    issuing every call again gives."""
    offs = np.array([[0, 0], [3, -2], [-4, 1], [2, 5], [-1, -3]])
    raw = torch.from_numpy(_stack(256, 5, offs, seed=21)).to(DEV)
    lv = swift.Level(64, 0.65, "hann", 1.0, 3.0)
    a1, t1, h1 = align.align_stack(raw, lv, stride=48, k=2, iters=4, graph=True)
    a2, t2, h2 = align.align_stack(raw, lv, stride=48, k=2, iters=4, graph=False)
    assert h1 == h2 and len(h1) == 4
    assert torch.equal(t1, t2) and torch.equal(a1, a2)
    # a reused aligner (every iteration of the second run a replay) gives the same again
    al = align.StackAligner(5, 256, 256, lv, 48, 2, device=DEV)
    al.run(raw, 4)
    a3, t3, h3 = al.run(raw, 4)
    assert h3 == h1 and torch.equal(t3, t1) and torch.equal(a3, a1)


def test_loop_recovers_known_offsets_and_stops_when_the_snr_settles():
    rng = np.random.default_rng(5)
    offs = rng.integers(-6, 7, (6, 2))
    raw = _stack(512, 6, offs, seed=14)
    lv = swift.Level(128, 0.65, "hann", 1.0, 3.0)
    aligned, theta, hist = align.align_stack(torch.from_numpy(raw).to(DEV), lv, stride=64, k=3, iters=10, tol=0.01)
    t = theta.cpu().numpy()[:, [2, 5]]
    rel = (t - t.mean(0)) + (offs - offs.mean(0))
    assert np.abs(rel).max() < 0.3, rel
    assert hist[-1] > 1.5 * hist[0]
    assert len(hist) < 10  # stopped by the SNR rule


def test_pyramid_loop_matches_the_oracle_and_recovers_offsets():
    """Three levels (4x, 2x, full resolution), offsets up to 40 px: the device
    pyramid against the oracle's pyramid (same readings) -- per-level median
    SNR histories within 2 %, final affines within 0.1 px at the section
    corners -- and the known offsets within 0.3 px."""
    from test_oracle_driver import PYRAMID, pyramid_stack
    offs = np.random.default_rng(3).integers(-40, 41, (4, 2))
    raw = pyramid_stack(512, 4, offs, seed=31)
    P = PYRAMID
    lvs = [swift.Level(n, 0.65, "hann", 1.0, 3.0) for n in P["sizes"]]
    olvs = [swim.Level(n, 0.65, swim.APOD_HANN, 1.0, 3.0) for n in P["sizes"]]
    aligned, theta, hists = align.align_pyramid(torch.from_numpy(raw).to(DEV), P["factors"], lvs, P["strides"],
                                                P["k"], P["iters"], P["tol"], margins=P["margins"])
    oa, ot, oh = driver.align_pyramid(raw, P["factors"], olvs, P["strides"], P["k"], P["iters"], P["tol"],
                                      margins=P["margins"])
    assert [len(h) for h in hists] == [len(h) for h in oh]
    for h, o in zip(hists, oh):
        np.testing.assert_allclose(h, o, rtol=2e-2)
    theta = theta.cpu().numpy()
    for z in range(4):
        assert np.abs(_corners(theta[z], 512, 512) - _corners(ot[z], 512, 512)).max() <= 0.1, z
    t = theta[:, [2, 5]]
    assert np.abs((t - t.mean(0)) + (offs - offs.mean(0))).max() < 0.3
    assert aligned.shape == (4, 512, 512)
