"""Mixed-size pyramid batches: schedules, the autotuner, and CUDA-graph replay.

Pyramid stand-in: one EM-like section pair and its 2x and 4x box
downsamples (powers-of-two pyramid, Sec. III "iscale"), windows of 64, 128
and 256 px at stride n/4, whitening exponents 0.5 / 0.65 / 0.8 per level.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import swim
from parity import compare, oracle_window

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402

DEV = "cuda:0"
LEVELS = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8)]


@pytest.fixture(scope="module")
def pyramid():
    a, b = synth.em_section_pair(1024, seed_content=51, seed_warp=52, seed_noise=(53, 54))
    imgs_a = [synth.box_downsample(a, 4), synth.box_downsample(a, 2), a]
    imgs_b = [synth.box_downsample(b, 4), synth.box_downsample(b, 2), b]
    orgs, lvls = [], []
    for k, (img, lv) in enumerate(zip(imgs_a, LEVELS)):
        o = synth.grid_origins(img.shape[0], lv.n, lv.n // 4)
        orgs.append(o)
        lvls.append(np.full(len(o), k, np.int32))
    org = np.concatenate(orgs).astype(np.int32)
    lvl = np.concatenate(lvls)
    perm = np.random.default_rng(55).permutation(len(org))
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    return dict(a=imgs_a, b=imgs_b, org=org[perm], lvl=lvl[perm],
                ta=[T(x) for x in imgs_a], tb=[T(x) for x in imgs_b], to=T(org[perm]), tl=T(lvl[perm]))


def _oracle_check(P, g, idx):
    for i in idx:
        l = int(P["lvl"][i])
        lv = LEVELS[l]
        olv = swim.Level(lv.n, lv.whiten_exponent, swim.APOD_HANN, 1.0, lv.snr_exclusion_radius)
        o, tied = oracle_window(swim.gather(P["b"][l], P["org"][i], lv.n), swim.gather(P["a"][l], P["org"][i], lv.n), olv)
        compare(g, i, o, tied, lv.n, f"pyramid level {l}")


def _close(g1, g2):
    ok = (g1["status"] == 0) & (g2["status"] == 0)
    assert (g1["status"] == g2["status"]).all()
    same_peak = (g1["dy"] == g2["dy"]) & (g1["dx"] == g2["dx"])
    assert same_peak[ok].mean() > 0.995  # near-ties may flip between schedules
    sel = ok & same_peak
    assert np.abs(g1["sx"][sel] - g2["sx"][sel]).max() <= 0.02
    assert (np.abs(g1["snr"][sel] - g2["snr"][sel]) <= 1e-3 * np.abs(g2["snr"][sel])).all()


@pytest.mark.parametrize("sched", [("fused", "fused", "fused"), ("stream", "stream", "stream"), ("stream", "fused", "stream")])
def test_every_schedule_matches_the_oracle(pyramid, sched):
    P = pyramid
    plan = swift.Plan(LEVELS, dtype="u8", max_windows=len(P["org"]))
    for l, s in enumerate(sched):
        plan.set_schedule(l, s)
    g = swift.decode(plan.match(P["ta"], P["tb"], P["to"], P["to"], level=P["tl"]))
    assert (g["status"] == 0).all()
    rng = np.random.default_rng(len(sched[0]))
    idx = np.concatenate([rng.choice(np.nonzero(P["lvl"] == l)[0], 6, replace=False) for l in range(3)])
    _oracle_check(P, g, idx)


def test_autotune_then_graph_replay(pyramid):
    P = pyramid
    plan = swift.Plan(LEVELS, dtype="u8", max_windows=len(P["org"]))
    base = swift.decode(plan.match(P["ta"], P["tb"], P["to"], P["to"], level=P["tl"]))
    chosen, out = plan.autotune(P["ta"], P["tb"], P["to"], P["to"], level=P["tl"])
    assert len(chosen) == 3 and all(c in ("fused", "stream") for c in chosen)
    tuned = swift.decode(out)
    _close(tuned, base)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out_g = plan.capture(P["ta"], P["tb"], P["to"], P["to"], level=P["tl"], stream=stream)
        ref = swift.decode(out_g).copy() if False else None
        out_g.fill_(-1)
        plan.replay(stream)
    stream.synchronize()
    g1 = swift.decode(out_g)
    direct = swift.decode(plan.match(P["ta"], P["tb"], P["to"], P["to"], level=P["tl"]))
    for k in g1:
        assert (g1[k] == direct[k]).all(), k
    # new contents in the same buffers: replay follows them
    with torch.cuda.stream(stream):
        for t in P["tb"]:
            t.copy_(torch.roll(t, shifts=(3, -2), dims=(0, 1)))
        plan.replay(stream)
    stream.synchronize()
    g2 = swift.decode(out_g)
    direct2 = swift.decode(plan.match(P["ta"], P["tb"], P["to"], P["to"], level=P["tl"]))
    for k in g2:
        assert (g2[k] == direct2[k]).all(), k
    assert not (g2["dx"] == g1["dx"]).all()


def test_four_sizes_64_to_512_in_one_call_and_one_graph():
    """Windows of 64, 128, 256 and 512 px mixed in one batch: one call, the
    autotuner (512 streams only), one graph replay; oracle parity on a sample."""
    a, b = synth.em_section_pair(1024, seed_content=57, seed_warp=58, seed_noise=(59, 60))
    levels = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8), swift.Level(512, 0.65, "hann", 1.0, 4.0)]
    imgs_a = [synth.box_downsample(a, 4), synth.box_downsample(a, 2), a, a]
    imgs_b = [synth.box_downsample(b, 4), synth.box_downsample(b, 2), b, b]
    orgs, lvls = [], []
    for k, (img, lv) in enumerate(zip(imgs_a, levels)):
        o = synth.grid_origins(img.shape[0], lv.n, lv.n // 2)
        orgs.append(o)
        lvls.append(np.full(len(o), k, np.int32))
    org = np.concatenate(orgs).astype(np.int32)
    lvl = np.concatenate(lvls)
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    ta, tb, to, tl = [T(x) for x in imgs_a], [T(x) for x in imgs_b], T(org), T(lvl)
    plan = swift.Plan(levels, dtype="u8", max_windows=len(org))
    chosen, _ = plan.autotune(ta, tb, to, to, level=tl)
    assert chosen[3] == "stream"
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out = plan.capture(ta, tb, to, to, level=tl, stream=stream)
        out.fill_(-1)
        plan.replay(stream)
    stream.synchronize()
    g = swift.decode(out)
    assert (g["status"] == 0).all()
    rng = np.random.default_rng(61)
    for l, lv in enumerate(levels):
        idx = rng.choice(np.nonzero(lvl == l)[0], 2, replace=False)
        olv = swim.Level(lv.n, lv.whiten_exponent, swim.APOD_HANN, 1.0, lv.snr_exclusion_radius)
        for i in idx:
            o, tied = oracle_window(swim.gather(imgs_b[l], org[i], lv.n), swim.gather(imgs_a[l], org[i], lv.n), olv)
            compare(g, i, o, tied, lv.n, f"four sizes level {l}")


def test_calls_on_two_streams_are_ordered_by_the_plan(pyramid):
    """One plan called on two non-blocking streams, each call issued while
    the other stream's call may still run, and graph replays alternating
    with direct calls: the calls share the plan's workspace, so each waits
    for the plan's previous call, and every result equals a lone call's."""
    P = pyramid
    args = (P["ta"], P["tb"], P["to"], P["to"])
    plan = swift.Plan(LEVELS, dtype="u8", max_windows=len(P["org"]))
    for l in range(len(LEVELS)):
        plan.set_schedule(l, "stream")
    want = swift.decode(plan.match(*args, level=P["tl"]))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.full((len(P["org"]), 8), -1, dtype=torch.int32, device=DEV) for _ in range(12)]
    torch.cuda.synchronize()
    for i in range(8):
        plan.match(*args, level=P["tl"], out=outs[i], stream=s1 if i % 2 == 0 else s2)
    with torch.cuda.stream(s1):
        g_out = plan.capture(*args, level=P["tl"], stream=s1)
    for i in range(8, 12):
        plan.replay(s2 if i % 2 == 0 else s1)
        plan.match(*args, level=P["tl"], out=outs[i], stream=s1 if i % 2 == 0 else s2)
    torch.cuda.synchronize()
    for out in outs + [g_out]:
        got = swift.decode(out)
        for k in want:
            assert (got[k] == want[k]).all(), k


def test_stale_ok_status_of_another_level_is_skipped_by_the_row_guard():
    """The statistics kernel is made to report every window of another level
    as OK (the state a raced or stale workspace could leave).  It runs for the
    512 x 512 level (windows up to 256 x 256 take their statistics in the row
    kernel, which derives the status itself).  The row kernels re-check each
    window's level from the batch's own arrays, so those windows are skipped:
    every result equals the normal call's, bit for bit.  Every origin here lies
    inside every level's images, so no read could leave an image even without
    the guard (the test does not rely on it for that)."""
    a, b = synth.em_section_pair(1024, seed_content=61, seed_warp=62, seed_noise=(63, 64))
    imgs_a, imgs_b = [synth.box_downsample(a, 2), a], [synth.box_downsample(b, 2), b]
    levels = [swift.Level(128, 0.65), swift.Level(512, 0.8)]
    o = synth.grid_origins(256, 128, 32)  # origins in [0, 128]: inside 512^2 for n = 128 and 1024^2 for n = 512
    org = np.concatenate([o, o]).astype(np.int32)
    lvl = np.concatenate([np.zeros(len(o), np.int32), np.ones(len(o), np.int32)])
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    ta, tb, to, tl = [T(x) for x in imgs_a], [T(x) for x in imgs_b], T(org), T(lvl)
    plan = swift.Plan(levels, dtype="u8", max_windows=len(org))
    for l in range(2):
        plan.set_schedule(l, "stream")
    base = plan.match(ta, tb, to, to, level=tl).clone()
    assert (swift.decode(base)["status"] == 0).all()
    plan.set_test_stale_status(True)
    stale = plan.match(ta, tb, to, to, level=tl)
    plan.set_test_stale_status(False)
    torch.cuda.synchronize()
    assert torch.equal(stale, base)


@pytest.mark.parametrize("sched", ["fused", "stream", "persistent"])
def test_level_offsets_give_the_level_array_results(pyramid, sched):
    """A batch sorted by level with its level offsets: each level's launches
    cover only its own windows; the results equal the level-array call's,
    bit for bit, in every schedule (the persistent one indexes the ranges
    itself)."""
    P = pyramid
    order = np.argsort(P["lvl"], kind="stable")
    org, lvl = P["org"][order], P["lvl"][order]
    offs = [0] + [int((lvl <= k).sum()) for k in range(3)]
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    plan = swift.Plan(LEVELS, dtype="u8", max_windows=len(org))
    for l in range(3):
        plan.set_schedule(l, sched if (sched != "fused" or LEVELS[l].n <= 256) else "stream")
    want = plan.match(P["ta"], P["tb"], T(org), T(org), level=T(lvl)).clone()
    got = plan.match(P["ta"], P["tb"], T(org), T(org), level_offsets=offs)
    got2 = plan.match(P["ta"], P["tb"], T(org), T(org), level=T(lvl), level_offsets=offs)
    torch.cuda.synchronize()
    assert torch.equal(got, want) and torch.equal(got2, want)


def test_bad_level_offsets_are_rejected(pyramid):
    P = pyramid
    plan = swift.Plan(LEVELS, dtype="u8", max_windows=len(P["org"]))
    B = len(P["org"])
    for offs in ([0, 10, 5, B], [1, 10, 20, B], [0, 10, 20, B - 1]):
        with pytest.raises(ValueError):
            plan.match(P["ta"], P["tb"], P["to"], P["to"], level_offsets=offs)
    # the C boundary checks them too
    import ctypes as C
    bt, keep, _, _ = plan._batch(P["ta"], P["tb"], P["to"], P["to"], None, None, [0, 10, 20, B])
    bad = (C.c_int64 * 4)(0, 10, 5, B)
    bt.level_offsets = bad
    out = torch.empty((B, 8), dtype=torch.int32, device=DEV)
    assert swift.lib.swift_match_batch(plan.handle, C.byref(bt), out.data_ptr(), None) == swift._lib.SWIFT_ERR_INVALID_ARG
