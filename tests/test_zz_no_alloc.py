"""The allocation-free entry point agrees with the plan-based one.

swift_match_batch_noalloc serves callers that cannot call cudaMalloc -- code
running inside another allocator's callback, real-time loops whose device
memory must stay fixed after start-up, processes whose memory pool belongs to a
framework.  It takes no plan and keeps its scratch in a static device array.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from parity import PEAK_RTOL, SNR_RTOL, SUBPIXEL_TOL

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402
from paper_1612_04787_gb300 import _lib  # noqa: E402

DEV = "cuda:0"


def noalloc_match(level, dtype, ref, mov, ref_origin, mov_origin, out):
    """Call swift_match_batch_noalloc through the C ABI (ctypes)."""
    patch = ref_origin is None
    ri = (_lib.SwiftImage * 1)(swift._image(ref, ref.dtype, patch))
    mi = (_lib.SwiftImage * 1)(swift._image(mov, mov.dtype, patch))
    B = ref.shape[0] if patch else ref_origin.shape[0]
    bt = _lib.SwiftBatch(ri, mi, None if patch else ref_origin.data_ptr(),
                         None if patch else mov_origin.data_ptr(), None, int(B), 1 if patch else 0)
    lv = (_lib.SwiftLevel * 1)(level.c())
    code = _lib.lib.swift_match_batch_noalloc(lv, _lib.DTYPE[dtype], C.byref(bt), out.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    return code


def assert_close(a, b):
    ok = a["status"] == 0
    assert (a["status"] == b["status"]).all()
    assert (a["dy"][ok] == b["dy"][ok]).all() and (a["dx"][ok] == b["dx"][ok]).all()
    assert np.abs(a["sy"][ok] - b["sy"][ok]).max(initial=0) <= SUBPIXEL_TOL
    assert np.abs(a["sx"][ok] - b["sx"][ok]).max(initial=0) <= SUBPIXEL_TOL
    assert (np.abs(a["snr"][ok] - b["snr"][ok]) <= SNR_RTOL * np.abs(b["snr"][ok])).all()
    assert (np.abs(a["peak"][ok] - b["peak"][ok]) <= PEAK_RTOL * np.abs(b["peak"][ok]) + 1e-6).all()


def test_noalloc_matches_plan_path_twice_in_a_row():
    a, b = synth.em_section_pair(1024, seed_content=31, seed_warp=32, seed_noise=(33, 34))
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    level = swift.Level(256, 0.65, "hann", 1.0, 3.0)
    ro = synth.random_origins(24, 1024, 1024, 256, seed=35)
    mo = np.clip(ro + np.random.default_rng(36).integers(-10, 11, ro.shape), 0, 768).astype(np.int32)
    tro, tmo = torch.from_numpy(ro).to(DEV), torch.from_numpy(mo).to(DEV)
    plan = swift.Plan([level], dtype="u8", max_windows=len(ro))
    want = swift.decode(plan.match(ta, tb, tro, tmo))
    for _ in range(2):  # the static scratch keeps the previous call's contents
        out = torch.full((len(ro), 8), -7, dtype=torch.int32, device=DEV)
        assert noalloc_match(level, "u8", ta, tb, tro, tmo, out) == _lib.SWIFT_OK
        torch.cuda.synchronize()
        assert_close(swift.decode(out), want)


def test_noalloc_float_patches_and_capacity_limit():
    a, _ = synth.em_section_pair(1024, seed_content=41, seed_warp=42, seed_noise=(43, 44))
    ref, mov, _ = synth.shifted_patches(a, 128, 20, seed=45)
    tr, tm = torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)
    level = swift.Level(128, 0.5, "tukey", 0.5, 2.0)
    plan = swift.Plan([level], dtype="f32", max_windows=20)
    want = swift.decode(plan.match(tr, tm))
    for _ in range(2):
        out = torch.zeros((20, 8), dtype=torch.int32, device=DEV)
        assert noalloc_match(level, "f32", tr, tm, None, None, out) == _lib.SWIFT_OK
        torch.cuda.synchronize()
        assert_close(swift.decode(out), want)
    # 256 x 256 windows: 31 fit in the static scratch, 32 do not
    big = torch.zeros((32, 256, 256), dtype=torch.float32, device=DEV)
    out = torch.zeros((32, 8), dtype=torch.int32, device=DEV)
    lv256 = swift.Level(256, 0.65)
    assert noalloc_match(lv256, "f32", big, big, None, None, out) == _lib.SWIFT_ERR_CAPACITY
    assert noalloc_match(lv256, "f32", big[:31], big[:31], None, None, out[:31]) == _lib.SWIFT_OK
    torch.cuda.synchronize()
    assert (swift.decode(out[:31])["status"] == swift.WIN_FLAT).all()


def test_noalloc_512_matches_plan_path():
    """512 x 512 windows: 7 fit in the static scratch; results equal the plan path's."""
    a, b = synth.em_section_pair(1024, seed_content=91, seed_warp=92, seed_noise=(93, 94))
    ro = np.array([[0, 0], [500, 100], [256, 300]], np.int32)
    mo = (ro + np.array([[3, -4], [0, 7], [-5, 2]])).clip(0, 512).astype(np.int32)
    lv = swift.Level(512, 0.65, "hann", 1.0, 3.0)
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    tro, tmo = torch.from_numpy(ro).to(DEV), torch.from_numpy(mo).to(DEV)
    want = swift.decode(swift.Plan([lv], dtype="u8", max_windows=3).match(ta, tb, tro, tmo))
    for _ in range(2):
        out = torch.empty((3, 8), dtype=torch.int32, device=DEV)
        assert noalloc_match(lv, "u8", ta, tb, tro, tmo, out) == _lib.SWIFT_OK
        torch.cuda.synchronize()
        assert_close(swift.decode(out), want)
    big = torch.zeros((8, 512, 512), dtype=torch.float32, device=DEV)
    out8 = torch.empty((8, 8), dtype=torch.int32, device=DEV)
    assert noalloc_match(lv, "f32", big, big, None, None, out8) == _lib.SWIFT_ERR_CAPACITY


def test_noalloc_64_without_taper_matches_plan_path():
    """64 x 64 windows with apodisation NONE: the tables the entry point
    computes on the device for this level equal the plan's host-built ones in
    effect (same results within the parity tolerances), on two calls in a row."""
    a, b = synth.em_section_pair(512, seed_content=71, seed_warp=72, seed_noise=(73, 74))
    ro = synth.random_origins(40, 512, 512, 64, seed=75)
    mo = np.clip(ro + np.random.default_rng(76).integers(-6, 7, ro.shape), 0, 448).astype(np.int32)
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    tro, tmo = torch.from_numpy(ro).to(DEV), torch.from_numpy(mo).to(DEV)
    lv = swift.Level(64, 0.65, "none", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=len(ro))
    plan.set_schedule(0, "stream")
    want = swift.decode(plan.match(ta, tb, tro, tmo))
    for _ in range(2):
        out = torch.full((len(ro), 8), -7, dtype=torch.int32, device=DEV)
        assert noalloc_match(lv, "u8", ta, tb, tro, tmo, out) == _lib.SWIFT_OK
        torch.cuda.synchronize()
        assert_close(swift.decode(out), want)


def test_noalloc_call_replays_from_a_captured_graph():
    """Every call builds its tables on the device (no host buffer), so a call
    can be captured into a CUDA graph: each replay gives the direct call's
    records bit for bit, also after the scratch held another level's tables."""
    a, b = synth.em_section_pair(1024, seed_content=81, seed_warp=82, seed_noise=(83, 84))
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    ro = synth.random_origins(20, 1024, 1024, 256, seed=85)
    mo = np.clip(ro + np.random.default_rng(86).integers(-8, 9, ro.shape), 0, 768).astype(np.int32)
    tro, tmo = torch.from_numpy(ro).to(DEV), torch.from_numpy(mo).to(DEV)
    lv = swift.Level(256, 0.7, "tukey", 0.6, 3.0)
    want = torch.empty((len(ro), 8), dtype=torch.int32, device=DEV)
    assert noalloc_match(lv, "u8", ta, tb, tro, tmo, want) == _lib.SWIFT_OK
    torch.cuda.synchronize()
    out = torch.full_like(want, -1)
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream(device=DEV)
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=st):
        code = noalloc_match(lv, "u8", ta, tb, tro, tmo, out)
    assert code == _lib.SWIFT_OK
    for k in range(3):
        out.fill_(-1)
        if k == 1:  # another level's call in between rewrites the scratch's tables
            other = torch.empty((4, 8), dtype=torch.int32, device=DEV)
            assert noalloc_match(swift.Level(128, 0.3), "u8", ta, tb, tro[:4], tmo[:4], other) == _lib.SWIFT_OK
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, want), k
