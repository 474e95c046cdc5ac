"""Lanes of a forward call: the streaming slices and fused launches of one call
spread over the call's stream and the plan's auxiliary stream, each lane with
its own part of the workspace.  Windows are independent, so the records must
equal the single-lane records bit for bit -- for one level, for a pyramid of
three levels (fused 64 x 64 beside streaming 128 x 128 / 256 x 256), for a
batch that fills several slices per lane, inside a captured graph, and when
the next call arrives on another stream."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402

DEV = "cuda:0"
T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731


def _per_lanes(plan, *args, **kw):
    out = {}
    for k in (1, 2):
        plan.set_lanes(k)
        assert plan.lanes == k
        out[k] = plan.match(*args, **kw).clone()
    torch.cuda.synchronize()
    return out[1], out[2]


def test_default_is_two_lanes_and_bad_values_are_rejected():
    plan = swift.Plan([swift.Level(256, 0.65)], dtype="u8", max_windows=16)
    assert plan.lanes == 2
    for bad in (0, 3, -1):
        with pytest.raises(swift.SwiftError):
            plan.set_lanes(bad)
    assert plan.lanes == 2


@pytest.mark.parametrize("n,count", [(256, 301), (128, 777)])
def test_one_level_equals_one_lane(n, count):
    a, b = synth.em_section_pair(1024, seed_content=201, seed_warp=202, seed_noise=(203, 204))
    ro = synth.random_origins(count, 1024, 1024, n, seed=205)
    mo = np.clip(ro + np.random.default_rng(206).integers(-9, 10, ro.shape), 0, 1024 - n).astype(np.int32)
    ro[::41] = -3  # some windows out of bounds
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=count)
    one, two = _per_lanes(plan, T(a), T(b), T(ro), T(mo))
    assert torch.equal(one, two)
    g = swift.decode(two)
    assert (g["status"][::41] == swift.WIN_OUT_OF_BOUNDS).all() and (g["status"] == 0).sum() > 0.9 * count


def test_several_slices_per_lane():
    """max_windows above the 2048-window slice: with two lanes the 5000
    windows go out as slices of 2048, 2048 and 904, two of them on one lane."""
    a, b = synth.em_section_pair(1024, seed_content=211, seed_warp=212, seed_noise=(213, 214))
    ro = synth.random_origins(5000, 1024, 1024, 128, seed=215)
    plan = swift.Plan([swift.Level(128, 0.65)], dtype="u8", max_windows=5000)
    one, two = _per_lanes(plan, T(a), T(b), T(ro), T(ro))
    assert torch.equal(one, two)
    assert (swift.decode(two)["status"] == 0).all()


def test_pyramid_levels_share_the_lanes():
    a, b = synth.em_section_pair(1024, seed_content=221, seed_warp=222, seed_noise=(223, 224))
    imgs_a = [synth.box_downsample(a, 4), synth.box_downsample(a, 2), a]
    imgs_b = [synth.box_downsample(b, 4), synth.box_downsample(b, 2), b]
    levels = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8)]
    orgs = [synth.grid_origins(img.shape[0], lv.n, lv.n // 4) for img, lv in zip(imgs_a, levels)]
    offs = [0] + list(np.cumsum([len(o) for o in orgs]))
    org = np.concatenate(orgs).astype(np.int32)
    lvl = np.concatenate([np.full(len(o), k, np.int32) for k, o in enumerate(orgs)])
    plan = swift.Plan(levels, dtype="u8", max_windows=len(org))
    args = ([T(x) for x in imgs_a], [T(x) for x in imgs_b], T(org), T(org))
    one, two = _per_lanes(plan, *args, level=T(lvl), level_offsets=offs)
    assert torch.equal(one, two)
    # the unsorted form (a per-window level index) too
    one_u, two_u = _per_lanes(plan, *args, level=T(lvl))
    assert torch.equal(one_u, one) and torch.equal(two_u, one)


def test_graph_replay_and_a_second_stream():
    a, b = synth.em_section_pair(1024, seed_content=231, seed_warp=232, seed_noise=(233, 234))
    ro = synth.grid_origins(1024, 256, 64).astype(np.int32)
    plan = swift.Plan([swift.Level(256, 0.65)], dtype="u8", max_windows=len(ro))
    ta, tb, to = T(a), T(b), T(ro)
    plan.set_lanes(1)
    want = plan.match(ta, tb, to, to).clone()
    plan.set_lanes(2)
    st = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(st):
        out = plan.capture(ta, tb, to, to, stream=st)
        for _ in range(3):
            out.zero_()
            plan.replay(stream=st)
    st.synchronize()
    assert torch.equal(out, want)
    # calls alternating between two streams on one plan (one workspace)
    st2 = torch.cuda.Stream(device=DEV)
    outs = [torch.full_like(want, -1) for _ in range(4)]
    torch.cuda.synchronize()
    for s, o in zip((st, st2, st, st2), outs):
        plan.match(ta, tb, to, to, out=o, stream=s)
    torch.cuda.synchronize()
    assert all(torch.equal(o, want) for o in outs)


def test_tensor_core_forms_on_two_lanes():
    """The BF16X2 / FP16X2 schedules spread their slices over the lanes too
    (40 windows: two slices of 20); the records equal one lane's."""
    a, _ = synth.em_section_pair(1024, seed_content=241, seed_warp=242, seed_noise=(243, 244))
    ref, mov, _ = synth.shifted_patches(a, 128, 40, seed=245)
    for prec in ("bf16x2", "fp16x2"):
        plan = swift.Plan([swift.Level(128, 0.65)], dtype="f32", precision=prec, max_windows=40)
        one, two = _per_lanes(plan, T(ref), T(mov))
        assert torch.equal(one, two), prec
        assert (swift.decode(two)["status"] == 0).all()
