"""The persistent schedule (opt-in): every window of every level in one launch.

Its work items run the same stage code as the five-kernel streaming schedule,
so its results must equal that schedule's bit for bit (which the streaming
schedule's own parity tests tie to the oracle); a pyramid batch must take one
launch; and its bounded waits must give up cleanly when made to run out."""
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
T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731


def _both(plan, levels, *args, **kw):
    out = {}
    for sched in ("stream", "persistent"):
        for l in range(levels):
            plan.set_schedule(l, sched)
        out[sched] = plan.match(*args, **kw).clone()
    torch.cuda.synchronize()
    return out["stream"], out["persistent"]


@pytest.mark.parametrize("n,count", [(256, 300), (128, 700), (64, 1500)])
def test_sections_equal_the_streaming_schedule(n, count):
    a, b = synth.em_section_pair(1024, seed_content=101, seed_warp=102, seed_noise=(103, 104))
    ro = synth.random_origins(count, 1024, 1024, n, seed=105)
    mo = np.clip(ro + np.random.default_rng(106).integers(-9, 10, ro.shape), 0, 1024 - n).astype(np.int32)
    ro[::37] = -5  # some windows out of bounds
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=count)
    s, p = _both(plan, 1, T(a), T(b), T(ro), T(mo))
    assert torch.equal(s, p)
    g = swift.decode(p)
    assert (g["status"][::37] == swift.WIN_OUT_OF_BOUNDS).all() and (g["status"] == 0).sum() > 0.9 * count


def test_float_patches_and_tukey_equal_the_streaming_schedule():
    a, _ = synth.em_section_pair(1024, seed_content=111, seed_warp=112, seed_noise=(113, 114))
    ref, mov, _ = synth.shifted_patches(a, 128, 257, seed=115)
    plan = swift.Plan([swift.Level(128, 0.3, "tukey", 0.5, 2.5)], dtype="f32", max_windows=257)
    s, p = _both(plan, 1, T(ref), T(mov))
    assert torch.equal(s, p)


def test_pyramid_is_one_launch_and_equals_the_streaming_schedule():
    a, b = synth.em_section_pair(1024, seed_content=121, seed_warp=122, seed_noise=(123, 124))
    imgs_a = [synth.box_downsample(a, 4), synth.box_downsample(a, 2), a]
    imgs_b = [synth.box_downsample(b, 4), synth.box_downsample(b, 2), b]
    levels = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8)]
    orgs, lvls = [], []
    for k, (img, lv) in enumerate(zip(imgs_a, levels)):
        o = synth.grid_origins(img.shape[0], lv.n, lv.n // 4)
        orgs.append(o)
        lvls.append(np.full(len(o), k, np.int32))
    perm = np.random.default_rng(125).permutation(sum(len(o) for o in orgs))
    org, lvl = np.concatenate(orgs)[perm].astype(np.int32), np.concatenate(lvls)[perm]
    plan = swift.Plan(levels, dtype="u8", max_windows=len(org))
    args = ([T(x) for x in imgs_a], [T(x) for x in imgs_b], T(org), T(org))
    s, p = _both(plan, 3, *args, level=T(lvl))
    assert torch.equal(s, p)
    plan.set_timing(True)
    plan.timings()
    plan.match(*args, level=T(lvl))
    t = plan.timings()
    plan.set_timing(False)
    assert set(t) == {"persistent"} and t["persistent"][1] == 1, t
    g = swift.decode(p)
    assert (g["status"] == 0).all()
    # a few windows of every level against the oracle
    rng = np.random.default_rng(126)
    for k, lv in enumerate(levels):
        olv = swim.Level(lv.n, lv.whiten_exponent, swim.APOD_HANN, 1.0, 3.0)
        for i in rng.choice(np.nonzero(lvl == k)[0], 4, replace=False):
            o, tied = oracle_window(swim.gather(imgs_b[k], org[i], lv.n), swim.gather(imgs_a[k], org[i], lv.n), olv)
            compare(g, i, o, tied, lv.n, f"level {k}")


def test_graph_replay_of_the_persistent_launch():
    a, b = synth.em_section_pair(1024, seed_content=131, seed_warp=132, seed_noise=(133, 134))
    ro = synth.grid_origins(1024, 256, 128).astype(np.int32)
    plan = swift.Plan([swift.Level(256, 0.65)], dtype="u8", max_windows=len(ro))
    plan.set_schedule(0, "persistent")
    ta, tb, to = T(a), T(b), T(ro)
    want = plan.match(ta, tb, to, to).clone()
    st = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(st):
        out = plan.capture(ta, tb, to, to, stream=st)
        for _ in range(3):
            out.zero_()
            plan.replay(stream=st)
    st.synchronize()
    assert torch.equal(out, want)


def test_small_batches():
    a, b = synth.em_section_pair(512, seed_content=141, seed_warp=142, seed_noise=(143, 144))
    plan = swift.Plan([swift.Level(256, 0.65)], dtype="u8", max_windows=8)
    for B in (1, 2, 5):
        ro = synth.random_origins(B, 512, 512, 256, seed=145 + B)
        s, p = _both(plan, 1, T(a), T(b), T(ro), T(ro))
        assert torch.equal(s, p)


def test_a_wait_that_runs_out_reports_timeouts_and_the_plan_recovers():
    """The test hook holds back the row items of one window: the wait for
    them gives up after its (shortened) bound, the launch stops its remaining
    work, and windows not finished by then report SWIFT_WIN_TIMEOUT; every
    other window's record equals the normal result, and the next call is
    normal again."""
    a, b = synth.em_section_pair(1024, seed_content=151, seed_warp=152, seed_noise=(153, 154))
    ro = synth.grid_origins(1024, 256, 64).astype(np.int32)  # 169 windows
    plan = swift.Plan([swift.Level(256, 0.65)], dtype="u8", max_windows=len(ro))
    plan.set_schedule(0, "persistent")
    ta, tb, to = T(a), T(b), T(ro)
    want = plan.match(ta, tb, to, to).clone()
    plan.set_test_hold(40)
    out = torch.full_like(want, -1)
    plan.match(ta, tb, to, to, out=out)
    torch.cuda.synchronize()
    plan.set_test_hold(-1)
    g = swift.decode(out)
    assert g["status"][40] == swift.WIN_TIMEOUT
    done = g["status"] != swift.WIN_TIMEOUT
    assert torch.equal(out[torch.from_numpy(done).to(DEV)], want[torch.from_numpy(done).to(DEV)])
    again = plan.match(ta, tb, to, to)
    torch.cuda.synchronize()
    assert torch.equal(again, want)
