"""The row kernel's tensor-map (TMA) tile copies of uint8 section windows.

A tile copy takes the rows of one row block from the 16-byte chunk that
holds the window's first column, so it starts aligned whatever the origin,
and the kernel reads the window from the origin's offset in that chunk.  The
pixels reaching the transforms are the same bytes as with plain loads, so
every record must equal the plain-load record bit for bit, in each of the
three modes (0 plain loads, 1 tile copies for unaligned windows only, 2 tile
copies for every window) -- at every window size, for windows touching the
images' right and bottom edges, for out-of-bounds and other-level windows,
and for images the maps cannot describe (a width or an address off a 16-byte
boundary), which load as with mode 0.  Parity against the FP64 oracle on
windows at every offset within a chunk closes the loop."""
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


def _per_mode(plan, *args, **kw):
    out = {}
    for mode in (0, 1, 2):
        plan.set_row_tma(mode)
        assert plan.row_tma == mode
        out[mode] = plan.match(*args, **kw).clone()
    torch.cuda.synchronize()
    return out


def _origins(count, h, w, n, seed):
    """Random origins, every x offset within a 16-byte chunk present, plus
    windows flush with the right and bottom edges and a few out of bounds."""
    rng = np.random.default_rng(seed)
    o = synth.random_origins(count, h, w, n, seed=seed)
    o[:16, 1] = (o[:16, 1] // 16) * 16 + np.arange(16)
    o[:16, 1] = np.minimum(o[:16, 1], w - n)
    o[16] = (h - n, w - n)
    o[17] = (h - n, w - n - 5)
    o[18] = (0, 0)
    o[19] = (rng.integers(0, h - n), w - n - 1)
    o[-1] = (-2, 7)
    o[-2] = (3, w - n + 1)
    return o.astype(np.int32)


def test_default_mode_and_bad_values_are_rejected():
    plan = swift.Plan([swift.Level(256, 0.65)], dtype="u8", max_windows=4)
    assert plan.row_tma == 1
    for bad in (-1, 3):
        with pytest.raises(swift.SwiftError):
            plan.set_row_tma(bad)
    assert plan.row_tma == 1


@pytest.mark.parametrize("n,count", [(64, 200), (128, 150), (256, 90), (512, 40)])
def test_modes_are_bit_identical(n, count):
    a, b = synth.em_section_pair(1024, seed_content=301, seed_warp=302, seed_noise=(303, 304))
    ro = _origins(count, 1024, 1024, n, seed=305 + n)
    mo = _origins(count, 1024, 1024, n, seed=306 + n)
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=count)
    out = _per_mode(plan, T(a), T(b), T(ro), T(mo))
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])
    g = swift.decode(out[2])
    assert (g["status"][-2:] == swift.WIN_OUT_OF_BOUNDS).all()
    assert (g["status"] == 0).sum() >= count - 4


def test_pyramid_with_other_level_windows():
    """Levels of 64, 128 and 256 in one call (each level's launches skip the
    other levels' windows before any load) on one lane and on two."""
    a, b = synth.em_section_pair(1024, seed_content=311, seed_warp=312, seed_noise=(313, 314))
    rng = np.random.default_rng(315)
    levels = [swift.Level(64, 0.65), swift.Level(128, 0.65), swift.Level(256, 0.65)]
    count = 300
    lvl = rng.integers(0, 3, count).astype(np.int32)
    ro = np.stack([synth.random_origins(count, 1024, 1024, 256, seed=316)[:, 0],
                   rng.integers(0, 1024 - 256, count)], 1).astype(np.int32)
    mo = np.clip(ro + rng.integers(-7, 8, ro.shape), 0, 1024 - 256).astype(np.int32)
    plan = swift.Plan(levels, dtype="u8", max_windows=count)
    for lanes in (1, 2):
        plan.set_lanes(lanes)
        out = _per_mode(plan, [T(a)] * 3, [T(b)] * 3, T(ro), T(mo), level=T(lvl))
        assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2]), lanes


def test_images_the_maps_cannot_describe_load_plainly():
    """A width off a 16-byte boundary (1000 columns) and an image whose first
    byte is off a 16-byte boundary (a view from column 3): no tile copies,
    the same records in every mode."""
    a, b = synth.em_section_pair(1024, seed_content=321, seed_warp=322, seed_noise=(323, 324))
    n, count = 128, 60
    ro = synth.random_origins(count, 1000, 1000, n, seed=325)
    mo = synth.random_origins(count, 1000, 1000, n, seed=326)
    plan = swift.Plan([swift.Level(n, 0.65)], dtype="u8", max_windows=count)
    narrow = _per_mode(plan, T(a[:1000, :1000]), T(b[:1000, :1000]), T(ro), T(mo))
    assert torch.equal(narrow[0], narrow[2])
    ta, tb = T(a), T(b)
    va, vb = ta[:, 3:1003], tb[:, 3:1003]
    assert va.data_ptr() % 16 == 3
    view = _per_mode(plan, va, vb, T(ro), T(mo))
    assert torch.equal(view[0], view[2])
    # the view is the same pixels as the 1000-column copy starting at column 3
    same = plan.match(T(a[:, 3:1003]), T(b[:, 3:1003]), T(ro), T(mo))
    assert torch.equal(view[2], same)


@pytest.mark.parametrize("n", [128, 256])
def test_tile_copies_match_the_oracle(n):
    """Mode 2 (every window through the tile copies) on windows at each of
    the 16 offsets within a chunk, against the FP64 oracle."""
    a, b = synth.em_section_pair(1024, seed_content=331, seed_warp=332, seed_noise=(333, 334))
    rng = np.random.default_rng(335 + n)
    ro = synth.random_origins(16, 1024, 1024, n, seed=336 + n)
    ro[:, 1] = np.minimum((ro[:, 1] // 16) * 16 + np.arange(16), 1024 - n)
    mo = np.clip(ro + rng.integers(-9, 10, ro.shape), 0, 1024 - n).astype(np.int32)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=16)
    plan.set_row_tma(2)
    g = swift.decode(plan.match(T(a), T(b), T(ro), T(mo)))
    olv = swim.Level(n, 0.65, swim.APOD_HANN, 1.0, 3.0)
    kinds = []
    for i in range(16):
        ref, tied = oracle_window(swim.gather(b, mo[i], n), swim.gather(a, ro[i], n), olv)
        kinds.append(compare(g, i, ref, tied, n, f"tma n={n} x={ro[i, 1]}"))
    assert kinds.count("exact") >= len(kinds) - 1


def test_tile_copy_wait_runs_out_and_is_reported():
    """The bounded wait on the tile copies, made to run out on purpose: with
    the test hook on, the copies expect 16 bytes that never arrive, the wait
    gives up after its bound and every window reports SWIFT_WIN_TIMEOUT (4);
    nothing faults and the same plan then gives its normal records."""
    a, b = synth.em_section_pair(1024, seed_content=341, seed_warp=342, seed_noise=(343, 344))
    n = 128
    ro = synth.random_origins(4, 1024, 1024, n, seed=345)
    ro[:, 1] = np.minimum(ro[:, 1] | 1, 1024 - n - 1)  # rows off a 16-byte boundary: tile copies by default
    plan = swift.Plan([swift.Level(n, 0.65)], dtype="u8", max_windows=4)
    args = (T(a), T(b), T(ro), T(ro))
    base = plan.match(*args).clone()
    assert (swift.decode(base)["status"] == 0).all()
    plan.set_test_stall(True)
    stalled = swift.decode(plan.match(*args))
    plan.set_test_stall(False)
    assert (stalled["status"] == 4).all(), stalled["status"]
    assert torch.equal(plan.match(*args), base)
