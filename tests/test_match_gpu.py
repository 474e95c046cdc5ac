"""Parity of the CUDA forward match against the FP64 oracle (through the C ABI).

Inputs are seeded synthetic stand-ins for the paper's ssEM sections: EM-like
uint8 section pairs (one warped affinely and smoothly), float32 patch pairs
with known band-limited shifts, and the 64 x 64 blurred-noise worked example.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import swim
from parity import compare, oracle_window

pytestmark = pytest.mark.gpu

swift = pytest.importorskip("paper_1612_04787_gb300") if torch.cuda.is_available() else None
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = "cuda:0"


def oracle_level(lv):
    apod = {"none": swim.APOD_NONE, "hann": swim.APOD_HANN, "tukey": swim.APOD_TUKEY}[lv.apod]
    return swim.Level(lv.n, lv.whiten_exponent, apod, lv.tukey_alpha, lv.snr_exclusion_radius)


@pytest.fixture(scope="module")
def sections():
    a, b = synth.em_section_pair(1024, seed_content=5, seed_warp=6, seed_noise=(7, 8))
    return a, b


def run_sections(a, b, ro, mo, lv, dtype="u8"):
    plan = swift.Plan([lv], dtype=dtype, max_windows=max(1, len(ro)))
    ta = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    tb = torch.from_numpy(np.ascontiguousarray(b)).to(DEV)
    tro = torch.from_numpy(ro.astype(np.int32)).to(DEV)
    tmo = torch.from_numpy(mo.astype(np.int32)).to(DEV)
    res = plan.match(ta, tb, tro, tmo)
    torch.cuda.synchronize()
    return swift.decode(res)


def check_sections(a, b, ro, mo, lv, g, where):
    olv = oracle_level(lv)
    kinds = []
    for i in range(len(ro)):
        r = swim.gather(a, ro[i], lv.n)
        m = swim.gather(b, mo[i], lv.n)
        if r is None or m is None:
            assert int(g["status"][i]) == swim.OUT_OF_BOUNDS
            continue
        ref, tied = oracle_window(m, r, olv)
        kinds.append(compare(g, i, ref, tied, lv.n, where))
    return kinds


def test_noise_pair_worked_example():
    ref, mov = synth.noise_pair(64, (-3, 5))
    lv = swift.Level(64, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", max_windows=1)
    tr = torch.from_numpy(ref.astype(np.float32)[None]).to(DEV)
    tm = torch.from_numpy(mov.astype(np.float32)[None]).to(DEV)
    g = swift.decode(plan.match(tr, tm))
    o, tied = oracle_window(mov.astype(np.float32).astype(np.float64), ref.astype(np.float32).astype(np.float64),
                            oracle_level(lv))
    assert (int(g["dy"][0]), int(g["dx"][0])) == (-3, 5)
    assert compare(g, 0, o, tied, 64, "noise pair") == "exact"


@pytest.mark.parametrize("n", [64, 128, 256])
@pytest.mark.parametrize("w", [0.0, 0.65, 1.0])
def test_sections_u8_parity(sections, n, w):
    a, b = sections
    rng = np.random.default_rng(n + int(100 * w))
    cnt = {64: 48, 128: 32, 256: 16}[n]
    ro = synth.random_origins(cnt, 1024, 1024, n, seed=n + 1)
    mo = np.clip(ro + rng.integers(-12, 13, ro.shape), 0, 1024 - n).astype(np.int32)
    lv = swift.Level(n, w, "hann", 1.0, 3.0)
    g = run_sections(a, b, ro, mo, lv)
    kinds = check_sections(a, b, ro, mo, lv, g, f"n={n} w={w}")
    assert kinds.count("exact") >= len(kinds) - 2


@pytest.mark.parametrize("apod,alpha", [("none", 1.0), ("tukey", 0.5), ("tukey", 0.25)])
def test_taper_variants(sections, apod, alpha):
    a, b = sections
    n = 128
    ro = synth.random_origins(12, 1024, 1024, n, seed=31)
    mo = ro.copy()
    lv = swift.Level(n, 0.5, apod, alpha, 2.5)
    g = run_sections(a, b, ro, mo, lv)
    check_sections(a, b, ro, mo, lv, g, f"{apod}({alpha})")


@pytest.mark.parametrize("n", [64, 128, 256])
@pytest.mark.parametrize("w", [0.0, 0.35, 1.0])
def test_exact_circular_shift_recovered(n, w):
    rng = np.random.default_rng(n)
    B = 6
    ref = rng.uniform(0, 255, (B, n, n)).astype(np.float32)
    d = rng.integers(-n // 2, n // 2, (B, 2))
    mov = np.stack([np.roll(ref[i], tuple(d[i]), axis=(0, 1)) for i in range(B)])
    lv = swift.Level(n, w, "none", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", max_windows=B)
    g = swift.decode(plan.match(torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)))
    np.testing.assert_array_equal(g["dy"], d[:, 0])
    np.testing.assert_array_equal(g["dx"], d[:, 1])
    if w == 1.0:
        np.testing.assert_allclose(g["peak"], 1.0 - 1.0 / n ** 2, rtol=1e-4)


@pytest.mark.parametrize("n", [128, 256])
def test_shifted_patches_f32(sections, n):
    a, _ = sections
    ref, mov, d = synth.shifted_patches(a, n, 8, seed=40 + n)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", max_windows=8)
    g = swift.decode(plan.match(torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)))
    olv = oracle_level(lv)
    for i in range(8):
        o, tied = oracle_window(mov[i].astype(np.float64), ref[i].astype(np.float64), olv)
        compare(g, i, o, tied, n, f"patch n={n}")
        # and the known shift is recovered to within a pixel
        assert abs(g["sy"][i] - d[i, 0]) < 1.0 and abs(g["sx"][i] - d[i, 1]) < 1.0


def test_staging_wait_runs_out_and_is_reported(sections):
    """The bounded wait of the float row staging, made to run out on purpose:
    with the test hook on, the copies expect 16 bytes that never arrive, the
    wait gives up after its bound and every window reports SWIFT_WIN_TIMEOUT
    (4); nothing faults, and the same plan then gives normal results (the
    context stays usable)."""
    a, _ = sections
    n = 128
    ref, mov, _ = synth.shifted_patches(a, n, 4, seed=77)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", max_windows=4)
    tr, tm = torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)
    base = swift.decode(plan.match(tr, tm))
    assert (base["status"] == 0).all()
    plan.set_test_stall(True)
    stalled = swift.decode(plan.match(tr, tm))
    plan.set_test_stall(False)
    assert (stalled["status"] == 4).all(), stalled["status"]
    again = swift.decode(plan.match(tr, tm))
    for k in base:
        assert (again[k] == base[k]).all(), k


@pytest.mark.parametrize("n", [128, 256])
def test_float_sections_aligned_and_unaligned_origins(sections, n):
    """float32 sections in section mode: windows whose rows start on 16-byte
    boundaries are staged by bulk asynchronous copies, the others by scalar
    loads; both kinds mixed in one call match the oracle."""
    a, b = sections
    fa = (a.astype(np.float32) * 0.5 - 3.0)
    fb = (b.astype(np.float32) * 0.5 - 3.0)
    rng = np.random.default_rng(n + 3)
    ro = synth.random_origins(8, 1024, 1024, n, seed=n + 4, margin=2)
    ro[::2] -= ro[::2] % 4  # x multiple of 4 floats: 16-byte aligned rows (pitch 1024 floats)
    mo = np.clip(ro + rng.integers(-4, 5, ro.shape), 0, 1024 - n).astype(np.int32)
    mo[0:4:2] = np.clip(ro[0:4:2] + np.array([[4, -8], [-4, 4]]), 0, 1024 - n)  # both rows aligned
    assert (ro[0:4:2, 1] % 4 == 0).all() and (mo[0:4:2, 1] % 4 == 0).all() and (mo[1::2, 1] % 4 != 0).any()
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    g = run_sections(fa, fb, ro, mo, lv, dtype="f32")
    assert (g["status"] == 0).all()
    check_sections(fa.astype(np.float64), fb.astype(np.float64), ro, mo, lv, g, f"float sections n={n}")


def test_full_size_section_pair_sampled_parity():
    """The benchmark's workload at full size and in its launch configuration:
    the 31 x 31 grid of 256^2 windows (stride 128) on the 4096^2 uint8 section
    pair with the bench's seeds, in one call.  96 sampled windows against the
    oracle; for every window, properties that hold at any size."""
    a, b = synth.em_section_pair(4096, seed_content=0, seed_warp=1, seed_noise=(2, 3))
    org = synth.grid_origins(4096, 256, 128).astype(np.int32)
    assert len(org) == 961
    lv = swift.Level(256, 0.65, "hann", 1.0, 3.0)
    g = run_sections(a, b, org, org, lv)
    assert (g["status"] == 0).all()
    assert ((g["dy"] >= -128) & (g["dy"] < 128) & (g["dx"] >= -128) & (g["dx"] < 128)).all()
    assert (np.abs(g["sy"] - g["dy"]) <= 0.5).all() and (np.abs(g["sx"] - g["dx"]) <= 0.5).all()
    assert np.isfinite(g["snr"]).all() and (g["snr"] > 0).all() and (g["peak"] > 0).all()
    olv = oracle_level(lv)
    for i in np.random.default_rng(961).choice(961, 96, replace=False):
        o, tied = oracle_window(swim.gather(b, org[i], 256), swim.gather(a, org[i], 256), olv)
        compare(g, int(i), o, tied, 256, "full-size sections")


def test_projection_reference(sections):
    a, b = sections
    n = 128
    stack = np.stack([a, np.roll(a, 1, axis=1), np.roll(a, -1, axis=0)])
    ro = synth.random_origins(6, 1024, 1024, n, seed=3, margin=2)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=6)
    g = swift.decode(plan.match(torch.from_numpy(stack).to(DEV), torch.from_numpy(b).to(DEV),
                                torch.from_numpy(ro).to(DEV), torch.from_numpy(ro).to(DEV)))
    olv = oracle_level(lv)
    for i in range(6):
        r = swim.project(list(stack), ro[i], n)
        m = swim.gather(b, ro[i], n)
        o, tied = oracle_window(m, r.astype(np.float32).astype(np.float64), olv)
        compare(g, i, o, tied, n, "projection")


def test_mixed_levels_one_call(sections):
    a, b = sections
    a2, b2 = synth.box_downsample(a, 2), synth.box_downsample(b, 2)
    a4, b4 = synth.box_downsample(a, 4), synth.box_downsample(b, 4)
    levels = [swift.Level(64, 0.5), swift.Level(128, 0.65), swift.Level(256, 0.8)]
    imgs_a, imgs_b = [a4, a2, a], [b4, b2, b]
    o = [synth.grid_origins(img.shape[0], lv.n, lv.n // 2)[::5] for img, lv in zip(imgs_a, levels)]
    lvl = np.concatenate([np.full(len(x), k, np.int32) for k, x in enumerate(o)])
    org = np.concatenate(o).astype(np.int32)
    perm = np.random.default_rng(0).permutation(len(org))
    org, lvl = org[perm], lvl[perm]
    plan = swift.Plan(levels, dtype="u8", max_windows=len(org))
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    g = swift.decode(plan.match([T(x) for x in imgs_a], [T(x) for x in imgs_b], T(org), T(org), level=T(lvl)))
    for i in range(len(org)):
        lv = levels[lvl[i]]
        r = swim.gather(imgs_a[lvl[i]], org[i], lv.n)
        m = swim.gather(imgs_b[lvl[i]], org[i], lv.n)
        ref, tied = oracle_window(m, r, oracle_level(lv))
        compare(g, i, ref, tied, lv.n, f"mixed level {lvl[i]}")


def test_status_codes_and_empty_batch():
    n = 64
    lv = swift.Level(n, 0.65, "hann")
    sec = torch.from_numpy(np.random.default_rng(1).integers(0, 256, (200, 300)).astype(np.uint8)).to(DEV)
    flat = torch.full((200, 300), 9, dtype=torch.uint8, device=DEV)
    plan = swift.Plan([lv], dtype="u8", max_windows=4)
    o = torch.tensor([[0, 0], [150, 10], [10, 250], [136, 236]], dtype=torch.int32, device=DEV)
    g = swift.decode(plan.match(sec, sec, o, o))
    assert list(g["status"]) == [0, 1, 1, 0]
    g = swift.decode(plan.match(flat, sec, o, o))
    assert list(g["status"]) == [2, 1, 1, 2]
    empty = torch.zeros((0, 2), dtype=torch.int32, device=DEV)
    out = plan.match(sec, sec, empty, empty)
    assert out.shape == (0, 8)
    fplan = swift.Plan([lv], dtype="f32", max_windows=2)
    p = torch.randn(2, n, n, device=DEV)
    q = p.clone()
    q[1, 5, 7] = float("nan")
    g = swift.decode(fplan.match(p, q))
    assert list(g["status"]) == [0, 3]
    with pytest.raises(swift.SwiftError):
        plan.match(sec, sec, torch.zeros((5, 2), dtype=torch.int32, device=DEV),
                   torch.zeros((5, 2), dtype=torch.int32, device=DEV))  # beyond max_windows


def test_deterministic(sections):
    a, b = sections
    n = 256
    ro = synth.random_origins(16, 1024, 1024, n, seed=9)
    lv = swift.Level(n, 0.65)
    plan = swift.Plan([lv], dtype="u8", max_windows=16)
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    r1 = plan.match(T(a), T(b), T(ro), T(ro)).clone()
    r2 = plan.match(T(a), T(b), T(ro), T(ro))
    assert torch.equal(r1, r2)


@pytest.mark.parametrize("n", [64, 256])
def test_persistent_loop_many_windows(sections, n):
    """Far more windows than resident clusters, with out-of-bounds windows
    mixed into every cluster's chain of staged loads."""
    a, b = sections
    rng = np.random.default_rng(77 + n)
    B = 1500 if n == 64 else 700
    ro = synth.random_origins(B, 1024, 1024, n, seed=n)
    mo = np.clip(ro + rng.integers(-6, 7, ro.shape), 0, 1024 - n).astype(np.int32)
    bad = rng.choice(B, B // 10, replace=False)
    mo[bad, 1] = 1024 - n + 1 + rng.integers(0, 40, len(bad))  # leaves the section
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    g = run_sections(a, b, ro, mo, lv)
    assert set(np.nonzero(g["status"] == swim.OUT_OF_BOUNDS)[0]) == set(bad)
    assert (g["status"][np.setdiff1d(np.arange(B), bad)] == 0).all()
    sample = rng.choice(np.setdiff1d(np.arange(B), bad), 24, replace=False)
    olv = oracle_level(lv)
    for i in sample:
        o, tied = oracle_window(swim.gather(b, mo[i], n), swim.gather(a, ro[i], n), olv)
        compare(g, i, o, tied, n, f"persistent n={n}")
    # the same pair anywhere in the batch gives bit-identical results
    ro2 = np.concatenate([ro[:1]] * 300)
    mo2 = np.concatenate([mo[sample[:1]]] * 300)
    ro2[:, :] = ro[sample[0]]
    g2 = run_sections(a, b, ro2, mo2, lv)
    for k in ("dy", "dx", "sy", "sx", "snr", "peak", "status"):
        assert (g2[k] == g2[k][0]).all()
        assert g2[k][0] == g[k][sample[0]]


def test_unaligned_section_width_uses_direct_loads(sections):
    a, b = sections
    n = 128
    aw, bw = np.ascontiguousarray(a[:, :1001]), np.ascontiguousarray(b[:, :1001])  # width % 16 != 0
    ro = synth.random_origins(20, 1024, 1001, n, seed=5)
    lv = swift.Level(n, 0.65)
    g = run_sections(aw, bw, ro, ro, lv)
    check_sections(aw, bw, ro, ro, lv, g, "width 1001")


@pytest.mark.parametrize("w", [0.0, 0.65, 1.0])
def test_sections_512_parity(w):
    """512 x 512 windows (streaming schedule, 16 x 32 radix)."""
    a, b = synth.em_section_pair(1024, seed_content=81, seed_warp=82, seed_noise=(83, 84))
    ro = np.array([[0, 0], [300, 200], [512, 512], [100, 480]], np.int32)
    rng = np.random.default_rng(int(10 * w))
    mo = np.clip(ro + rng.integers(-20, 21, ro.shape), 0, 1024 - 512).astype(np.int32)
    lv = swift.Level(512, w, "hann", 1.0, 4.0)
    g = run_sections(a, b, ro, mo, lv)
    kinds = check_sections(a, b, ro, mo, lv, g, f"512 w={w}")
    assert kinds.count("exact") >= 3


def test_512_schedule_and_warp_limits():
    plan = swift.Plan([swift.Level(512, 0.65, "hann", 1.0, 3.0)], dtype="u8", max_windows=4)
    with pytest.raises(swift.SwiftError) as e:
        plan.set_schedule(0, "fused")
    assert "UNSUPPORTED" in str(e.value)
    sec = torch.zeros((1024, 1024), dtype=torch.uint8, device=DEV)
    org = torch.zeros((2, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(swift.SwiftError) as e:
        plan.match(sec, sec, org, org, affine=torch.zeros((2, 6), dtype=torch.float32, device=DEV))
    assert "UNSUPPORTED" in str(e.value)


@pytest.mark.parametrize("n", [128, 256])
@pytest.mark.parametrize("radius", [0.0, 0.9, 1.0, 7.9, 8.0, 20.0])
def test_exclusion_radius_range(sections, n, radius):
    """The finalize in its two forms: folded into the last inverse-row block
    (radius below 8 px: the rows within the radius recomputed) and as a kernel
    of its own (8 px and more, several chunks of row pairs at 20 px), and the
    smallest radii (the parabola's neighbours still recomputed)."""
    a, b = sections
    ro = synth.random_origins(10, 1024, 1024, n, seed=int(10 * radius) + n)
    mo = np.clip(ro + np.random.default_rng(n).integers(-6, 7, ro.shape), 0, 1024 - n).astype(np.int32)
    lv = swift.Level(n, 0.65, "hann", 1.0, radius)
    g = run_sections(a, b, ro, mo, lv)
    check_sections(a, b, ro, mo, lv, g, f"n={n} r={radius}")
