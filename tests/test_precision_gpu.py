"""Tensor-core precision variant against the FP64 oracle (through the C ABI).

The transforms run as BF16 or FP16 DFT-matrix GEMMs on the tensor cores with
FP32 accumulation and hi+lo split operands (three products per term); the
statistics, SNR and subpixel fit are the FP64-accumulated kernels of the FP32
path.  Inputs: float32 patch pairs with known band-limited subpixel shifts
cut from an EM-like section (the precision workload), and uint8 section
windows including a projected (multi-section) reference.
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
PRECISIONS = ["bf16x2", "fp16x2"]


def oracle_level(lv):
    apod = {"none": swim.APOD_NONE, "hann": swim.APOD_HANN, "tukey": swim.APOD_TUKEY}[lv.apod]
    return swim.Level(lv.n, lv.whiten_exponent, apod, lv.tukey_alpha, lv.snr_exclusion_radius)


@pytest.fixture(scope="module")
def section():
    a, _ = synth.em_section_pair(1024, seed_content=60, seed_warp=61, seed_noise=(62, 63))
    return a


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n", [128, 256])
@pytest.mark.parametrize("w", [0.0, 0.65, 1.0])
def test_patches_parity(section, prec, n, w):
    cnt = {128: 12, 256: 6}[n]
    ref, mov, d = synth.shifted_patches(section, n, cnt, seed=10 + n)
    lv = swift.Level(n, w, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", precision=prec, max_windows=cnt)
    g = swift.decode(plan.match(torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)))
    torch.cuda.synchronize()
    olv = oracle_level(lv)
    for i in range(cnt):
        o, tied = oracle_window(mov[i].astype(np.float64), ref[i].astype(np.float64), olv)
        compare(g, i, o, tied, n, f"{prec} n={n} w={w}")


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n", [128, 256])
def test_sections_u8_parity(prec, n):
    a, b = synth.em_section_pair(1024, seed_content=5, seed_warp=6, seed_noise=(7, 8))
    cnt = {128: 16, 256: 8}[n]
    ro = synth.random_origins(cnt, 1024, 1024, n, seed=n + 3)
    rng = np.random.default_rng(n)
    mo = np.clip(ro + rng.integers(-12, 13, ro.shape), 0, 1024 - n).astype(np.int32)
    mo[0] = (1024 - n + 5, 0)  # out of bounds
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", precision=prec, max_windows=cnt)
    res = plan.match(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV),
                     torch.from_numpy(ro.astype(np.int32)).to(DEV), torch.from_numpy(mo).to(DEV))
    g = swift.decode(res)
    olv = oracle_level(lv)
    assert int(g["status"][0]) == swim.OUT_OF_BOUNDS
    for i in range(1, cnt):
        o, tied = oracle_window(swim.gather(b, mo[i], n), swim.gather(a, ro[i], n), olv)
        compare(g, i, o, tied, n, f"{prec} sections n={n}")


@pytest.mark.parametrize("prec", PRECISIONS)
def test_projected_reference(prec):
    """Reference = mean of three sections (the paper's projection), u8."""
    stack = synth.section_stack(512, depth=4, seed=20)
    n = 128
    ro = synth.random_origins(8, 512, 512, n, seed=4)
    mo = ro.copy()
    lv = swift.Level(n, 0.5, "tukey", 0.5, 2.0)
    plan = swift.Plan([lv], dtype="u8", precision=prec, max_windows=8)
    refs = torch.from_numpy(np.ascontiguousarray(stack[1:])).to(DEV)
    mov = torch.from_numpy(np.ascontiguousarray(stack[0])).to(DEV)
    g = swift.decode(plan.match(refs, mov, torch.from_numpy(ro).to(DEV), torch.from_numpy(mo).to(DEV)))
    olv = oracle_level(lv)
    for i in range(8):
        r = swim.project(stack[1:], ro[i], n)
        o, tied = oracle_window(swim.gather(stack[0], mo[i], n), r, olv)
        compare(g, i, o, tied, n, f"{prec} projection")


@pytest.mark.parametrize("prec", PRECISIONS)
def test_slices_and_empty(section, prec):
    """More windows than one workspace slice; an empty batch is a no-op."""
    n = 128
    cnt = 2048 + 40
    ref, mov, d = synth.shifted_patches(section, n, 64, seed=3)
    idx = np.arange(cnt) % 64
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="f32", precision=prec, max_windows=cnt)
    tr, tm = torch.from_numpy(ref[idx]).to(DEV), torch.from_numpy(mov[idx]).to(DEV)
    g = swift.decode(plan.match(tr, tm))
    for k in ("dy", "dx", "sy", "sx", "snr", "peak"):
        v = np.asarray(g[k]).reshape(-1)
        assert np.array_equal(v[:40], v[2048:]), k  # the second slice repeats the first windows
    assert (np.asarray(g["status"]) == 0).all()
    sec = torch.zeros((512, 512), dtype=torch.float32, device=DEV)
    empty = torch.zeros((0, 2), dtype=torch.int32, device=DEV)
    assert plan.match(sec, sec, empty, empty).shape[0] == 0


@pytest.mark.parametrize("prec", PRECISIONS)
def test_agrees_with_fp32_path(section, prec):
    """Same integer peaks as the FP32 path; subpixel and SNR within tolerance."""
    n = 256
    ref, mov, d = synth.shifted_patches(section, n, 32, seed=99)
    tr, tm = torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    g32 = swift.decode(swift.Plan([lv], dtype="f32", max_windows=32).match(tr, tm))
    gtc = swift.decode(swift.Plan([lv], dtype="f32", precision=prec, max_windows=32).match(tr, tm))
    assert np.array_equal(np.asarray(g32["dy"]), np.asarray(gtc["dy"]))
    assert np.array_equal(np.asarray(g32["dx"]), np.asarray(gtc["dx"]))
    assert np.abs(np.asarray(g32["sy"]) - np.asarray(gtc["sy"])).max() <= 0.02
    assert np.abs(np.asarray(g32["sx"]) - np.asarray(gtc["sx"])).max() <= 0.02
    rel = np.abs(np.asarray(g32["snr"]) - np.asarray(gtc["snr"])) / np.abs(np.asarray(g32["snr"]))
    assert rel.max() <= 2e-3
    # the known shift of the generator is recovered to well within a pixel
    assert np.abs(np.asarray(gtc["sy"]) - d[:, 0]).max() < 0.5
    assert np.abs(np.asarray(gtc["sx"]) - d[:, 1]).max() < 0.5


def test_reduced_precision_rejects_warp():
    n = 128
    plan = swift.Plan([swift.Level(n, 0.65, "hann", 1.0, 3.0)], dtype="u8", precision="bf16x2", max_windows=4)
    a = torch.zeros((512, 512), dtype=torch.uint8, device=DEV)
    o = torch.zeros((4, 2), dtype=torch.int32, device=DEV) + 100
    aff = torch.zeros((4, 6), dtype=torch.float32, device=DEV)
    with pytest.raises(swift.SwiftError) as e:
        plan.match(a, a, o, o, affine=aff)
    assert "UNSUPPORTED" in str(e.value)
