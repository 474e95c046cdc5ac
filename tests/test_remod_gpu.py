"""Pyramid (iscale) and Z-model (remod) kernels against the oracle, through
the C ABI: bit-exact (integer sums, exact rounding, one IEEE division)."""
import numpy as np
import pytest
import torch

import synth
from oracle import remod

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("f", [2, 3, 5])
def test_downsample_uint8_bit_exact(f):
    a, _ = synth.em_section_pair(512, seed_content=61, seed_warp=62, seed_noise=(63, 64))
    img = np.ascontiguousarray(a[:301, :443])
    got = swift.downsample(torch.from_numpy(img).to(DEV), f).cpu().numpy()
    np.testing.assert_array_equal(got, remod.downsample(img, f))


@pytest.mark.parametrize("f", [2, 4])
def test_downsample_uint8_batch_vector_path(f):
    """A batch of aligned sections (the 8/16-byte vector path) in one launch."""
    stack = synth.section_stack(256, depth=3, seed=8 + f)
    got = swift.downsample(torch.from_numpy(stack).to(DEV), f).cpu().numpy()
    for z in range(3):
        np.testing.assert_array_equal(got[z], remod.downsample(stack[z], f))


@pytest.mark.parametrize("width", [264, 256])  # 2x: four outputs per thread (W = 132), eight (W = 128)
def test_downsample_uint8_2x_vector_widths(width):
    rng = np.random.default_rng(width)
    img = rng.integers(0, 256, (2, 40, width)).astype(np.uint8)
    got = swift.downsample(torch.from_numpy(img).to(DEV), 2).cpu().numpy()
    for z in range(2):
        np.testing.assert_array_equal(got[z], remod.downsample(img[z], 2))


@pytest.mark.parametrize("f", [2, 4])
def test_downsample_float32_bit_exact(f):
    rng = np.random.default_rng(f)
    img = rng.uniform(-50, 300, (130, 257)).astype(np.float32)
    got = swift.downsample(torch.from_numpy(img).to(DEV), f).cpu().numpy()
    np.testing.assert_array_equal(got, remod.downsample(img, f))


@pytest.mark.parametrize("k", [1, 4])
@pytest.mark.parametrize("width", [256, 260, 257])  # 16-pixel, 4-pixel and scalar paths
def test_zmodel_bit_exact(k, width):
    rng = np.random.default_rng(k + width)
    stack = rng.integers(0, 256, (9, 40, width)).astype(np.uint8)
    valid = np.ones(9, bool)
    valid[[3, 7]] = False
    got = swift.zmodel(torch.from_numpy(stack).to(DEV), k, valid=torch.from_numpy(valid.astype(np.uint8))).cpu().numpy()
    np.testing.assert_array_equal(got, remod.zmodel(stack, k, valid))
    got = swift.zmodel(torch.from_numpy(stack).to(DEV), k).cpu().numpy()
    np.testing.assert_array_equal(got, remod.zmodel(stack, k))


def test_zmodel_feeds_the_match_as_a_reference():
    """The model of section z (from a drifting stack) matches section z at a
    near-zero shift with a higher SNR than the single neighbour section."""
    stack = synth.section_stack(512, depth=5, seed=71)
    ts = torch.from_numpy(stack).to(DEV)
    model = swift.zmodel(ts, 2)
    n = 128
    org = torch.from_numpy(synth.grid_origins(512, n, 96)).to(DEV)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="f32", max_windows=int(org.shape[0]))
    r_model = swift.decode(plan.match(model[2].contiguous(), ts[2].float().contiguous(), org, org))
    r_single = swift.decode(plan.match(ts[1].float().contiguous(), ts[2].float().contiguous(), org, org))
    assert (r_model["status"] == 0).all()
    assert np.median(r_model["snr"]) > np.median(r_single["snr"])
    assert np.abs(r_model["sy"]).max() < 2.0 and np.abs(r_model["sx"]).max() < 2.0


@pytest.mark.parametrize("width", [256, 260, 257])  # 16-pixel, 4-pixel and scalar paths
def test_zmodel_uint8_bit_exact(width):
    rng = np.random.default_rng(width)
    stack = rng.integers(0, 256, (7, 33, width)).astype(np.uint8)
    got = swift.zmodel(torch.from_numpy(stack).to(DEV), 3, dtype=torch.uint8).cpu().numpy()
    np.testing.assert_array_equal(got, remod.zmodel(stack, 3, dtype=np.uint8))
