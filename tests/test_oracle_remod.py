"""Pins of the pyramid (iscale) and model (remod) oracle against closed forms
and hand-worked values."""
import numpy as np
import pytest

from oracle import remod


def test_downsample_identity_constant_and_ramp():
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (13, 17)).astype(np.uint8)
    np.testing.assert_array_equal(remod.downsample(img, 1), img)
    assert (remod.downsample(np.full((12, 9), 77, np.uint8), 3) == 77).all()
    # a linear ramp's block means are the ramp at the block centres (exact in float32)
    y, x = np.meshgrid(np.arange(20.0), np.arange(30.0), indexing="ij")
    ramp = (2.0 * y + 0.5 * x).astype(np.float32)
    out = remod.downsample(ramp, 5)
    yc, xc = np.meshgrid(5 * np.arange(4) + 2.0, 5 * np.arange(6) + 2.0, indexing="ij")
    np.testing.assert_allclose(out, 2.0 * yc + 0.5 * xc, rtol=1e-6)
    assert out.shape == (4, 6)


def test_downsample_uint8_rounding_by_hand():
    # 2 x 2 blocks with sums 2 (mean 0.5 -> 0), 6 (1.5 -> 2), 10 (2.5 -> 2), 3 (0.75 -> 1)
    img = np.array([[0, 1, 1, 2, 2, 3, 0, 1],
                    [0, 1, 1, 2, 2, 3, 1, 1]], np.uint8)
    np.testing.assert_array_equal(remod.downsample(img, 2), [[0, 2, 2, 1]])
    # odd sizes drop the partial edge blocks
    assert remod.downsample(np.zeros((7, 11), np.uint8), 3).shape == (2, 3)


def test_downsample_preserves_mass():
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 100, (40, 60)).astype(np.float32)
    out = remod.downsample(img, 4)
    assert abs(float(out.sum()) * 16 - float(img.sum())) < 1e-3 * float(img.sum())


def test_zmodel_linear_in_z_and_constants():
    Z, k = 9, 2
    base = np.arange(12 * 10, dtype=np.int64).reshape(12, 10) % 50
    stack = np.stack([base + 10 * z for z in range(Z)]).astype(np.uint8)
    out = remod.zmodel(stack, k)
    for z in range(k, Z - k):  # symmetric neighbourhoods: the mean of z +- 1..k is z
        np.testing.assert_array_equal(out[z], stack[z].astype(np.float32))
    # at the first section the neighbours are 1..k
    np.testing.assert_allclose(out[0], base + 10 * np.mean(np.arange(1, k + 1)), rtol=1e-6)


def test_zmodel_excludes_damaged_sections_and_handles_isolation():
    stack = np.stack([np.full((4, 5), v, np.uint8) for v in (10, 20, 30, 40, 50)])
    valid = np.array([1, 1, 0, 1, 1], bool)
    out = remod.zmodel(stack, 1, valid)
    np.testing.assert_allclose(out[:, 0, 0], [20, 10, 30, 50, 40])  # z=2 takes (20 + 40) / 2
    st2 = np.stack([np.full((4, 5), v, np.uint8) for v in (10, 20, 35, 40, 70)])
    iso = remod.zmodel(st2, 1, np.array([1, 0, 1, 0, 1], bool))
    # sections 0, 2, 4 have no valid neighbour (their own value); 1 and 3 average their neighbours
    np.testing.assert_allclose(iso[:, 0, 0], [10, 22.5, 35, 52.5, 70])
    out0 = remod.zmodel(stack, 0)  # k = 0: no neighbours, the section itself
    np.testing.assert_array_equal(out0, stack.astype(np.float32))


def test_zmodel_uint8_rounds_the_exact_mean_half_to_even():
    # neighbour sums over 2 sections: (1 + 2) / 2 = 1.5 -> 2, (2 + 3) / 2 = 2.5 -> 2, (4 + 5) / 2 = 4.5 -> 4
    stack = np.stack([np.array([[1, 2, 4]], np.uint8), np.zeros((1, 3), np.uint8), np.array([[2, 3, 5]], np.uint8)])
    out = remod.zmodel(stack, 1, dtype=np.uint8)
    np.testing.assert_array_equal(out[1], [[2, 2, 4]])
    np.testing.assert_array_equal(out[0], stack[1])  # single neighbour: exact
    assert out.dtype == np.uint8
