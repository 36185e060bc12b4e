"""Pins for the oracle's scaled local thickness (LT at 1/s resolution,
brought back to full resolution; the reduced-resolution option of the fast
local-thickness work the paper builds on, Sec. 1 and Sec. 4).

Independent references: scale 1 is the exact LT; an object made of s^d blocks
is sampled without loss, so its scaled LT is exactly s^2 times the LT of the
block-level object; a 3x3 square worked by hand exercises the
neighbouring-block rule.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.usefixtures("built_cpu_parts")


def _random_labelled(rng, shape, p=0.75):
    mask = (rng.random(shape) < p).astype(np.uint8)
    half = (np.indices(shape)[-1] >= shape[-1] // 2).astype(np.uint32)
    return mask, mask.astype(np.uint32) * (1 + half)


@pytest.mark.parametrize("shape", [(13, 17), (7, 9, 11)])
def test_scale_one_is_exact(shape):
    rng = np.random.default_rng(len(shape))
    mask, labels = _random_labelled(rng, shape)
    exact = oracle.lt2(oracle.dt2(mask), labels)
    assert np.array_equal(oracle.lt2_scaled(mask, labels, 1), exact)


@pytest.mark.parametrize("s,shape", [(2, (6, 7)), (3, (5, 4)), (2, (4, 5, 3)), (4, (3, 3, 2))])
def test_block_objects_scale_exactly(s, shape):
    rng = np.random.default_rng(s * 10 + len(shape))
    mask_l, labels_l = _random_labelled(rng, shape)
    block = np.ones((s,) * len(shape), np.uint8)
    mask = np.kron(mask_l, block).astype(np.uint8)
    labels = np.kron(labels_l, block.astype(np.uint32)).astype(np.uint32)
    low = oracle.lt2(oracle.dt2(mask_l), labels_l).astype(np.int64)
    want = (s * s * np.kron(low, block.astype(np.int64))).astype(np.uint32)
    assert np.array_equal(oracle.lt2_scaled(mask, labels, s), want)


def test_hand_worked_square():
    """3x3 square in a 4x4 image, s = 2. Blocks (0,0) samples (1,1): inside;
    the other three blocks sample background. The low-res object is one
    voxel with LT2 = 1, so its block gets 4; the five voxels in blocks of
    another label take the neighbouring block's 4. The exact LT2 of the 3x3
    square is 4 everywhere too (the centre's ball, DT2 = 4, holds it)."""
    m = np.zeros((4, 4), np.uint8)
    m[:3, :3] = 1
    out = oracle.lt2_scaled(m, m.astype(np.uint32), 2)
    want = np.zeros((4, 4), np.uint32)
    want[:3, :3] = 4
    assert np.array_equal(out, want)
    assert np.array_equal(oracle.lt2(oracle.dt2(m), m.astype(np.uint32)), want)
