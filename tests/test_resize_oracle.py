"""Pins of the S0 resize oracle (CPU): target sizes by hand, the overlap
formula against brute force on a finely replicated grid, exact 2x reduction
as 2x2 means, and constants."""
import numpy as np
import pytest

from oracle import resize_oracle as R


def test_target_sizes():
    assert R.target_size(1280, 720, 640) == (640, 360)
    assert R.target_size(700, 1280, 640) == (350, 640)
    assert R.target_size(600, 400, 640) == (600, 400)
    assert R.target_size(1280, 333, 640) == (640, 166)      # 166.5, tie to even
    assert R.target_size(1280, 335, 640) == (640, 168)      # 167.5, tie to even
    assert R.target_size(800, 800, 0) == (800, 800)


@pytest.mark.parametrize("shape,max_side", [((9, 13), 7), ((11, 6), 5), ((17, 17), 10), ((8, 15), 12)])
def test_matches_brute_force_on_replicated_grid(shape, max_side):
    rng = np.random.default_rng(sum(shape) + max_side)
    img = rng.integers(0, 256, shape).astype(np.uint8)
    H, W = shape
    W2, H2 = R.target_size(W, H, max_side)
    # each input pixel becomes an H2 x W2 block; each output pixel is then an H x W block
    fine = np.repeat(np.repeat(img.astype(np.int64), H2, axis=0), W2, axis=1)
    sums = fine.reshape(H2, H, W2, W).sum(axis=(1, 3))
    want = np.array([[R.round_half_even_div(int(s), W * H) for s in row] for row in sums], np.uint8)
    np.testing.assert_array_equal(R.resize(img, max_side), want)


def test_exact_halving_is_2x2_means():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (10, 16)).astype(np.uint8)
    got = R.resize(img, 8)
    s = img.astype(np.int64).reshape(5, 2, 8, 2).sum(axis=(1, 3))
    want = np.vectorize(lambda v: R.round_half_even_div(int(v), 4))(s)
    np.testing.assert_array_equal(got, want)


def test_constant_and_identity():
    img = np.full((30, 45), 77, np.uint8)
    np.testing.assert_array_equal(R.resize(img, 20), np.full((13, 20), 77, np.uint8))
    img = np.random.default_rng(4).integers(0, 256, (30, 45)).astype(np.uint8)
    np.testing.assert_array_equal(R.resize(img, 45), img)
