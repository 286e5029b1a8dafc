"""Match checks on the paired warped copies of the 640x480 workload images
(synth.warp_params / warp_image: rotation 0-45 deg, scale 0.7-1.4 about the
centre, bilinear, fill 128).

The features of an image and of its warped copy are matched by nearest
descriptor with the ratio test (0.8); a match is an inlier when the warp's
affine map sends the first point within 3 px of the second.  Orientation
normalisation (Alg. 2 stage A) and the scale space make the descriptors of
the same structure agree under rotation and scale, so most ratio-test
matches are inliers; a descriptor frame rotated the wrong way, or a wrong
scale, leaves few.  The oracle is checked on the CPU; the CUDA path on the GPU
must find as many inliers as the oracle, within a few percent.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1705_09776_gb300 import synth

SEEDS = [synth.image_seed(1, i) for i in (0, 2, 3, 5)]


def _pair(seed):
    img = synth.blob_image(seed)
    ang, sc = synth.warp_params(seed)
    warped, A = synth.warp_image(img, ang, sc)
    return img, warped, A


def _inliers(k1, d1, k2, d2, A):
    D = ((d1[:, None, :].astype(np.float64) - d2[None, :, :]) ** 2).sum(-1)
    o = np.argsort(D, axis=1)[:, :2]
    r = np.arange(len(d1))
    good = D[r, o[:, 0]] < 0.8 ** 2 * D[r, o[:, 1]]
    pred = np.stack([k1["x"], k1["y"], np.ones(len(k1))], 1) @ A.T
    err = np.hypot(pred[:, 0] - k2["x"][o[:, 0]], pred[:, 1] - k2["y"][o[:, 0]])
    return int(good.sum()), int((good & (err < 3.0)).sum())


@pytest.mark.parametrize("seed", SEEDS)
def test_oracle_matches_its_warped_copy(seed):
    img, warped, A = _pair(seed)
    k1, d1, _ = O.extract(img, O.params())
    k2, d2, _ = O.extract(warped, O.params())
    good, inl = _inliers(k1, d1, k2, d2, A)
    assert inl >= 80 and inl >= 0.75 * good, (good, inl)


@pytest.mark.gpu
def test_gpu_matches_its_warped_copy_like_the_oracle():
    from paper_1705_09776_gb300 import cdvs
    ctx = cdvs.Context(0)
    for seed in SEEDS:
        img, warped, A = _pair(seed)
        gk, gd, gc, _ = ctx.extract([img, warped])
        n0 = int(gc[0])
        g_good, g_inl = _inliers(gk[:n0], gd[:n0], gk[n0:], gd[n0:], A)
        k1, d1, _ = O.extract(img, O.params())
        k2, d2, _ = O.extract(warped, O.params())
        o_good, o_inl = _inliers(k1, d1, k2, d2, A)
        assert g_inl >= 0.75 * g_good, (seed, g_good, g_inl)
        assert abs(g_inl - o_inl) <= max(5, 0.05 * o_inl), (seed, g_inl, o_inl)
