"""Uneven batches (S0 resize to a common scale, then the whole path).

* cdvs_resize is bit-exact against the S0 oracle (exact integer area means),
  on random small sizes and on a full-size 1280 x 720 -> 640 x 360 image;
* extraction of an uneven batch with max_side = 640 equals, record for
  record and bit for bit, extraction of the oracle-resized images with no
  resize -- the resize is the only thing max_side adds;
* one uneven image end to end against the FP64 oracle on its resized form,
  with the parity bracketing of the other end-to-end tests.
"""
import numpy as np
import pytest

import parity as PT
from oracle import oracle as O
from oracle import resize_oracle as R
from paper_1705_09776_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1705_09776_gb300 import cdvs
    return cdvs, cdvs.Context(0)


def _uneven(n, seed, scale=1.0):
    out = []
    for i, (w, h) in enumerate(synth.uneven_sizes(n, base_seed=seed)):
        w, h = max(16, int(w * scale)), max(16, int(h * scale))
        out.append(synth.blob_image(synth.image_seed(seed, i), width=w, height=h,
                                    n_blobs=max(8, int(200 * w * h / (640 * 480)))))
    return out


def test_resize_bit_exact_small(env):
    cdvs, ctx = env
    rng = np.random.default_rng(1)
    imgs = [rng.integers(0, 256, (int(rng.integers(20, 200)), int(rng.integers(20, 200)))).astype(np.uint8)
            for _ in range(12)]
    for max_side in (17, 64, 150, 0):
        got = ctx.resize(imgs, max_side)
        for im, g in zip(imgs, got):
            np.testing.assert_array_equal(g, R.resize(im, max_side))


def test_resize_bit_exact_full_size(env):
    cdvs, ctx = env
    img = synth.blob_image(synth.image_seed(77, 0), width=1280, height=720, n_blobs=600)
    g = ctx.resize([img], 640)[0]
    assert g.shape == (360, 640)
    np.testing.assert_array_equal(g, R.resize(img, 640))


def test_uneven_batch_equals_extraction_of_resized_images(env):
    cdvs, ctx = env
    imgs = _uneven(6, seed=3)
    k1, d1, c1, _ = ctx.extract(imgs, cdvs.params(max_side=640))
    small = [R.resize(im, 640) for im in imgs]
    assert any(s.shape != im.shape for s, im in zip(small, imgs))
    k0, d0, c0, _ = ctx.extract(small)
    assert np.array_equal(c0, c1)
    assert np.array_equal(k0.view(np.uint8), k1.view(np.uint8))
    assert np.array_equal(d0, d1)


def test_uneven_image_end_to_end_vs_oracle(env):
    cdvs, ctx = env
    img = _uneven(1, seed=9, scale=0.5)[0]           # a smaller uneven image, resized to max side 256
    small = R.resize(img, 256)
    gk, gd, cnt, st = ctx.extract([img], cdvs.params(max_side=256))
    assert st == cdvs.CDVS_OK
    ek, ed, _ = O.extract(small, O.params())
    lk, _, _ = O.extract(small, O.params(margin=PT.MARGIN))
    sk, _, _ = O.extract(small, O.params(margin=-PT.MARGIN))

    def points(r, key):
        return r[np.unique(r[key], return_index=True)[1]]

    gp, ep = points(gk, "parent_id"), points(ek, "parent")
    agree, n_dis, n_exc, n = PT.point_agreement(gp, ep, points(lk, "parent"), points(sk, "parent"))
    assert agree >= PT.AGREE, (agree, n_dis, n_exc, n)


def test_graph_mode_matches_direct_launches(env):
    """cdvs_set_graph: device-resident calls captured into one CUDA graph --
    a first capture, an in-place update on the same shapes, a new shape
    (re-instantiated), and a resized uneven batch -- give exactly the
    records of direct launches."""
    import torch
    cdvs, ctx = env
    batches = [[synth.blob_image(synth.image_seed(61, i)) for i in range(4)],
               [synth.blob_image(synth.image_seed(62, i)) for i in range(4)],
               [synth.blob_image(synth.image_seed(63, i), width=320, height=200, n_blobs=60) for i in range(3)],
               _uneven(3, seed=64)]

    def run(imgs, p):
        n = len(imgs)
        flat = np.concatenate([im.ravel() for im in imgs])
        dev = torch.from_numpy(flat).cuda()
        offs = np.cumsum([0] + [im.size for im in imgs])
        sizes = np.array([(im.shape[1], im.shape[0], im.shape[1]) for im in imgs], cdvs.IMAGE_DESC_DTYPE)
        cap = n * 300 * 4
        kp = torch.zeros(cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        desc = torch.zeros(cap, 128, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        ctx.extract_raw(n, [dev.data_ptr() + int(o) for o in offs[:-1]], sizes, p, kp, desc, cap, cnt,
                        cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE, torch.cuda.current_stream())
        torch.cuda.synchronize()
        c = cnt.cpu().numpy()
        t = int(c.sum())
        return c, kp.cpu().numpy()[:t * cdvs.KEYPOINT_DTYPE.itemsize].copy(), desc.cpu().numpy()[:t].copy()

    p = cdvs.params(max_side=640)
    ref = [run(b, p) for b in batches]
    ctx.set_graph(True)
    try:
        for rep in range(2):
            for b, r in zip(batches, ref):
                got = run(b, p)
                assert np.array_equal(got[0], r[0])
                assert np.array_equal(got[1], r[1])
                assert np.array_equal(got[2], r[2])
    finally:
        ctx.set_graph(False)


def _highres(w, h, seed, i=0):
    k = w * h / (640 * 480)
    return synth.blob_image(synth.image_seed(seed, i), w, h, n_blobs=int(round(200 * k)), sigma_range=(4.8, 64.0))


def test_highres_six_octaves_2000_points_vs_oracle(env):
    """The high-resolution configuration (6 octaves, N = 2000, blobs x3.2) on a
    1024 x 768 image against the oracle, with the parity bracketing."""
    cdvs, ctx = env
    img = _highres(1024, 768, seed=5)
    p = cdvs.params(num_octaves=6, max_keypoints=2000)
    gk, gd, cnt, st = ctx.extract([img], p)
    assert st == cdvs.CDVS_OK and 300 < cnt[0]
    op = dict(num_octaves=6, max_keypoints=2000)
    ek, ed, _ = O.extract(img, O.params(**op), cap=16384)
    lk, _, _ = O.extract(img, O.params(margin=PT.MARGIN, **op), cap=16384)
    sk, _, _ = O.extract(img, O.params(margin=-PT.MARGIN, **op), cap=16384)

    def points(r, key):
        return r[np.unique(r[key], return_index=True)[1]]

    gp, ep = points(gk, "parent_id"), points(ek, "parent")
    assert (gp["octave"] >= 4).any()                  # the added octaves contribute
    agree, n_dis, n_exc, n = PT.point_agreement(gp, ep, points(lk, "parent"), points(sk, "parent"))
    assert agree >= PT.AGREE, (agree, n_dis, n_exc, n)


def test_highres_full_size_runs_and_is_deterministic(env):
    cdvs, ctx = env
    imgs = [_highres(2048, 1536, seed=5, i=i) for i in range(2)]
    p = cdvs.params(num_octaves=6, max_keypoints=2000)
    a = ctx.extract(imgs, p)
    b = ctx.extract(imgs, p)
    assert (a[2] <= 2000 * p["max_orientations"][0]).all() and (a[2] > 1000).all()
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8)) and np.array_equal(a[1], b[1])
    assert len(np.unique(a[0][a[0]["image"] == 0]["parent_id"])) <= 2000
