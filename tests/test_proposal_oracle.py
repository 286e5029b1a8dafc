"""Pins of the proposal-network oracle (CPU only): the convolution against
scipy's 2-D correlation, the analytic gradient against central finite
differences of the loss, pooling and the loss against closed forms, and the
BF16 rounding against hand-worked values."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import proposal_oracle as PO


def _theta(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in PO.SHAPES:
        fan_in = int(np.prod(shp[1:])) if len(shp) > 1 else 16
        p[name] = rng.normal(0.0, scale / np.sqrt(fan_in), shp)
        if name.startswith("b"):
            p[name] = rng.normal(0.05, 0.05, shp)
    return PO.pack(p)


@pytest.mark.parametrize("stride", [1, 2])
@pytest.mark.parametrize("shape", [(9, 14), (10, 7), (16, 16)])
def test_conv_matches_scipy_correlation(stride, shape):
    rng = np.random.default_rng(1)
    a = rng.normal(size=(3,) + shape)
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = PO.conv3x3(a, w, b, stride)
    for co in range(4):
        full = sum(correlate2d(a[ci], w[co, ci], mode="same", boundary="fill") for ci in range(3)) + b[co]
        np.testing.assert_allclose(got[co], full[::stride, ::stride], rtol=1e-12, atol=1e-12)
    assert got.shape[1:] == (PO.out_size(shape[0], stride), PO.out_size(shape[1], stride))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    imgs = [rng.integers(0, 256, (37, 53)).astype(np.uint8), rng.integers(0, 256, (32, 48)).astype(np.uint8)]
    labels = [rng.integers(0, 2, (-(-im.shape[0] // 16), -(-im.shape[1] // 16))).astype(float) for im in imgs]
    theta = _theta(3)
    _, g = PO.loss_and_grad(imgs, labels, theta, bf16=False)
    # every head parameter and bias, and a sample of each weight tensor
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in PO.SHAPES])
    idx = []
    for k, (name, _) in enumerate(PO.SHAPES):
        span = np.arange(offs[k], offs[k + 1])
        idx += list(span) if span.size <= 16 else list(rng.choice(span, 12, replace=False))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (PO.loss_and_grad(imgs, labels, tp, bf16=False)[0] - PO.loss_and_grad(imgs, labels, tm, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_pooling_and_loss_closed_forms():
    a = np.full((16, 10, 13), 2.5)
    P = PO.pool_cells(a, 3, 4)
    np.testing.assert_allclose(P, 2.5)
    a = np.arange(16 * 5 * 5, dtype=float).reshape(16, 5, 5)
    P = PO.pool_cells(a, 2, 2)
    np.testing.assert_allclose(P[:, 1, 1], a[:, 4, 4])                 # ragged corner cell: one position
    np.testing.assert_allclose(P[:, 0, 0], a[:, :4, :4].mean(axis=(1, 2)))
    assert PO.bce_with_logits(0.0, 1.0) == pytest.approx(np.log(2.0))
    assert PO.bce_with_logits(40.0, 1.0) == pytest.approx(np.exp(-40.0), rel=1e-6)
    assert PO.bce_with_logits(-40.0, 1.0) == pytest.approx(40.0, rel=1e-12)


def test_bf16_rounding_hand_values():
    u = 2.0 ** -7   # BF16 spacing at 1
    vals = np.array([1.0, 1 + u / 2, 1 + 1.5 * u, 1 + u / 2 + 2.0 ** -20, -3.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -3.0, 0.0])
    np.testing.assert_array_equal(PO.bf16_round(vals), want)
    # inputs (u8 - 128) / 64 are exact in BF16
    x = (np.arange(256) - 128.0) / 64.0
    np.testing.assert_array_equal(PO.bf16_round(x), x)


def test_sizes_and_descent_step():
    img = np.random.default_rng(4).integers(0, 256, (100, 70)).astype(np.uint8)
    z, c = PO.forward(img, _theta(5))
    assert z.shape == (7, 5) and c["a1"].shape == (16, 50, 35) and c["a3"].shape == (16, 25, 18)
    y = (np.random.default_rng(6).random(z.shape) < 0.3).astype(float)
    l0, g = PO.loss_and_grad([img], [y], _theta(5), bf16=False)
    l1, _ = PO.loss_and_grad([img], [y], _theta(5) - 0.05 * g / np.linalg.norm(g), bf16=False)
    assert l1 < l0


def test_block_labels():
    y = PO.block_labels([(0.0, 0.0), (15.4, 2.0), (15.6, 2.0), (639.0, 479.0)], 480, 640)
    assert y.shape == (30, 40) and y.sum() == 3
    assert y[0, 0] == 1 and y[0, 1] == 1 and y[29, 39] == 1
