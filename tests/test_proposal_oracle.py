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


def test_forward_by_hand_on_constant_images():
    """The whole forward pass worked by hand.  Channel 0 only: centre taps of
    1 in all three layers (the centre tap reads the input at (s y, s x)), one
    extra corner tap of 2^-9 in conv2, head weight 1, head bias 0.25.  On a
    constant 64 x 64 image the block (1, 1) is interior at every layer, so
    x = (u - 128) / 64, A1 = relu(x), z2 = A1 (1 + 2^-9), A3 = relu(A2) and the
    logit is A3 + 0.25.  In BF16 mode A2 is rounded: 1 + 2^-9 lies below half
    a BF16 ulp above 1 (2^-8), so it rounds to 1."""
    p = {name: np.zeros(shp) for name, shp in PO.SHAPES}
    p["W1"][0, 0, 1, 1] = 1.0
    p["W2"][0, 0, 1, 1] = 1.0
    p["W2"][0, 0, 0, 0] = 2.0 ** -9
    p["W3"][0, 0, 1, 1] = 1.0
    p["Wh"][0] = 1.0
    p["bh"][0] = 0.25
    theta = PO.pack(p)
    cases = [(192, 1.25, 1.25 + 2.0 ** -9),          # x = 1
             (160, 0.75, 0.75 + 2.0 ** -10),         # x = 0.5
             (100, 0.25, 0.25)]                      # x < 0: every activation is 0
    for u, want_bf16, want_fp64 in cases:
        img = np.full((64, 64), u, np.uint8)
        z16, _ = PO.forward(img, theta, bf16=True)
        z64, _ = PO.forward(img, theta, bf16=False)
        assert z16.shape == (4, 4)
        assert z16[1, 1] == want_bf16, (u, z16[1, 1])
        assert z64[1, 1] == want_fp64, (u, z64[1, 1])


def test_forward_rounds_the_weights_and_a1_to_bf16():
    """Channel 0 only: W1 centre 1 and corner 2^-9, W2 centre 1, W3 centre
    1 + 2^-9, head weight 1.  On a constant image of 192 (x = 1) an interior
    z1 is 1 + 2^-9, which BF16 rounds to 1 (below half an ulp above 1), and
    so is W3's centre; A3 is not rounded.  So the logit of the interior block
    is 1 in BF16 mode and (1 + 2^-9)^2 in FP64, and A1 is 1 in BF16 mode."""
    p = {name: np.zeros(shp) for name, shp in PO.SHAPES}
    p["W1"][0, 0, 1, 1] = 1.0
    p["W1"][0, 0, 0, 0] = 2.0 ** -9
    p["W2"][0, 0, 1, 1] = 1.0
    p["W3"][0, 0, 1, 1] = 1.0 + 2.0 ** -9
    p["Wh"][0] = 1.0
    theta = PO.pack(p)
    img = np.full((64, 64), 192, np.uint8)
    z16, c16 = PO.forward(img, theta, bf16=True)
    z64, c64 = PO.forward(img, theta, bf16=False)
    assert c16["a1"][0, 10, 10] == 1.0
    assert c64["a1"][0, 10, 10] == 1.0 + 2.0 ** -9
    assert z16[1, 1] == 1.0
    assert z64[1, 1] == (1.0 + 2.0 ** -9) ** 2


def test_flat_parameter_layout():
    """The flat parameter vector the GPU also reads: W1 (144), b1 (16), W2
    (2304), b2 (16), W3 (2304), b3 (16), Wh (16), bh (1) in that order, 4817
    values, each weight tensor row-major over [co][ci][ky][kx]."""
    assert PO.N_PARAMS == 4817
    p = PO.unpack(np.arange(4817, dtype=np.float64))
    starts = {"W1": 0, "b1": 144, "W2": 160, "b2": 2464, "W3": 2480, "b3": 4784, "Wh": 4800, "bh": 4816}
    for name, first in starts.items():
        assert p[name].ravel()[0] == first, name
    assert p["W2"][1, 2, 0, 1] == 160 + ((1 * 16 + 2) * 3 + 0) * 3 + 1
    assert p["W1"][3, 0, 2, 1] == (3 * 3 + 2) * 3 + 1
    np.testing.assert_array_equal(PO.pack(p), np.arange(4817))
