"""FP64 oracle of the learned block-proposal network (numpy).

TEST INFRASTRUCTURE ONLY: the tests are the only users; the product path
never imports this module.

The paper detects interest points with ALP over the whole image (Sec. IV-A,
Alg. 1).  Its learned extension here is a small CNN that looks at an 8-bit
image and gives one logit per 16x16 block, trained on labels the plain
detector produces, so that detection can skip blocks where no interest point
is likely.  The network (a reading of the extension, not of the paper):

    x  = (u8 - 128) / 64                                  1 x H  x W
    Z1 = conv3x3(x,  W1, stride 2, pad 1) + b1,  A1 = relu(Z1)   16 x H1 x W1
    Z2 = conv3x3(A1, W2, stride 2, pad 1) + b2,  A2 = relu(Z2)   16 x H2 x W2
    Z3 = conv3x3(A2, W3, stride 1, pad 1) + b3,  A3 = relu(Z3)   16 x H2 x W2
    P  = mean of A3 over each 4x4 cell (cells clipped to H2 x W2)   16 x Th x Tw
    z  = Wh . P + bh                                      one logit per block
    loss = mean over blocks of  softplus(z) - y z        (BCE with logits)

with H1 = ceil(H/2), H2 = ceil(H1/2), Th = ceil(H/16) (and the same for
widths).  "conv3x3" is cross-correlation, W[co][ci][ky][kx] applied at
input (s*y + ky - 1, s*x + kx - 1), zero outside the input.

BF16 mode rounds (to nearest, ties to even) what the GPU stores in BF16: the
weights W1, W2, W3, Wh, the input x (exact) and the activations A1 and A2.
Biases, A3, P and every accumulation stay in the oracle's FP64.  The backward
pass differentiates that forward treating each rounding as the identity.

The flat parameter vector (FP32 on the GPU) is W1 (144), b1 (16), W2 (2304),
b2 (16), W3 (2304), b3 (16), Wh (16), bh (1): 4817 values.
"""
from __future__ import annotations

import numpy as np

C = 16  # channels of every hidden layer
SHAPES = [("W1", (C, 1, 3, 3)), ("b1", (C,)), ("W2", (C, C, 3, 3)), ("b2", (C,)),
          ("W3", (C, C, 3, 3)), ("b3", (C,)), ("Wh", (C,)), ("bh", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Flat vector -> dict of arrays (FP64 copies)."""
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp).copy()
        o += n
    assert o == theta.size == N_PARAMS
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64.
    The value is first rounded to FP32 (what the GPU holds), then its 16 low
    bits are rounded away."""
    f = np.asarray(a, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def out_size(n, stride):
    """Output length of a 3-tap convolution with padding 1."""
    return (n - 1) // stride + 1


def conv3x3(a, w, b, stride):
    """a: (ci, H, W); w: (co, ci, 3, 3); b: (co,).  Plain definition: a sum
    over the 9 taps and the input channels of shifted, strided inputs."""
    ci, H, W = a.shape
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    pad = np.zeros((ci, H + 2, W + 2))
    pad[:, 1:H + 1, 1:W + 1] = a
    out = np.zeros((w.shape[0], Ho, Wo))
    for ky in range(3):
        for kx in range(3):
            # input (s*y + ky - 1) sits at padded row s*y + ky
            win = pad[:, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("oc,chw->ohw", w[:, :, ky, kx], win)
    return out + b[:, None, None]


def conv3x3_backward(a, w, dz, stride):
    """Gradients of conv3x3(a, w, b, stride) given dL/dout = dz: (da, dw, db)."""
    ci, H, W = a.shape
    co, Ho, Wo = dz.shape
    pad = np.zeros((ci, H + 2, W + 2))
    pad[:, 1:H + 1, 1:W + 1] = a
    dpad = np.zeros_like(pad)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(ky, ky + stride * (Ho - 1) + 1, stride),
                  slice(kx, kx + stride * (Wo - 1) + 1, stride))
            dw[:, :, ky, kx] = np.einsum("ohw,chw->oc", dz, pad[sl])
            dpad[sl] += np.einsum("oc,ohw->chw", w[:, :, ky, kx], dz)
    return dpad[:, 1:H + 1, 1:W + 1], dw, dz.sum(axis=(1, 2))


def pool_cells(a3, th, tw):
    """Mean of a3 (c, H2, W2) over 4x4 cells clipped to the array."""
    c, H2, W2 = a3.shape
    out = np.zeros((c, th, tw))
    for ty in range(th):
        for tx in range(tw):
            cell = a3[:, 4 * ty:min(4 * ty + 4, H2), 4 * tx:min(4 * tx + 4, W2)]
            out[:, ty, tx] = cell.mean(axis=(1, 2)) if cell.size else 0.0
    return out


def forward(img, theta, bf16=True):
    """One image (H, W) uint8 -> (logits (Th, Tw), cache for backward)."""
    p = unpack(theta)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    H, W = img.shape
    th, tw = -(-H // 16), -(-W // 16)
    x = rnd((np.asarray(img, np.float64) - 128.0) / 64.0)[None]
    w1, w2, w3, wh = rnd(p["W1"]), rnd(p["W2"]), rnd(p["W3"]), rnd(p["Wh"])
    z1 = conv3x3(x, w1, p["b1"], 2)
    a1 = rnd(np.maximum(z1, 0.0))
    z2 = conv3x3(a1, w2, p["b2"], 2)
    a2 = rnd(np.maximum(z2, 0.0))
    z3 = conv3x3(a2, w3, p["b3"], 1)
    a3 = np.maximum(z3, 0.0)
    P = pool_cells(a3, th, tw)
    z = np.einsum("c,chw->hw", wh, P) + p["bh"][0]
    cache = dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, P=P, w1=w1, w2=w2, w3=w3, wh=wh, th=th, tw=tw)
    return z, cache


def bce_with_logits(z, y):
    """Elementwise softplus(z) - y z, in the overflow-free form."""
    return np.maximum(z, 0.0) - y * z + np.log1p(np.exp(-np.abs(z)))


def loss_and_grad(imgs, labels, theta, bf16=True):
    """Mean BCE over every block of every image, and its gradient with
    respect to the flat parameters."""
    n_blocks = sum(l.size for l in labels)
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    loss = 0.0
    for img, y in zip(imgs, labels):
        z, c = forward(img, theta, bf16)
        y = np.asarray(y, np.float64)
        loss += bce_with_logits(z, y).sum()
        dz = (1.0 / (1.0 + np.exp(-z)) - y) / n_blocks
        g["Wh"] += np.einsum("hw,chw->c", dz, c["P"])
        g["bh"] += dz.sum()
        dP = c["wh"][:, None, None] * dz[None]
        # each cell's mean spreads its gradient evenly over its positions
        da3 = np.zeros_like(c["a3"])
        H2, W2 = da3.shape[1:]
        for ty in range(c["th"]):
            for tx in range(c["tw"]):
                ys, xs = slice(4 * ty, min(4 * ty + 4, H2)), slice(4 * tx, min(4 * tx + 4, W2))
                n = (ys.stop - ys.start) * (xs.stop - xs.start)
                if n > 0:
                    da3[:, ys, xs] = dP[:, ty, tx][:, None, None] / n
        dz3 = da3 * (c["z3"] > 0)
        da2, dw3, db3 = conv3x3_backward(c["a2"], c["w3"], dz3, 1)
        dz2 = da2 * (c["z2"] > 0)
        da1, dw2, db2 = conv3x3_backward(c["a1"], c["w2"], dz2, 2)
        dz1 = da1 * (c["z1"] > 0)
        _, dw1, db1 = conv3x3_backward(c["x"], c["w1"], dz1, 2)
        for k, v in (("W1", dw1), ("b1", db1), ("W2", dw2), ("b2", db2), ("W3", dw3), ("b3", db3)):
            g[k] += v
    return loss / n_blocks, pack(g)


def block_labels(points_xy, height, width):
    """1 for every 16x16 block holding at least one of the points (x, y in
    image pixels, pixel centres at integers), else 0."""
    th, tw = -(-height // 16), -(-width // 16)
    y = np.zeros((th, tw))
    for x, yy in points_xy:
        bx = min(max(int(np.floor(x + 0.5)) // 16, 0), tw - 1)
        by = min(max(int(np.floor(yy + 0.5)) // 16, 0), th - 1)
        y[by, bx] = 1.0
    return y
