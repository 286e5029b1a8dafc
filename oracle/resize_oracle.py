"""Oracle of the S0 resize that brings uneven inputs to a common scale.

TEST INFRASTRUCTURE ONLY: the tests are the only users.

The paper's encoder scales images so that their larger side is 640 px before
detection (its experiments use VGA-sized images); the method of resampling is
not stated.  The reading here is area averaging: output pixel (x', y') of a
W' x H' image is the mean of the W x H input over the rectangle
[x' W / W', (x' + 1) W / W') x [y' H / H', (y' + 1) H / H'], the input being
constant on each pixel, rounded to the nearest integer with ties to even.

Scaled by W' (and H'), input column x covers [x W', (x + 1) W') and output
column x' covers [x' W, (x' + 1) W), so every overlap is an integer and the
mean is an exact ratio of integers:

    out = round( sum_x sum_y in[y][x] * ox(x', x) * oy(y', y) / (W H) ).

Sizes: an image whose larger side exceeds max_side is scaled so that that
side becomes max_side and the other side round(side * max_side / larger)
(ties to even, at least 1); max_side = 0 or a smaller image leaves it as is.
"""
from __future__ import annotations

import numpy as np


def round_half_even_div(num: int, den: int) -> int:
    q, r = divmod(num, den)
    if 2 * r > den or (2 * r == den and q % 2 == 1):
        q += 1
    return q


def target_size(width: int, height: int, max_side: int):
    """(W', H') of the resized image."""
    if max_side <= 0 or max(width, height) <= max_side:
        return width, height
    if width >= height:
        return max_side, max(1, round_half_even_div(height * max_side, width))
    return max(1, round_half_even_div(width * max_side, height)), max_side


def overlap(o: int, i: int, n_in: int, n_out: int) -> int:
    """Length of [i n_out, (i + 1) n_out) intersected with [o n_in, (o + 1) n_in)."""
    return max(0, min((o + 1) * n_in, (i + 1) * n_out) - max(o * n_in, i * n_out))


def resize(img: np.ndarray, max_side: int) -> np.ndarray:
    H, W = img.shape
    W2, H2 = target_size(W, H, max_side)
    if (W2, H2) == (W, H):
        return img.copy()
    v = img.astype(np.int64)
    out = np.zeros((H2, W2), np.uint8)
    for y2 in range(H2):
        # input rows that overlap output row y2: [y2 H / H2, (y2 + 1) H / H2)
        ys = range((y2 * H) // H2, min(-(-((y2 + 1) * H) // H2), H))
        for x2 in range(W2):
            xs = range((x2 * W) // W2, min(-(-((x2 + 1) * W) // W2), W))
            s = 0
            for y in ys:
                wy = overlap(y2, y, H, H2)
                for x in xs:
                    s += int(v[y, x]) * overlap(x2, x, W, W2) * wy
            out[y2, x2] = round_half_even_div(s, W * H)
    return out
