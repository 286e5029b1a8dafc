"""Coefficients of the arctangent used by the descriptor kernel.

atan(t) on [0, 1] is approximated by an odd polynomial t * P(t^2) of degree 15
(8 coefficients).  The coefficients come from Lawson's algorithm: weighted
least squares on a dense grid, with the weights multiplied by the absolute
error after every solve, which converges to the minimax (equal-ripple) fit.
Run as a script to print the coefficients (as FP32) and the maximum error of
the FP32 Horner evaluation; describe.cu holds the printed values.
"""
import numpy as np

N_COEF = 8


def fit(n_coef=N_COEF, iters=200):
    t = np.sort(np.concatenate([0.5 + 0.5 * np.cos(np.linspace(0.0, np.pi, 4000)), np.linspace(0.0, 1.0, 4000)]))
    z = t * t
    V = np.stack([t * z ** k for k in range(n_coef)], 1)
    y = np.arctan(t)
    w = np.ones_like(t)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], y * sw, rcond=None)
        w = w * np.abs(V @ c - y)
        w /= w.sum()
    return c.astype(np.float32)


def eval_f32(c, t):
    """Horner in FP32 with one rounding per step, like the kernel's FMAs."""
    t = np.asarray(t, np.float64)
    z = (t * t).astype(np.float32).astype(np.float64)
    p = np.float64(c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p * z + np.float64(c[k])).astype(np.float32).astype(np.float64)
    return (p * t).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    tt = np.linspace(0.0, 1.0, 1_000_001)
    err = np.max(np.abs(eval_f32(c, tt).astype(np.float64) - np.arctan(tt)))
    for k, v in enumerate(c):
        print(f"c{2 * k + 1} = {float(v):.9e}f")
    print(f"max |error| on [0, 1] (FP32 evaluation): {err:.3e} rad")
