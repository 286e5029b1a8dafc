"""The descriptor kernel's arctangent: its constants are the ones fit_atan.py
prints, and that polynomial, evaluated in FP32 with the kernel's octant
reconstruction, stays within 4e-7 rad of the true atan2: the fit error plus
the FP32 rounding of pi - r, half an ulp of pi (well inside the
1e-4 bin-boundary margin the parity tests bracket)."""
import importlib.util
import pathlib
import re

import numpy as np

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_1705_09776_gb300" / "csrc"


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_atan", CSRC / "fit_atan.py")
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _kernel_coefficients():
    src = (CSRC / "describe.cu").read_text()
    body = src[src.index("float atan2_poly("):]
    body = body[:body.index("return copysignf")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    # Horner runs from the highest coefficient down
    return np.array(vals[::-1], np.float32)


def test_kernel_constants_are_the_fit():
    m = _fit_module()
    np.testing.assert_allclose(_kernel_coefficients(), m.fit(), rtol=2e-6, atol=1e-9)


def _atan2_f32(c, y, x):
    y = np.asarray(y, np.float32)
    x = np.asarray(x, np.float32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    t = np.where(mx >= 1e-30, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    p = _fit_module().eval_f32(c, t).astype(np.float32)
    r = np.where(ay > ax, np.float32(np.pi / 2) - p, p).astype(np.float32)
    r = np.where(x < 0, np.float32(np.pi) - r, r).astype(np.float32)
    return np.copysign(r, y)


def test_atan2_error_bound_all_octants():
    rng = np.random.default_rng(7)
    ang = rng.uniform(-np.pi, np.pi, 200000)
    mag = rng.uniform(0.01, 400.0, ang.size)
    y, x = (mag * np.sin(ang)).astype(np.float32), (mag * np.cos(ang)).astype(np.float32)
    got = _atan2_f32(_kernel_coefficients(), y, x).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    d = np.abs(np.angle(np.exp(1j * (got - ref))))
    assert d.max() < 4e-7
    # axes and diagonals
    for yy, xx, want in ((0, 1, 0.0), (1, 0, np.pi / 2), (0, -1, np.pi), (-1, 0, -np.pi / 2), (1, 1, np.pi / 4),
                         (-1, -1, -3 * np.pi / 4)):
        assert abs(_atan2_f32(_kernel_coefficients(), yy, xx) - want) < 4e-7
