"""Pins of the FP64 oracle to the paper and to mathematics (CPU only).

Each test checks the oracle against something other than itself: a closed
form, an invariant, a library routine the definition reduces to, brute force,
or values printed in the paper.  They are chosen so that a dropped term, a
wrong sign or index, or a transposed operand in any step fails one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import oracle as O
from paper_1705_09776_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def P():
    return O.params()


# ---------------------------------------------------------------- S1 filters

@pytest.mark.parametrize("tau", [0.8, 1.2262, 1.52, 2.49, 3.161])
def test_taps_sum_to_one_symmetric_and_variance(tau):
    g = O.gaussian_taps(tau)
    r = (g.size - 1) // 2
    assert r == math.ceil(4 * tau)
    assert abs(g.sum() - 1.0) < 1e-15
    assert np.array_equal(g, g[::-1])
    # second moment of the sampled, 4-sigma-truncated Gaussian is tau^2 up to
    # the truncated tail (relative loss < 2e-3 at 4 sigma)
    p = np.arange(-r, r + 1)
    var = float((p * p * g).sum())
    assert abs(var / (tau * tau) - 1.0) < 2e-3


def test_tau_zero_is_identity():
    assert np.array_equal(O.gaussian_taps(0.0), np.array([1.0]))


def test_separable_equals_bruteforce_2d_and_library():
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 255, size=(23, 31))
    g = O.gaussian_taps(1.953)
    sep = O.filter_separable(img, g)
    bf = O.filter_2d(img, g)
    lib = ndi.correlate(img, np.outer(g, g), mode="nearest")
    assert np.max(np.abs(sep - bf)) <= 1e-12 * np.max(np.abs(bf))
    assert np.max(np.abs(sep - lib)) <= 1e-12 * np.max(np.abs(lib))


def test_constant_stays_constant_and_impulse_gives_kernel():
    g = O.gaussian_taps(2.49)
    c = O.filter_separable(np.full((40, 50), 77.0), g)
    assert np.max(np.abs(c - 77.0)) < 1e-12
    imp = np.zeros((41, 41))
    imp[20, 20] = 1.0
    out = O.filter_separable(imp, g)
    r = (g.size - 1) // 2
    assert np.max(np.abs(out[20 - r:21 + r, 20 - r:21 + r] - np.outer(g, g))) < 1e-16
    # nothing outside the support
    mask = np.ones_like(out, bool)
    mask[20 - r:21 + r, 20 - r:21 + r] = False
    assert np.all(out[mask] == 0.0)
    # an off-centre impulse lands at the same offset (no transposition)
    imp2 = np.zeros((41, 41))
    imp2[10, 30] = 1.0
    assert np.unravel_index(np.argmax(O.filter_separable(imp2, g)), (41, 41)) == (10, 30)


def test_scale_schedule(P):
    s = [O.scale(P, k) for k in range(4)]
    assert s[0] == pytest.approx(1.6) and s[3] == pytest.approx(3.2)
    assert s[1] / s[0] == pytest.approx(2 ** (1 / 3))
    # radii of the level filters: octave 0 assumes 0.5 px input blur, later
    # octaves start from a sigma0-blurred base
    r0 = [(O.gaussian_taps(O.tau(P, 0, k)).size - 1) // 2 for k in range(4)]
    r1 = [(O.gaussian_taps(O.tau(P, 1, k)).size - 1) // 2 for k in range(4)]
    assert r0 == [7, 8, 10, 13]
    assert r1 == [0, 5, 8, 12]


def test_levels_compose_to_the_nominal_blur(P):
    """Filtering a level further by tau' equals (within sampling/truncation
    error) filtering the base by sqrt(tau^2 + tau'^2): the levels carry the
    blurs the schedule claims."""
    rng = np.random.default_rng(2)
    img = ndi.gaussian_filter(rng.uniform(0, 255, (64, 64)), 2.0)
    lv = O.scale_space(img.astype(np.uint8), P)
    base = img.astype(np.uint8).astype(np.float64)
    t1, t3 = O.tau(P, 0, 1), O.tau(P, 0, 3)
    extra = math.sqrt(t3 * t3 - t1 * t1)
    g_extra = O.gaussian_taps(extra)
    a = O.filter_separable(lv[0][1], g_extra)
    b = lv[0][3]
    inner = (slice(16, 48), slice(16, 48))
    assert np.max(np.abs(a[inner] - b[inner])) < 1e-2
    assert np.max(np.abs(O.filter_separable(base, O.gaussian_taps(t3))[inner] - b[inner])) < 1e-12


# --------------------------------------------------------------- S2 Laplacian

def test_laplacian_exact_on_quadratic_and_ramp():
    y, x = np.mgrid[0:20, 0:30].astype(np.float64)
    q = x * x + y * y
    L = O.laplacian(q, 2.0)
    assert np.all(L[1:-1, 1:-1] == 4.0 * 4.0)
    ramp = 3.0 * x - 2.0 * y + 7.0
    assert np.all(O.laplacian(ramp, 1.7)[1:-1, 1:-1] == 0.0)
    # sign: a bright spot has a negative Laplacian
    spot = np.zeros((9, 9))
    spot[4, 4] = 1.0
    assert O.laplacian(spot, 1.0)[4, 4] == -4.0


# --------------------------------------------------------------- S3 ALP fit

def test_alp_exact_on_cubic_data(P):
    rng = np.random.default_rng(3)
    beta = O.alp_matrix(P)
    s = np.array([O.scale(P, k) for k in range(4)])
    for _ in range(50):
        c = rng.normal(size=4) * np.array([10, 10, 5, 2])
        Lk = c[0] + c[1] * s + c[2] * s ** 2 + c[3] * s ** 3
        a = O.alp_fit(beta, Lk)
        assert np.allclose(a, c, rtol=1e-10, atol=1e-10 * np.abs(c).max())


def test_alp_least_squares_for_more_scales():
    P6 = O.params(scales_per_octave=6)
    beta = O.alp_matrix(P6)
    s = np.array([O.scale(P6, k) for k in range(6)])
    c = np.array([1.0, -2.0, 0.5, 0.25])
    a = O.alp_fit(beta, c[0] + c[1] * s + c[2] * s ** 2 + c[3] * s ** 3)
    assert np.allclose(a, c, rtol=1e-10)
    # the fit of non-cubic data is the least-squares one (library lstsq)
    Lk = np.sin(s)
    V = np.vander(s, 4, increasing=True)
    ref = np.linalg.lstsq(V, Lk, rcond=None)[0]
    assert np.allclose(O.alp_fit(beta, Lk), ref, rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------- S4 extremum logic

def _cubic_from_dp_roots(r1, r2, k, c0):
    # p'(s) = 3k (s - r1)(s - r2)  =>  p = k s^3 - 1.5k(r1+r2) s^2 + 3k r1 r2 s + c0
    return np.array([c0, 3 * k * r1 * r2, -1.5 * k * (r1 + r2), k])


def test_extremum_is_analytic_root(P):
    # p' = -3 (s-2)(s-3): minimum at 2, maximum at 3; c0 makes |p(3)| larger
    a = _cubic_from_dp_roots(2.0, 3.0, -1.0, 20.0)
    t, s, v = O.alp_extremum(a, P)
    assert t == +1 and abs(s - 3.0) <= 1e-12 and abs(v - O.cubic(a, 3.0)) < 1e-12
    # with a strongly negative offset the minimum at 2 has the larger |p|
    a = _cubic_from_dp_roots(2.0, 3.0, -1.0, -40.0)
    t, s, v = O.alp_extremum(a, P)
    assert t == -1 and abs(s - 2.0) <= 1e-12
    # root outside [s0, s3] -> nothing
    a = _cubic_from_dp_roots(1.0, 4.0, 1.0, 50.0)
    assert O.alp_extremum(a, P)[0] == 0
    # below contrast
    a = _cubic_from_dp_roots(2.0, 3.0, -1.0, 13.75)   # p(3) = 0.25, p(2) = -0.25
    assert abs(O.cubic(a, 3.0)) < 4 and abs(O.cubic(a, 2.0)) < 4
    assert O.alp_extremum(a, P)[0] == 0
    # quadratic p (a3 = 0): single root of the linear derivative
    a = np.array([30.0, -12.0, 2.5, 0.0])      # p' = 5 s - 12 -> s = 2.4, minimum
    t, s, v = O.alp_extremum(a, P)
    assert t == -1 and abs(s - 2.4) < 1e-15 and v == pytest.approx(30 - 12 * 2.4 + 2.5 * 2.4 ** 2)


def test_extremum_matches_dense_grid_search(P):
    """Brute force: local extrema of p on a dense grid over [s0, s3], with the
    contrast rule and the larger-|p| choice, agree with the root logic."""
    rng = np.random.default_rng(11)
    s0, s3 = O.scale(P, 0), O.scale(P, 3)
    grid = np.linspace(s0, s3, 10001)
    h = grid[1] - grid[0]
    n_checked = {0: 0, 1: 0, -1: 0}
    for _ in range(3000):
        a = rng.normal(size=4) * np.array([20, 40, 15, 3])
        p = a[0] + a[1] * grid + a[2] * grid ** 2 + a[3] * grid ** 3
        inner = p[1:-1]
        ismax = (inner > p[:-2]) & (inner > p[2:])
        ismin = (inner < p[:-2]) & (inner < p[2:])
        cands = []
        for i in np.nonzero(ismax | ismin)[0]:
            if abs(inner[i]) >= 4.0:
                cands.append((abs(inner[i]), grid[i + 1], +1 if ismax[i] else -1))
        t, s, v = O.alp_extremum(a, P)
        # skip draws whose decision sits within grid resolution of a threshold
        near = any(abs(abs(x[0]) - 4.0) < 1e-3 for x in cands) or \
            (t and (abs(s - s0) < 2 * h or abs(s3 - s) < 2 * h or abs(abs(v) - 4.0) < 1e-3))
        if near:
            continue
        if not cands:
            assert t == 0
        else:
            best = max(cands, key=lambda x: x[0])
            if len(cands) == 2 and abs(cands[0][0] - cands[1][0]) < 1e-3:
                continue
            assert t == best[2]
            assert abs(s - best[1]) <= 1.5 * h
        n_checked[t] += 1
    assert min(n_checked.values()) > 100


# ---------------------------------------------------------------- S5 refine

def test_refine_exact_on_quadratic_bump(P):
    rng = np.random.default_rng(4)
    for _ in range(200):
        x0, y0 = rng.uniform(-0.49, 0.49, 2)
        a = rng.uniform(10, 50)
        c = rng.uniform(0.5, 2.0)
        yy, xx = np.mgrid[-1:2, -1:2].astype(np.float64)
        q = a - c * (xx - x0) ** 2 - 2 * c * (yy - y0) ** 2
        ok, out = O.refine(q, P)
        assert ok
        assert abs(out[0] - x0) < 1e-12 and abs(out[1] - y0) < 1e-12
        assert abs(out[2] - a) < 1e-10
        assert out[3] == pytest.approx((3 * c) ** 2 / (2 * c * c))   # (-2c-4c)^2 / (8c^2)
        # minimum: negate
        ok, out = O.refine(-q, P)
        assert ok and abs(out[0] - x0) < 1e-12 and abs(out[2] + a) < 1e-10


def test_refine_rejections(P):
    yy, xx = np.mgrid[-1:2, -1:2].astype(np.float64)
    # offset beyond 0.5
    q = 30 - (xx - 0.6) ** 2 - (yy) ** 2
    assert not O.refine(q, P)[0]
    # saddle
    q = 30 - xx ** 2 + yy ** 2
    assert not O.refine(q, P)[0]
    # edge ratio: Hessian diag(-2a, -2b); (a+b)^2/(ab) = 12.1 exactly at a = 10 b
    b = 0.5
    q = 30 - 10 * b * xx ** 2 - b * yy ** 2
    assert not O.refine(q, P)[0]          # ratio == 12.1 -> rejected
    q = 30 - 9.99 * b * xx ** 2 - b * yy ** 2
    assert O.refine(q, P)[0]
    # refined response below T
    q = 3.9 - 0.1 * xx ** 2 - 0.1 * yy ** 2
    assert not O.refine(q, P)[0]


# ---------------------------------------------- S1-S5 closed-form blob scale

@pytest.mark.parametrize("b,octave", [(3.0, 0), (4.0, 1), (6.0, 1), (10.0, 2)])
def test_blob_scale_closed_form(P, b, octave):
    """A centred isotropic Gaussian blob of std b: the scale-normalised LoG at
    its centre, -2 A b^2 t^2 / (b^2 + t^2)^2, is extremal at t = b.  The
    detector finds a minimum at the centre pixel with sigma within 5% of b
    (cubic fit and discretisation), in the octave whose range holds b."""
    n = 161
    c = 80
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    img = 60.0 + 150.0 * np.exp(-((xx - c) ** 2 + (yy - c) ** 2) / (2 * b * b))
    img = np.rint(img).astype(np.uint8)
    kp, d, nc = O.extract(img, P)
    assert kp.size >= 1
    k = kp[np.argmax(np.abs(kp["response"]))]
    assert k["type"] == -1 and k["response"] < 0
    assert k["octave"] == octave
    assert abs(k["x"] - c) < 1e-9 and abs(k["y"] - c) < 1e-9
    assert abs(k["sigma"] / b - 1.0) < 0.05


# ------------------------------------------------------- S6 decimation

def test_decimation_identity_and_coordinates(P):
    img = synth.blob_image(synth.image_seed(7, 0), 97, 75, n_blobs=20)
    lv = O.scale_space(img, P)
    dims = O.octave_dims(97, 75, P)
    assert dims == [(97, 75), (49, 38), (25, 19), (13, 10)]
    for o in range(1, len(lv)):
        assert np.array_equal(lv[o][0], lv[o - 1][3][::2, ::2])
    c = O.candidates(img, P)
    for k in c:
        s = 2.0 ** k["octave"]
        assert k["x"] == k["xo"] * s and k["y"] == k["yo"] * s and k["sigma"] == k["so"] * s


# ------------------------------------------------------- S7 dedupe

def _kp(x, y, sigma, r, o):
    k = np.zeros(1, O.KP_DTYPE)
    k["x"], k["y"], k["sigma"], k["response"], k["octave"] = x, y, sigma, r, o
    k["xo"], k["yo"], k["so"] = x / 2 ** o, y / 2 ** o, sigma / 2 ** o
    return k


def test_dedupe_rules(P):
    c = np.concatenate([
        _kp(100, 100, 3.2, -20, 0), _kp(101, 99, 3.3, -25, 1),     # pair: second wins
        _kp(200, 50, 3.0, 30, 0), _kp(202, 52, 3.0, 30, 1),         # tie at the window edge: finer wins
        _kp(300, 300, 3.0, 10, 0), _kp(300, 300, 3.0, 50, 0),       # same octave: never duplicates
        _kp(400, 100, 3.0, 10, 0), _kp(400, 100, 3.0, 50, 2),       # octaves 0 and 2, same place and scale: not adjacent
        _kp(500, 100, 3.0, 10, 0), _kp(500, 100, 3.0 * 2 ** (1 / 3) * 1.001, 50, 1),  # outside sigma window
        _kp(600, 100, 6.0, 10, 1), _kp(604, 100, 6.0, 50, 2),       # |dx| = 4 = 2^2 inclusive -> dup
        _kp(50, 400, 6.0, 10, 1), _kp(54.01, 400, 6.0, 50, 2),      # just outside the box
    ])
    keep = O.dedupe(c, P)
    assert keep.tolist() == [False, True, True, False, True, True, True, True, True, True,
                             False, True, True, True]
    # permutation invariance of the decision
    rng = np.random.default_rng(0)
    perm = rng.permutation(c.size)
    keep_p = O.dedupe(c[perm], P)
    assert np.array_equal(keep_p, keep[perm])


def test_dedupe_random_invariants(P):
    rng = np.random.default_rng(9)
    n = 400
    c = np.zeros(n, O.KP_DTYPE)
    c["octave"] = rng.integers(0, 4, n)
    c["x"] = rng.uniform(0, 64, n)
    c["y"] = rng.uniform(0, 64, n)
    c["sigma"] = 1.6 * 2.0 ** (c["octave"] + rng.uniform(0, 1, n))
    c["response"] = rng.normal(0, 20, n)
    keep = O.dedupe(c, P)
    # every removed point has a kept-or-removed adjacent-octave duplicate with larger |r|;
    # the point of largest |r| in the set is never removed
    assert keep[np.argmax(np.abs(c["response"]))]
    # scaling all coordinates by 2 and shifting octaves by one keeps decisions
    c2 = c.copy()
    c2["x"] *= 2
    c2["y"] *= 2
    c2["sigma"] *= 2
    c2["octave"] += 1
    assert np.array_equal(O.dedupe(c2, P), keep)


# ------------------------------------------------------- S8 selection

def test_selection_order_and_cap():
    P = O.params(max_keypoints=5)
    c = np.concatenate([_kp(10, 5, 2, 7, 0), _kp(3, 5, 2, -7, 0), _kp(1, 9, 2, 9, 0),
                        _kp(8, 1, 2, 7, 0), _kp(1, 1, 2, 1, 0), _kp(2, 2, 2, 100, 0),
                        _kp(5, 5, 2, 0.5, 0)])
    order = O.dedupe_select(c, P)
    # |r| desc, then y asc, then x asc
    assert order.tolist() == [5, 2, 3, 1, 0]


# ------------------------------------------------- S9/S10 rotation invariance

@pytest.fixture(scope="module")
def rot_pair():
    img = synth.blob_image(synth.image_seed(21, 0), 641, 481, n_blobs=120)
    return img, np.ascontiguousarray(np.rot90(img))


def _match_rot(kpa, kpb, W):
    # (x, y) in A -> (y, W - 1 - x) in B
    out = []
    for i, k in enumerate(kpa):
        xb, yb = k["y"], W - 1 - k["x"]
        d = np.abs(kpb["x"] - xb) + np.abs(kpb["y"] - yb) + np.abs(kpb["sigma"] - k["sigma"])
        j = int(np.argmin(d))
        out.append((i, j, d[j]))
    return out


def test_rotation_90_oriented(rot_pair):
    img, rot = rot_pair
    P = O.params()
    ka, da, _ = O.extract(img, P)
    kb, db, _ = O.extract(rot, P)
    assert ka.size == kb.size and ka.size > 200
    W = img.shape[1]
    for i, j, dist in _match_rot(ka, kb, W):
        assert dist < 1e-9
        dth = (ka["theta"][i] - math.pi / 2 - kb["theta"][j]) % (2 * math.pi)
        dth = min(dth, 2 * math.pi - dth)
        if dth > 1e-9:
            # same point, another orientation copy
            continue
        assert np.max(np.abs(da[i] - db[j])) < 1e-9
    # every record found its rotated twin with the same theta - pi/2
    th_a = sorted((round(k["x"], 6), round(k["y"], 6), round((k["theta"] - math.pi / 2) % (2 * math.pi), 6))
                  for k in ka)
    th_b = sorted((round(W - 1 - k["y"], 6), round(k["x"], 6), round(k["theta"], 6)) for k in kb)
    assert th_a == th_b


def test_rotation_90_upright_permutes_bins(rot_pair):
    img, rot = rot_pair
    P = O.params(upright=1)
    ka, da, _ = O.extract(img, P)
    kb, db, _ = O.extract(rot, P)
    W = img.shape[1]
    # cell (cx, cy) of A goes to (cy, 3 - cx) of B; orientation bin b -> b - 2 (mod 8)
    perm = np.zeros(128, int)
    for cy in range(4):
        for cx in range(4):
            for b in range(8):
                perm[(cy * 4 + cx) * 8 + b] = ((3 - cx) * 4 + cy) * 8 + (b - 2) % 8
    for i, j, dist in _match_rot(ka, kb, W):
        assert dist < 1e-9
        assert np.max(np.abs(db[j][perm] - da[i])) < 1e-9
        assert np.max(np.abs(da[i] - db[j])) > 1e-3   # really a permutation, not identity


# ------------------------------------------------------- S9 orientation

@pytest.mark.parametrize("phi_deg", [5.0, 101.0, 203.0, 333.0])
def test_orientation_of_a_ramp(P, phi_deg):
    phi = math.radians(phi_deg)
    yy, xx = np.mgrid[0:60, 0:60].astype(np.float64)
    G = 3.0 * (math.cos(phi) * xx + math.sin(phi) * yy)
    th, hist = O.orientations(G, 30.2, 29.7, 2.0, P)
    b = int(math.floor(36 * phi / (2 * math.pi))) % 36
    assert np.count_nonzero(hist) == 1 and hist[b] > 0
    assert th.size == 1 and abs(th[0] - 2 * math.pi * (b + 0.5) / 36) < 1e-12


def test_orientation_peaks_rule(P):
    """Two ramps in the two halves of a patch give two dominant bins: every
    local maximum above 0.8 of the highest is returned, by value, and no
    other bin is."""
    yy, xx = np.mgrid[0:61, 0:61].astype(np.float64)
    G = np.where(yy < 30, 3.0 * xx, 2.7 * yy + 3.0 * 30)   # gradient along x above, along y below
    th, hist = O.orientations(G, 30, 30, 2.0, P)
    l, r = np.roll(hist, 1), np.roll(hist, -1)
    want = [b for b in range(36) if hist[b] > l[b] and hist[b] > r[b] and hist[b] > 0.8 * hist.max()]
    want = sorted(want, key=lambda b: (-hist[b], b))[:4]
    got = [int(t * 36 / (2 * math.pi)) % 36 for t in th]
    assert got == want and len(got) >= 1


@pytest.mark.parametrize("x0", [5.5, 5.83, 5.21, 0.3, 35.9, 17.64])
def test_orientation_peak_is_the_parabola_vertex(P, x0):
    """Three bins sampled from an exact parabola y = A - B (x - x0)^2 at the
    bin centres (bin b is centred at b + 1/2, in bin units): the refined angle
    is the parabola's own vertex, 2 pi x0 / 36, on either side of the centre
    and across the wrap at bin 0 / 35."""
    A, Bc = 10.0, 1.7
    b = int(math.floor(x0))
    h = np.zeros(36)
    for j in (b - 1, b, b + 1):
        h[j % 36] = A - Bc * ((j + 0.5) - x0) ** 2
    th = O.orientation_peaks(h, P)
    assert th.size == 1
    want = (2 * math.pi * x0 / 36) % (2 * math.pi)
    assert abs(th[0] - want) < 1e-12, (th[0], want)


def test_orientation_peak_ratio_and_order(P):
    """Sec. IV-B: a bin is an orientation when it is a local maximum above
    0.8 x the highest bin (strictly); peaks come out by value, at most 4."""
    def peaks(vals):
        h = np.zeros(36)
        for b, v in vals.items():
            h[b] = v
        return [int(round(t * 36 / (2 * math.pi) - 0.5)) % 36 for t in O.orientation_peaks(h, P)]

    assert peaks({3: 1.0, 20: 0.85}) == [3, 20]
    assert peaks({3: 0.85, 20: 1.0}) == [20, 3]        # by value, not by bin
    assert peaks({3: 1.0, 20: 0.75}) == [3]
    assert peaks({3: 1.0, 20: 0.8}) == [3]             # strictly above 0.8 x max
    assert peaks({3: 1.0, 20: 0.8000001}) == [3, 20]
    assert peaks({3: 1.0, 9: 1.0}) == [3, 9]           # equal values: lower bin first
    six = {2: 0.95, 8: 0.99, 14: 0.96, 20: 1.0, 26: 0.98, 32: 0.97}
    assert peaks(six) == [20, 8, 26, 32]               # the 4 largest, by value
    assert peaks({4: 1.0, 5: 1.0}) == []               # a plateau is not strictly above its neighbour
    assert peaks({4: 1.0, 5: 0.9}) == [4]              # a shoulder is no peak


def _voters(shape, spec):
    """A patch whose only non-zero central-difference gradients inside the
    sampling disc are chosen pixels: for a pixel P and an outward unit step
    e, G = a at P + e gives P the gradient a e and moves the other three
    pixels that see it (P + 2e, P + e +- e_perp) further out."""
    G = np.zeros(shape)
    for (u, v), (ex, ey), a in spec:
        G[v + ey, u + ex] += a
    return G


def test_orientation_vote_weight_closed_form(P):
    """Alg. 2 stage A with one gradient sample inside the disc: the bin of its
    angle gets |g| exp(-d^2 / (2 (1.5 sigma)^2)), every other bin nothing.
    sigma = 2: disc radius 3.96 x 2 = 7.92 px, the voter at d = 7.7 px
    (gradient along +x, bin 0) and the others of its bump beyond 8.7 px."""
    xo, yo, so = 30.3, 30.0, 2.0
    G = _voters((61, 61), [((38, 30), (1, 0), 1.0)])
    th, h = O.orientations(G, xo, yo, so, P)
    want = math.exp(-7.7 ** 2 / (2 * (1.5 * 2.0) ** 2))
    assert h[0] == pytest.approx(want, rel=1e-12)
    assert np.count_nonzero(h) == 1
    assert th.size == 1 and abs(th[0] - 2 * math.pi * 0.5 / 36) < 1e-12


@pytest.mark.parametrize("ratio,n_peaks", [(0.85, 2), (0.75, 1), (1 / 0.85, 2), (1 / 0.75, 1)])
def test_orientation_two_voters_peak_rule(P, ratio, n_peaks):
    """Two gradient samples at d = 7.7 px (angle 0, bin 0) and d' = 7.3 px
    (angle pi, bin 18), with magnitudes set so that their weighted votes are
    in a given ratio: with the weight window exp(-d^2 / (2 (1.5 sigma)^2))
    the weaker one is an orientation at 0.85 of the stronger and not at 0.75,
    and the stronger comes first."""
    xo, yo, so = 30.3, 30.0, 2.0
    w = lambda d: math.exp(-d * d / 18.0)
    a2 = ratio * w(7.7) / w(7.3)   # vote(bin 18) / vote(bin 0) = ratio
    G = _voters((61, 61), [((38, 30), (1, 0), 1.0), ((23, 30), (-1, 0), a2)])
    th, h = O.orientations(G, xo, yo, so, P)
    assert np.count_nonzero(h) == 2
    assert h[18] / h[0] == pytest.approx(ratio, rel=1e-12)
    bins = [int(round(t * 36 / (2 * math.pi) - 0.5)) % 36 for t in th]
    strong, weak = (0, 18) if ratio < 1 else (18, 0)
    assert bins == [strong, weak][:n_peaks]


# ------------------------------------------------------- S10 descriptor

def test_descriptor_normalisation(P):
    img = synth.blob_image(synth.image_seed(1, 0))
    kp, d, _ = O.extract(img, P)
    n = np.linalg.norm(d, axis=1)
    assert np.allclose(n, 1.0, atol=1e-12)
    assert np.all(d >= 0)
    # after clamping at 0.2 and renormalising, no element exceeds 0.2 / ||clamped||
    # and the descriptor of a flat patch is all zeros
    flat = np.full((50, 50), 9.0)
    assert np.all(O.descriptor(flat, 25, 25, 2.0, 0.3, P) == 0.0)


def test_descriptor_of_a_ramp_uses_only_two_orientation_bins(P):
    phi = math.radians(40.0)
    yy, xx = np.mgrid[0:80, 0:80].astype(np.float64)
    G = 2.0 * (math.cos(phi) * xx + math.sin(phi) * yy)
    theta = 0.1
    d = O.descriptor(G, 40, 40, 2.0, theta, P).reshape(16, 8)
    ob = 8 * ((phi - theta) % (2 * math.pi)) / (2 * math.pi)
    b0 = int(math.floor(ob))
    used = np.nonzero(d.sum(axis=0))[0].tolist()
    assert used == sorted([b0 % 8, (b0 + 1) % 8])
    # trilinear split between the two bins in the ratio of the distances
    # (clamping at 0.2 then renormalising keeps the ratio in every cell whose
    # two values are both below the clamped maximum)
    f = ob - b0
    top = d.max()
    n_cells = 0
    for cell in d:
        if cell.max() < top - 1e-12 and cell[b0 % 8] > 0:
            assert cell[(b0 + 1) % 8] / cell[b0 % 8] == pytest.approx(f / (1 - f), rel=1e-9)
            n_cells += 1
    assert n_cells >= 4


def test_descriptor_single_vote_by_hand(P):
    """Alg. 2 stage B with one gradient sample inside the 6 sigma disc: its
    vote lands in the cells and bins predicted by hand from cells of side
    3 sigma centred on the keypoint (cell coordinate u + 1.5), the weight
    |g| exp(-(u^2 + v^2) / 8) with (u, v) in cells, and the trilinear split.

    sigma = 1.25: disc radius 7.5 px, cell side 3.75 px.  The voter sits 6.75
    px right of the keypoint (u = 1.8 cells, v = 0) with gradient (1, 0); the
    rest of its bump lies beyond 7.8 px."""
    xo, yo, so = 30.25, 30.0, 1.25
    G = _voters((61, 61), [((37, 30), (1, 0), 1.0)])
    wgt = math.exp(-(1.8 ** 2) / 8.0)
    # theta = 0: x cell 1.8 + 1.5 = 3.3 -> cell 3 with 0.7 (cell 4 is outside
    # the grid); y cell 1.5 -> cells 1 and 2 with 0.5 each; angle 0 -> bin 0
    h = O.descriptor_hist(G, xo, yo, so, 0.0, P)
    want = np.zeros((4, 4, 8))
    want[1, 3, 0] = want[2, 3, 0] = wgt * 0.7 * 0.5
    assert np.allclose(h, want, rtol=0, atol=1e-13), np.argwhere(h != 0)
    # theta = pi / 2: the offset rotates by -pi / 2 to (0, -1.8) cells, so y
    # cell -0.3 -> row 0 with 0.7 (row -1 is outside); x cell 1.5 -> cells 1
    # and 2 with 0.5; the angle relative to theta is 3 pi / 2 -> bin 6
    h = O.descriptor_hist(G, xo, yo, so, math.pi / 2, P)
    want = np.zeros((4, 4, 8))
    want[0, 1, 6] = want[0, 2, 6] = wgt * 0.7 * 0.5
    assert np.allclose(h, want, rtol=0, atol=1e-13), np.argwhere(h != 0)


def test_descriptor_single_vote_off_axis(P):
    """An off-axis voter: offset (6, 3) px at sigma = 1.15 (disc 6.9 px, cell
    side 3.45 px), gradient (2, 0), orientation theta = 0.  Cells: x = 6 / 3.45
    + 1.5, y = 3 / 3.45 + 1.5; weight 2 exp(-((6^2 + 3^2) / 3.45^2) / 8); the
    orientation split of angle 0 - theta."""
    xo, yo, so = 30.0, 30.0, 1.15
    G = _voters((61, 61), [((36, 33), (1, 0), 2.0)])
    cx, cy = 6 / 3.45 + 1.5, 3 / 3.45 + 1.5          # 3.2391.., 2.3695..
    fx, fy = cx - 3, cy - 2
    wgt = 2.0 * math.exp(-(45 / 3.45 ** 2) / 8.0)
    h = O.descriptor_hist(G, xo, yo, so, 0.0, P)
    want = np.zeros((4, 4, 8))
    want[2, 3, 0] = wgt * (1 - fy) * (1 - fx)
    want[3, 3, 0] = wgt * fy * (1 - fx)
    assert np.allclose(h, want, rtol=0, atol=1e-13), np.argwhere(h != 0)
    # theta = -pi / 8 (i.e. 15 pi / 8): the gradient is at +pi / 8 relative to
    # theta, half-way between bins 0 and 1 (bin width pi / 4)
    t = -math.pi / 8
    h = O.descriptor_hist(G, xo, yo, so, t, P)
    u = (math.cos(t) * 6 + math.sin(t) * 3) / 3.45
    v = (-math.sin(t) * 6 + math.cos(t) * 3) / 3.45
    assert u * u + v * v == pytest.approx(45 / 3.45 ** 2, rel=1e-12)   # rotation keeps the radius
    cx, cy = u + 1.5, v + 1.5                         # 2.774.., 2.969..
    assert (math.floor(cx), math.floor(cy)) == (2, 2)
    fx, fy = cx - 2, cy - 2
    want = np.zeros((4, 4, 8))
    for yy, wy in ((2, 1 - fy), (3, fy)):
        for xx, wx in ((2, 1 - fx), (3, fx)):
            want[yy, xx, 0] = want[yy, xx, 1] = wgt * wy * wx * 0.5
    assert np.allclose(h, want, rtol=0, atol=1e-13), np.argwhere(h != 0)


# ------------------------------------------------------- S11 transform + ternary

def _golden_sets():
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "transform_sets.txt"))
            if l.strip() and not l.startswith("#")]
    M = np.array(rows)
    return M[:8], M[8:]


def test_transform_matches_printed_sets():
    A, B = _golden_sets()
    for cell in range(16):
        cy, cx = divmod(cell, 4)
        M = A if (cx + cy) % 2 == 0 else B
        for j in range(8):
            e = np.zeros(128)
            e[cell * 8 + j] = 1.0
            v = O.transform(e)
            assert np.array_equal(v[cell * 8:cell * 8 + 8], M[:, j])
            assert np.count_nonzero(v) == np.count_nonzero(M[:, j])


def test_ternary_values_and_thresholds():
    rng = np.random.default_rng(1)
    v = rng.normal(size=128)
    lo = np.full(128, -0.3)
    hi = np.full(128, 0.3)
    q = O.ternary(v, lo, hi)
    assert set(np.unique(q)).issubset({-1, 0, 1})
    assert np.array_equal(q, np.where(v < -0.3, -1, np.where(v > 0.3, 1, 0)))


def test_extremum_tie_goes_to_the_smaller_sigma(P):
    """Sec. III-A with two qualifying roots of equal |p|: p(s) = 32 ((s - 2.5)^3
    - 0.75 (s - 2.5)) has p' = 96 (s - 2)(s - 3), p(2) = 8 (a maximum) and
    p(3) = -8 (a minimum), all exact in binary.  Both lie in [1.6, 3.2] and
    reach the contrast 4, so the tie rule decides: the smaller sigma."""
    a = np.array([-440.0, 576.0, -240.0, 32.0])
    assert O.alp_extremum(a, P) == (1, 2.0, 8.0)
    assert O.alp_extremum(-a, P) == (-1, 2.0, -8.0)   # the mirrored cubic: a minimum at 2


def test_descriptor_level_is_the_nearest_in_log_scale(P):
    """Alg. 2 reads the Gaussian level nearest to sigma in log scale: level k
    of s_k = sigma0 2^(k/3), so t = 3 log2(sigma/sigma0) rounds to the
    nearest integer, clamped to 0..3."""
    for t, k in [(-0.7, 0), (0.0, 0), (0.4, 0), (0.6, 1), (1.4, 1), (1.6, 2), (2.6, 3), (3.0, 3), (3.8, 3)]:
        assert O.desc_level(P, 1.6 * 2.0 ** (t / 3.0)) == k, t


@pytest.mark.parametrize("radius,inside", [(4.0, False), (4.0 + 1e-9, True)])
def test_orientation_disc_is_open(radius, inside):
    """Sec. IV-B takes the pixels closer than the radius: a voter at distance
    exactly 4 px (sigma = 1, radius 4 sigma) votes nothing, one just inside the
    radius votes |g| exp(-d^2 / (2 (1.5 sigma)^2)) into bin 0.  The voter's bump
    pixels lie 5 px or more away."""
    p = O.params(ori_radius=radius)
    G = _voters((41, 41), [((24, 20), (1, 0), 1.0)])
    th, h = O.orientations(G, 20.0, 20.0, 1.0, p)
    if inside:
        assert h[0] == pytest.approx(math.exp(-16.0 / (2 * 1.5 ** 2)), rel=1e-12)
        assert np.count_nonzero(h) == 1
    else:
        assert not h.any() and th.size == 0


def test_descriptor_clamp_level(P):
    """Alg. 2 stage B normalises the 128 sums, clamps at 0.2 and normalises
    again.  With n = h / |h| and d the descriptor, every entry with n > 0.2
    takes the same value max(d), and every other entry keeps its ratio to the
    clamped ones: d_i / max(d) = n_i / 0.2.  That fixes the clamp level from
    the two outputs without redoing the normalisation."""
    img = synth.blob_image(synth.image_seed(23, 0), 96, 96, n_blobs=6).astype(np.float64)
    G = O.filter_separable(img, O.gaussian_taps(2.0))
    for xo, yo, so, theta in [(48.3, 47.6, 2.2, 0.4), (40.0, 55.5, 3.0, 2.0)]:
        h = O.descriptor_hist(G, xo, yo, so, theta, P).ravel()
        d = O.descriptor(G, xo, yo, so, theta, P)
        n = h / np.linalg.norm(h)
        big = n > 0.2
        assert big.any() and (~big & (n > 0)).any()
        assert np.allclose(d[big], d.max(), rtol=1e-13, atol=0)
        np.testing.assert_allclose(d[~big] / d.max(), n[~big] / 0.2, rtol=1e-12, atol=1e-15)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-12


def test_ternary_thresholds_are_strict():
    """Sec. III-C: an element is -1 below its lower threshold and +1 above its
    upper one; an element equal to either threshold is 0."""
    lo, hi = np.full(128, -0.25), np.full(128, 0.5)
    v = np.zeros(128)
    v[:4] = [-0.25, 0.5, -0.2500001, 0.5000001]
    q = O.ternary(v, lo, hi)
    assert q[:4].tolist() == [0, 0, -1, 1] and not q[4:].any()


def test_octave_needs_three_pixels_per_side(P):
    """Alg. 1 builds octaves while both sides are at least 3 px (the 3 x 3
    neighbour test needs an interior pixel); each octave is ceil(side / 2) of
    the previous one."""
    assert O.octave_dims(10, 5, P) == [(10, 5), (5, 3)]          # next would be 3 x 2
    assert O.octave_dims(3, 3, P) == [(3, 3)]
    assert O.octave_dims(2, 40, P) == []
    assert O.octave_dims(40, 40, P) == [(40, 40), (20, 20), (10, 10), (5, 5)]


def test_contrast_and_scale_range_are_inclusive():
    """Sec. III-A: a root counts when |p| >= T and sigma lies in the closed
    range [s_0, s_3].  p(s) = 2 s^3 - 21 s^2 + 60 s + a0 has p' = 6 (s - 2)(s - 5)
    (roots exact in binary), a maximum at 2 and p(2) = a0 + 52."""
    P = O.params()
    assert O.alp_extremum(np.array([-48.0, 60.0, -21.0, 2.0]), P) == (1, 2.0, 4.0)   # |p| = T = 4
    assert O.alp_extremum(np.array([-48.5, 60.0, -21.0, 2.0]), P)[0] == 0           # |p| = 3.5 < T
    P2 = O.params(sigma0=2.0)                                                        # range [2, 4]
    assert O.alp_extremum(np.array([-44.0, 60.0, -21.0, 2.0]), P2) == (1, 2.0, 8.0)  # root at s_0
    P3 = O.params(sigma0=2.0000001)
    assert O.alp_extremum(np.array([-44.0, 60.0, -21.0, 2.0]), P3)[0] == 0           # just outside


def test_refine_offset_limit_is_inclusive(P):
    """Alg. 1 stage B keeps a point whose offset is at most offset_max (0.5):
    q with left 0, centre 8, right 8, top and bottom 0 gives g = (4, 0),
    H = diag(-8, -16), delta = (0.5, 0), p-hat = 8 + 0.5 * 4 * 0.5 = 9 and
    tr^2 / det = 576 / 128 = 4.5, all exact.  A right value of 8.5 moves the
    offset to 4.25 / 7.5 > 0.5 and drops it."""
    q = np.array([[0.0, 0.0, 0.0], [0.0, 8.0, 8.0], [0.0, 0.0, 0.0]])
    ok, out = O.refine(q, P)
    assert ok == 1 and out.tolist() == [0.5, 0.0, 9.0, 4.5]
    q[1, 2] = 8.5
    assert O.refine(q, P)[0] == 0


@pytest.mark.parametrize("radius,inside", [(4.0, False), (4.0 + 1e-9, True)])
def test_descriptor_disc_is_open(radius, inside):
    """Alg. 2 stage B samples the pixels closer than desc_radius * sigma: a
    voter at exactly 4 px (sigma = 1, radius 4) votes nothing; just inside it
    votes.  Its bump pixels lie 5 px or more away."""
    p = O.params(desc_radius=radius)
    G = _voters((41, 41), [((24, 20), (1, 0), 1.0)])
    h = O.descriptor_hist(G, 20.0, 20.0, 1.0, 0.0, p)
    assert bool(h.any()) == inside


def test_selection_ties_by_sigma_then_octave():
    """Eq. 5's order is total: |response| descending, then y, x, sigma and
    octave ascending.  Five records equal in |response|, y and x (one of them
    negative) sort by sigma, then by octave."""
    c = np.concatenate([_kp(10, 10, 3.0, 5, 1), _kp(10, 10, 2.0, -5, 1), _kp(10, 10, 2.0, 5, 0),
                        _kp(10, 10, 2.0, 5, 2), _kp(10, 10, 2.5, 5, 0)])
    P = O.params()
    keep = np.ones(c.size, np.uint8)
    order = np.zeros(c.size, np.int32)
    n = O.lib().oracle_select(O._p(c), O._p(keep), c.size, O._p(P), O._p(order))
    assert order[:n].tolist() == [2, 1, 3, 4, 0]


@pytest.mark.parametrize("ori_margin,bin_", [(0.0, 35), (1e-3, 0), (-1e-3, 35)])
def test_orientation_bin_bracketing_direction(ori_margin, bin_):
    """The bracketing runs move a vote within ori_margin (a fraction of a bin)
    of a bin edge across that edge.  One voter at d = 7.7 px (sigma = 2) with
    gradient (1, -1e-4): angle -1e-4 rad, 5.7e-4 of a bin below the edge of
    bin 0, so it lands in bin 35, and in bin 0 once ori_margin = 1e-3 moves it
    up; a negative margin moves only votes just above an edge.  Its tilt
    leaves one other pixel of weight 1e-4 in bin 0."""
    p = O.params(ori_margin=ori_margin)
    G = _voters((61, 61), [((38, 30), (1, 0), 1.0), ((38, 30), (0, -1), 1e-4)])
    _, h = O.orientations(G, 30.3, 30.0, 2.0, p)
    w = math.sqrt(1 + 1e-8) * math.exp(-7.7 ** 2 / (2 * (1.5 * 2.0) ** 2))
    assert h[bin_] == pytest.approx(w, rel=1e-3)
    others = np.delete(h, [bin_, 0])
    assert not others.any()


def test_p_ss_is_the_cubics_second_derivative(P):
    """p_ss of a record is d2p/dsigma2 of its pixel's ALP cubic at sigma*, and
    sigma* is a root of dp/dsigma.  The cubic is rebuilt from the separately
    pinned steps: levels, scale-normalised Laplacians and the ALP fit."""
    img = synth.blob_image(synth.image_seed(24, 0), 120, 90, n_blobs=12)
    levels = O.scale_space(img, P)
    beta = O.alp_matrix(P)
    L = [O.laplacian(levels[0][k], O.scale(P, k)) for k in range(4)]
    c = O.candidates(img, P)
    c = c[c["octave"] == 0]
    assert c.size >= 5
    for k in c:
        x, y = int(round(k["xo"])), int(round(k["yo"]))
        a = O.alp_fit(beta, np.array([Lk[y, x] for Lk in L]))
        s = k["so"]
        assert abs(3 * a[3] * s * s + 2 * a[2] * s + a[1]) <= 1e-9 * (abs(a[1]) + abs(a[2] * s) + abs(a[3] * s * s))
        assert k["p_ss"] == pytest.approx(6 * a[3] * s + 2 * a[2], rel=1e-12, abs=1e-12)


def test_laplacian_clamps_to_the_edge():
    """Alg. 1's 5-point Laplacian reads the edge pixel again outside the level.
    On G = x + 5 (20 x 30): at x = 0 the left sample is G(0) = 5, so the sum
    is 5 + 6 + 5 + 5 - 4 * 5 = 1; at x = 29 the right sample is G(29), giving
    -1; interior columns give 0.  Scaled by s^2 = 4."""
    y, x = np.mgrid[0:20, 0:30].astype(np.float64)
    L = O.laplacian(x + 5.0, 2.0)
    assert np.all(L[:, 0] == 4.0) and np.all(L[:, -1] == -4.0) and np.all(L[:, 1:-1] == 0.0)
    L = O.laplacian(y + 5.0, 2.0)
    assert np.all(L[0, :] == 4.0) and np.all(L[-1, :] == -4.0) and np.all(L[1:-1, :] == 0.0)


def test_detection_covers_every_interior_pixel(P):
    """Alg. 1's 3 x 3 test runs at every pixel that has all eight neighbours:
    bright 3 x 3 dots centred on rows 1 and 62 and columns 1 and 78 of a flat
    64 x 80 image give extrema on those rows and columns of the first octave
    (a refined position stays within 0.5 px of its pixel)."""
    img = np.full((64, 80), 100, np.uint8)
    for x, y in [(40, 1), (40, 62), (1, 30), (78, 30)]:
        img[y - 1:y + 2, x - 1:x + 2] = 200
    c = O.candidates(img, P)
    c = c[c["octave"] == 0]
    ys, xs = np.rint(c["yo"]).astype(int), np.rint(c["xo"]).astype(int)
    assert ys.min() == 1 and ys.max() == 62 and xs.min() == 1 and xs.max() == 78


def test_describe_reads_the_nearest_level(P):
    """Alg. 2 describes a point on the Gaussian level of its octave nearest to
    its scale: the pipeline's descriptors equal the stage run by hand on level
    desc_level(sigma) of that octave, for points of levels 0 to 3 in octaves 0
    and 1."""
    img = synth.blob_image(synth.image_seed(25, 0), 96, 80, n_blobs=10)
    levels = O.scale_space(img, P)
    pts = np.concatenate([_kp(40.3, 37.6, 1.6 * 2 ** (t / 3) * 2 ** o, 9.0, o)
                          for o in (0, 1) for t in (0.0, 1.1, 1.9, 3.0)])
    kp, d = O.describe(img, pts, O.params(upright=1))
    assert len(kp) == len(pts)
    for r, dr in zip(kp, d):
        k = O.desc_level(P, r["so"])
        want = O.descriptor(levels[r["octave"]][k], r["xo"], r["yo"], r["so"], 0.0, P)
        np.testing.assert_array_equal(dr, want)
    assert sorted({O.desc_level(P, r["so"]) for r in kp}) == [0, 1, 2, 3]


@pytest.mark.parametrize("right,n_points", [(1.0, 0), (1.25, 1)])
def test_neighbour_test_is_strict(P, right, n_points):
    """Alg. 1's 3 x 3 test wants the centre strictly beyond all 8 neighbours.
    Levels G_k = c_k B, B a horizontal domino (1 and `right` at (9, 8) and
    (10, 8)), c_k = w_k / s_k^2 with w = 100 (1, 3, 3, 1): every response is
    B's Laplacian times one cubic in sigma with a maximum inside the octave.
    With equal pixels the two responses tie exactly (the same operations on
    the same values), so neither is a minimum and nothing is found; the ring
    around them ties too.  With 1.25 on the right, that pixel is a strict
    minimum and is found."""
    B = np.zeros((16, 20))
    B[8, 9], B[8, 10] = 1.0, right
    w = 100.0 * np.array([1.0, 3.0, 3.0, 1.0])
    levels = np.stack([w[k] / O.scale(P, k) ** 2 * B for k in range(4)])
    c = O.detect_levels(levels, 0, P)
    assert len(c) == n_points
    if n_points:
        assert c[0]["type"] == -1 and abs(c[0]["xo"] - 10) <= 0.5 and c[0]["yo"] == 8.0
