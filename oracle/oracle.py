"""ctypes wrapper of the FP64 CPU oracle (cdvs_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg are the only users.  The product path never
imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libcdvs_oracle.so")
SRC = os.path.join(HERE, "cdvs_oracle.c")

PARAMS_DTYPE = np.dtype([
    ("num_octaves", "<i4"), ("scales_per_octave", "<i4"),
    ("sigma0", "<f8"), ("sigma_in", "<f8"), ("contrast_T", "<f8"), ("edge_r", "<f8"),
    ("offset_max", "<f8"), ("ori_radius", "<f8"), ("ori_peak_ratio", "<f8"),
    ("ori_weight_sigma", "<f8"), ("desc_radius", "<f8"), ("cell_side", "<f8"),
    ("desc_weight_sigma", "<f8"), ("dedupe_dlog2", "<f8"),
    ("max_keypoints", "<i4"), ("max_orientations", "<i4"), ("upright", "<i4"), ("pad0", "<i4"),
    ("margin", "<f8"), ("ori_margin", "<f8"),
], align=True)

KP_DTYPE = np.dtype([
    ("x", "<f8"), ("y", "<f8"), ("sigma", "<f8"),
    ("xo", "<f8"), ("yo", "<f8"), ("so", "<f8"),
    ("theta", "<f8"), ("response", "<f8"), ("p_ss", "<f8"), ("ratio", "<f8"),
    ("octave", "<i4"), ("scale_idx", "<i4"), ("type", "<i4"), ("parent", "<i4"),
], align=True)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, FP contraction off so x86 and
    Arm builds round alike)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "cdvs_oracle.h"))):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        i32, f64, sz = C.c_int, C.c_double, C.c_size_t
        sig = {
            "oracle_params_default": (None, [P]),
            "oracle_octave_dims": (i32, [i32, i32, P, P, P]),
            "oracle_levels_size": (sz, [i32, i32, P]),
            "oracle_level_offset": (sz, [i32, i32, P, i32, i32]),
            "oracle_scale": (f64, [P, i32]),
            "oracle_tau": (f64, [P, i32, i32]),
            "oracle_gaussian_taps": (i32, [f64, P, i32]),
            "oracle_filter_separable": (None, [P, i32, i32, P, i32, P]),
            "oracle_filter_2d": (None, [P, i32, i32, P, i32, P]),
            "oracle_scale_space": (i32, [P, i32, i32, i32, P, P]),
            "oracle_laplacian": (None, [P, i32, i32, f64, P]),
            "oracle_alp_matrix": (i32, [P, P]),
            "oracle_alp_fit": (None, [P, P, i32, P]),
            "oracle_cubic": (f64, [P, f64]),
            "oracle_alp_extremum": (i32, [P, P, P, P]),
            "oracle_refine": (i32, [P, P, P]),
            "oracle_detect_levels": (i32, [P, i32, i32, i32, P, P, i32]),
            "oracle_dedupe": (None, [P, i32, P, P]),
            "oracle_select": (i32, [P, P, i32, P, P]),
            "oracle_orientations": (i32, [P, i32, i32, f64, f64, f64, P, P, P]),
            "oracle_descriptor": (None, [P, i32, i32, f64, f64, f64, f64, P, P]),
            "oracle_orientation_peaks": (i32, [P, P, P]),
            "oracle_descriptor_hist": (None, [P, i32, i32, f64, f64, f64, f64, P, P]),
            "oracle_desc_level": (i32, [P, f64]),
            "oracle_extract": (i32, [P, i32, i32, i32, P, P, P, i32, P]),
            "oracle_candidates": (i32, [P, i32, i32, i32, P, P, i32]),
            "oracle_dedupe_select": (i32, [P, i32, P, P]),
            "oracle_describe": (i32, [P, i32, i32, i32, P, P, i32, P, P, i32]),
            "oracle_extract_batch": (i32, [i32, P, P, P, P, P, P, P, i32, P, i32]),
            "oracle_num_threads": (i32, []),
            "oracle_transform": (None, [P, P]),
            "oracle_ternary": (None, [P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def params(**kw) -> np.ndarray:
    """Default oracle parameters (a one-element structured array), with overrides."""
    p = np.zeros(1, dtype=PARAMS_DTYPE)
    lib().oracle_params_default(_p(p))
    for k, v in kw.items():
        p[k] = v
    return p


def octave_dims(W, H, p):
    Wo = np.zeros(16, np.int32)
    Ho = np.zeros(16, np.int32)
    n = lib().oracle_octave_dims(W, H, _p(p), _p(Wo), _p(Ho))
    return [(int(Wo[i]), int(Ho[i])) for i in range(n)]


def scale(p, k):
    return lib().oracle_scale(_p(p), k)


def tau(p, o, k):
    return lib().oracle_tau(_p(p), o, k)


def gaussian_taps(t: float) -> np.ndarray:
    buf = np.zeros(1025, np.float64)
    r = lib().oracle_gaussian_taps(float(t), _p(buf), buf.size)
    assert r >= 0
    return buf[:2 * r + 1].copy()


def filter_separable(img: np.ndarray, taps: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(img, np.float64)
    t = np.ascontiguousarray(taps, np.float64)
    out = np.empty_like(a)
    lib().oracle_filter_separable(_p(a), a.shape[1], a.shape[0], _p(t), (t.size - 1) // 2, _p(out))
    return out


def filter_2d(img: np.ndarray, taps: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(img, np.float64)
    t = np.ascontiguousarray(taps, np.float64)
    out = np.empty_like(a)
    lib().oracle_filter_2d(_p(a), a.shape[1], a.shape[0], _p(t), (t.size - 1) // 2, _p(out))
    return out


def scale_space(img: np.ndarray, p) -> list:
    """levels[o][k] as 2-D float64 arrays."""
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    n = lib().oracle_levels_size(W, H, _p(p))
    buf = np.empty(n, np.float64)
    O = lib().oracle_scale_space(_p(img), W, H, W, _p(p), _p(buf))
    dims = octave_dims(W, H, p)
    K = int(p["scales_per_octave"][0])
    out, off = [], 0
    for o in range(O):
        w, h = dims[o]
        lv = []
        for k in range(K):
            lv.append(buf[off:off + w * h].reshape(h, w))
            off += w * h
        out.append(lv)
    return out


def laplacian(G: np.ndarray, s: float) -> np.ndarray:
    a = np.ascontiguousarray(G, np.float64)
    out = np.empty_like(a)
    lib().oracle_laplacian(_p(a), a.shape[1], a.shape[0], float(s), _p(out))
    return out


def alp_matrix(p) -> np.ndarray:
    K = int(p["scales_per_octave"][0])
    b = np.zeros(4 * K, np.float64)
    assert lib().oracle_alp_matrix(_p(p), _p(b)) == 0
    return b.reshape(4, K)


def alp_fit(beta: np.ndarray, Lk: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(beta, np.float64)
    L = np.ascontiguousarray(Lk, np.float64)
    a = np.zeros(4, np.float64)
    lib().oracle_alp_fit(_p(b), _p(L), L.size, _p(a))
    return a


def cubic(a, s):
    a = np.ascontiguousarray(a, np.float64)
    return lib().oracle_cubic(_p(a), float(s))


def alp_extremum(a, p):
    a = np.ascontiguousarray(a, np.float64)
    s = np.zeros(1)
    v = np.zeros(1)
    t = lib().oracle_alp_extremum(_p(a), _p(p), _p(s), _p(v))
    return t, float(s[0]), float(v[0])


def refine(q3x3, p):
    q = np.ascontiguousarray(np.asarray(q3x3, np.float64).reshape(9))
    out = np.zeros(4)
    ok = lib().oracle_refine(_p(q), _p(p), _p(out))
    return ok, out


def detect_levels(levels: np.ndarray, octave: int, p, cap: int = 100000) -> np.ndarray:
    """S2-S5 on given levels of one octave: levels (K, H, W) float64."""
    a = np.ascontiguousarray(levels, np.float64)
    out = np.zeros(cap, KP_DTYPE)
    n = lib().oracle_detect_levels(_p(a), a.shape[2], a.shape[1], int(octave), _p(p), _p(out), cap)
    assert n <= cap
    return out[:n].copy()


def dedupe(cands: np.ndarray, p) -> np.ndarray:
    c = np.ascontiguousarray(cands, KP_DTYPE)
    keep = np.zeros(max(1, c.size), np.uint8)
    lib().oracle_dedupe(_p(c), c.size, _p(p), _p(keep))
    return keep[:c.size].astype(bool)


def dedupe_select(cands: np.ndarray, p) -> np.ndarray:
    c = np.ascontiguousarray(cands, KP_DTYPE)
    order = np.zeros(max(1, c.size), np.int32)
    n = lib().oracle_dedupe_select(_p(c), c.size, _p(p), _p(order))
    return order[:n].copy()


def orientations(G, xo, yo, so, p):
    a = np.ascontiguousarray(G, np.float64)
    th = np.zeros(36)
    hist = np.zeros(36)
    n = lib().oracle_orientations(_p(a), a.shape[1], a.shape[0], float(xo), float(yo), float(so),
                                  _p(p), _p(th), _p(hist))
    return th[:n].copy(), hist


def descriptor(G, xo, yo, so, theta, p):
    a = np.ascontiguousarray(G, np.float64)
    d = np.zeros(128)
    lib().oracle_descriptor(_p(a), a.shape[1], a.shape[0], float(xo), float(yo), float(so),
                            float(theta), _p(p), _p(d))
    return d


def orientation_peaks(hist36, p):
    """The S9 peak rule alone on a given 36-bin histogram."""
    h = np.ascontiguousarray(hist36, np.float64).reshape(36)
    th = np.zeros(36)
    n = lib().oracle_orientation_peaks(_p(h), _p(p), _p(th))
    return th[:n].copy()


def descriptor_hist(G, xo, yo, so, theta, p):
    """The S10 votes alone: 128 unnormalised sums, shape (4, 4, 8) = (cy, cx, bin)."""
    a = np.ascontiguousarray(G, np.float64)
    d = np.zeros(128)
    lib().oracle_descriptor_hist(_p(a), a.shape[1], a.shape[0], float(xo), float(yo), float(so),
                                 float(theta), _p(p), _p(d))
    return d.reshape(4, 4, 8)


def desc_level(p, so):
    return lib().oracle_desc_level(_p(p), float(so))


def candidates(img: np.ndarray, p, cap: int = 200000) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    out = np.zeros(cap, KP_DTYPE)
    n = lib().oracle_candidates(_p(img), W, H, W, _p(p), _p(out), cap)
    assert n <= cap
    return out[:n].copy()


def extract(img: np.ndarray, p, cap: int = 4096):
    """(records, descriptors, n_candidates) of one image."""
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    kp = np.zeros(cap, KP_DTYPE)
    d = np.zeros((cap, 128), np.float64)
    nc = np.zeros(1, np.int32)
    n = lib().oracle_extract(_p(img), W, H, W, _p(p), _p(kp), _p(d), cap, _p(nc))
    assert n <= cap
    return kp[:n].copy(), d[:n].copy(), int(nc[0])


def describe(img: np.ndarray, pts: np.ndarray, p, cap: int = 8192):
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    pts = np.ascontiguousarray(pts, KP_DTYPE)
    kp = np.zeros(cap, KP_DTYPE)
    d = np.zeros((cap, 128), np.float64)
    n = lib().oracle_describe(_p(img), W, H, W, _p(p), _p(pts), pts.size, _p(kp), _p(d), cap)
    assert n <= cap
    return kp[:n].copy(), d[:n].copy()


def extract_batch(imgs, p, cap: int = 2048, n_threads: int = 0):
    """Image-parallel oracle over a list of 2-D uint8 arrays."""
    imgs = [np.ascontiguousarray(a, np.uint8) for a in imgs]
    n = len(imgs)
    ptrs = (C.c_void_p * n)(*[a.ctypes.data for a in imgs])
    W = np.array([a.shape[1] for a in imgs], np.int32)
    H = np.array([a.shape[0] for a in imgs], np.int32)
    kp = np.zeros(n * cap, KP_DTYPE)
    d = np.zeros((n * cap, 128), np.float64)
    counts = np.zeros(n, np.int32)
    lib().oracle_extract_batch(n, C.cast(ptrs, C.c_void_p), _p(W), _p(H), _p(W), _p(p), _p(kp),
                               _p(d), cap, _p(counts), n_threads)
    return kp.reshape(n, cap), d.reshape(n, cap, 128), counts


def num_threads() -> int:
    return lib().oracle_num_threads()


def transform(desc: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(desc, np.float64).reshape(128)
    v = np.zeros(128)
    lib().oracle_transform(_p(d), _p(v))
    return v


def ternary(v: np.ndarray, t_lo: np.ndarray, t_hi: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(v, np.float64).reshape(128)
    lo = np.ascontiguousarray(t_lo, np.float64)
    hi = np.ascontiguousarray(t_hi, np.float64)
    q = np.zeros(128, np.int8)
    lib().oracle_ternary(_p(v), _p(lo), _p(hi), _p(q))
    return q
