"""Python binding of the CDVS C ABI (include/cdvs.h) -- argument marshalling only.

Every step of the method runs in libcdvs.so's CUDA kernels.  Importing this
module loads the library and raises if it is missing: there is no CPU
fallback.  Host arrays are numpy; device buffers are torch CUDA tensors (torch
is used only for device memory and streams).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

CDVS_OK = 0
CDVS_INVALID_ARGUMENT = 1
CDVS_UNSUPPORTED_SIZE = 2
CDVS_OUT_OF_MEMORY = 3
CDVS_CAPACITY_TRUNCATED = 4
CDVS_DEVICE_TIMEOUT = 5
CDVS_CUDA_ERROR = 6
STATUS_NAMES = {0: "OK", 1: "INVALID_ARGUMENT", 2: "UNSUPPORTED_SIZE", 3: "OUT_OF_MEMORY",
                4: "CAPACITY_TRUNCATED", 5: "DEVICE_TIMEOUT", 6: "CUDA_ERROR"}

CDVS_INPUT_DEVICE = 0x1
CDVS_OUTPUT_DEVICE = 0x2
CDVS_ASYNC = 0x4
CDVS_STORAGE_FP32 = 0
CDVS_STORAGE_FP16 = 1

PARAMS_DTYPE = np.dtype([
    ("num_octaves", "<i4"), ("scales_per_octave", "<i4"),
    ("sigma0", "<f4"), ("sigma_in", "<f4"), ("contrast_T", "<f4"), ("edge_r", "<f4"),
    ("offset_max", "<f4"), ("ori_radius", "<f4"), ("ori_peak_ratio", "<f4"),
    ("ori_weight_sigma", "<f4"), ("desc_radius", "<f4"), ("cell_side", "<f4"),
    ("desc_weight_sigma", "<f4"), ("dedupe_dlog2", "<f4"),
    ("max_keypoints", "<i4"), ("max_orientations", "<i4"), ("upright", "<i4"), ("storage", "<i4"),
    ("use_proposal", "<i4"), ("proposal_threshold", "<f4"), ("max_side", "<i4"),
])
KEYPOINT_DTYPE = np.dtype([
    ("x", "<f4"), ("y", "<f4"), ("sigma", "<f4"), ("theta", "<f4"), ("response", "<f4"),
    ("p_ss", "<f4"), ("ratio", "<f4"), ("octave", "<i2"), ("scale_idx", "<i2"), ("type", "<i2"),
    ("reserved", "<i2"), ("image", "<i4"), ("parent_id", "<i4"),
])
IMAGE_DESC_DTYPE = np.dtype([("width", "<i4"), ("height", "<i4"), ("pitch_bytes", "<i4")])
assert PARAMS_DTYPE.itemsize == 84 and KEYPOINT_DTYPE.itemsize == 44
PROPOSAL_PARAMS = 4817
PROPOSAL_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_weights.npz")


def load_proposal_weights(path=None, highres=False):
    """(theta, threshold) of a trained block proposal (train_proposal.py): the
    threshold chosen on 640 x 480 images, or with highres=True the one chosen
    on images with the high-resolution workload's statistics."""
    d = np.load(path or PROPOSAL_WEIGHTS)
    key = "threshold_zoom" if highres and "threshold_zoom" in d else "threshold"
    return d["theta"].astype(np.float32), float(d[key])

EXPORTED = ["cdvs_params_default", "cdvs_create", "cdvs_destroy", "cdvs_last_error", "cdvs_extract",
            "cdvs_candidates", "cdvs_dedupe_select", "cdvs_describe", "cdvs_scale_space",
            "cdvs_rank_host", "cdvs_transform_ternary", "cdvs_profile", "cdvs_profile_read", "cdvs_wait",
            "cdvs_dedupe_select_noalloc", "cdvs_set_proposal", "cdvs_proposal_logits",
            "cdvs_proposal_train_step", "cdvs_resize", "cdvs_set_graph", "cdvs_set_scfv_model", "cdvs_scfv",
            "cdvs_inject_alloc_failures", "cdvs_set_candidate_capacity", "cdvs_set_detect_variant",
            "cdvs_detect_tuning", "cdvs_probe_fp32_rate", "cdvs_inject_scfv_wait_timeouts"]
STAGES = ["detect", "select", "describe", "offsets", "pack", "detect_octave0", "proposal"]


class CdvsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(build_if_missing: bool = True):
    """Loads libcdvs.so (building it first if allowed).  Raises when it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB_PATH):
        raise ImportError(f"CDVS CUDA library not built: {_build.LIB_PATH} is missing")
    L = C.CDLL(_build.LIB_PATH)
    P, i32, u32, sz = C.c_void_p, C.c_int32, C.c_uint32, C.c_size_t
    sig = {
        "cdvs_params_default": (None, [P]),
        "cdvs_create": (i32, [P, C.c_int, sz]),
        "cdvs_destroy": (None, [P]),
        "cdvs_last_error": (C.c_char_p, [P]),
        "cdvs_extract": (i32, [P, i32, P, P, P, P, P, i32, P, u32, P]),
        "cdvs_candidates": (i32, [P, i32, P, P, P, P, i32, P, u32, P]),
        "cdvs_dedupe_select": (i32, [P, i32, P, P, P, i32, P, P, i32, P, u32, P]),
        "cdvs_describe": (i32, [P, i32, P, P, P, P, P, i32, P, P, i32, P, u32, P]),
        "cdvs_scale_space": (i32, [P, P, P, P, P, sz, P, u32, P]),
        "cdvs_rank_host": (i32, [P, i32, i32, P]),
        "cdvs_transform_ternary": (i32, [P, i32, P, P, P, P]),
        "cdvs_profile": (i32, [P, i32]),
        "cdvs_wait": (i32, [P, P]),
        "cdvs_profile_read": (i32, [P, P, P, i32, i32]),
        "cdvs_dedupe_select_noalloc": (i32, [P, i32, i32, i32, P, P, P, P, P]),
        "cdvs_set_proposal": (i32, [P, P, i32]),
        "cdvs_resize": (i32, [P, i32, P, P, i32, P, sz, P, u32, P]),
        "cdvs_set_graph": (i32, [P, i32]),
        "cdvs_set_scfv_model": (i32, [P, P]),
        "cdvs_scfv": (i32, [P, i32, P, P, i32, P, P, P, P, P, u32, P]),
        "cdvs_proposal_logits": (i32, [P, i32, P, P, P, i32, u32, P]),
        "cdvs_proposal_train_step": (i32, [P, P, i32, i32, i32, i32, P, P, P, P, P, P, P, i32, C.c_float, i32, P]),
        "cdvs_inject_alloc_failures": (None, [i32]),
        "cdvs_set_candidate_capacity": (i32, [P, i32]),
        "cdvs_set_detect_variant": (i32, [P, i32]),
        "cdvs_detect_tuning": (i32, [P, P, i32]),
        "cdvs_probe_fp32_rate": (i32, [P, P]),
        "cdvs_inject_scfv_wait_timeouts": (None, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a) -> int:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def params(**kw) -> np.ndarray:
    """cdvs_params with the library defaults and the given overrides (1-element array)."""
    p = np.zeros(1, PARAMS_DTYPE)
    load().cdvs_params_default(p.ctypes.data)
    for k, v in kw.items():
        p[k] = v
    return p


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Context:
    """A cdvs_ctx on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self._L = load()
        h = C.c_void_p()
        st = self._L.cdvs_create(C.byref(h), device, workspace_bytes)
        if st != CDVS_OK:
            raise CdvsError(st, f"cdvs_create(device={device}) failed")
        self.handle = h.value
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self._L.cdvs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._L.cdvs_last_error(self.handle).decode()

    def _check(self, st, allow_truncated=True):
        if st == CDVS_OK or (allow_truncated and st == CDVS_CAPACITY_TRUNCATED):
            return st
        raise CdvsError(st, self.last_error())

    def wait(self, stream=None):
        """cdvs_wait: synchronises the stream of CDVS_ASYNC extractions and
        returns their combined status (raises on errors other than truncation)."""
        return self._check(self._L.cdvs_wait(self.handle, _stream_handle(stream)))

    def set_candidate_capacity(self, per_image: int):
        """cdvs_set_candidate_capacity: 0 = from the image size."""
        self._check(self._L.cdvs_set_candidate_capacity(self.handle, int(per_image)))

    def set_detect_variant(self, variant: int):
        """cdvs_set_detect_variant: -1 = tuned (default), 0..3 = a fixed work shape."""
        self._check(self._L.cdvs_set_detect_variant(self.handle, int(variant)))

    def detect_tuning(self) -> dict:
        """cdvs_detect_tuning as a dict."""
        import json
        n = self._L.cdvs_detect_tuning(self.handle, None, 0)
        buf = C.create_string_buffer(n + 1)
        self._L.cdvs_detect_tuning(self.handle, buf, n + 1)
        return json.loads(buf.value.decode())

    def probe_fp32_rate(self) -> float:
        """cdvs_probe_fp32_rate: the measured packed-FP32 FMA rate, TFLOP/s."""
        v = C.c_double(0.0)
        self._check(self._L.cdvs_probe_fp32_rate(self.handle, C.byref(v)))
        return float(v.value)

    def set_graph(self, enable: bool):
        """Device-resident extractions through one CUDA graph (cdvs_set_graph)."""
        self._check(self._L.cdvs_set_graph(self.handle, 1 if enable else 0))

    # ------------------------------------------------------------ SCFV
    def set_scfv_model(self, model):
        """model: mapping with pca_mean (128), pca (32 x 128), weights (512),
        means (512 x 32), variances (512 x 32)."""
        arrs = [np.ascontiguousarray(model[k], np.float32) for k in
                ("pca_mean", "pca", "weights", "means", "variances")]
        st = (C.c_void_p * 5)(*[a.ctypes.data for a in arrs])
        self._check(self._L.cdvs_set_scfv_model(self.handle, C.cast(st, C.c_void_p)))

    def scfv(self, desc, counts, n_select=64):
        """Host SCFV of a batch: desc (sum(counts) x 128 float32, image order),
        counts per image.  Returns g_mu, g_sigma (n x 512 x 32), delta (n x
        512), order (n x 512) and bits (n x n_select uint32)."""
        d = np.ascontiguousarray(desc, np.float32)
        cnt = np.ascontiguousarray(counts, np.int32)
        n = len(cnt)
        g_mu = np.zeros((n, 512, 32), np.float32)
        g_sig = np.zeros((n, 512, 32), np.float32)
        delta = np.zeros((n, 512), np.float32)
        order = np.zeros((n, 512), np.int32)
        bits = np.zeros((n, max(n_select, 1)), np.uint32)
        self._check(self._L.cdvs_scfv(self.handle, n, d.ctypes.data, cnt.ctypes.data, int(n_select),
                                      g_mu.ctypes.data, g_sig.ctypes.data, delta.ctypes.data, order.ctypes.data,
                                      bits.ctypes.data, 0, None))
        return g_mu, g_sig, delta, order, bits[:, :n_select]

    # ------------------------------------------------------------ S0
    def resize(self, images, max_side):
        """cdvs_resize on host images: the list of resized uint8 arrays."""
        imgs, sizes, ptrs = self._host_images(images)
        out_sizes = np.zeros(len(imgs), IMAGE_DESC_DTYPE)
        cap = sum(a.size for a in imgs) + 16
        out = np.zeros(cap, np.uint8)
        self._check(self._L.cdvs_resize(self.handle, len(imgs), C.cast(ptrs, C.c_void_p), sizes.ctypes.data,
                                        int(max_side), out.ctypes.data, cap, out_sizes.ctypes.data, 0, None))
        res, o = [], 0
        for d in out_sizes:
            w, h = int(d["width"]), int(d["height"])
            res.append(out[o:o + w * h].reshape(h, w).copy())
            o += w * h
        return res

    # ------------------------------------------------------------ proposal
    def set_proposal(self, theta):
        """Network parameters (PROPOSAL_PARAMS floats) for use_proposal = 1."""
        t = np.ascontiguousarray(theta, np.float32)
        self._check(self._L.cdvs_set_proposal(self.handle, t.ctypes.data, int(t.size)))

    def proposal_logits(self, images):
        """Logits of the 16x16 blocks of each image: a list of (ceil(H/16), ceil(W/16)) arrays."""
        imgs, sizes, ptrs = self._host_images(images)
        shapes = [(-(-a.shape[0] // 16), -(-a.shape[1] // 16)) for a in imgs]
        out = np.zeros(sum(h * w for h, w in shapes), np.float32)
        self._check(self._L.cdvs_proposal_logits(self.handle, len(imgs), C.cast(ptrs, C.c_void_p), sizes.ctypes.data,
                                                 out.ctypes.data, out.size, 0, None))
        res, o = [], 0
        for h, w in shapes:
            res.append(out[o:o + h * w].reshape(h, w))
            o += h * w
        return res

    def proposal_train_step(self, images, labels, theta, adam_m, adam_v, grad, loss=None, logits=None,
                            step=1, lr=0.0, bf16=True, stream=None):
        """One training step on device tensors: images (B, H, W) uint8, labels
        (B, ceil(H/16), ceil(W/16)) float32 or None; theta, adam_m, adam_v,
        grad: PROPOSAL_PARAMS float32; loss: 1 float32; logits like labels."""
        B, H, W = images.shape
        st = self._L.cdvs_proposal_train_step(self.handle, _ptr(images), B, W, H, W, _ptr(labels), _ptr(theta),
                                              _ptr(adam_m), _ptr(adam_v), _ptr(grad), _ptr(loss), _ptr(logits),
                                              int(step), float(lr), 1 if bf16 else 0, _stream_handle(stream))
        return self._check(st)

    # ------------------------------------------------------------ measurement
    def profile(self, enable: bool):
        self._check(self._L.cdvs_profile(self.handle, 1 if enable else 0))

    def profile_read(self, reset: bool = True):
        """{stage: (ms, launches)} accumulated since the last reset."""
        ms = np.zeros(len(STAGES), np.float64)
        nl = np.zeros(len(STAGES), np.int32)
        n = self._L.cdvs_profile_read(self.handle, ms.ctypes.data, nl.ctypes.data, len(STAGES), 1 if reset else 0)
        if n < 0:
            raise CdvsError(CDVS_CUDA_ERROR, "cdvs_profile_read")
        return {s: (float(ms[i]), int(nl[i])) for i, s in enumerate(STAGES)}

    # ------------------------------------------------------------ host batches
    @staticmethod
    def _host_images(images):
        imgs = [np.ascontiguousarray(a, np.uint8) for a in images]
        sizes = np.zeros(len(imgs), IMAGE_DESC_DTYPE)
        for i, a in enumerate(imgs):
            sizes[i] = (a.shape[1], a.shape[0], a.strides[0])
        ptrs = (C.c_void_p * len(imgs))(*[a.ctypes.data for a in imgs])
        return imgs, sizes, ptrs

    def extract(self, images, p=None, capacity=None, stream=None, flags=0):
        """cdvs_extract on a list of 2-D uint8 numpy arrays.  Returns (records,
        descriptors (n x 128 float32), per-image counts, status)."""
        p = params() if p is None else p
        imgs, sizes, ptrs = self._host_images(images)
        n = len(imgs)
        if capacity is None:
            capacity = n * int(p["max_keypoints"][0]) * int(p["max_orientations"][0])
        kp = np.zeros(capacity, KEYPOINT_DTYPE)
        desc = np.zeros((capacity, 128), np.float32)
        cnt = np.zeros(n, np.int32)
        st = self._L.cdvs_extract(self.handle, n, C.cast(ptrs, C.c_void_p), sizes.ctypes.data, p.ctypes.data,
                                  kp.ctypes.data, desc.ctypes.data, capacity, cnt.ctypes.data, flags,
                                  _stream_handle(stream))
        self._check(st)
        tot = int(cnt.sum())
        return kp[:tot].copy(), desc[:tot].copy(), cnt, st

    def extract_raw(self, n, image_ptrs, sizes, p, kp_out, desc_out, capacity, counts, flags, stream=None):
        """cdvs_extract with caller-provided pointers (ints) -- no copies here.
        With CDVS_ASYNC in flags the call returns once the batch is enqueued;
        wait() completes the outstanding calls and returns their status."""
        ptrs = (C.c_void_p * n)(*image_ptrs)
        st = self._L.cdvs_extract(self.handle, n, C.cast(ptrs, C.c_void_p), _ptr(sizes), _ptr(p), _ptr(kp_out),
                                  _ptr(desc_out), capacity, _ptr(counts), flags, _stream_handle(stream))
        return self._check(st)

    def candidates(self, images, p=None, capacity=None):
        p = params() if p is None else p
        imgs, sizes, ptrs = self._host_images(images)
        n = len(imgs)
        if capacity is None:
            capacity = sum(a.size // 4 for a in imgs) + 4096
        kp = np.zeros(capacity, KEYPOINT_DTYPE)
        cnt = np.zeros(n, np.int32)
        st = self._L.cdvs_candidates(self.handle, n, C.cast(ptrs, C.c_void_p), sizes.ctypes.data, p.ctypes.data,
                                     kp.ctypes.data, capacity, cnt.ctypes.data, 0, None)
        self._check(st)
        return kp[:int(cnt.sum())].copy(), cnt, st

    def dedupe_select(self, shapes, cand_lists, p=None):
        """shapes: [(H, W)]; cand_lists: one KEYPOINT_DTYPE array per image."""
        p = params() if p is None else p
        n = len(shapes)
        sizes = np.zeros(n, IMAGE_DESC_DTYPE)
        for i, (h, w) in enumerate(shapes):
            sizes[i] = (w, h, w)
        stride = max(1, max(len(c) for c in cand_lists))
        cand = np.zeros(n * stride, KEYPOINT_DTYPE)
        cnt = np.zeros(n, np.int32)
        for i, c in enumerate(cand_lists):
            cand[i * stride:i * stride + len(c)] = c
            cnt[i] = len(c)
        cap = n * int(p["max_keypoints"][0])
        out = np.zeros(cap, KEYPOINT_DTYPE)
        oc = np.zeros(n, np.int32)
        st = self._L.cdvs_dedupe_select(self.handle, n, sizes.ctypes.data, cand.ctypes.data, cnt.ctypes.data,
                                        stride, p.ctypes.data, out.ctypes.data, cap, oc.ctypes.data, 0, None)
        self._check(st)
        return out[:int(oc.sum())].copy(), oc, st

    def describe(self, images, point_lists, p=None, capacity=None):
        p = params() if p is None else p
        imgs, sizes, ptrs = self._host_images(images)
        n = len(imgs)
        stride = max(1, max(len(c) for c in point_lists))
        pts = np.zeros(n * stride, KEYPOINT_DTYPE)
        npts = np.zeros(n, np.int32)
        for i, c in enumerate(point_lists):
            pts[i * stride:i * stride + len(c)] = c
            npts[i] = len(c)
        if capacity is None:
            capacity = int(npts.sum()) * int(p["max_orientations"][0]) + 1
        kp = np.zeros(capacity, KEYPOINT_DTYPE)
        desc = np.zeros((capacity, 128), np.float32)
        cnt = np.zeros(n, np.int32)
        st = self._L.cdvs_describe(self.handle, n, C.cast(ptrs, C.c_void_p), sizes.ctypes.data, p.ctypes.data,
                                   pts.ctypes.data, npts.ctypes.data, stride, kp.ctypes.data, desc.ctypes.data,
                                   capacity, cnt.ctypes.data, 0, None)
        self._check(st)
        tot = int(cnt.sum())
        return kp[:tot].copy(), desc[:tot].copy(), cnt, st

    def scale_space(self, image, p=None):
        """Gaussian levels of one image minus 128: levels[o][k] (float32 2-D arrays)."""
        p = params() if p is None else p
        img = np.ascontiguousarray(image, np.uint8)
        size = np.array([(img.shape[1], img.shape[0], img.strides[0])], IMAGE_DESC_DTYPE)
        cap = 4 * img.size * 2 + 1024
        out = np.zeros(cap, np.float32)
        no = np.zeros(1, np.int32)
        st = self._L.cdvs_scale_space(self.handle, img.ctypes.data, size.ctypes.data, p.ctypes.data,
                                      out.ctypes.data, cap, no.ctypes.data, 0, None)
        self._check(st, allow_truncated=False)
        levels, off = [], 0
        w, h = img.shape[1], img.shape[0]
        for o in range(int(no[0])):
            lv = []
            for k in range(4):
                lv.append(out[off:off + w * h].reshape(h, w).copy())
                off += w * h
            levels.append(lv)
            w, h = (w + 1) // 2, (h + 1) // 2
        return levels


NOALLOC_MAX_CANDIDATES = 16384


def dedupe_select_noalloc(cand_dev, n_cand, width, height, p, sel_out_dev, sel_count_dev, stream=None,
                          status_dev=None) -> int:
    """cdvs_dedupe_select_noalloc on device buffers (torch tensors or device
    addresses as ints): no memory is allocated by the library.  Returns the
    call's status code (asynchronous: outputs, and the device status word
    when given, are ready once `stream` is)."""
    def addr(x):
        return x if isinstance(x, int) or x is None else x.data_ptr()
    return load().cdvs_dedupe_select_noalloc(addr(cand_dev), n_cand, width, height, p.ctypes.data,
                                             addr(sel_out_dev), addr(sel_count_dev), addr(status_dev),
                                             _stream_handle(stream))


def inject_alloc_failures(count: int) -> None:
    """Testing hook: the next `count` workspace allocations fail as if the
    device were out of memory."""
    load().cdvs_inject_alloc_failures(int(count))


def inject_scfv_wait_timeouts(count: int) -> None:
    """Testing hook: the next `count` SCFV calls leave their tensor-core
    products unissued, so the bounded wait in the posterior kernel runs out."""
    load().cdvs_inject_scfv_wait_timeouts(int(count))


def rank_host(pts: np.ndarray, max_keypoints: int) -> np.ndarray:
    pts = np.ascontiguousarray(pts, KEYPOINT_DTYPE)
    order = np.zeros(max(1, pts.size), np.int32)
    m = load().cdvs_rank_host(pts.ctypes.data, pts.size, max_keypoints, order.ctypes.data)
    return order[:m].copy()


def transform_ternary(desc: np.ndarray, t_lo: np.ndarray, t_hi: np.ndarray):
    d = np.ascontiguousarray(desc, np.float32).reshape(-1, 128)
    lo = np.ascontiguousarray(t_lo, np.float64)
    hi = np.ascontiguousarray(t_hi, np.float64)
    q = np.zeros(d.shape, np.int8)
    v = np.zeros(d.shape, np.float64)
    st = load().cdvs_transform_ternary(d.ctypes.data, d.shape[0], lo.ctypes.data, hi.ctypes.data,
                                       q.ctypes.data, v.ctypes.data)
    if st != CDVS_OK:
        raise CdvsError(st, "cdvs_transform_ternary")
    return q, v
