"""Asynchronous extraction (CDVS_ASYNC + cdvs_wait) through the C ABI.

* batches enqueued back to back without host synchronisation -- more calls
  than the context has staging sets, different shapes, direct launches and
  the CUDA graph, device buffers or host buffers (page-locked or not) --
  give exactly the records of synchronous calls;
* the truncation of any call since the last cdvs_wait is reported by it, and
  only once;
* the flag's preconditions: cdvs_extract only, and no other call on the
  context while asynchronous calls are pending.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1705_09776_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1705_09776_gb300 import cdvs
    return cdvs, cdvs.Context(0)


def _batch(seed, n, w=640, h=480):
    return [synth.blob_image(synth.image_seed(seed, i), width=w, height=h,
                             n_blobs=max(8, int(200 * w * h / (640 * 480)))) for i in range(n)]


class _Dev:
    """One batch on the device with its own output buffers."""

    def __init__(self, cdvs, imgs, cap_per_image=1200):
        import torch
        self.n = len(imgs)
        flat = np.concatenate([im.ravel() for im in imgs])
        self.img = torch.from_numpy(flat).cuda()
        offs = np.cumsum([0] + [im.size for im in imgs])
        self.ptrs = [self.img.data_ptr() + int(o) for o in offs[:-1]]
        self.sizes = np.array([(im.shape[1], im.shape[0], im.shape[1]) for im in imgs], cdvs.IMAGE_DESC_DTYPE)
        self.cap = self.n * cap_per_image
        self.kp = torch.zeros(self.cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        self.desc = torch.zeros(self.cap, 128, dtype=torch.float32, device="cuda")
        self.cnt = torch.zeros(self.n, dtype=torch.int32, device="cuda")

    def run(self, cdvs, ctx, p, flags, stream):
        return ctx.extract_raw(self.n, self.ptrs, self.sizes, p, self.kp, self.desc, self.cap, self.cnt,
                               flags, stream)

    def result(self, cdvs):
        c = self.cnt.cpu().numpy()
        t = min(int(c.sum()), self.cap)
        return c, self.kp.cpu().numpy()[:t * cdvs.KEYPOINT_DTYPE.itemsize].copy(), self.desc.cpu().numpy()[:t].copy()


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("graph", [False, True])
def test_async_batches_equal_synchronous_calls(env, graph):
    import torch
    cdvs, ctx = env
    stream = torch.cuda.current_stream()
    dev = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE
    p = cdvs.params()
    batches = [_Dev(cdvs, _batch(71, 4)), _Dev(cdvs, _batch(72, 3, 320, 200)), _Dev(cdvs, _batch(73, 5)),
               _Dev(cdvs, _batch(74, 2, 333, 257)), _Dev(cdvs, _batch(75, 4))]
    ref = []
    for b in batches:
        b.run(cdvs, ctx, p, dev, stream)
        torch.cuda.synchronize()
        ref.append(b.result(cdvs))
        b.cnt.zero_()
        b.kp.zero_()
        b.desc.zero_()
    ctx.set_graph(graph)
    try:
        for b in batches:  # five calls in flight on two staging sets
            assert b.run(cdvs, ctx, p, dev | cdvs.CDVS_ASYNC, stream) == cdvs.CDVS_OK
        assert ctx.wait(stream) == cdvs.CDVS_OK
    finally:
        ctx.set_graph(False)
    for b, r in zip(batches, ref):
        assert _same(b.result(cdvs), r)


def test_async_truncation_is_reported_by_wait(env):
    import torch
    cdvs, ctx = env
    stream = torch.cuda.current_stream()
    dev = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE
    full = _Dev(cdvs, _batch(81, 3))
    small = _Dev(cdvs, _batch(81, 3), cap_per_image=20)
    p = cdvs.params()
    full.run(cdvs, ctx, p, dev | cdvs.CDVS_ASYNC, stream)
    small.run(cdvs, ctx, p, dev | cdvs.CDVS_ASYNC, stream)
    full.run(cdvs, ctx, p, dev | cdvs.CDVS_ASYNC, stream)
    assert ctx.wait(stream) == cdvs.CDVS_CAPACITY_TRUNCATED
    assert ctx.wait(stream) == cdvs.CDVS_OK  # reported once
    full.run(cdvs, ctx, p, dev | cdvs.CDVS_ASYNC, stream)
    assert ctx.wait(stream) == cdvs.CDVS_OK
    # the truncated call kept the first records of the batch
    c_full, kp_full, d_full = full.result(cdvs)
    c_small, kp_small, d_small = small.result(cdvs)
    assert c_small.sum() == small.cap
    assert np.array_equal(kp_small, kp_full[:len(kp_small)]) and np.array_equal(d_small, d_full[:len(d_small)])


def test_async_preconditions(env):
    import torch
    cdvs, ctx = env
    stream = torch.cuda.current_stream()
    dev = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE
    b = _Dev(cdvs, _batch(91, 2))
    p = cdvs.params()
    # cdvs_extract only
    img = np.zeros((64, 64), np.uint8)
    sz = np.array([(64, 64, 64)], cdvs.IMAGE_DESC_DTYPE)
    ptrs = (C.c_void_p * 1)(img.ctypes.data)
    kp = np.zeros(64, cdvs.KEYPOINT_DTYPE)
    cnt = np.zeros(1, np.int32)
    st = ctx._L.cdvs_candidates(ctx.handle, 1, C.cast(ptrs, C.c_void_p), sz.ctypes.data, p.ctypes.data,
                                kp.ctypes.data, 64, cnt.ctypes.data, cdvs.CDVS_ASYNC, None)
    assert st == cdvs.CDVS_INVALID_ARGUMENT
    # with calls pending, a synchronous call is refused until cdvs_wait
    b.run(cdvs, ctx, p, dev | cdvs.CDVS_ASYNC, stream)
    with pytest.raises(cdvs.CdvsError) as ei:
        b.run(cdvs, ctx, p, dev, stream)
    assert ei.value.status == cdvs.CDVS_INVALID_ARGUMENT
    with pytest.raises(cdvs.CdvsError):
        ctx.extract([np.zeros((64, 64), np.uint8)])
    assert ctx.wait(stream) == cdvs.CDVS_OK
    assert b.run(cdvs, ctx, p, dev, stream) == cdvs.CDVS_OK
    assert ctx.wait(stream) == cdvs.CDVS_OK  # nothing pending


@pytest.mark.parametrize("pinned", [True, False])
def test_async_host_buffers_equal_synchronous_calls(env, pinned):
    """Host images in, host records out: each call's records reach its own
    buffers after cdvs_wait, equal to a synchronous call's, while later
    batches were enqueued behind it."""
    import torch
    cdvs, ctx = env
    stream = torch.cuda.current_stream()
    batches = [_batch(101, 4), _batch(102, 3, 320, 200), _batch(103, 5), _batch(104, 2, 333, 257)]
    ref = [ctx.extract(b) for b in batches]

    def host(shape, dtype):
        t = torch.zeros(shape, dtype=dtype)
        return t.pin_memory() if pinned else t

    outs = []
    for b in batches:
        n = len(b)
        flat = host((sum(im.size for im in b),), torch.uint8)
        flat.numpy()[:] = np.concatenate([im.ravel() for im in b])
        offs = np.cumsum([0] + [im.size for im in b])
        ptrs = [flat.data_ptr() + int(o) for o in offs[:-1]]
        sizes = np.array([(im.shape[1], im.shape[0], im.shape[1]) for im in b], cdvs.IMAGE_DESC_DTYPE)
        cap = n * 1200
        kp = host((cap * cdvs.KEYPOINT_DTYPE.itemsize,), torch.uint8)
        desc = host((cap, 128), torch.float32)
        cnt = host((n,), torch.int32)
        assert ctx.extract_raw(n, ptrs, sizes, cdvs.params(), kp, desc, cap, cnt, cdvs.CDVS_ASYNC,
                               stream) == cdvs.CDVS_OK
        outs.append((flat, kp, desc, cnt))
    assert ctx.wait(stream) == cdvs.CDVS_OK
    for (flat, kp, desc, cnt), (rk, rd, rc, _) in zip(outs, ref):
        c = cnt.numpy()
        t = int(c.sum())
        assert np.array_equal(c, rc)
        assert np.array_equal(kp.numpy()[:t * cdvs.KEYPOINT_DTYPE.itemsize], rk.view(np.uint8).ravel())
        assert np.array_equal(desc.numpy()[:t], rd)


def test_async_mixed_host_and_device_outputs(env):
    """Host outputs, then device outputs, then host outputs again: the third
    call reuses the first call's staging set, so the first call's records
    must leave before the third call packs its own."""
    import torch
    cdvs, ctx = env
    stream = torch.cuda.current_stream()
    a, b, c = _batch(111, 3), _batch(112, 2, 320, 200), _batch(113, 4)
    ref = [ctx.extract(x) for x in (a, c)]
    dev_b = _Dev(cdvs, b)
    dev_b.run(cdvs, ctx, cdvs.params(), cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE, stream)
    torch.cuda.synchronize()
    ref_b = dev_b.result(cdvs)

    def host_call(imgs):
        n = len(imgs)
        flat = torch.from_numpy(np.concatenate([im.ravel() for im in imgs])).pin_memory()
        offs = np.cumsum([0] + [im.size for im in imgs])
        sizes = np.array([(im.shape[1], im.shape[0], im.shape[1]) for im in imgs], cdvs.IMAGE_DESC_DTYPE)
        cap = n * 1200
        kp = torch.zeros(cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        desc = torch.zeros(cap, 128, dtype=torch.float32).pin_memory()
        cnt = torch.zeros(n, dtype=torch.int32).pin_memory()
        ctx.extract_raw(n, [flat.data_ptr() + int(o) for o in offs[:-1]], sizes, cdvs.params(), kp, desc, cap,
                        cnt, cdvs.CDVS_ASYNC, stream)
        return flat, kp, desc, cnt

    out_a = host_call(a)
    dev_b.run(cdvs, ctx, cdvs.params(), cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE | cdvs.CDVS_ASYNC, stream)
    out_c = host_call(c)
    assert ctx.wait(stream) == cdvs.CDVS_OK
    assert _same(dev_b.result(cdvs), ref_b)
    for (flat, kp, desc, cnt), (rk, rd, rc, _) in zip((out_a, out_c), ref):
        t = int(cnt.numpy().sum())
        assert np.array_equal(cnt.numpy(), rc)
        assert np.array_equal(kp.numpy()[:t * cdvs.KEYPOINT_DTYPE.itemsize], rk.view(np.uint8).ravel())
        assert np.array_equal(desc.numpy()[:t], rd)
