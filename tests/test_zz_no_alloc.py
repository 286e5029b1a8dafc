"""cdvs_dedupe_select_noalloc: the allocation-free selection entry point.

Some callers cannot call cudaMalloc -- code that runs within a device-memory
budget fixed at start-up, or code that must not allocate while other threads
capture CUDA graphs.  For them the library offers one entry point whose
scratch lives in a fixed array inside the library.  This file checks, through
the C ABI, that it selects exactly what cdvs_dedupe_select selects, on two
calls in a row (the second call must not see the first call's leftovers), and
that it refuses more candidates than its array holds.  It is collected last,
so a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1705_09776_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1705_09776_gb300 import cdvs
    torch.cuda.init()
    return cdvs, cdvs.Context(0), torch


def _noalloc(cdvs, torch, cands, shape, p, with_status=False):
    N = int(p["max_keypoints"][0])
    rec = cdvs.KEYPOINT_DTYPE.itemsize
    d_in = torch.from_numpy(np.ascontiguousarray(cands).view(np.uint8).copy()).cuda()
    d_out = torch.zeros(N * rec, dtype=torch.uint8, device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = cdvs.dedupe_select_noalloc(d_in if len(cands) else None, len(cands), shape[1], shape[0], p, d_out, d_cnt,
                                    torch.cuda.current_stream(), d_st)
    torch.cuda.synchronize()
    n = int(d_cnt.cpu().item())
    out = d_out.cpu().numpy()[:n * rec].view(cdvs.KEYPOINT_DTYPE)
    if with_status:
        return st, out, int(d_st.cpu().item())
    return st, out


def test_noalloc_matches_dedupe_select_twice(env):
    cdvs, ctx, torch = env
    p = cdvs.params()
    for seed in (11, 12):   # two calls in a row, different images
        img = synth.blob_image(synth.image_seed(seed, 0))
        cands, cnt, st = ctx.candidates([img])
        assert st == cdvs.CDVS_OK and 300 < len(cands) < cdvs.NOALLOC_MAX_CANDIDATES
        ref, rc, st = ctx.dedupe_select([img.shape], [cands], p)
        assert st == cdvs.CDVS_OK
        st, got, dst = _noalloc(cdvs, torch, cands, img.shape, p, with_status=True)
        assert st == cdvs.CDVS_OK and dst == cdvs.CDVS_OK
        assert len(got) == rc[0] == 300
        assert np.array_equal(got["parent_id"], ref["parent_id"])
        assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))


def test_noalloc_limits(env):
    cdvs, ctx, torch = env
    p = cdvs.params()
    too_many = np.zeros(cdvs.NOALLOC_MAX_CANDIDATES + 1, cdvs.KEYPOINT_DTYPE)
    st, _ = _noalloc(cdvs, torch, too_many, (480, 640), p)
    assert st == cdvs.CDVS_UNSUPPORTED_SIZE
    # an empty list selects nothing
    st, got = _noalloc(cdvs, torch, np.zeros(0, cdvs.KEYPOINT_DTYPE), (480, 640), p)
    assert st == cdvs.CDVS_OK and len(got) == 0


def test_noalloc_records_out_of_range_are_left_out_and_reported(env):
    """A record whose octave is not one of the image's octaves is left out,
    the device status word says CDVS_INVALID_ARGUMENT, and the others are
    selected as cdvs_dedupe_select selects them."""
    cdvs, ctx, torch = env
    p = cdvs.params()
    img = synth.blob_image(synth.image_seed(13, 0))
    cands, cnt, st = ctx.candidates([img])
    bad = cands.copy()
    bad["octave"][3] = 4           # a 640 x 480 image has octaves 0..3
    bad["octave"][7] = -2
    keep = np.ones(len(bad), bool)
    keep[[3, 7]] = False
    ref, rc, st = ctx.dedupe_select([img.shape], [cands[keep]], p)
    st, got, dst = _noalloc(cdvs, torch, bad, img.shape, p, with_status=True)
    assert st == cdvs.CDVS_OK and dst == cdvs.CDVS_INVALID_ARGUMENT
    idx = np.nonzero(keep)[0]
    assert np.array_equal(got["parent_id"], idx[ref["parent_id"]])


def test_noalloc_ties_beyond_the_list(env):
    """5000 equal responses and N = 2048: the tie list (4096 entries) cannot
    hold them all, and the selection is still exact and complete."""
    cdvs, ctx, torch = env
    rng = np.random.default_rng(31)
    n = 5000
    rec = np.zeros(n, cdvs.KEYPOINT_DTYPE)
    rec["x"] = rng.integers(1, 639, n) + rng.uniform(-0.5, 0.5, n)
    rec["y"] = rng.integers(1, 479, n) + rng.uniform(-0.5, 0.5, n)
    rec["sigma"] = 1.6 * 2 ** rng.uniform(0, 1, n)
    rec["response"] = 10.0
    p = cdvs.params(max_keypoints=2048)
    ref, rc, st = ctx.dedupe_select([(480, 640)], [rec], p)
    assert st == cdvs.CDVS_OK and rc[0] == 2048
    st, got, dst = _noalloc(cdvs, torch, rec, (480, 640), p, with_status=True)
    assert st == cdvs.CDVS_OK and dst == cdvs.CDVS_OK
    assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))
