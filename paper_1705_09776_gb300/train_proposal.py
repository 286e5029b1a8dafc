"""Trains the learned block proposal on the GPU and writes its parameters.

    python -m paper_1705_09776_gb300.train_proposal [--train 16384] [--out PATH]

Labels come from the plain detector: a 16x16 block is positive when a
first-octave record of cdvs_extract (after the cross-octave check and the
selection, Sec. III-B) lies in it.  The images are the seeded synthetic
blob images (seeds 1000000 + i for training, 3000000 + i for choosing the
threshold).  A fraction of them (--zoom) carries the statistics of the
high-resolution workload at 640 x 480: the blobs 3.2 times larger and as
many per pixel as in a 2048 x 1536 image (200 / 10.24 of them), so one
network serves both scales.  Training runs the library's own forward,
backward and Adam kernels (cdvs_proposal_train_step, BF16 as in
inference).  Each kind of validation image gets its own threshold: the
largest of a fixed list whose masked extraction keeps at least `--keep` of
the plain detector's records on those images.  The
output .npz holds `theta` (FP32), `threshold` (640 x 480 images),
`threshold_zoom` (images with the high-resolution statistics) and the
training record.
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import synth

TRAIN_BASE, VAL_BASE = 1_000_000, 3_000_000
ZOOM_TRAIN_BASE, ZOOM_VAL_BASE = 5_000_000, 6_000_000
ZOOM = 3.2   # blob scale of the 2048 x 1536 workload against the 640 x 480 one
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "proposal_weights.npz")
THRESHOLDS = (0.5, 0.4, 0.3, 0.2, 0.15, 0.1, 0.07, 0.05, 0.03, 0.02, 0.01)


def _gen(args):
    base, i, zoom = args
    if zoom:
        # a 640 x 480 window of the high-resolution workload: blobs ZOOM times
        # larger, as many per pixel as there
        return synth.blob_image(synth.image_seed(base, i), n_blobs=int(round(200 / (ZOOM * ZOOM))),
                                sigma_range=(1.5 * ZOOM, 20.0 * ZOOM))
    return synth.blob_image(synth.image_seed(base, i))


def make_images(base: int, n: int, procs: int, zoom: bool = False) -> np.ndarray:
    """Seeded images, generated in a spawn pool (call before CUDA starts)."""
    import multiprocessing as mp
    if n == 0:
        return np.zeros((0, 480, 640), np.uint8)
    with mp.get_context("spawn").Pool(procs) as pool:
        return np.stack(pool.map(_gen, [(base, i, zoom) for i in range(n)], chunksize=16))


def block_labels(records, n_images: int, height: int, width: int) -> np.ndarray:
    """(n, ceil(H/16), ceil(W/16)) float32: 1 where a first-octave record lies."""
    th, tw = -(-height // 16), -(-width // 16)
    y = np.zeros((n_images, th, tw), np.float32)
    r = records[records["octave"] == 0]
    bx = np.clip(np.floor(r["x"] + 0.5).astype(np.int64) // 16, 0, tw - 1)
    by = np.clip(np.floor(r["y"] + 0.5).astype(np.int64) // 16, 0, th - 1)
    y[r["image"], by, bx] = 1.0
    return y


def record_keys(records) -> set:
    """Exact identity of records: image, octave and the bits of x, y, sigma, theta."""
    k = np.stack([records["image"], records["octave"], records["x"].view(np.int32), records["y"].view(np.int32),
                  records["sigma"].view(np.int32), records["theta"].view(np.int32)], 1)
    return set(map(tuple, k.tolist()))


def extract_batches(ctx, cdvs, images, p, batch=256):
    recs, counts = [], []
    for b0 in range(0, len(images), batch):
        k, _, c, _ = ctx.extract(list(images[b0:b0 + batch]), p)
        k = k.copy()
        k["image"] += b0
        recs.append(k)
        counts.append(c)
    return np.concatenate(recs), np.concatenate(counts)


def recall(plain_keys: set, masked) -> float:
    return len(plain_keys & record_keys(masked)) / max(len(plain_keys), 1)


def init_theta(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases except a negative head bias (positives are rare)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 9), 144), np.zeros(16), rng.normal(0, np.sqrt(2 / 144), 2304), np.zeros(16),
             rng.normal(0, np.sqrt(2 / 144), 2304), np.zeros(16), rng.normal(0, np.sqrt(1 / 16), 16), [-2.0]]
    return np.concatenate(parts).astype(np.float32)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=16384)
    ap.add_argument("--val", type=int, default=512)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--keep", type=float, default=0.995)
    ap.add_argument("--zoom", type=float, default=0.25,
                    help="fraction of training and validation images with the high-resolution statistics")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=DEFAULT_OUT)
    a = ap.parse_args(argv)
    t0 = time.time()
    nz, nzv = int(round(a.train * a.zoom)), int(round(a.val * a.zoom))
    train = np.concatenate([make_images(TRAIN_BASE, a.train - nz, a.procs),
                            make_images(ZOOM_TRAIN_BASE, nz, a.procs, zoom=True)])
    vals = [make_images(VAL_BASE, a.val - nzv, a.procs)]
    if nzv:
        vals.append(make_images(ZOOM_VAL_BASE, nzv, a.procs, zoom=True))
    t_gen = time.time() - t0

    import torch

    from . import cdvs
    ctx = cdvs.Context(0)
    H, W = train.shape[1:]
    plain = cdvs.params()
    rec, _ = extract_batches(ctx, cdvs, train, plain)
    labels = block_labels(rec, len(train), H, W)
    print(f"labels: {labels.mean():.4f} of blocks positive, {len(rec) / len(train):.1f} records/img", flush=True)

    dev_img = torch.from_numpy(train).cuda()
    dev_lab = torch.from_numpy(labels).cuda()
    theta = torch.from_numpy(init_theta()).cuda()
    m, v, g = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    steps_per_epoch = len(train) // a.batch
    total = steps_per_epoch * a.epochs
    order = np.random.default_rng(1).permutation(len(train))
    hist = []
    t1 = time.time()
    step = 0
    for ep in range(a.epochs):
        perm = np.roll(order, ep * 7919)
        for s in range(steps_per_epoch):
            step += 1
            lr = a.lr * 0.5 * (1 + np.cos(np.pi * (step - 1) / total))   # cosine decay
            idx = torch.from_numpy(np.sort(perm[s * a.batch:(s + 1) * a.batch])).cuda()
            bi = dev_img.index_select(0, idx).contiguous()
            bl = dev_lab.index_select(0, idx).contiguous()
            ctx.proposal_train_step(bi, bl, theta, m, v, g, loss, None, step=step, lr=lr, bf16=True)
            if step % 50 == 0 or step == total:
                hist.append((step, float(loss.item())))
                print(f"step {step}/{total} loss {hist[-1][1]:.4f}", flush=True)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    th = theta.cpu().numpy()

    # thresholds: per kind of validation image, the largest whose masked
    # extraction keeps `keep` of the plain detector's records
    ctx.set_proposal(th)
    vkeys = [record_keys(extract_batches(ctx, cdvs, v, plain)[0]) for v in vals]
    chosen = [None] * len(vals)
    table = []
    for t in THRESHOLDS:
        rs = [recall(k, extract_batches(ctx, cdvs, v, cdvs.params(use_proposal=1, proposal_threshold=t))[0])
              for k, v in zip(vkeys, vals)]
        table.append([t] + rs)
        print(f"threshold {t}: recall " + ", ".join(f"{r:.5f}" for r in rs), flush=True)
        for j, r in enumerate(rs):
            if chosen[j] is None and r >= a.keep:
                chosen[j] = t
        if all(c is not None for c in chosen):
            break
    chosen = [THRESHOLDS[-1] if c is None else c for c in chosen]
    np.savez(a.out, theta=th, threshold=np.float32(chosen[0]),
             threshold_zoom=np.float32(chosen[-1]), loss_history=np.array(hist, np.float64),
             recall_table=np.array(table, np.float64),
             config=np.array([a.train, a.val, a.batch, a.epochs, a.lr, a.keep, a.zoom], np.float64),
             seconds=np.array([t_gen, t_train], np.float64))
    print(f"wrote {a.out}: thresholds {chosen}, gen {t_gen:.1f} s, train {t_train:.1f} s", flush=True)


if __name__ == "__main__":
    main()
