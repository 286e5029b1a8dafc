"""Writes scfv_model.npz: the stand-in for the SCFV aggregation model of the
CDVS global descriptor (Sec. III-D: a PCA from 128 to 32 dimensions and a
512-component diagonal GMM; the normative matrices are not available).

* PCA: mean and the 32 leading eigenvectors (rows, unit length, sign fixed
  so the largest component is positive) of the covariance of the oracle's
  descriptors of seeded calibration images;
* GMM: 512 components, uniform weights, means = 512 PCA-projected
  descriptors drawn with a seeded permutation, diagonal variances = a quarter
  of the per-dimension variance of the projected data.

Calls only the oracle.  Run from the repository root:
    python tests/golden/make_scfv_model.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402
from paper_1705_09776_gb300 import synth  # noqa: E402

SEED = 0x5CF7
N_IMAGES = 48
N_COMP, DIM = 512, 32


def compute():
    """The model's arrays, as written to scfv_model.npz (without the source note)."""
    imgs = [synth.blob_image(synth.image_seed(SEED, i)) for i in range(N_IMAGES)]
    kp, d, counts = O.extract_batch(imgs, O.params(), cap=2048)
    X = np.concatenate([d[b, :counts[b]] for b in range(N_IMAGES)])
    mean = X.mean(axis=0)
    cov = np.cov((X - mean).T)
    vals, vecs = np.linalg.eigh(cov)
    P = vecs[:, ::-1][:, :DIM].T.copy()                       # 32 x 128, leading first
    P *= np.sign(P[np.arange(DIM), np.abs(P).argmax(axis=1)])[:, None]
    Y = (X - mean) @ P.T
    perm = np.random.default_rng(SEED).permutation(len(Y))[:N_COMP]
    means = Y[perm]
    var = np.tile(Y.var(axis=0) / 4.0, (N_COMP, 1))
    w = np.full(N_COMP, 1.0 / N_COMP)
    return dict(pca_mean=mean.astype(np.float32), pca=P.astype(np.float32), weights=w.astype(np.float32),
                means=means.astype(np.float32), variances=var.astype(np.float32)), len(X)


def main():
    model, n = compute()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scfv_model.npz")
    np.savez(out, **model, source=np.array(f"oracle descriptors of {N_IMAGES} seeded 640x480 images, "
                                           f"seed 0x{SEED:X}, {n} records"))
    print("wrote", out, "from", n, "descriptors")


if __name__ == "__main__":
    main()
