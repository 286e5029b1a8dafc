"""Writes ternary_thresholds.json: the stand-in for the ternary quantisation
thresholds of the CDVS descriptor compression (Sec. III-C learns them offline
from the distribution of each transformed element; the normative table is not
available).  For element j the two thresholds are the 1/3 and 2/3 quantiles of
v_j over the oracle's descriptors of seeded calibration images.

Calls only the oracle.  Run from the repository root:
    python tests/golden/make_ternary_thresholds.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402
from paper_1705_09776_gb300 import synth  # noqa: E402

SEED = 0xCA11B
N_IMAGES = 100


def compute():
    """The thresholds as written to ternary_thresholds.json."""
    p = O.params()
    imgs = [synth.blob_image(synth.image_seed(SEED, i)) for i in range(N_IMAGES)]
    kp, d, counts = O.extract_batch(imgs, p, cap=2048)
    V = []
    for b in range(N_IMAGES):
        for i in range(counts[b]):
            V.append(O.transform(d[b, i]))
    V = np.array(V)
    lo = np.quantile(V, 1.0 / 3.0, axis=0)
    hi = np.quantile(V, 2.0 / 3.0, axis=0)
    return {"source": "oracle descriptors of %d seeded 640x480 images, base seed 0x%X" % (N_IMAGES, SEED),
            "n_descriptors": int(V.shape[0]), "t_lo": lo.tolist(), "t_hi": hi.tolist()}


def main():
    out = compute()
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "ternary_thresholds.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote thresholds from", out["n_descriptors"], "descriptors")


if __name__ == "__main__":
    main()
