"""What a perfect block proposal would skip (CPU, run by hand):

    python tests/proposal_ceiling.py [n_images] [n_workloads]

For 640 x 480 blob images of several densities and noise levels, the blocks
holding a first-octave record of the FP64 oracle's extraction (the records a
mask must keep, by exact identity) are proposed and every other block is not.
The first-octave tiles then take their modes by the library's rule (bench.py's
tile_modes: detect near a proposed block, keep the levels within the
descriptor reach of a detecting tile, else level 3 only).  Prints the share of
tiles per mode; the share not detecting is the most any mask can take out of
detection on that workload.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1705_09776_gb300 import cdvs, synth  # noqa: E402

WORKLOADS = [(200, 4.0), (60, 4.0), (20, 4.0), (20, 1.0), (6, 1.0)]   # (blobs, noise std)


def main():
    n_images = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    workloads = WORKLOADS[:int(sys.argv[2])] if len(sys.argv) > 2 else WORKLOADS
    p = cdvs.params()
    reach = max(float(p["desc_radius"][0]), float(p["ori_radius"][0])) * 2 * float(p["sigma0"][0]) * 1.001 + 2
    P = O.params()
    for n_blobs, noise in workloads:
        counts = np.zeros(3, np.int64)
        for i in range(n_images):
            img = synth.blob_image(synth.image_seed(900 + n_blobs, i), n_blobs=n_blobs, noise_std=noise)
            kp, _, _ = O.extract(img, P)
            k0 = kp[kp["octave"] == 0]
            z = -np.ones((30, 40))
            for x, y in zip(k0["x"], k0["y"]):
                z[min(int(np.floor(y + 0.5)) // 16, 29), min(int(np.floor(x + 0.5)) // 16, 39)] = 1.0
            counts += bench.tile_modes([z], 0.0, 480, 640, reach)
        share = counts / counts.sum()
        print(f"{n_blobs:3d} blobs, noise {noise}: detect {share[2]:.3f}, levels only {share[1]:.3f}, "
              f"level 3 only {share[0]:.3f}; out of detection {1 - share[2]:.3f}")


if __name__ == "__main__":
    main()
