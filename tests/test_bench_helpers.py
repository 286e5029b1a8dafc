"""CPU checks of the measurement helpers in bench.py: the algorithmic counts the
roofline divides by, the hash-keyed DRAM traffic record, and the first-octave
tile modes the learned leg reports.

The counts are pinned to a hand count of the method at 640 x 480: level
filters of radius ceil(4 tau) with tau = sqrt(s_k^2 - 0.5^2), s_k = 1.6 * 2^(k/3)
(radii 7, 8, 10, 13: 80 taps over the four levels, two passes, an FMA = 2
flops), a 5-point Laplacian scaled by s_k^2 (7 flops per level), the cubic fit
(4 coefficients x 4 samples x 2 = 32 flops) and the root test (25): 405 flops
per pixel; bytes = the 8-bit input + four FP32 levels + the FP32 decimated base.
"""
import json
import math

import numpy as np

import bench
from paper_1705_09776_gb300 import synth  # noqa: F401  (the package imports without a GPU)


def _params():
    p = np.zeros(1, [("sigma0", "<f4"), ("sigma_in", "<f4"), ("num_octaves", "<i4")])
    p["sigma0"], p["sigma_in"], p["num_octaves"] = 1.6, 0.5, 4
    return p


def test_detect_counts_octave0_by_hand():
    flops, byts = bench.detect_counts(_params(), 640, 480)
    radii = [math.ceil(4 * math.sqrt((1.6 * 2 ** (k / 3)) ** 2 - 0.25)) for k in range(4)]
    assert radii == [7, 8, 10, 13]
    assert flops[0] == 405 * 640 * 480
    assert byts[0] == 640 * 480 + 4 * 4 * 640 * 480 + 4 * 320 * 240
    # later octaves: base sigma0, level 0 is the identity (no taps), the base
    # is an FP32 level written by the previous octave
    assert len(flops) == 4 and flops[1] < flops[0] / 4 + 1
    assert byts[1] == 4 * 320 * 240 + 4 * 3 * 320 * 240 + 4 * 160 * 120
    assert byts[3] == 4 * 80 * 60 + 4 * 3 * 80 * 60  # the last octave writes no decimated base


def test_traffic_record_is_keyed_on_the_kernel_source(tmp_path, monkeypatch):
    rec = {"variants": {"2": {"dram_bytes_per_image_octave0": 4.6e6}}, "kernel_sha256": bench.kernel_sha()}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.load_traffic(2)["dram_bytes_per_image_octave0"] == 4.6e6
    assert bench.load_traffic(1) is None
    rec["kernel_sha256"] = "0" * 64  # taken on another kernel: no traffic figure
    f.write_text(json.dumps(rec))
    assert bench.load_traffic(2) is None


def test_committed_traffic_record_matches_the_sources():
    """The committed ncu figures were taken on the K1 sources in the tree."""
    assert all(bench.load_traffic(v) is not None for v in range(4))


def test_tile_modes_rule():
    """Detect where a block with logit above the threshold lies within one block
    of the tile; keep the levels of tiles within the descriptor reach of a
    detecting tile; the rest only feed the next octave."""
    H, W = 64, 256                      # 2 x 2 tiles of 128 x 32, 4 x 16 blocks
    logits = np.full((H // 16, W // 16), -10.0, np.float32)
    # counts = [next-octave base only, levels only, detect]
    assert bench.tile_modes([logits], 0.0, H, W, reach=0.0).tolist() == [4, 0, 0]
    logits[0, 0] = 10.0                 # block (0, 0): only tile (0, 0) is within one block
    assert bench.tile_modes([logits], 0.0, H, W, reach=0.0).tolist() == [3, 0, 1]
    # a reach of one tile row and one tile column keeps the neighbours' levels
    assert bench.tile_modes([logits], 0.0, H, W, reach=32.0).tolist() == [0, 3, 1]
    logits[0, 15] = 10.0                # block (0, 15) lies within one block of tile (0, 1) only
    assert bench.tile_modes([logits], 0.0, H, W, reach=0.0).tolist() == [2, 0, 2]
    logits[1, 7] = 10.0                 # block (1, 7) lies within one block of all four tiles
    assert bench.tile_modes([logits], 0.0, H, W, reach=0.0).tolist() == [0, 0, 4]


def test_break_even_share_by_hand():
    # network 0.5 ms; masking every tile saves 1.86 - 0.69 = 1.17 ms
    assert abs(bench.break_even_share(0.5, 1.86, 0.69) - 0.5 / 1.17) < 1e-12
    # a network as costly as the whole saving breaks even only at every tile
    assert abs(bench.break_even_share(1.0, 2.0, 1.0) - 1.0) < 1e-12
    # no saving (or a slower masked octave): never pays
    assert bench.break_even_share(0.5, 1.0, 1.0) is None
    assert bench.break_even_share(0.5, 1.0, 1.2) is None
    assert bench.break_even_share(0.5, float("nan"), 0.7) is None
