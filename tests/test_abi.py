"""The C ABI library on the CPU: it loads, exports every symbol include/cdvs.h
declares, and its host-side parts (selection order, transform + ternary
quantisation) agree bit for bit with the oracle.  No GPU compute here."""
import json
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1705_09776_gb300 import build as B
from paper_1705_09776_gb300 import cdvs
from paper_1705_09776_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cdvs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cdvs_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert set(declared) == set(cdvs.EXPORTED)
    L = cdvs.load()
    for s in declared:
        assert getattr(L, s) is not None


def test_params_defaults_and_struct_sizes():
    p = cdvs.params()
    assert p["num_octaves"][0] == 4 and p["scales_per_octave"][0] == 4
    assert p["sigma0"][0] == np.float32(1.6) and p["ori_radius"][0] == np.float32(3.96)
    assert p["ori_peak_ratio"][0] == np.float32(0.8) and p["desc_radius"][0] == np.float32(6.0)
    assert p["cell_side"][0] == np.float32(3.0) and p["max_keypoints"][0] == 300
    # the oracle's defaults are the same method parameters
    q = O.params()
    for k in ["num_octaves", "scales_per_octave", "max_keypoints", "max_orientations", "upright"]:
        assert int(p[k][0]) == int(q[k][0])
    for k in ["sigma0", "sigma_in", "contrast_T", "edge_r", "offset_max", "ori_radius", "ori_peak_ratio",
              "ori_weight_sigma", "desc_radius", "cell_side", "desc_weight_sigma", "dedupe_dlog2"]:
        assert p[k][0] == np.float32(q[k][0]), k


def test_create_fails_cleanly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cdvs.CdvsError):
        cdvs.Context(0)


def test_rank_host_matches_oracle_selection_order():
    rng = np.random.default_rng(3)
    n = 500
    pts = np.zeros(n, cdvs.KEYPOINT_DTYPE)
    pts["x"] = rng.integers(0, 50, n).astype(np.float32)
    pts["y"] = rng.integers(0, 50, n).astype(np.float32)
    pts["sigma"] = rng.choice([2.0, 3.0], n).astype(np.float32)
    pts["response"] = rng.choice([-9.0, 5.0, 7.5, -7.5, 12.0], n).astype(np.float32)   # many ties
    pts["octave"] = rng.integers(0, 2, n)
    order = cdvs.rank_host(pts, 200)
    ok = np.zeros(n, O.KP_DTYPE)
    for f in ["x", "y", "sigma", "response", "octave"]:
        ok[f] = pts[f]
    P = O.params(max_keypoints=200)
    keep = np.ones(n, np.uint8)
    ref = np.zeros(n, np.int32)
    m = O.lib().oracle_select(O._p(ok), O._p(keep), n, O._p(P), O._p(ref))
    assert m == 200
    # identical (x, y, sigma, octave, response) points may swap; compare the keys
    key = lambda i: (pts["response"][i], pts["y"][i], pts["x"][i], pts["sigma"][i], pts["octave"][i])
    assert [key(i) for i in order] == [key(i) for i in ref[:m]]


def test_transform_ternary_bit_exact_with_oracle():
    th = json.load(open(os.path.join(ROOT, "tests", "golden", "ternary_thresholds.json")))
    lo, hi = np.array(th["t_lo"]), np.array(th["t_hi"])
    img = synth.blob_image(synth.image_seed(5, 0))
    kp, d, _ = O.extract(img, O.params())
    d32 = d.astype(np.float32)
    q, v = cdvs.transform_ternary(d32, lo, hi)
    for i in range(d32.shape[0]):
        vo = O.transform(d32[i].astype(np.float64))
        assert np.array_equal(v[i], vo)
        assert np.array_equal(q[i], O.ternary(vo, lo, hi))
    # the stand-in thresholds split every element roughly in thirds on fresh images
    frac = [(q == s).mean() for s in (-1, 0, 1)]
    assert all(0.2 < f < 0.5 for f in frac), frac


def test_header_constants_match_the_binding():
    """Every flag, storage type and size the header defines has the same value
    in the Python binding."""
    src = open(os.path.join(ROOT, "include", "cdvs.h")).read()
    defs = {k: int(v, 0) for k, v in re.findall(r"#define (CDVS_[A-Z0-9_]+) (0x[0-9a-fA-F]+|[0-9]+)u?\b", src)}
    assert {"CDVS_INPUT_DEVICE", "CDVS_OUTPUT_DEVICE", "CDVS_ASYNC", "CDVS_STORAGE_FP16"} <= set(defs)
    for k, v in defs.items():
        py = k if hasattr(cdvs, k) else k[len("CDVS_"):]
        if hasattr(cdvs, py):
            assert getattr(cdvs, py) == v, k
    assert cdvs.PROPOSAL_PARAMS == defs["CDVS_PROPOSAL_PARAMS"]
    # the status codes of the enum
    enum = dict((n, int(v)) for n, v in re.findall(r"\b(CDVS_[A-Z_]+) = ([0-9]+)", src))
    for n, v in enum.items():
        assert getattr(cdvs, n) == v, n


def test_names_the_readme_examples_use_exist():
    """The README's examples call these parameters, functions and methods."""
    p = cdvs.params(max_keypoints=2000, num_octaves=6, storage=cdvs.CDVS_STORAGE_FP16, max_side=640,
                    use_proposal=1, proposal_threshold=0.1)
    assert int(p["max_keypoints"][0]) == 2000 and int(p["max_side"][0]) == 640
    for name in ("rank_host", "transform_ternary", "load_proposal_weights", "CDVS_ASYNC"):
        assert hasattr(cdvs, name), name
    for name in ("extract", "extract_raw", "wait", "set_graph", "candidates", "dedupe_select", "describe",
                 "set_scfv_model", "scfv", "set_proposal"):
        assert callable(getattr(cdvs.Context, name)), name
    theta, thr = cdvs.load_proposal_weights()
    assert 0.0 < thr < 1.0 and theta.ndim == 1
