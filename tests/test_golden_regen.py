"""The stored stand-in tables are what their committed scripts write from the
oracle: tests/golden/make_scfv_model.py and make_ternary_thresholds.py
recomputed here must reproduce scfv_model.npz and ternary_thresholds.json."""
import importlib.util
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(GOLDEN, name + ".py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_scfv_model_is_reproduced():
    model, n = _load("make_scfv_model").compute()
    stored = np.load(os.path.join(GOLDEN, "scfv_model.npz"))
    assert f"{n} records" in str(stored["source"])
    for k, v in model.items():
        # eigenvectors from another LAPACK build may differ in the last bits
        np.testing.assert_allclose(v, stored[k], rtol=1e-5, atol=1e-6, err_msg=k)


def test_ternary_thresholds_are_reproduced():
    out = _load("make_ternary_thresholds").compute()
    stored = json.load(open(os.path.join(GOLDEN, "ternary_thresholds.json")))
    assert out["n_descriptors"] == stored["n_descriptors"] and out["source"] == stored["source"]
    np.testing.assert_allclose(out["t_lo"], stored["t_lo"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["t_hi"], stored["t_hi"], rtol=1e-12, atol=1e-15)
