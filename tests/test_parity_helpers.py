"""The matching and classification that every GPU parity test relies on
(tests/parity.py), on hand-built records: one-to-one pairing, duplicates,
missing and extra points, margin cases and tolerances."""
import numpy as np

import parity as PT
from oracle import oracle as O


def _recs(spec):
    """Records from (x, y, sigma, octave, theta) tuples, image px."""
    r = np.zeros(len(spec), O.KP_DTYPE)
    for i, (x, y, s, o, t) in enumerate(spec):
        r[i]["x"], r[i]["y"], r[i]["sigma"], r[i]["octave"], r[i]["theta"] = x, y, s, o, t
        r[i]["parent"] = i
    return r


def _descs(n, seed=0):
    d = np.abs(np.random.default_rng(seed).normal(size=(n, 128)))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


ORACLE = _recs([(10, 10, 2.0, 0, 0.5), (40, 12, 2.5, 0, 1.0), (40, 12, 2.5, 0, 2.5),
                (80, 64, 5.0, 1, 3.0), (120, 30, 3.1, 0, 6.0)])
DESC = _descs(len(ORACLE))


def test_max_matching_finds_the_larger_pairing():
    # greedy in index order would give left 0 the right vertex 0 and leave left 1 unpaired
    owner = PT.max_matching([[0, 1], [0]], 2)
    assert sorted(owner.tolist()) == [0, 1] and owner[0] == 1 and owner[1] == 0
    owner = PT.max_matching([[0], [0], [1, 2], [2]], 3)
    assert (owner >= 0).sum() == 3
    assert PT.max_matching([[], []], 2).tolist() == [-1, -1]


def test_identical_records_are_all_good():
    runs = [(ORACLE, DESC)] * 3
    assert PT.record_agreement(ORACLE, DESC, runs) == (5, 0, 0)
    assert PT.good_pairs(ORACLE, DESC, ORACLE, DESC) == [(i, i) for i in range(5)]
    pts = ORACLE[[0, 1, 3, 4]]
    assert PT.point_agreement(pts, pts, pts, pts) == (1.0, 0, 0, 4)


def test_a_duplicated_record_is_bad_even_when_a_perturbed_run_has_it():
    gk = np.concatenate([ORACLE, ORACLE[:1]])
    gd = np.concatenate([DESC, DESC[:1]])
    runs = [(ORACLE, DESC)] * 3
    assert PT.record_agreement(gk, gd, runs) == (5, 0, 1)
    assert len(PT.good_pairs(gk, gd, ORACLE, DESC)) == 5


def test_duplicated_and_missing_points_disagree():
    pts = ORACLE[[0, 1, 3, 4]]
    dup = np.concatenate([pts, pts[:1]])
    assert PT.point_agreement(dup, pts, pts, pts)[1:] == (1, 0, 4)
    assert PT.point_agreement(pts[:3], pts, pts, pts)[1:] == (1, 0, 4)
    # a missing point that only one perturbed run has is a margin point
    assert PT.point_agreement(pts[:3], pts, pts[:3], pts)[1:] == (0, 1, 4)
    # an extra GPU point the loose run has is a margin point; otherwise it disagrees
    extra = _recs([(300, 200, 4.0, 0, 0.0)])
    g = np.concatenate([pts, extra])
    assert PT.point_agreement(g, pts, np.concatenate([pts, extra]), pts)[1:] == (0, 1, 4)
    assert PT.point_agreement(g, pts, pts, pts)[1:] == (1, 0, 4)


def test_point_window_and_octave():
    pts = ORACLE[[0]]
    near = _recs([(10.49, 9.51, 2.0 * np.exp(0.0099), 0, 0.0)])
    assert PT.point_agreement(near, pts, pts, pts)[1:] == (0, 0, 1)
    # (20, 20, 4.0) in octave 1 has the octave coordinates (10, 10, 2.0) of the oracle's point
    for far in [(10.51, 10, 2.0, 0, 0.0), (10, 10, 2.0 * np.exp(0.0101), 0, 0.0), (20, 20, 4.0, 1, 0.0)]:
        assert PT.point_agreement(_recs([far]), pts, pts, pts)[1] == 2   # extra and missing


def test_orientation_and_descriptor_tolerances():
    runs = [(ORACLE, DESC)] * 3
    gk, gd = ORACLE.copy(), DESC.copy()
    gk["theta"][0] += 0.9 * PT.THETA_TOL
    gd[1] += 0.9 * PT.DESC_TOL / np.sqrt(128)          # relative L2 0.9e-3
    assert PT.record_agreement(gk, gd, runs) == (5, 0, 0)
    gk["theta"][0] += 0.2 * PT.THETA_TOL
    gd[1] += 0.2 * PT.DESC_TOL / np.sqrt(128)
    assert PT.record_agreement(gk, gd, runs) == (3, 0, 2)
    # theta wraps at 2 pi: 5e-5 and 2 pi - 3e-5 are 8e-5 apart
    ek = ORACLE.copy()
    ek["theta"][4] = 5e-5
    gk, gd = ek.copy(), DESC.copy()
    gk["theta"][4] = 2 * np.pi - 3e-5
    assert PT.record_agreement(gk, gd, [(ek, DESC)] * 3) == (5, 0, 0)
    gk["theta"][4] = 2 * np.pi - 6e-5
    assert PT.record_agreement(gk, gd, [(ek, DESC)] * 3) == (4, 0, 1)


def test_a_record_only_a_perturbed_run_explains_is_a_margin_case():
    gk, gd = ORACLE.copy(), DESC.copy()
    gk["theta"][2] = 2.6                                  # a different orientation copy
    other = ORACLE.copy()
    other["theta"][2] = 2.6
    assert PT.record_agreement(gk, gd, [(ORACLE, DESC), (other, DESC), (ORACLE, DESC)]) == (4, 1, 0)
    assert PT.record_agreement(gk, gd, [(ORACLE, DESC)] * 3) == (4, 0, 1)
    # the oracle at the GPU's own point explains it too
    assert PT.record_agreement(gk, gd, [(ORACLE, DESC)] * 3,
                               at_point=lambda i: (gk[i:i + 1], gd[i:i + 1])) == (4, 1, 0)
