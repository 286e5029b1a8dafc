"""Matching of GPU records to oracle records, shared by the GPU parity tests.

Tolerances (the CUDA path computes in FP32, the oracle in FP64):
  * two points match when they are in the same octave, within 0.5 octave px
    in x and y, and within 0.01 in |log sigma|;
  * position <= 0.01 octave px, relative scale <= 1e-3, descriptor relative L2
    <= 1e-3 for matched points;
  * at least 99.5% of the oracle's points are matched, not counting those the
    oracle itself decides within a relative 1e-4 of a threshold (points that
    appear or vanish when every threshold is moved by 1e-4: the "margin" set).
"""
import numpy as np

POS_TOL = 0.01        # octave px
SCALE_TOL = 1e-3      # relative
DESC_TOL = 1e-3       # relative L2
THETA_TOL = 1e-4      # rad: the same orientation (FP32 histogram sums shift a peak by ~1e-6 rad)
THETA_ID = 2e-2       # rad: records closer than this are taken as the same orientation copy
AGREE = 0.995
MARGIN = 1e-4


def octave_coords(r):
    s = 2.0 ** r["octave"].astype(np.float64)
    return r["x"] / s, r["y"] / s, r["sigma"] / s


def candidates(a, b):
    """For each record of a, the indices of the records of b that match it
    (same octave, |dx|, |dy| < 0.5 octave px, |dlog sigma| < 0.01), nearest
    first (ties by index)."""
    out = [np.zeros(0, np.int64) for _ in range(len(a))]
    if len(a) == 0 or len(b) == 0:
        return out
    ax, ay, asg = octave_coords(a)
    bx, by, bsg = octave_coords(b)
    for i in range(len(a)):
        m = (b["octave"] == a["octave"][i]) & (np.abs(bx - ax[i]) < 0.5) & (np.abs(by - ay[i]) < 0.5) & \
            (np.abs(np.log(bsg / asg[i])) < 0.01)
        idx = np.nonzero(m)[0]
        d = (bx[idx] - ax[i]) ** 2 + (by[idx] - ay[i]) ** 2
        out[i] = idx[np.argsort(d, kind="stable")]
    return out


def match(a, b):
    """For each record of a, the index of the nearest record of b that matches
    it, else -1 (several records of a may name the same record of b)."""
    return np.array([c[0] if c.size else -1 for c in candidates(a, b)], np.int64)


def max_matching(adj, n_right):
    """A maximum one-to-one pairing of left vertices i with right vertices in
    adj[i] (breadth-first augmenting paths).  Returns, per right vertex, its
    left partner or -1."""
    owner = np.full(n_right, -1, np.int64)
    held = {}  # left vertex -> the right vertex it holds
    for root in range(len(adj)):
        if len(adj[root]) == 0:
            continue
        parent = {}  # right vertex -> the left vertex that reached it
        seen_left = {root}
        queue = [root]
        free = -1
        while queue and free < 0:
            nxt = []
            for i in queue:
                for j in adj[i]:
                    j = int(j)
                    if j in parent:
                        continue
                    parent[j] = i
                    if owner[j] < 0:
                        free = j
                        break
                    k = int(owner[j])
                    if k not in seen_left:
                        seen_left.add(k)
                        nxt.append(k)
                if free >= 0:
                    break
            queue = nxt
        if free < 0:
            continue
        j = free
        while True:  # flip the path: every left vertex on it moves to the right vertex that reached it
            i = parent[j]
            prev = held.get(i, -1)
            owner[j] = i
            held[i] = j
            if i == root:
                break
            j = prev
    return owner


def keyset(r):
    """Point identity used to compare oracle runs with each other."""
    x, y, s = octave_coords(r)
    return [(int(o), round(float(xx), 3), round(float(yy), 3), round(float(np.log(ss)), 3))
            for o, xx, yy, ss in zip(r["octave"], x, y, s)]


def point_agreement(gpu, exact, loose, strict):
    """Agreement of the GPU point set with the oracle's, excluding margin points.

    GPU and oracle points pair one to one (a maximum matching over matching
    pairs).  An oracle point left unpaired is missing; it is in the margin set
    when it is not in both the loose and the strict oracle result.  A GPU point
    with no matching oracle point is extra, and a margin case when the loose
    run has it; a GPU point whose matching oracle points are all paired with
    other GPU points is a duplicate and always a disagreement.

    Returns (agreement, n_disagree, n_excluded, n_oracle)."""
    cand = candidates(gpu, exact)
    owner = max_matching(cand, len(exact))
    paired_gpu = np.zeros(len(gpu), bool)
    paired_gpu[owner[owner >= 0]] = True
    e_in_loose = match(exact, loose) >= 0
    e_in_strict = match(exact, strict) >= 0
    g_in_loose = match(gpu, loose) >= 0
    has_cand = np.array([c.size > 0 for c in cand], bool)
    # oracle points missing on the GPU
    miss = owner < 0
    miss_margin = miss & ~(e_in_loose & e_in_strict)
    # GPU points absent from the oracle, and duplicates
    extra = ~paired_gpu & ~has_cand
    extra_margin = extra & g_in_loose
    dup = ~paired_gpu & has_cand
    n_dis = int((miss & ~miss_margin).sum() + (extra & ~extra_margin).sum() + dup.sum())
    n_exc = int(miss_margin.sum() + extra_margin.sum())
    n = max(1, len(exact))
    return 1.0 - n_dis / n, n_dis, n_exc, len(exact)


def ang(a, b):
    d = abs(a - b) % (2 * np.pi)
    return min(d, 2 * np.pi - d)


def good_edges(gk, gd, ek, ed):
    """For each GPU record i, the oracle records j it may pair with: the same
    point, theta within THETA_TOL and a descriptor within DESC_TOL."""
    adj = []
    m0 = match(gk, ek)
    for i in range(len(gk)):
        if m0[i] < 0:
            adj.append([])
            continue
        same_pt = np.nonzero(match(ek, gk[i:i + 1]) == 0)[0]
        adj.append([int(j) for j in same_pt
                    if ang(ek["theta"][j], gk["theta"][i]) <= THETA_TOL and rel_l2(gd[i], ed[j]) <= DESC_TOL])
    return adj


def record_agreement(gk, gd, runs, at_point=None):
    """Orientation and descriptor agreement of GPU records with the oracle.

    runs[0] = (records, descriptors) of the oracle itself; runs[1:] = the
    oracle with every threshold, every orientation-bin boundary and the
    sampling-disc radii moved by a relative 1e-4 (both ways).  GPU records pair
    one to one with the oracle's records of the same point, theta within
    THETA_TOL and a descriptor within DESC_TOL (a maximum matching): each pair
    is good.  An unpaired GPU record that has such a partner, all of them
    paired with other GPU records, is a duplicate: bad.  Any other unpaired
    GPU record of an oracle point is a margin case when only a perturbed oracle
    run has such a record (a gradient sample on a histogram bin boundary, a
    peak on the 0.8 x max line, a pixel on the edge of the sampling disc), and
    bad otherwise.  GPU records of points the oracle lacks are left to
    point_agreement.

    at_point(i), when given, returns the oracle's (records, descriptors) for
    the point of GPU record i as the GPU found it.  Alg. 2 is discontinuous in
    the point (a pixel enters or leaves the sampling disc), so where the
    end-to-end points differ by FP32 rounding (far inside POS_TOL) a record
    that the oracle reproduces at the GPU's own point is a margin case too.
    Returns (good, margin, bad)."""
    ek, ed = runs[0]
    adj = good_edges(gk, gd, ek, ed)
    owner = max_matching(adj, len(ek))
    paired = np.zeros(len(gk), bool)
    paired[owner[owner >= 0]] = True
    good = int(paired.sum())
    margin = bad = 0
    m0 = match(gk, ek)
    alt_m = [match(gk, r[0]) for r in runs[1:]]
    for i in range(len(gk)):
        if paired[i] or m0[i] < 0:
            continue  # paired, or a point-level disagreement (counted by point_agreement)
        if adj[i]:
            bad += 1  # a duplicate of oracle records already paired
            continue
        # not explained by the oracle itself: a margin case when a perturbed
        # oracle run has the same orientation and descriptor
        hit = False
        for (rk, rd), mm in zip(runs[1:], alt_m):
            if mm[i] < 0:
                continue
            pts = np.nonzero(match(rk, gk[i:i + 1]) == 0)[0]
            if any(ang(rk["theta"][j], gk["theta"][i]) <= THETA_TOL and rel_l2(gd[i], rd[j]) <= DESC_TOL
                   for j in pts):
                hit = True
        if not hit and at_point is not None:
            rk, rd = at_point(i)
            hit = any(ang(rk["theta"][j], gk["theta"][i]) <= THETA_TOL and rel_l2(gd[i], rd[j]) <= DESC_TOL
                      for j in range(len(rk)))
        if hit:
            margin += 1
        else:
            bad += 1
    return good, margin, bad


def good_pairs(gk, gd, ek, ed):
    """(i, j) pairs of GPU record i and oracle record j, one to one, for the
    same point with theta within THETA_TOL and a descriptor within DESC_TOL."""
    owner = max_matching(good_edges(gk, gd, ek, ed), len(ek))
    return sorted((int(owner[j]), int(j)) for j in range(len(ek)) if owner[j] >= 0)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


# Counts that the GPU tests report (printed at the end of the pytest run by
# tests/conftest.py, so a run's tail shows the good / margin / bad splits and
# the excluded counts, not only pass or fail).
REPORT = []


def report(name, **counts):
    REPORT.append((name, counts))
