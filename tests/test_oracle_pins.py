"""Pins for the CPU oracle: values fixed by the paper and by mathematics, not by the oracle.

Each test checks the oracle against something computed another way: a
hand-derived set, a textbook range query, a polar closed form, the epipolar
constraint of noise-free projections, an independent numpy / decimal brute
force.  A dropped term, a wrong sign or index, or a transposed F in the
oracle fails at least one of them.
"""
import json
import math
import os
from bisect import bisect_left, bisect_right
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import synth


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _rows(c):
    off, idx = c["offsets"], c["idx"]
    return [list(idx[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


# --------------------------------------------------------------------------
# Candidate sets (Eq. 3, Eq. 4)
# --------------------------------------------------------------------------

def test_golden_tiny_scenes(golden_dir):
    g = _load(golden_dir, "tiny_scenes.json")
    for sc in g["scenes"]:
        c = oracle.candidates(np.array(sc["queries"], float), np.array(sc["refs"], float),
                              np.array(sc["F"], float), sc["eps"] if np.isscalar(sc["eps"])
                              else np.array(sc["eps"], float))
        assert _rows(c) == sc["expected"], sc["name"]
        assert list(c["degenerate"]) == sc["degenerate"], sc["name"]


def test_rectified_matches_sorted_range_query():
    """t = (1,0,0), K = I, R = I: C_i = {j : |y_j - y_i| <= eps}; a textbook
    range query over the references sorted by y gives the same set."""
    rng = np.random.default_rng(11)
    F = synth.skew([1.0, 0.0, 0.0])
    xy1 = rng.uniform(0, 500, size=(300, 2))
    xy2 = rng.uniform(0, 500, size=(3000, 2))
    # integer y values make some distances land exactly on eps
    xy1[:50, 1] = np.round(xy1[:50, 1])
    xy2[:500, 1] = np.round(xy2[:500, 1])
    eps = 2.0
    c = oracle.candidates(xy1, xy2, F, eps)
    order = np.argsort(xy2[:, 1], kind="stable")
    ys = list(xy2[order, 1])
    for i, row in enumerate(_rows(c)):
        y = xy1[i, 1]
        lo = bisect_left(ys, y - eps)
        hi = bisect_right(ys, y + eps)
        want = sorted(int(j) for j in order[lo:hi])
        assert row == want, i
    # the integer rows include pairs exactly at distance eps
    assert any(abs(abs(xy2[j, 1] - xy1[i, 1]) - eps) == 0 for i in range(50) for j in _rows(c)[i])


def test_forward_motion_polar_closed_form():
    """t = (0,0,1), K = I, R = I: every line passes through the epipole at the
    origin, and the distance of p to the line at angle alpha is
    r |sin(theta - alpha)| in polar coordinates."""
    rng = np.random.default_rng(12)
    F = synth.skew([0.0, 0.0, 1.0])
    xy1 = rng.uniform(-300, 300, size=(200, 2))
    xy2 = rng.uniform(-300, 300, size=(4000, 2))
    eps = 1.5
    c = oracle.candidates(xy1, xy2, F, eps)
    r = np.hypot(xy2[:, 0], xy2[:, 1])
    th = np.arctan2(xy2[:, 1], xy2[:, 0])
    for i, row in enumerate(_rows(c)):
        alpha = math.atan2(xy1[i, 1], xy1[i, 0])
        d = r * np.abs(np.sin(th - alpha))
        clear = np.abs(d - eps) > 1e-9
        want = set(np.nonzero((d <= eps) & clear)[0])
        got = set(row)
        assert want <= got
        assert got - want <= set(np.nonzero(~clear)[0])
        for j in (0, 7, 99):
            assert abs(oracle.point_line_distance(F, *xy1[i], *xy2[j]) - d[j]) < 1e-9


def test_true_correspondences_lie_on_their_lines():
    """Noise-free projections of 3D points satisfy p2^T F p1 = 0 (Sec. 3), so
    their distance to the epipolar line F p1 is ~0; with F^T instead of F
    (a transposed operand) they are not."""
    rng = np.random.default_rng(13)
    K1 = synth.intrinsics(800.0, 1000, 800)
    K2 = synth.intrinsics(900.0, 1000, 800)
    R = synth.rotation([0.3, -1.0, 0.2], 12.0)
    t = np.array([0.7, -0.2, 0.3])
    F = synth.fundamental(K1, K2, R, t)
    X = np.c_[rng.uniform(-2, 2, 200), rng.uniform(-2, 2, 200), rng.uniform(4, 9, 200)]
    p1 = (K1 @ X.T).T
    p1 = p1[:, :2] / p1[:, 2:]
    X2 = X @ R.T + t
    p2 = (K2 @ X2.T).T
    p2 = p2[:, :2] / p2[:, 2:]
    d = np.array([oracle.point_line_distance(F, *p1[k], *p2[k]) for k in range(200)])
    assert d.max() < 1e-7
    dT = np.array([oracle.point_line_distance(F.T, *p1[k], *p2[k]) for k in range(200)])
    assert np.median(dT) > 1.0


def test_degenerate_line_has_empty_set():
    F = synth.skew([0.0, 0.0, 1.0])
    c = oracle.candidates(np.array([[0.0, 0.0], [1.0, 0.0]]), np.array([[0.0, 0.0], [5.0, 0.0]]), F, 1.0)
    assert list(c["degenerate"]) == [1, 0]
    assert _rows(c) == [[], [0, 1]]


def test_boundary_list():
    """Pairs within 1e-9 px of the tolerance are listed apart (and still decided by <=)."""
    F = synth.skew([1.0, 0.0, 0.0])
    xy1 = np.array([[0.0, 10.0]])
    xy2 = np.array([[0.0, 12.0], [0.0, 12.0 + 5e-10], [0.0, 12.0 - 5e-10], [0.0, 12.1], [0.0, 8.0]])
    c = oracle.candidates(xy1, xy2, F, 2.0)
    assert _rows(c) == [[0, 2, 4]]
    assert list(c["bidx"]) == [0, 1, 2, 4]


# --------------------------------------------------------------------------
# Epipole and angular intervals (Sec. 4.2, Algorithm 1)
# --------------------------------------------------------------------------

def test_epipole_is_K_t():
    """For F = K2^-T [t]x R K1^-1, F^T (K2 t) = 0, so e2 ~ K2 t (up to scale)."""
    for seed in range(5):
        rng = np.random.default_rng(seed)
        K1 = synth.intrinsics(rng.uniform(300, 5000), 640, 480)
        K2 = synth.intrinsics(rng.uniform(300, 5000), 640, 480)
        R = synth.rotation(rng.normal(size=3), rng.uniform(0, 30))
        t = rng.normal(size=3)
        e = oracle.epipole(synth.fundamental(K1, K2, R, t))
        want = K2 @ t
        want = want / np.linalg.norm(want)
        assert min(np.linalg.norm(e - want), np.linalg.norm(e + want)) < 1e-10


def test_intervals_tangent_closed_form():
    """delta_j = asin(eps / d_j): the line through the epipole at angle
    theta_j +- delta_j is tangent to the eps-circle around p_j (Sec. 4.1,
    Eq. delta), and the line at theta_j passes through p_j."""
    K = synth.intrinsics(500.0, 640, 480)
    R = synth.rotation([0, 1, 0], 3.0)
    t = np.array([0.2, 0.1, 1.0])
    F = synth.fundamental(K, K, R, t)
    rng = np.random.default_rng(3)
    xy2 = rng.uniform([0, 0], [640, 480], size=(500, 2))
    eps = rng.uniform(0.5, 5.0, size=500)
    theta, delta, e = oracle.intervals(F, xy2, eps)
    assert np.all((theta >= 0) & (theta < math.pi))
    d = np.hypot(xy2[:, 0] - e[0], xy2[:, 1] - e[1])
    far = d > eps
    for s in (-1.0, 1.0):
        a = theta + s * delta
        # distance of p_j from the line through e with direction (cos a, sin a)
        dist = np.abs((xy2[:, 0] - e[0]) * np.sin(a) - (xy2[:, 1] - e[1]) * np.cos(a))
        assert np.allclose(dist[far], eps[far], rtol=0, atol=1e-9)
    dist0 = np.abs((xy2[:, 0] - e[0]) * np.sin(theta) - (xy2[:, 1] - e[1]) * np.cos(theta))
    assert dist0.max() < 1e-9
    assert np.all(delta[~far] == math.pi / 2)


def test_intervals_near_epipole_full():
    F = synth.skew([0.0, 0.0, 1.0])
    theta, delta, e = oracle.intervals(F, np.array([[0.0, 0.0], [0.3, 0.4], [3.0, 4.0]]), 1.0)
    assert np.allclose(e, 0.0)
    assert delta[0] == delta[1] == math.pi / 2
    assert abs(delta[2] - math.asin(0.2)) < 1e-15


# --------------------------------------------------------------------------
# Descriptor matching (Sec. 4.3)
# --------------------------------------------------------------------------

def _golden_match(g, key, kind):
    s = g[key]
    out = oracle.match(np.array(s["queries"], float), np.array(s["refs"], float),
                       np.array(g["F"], float), g["eps"], np.array(s["desc1"], np.uint8),
                       np.array(s["desc2"], np.uint8), kind, s["dim"])
    assert list(out["best"]) == s["best"]
    assert list(out["second"]) == s["second"]
    assert list(out["flags"]) == s["flags"]
    for got, want in zip(out["best_d"], s["best_d"]):
        assert (want is None and got == math.inf) or got == want
    for got, want in zip(out["second_d"], s["second_d"]):
        assert (want is None and got == math.inf) or got == want


def test_golden_matches(golden_dir):
    g = _load(golden_dir, "tiny_matches.json")
    _golden_match(g, "u8", 0)
    _golden_match(g, "bin", 2)


def _decimal_ratio_pass(d1sq, d2sq, num=4, den=5):
    getcontext().prec = 60
    return Decimal(int(d1sq)).sqrt() < Decimal(num) / Decimal(den) * Decimal(int(d2sq)).sqrt()


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_infinite_eps_is_exhaustive_nearest_neighbour(kind):
    """eps larger than any distance: C_i is every reference and matching is
    plain exhaustive nearest neighbour; compare with an independent numpy
    brute force (argsort by (distance, index)) and a decimal ratio test."""
    rng = np.random.default_rng(20 + kind)
    m, n = 40, 60
    F = synth.fundamental(synth.intrinsics(500, 640, 480), synth.intrinsics(500, 640, 480),
                          synth.rotation([0, 1, 0], 10), [0.3, 0.0, 0.03])
    xy1 = rng.uniform([0, 0], [640, 480], (m, 2))
    xy2 = rng.uniform([0, 0], [640, 480], (n, 2))
    if kind == 0:
        d1 = rng.integers(0, 8, (m, 16), dtype=np.uint8)   # small alphabet: many ties
        d2 = rng.integers(0, 8, (n, 16), dtype=np.uint8)
        D = ((d1[:, None, :].astype(np.int64) - d2[None, :, :].astype(np.int64)) ** 2).sum(-1)
        dim = 16
    elif kind == 2:
        d1 = rng.integers(0, 256, (m, 4), dtype=np.uint8)
        d2 = rng.integers(0, 256, (n, 4), dtype=np.uint8)
        D = np.array([[sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(d1[i], d2[j]))
                       for j in range(n)] for i in range(m)])
        dim = 32
    else:
        d1 = rng.random((m, 8)).astype(np.float32)
        d2 = rng.random((n, 8)).astype(np.float32)
        D = ((d1[:, None, :].astype(np.float64) - d2[None, :, :].astype(np.float64)) ** 2).sum(-1)
        dim = 8
    out = oracle.match(xy1, xy2, F, 1e12, d1, d2, kind, dim)
    for i in range(m):
        order = np.lexsort((np.arange(n), D[i]))
        assert out["best"][i] == order[0] and out["second"][i] == order[1]
        tol = 1e-12 * D[i, order[1]] if kind == 1 else 0   # numpy sums pairwise
        assert abs(out["best_d"][i] - D[i, order[0]]) <= tol
        assert abs(out["second_d"][i] - D[i, order[1]]) <= tol
        if kind == 0:
            want = _decimal_ratio_pass(D[i, order[0]], D[i, order[1]])
        elif kind == 2:
            want = D[i, order[0]] / D[i, order[1]] < 0.8 if D[i, order[1]] else False
        else:
            want = math.sqrt(D[i, order[0]]) < 0.8 * math.sqrt(D[i, order[1]])
        assert bool(out["flags"][i] & oracle.FLAG_RATIO_PASS) == bool(want)
        assert out["ncand"][i] == n


def test_exclude_boundary_changes_only_boundary_queries():
    F = synth.skew([1.0, 0.0, 0.0])
    xy1 = np.array([[0.0, 10.0], [0.0, 50.0]])
    xy2 = np.array([[0.0, 12.0], [0.0, 10.5], [0.0, 50.0]])
    d1 = np.array([[0, 0], [0, 0]], np.uint8)
    d2 = np.array([[0, 0], [3, 0], [0, 0]], np.uint8)
    a = oracle.match(xy1, xy2, F, 2.0, d1, d2, 0, 2)
    b = oracle.match(xy1, xy2, F, 2.0, d1, d2, 0, 2, exclude_boundary=True)
    assert a["best"][0] == 0 and b["best"][0] == 1
    assert a["best"][1] == b["best"][1] == 2


def test_mutual_matching_hand_case_and_symmetry():
    """A hand-built pair: F = [x]_x (lines y = y1 in both directions), two
    points per image on the same rows; descriptors make 0 <-> 1 and 1 <-> 0
    mutual, while query 2's best (reference 1) prefers query 1."""
    F = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])  # [e_x]_x: p2^T F p1 = y1 - y2
    xy1 = np.array([[10.0, 5.0], [20.0, 7.0], [30.0, 7.0]])
    xy2 = np.array([[40.0, 5.0], [50.0, 7.0]])
    d1 = np.array([[0] * 15 + [0], [0] * 15 + [100], [0] * 15 + [110]], np.uint8)
    d2 = np.array([[0] * 15 + [1], [0] * 15 + [101]], np.uint8)
    fw, rv = oracle.match_mutual(xy1, xy2, F, 0.5, 0.5, d1, d2, 0, 16)
    assert list(fw["best"]) == [0, 1, 1]
    assert list(rv["best"]) == [0, 1]
    mf = (fw["flags"] & oracle.FLAG_MUTUAL) != 0
    mr = (rv["flags"] & oracle.FLAG_MUTUAL) != 0
    assert list(mf) == [True, True, False] and list(mr) == [True, True]
    # symmetry on a random scene: mutual rows pair up one to one
    sc = synth.config1(seed=2, scale=0.2)
    fw, rv = oracle.match_mutual(sc.xy1, sc.xy2, sc.F, 2.0, 2.0, sc.desc1, sc.desc2, sc.kind, sc.dim)
    mf = np.nonzero(fw["flags"] & oracle.FLAG_MUTUAL)[0]
    mr = np.nonzero(rv["flags"] & oracle.FLAG_MUTUAL)[0]
    assert len(mf) == len(mr) > 0
    assert sorted(fw["best"][mf]) == sorted(mr) and sorted(rv["best"][mr]) == sorted(mf)
