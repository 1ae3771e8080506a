"""CPU oracle for exact epipolar-guided matching.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library never does.  It shares no code with
the CUDA path.  Everything is FP64.

- ``candidates`` / ``match``: brute force over all (query, reference) pairs
  (plain C, ``egm_oracle.c``), following Sec. 3 Eqs. 3-4 and Sec. 4.3.
- ``epipole``: the null vector of F^T (Algorithm 1, preprocessing) from an SVD.
- ``intervals``: the angular interval of every reference keypoint as seen from
  the epipole, theta_j = atan2(y_j - y_e, x_j - x_e) and
  delta_j = asin(eps_j / ||p_j - e||) (Sec. 4.2), folded into [0, pi)
  (Sec. 4.2: lines are undirected, so angles are taken mod pi); keypoints within eps of the epipole get the
  full interval (Algorithm 1; Sec. 4.4 "Keypoints near the epipole").
- ``match_mutual``: matching in both directions (the reverse with F^T and the
  roles of the images swapped, Sec. 3) and the cross-check: i -> j is mutual
  when j's best in the reverse direction is i.
- ``mlp``: the learned-tolerance network in FP64 (see ``oracle/mlp.py``).
- ``gms``: the grid motion-statistics filter of the matches (see ``oracle/gms.py``).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

FLAG_HAS_BEST = 1
FLAG_RATIO_PASS = 2
FLAG_NO_SECOND = 4
FLAG_DEGENERATE_LINE = 8
FLAG_MUTUAL = 16
BOUNDARY_BAND = 1e-9

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.oracle_num_threads.restype = C.c_int
        lib.oracle_point_line_distance.restype = C.c_double
        lib.oracle_point_line_distance.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double]
        lib.oracle_candidates.restype = C.c_int
        lib.oracle_candidates.argtypes = [C.c_int64, P, C.c_int64, P, P, P, C.c_double,
                                          P, P, P, P, P, P, P]
        lib.oracle_match.restype = C.c_int
        lib.oracle_match.argtypes = [C.c_int64, P, C.c_int64, P, P, P, C.c_double,
                                     C.c_int, C.c_int, P, P, C.c_int, C.c_int, C.c_int,
                                     P, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def point_line_distance(F, x1, y1, x2, y2) -> float:
    """Eq. 3 for one pair: distance of (x2, y2) to the epipolar line F (x1, y1, 1)^T."""
    F = _f64(F, (9,))
    return float(_load().oracle_point_line_distance(_p(F), x1, y1, x2, y2))


def _eps_args(eps, n):
    if eps is None:
        raise ValueError("eps required")
    if np.ndim(eps) == 0:
        return None, float(eps)
    e = _f64(eps)
    if e.shape != (n,):
        raise ValueError("per-keypoint eps must have shape (n,)")
    return e, 0.0


def candidates(xy1, xy2, F, eps):
    """Exact candidate sets by brute force (Eq. 4).

    Returns dict(offsets (m+1,), idx, boffsets, bidx, degenerate (m,)) where
    row i of (offsets, idx) is C_i ascending in j and row i of (boffsets, bidx)
    lists the pairs with |dist - eps_j| < 1e-9 px (decided in FP64 by Eq. 4
    like every other pair, but reported apart).
    """
    lib = _load()
    xy1 = _f64(xy1)
    xy2 = _f64(xy2)
    F = _f64(F, (9,))
    m, n = xy1.shape[0], xy2.shape[0]
    e, es = _eps_args(eps, n)
    counts = np.zeros(m, np.int64)
    bcounts = np.zeros(m, np.int64)
    deg = np.zeros(m, np.uint8)
    lib.oracle_candidates(m, _p(xy1), n, _p(xy2), _p(F), _p(e), es, _p(counts), _p(bcounts),
                          None, None, None, None, _p(deg))
    off = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    boff = np.zeros(m + 1, np.int64)
    np.cumsum(bcounts, out=boff[1:])
    idx = np.zeros(max(int(off[-1]), 1), np.int32)
    bidx = np.zeros(max(int(boff[-1]), 1), np.int32)
    lib.oracle_candidates(m, _p(xy1), n, _p(xy2), _p(F), _p(e), es, None, None,
                          _p(off), _p(idx), _p(boff), _p(bidx), _p(deg))
    return dict(offsets=off, idx=idx[: off[-1]], boffsets=boff, bidx=bidx[: boff[-1]],
                degenerate=deg)


def _row_bytes(kind, dim):
    return dim if kind == 0 else dim // 8 if kind == 2 else 4 * dim


def match(xy1, xy2, F, eps, desc1, desc2, kind, dim, ratio=(4, 5), exclude_boundary=False):
    """Candidate-restricted matching with best / second best and the ratio test.

    Returns dict(best, second (int32, -1 if none), best_d, second_d (float64,
    squared L2 or Hamming count, +inf if none), flags (uint8), ncand (int64)).
    """
    lib = _load()
    xy1 = _f64(xy1)
    xy2 = _f64(xy2)
    F = _f64(F, (9,))
    m, n = xy1.shape[0], xy2.shape[0]
    e, es = _eps_args(eps, n)
    rb = _row_bytes(kind, dim)
    d1 = np.ascontiguousarray(desc1)
    d2 = np.ascontiguousarray(desc2)
    if d1.nbytes != m * rb or d2.nbytes != n * rb:
        raise ValueError("descriptor arrays do not match kind/dim")
    out = dict(best=np.empty(m, np.int32), second=np.empty(m, np.int32),
               best_d=np.empty(m, np.float64), second_d=np.empty(m, np.float64),
               flags=np.empty(m, np.uint8), ncand=np.empty(m, np.int64))
    lib.oracle_match(m, _p(xy1), n, _p(xy2), _p(F), _p(e), es, int(kind), int(dim),
                     _p(d1), _p(d2), int(ratio[0]), int(ratio[1]), int(bool(exclude_boundary)),
                     _p(out["best"]), _p(out["second"]), _p(out["best_d"]), _p(out["second_d"]),
                     _p(out["flags"]), _p(out["ncand"]))
    return out


def match_mutual(xy1, xy2, F, eps2, eps1, desc1, desc2, kind, dim, ratio=(4, 5), exclude_boundary=False):
    """Both directions and the cross-check.  Returns (forward, reverse): the
    dicts of ``match`` for image 1 -> 2 (F, tolerance eps2 of the image-2
    keypoints) and image 2 -> 1 (F^T, tolerance eps1 of the image-1
    keypoints), with FLAG_MUTUAL added to every row whose best match has that
    row as its own best."""
    F = _f64(F, (3, 3))
    fw = match(xy1, xy2, F, eps2, desc1, desc2, kind, dim, ratio, exclude_boundary)
    rv = match(xy2, xy1, F.T.copy(), eps1, desc2, desc1, kind, dim, ratio, exclude_boundary)
    for a, b in ((fw, rv), (rv, fw)):
        for i, j in enumerate(a["best"]):
            if j >= 0 and b["best"][j] == i:
                a["flags"][i] |= FLAG_MUTUAL
    return fw, rv


def match_scene(sc, ratio=(4, 5), exclude_boundary=False, eps=None):
    return match(sc.xy1, sc.xy2, sc.F, sc.eps if eps is None else eps, sc.desc1, sc.desc2,
                 sc.kind, sc.dim, ratio=ratio, exclude_boundary=exclude_boundary)


def epipole(F):
    """e2 = null(F^T) (Algorithm 1): right singular vector of F^T for the smallest
    singular value, homogeneous, scaled to unit norm with e_w >= 0."""
    F = _f64(F, (3, 3))
    _, s, vt = np.linalg.svd(F.T)
    e = vt[-1]
    if e[2] < 0 or (e[2] == 0 and (e[0] < 0 or (e[0] == 0 and e[1] < 0))):
        e = -e
    return e / np.linalg.norm(e)


def intervals(F, xy2, eps):
    """Angular interval (theta_j, delta_j) of every reference keypoint (Sec. 4.2).

    theta_j = atan2(y_j - y_e, x_j - x_e) mod pi (Eq. theta and the reduced
    domain [0, pi)); delta_j = asin(eps_j / ||p_j - e||) (Eq. delta); keypoints
    with ||p_j - e|| <= eps_j get delta = pi/2, i.e. the full domain
    (Algorithm 1).  Returns (theta, delta, e_xy) or raises for an epipole at
    infinity (e_w == 0), where the intervals are undefined.
    """
    e = epipole(F)
    if e[2] == 0.0:
        raise ValueError("epipole at infinity: angular intervals undefined")
    ex, ey = e[0] / e[2], e[1] / e[2]
    xy2 = _f64(xy2)
    n = xy2.shape[0]
    eps = np.broadcast_to(np.asarray(eps, np.float64), (n,))
    theta = np.empty(n)
    delta = np.empty(n)
    for j in range(n):
        dx, dy = xy2[j, 0] - ex, xy2[j, 1] - ey
        d = math.hypot(dx, dy)
        th = math.atan2(dy, dx) % math.pi
        if th >= math.pi:
            th = 0.0
        theta[j] = th
        delta[j] = math.pi / 2 if d <= eps[j] else math.asin(eps[j] / d)
    return theta, delta, np.array([ex, ey])
