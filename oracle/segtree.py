"""CPU baseline: the paper's centred segment tree (Sec. 4.4) on the host
cores, in plain C with OpenMP (``segtree.c``).

TEST AND BENCHMARK INFRASTRUCTURE ONLY: the benchmark times it beside the
brute-force oracle; the tests check it against the oracle.  ``exact=False`` is
the paper's method as described (interval stabbing only); ``exact=True``
widens the intervals by a proven pad and applies the point-to-line test of
Eq. 3 / Eq. 4 to every candidate, so its sets equal the brute force.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _build.build()
        lib = C.CDLL(_build.SEG_LIB)
        vp, i64, d, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
        lib.segtree_num_threads.restype = C.c_int
        lib.segtree_candidates.restype = C.c_int
        lib.segtree_candidates.argtypes = [i64, vp, i64, vp, vp, vp, d, i32, i32, i32, vp, vp, vp]
        lib.segtree_match.restype = C.c_int
        lib.segtree_match.argtypes = [i64, vp, i64, vp, vp, vp, d, i32, i32, i32, i32, i32, vp, vp, i32, i32,
                                      vp, vp, vp, vp, vp, vp, vp]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return _load().segtree_num_threads()


def _eps(eps, n):
    if np.ndim(eps) == 0:
        return None, float(eps)
    e = np.ascontiguousarray(eps, np.float64)
    assert e.shape == (n,)
    return e, 0.0


def candidates(xy1, xy2, F, eps, width, height, exact=True):
    """CSR candidate sets (offsets [m + 1] int64, idx int32, ascending j)."""
    lib = _load()
    xy1 = np.ascontiguousarray(xy1, np.float64).reshape(-1, 2)
    xy2 = np.ascontiguousarray(xy2, np.float64).reshape(-1, 2)
    F = np.ascontiguousarray(F, np.float64).reshape(9)
    m, n = xy1.shape[0], xy2.shape[0]
    e, es = _eps(eps, n)
    counts = np.zeros(m, np.int64)
    st = lib.segtree_candidates(m, _p(xy1), n, _p(xy2), _p(F), _p(e), es, int(width), int(height), int(exact),
                                _p(counts), None, None)
    if st != 0:
        raise RuntimeError(f"segtree_candidates: {st}")
    off = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    idx = np.zeros(max(int(off[-1]), 1), np.int32)
    lib.segtree_candidates(m, _p(xy1), n, _p(xy2), _p(F), _p(e), es, int(width), int(height), int(exact), None,
                           _p(off), _p(idx))
    return {"offsets": off, "idx": idx[:off[-1]]}


def match(xy1, xy2, F, eps, desc1, desc2, kind, dim, width, height, exact=True, ratio=(4, 5)):
    """Outputs as the oracle's match(); also 'build_s' and 'match_s' (wall time)."""
    lib = _load()
    xy1 = np.ascontiguousarray(xy1, np.float64).reshape(-1, 2)
    xy2 = np.ascontiguousarray(xy2, np.float64).reshape(-1, 2)
    F = np.ascontiguousarray(F, np.float64).reshape(9)
    desc1 = np.ascontiguousarray(desc1)
    desc2 = np.ascontiguousarray(desc2)
    m, n = xy1.shape[0], xy2.shape[0]
    e, es = _eps(eps, n)
    out = {"best": np.empty(m, np.int32), "second": np.empty(m, np.int32), "best_d": np.empty(m, np.float64),
           "second_d": np.empty(m, np.float64), "flags": np.empty(m, np.uint8), "ncand": np.empty(m, np.int64)}
    secs = np.zeros(2, np.float64)
    st = lib.segtree_match(m, _p(xy1), n, _p(xy2), _p(F), _p(e), es, int(width), int(height), int(exact),
                           int(kind), int(dim), _p(desc1), _p(desc2), int(ratio[0]), int(ratio[1]), _p(out["best"]),
                           _p(out["second"]), _p(out["best_d"]), _p(out["second_d"]), _p(out["flags"]),
                           _p(out["ncand"]), _p(secs))
    if st != 0:
        raise RuntimeError(f"segtree_match: {st}")
    out["build_s"], out["match_s"] = float(secs[0]), float(secs[1])
    return out


def match_scene(sc, exact=True, ratio=(4, 5)):
    return match(sc.xy1, sc.xy2, sc.F, sc.eps, sc.desc1, sc.desc2, sc.kind, sc.dim, sc.width, sc.height,
                 exact=exact, ratio=ratio)
