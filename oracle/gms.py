"""Grid-based motion statistics (GMS) filter, FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline); the CUDA
library never imports it and shares no code with it.

The paper filters its guided matches with GMS (Bian et al., CVPR 2017), with
the neighbour threshold fixed to 6 (Sec. 5.1, "Baselines"; Sec. 4.3 names GMS
as the filter suited to guided matching).  GMS itself is written here from the
published algorithm:

1. Both images are cut into G x G cells.  For a grid shift (sx, sy) in
   {0, 1/2}^2 the image-1 cell of x is floor(x * G / W1 + sx) (clamped to
   0 .. G, so a shifted grid has G + 1 columns); the image-2 cell of x is
   floor(x * G / W2) (clamped to 0 .. G - 1).  Same for y.
2. M[c][d] counts the input matches from image-1 cell c to image-2 cell d,
   N[c] the input matches in image-1 cell c.
3. For every image-1 cell c with N[c] > 0, d*(c) is the image-2 cell with the
   most matches from c (the lowest index dy * G + dx on ties).
4. S(c) sums M[c + o][d*(c) + o] over the 3 x 3 offsets o, skipping cells
   outside either grid; the threshold is alpha * sqrt(n(c)) with n(c) the sum
   of N over the (in-grid) 3 x 3 neighbourhood of c divided by 9, the mean
   count of the nine cells.
5. Under this shift a match from c to d is kept iff d == d*(c) and
   S(c) > alpha * sqrt(n(c)).
6. The result is the union over the four shifts.

The input matches are the rows i whose best[i] is a valid index and whose
flags contain every bit of `require`.  The threshold is evaluated in FP64 as
alpha * sqrt(sum / 9) (one rounding per operation).
"""
from __future__ import annotations

import numpy as np

FLAG_GMS = 32
SHIFTS = ((0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5))


def _cells(v, g, size, shift, top):
    """floor(v * g / size + shift), clamped to [0, top] (step 1)."""
    t = np.floor((np.asarray(v, np.float64) * float(g)) / float(size) + shift)
    t = np.where(np.isnan(t), 0.0, t)
    return np.clip(t, 0, top).astype(np.int64)


def gms_one_shift(xy1, xy2, qi, rj, size1, size2, grid, alpha, shift):
    """Keep mask of the matches (qi[k], rj[k]) under one grid shift (steps 1-5)."""
    G = int(grid)
    G1 = G + 1
    c = _cells(xy1[qi, 1], G, size1[1], shift[1], G) * G1 + _cells(xy1[qi, 0], G, size1[0], shift[0], G)
    d = _cells(xy2[rj, 1], G, size2[1], 0.0, G - 1) * G + _cells(xy2[rj, 0], G, size2[0], 0.0, G - 1)
    M = np.zeros((G1 * G1, G * G), np.int64)
    np.add.at(M, (c, d), 1)
    N = M.sum(axis=1)
    best = np.full(G1 * G1, -1, np.int64)
    for cell in range(G1 * G1):
        if N[cell] == 0:
            continue
        dstar = int(np.argmax(M[cell]))  # first maximum: lowest index
        cx, cy = cell % G1, cell // G1
        dx, dy = dstar % G, dstar // G
        S = 0
        total = 0
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                ax, ay = cx + ox, cy + oy
                if not (0 <= ax < G1 and 0 <= ay < G1):
                    continue
                total += int(N[ay * G1 + ax])
                bx, by = dx + ox, dy + oy
                if 0 <= bx < G and 0 <= by < G:
                    S += int(M[ay * G1 + ax, by * G + bx])
        if float(S) > float(alpha) * np.sqrt(float(total) / 9.0):
            best[cell] = dstar
    return best[c] == d


def gms(xy1, xy2, best, flags, size1, size2, require=1, grid=20, alpha=6.0):
    """flags with FLAG_GMS set on the input matches GMS keeps and cleared
    elsewhere (step 6: union over the four shifts)."""
    xy1 = np.asarray(xy1, np.float64).reshape(-1, 2)
    xy2 = np.asarray(xy2, np.float64).reshape(-1, 2)
    best = np.asarray(best, np.int64)
    flags = np.asarray(flags, np.uint8)
    n = xy2.shape[0]
    sel = (best >= 0) & (best < n) & ((flags & require) == require)
    qi = np.nonzero(sel)[0]
    rj = best[qi]
    keep = np.zeros(qi.shape[0], bool)
    for s in SHIFTS:
        keep |= gms_one_shift(xy1, xy2, qi, rj, size1, size2, grid, alpha, s)
    out = flags & np.uint8(0xFF ^ FLAG_GMS)
    out[qi[keep]] |= np.uint8(FLAG_GMS)
    return out
