"""Pins of the GMS oracle (oracle/gms.py) to values fixed by the GMS rule
itself (Bian et al. 2017; the paper's filter with threshold 6, Sec. 5.1):
closed-form thresholds on hand-built match sets, the tie rule, neighbour
support, and the two limiting motion fields."""
import numpy as np

from oracle import gms as G

W, H = 640, 480  # 20 x 20 cells of 32 x 24 px


def run(p1, p2, alpha=6.0, grid=20, flags=None, require=1):
    p1 = np.asarray(p1, np.float64).reshape(-1, 2)
    p2 = np.asarray(p2, np.float64).reshape(-1, 2)
    m = p1.shape[0]
    best = np.arange(m, dtype=np.int64)
    if flags is None:
        flags = np.ones(m, np.uint8)
    out = G.gms(p1, p2, best, flags, (W, H), (W, H), require=require, grid=grid, alpha=alpha)
    return (out & G.FLAG_GMS) != 0


def dupes(k, a=(123.5, 77.5), b=(400.5, 300.5)):
    return np.tile(a, (k, 1)), np.tile(b, (k, 1))


def test_duplicate_cluster_threshold_closed_form():
    # k identical matches: S = k and the neighbourhood holds k, so the rule is
    # k > alpha * sqrt(k / 9), i.e. k > alpha^2 / 9 (4 for alpha = 6)
    for k, want in ((1, False), (4, False), (5, True), (30, True)):
        assert run(*dupes(k)).tolist() == [want] * k, k
    for k, want in ((1, False), (2, True)):  # alpha = 3: k > 1
        assert run(*dupes(k), alpha=3.0).tolist() == [want] * k, k
    # alpha = 7.5: k > 6.25
    assert not run(*dupes(6), alpha=7.5).any() and run(*dupes(7), alpha=7.5).all()


def test_neighbour_support():
    # k matches A -> A' and k matches B -> B', B = A + one cell, B' = A' + one
    # cell: S = 2k against 6 sqrt(2k / 9), kept iff k > 2; alone, k = 3 fails
    A, A2 = (100.0, 100.0), (300.0, 200.0)
    B, B2 = (132.0, 100.0), (332.0, 200.0)
    for k, want in ((2, False), (3, True)):
        p1 = np.vstack([np.tile(A, (k, 1)), np.tile(B, (k, 1))])
        p2 = np.vstack([np.tile(A2, (k, 1)), np.tile(B2, (k, 1))])
        assert run(p1, p2).tolist() == [want] * (2 * k), k
    assert not run(*dupes(3, A, A2)).any()
    # the neighbour must move the same way: B -> B' - one cell gives no support
    p1 = np.vstack([np.tile(A, (3, 1)), np.tile(B, (3, 1))])
    p2 = np.vstack([np.tile(A2, (3, 1)), np.tile((268.0, 200.0), (3, 1))])
    assert not run(p1, p2).any()


def test_argmax_ties_to_the_lower_cell():
    # 10 matches to each of two far-apart cells: S = 10 > 6 sqrt(20 / 9) = 8.94
    # for the winner; the tie goes to the lower cell index (dy * 20 + dx)
    lo, hi = (40.0, 30.0), (600.0, 450.0)
    p1 = np.tile((320.5, 240.5), (20, 1))
    p2 = np.vstack([np.tile(hi, (10, 1)), np.tile(lo, (10, 1))])
    keep = run(p1, p2)
    assert keep.tolist() == [False] * 10 + [True] * 10
    # with 11 to the higher cell it wins
    p1 = np.tile((320.5, 240.5), (21, 1))
    p2 = np.vstack([np.tile(hi, (11, 1)), np.tile(lo, (10, 1))])
    assert run(p1, p2).tolist() == [True] * 11 + [False] * 10


def test_cell_aligned_translation_keeps_everything():
    # p2 = p1 + one cell in x and y: every cell maps to one cell in the
    # unshifted grid, with ~12 matches per cell all matches pass there
    rng = np.random.default_rng(0)
    p1 = rng.uniform([0, 0], [W - 32, H - 24], (4000, 2))
    p2 = p1 + np.array([32.0, 24.0])
    assert run(p1, p2).all()


def test_random_motion_keeps_nothing():
    # uniform random destinations: a cell's matches scatter, so S stays far
    # below the threshold (~6 sqrt(10) with ~10 matches per cell)
    rng = np.random.default_rng(1)
    p1 = rng.uniform([0, 0], [W, H], (4000, 2))
    p2 = rng.uniform([0, 0], [W, H], (4000, 2))
    assert not run(p1, p2).any()


def test_shift_union():
    # a cluster straddling a cell boundary of the unshifted grid is split
    # there into 3 + 3 (no support: neighbouring cells must move to
    # neighbouring cells, here both halves land in one cell) and whole in the
    # grid shifted by half a cell, where it passes (6 > 6 sqrt(6 / 9) = 4.9)
    p1 = np.vstack([np.tile((63.0, 100.0), (3, 1)), np.tile((65.0, 100.0), (3, 1))])
    p2 = np.vstack([np.tile((300.0, 200.0), (3, 1)), np.tile((302.0, 200.0), (3, 1))])
    keep = G.gms_one_shift(p1, p2, np.arange(6), np.arange(6), (W, H), (W, H), 20, 6.0, (0.0, 0.0))
    assert not keep.any()
    keep = G.gms_one_shift(p1, p2, np.arange(6), np.arange(6), (W, H), (W, H), 20, 6.0, (0.5, 0.0))
    assert keep.all()
    assert run(p1, p2).all()


def test_require_mask_and_invalid_rows():
    p1, p2 = dupes(8)
    flags = np.array([1, 1, 3, 3, 3, 3, 3, 3 | G.FLAG_GMS], np.uint8)
    keep = run(p1, p2, flags=flags, require=2)   # 6 inputs: 6 > 4
    assert keep.tolist() == [False, False] + [True] * 6
    flags = np.array([3, 3, 3, 3, 1, 1, 1, 1 | G.FLAG_GMS], np.uint8)
    keep = run(p1, p2, flags=flags, require=2)   # 4 inputs: fail; the stale bit is cleared
    assert not keep.any()
    best = np.array([0, -1, 5, 1], np.int64)      # -1 and out of range are not inputs
    out = G.gms(p1[:4], p2[:2], best, np.full(4, G.FLAG_GMS | 1, np.uint8), (W, H), (W, H))
    assert ((out & G.FLAG_GMS) == 0).all() and ((out & 1) == 1).all()
