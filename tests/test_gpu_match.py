"""Mutual matching (egm_match_mutual) and the compact match list
(egm_compact_matches) against the oracle, and matching recall on the
synthetic ground truth."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import _scene, check_matches

pytestmark = pytest.mark.gpu

FORM_AUTO, FORM_PLAIN, FORM_BANDED = 0, 1, 2
KEYS = ("best", "second", "flags", "best_d", "second_d")
RATIO, MUTUAL = 2, 16


@pytest.fixture(scope="module")
def mt():
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_2603_18401_gb300 import Matcher

    m = Matcher(0)
    yield m
    torch.cuda.synchronize()
    m.close()


def mutual(mt, sc, eps1, form=FORM_AUTO):
    torch = mt.torch
    d = mt.to_device(sc)
    e1 = eps1 if np.ndim(eps1) == 0 else torch.as_tensor(eps1, dtype=torch.float64).to(mt.device)
    mt.set_params(form=form)
    try:
        o = mt.match_mutual(d["xy1"], d["xy2"], d["F"], d["eps"], e1, d["desc1"], d["desc2"], d["kind"], d["dim"],
                            d["width"], d["height"])
    finally:
        mt.set_params(form=FORM_AUTO)
    return {k: v.cpu().numpy() for k, v in o.items()}, o


def check_mutual(out, sc, eps1):
    fw, rv = oracle.match_mutual(sc.xy1, sc.xy2, sc.F, sc.eps, eps1, sc.desc1, sc.desc2, sc.kind, sc.dim)
    m = sc.m
    check_matches({k: out[k][:m] for k in KEYS}, sc, ref=fw)
    rev = synth.Scene(xy1=sc.xy2, xy2=sc.xy1, F=np.ascontiguousarray(sc.F.T), eps=eps1, desc1=sc.desc2,
                      desc2=sc.desc1, kind=sc.kind, dim=sc.dim, width=sc.width, height=sc.height,
                      gt=np.zeros((0, 2), np.int64))
    check_matches({k: out[k][m:] for k in KEYS}, rev, ref=rv)
    return fw, rv


@pytest.mark.parametrize("form", [FORM_PLAIN, FORM_BANDED])
def test_mutual_config1_and_config2(mt, form):
    for sc in (synth.config1(), synth.config2("far", 2.0, scale=0.25), synth.config2("inside", 4.0, scale=0.25)):
        out, _ = mutual(mt, sc, 2.0 if np.ndim(sc.eps) == 0 else sc.eps, form)
        check_mutual(out, sc, 2.0)


def test_mutual_binary_float_and_per_keypoint_eps(mt):
    rng = np.random.default_rng(4)
    for sc in (synth.config3(seed=7, npairs=2, scale=0.1)[1], synth.config4(seed=1, npairs=1, scale=0.1)[0]):
        out, _ = mutual(mt, sc, 2.0)
        check_mutual(out, sc, 2.0)
    K = synth.intrinsics(500.0, 640, 480)
    F = synth.fundamental(K, K, synth.rotation([0, 1, 0], 6), [0.3, 0.05, 0.03])
    sc = _scene(rng.uniform([0, 0], [640, 480], (700, 2)), rng.uniform([0, 0], [640, 480], (900, 2)), F,
                rng.uniform(0.5, 6.0, 900), dim=128)
    eps1 = rng.uniform(0.5, 6.0, 700)
    out, _ = mutual(mt, sc, eps1)
    check_mutual(out, sc, eps1)


def test_mutual_rejects_inconsistent_pairs(mt):
    from paper_2603_18401_gb300 import EgmError, _egm
    import ctypes as C

    sc = synth.config1(scale=0.1)
    d = mt.to_device(sc)
    fwd = mt.make_pair(d["xy1"], d["xy2"], d["F"], 2.0, d["desc1"], d["desc2"], 0, 128)
    rev = mt.make_pair(d["xy1"], d["xy2"], d["F"], 2.0, d["desc1"], d["desc2"], 0, 128)  # sizes not swapped
    o = mt._alloc_out(2 * sc.m, False, 0)
    s = mt._out_struct(o, 0)
    if sc.m != sc.n:
        assert mt.lib.egm_match_mutual(mt.ctx, C.byref(fwd), C.byref(rev), C.byref(s)) == _egm.EGM_ERR_ARG
    assert mt.lib.egm_match_mutual(mt.ctx, None, C.byref(rev), C.byref(s)) == _egm.EGM_ERR_ARG
    del EgmError


@pytest.mark.parametrize("m", [0, 1, 777, 2048, 2049, 40000])
def test_compact_matches(mt, m):
    torch = mt.torch
    rng = np.random.default_rng(m)
    flags = rng.integers(0, 32, m).astype(np.uint8)
    best = rng.integers(-1, 1000, m).astype(np.int32)
    f, b = torch.as_tensor(flags).to(mt.device), torch.as_tensor(best).to(mt.device)
    for req in (0, RATIO, RATIO | MUTUAL, 31):
        qi, rj = mt.compact_matches(f, b, req)
        sel = np.nonzero((flags & req) == req)[0]
        assert np.array_equal(qi.cpu().numpy(), sel)
        assert np.array_equal(rj.cpu().numpy(), best[sel])


def recall_precision(qi, rj, gt):
    truth = set(map(tuple, gt.tolist()))
    got = set(zip(qi.tolist(), rj.tolist()))
    tp = len(got & truth)
    return tp / max(len(truth), 1), tp / max(len(got), 1)


def test_matching_recall_on_synthetic_ground_truth(mt):
    """Ratio-passing mutual matches against the scenes' true pairs: the GPU
    list equals the oracle's, so its recall and precision do too."""
    for sc in (synth.config1(), synth.config2("inside", 2.0), synth.config2("far", 2.0)):
        out, dev = mutual(mt, sc, 2.0)
        qi, rj = mt.compact_matches(dev["flags"][:sc.m], dev["best"][:sc.m], RATIO | MUTUAL)
        qi, rj = qi.cpu().numpy(), rj.cpu().numpy()
        fw, _ = oracle.match_mutual(sc.xy1, sc.xy2, sc.F, sc.eps, 2.0, sc.desc1, sc.desc2, sc.kind, sc.dim)
        sel = np.nonzero((fw["flags"] & (RATIO | MUTUAL)) == (RATIO | MUTUAL))[0]
        assert np.array_equal(qi, sel) and np.array_equal(rj, fw["best"][sel])
        rec, prec = recall_precision(qi, rj, sc.gt)
        assert rec > 0.85 and prec > 0.97, (rec, prec)


# ------------------------------------------------------------------ GMS
def gms_both(mt, xy1, xy2, best, flags, size1, size2, require=1, grid=20, alpha=6.0):
    """egm_gms on the device and the oracle on the same inputs: identical flags."""
    from oracle import gms as ogms

    torch = mt.torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(mt.device)
    f = dev(flags)
    mt.gms(dev(xy1), dev(xy2), dev(best.astype(np.int32)), f, size1, size2, require, grid, alpha)
    got = f.cpu().numpy()
    want = ogms.gms(xy1, xy2, best, flags, size1, size2, require=require, grid=grid, alpha=alpha)
    assert np.array_equal(got, want), (int((got != want).sum()), grid, alpha, require)
    return got


def test_gms_on_matches_of_the_configs(mt):
    for sc in (synth.config1(), synth.config2("inside", 2.0), synth.config2("far", 4.0),
               synth.config2("infinity", 1.0)):
        o = run_match(mt, sc)
        size = (sc.width, sc.height)
        for req, grid, alpha in ((1, 20, 6.0), (RATIO, 20, 6.0), (1, 7, 4.5), (1, 48, 6.0), (1, 1, 2.0)):
            got = gms_both(mt, sc.xy1, sc.xy2, o["best"], o["flags"], size, size, req, grid, alpha)
        # GMS alone on the nearest neighbours (the paper's default filter):
        # far more precise than its input, still most of the true pairs
        got = gms_both(mt, sc.xy1, sc.xy2, o["best"], o["flags"], size, size)
        truth = set(map(tuple, sc.gt.tolist()))
        prec = lambda rows: np.mean([(i, o["best"][i]) in truth for i in rows])
        kept = np.nonzero(got & 32)[0]
        inputs = np.nonzero(o["best"] >= 0)[0]
        assert len(kept) > 0.5 * len(truth) and prec(kept) > prec(inputs) + 0.15, (len(kept), prec(kept))


def run_match(mt, sc):
    d = mt.to_device(sc)
    o = mt.match(d["xy1"], d["xy2"], d["F"], d["eps"], d["desc1"], d["desc2"], d["kind"], d["dim"], d["width"],
                 d["height"])
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("m", [0, 1, 5, 1000, 70000])
def test_gms_edge_cases(mt, m):
    rng = np.random.default_rng(m + 3)
    n = max(m // 2, 1)
    # clustered motion plus noise, points outside the image, duplicates, invalid rows
    xy1 = rng.uniform([-50, -50], [1100, 800], (m, 2))
    xy2 = rng.uniform([-50, -50], [900, 700], (n, 2))
    best = rng.integers(-2, n + 2, m)
    if m >= 1000:
        k = m // 3
        xy1[:k] = rng.uniform([0, 0], [1000, 700], (k, 2))
        best[:k] = np.arange(k) % n
        xy2[best[:k]] = xy1[:k] * 0.8 + 20.0
        xy1[k:k + 50] = xy1[0]
    flags = rng.integers(0, 64, m).astype(np.uint8)
    for req in (0, 1, 3):
        gms_both(mt, xy1, xy2, best, flags, (1024, 768), (800, 600), req)
    gms_both(mt, xy1, xy2, best, flags, (1024, 768), (800, 600), 0, 13, 3.0)


def test_gms_rejects_bad_arguments(mt):
    from paper_2603_18401_gb300 import EgmError

    torch = mt.torch
    xy = torch.zeros((4, 2), dtype=torch.float64, device=mt.device)
    best = torch.zeros(4, dtype=torch.int32, device=mt.device)
    f = torch.zeros(4, dtype=torch.uint8, device=mt.device)
    for kw in (dict(grid=0), dict(grid=49), dict(alpha=0.0), dict(alpha=float("inf")), dict(size1=(0, 10))):
        args = dict(size1=(10, 10), size2=(10, 10), grid=20, alpha=6.0)
        args.update(kw)
        with pytest.raises(EgmError):
            mt.gms(xy, xy, best, f, args["size1"], args["size2"], 1, args["grid"], args["alpha"])


def test_gms_batch_equals_per_pair_oracle(mt):
    """egm_gms_batch over pairs of different sizes (one empty) in one call:
    every pair's flags equal the oracle's for that pair alone."""
    from oracle import gms as ogms

    torch = mt.torch
    rng = np.random.default_rng(21)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(mt.device)
    items, want = [], []
    for k, m in enumerate([3000, 0, 800, 12000, 1]):
        n = max(m, 5)
        xy1 = rng.uniform([0, 0], [1200, 900], (m, 2))
        xy2 = rng.uniform([0, 0], [1000, 800], (n, 2))
        best = rng.integers(-1, n, m)
        kk = m // 2
        xy2[best[:kk]] = xy1[:kk] * 0.7 + 30.0   # a coherent part
        flags = rng.integers(0, 64, m).astype(np.uint8)
        size1, size2 = (1200, 900), (1000, 800)
        want.append(ogms.gms(xy1, xy2, best, flags, size1, size2, require=1, grid=20, alpha=6.0))
        items.append((dev(xy1), dev(xy2), dev(best.astype(np.int32)), dev(flags), size1, size2))
    mt.gms_batch(items, require=1, grid=20, alpha=6.0)
    for (_, _, _, f, _, _), w in zip(items, want):
        assert np.array_equal(f.cpu().numpy(), w)


def test_mutual_from_one_pair_equals_two_pair_call(mt):
    """egm_match_mutual_pair forms the reverse direction (F^T on the device,
    image-1 tolerances) itself: its outputs equal egm_match_mutual's with the
    caller-built reverse pair and the oracle's cross-check, with scalar and
    per-keypoint image-1 tolerances, on consecutive calls of different pairs."""
    torch = mt.torch
    rng = np.random.default_rng(31)
    for sc, eps1 in ((synth.config1(seed=6), 2.0), (synth.config2("far", 2.0, scale=0.25), None)):
        if eps1 is None:
            eps1 = rng.uniform(0.5, 4.0, sc.m)
        d = mt.to_device(sc)
        e1 = eps1 if np.ndim(eps1) == 0 else torch.as_tensor(eps1, dtype=torch.float64).to(mt.device)
        o = mt.match_mutual_pair(d["xy1"], d["xy2"], d["F"], d["eps"], e1, d["desc1"], d["desc2"], d["kind"],
                                 d["dim"], d["width"], d["height"])
        got = {k: v.cpu().numpy() for k, v in o.items()}
        ref, _ = mutual(mt, sc, eps1)
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), k
        check_mutual(got, sc, eps1)
