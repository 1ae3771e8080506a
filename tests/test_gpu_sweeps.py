"""Exactness across the tolerance and pose-noise ranges of the paper's
sweeps (Sec. 5.3: tolerances up to 200 px; Sec. 5.5: pose noise up to level
3.3 at 200 px), and the brute-force limit of a tolerance covering the image."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import check_candidates, check_matches

pytestmark = pytest.mark.gpu

FORM_PLAIN, FORM_BANDED = 1, 2


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


def run(mt, sc, F=None, eps=None, form=0, csr=False, cap=None):
    d = mt.to_device(sc)
    if F is not None:
        d["F"] = mt.torch.as_tensor(np.ascontiguousarray(F).reshape(9)).to(mt.device)
    mt.set_params(form=form)
    try:
        o = mt.match(d["xy1"], d["xy2"], d["F"], d["eps"] if eps is None else eps, d["desc1"], d["desc2"],
                     d["kind"], d["dim"], d["width"], d["height"], csr=csr, cand_capacity=cap)
    finally:
        mt.set_params(form=0)
    return {k: v.cpu().numpy() for k, v in o.items()}


def with_(sc, F=None, eps=None):
    return synth.Scene(xy1=sc.xy1, xy2=sc.xy2, F=sc.F if F is None else F, eps=sc.eps if eps is None else eps,
                       desc1=sc.desc1, desc2=sc.desc2, kind=sc.kind, dim=sc.dim, width=sc.width,
                       height=sc.height, gt=sc.gt, meta=sc.meta)


@pytest.mark.parametrize("pose", ["inside", "far", "infinity"])
@pytest.mark.parametrize("eps", [20.0, 50.0, 200.0])
def test_large_tolerance_both_forms(mt, pose, eps):
    sc = synth.config2(pose, eps, scale=0.2)
    ref = oracle.match_scene(sc)
    out = run(mt, sc, form=FORM_PLAIN, csr=True)
    check_candidates(out, sc)
    check_matches(out, sc, ref=ref)
    check_matches(run(mt, sc, form=FORM_BANDED), sc, ref=ref)


@pytest.mark.parametrize("level", [0.5, 1.0, 2.0, 3.3])
def test_noisy_pose_at_200px(mt, level):
    sc = synth.config2("far" if level < 2 else "inside", 200.0, scale=0.2)
    F = synth.perturb_pose(sc, level, seed=int(level * 10))
    s2 = with_(sc, F=F)
    ref = oracle.match_scene(s2)
    out = run(mt, sc, F=F, form=FORM_PLAIN, csr=True)
    check_candidates(out, s2)
    check_matches(out, s2, ref=ref)
    check_matches(run(mt, sc, F=F, form=FORM_BANDED), s2, ref=ref)


def test_full_size_200px_sampled_rows(mt):
    """25,000 keypoints per image at 200 px (the tolerance sweep's largest
    setting): every output of 600 sampled queries against the oracle."""
    sc = synth.config2("inside", 200.0, seed=5, scale=25000 / 16384)
    out = run(mt, sc)
    rows = np.sort(np.random.default_rng(0).choice(sc.m, 600, replace=False))
    ref = oracle.match(sc.xy1[rows], sc.xy2, sc.F, sc.eps, sc.desc1[rows], sc.desc2, sc.kind, sc.dim)
    sub = with_(sc)
    sub.xy1, sub.desc1 = sc.xy1[rows], sc.desc1[rows]
    check_matches({k: v[rows] for k, v in out.items()}, sub, ref=ref)


def test_tolerance_covering_the_image_is_brute_force(mt):
    """eps far beyond the image: every reference is a candidate, so the best
    match is the exhaustive nearest neighbour (numpy over all pairs)."""
    sc = synth.config1(seed=2)
    for form in (FORM_PLAIN, FORM_BANDED):
        out = run(mt, sc, eps=1e7, form=form)
        d = ((sc.desc1[:, None, :].astype(np.int64) - sc.desc2[None, :, :].astype(np.int64)) ** 2).sum(-1)
        order = np.argsort(d, axis=1, kind="stable")  # ties: lower index first
        assert np.array_equal(out["best"], order[:, 0])
        assert np.array_equal(out["second"], order[:, 1])
        assert np.array_equal(out["best_d"], d[np.arange(sc.m), order[:, 0]].astype(np.float32))


@pytest.mark.parametrize("count", [50000])
def test_scalability_size_sampled_rows(mt, count):
    """50,000 keypoints per image at 50 px (the largest size of the paper's
    scalability runs, Sec. 5.4), in both forms: every output of 500 sampled
    queries against the oracle."""
    sc = synth.config2("far", 50.0, seed=9, scale=count / 16384)
    rows = np.sort(np.random.default_rng(1).choice(sc.m, 500, replace=False))
    ref = oracle.match(sc.xy1[rows], sc.xy2, sc.F, sc.eps, sc.desc1[rows], sc.desc2, sc.kind, sc.dim)
    sub = with_(sc)
    sub.xy1, sub.desc1 = sc.xy1[rows], sc.desc1[rows]
    for form in (FORM_PLAIN, FORM_BANDED):
        out = run(mt, sc, form=form)
        check_matches({k: v[rows] for k, v in out.items()}, sub, ref=ref)
