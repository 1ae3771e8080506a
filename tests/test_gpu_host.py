"""Host-memory entry points: egm_match_batch_host (uploads overlapped with
matching) and egm_match_pair_host give the device path's outputs."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KEYS = (("best", np.int32), ("second", np.int32), ("best_d", np.float32), ("second_d", np.float32),
        ("flags", np.uint8))


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


def host_structs(mt, sc, pinned, eps_array=None):
    """egm_pair / egm_out with host pointers; returns (pair, out, buffers)."""
    from paper_2603_18401_gb300 import _egm

    torch = mt.torch

    def arr(a):
        a = np.ascontiguousarray(a)
        return torch.from_numpy(a).pin_memory().numpy() if pinned else a.copy()

    keep = {k: arr(getattr(sc, k)) for k in ("xy1", "xy2", "desc1", "desc2")}
    keep["F"] = arr(np.asarray(sc.F, np.float64).reshape(9))
    if eps_array is not None:
        keep["eps2"] = arr(np.asarray(eps_array, np.float64))
    outs = {k: arr(np.zeros(sc.m, dt)) for k, dt in KEYS}
    hp = lambda a: a.ctypes.data_as(C.c_void_p)
    p = _egm.egm_pair()
    p.xy1, p.xy2, p.F = hp(keep["xy1"]), hp(keep["xy2"]), hp(keep["F"])
    p.eps2 = hp(keep["eps2"]) if eps_array is not None else None
    p.eps_scalar = float(sc.eps) if eps_array is None else 0.0
    p.desc1, p.desc2 = hp(keep["desc1"]), hp(keep["desc2"])
    p.m, p.n, p.kind, p.dim, p.width, p.height = sc.m, sc.n, sc.kind, sc.dim, sc.width, sc.height
    o = _egm.egm_out()
    o.best, o.second, o.best_d, o.second_d, o.flags = (hp(outs["best"]), hp(outs["second"]), hp(outs["best_d"]),
                                                       hp(outs["second_d"]), hp(outs["flags"]))
    return p, o, (keep, outs)


def device_outputs(mt, sc, eps_array=None):
    d = mt.to_device(sc)
    eps = d["eps"] if eps_array is None else mt.torch.as_tensor(eps_array).to(mt.device)
    o = mt.match(d["xy1"], d["xy2"], d["F"], eps, d["desc1"], d["desc2"], d["kind"], d["dim"], d["width"],
                 d["height"])
    return {k: v.cpu().numpy() for k, v in o.items()}


def scenes():
    rng = np.random.default_rng(3)
    out = [(synth.config1(), None), (synth.config2("far", 4.0, scale=0.3), None),
           (synth.config3(seed=2, npairs=2, scale=0.2)[1], None),
           (synth.config4(seed=0, npairs=1, scale=0.1)[0], None)]
    sc = synth.config2("inside", 2.0, scale=0.2)
    out.append((sc, rng.uniform(0.5, 5.0, sc.n)))
    return out


@pytest.mark.parametrize("pinned", [True, False])
def test_batch_host_equals_device_path(mt, pinned):
    items = scenes()
    structs = [host_structs(mt, sc, pinned, e) for sc, e in items]
    assert mt.egm_match_batch_host([s[0] for s in structs], [s[1] for s in structs]) == 0
    for (sc, e), (_, _, (_, outs)) in zip(items, structs):
        ref = device_outputs(mt, sc, e)
        for k, _ in KEYS:
            assert np.array_equal(outs[k], ref[k]), k


def test_pair_host_equals_device_path(mt):
    for sc, e in scenes()[:3]:
        p, o, (_, outs) = host_structs(mt, sc, True, e)
        assert mt.egm_match_pair_host(p, o) == 0
        ref = device_outputs(mt, sc, e)
        for k, _ in KEYS:
            assert np.array_equal(outs[k], ref[k]), k


def test_batch_host_rejects_candidate_lists_and_missing_descriptors(mt):
    from paper_2603_18401_gb300 import _egm

    sc = synth.config1(scale=0.1)
    p, o, keep = host_structs(mt, sc, False)
    offs = np.zeros(sc.m + 1, np.int64)
    o.cand_offsets = offs.ctypes.data_as(C.c_void_p)
    assert mt.egm_match_batch_host([p], [o]) == _egm.EGM_ERR_ARG
    p2, o2, keep2 = host_structs(mt, sc, False)
    p2.desc1 = None
    assert mt.egm_match_batch_host([p2], [o2]) == _egm.EGM_ERR_ARG
    assert mt.egm_match_batch_host([], []) == 0
    del keep, keep2
