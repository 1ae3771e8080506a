"""egm_match_pair_static: matching for callers that cannot allocate device memory.

The entry point keeps all of its scratch in a fixed device array inside the
library instead of allocating it, so code that runs under another owner's
allocator, or in loops that must not stall in cudaMalloc / cudaFree, can still
match a pair.  Each case calls it twice in a row and compares it with
egm_match_pair (the context path) and with the CPU oracle.  This file runs
last so that a failure here comes after every other test; it must pass alone
in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_2603_18401_gb300 import Matcher, _egm

    mt = Matcher(0)
    yield mt, _egm, torch
    torch.cuda.synchronize()
    mt.close()


def _call_static(mt, _egm, pair, out_struct, stream):
    p = _egm.egm_params()
    mt.lib.egm_default_params(C.byref(p))
    return mt.lib.egm_match_pair_static(C.byref(pair), C.byref(out_struct), C.byref(p),
                                        C.c_void_p(stream.cuda_stream))


def _compare(mt, _egm, torch, sc, csr):
    d = mt.to_device(sc)
    pair = mt.make_pair(d["xy1"], d["xy2"], d["F"], d["eps"], d["desc1"], d["desc2"], d["kind"], d["dim"],
                        d["width"], d["height"])
    cap = 64 * sc.m
    ref = mt._alloc_out(sc.m, csr, cap)
    assert mt.egm_match_pair(pair, mt._out_struct(ref, cap)) == 0
    stream = torch.cuda.current_stream()
    outs = []
    for call in range(2):
        got = mt._alloc_out(sc.m, csr, cap)
        for o in got.values():
            o.fill_(-7 if o.dtype != torch.uint8 else 77)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call_static(mt, _egm, pair, mt._out_struct(got, cap), stream) == 0
        torch.cuda.synchronize()
        if call == 1:
            # the device's free memory is unchanged by a call after the first
            assert torch.cuda.mem_get_info()[0] == free0
        outs.append(got)
    for got in outs:
        # integer descriptors: distances are exact integers on both paths
        for k in ("best", "second", "flags", "best_d", "second_d"):
            assert torch.equal(got[k], ref[k]), k
        if csr:
            n = int(ref["cand_total"].item())
            assert int(got["cand_total"].item()) == n
            assert torch.equal(got["cand_offsets"], ref["cand_offsets"])
            assert torch.equal(got["cand_idx"][:n], ref["cand_idx"][:n])
    # and directly against the oracle
    got = {k: v.cpu().numpy() for k, v in outs[-1].items()}
    want = oracle.match_scene(sc)
    bad = np.zeros(sc.m, bool)
    for k in ("best", "second", "flags"):
        bad |= got[k] != want[k]
    if bad.any():
        # only queries with a pair within 1e-9 px of eps may differ: they must
        # then equal the oracle's answer with those pairs excluded
        alt = oracle.match_scene(sc, exclude_boundary=True)
        for k in ("best", "second", "flags"):
            assert np.array_equal(got[k][bad], alt[k][bad]), k
    ok = ~bad & (want["best"] >= 0)
    assert np.array_equal(got["best_d"][ok], want["best_d"][ok].astype(np.float32))
    if csr:
        c = oracle.candidates(sc.xy1, sc.xy2, sc.F, sc.eps)
        n = int(got["cand_total"][0])
        assert np.array_equal(got["cand_offsets"], c["offsets"])
        assert np.array_equal(got["cand_idx"][:n], c["idx"])


def test_static_scratch_matches_match_pair_twice(env):
    mt, _egm, torch = env
    # two pairs one after the other: the second must not see the first's state
    _compare(mt, _egm, torch, synth.config2("inside", 2.0), csr=True)
    _compare(mt, _egm, torch, synth.config2("far", 4.0, scale=0.5), csr=False)


def test_static_scratch_binary_and_per_keypoint_eps(env):
    mt, _egm, torch = env
    sc = synth.config3(seed=4, npairs=2, scale=0.4)[1]          # 256-bit binary descriptors
    assert sc.kind == synth.DESC_BIN256
    _compare(mt, _egm, torch, sc, csr=True)
    sc = synth.config1(seed=2)
    sc.eps = np.random.default_rng(3).uniform(0.5, 6.0, sc.n)   # one tolerance per image-2 keypoint
    _compare(mt, _egm, torch, sc, csr=True)


def test_static_scratch_rejects_oversized_pairs(env):
    mt, _egm, torch = env
    sc = synth.config1(scale=0.25)
    d = mt.to_device(sc)
    big = torch.zeros((16385, 2), dtype=torch.float64, device=mt.device)
    pair = mt.make_pair(d["xy1"], big, d["F"], 2.0, None, None, 0, 128, 640, 480)
    out = mt._alloc_out(sc.m, True, 16)
    assert _call_static(mt, _egm, pair, mt._out_struct(out, 16), torch.cuda.current_stream()) == -4
