"""egm_match_pair_static: matching for callers that cannot allocate device memory.

The entry point keeps all of its scratch in a fixed device array inside the
library instead of allocating it, so code that runs under another owner's
allocator, or in loops that must not stall in cudaMalloc / cudaFree, can still
match a pair.  This file runs last so that a failure here comes after every
other test; it must pass alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

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
    got = mt._alloc_out(sc.m, csr, cap)
    for o in got.values():
        o.fill_(-7 if o.dtype != torch.uint8 else 77)
    stream = torch.cuda.current_stream()
    assert _call_static(mt, _egm, pair, mt._out_struct(got, cap), stream) == 0
    torch.cuda.synchronize()
    # integer descriptors: distances are exact integers on both paths
    for k in ("best", "second", "flags", "best_d", "second_d"):
        assert torch.equal(got[k], ref[k]), k
    if csr:
        n = int(ref["cand_total"].item())
        assert int(got["cand_total"].item()) == n
        assert torch.equal(got["cand_offsets"], ref["cand_offsets"])
        assert torch.equal(got["cand_idx"][:n], ref["cand_idx"][:n])


def test_static_scratch_matches_match_pair_twice(env):
    mt, _egm, torch = env
    # two calls in a row on different pairs: the second must not see the first's state
    _compare(mt, _egm, torch, synth.config2("inside", 2.0), csr=True)
    _compare(mt, _egm, torch, synth.config2("far", 4.0, scale=0.5), csr=False)


def test_static_scratch_rejects_oversized_pairs(env):
    mt, _egm, torch = env
    sc = synth.config1(scale=0.25)
    d = mt.to_device(sc)
    big = torch.zeros((16385, 2), dtype=torch.float64, device=mt.device)
    pair = mt.make_pair(d["xy1"], big, d["F"], 2.0, None, None, 0, 128, 640, 480)
    out = mt._alloc_out(sc.m, True, 16)
    assert _call_static(mt, _egm, pair, mt._out_struct(out, 16), torch.cuda.current_stream()) == -4
