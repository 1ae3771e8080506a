"""Exact epipolar-guided matching on GB300 (sm_103a).

Python face of libegm.so.  PyTorch supplies device memory and streams; every
step of the matching path runs in the library's CUDA kernels (see
include/egm.h).  Importing works without a GPU; creating a ``Matcher`` needs
the built library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes as C

from . import _egm
from ._egm import (EGM_DESC_BIN, EGM_DESC_F32_L2, EGM_DESC_U8_L2, EGM_ERR_CAPACITY,
                   EGM_FLAG_DEGENERATE_LINE, EGM_FLAG_GMS, EGM_FLAG_HAS_BEST, EGM_FLAG_MUTUAL, EGM_FLAG_NO_SECOND,
                   EGM_FLAG_RATIO_PASS, EGM_OK, EgmError, check, load)

__all__ = ["Matcher", "TolNet", "EgmError", "load", "row_bytes", "EGM_DESC_U8_L2", "EGM_DESC_F32_L2",
           "EGM_DESC_BIN", "EGM_FLAG_HAS_BEST", "EGM_FLAG_RATIO_PASS", "EGM_FLAG_NO_SECOND",
           "EGM_FLAG_DEGENERATE_LINE", "EGM_FLAG_MUTUAL", "EGM_FLAG_GMS"]


def row_bytes(kind: int, dim: int) -> int:
    return dim if kind == EGM_DESC_U8_L2 else 4 * dim if kind == EGM_DESC_F32_L2 else dim // 8


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Matcher:
    """One libegm context bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None, ratio=(4, 5)):
        import torch

        self.torch = torch
        self.lib = load()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        ctx = C.c_void_p()
        check(self.lib.egm_create(C.byref(ctx), device, C.c_void_p(stream.cuda_stream)), "egm_create")
        self.ctx = ctx
        p = _egm.egm_params()
        self.lib.egm_default_params(C.byref(p))
        p.ratio_num, p.ratio_den = int(ratio[0]), int(ratio[1])
        check(self.lib.egm_set_params(self.ctx, C.byref(p)), "egm_set_params")
        self._keep = []

    def close(self):
        if getattr(self, "ctx", None) is not None:
            self.lib.egm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- params
    def set_params(self, ratio=None, sync=None, form=None, band_tile=None, float_pass=None, timeout_check=None,
                   tune=None):
        """ratio (num, den); sync; form (EGM_FORM_*); band_tile (0: tuned, k > 0: shape k - 1);
        float_pass (EGM_FLOAT_PASS_*); timeout_check (1: the banded kernel's timeout path, no results);
        tune (1: timed choice of form and shape per regime, 0: fixed rule)."""
        p = _egm.egm_params()
        check(self.lib.egm_get_params(self.ctx, C.byref(p)), "egm_get_params")
        if ratio is not None:
            p.ratio_num, p.ratio_den = int(ratio[0]), int(ratio[1])
        if sync is not None:
            p.sync = int(bool(sync))
        if form is not None:
            p.form = int(form)
        if band_tile is not None:
            p.band_tile = int(band_tile)
        if float_pass is not None:
            p.float_pass = int(float_pass)
        if timeout_check is not None:
            p.timeout_check = int(timeout_check)
        if tune is not None:
            p.tune = int(tune)
        check(self.lib.egm_set_params(self.ctx, C.byref(p)), "egm_set_params")

    def tuner_export(self) -> bytes:
        """The tuner's cache (egm_tuner_export) as bytes."""
        n = C.c_int64()
        check(self.lib.egm_tuner_export(self.ctx, None, 0, C.byref(n)), "egm_tuner_export")
        buf = C.create_string_buffer(max(int(n.value), 1))
        check(self.lib.egm_tuner_export(self.ctx, buf, int(n.value), C.byref(n)), "egm_tuner_export")
        return buf.raw[:int(n.value)]

    def tuner_import(self, data: bytes):
        check(self.lib.egm_tuner_import(self.ctx, data, len(data)), "egm_tuner_import")

    def tuner_entries(self) -> list:
        """The cache as dicts: regime key fields, chosen form and shape, timings (ms)."""
        import struct
        raw = self.tuner_export()
        magic, version, count, sms = struct.unpack_from("<4sIII", raw, 0)
        out = []
        for k in range(count):
            key, form, shape, ms_plain, ms_band = struct.unpack_from("<Qiiff", raw, 16 + 24 * k)
            out.append({"tiles_log2": key & 63, "one_pair": bool((key >> 6) & 1), "kinds": (key >> 8) & 7,
                        "candidates_log2": (key >> 12) & 15, "form": "banded" if form == 2 else "plain",
                        "band_tile": shape, "ms_plain": ms_plain, "ms_band": ms_band})
        return out

    def reserve(self, queries: int, refs: int, pairs: int = 1):
        check(self.lib.egm_reserve(self.ctx, int(queries), int(refs), int(pairs)), "egm_reserve")

    def sync(self) -> int:
        return self.lib.egm_sync(self.ctx)

    def set_counters(self, on: bool):
        check(self.lib.egm_set_counters(self.ctx, int(bool(on))), "egm_set_counters")

    def set_timing(self, on: bool):
        check(self.lib.egm_set_timing(self.ctx, int(bool(on))), "egm_set_timing")

    def timing(self) -> dict:
        t = _egm.egm_timing()
        check(self.lib.egm_get_timing(self.ctx, C.byref(t)), "egm_get_timing")
        return {k: (int(getattr(t, k)) if k in ("calls", "banded_calls") else float(getattr(t, k)))
                for k, _ in t._fields_}

    def stats(self) -> dict:
        s = _egm.egm_stats()
        check(self.lib.egm_get_stats(self.ctx, C.byref(s)), "egm_get_stats")
        return {k: int(getattr(s, k)) for k, _ in s._fields_}

    # ------------------------------------------------------------ helpers
    def to_device(self, scene):
        """Device tensors for a synth.Scene-like object (xy1, xy2, F, eps, desc1, desc2, ...)."""
        torch = self.torch
        dev = self.device
        d = dict(xy1=torch.as_tensor(scene.xy1, dtype=torch.float64).to(dev).contiguous(),
                 xy2=torch.as_tensor(scene.xy2, dtype=torch.float64).to(dev).contiguous(),
                 F=torch.as_tensor(scene.F, dtype=torch.float64).reshape(9).to(dev).contiguous(),
                 kind=int(scene.kind), dim=int(scene.dim), width=int(scene.width),
                 height=int(scene.height))
        import numpy as np
        if np.ndim(scene.eps) == 0:
            d["eps"] = float(scene.eps)
        else:
            d["eps"] = torch.as_tensor(scene.eps, dtype=torch.float64).to(dev).contiguous()
        for k in ("desc1", "desc2"):
            v = getattr(scene, k)
            d[k] = None if v is None else torch.as_tensor(v).to(dev).contiguous()
        return d

    def make_pair(self, xy1, xy2, F, eps, desc1=None, desc2=None, kind=EGM_DESC_U8_L2, dim=128,
                  width=640, height=480) -> _egm.egm_pair:
        p = _egm.egm_pair()
        p.xy1, p.xy2, p.F = _ptr(xy1), _ptr(xy2), _ptr(F)
        if isinstance(eps, (int, float)):
            p.eps2, p.eps_scalar = None, float(eps)
        else:
            p.eps2, p.eps_scalar = _ptr(eps), 0.0
        p.desc1, p.desc2 = _ptr(desc1), _ptr(desc2)
        p.m, p.n = int(xy1.shape[0]), int(xy2.shape[0])
        p.kind, p.dim, p.width, p.height = int(kind), int(dim), int(width), int(height)
        self._keep = [xy1, xy2, F, eps, desc1, desc2]
        return p

    def _alloc_out(self, M, csr, cap):
        torch = self.torch
        dev = self.device
        o = dict(best=torch.empty(M, dtype=torch.int32, device=dev),
                 second=torch.empty(M, dtype=torch.int32, device=dev),
                 best_d=torch.empty(M, dtype=torch.float32, device=dev),
                 second_d=torch.empty(M, dtype=torch.float32, device=dev),
                 flags=torch.empty(M, dtype=torch.uint8, device=dev))
        if csr:
            o["cand_offsets"] = torch.empty(M + 1, dtype=torch.int64, device=dev)
            o["cand_idx"] = torch.empty(max(int(cap), 1), dtype=torch.int32, device=dev)
            o["cand_total"] = torch.zeros(1, dtype=torch.int64, device=dev)
        return o

    @staticmethod
    def _out_struct(o, cap):
        s = _egm.egm_out()
        s.best, s.second = _ptr(o["best"]), _ptr(o["second"])
        s.best_d, s.second_d, s.flags = _ptr(o["best_d"]), _ptr(o["second_d"]), _ptr(o["flags"])
        if "cand_offsets" in o:
            s.cand_offsets, s.cand_idx = _ptr(o["cand_offsets"]), _ptr(o["cand_idx"])
            s.cand_total, s.cand_capacity = _ptr(o["cand_total"]), int(cap)
        return s

    # -------------------------------------------------------------- calls
    def egm_match_pair(self, pair: _egm.egm_pair, out: _egm.egm_out) -> int:
        return self.lib.egm_match_pair(self.ctx, C.byref(pair), C.byref(out))

    def egm_match_batch(self, pairs, out: _egm.egm_out) -> int:
        arr = (_egm.egm_pair * len(pairs))(*pairs)
        return self.lib.egm_match_batch(self.ctx, arr, len(pairs), C.byref(out))

    def egm_match_pair_host(self, pair: _egm.egm_pair, out: _egm.egm_out) -> int:
        return self.lib.egm_match_pair_host(self.ctx, C.byref(pair), C.byref(out))

    def egm_match_batch_host(self, pairs, outs) -> int:
        """egm_match_batch_host over lists of egm_pair / egm_out structs holding host pointers."""
        n = len(pairs)
        pa = (_egm.egm_pair * n)(*pairs)
        oa = (_egm.egm_out * n)(*outs)
        return self.lib.egm_match_batch_host(self.ctx, pa, n, oa)

    def match(self, xy1, xy2, F, eps, desc1=None, desc2=None, kind=EGM_DESC_U8_L2, dim=128,
              width=640, height=480, csr=False, cand_capacity=None, out=None):
        """Match one pair of device tensors; returns a dict of device tensors."""
        pair = self.make_pair(xy1, xy2, F, eps, desc1, desc2, kind, dim, width, height)
        return self._run([pair], csr, cand_capacity, out, batch=False)

    def match_batch(self, items, csr=False, cand_capacity=None, out=None):
        """items: list of dicts as produced by to_device(); outputs concatenated in pair order."""
        pairs, keep = [], []
        for it in items:
            pairs.append(self.make_pair(it["xy1"], it["xy2"], it["F"], it["eps"], it.get("desc1"),
                                        it.get("desc2"), it["kind"], it["dim"], it["width"],
                                        it["height"]))
            keep.append(self._keep)
        self._keep = keep
        return self._run(pairs, csr, cand_capacity, out, batch=True)

    def _run(self, pairs, csr, cap, out, batch):
        M = sum(int(p.m) for p in pairs)
        if csr and cap is None:
            cap = 64 * max(M, 1)
        o = out if out is not None else self._alloc_out(M, csr, cap or 0)
        s = self._out_struct(o, cap or 0)
        st = self.egm_match_batch(pairs, s) if batch else self.egm_match_pair(pairs[0], s)
        if st == EGM_ERR_CAPACITY and csr and out is None:
            need = int(o["cand_total"].item())
            return self._run(pairs, csr, need, None, batch)
        check(st, "egm_match_batch" if batch else "egm_match_pair")
        if csr:
            o["cand_idx"] = o["cand_idx"][: int(o["cand_offsets"][-1].item())]
        return o

    def graph_create(self, items, out, cand_capacity=0):
        """egm_graph_create over device items (as from to_device) and output tensors."""
        pairs, keep = [], []
        for it in items:
            pairs.append(self.make_pair(it["xy1"], it["xy2"], it["F"], it["eps"], it.get("desc1"),
                                        it.get("desc2"), it["kind"], it["dim"], it["width"], it["height"]))
            keep.append(self._keep)
        arr = (_egm.egm_pair * len(pairs))(*pairs)
        s = self._out_struct(out, cand_capacity)
        g = C.c_void_p()
        check(self.lib.egm_graph_create(self.ctx, arr, len(pairs), C.byref(s), C.byref(g)), "egm_graph_create")
        return _Graph(self, g, keep, out)

    def match_host(self, scene, csr=False, cand_capacity=None):
        """egm_match_pair_host on host (numpy) arrays; returns numpy outputs."""
        import numpy as np

        xy1 = np.ascontiguousarray(scene.xy1, np.float64)
        xy2 = np.ascontiguousarray(scene.xy2, np.float64)
        F = np.ascontiguousarray(scene.F, np.float64).reshape(9)
        d1 = np.ascontiguousarray(scene.desc1)
        d2 = np.ascontiguousarray(scene.desc2)
        p = _egm.egm_pair()
        hp = lambda a: a.ctypes.data_as(C.c_void_p)
        p.xy1, p.xy2, p.F = hp(xy1), hp(xy2), hp(F)
        if np.ndim(scene.eps) == 0:
            p.eps2, p.eps_scalar = None, float(scene.eps)
            eps = None
        else:
            eps = np.ascontiguousarray(scene.eps, np.float64)
            p.eps2, p.eps_scalar = hp(eps), 0.0
        p.desc1, p.desc2 = hp(d1), hp(d2)
        p.m, p.n = xy1.shape[0], xy2.shape[0]
        p.kind, p.dim, p.width, p.height = scene.kind, scene.dim, scene.width, scene.height
        m = p.m
        o = dict(best=np.empty(m, np.int32), second=np.empty(m, np.int32),
                 best_d=np.empty(m, np.float32), second_d=np.empty(m, np.float32),
                 flags=np.empty(m, np.uint8))
        s = _egm.egm_out()
        s.best, s.second, s.best_d = hp(o["best"]), hp(o["second"]), hp(o["best_d"])
        s.second_d, s.flags = hp(o["second_d"]), hp(o["flags"])
        if csr:
            cap = cand_capacity or 64 * max(m, 1)
            o["cand_offsets"] = np.empty(m + 1, np.int64)
            o["cand_idx"] = np.empty(cap, np.int32)
            o["cand_total"] = np.zeros(1, np.int64)
            s.cand_offsets, s.cand_idx, s.cand_total = (hp(o["cand_offsets"]), hp(o["cand_idx"]),
                                                        hp(o["cand_total"]))
            s.cand_capacity = cap
        check(self.egm_match_pair_host(p, s), "egm_match_pair_host")
        return o

    def match_mutual(self, xy1, xy2, F, eps2, eps1, desc1, desc2, kind=EGM_DESC_U8_L2, dim=128,
                     width2=640, height2=480, width1=None, height1=None):
        """egm_match_mutual: device tensors of one pair and the tolerance of each
        image's keypoints (eps1 for the reverse direction).  Returns the outputs
        of m + n rows: forward results, then reverse results."""
        torch = self.torch
        fwd = self.make_pair(xy1, xy2, F, eps2, desc1, desc2, kind, dim, width2, height2)
        keep = self._keep
        Ft = F.reshape(3, 3).t().contiguous().reshape(9)
        rev = self.make_pair(xy2, xy1, Ft, eps1, desc2, desc1, kind, dim,
                             width1 if width1 is not None else width2, height1 if height1 is not None else height2)
        self._keep = [keep, self._keep, Ft]
        o = self._alloc_out(int(xy1.shape[0]) + int(xy2.shape[0]), False, 0)
        s = self._out_struct(o, 0)
        check(self.lib.egm_match_mutual(self.ctx, C.byref(fwd), C.byref(rev), C.byref(s)), "egm_match_mutual")
        del torch
        return o

    def match_mutual_pair(self, xy1, xy2, F, eps2, eps1, desc1, desc2, kind=EGM_DESC_U8_L2, dim=128,
                          width2=640, height2=480, width1=None, height1=None):
        """egm_match_mutual_pair: as match_mutual, the reverse direction formed by the library."""
        fwd = self.make_pair(xy1, xy2, F, eps2, desc1, desc2, kind, dim, width2, height2)
        keep = self._keep
        e1p, e1s = (None, float(eps1)) if isinstance(eps1, (int, float)) else (_ptr(eps1), 0.0)
        o = self._alloc_out(int(xy1.shape[0]) + int(xy2.shape[0]), False, 0)
        s = self._out_struct(o, 0)
        check(self.lib.egm_match_mutual_pair(self.ctx, C.byref(fwd), e1p, e1s,
                                             int(width1 if width1 is not None else width2),
                                             int(height1 if height1 is not None else height2), C.byref(s)),
              "egm_match_mutual_pair")
        self._keep = [keep, eps1]
        return o

    def compact_matches(self, flags, best, require):
        """egm_compact_matches: (i, best[i]) of the rows whose flags contain `require`."""
        torch = self.torch
        m = int(flags.shape[0])
        qi = torch.empty(max(m, 1), dtype=torch.int32, device=self.device)
        rj = torch.empty(max(m, 1), dtype=torch.int32, device=self.device)
        cnt = torch.empty(1, dtype=torch.int64, device=self.device)
        check(self.lib.egm_compact_matches(self.ctx, _ptr(flags), _ptr(best), m, int(require), _ptr(qi), _ptr(rj),
                                           _ptr(cnt)), "egm_compact_matches")
        k = int(cnt.item())
        return qi[:k], rj[:k]

    def gms(self, xy1, xy2, best, flags, size1, size2, require=EGM_FLAG_HAS_BEST, grid=20, alpha=6.0):
        """egm_gms: sets EGM_FLAG_GMS in `flags` (in place) on the input matches
        the grid motion-statistics filter keeps; size1, size2 = (width, height)."""
        m, n = int(xy1.shape[0]), int(xy2.shape[0])
        check(self.lib.egm_gms(self.ctx, _ptr(xy1), m, _ptr(xy2), n, _ptr(best), _ptr(flags), int(size1[0]),
                               int(size1[1]), int(size2[0]), int(size2[1]), int(require), int(grid), float(alpha)),
              "egm_gms")
        return flags

    def gms_batch(self, items, require=EGM_FLAG_HAS_BEST, grid=20, alpha=6.0):
        """egm_gms_batch: items of (xy1, xy2, best, flags, size1, size2) device
        tensors; every flags tensor is updated in place."""
        arr = (_egm.egm_gms_pair * len(items))()
        for k, (xy1, xy2, best, flags, size1, size2) in enumerate(items):
            q = arr[k]
            q.xy1, q.xy2, q.best, q.flags = _ptr(xy1), _ptr(xy2), _ptr(best), _ptr(flags)
            q.m, q.n = int(xy1.shape[0]), int(xy2.shape[0])
            q.width1, q.height1, q.width2, q.height2 = int(size1[0]), int(size1[1]), int(size2[0]), int(size2[1])
        check(self.lib.egm_gms_batch(self.ctx, arr, len(items), int(require), int(grid), float(alpha)),
              "egm_gms_batch")

    def tolnet(self, params) -> "TolNet":
        """A learned-tolerance network on this context (egm_mlp_create)."""
        return TolNet(self, params)

    def residuals(self, xy1, xy2, F, qi, rj):
        """Exact distances [k] float64 of the pairs (qi[t], rj[t]) from their epipolar lines."""
        torch = self.torch
        pair = self.make_pair(xy1, xy2, F, 0.0)
        qi = torch.as_tensor(qi, dtype=torch.int32).to(self.device).contiguous()
        rj = torch.as_tensor(rj, dtype=torch.int32).to(self.device).contiguous()
        out = torch.empty(qi.shape[0], dtype=torch.float64, device=self.device)
        check(self.lib.egm_pair_residuals(self.ctx, C.byref(pair), _ptr(qi), _ptr(rj), qi.shape[0], _ptr(out)),
              "egm_pair_residuals")
        self.sync()
        return out

    def intervals(self, xy2, F, eps, width, height):
        """egm_intervals: (theta, delta, e3, mode) as device tensors."""
        torch = self.torch
        n = int(xy2.shape[0])
        xy1 = torch.zeros((0, 2), dtype=torch.float64, device=self.device)
        pair = self.make_pair(xy1, xy2, F, eps, None, None, EGM_DESC_U8_L2, 128, width, height)
        th = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        de = torch.empty_like(th)
        e3 = torch.empty(3, dtype=torch.float64, device=self.device)
        mode = torch.empty(1, dtype=torch.int32, device=self.device)
        st = self.lib.egm_intervals(self.ctx, C.byref(pair), _ptr(th), _ptr(de), _ptr(e3), _ptr(mode))
        check(st, "egm_intervals")
        return th[:n], de[:n], e3, int(mode.item())


class TolNet:
    """Learned per-keypoint tolerance (egm_mlp): eps = softplus(MLP(features)) + 0.25 px.

    Features are [n, 5] float32 device rows (scale, orientation, response,
    x / W, y / H); parameters a flat float32 vector of EGM_MLP_PARAMS values.
    """

    def __init__(self, mt: Matcher, params):
        import numpy as np

        self.mt, self.lib, self.torch = mt, mt.lib, mt.torch
        p = np.ascontiguousarray(np.asarray(params, np.float32))
        if p.size != _egm.EGM_MLP_PARAMS:
            raise ValueError(f"expected {_egm.EGM_MLP_PARAMS} parameters, got {p.size}")
        h = C.c_void_p()
        check(self.lib.egm_mlp_create(mt.ctx, p.ctypes.data_as(C.c_void_p), C.byref(h)), "egm_mlp_create")
        self.handle = h

    def _feat(self, feat):
        t = self.torch.as_tensor(feat, dtype=self.torch.float32).to(self.mt.device).contiguous()
        if t.ndim != 2 or t.shape[1] != 5:
            raise ValueError("features must be [n, 5]")
        return t

    def infer(self, feat):
        """eps [n] float64 on the device."""
        f = self._feat(feat)
        eps = self.torch.empty(f.shape[0], dtype=self.torch.float64, device=self.mt.device)
        check(self.lib.egm_mlp_infer(self.handle, _ptr(f), f.shape[0], _ptr(eps)), "egm_mlp_infer")
        return eps

    def set_fallback(self, eps_px):
        """Tolerance given to samples without a finite network output (default 2 px)."""
        check(self.lib.egm_mlp_set_fallback(self.handle, float(eps_px)), "egm_mlp_set_fallback")

    def grad(self, feat, resid, quantile):
        """(gradient [EGM_MLP_PARAMS] float32, mean pinball loss) on the device."""
        torch = self.torch
        f = self._feat(feat)
        r = torch.as_tensor(resid, dtype=torch.float32).to(self.mt.device).contiguous()
        g = torch.empty(_egm.EGM_MLP_PARAMS, dtype=torch.float32, device=self.mt.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.mt.device)
        check(self.lib.egm_mlp_grad(self.handle, _ptr(f), _ptr(r), f.shape[0], float(quantile), _ptr(g),
                                    _ptr(loss)), "egm_mlp_grad")
        return g, loss

    def train_step(self, feat, resid, lr, quantile, loss=None):
        """One Adam step; loss (a [1] float32 device tensor, optional) receives the batch loss."""
        check(self.lib.egm_mlp_train_step(self.handle, _ptr(feat), _ptr(resid), feat.shape[0], float(lr),
                                          float(quantile), _ptr(loss)), "egm_mlp_train_step")

    def state(self):
        import numpy as np

        n = _egm.EGM_MLP_PARAMS
        p, m, v = (np.empty(n, np.float32) for _ in range(3))
        step = C.c_int64()
        check(self.lib.egm_mlp_get_state(self.handle, p.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                         v.ctypes.data_as(C.c_void_p), C.byref(step)), "egm_mlp_get_state")
        return dict(params=p, adam_m=m, adam_v=v, step=int(step.value))

    def load_state(self, st):
        import numpy as np

        a = [np.ascontiguousarray(np.asarray(st[k], np.float32)) for k in ("params", "adam_m", "adam_v")]
        check(self.lib.egm_mlp_set_state(self.handle, *(x.ctypes.data_as(C.c_void_p) for x in a),
                                         int(st["step"])), "egm_mlp_set_state")

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.lib.egm_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Graph:
    """A captured batch (egm_graph); launch() replays it on the matcher's stream."""

    def __init__(self, mt, handle, keep, out):
        self.mt, self.handle, self._keep, self.out = mt, handle, keep, out

    def launch(self) -> int:
        return self.mt.lib.egm_graph_launch(self.handle)

    def close(self):
        if self.handle is not None:
            self.mt.lib.egm_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
