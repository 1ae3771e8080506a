#!/usr/bin/env python
"""Throughput benchmark: query keypoints matched per second at exact candidate sets.

Workload (one GPU): the high-resolution single-pair configuration -- nine
image pairs of 6048x4032 px with 16384 keypoints per image (70% true
projections), epipole inside / far outside / at infinity, eps in {1, 2, 4} px,
128-d uint8 descriptors.  One step matches all nine pairs, one pair per
egm_match_pair call, in the library's automatic form (the plain form on
sparse pairs, the banded tensor-core form where about 32 or more candidates
per query are expected; --form forces one).  Inputs are resident in HBM
before the timed region; L2 is flushed (a 256 MiB write) before every step
and the flush is outside the CUDA-event-timed interval.

Beside the headline: the same single-pair step in each forced form, the same
nine pairs as one batched call, the batched configuration (256 pairs, one
CUDA-graph launch per step) in both forms, the float-descriptor batch, the
end-to-end rate through host buffers, per-stage times, the roofline of the
dominant kernel, mutual matching and GMS, the tolerance / scalability /
pose-noise sweeps, the learned-tolerance kernels, and the CPU leg (the oracle
and the paper's segment tree on the host cores).

--impl reference times the CPU oracle (the plain brute-force definition) on
the host cores instead: the paper publishes no code or GPU number, so the
oracle is the reference arm.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, every rank runs the same workload on its own GPU (replicas: the
pairs are independent) and `value` is the total over ranks divided by the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "query keypoints matched/sec per GB300 at exact candidate sets; pairs/sec batched"
WORKLOAD = "6048x4032 single pairs, 16384 keypoints/image, epipole inside/far/infinity x eps {1,2,4} px, 128-d uint8"
POSES = ("inside", "far", "infinity")
EPS = (1.0, 2.0, 4.0)
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--form", choices=["auto", "plain", "banded"], default="auto")
    ap.add_argument("--compare-steps", type=int, default=200)
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-form comparison legs")
    ap.add_argument("--no-mlp", action="store_true", help="skip the learned-tolerance leg")
    ap.add_argument("--no-learned-experiment", action="store_true",
                    help="skip the config-5 train / test experiment (learned vs fixed tolerance)")
    ap.add_argument("--learned-pairs", type=int, default=512)
    ap.add_argument("--no-float", action="store_true", help="skip the float-descriptor batch")
    ap.add_argument("--float-pairs", type=int, default=64)
    ap.add_argument("--no-matching", action="store_true", help="skip the mutual-matching leg")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the tolerance and pose-noise sweeps")
    ap.add_argument("--batched-only", action="store_true", help="run only the batched configuration")
    return ap.parse_args()


def scenes():
    import synth

    return [synth.config2(p, e) for p in POSES for e in EPS]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def desc_row_bytes(kind, dim):
    """Native descriptor row D in bytes: u8 dim, binary dim / 8, float 4 dim."""
    return dim if kind == 0 else dim // 8 if kind == 2 else 4 * dim


def algorithmic_bytes(sc):
    """What the method must move for one pair, each input read once and each
    output written once: per query its keypoint (16 B), descriptor (D) and
    result (17 B: best, second, two distances, flags); per reference its
    keypoint (16 B), descriptor (D) and, when per keypoint, its tolerance
    (8 B); per pair F (72 B).  Tile re-reads, sorted copies and scratch
    records are not counted."""
    import numpy as np

    D = desc_row_bytes(sc.kind, sc.dim)
    per_ref = 16 + D + (0 if np.ndim(sc.eps) == 0 else 8)
    return sc.m * (16 + D + 17) + sc.n * per_ref + 72


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples during the timed region: every 50 ms, and one at each end."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def _once(self):
        """One synchronous sample (a query only), appended to the record."""
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            self.extra.append(r.stdout)
        except (OSError, subprocess.SubprocessError):
            pass

    def start(self):
        """Starts the periodic sampler (every 50 ms); `edge` also takes one
        sample at once, so that even a timed region shorter than the period
        has a sample at each end."""
        self.extra = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def edge(self):
        if self.p is not None:
            self._once()

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._once()
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        periodic = self.f.read().splitlines()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        edge_lines = [ln for out in self.extra for ln in out.splitlines()]
        for line in periodic + edge_lines:
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                smax.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "samples_periodic": len(periodic), "samples_at_edges": len(edge_lines),
                "reasons": sorted(reasons)}


def max_sm_mhz(device):
    """The device's largest SM clock as nvidia-smi reports it (a query only),
    else GB300's 2070 MHz."""
    try:
        import torch

        idx = torch.device(device).index or 0
        r = subprocess.run(["nvidia-smi", "-i", str(idx), "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                           capture_output=True, text=True, timeout=10)
        return float(r.stdout.strip().splitlines()[0])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return 2070.0


# ------------------------------------------------------------------ distributed
# One process per GPU, replicas of the same workload (the pairs are
# independent: no data-path collective).  The process group only carries the
# barriers around the timed regions and the max over ranks of the times: NCCL
# on GPUs, gloo where there is none (the multi-process tests on CPU).
def dist_setup(gpus, backend=None):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, local):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = f"cuda:{local}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, timed by the slowest rank."""
    return world * units_per_rank / seconds_max


# ------------------------------------------------------------------ oracle (CPU)
def cpu_oracle_rate(scs, seconds):
    """The oracle as it stands on the host cores: queries per second over a
    bounded sample (pairs cycled until `seconds` have elapsed)."""
    import oracle

    n_q, t0, k = 0, time.perf_counter(), 0
    while True:
        sc = scs[k % len(scs)]
        oracle.match_scene(sc)
        n_q += sc.m
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n_q / el, oracle.num_threads(), k, el


def cpu_segtree_rate(scs, seconds):
    """The paper's own method (centred segment tree, Sec. 4.4) in C on the
    host cores, in its exact form (pad + distance test) and as the paper
    describes it (stabbing only): queries per second including the index
    build, over the pairs cycled for about `seconds` each."""
    from oracle import segtree

    out = {}
    for name, exact in (("exact", True), ("paper", False)):
        segtree.match_scene(scs[0], exact=exact)  # load / build
        n_q, k, b, mtime, t0 = 0, 0, 0.0, 0.0, time.perf_counter()
        while True:
            sc = scs[k % len(scs)]
            r = segtree.match_scene(sc, exact=exact)
            b += r["build_s"]
            mtime += r["match_s"]
            n_q += sc.m
            k += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
        out[name] = {"value": n_q / el, "unit": "queries/s", "pairs": k, "seconds": el,
                     "build_ms_per_pair": 1e3 * b / k, "match_ms_per_pair": 1e3 * mtime / k}
    out["cores"] = segtree.num_threads()
    out["kind"] = "the paper's centred segment tree in C (OpenMP: intervals, subtree tasks, queries)"
    return out


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores, on the same
    workload and step as our arm (one step = the nine config pairs), so that
    the two lines time the same work per step."""
    rank, world, local = dist_setup(args.gpus)
    if rank != 0:
        return
    scs = scenes()
    import oracle

    oracle.match_scene(scs[0])  # load / build

    def step():
        for sc in scs:
            oracle.match_scene(sc)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    total = time.perf_counter() - t0
    q_per_step = sum(sc.m for sc in scs)
    value = q_per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs_per_step": len(scs), "queries_per_step": q_per_step,
                   "form": "CPU oracle: FP64 brute force over every (query, reference) pair",
                   "parallelism": f"OpenMP over queries, {oracle.num_threads()} threads"},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{args.steps} timed steps of the nine config pairs ({q_per_step} queries each)"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours
KERNEL_SOURCES = {"band_kernel": ("band.cu", "tc.cuh", "egm_internal.cuh"),
                  "stab_kernel": ("stab.cu", "egm_internal.cuh"),
                  "stab_pair_kernel": ("stab.cu", "egm_internal.cuh")}


def source_hash(kernel):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2603_18401_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_profile(kernel, workload="config2"):
    """Counters of the committed ncu summary of `kernel` on this workload, if
    it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return d if d.get("source_sha256") == source_hash(kernel) else None


def matching_leg(mt, torch, stream, scs, dev, steps):
    """Mutual matching (both directions, cross-check) of the single-pair scenes
    and the compact list of ratio-passing mutual matches; recall and precision
    against the true pairs of the synthetic scenes."""
    RATIO_MUTUAL = 2 | 16

    def one(s, d):
        o = mt.match_mutual(d["xy1"], d["xy2"], d["F"], d["eps"], 2.0, d["desc1"], d["desc2"], d["kind"],
                            d["dim"], d["width"], d["height"])
        return mt.compact_matches(o["flags"][:s.m], o["best"][:s.m], RATIO_MUTUAL)

    tp = n_true = n_got = 0
    for s, d in zip(scs, dev):
        qi, rj = one(s, d)
        got = set(zip(qi.cpu().numpy().tolist(), rj.cpu().numpy().tolist()))
        truth = set(map(tuple, s.gt.tolist()))
        tp += len(got & truth)
        n_true += len(truth)
        n_got += len(got)
    mt.set_params(sync=False)
    for _ in range(3):
        for s, d in zip(scs, dev):
            one(s, d)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = max(steps // 10, 5)
    for _ in range(reps):
        for s, d in zip(scs, dev):
            one(s, d)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    q = sum(s.m + s.n for s in scs)
    mutual = {"workload": "the nine single pairs, both directions (eps 2 px for image-1 keypoints)",
              "queries_per_s": q / (ms * 1e-3), "ms_per_step": ms, "matches": n_got,
              "recall": tp / max(n_true, 1), "precision": tp / max(n_got, 1),
              "filter": "ratio test (4/5) and mutual", "api": "egm_match_mutual + egm_compact_matches"}

    # GMS on the nearest neighbours (the paper's default filter, threshold 6)
    HAS_GMS = 1 | 32

    def gms_one(s, d):
        o = mt.match(d["xy1"], d["xy2"], d["F"], d["eps"], d["desc1"], d["desc2"], d["kind"], d["dim"],
                     d["width"], d["height"])
        mt.gms(d["xy1"], d["xy2"], o["best"], o["flags"], (s.width, s.height), (s.width, s.height))
        return mt.compact_matches(o["flags"], o["best"], HAS_GMS)

    tp = n_true = n_got = 0
    for s, d in zip(scs, dev):
        qi, rj = gms_one(s, d)
        got = set(zip(qi.cpu().numpy().tolist(), rj.cpu().numpy().tolist()))
        truth = set(map(tuple, s.gt.tolist()))
        tp += len(got & truth)
        n_true += len(truth)
        n_got += len(got)
    for _ in range(3):
        for s, d in zip(scs, dev):
            gms_one(s, d)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for s, d in zip(scs, dev):
            gms_one(s, d)
    e1.record(stream)
    torch.cuda.synchronize()
    gms_ms = e0.elapsed_time(e1) / reps
    q = sum(s.m for s in scs)
    gms = {"workload": "the nine single pairs", "queries_per_s": q / (gms_ms * 1e-3), "ms_per_step": gms_ms,
           "matches": n_got, "recall": tp / max(n_true, 1), "precision": tp / max(n_got, 1),
           "filter": "GMS (20 x 20 cells, alpha 6, four grid shifts) on the nearest neighbours",
           "api": "egm_match_pair + egm_gms + egm_compact_matches"}
    return {"mutual_ratio": mutual, "gms": gms, "timing": "CUDA events; each call reads the match count back"}


def sweeps_leg(mt, torch, stream, reps):
    """Analogues of the paper's tolerance sweep (Sec. 5.3: 25,000 keypoints
    per image, tolerance up to 200 px) and pose-noise sweep (Sec. 5.5: noise
    levels 0 to 3.3 at 200 px, against brute-force matching) on synthetic
    6048x4032 pairs."""
    import numpy as np
    import synth

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def quality(sc, o):
        best, flags = o["best"].cpu().numpy(), o["flags"].cpu().numpy()
        ok = np.nonzero(flags & 2)[0]
        got = set(zip(ok.tolist(), best[ok].tolist()))
        truth = set(map(tuple, sc.gt.tolist()))
        tp = len(got & truth)
        return tp / max(len(truth), 1), tp / max(len(got), 1)

    out = {}
    sc = synth.config2("inside", 2.0, seed=5, scale=25000 / 16384)
    d = mt.to_device(sc)
    args = lambda eps, F=None: (d["xy1"], d["xy2"], d["F"] if F is None else F, eps, d["desc1"], d["desc2"],
                                d["kind"], d["dim"], d["width"], d["height"])
    rows = []
    for eps in (1.0, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0, 200.0):
        o = mt.match(*args(eps), csr=True)
        kbar = int(o["cand_offsets"][-1].item()) / sc.m
        rec, prec = quality(sc, o)
        row = {"eps_px": eps, "candidates_per_query": kbar, "matching_recall": rec, "matching_precision": prec}
        for name, form in (("auto", 0), ("plain", 1), ("banded", 2)):
            mt.set_params(form=form)
            row[f"{name}_ms"] = timed(lambda: mt.match(*args(eps)))
        mt.set_params(form=0)
        row["candidates_csr_ms"] = timed(lambda: mt.match(*args(eps), csr=True))
        rows.append(row)
    out["tolerance"] = {"workload": "one 6048x4032 pair, 25,000 keypoints per image (17,500 true), epipole "
                                    "inside, u8 128-d; matching time per pair (CUDA events, L2 warm)",
                        "rows": rows}

    # keypoint counts (Sec. 5.4: 5,000 to 50,000 keypoints at 50 px)
    rows = []
    for count in (5000, 10000, 25000, 50000):
        sc = synth.config2("far", 50.0, seed=9, scale=count / 16384)
        d = mt.to_device(sc)
        o = mt.match(*args(50.0), csr=True)
        kbar = int(o["cand_offsets"][-1].item()) / sc.m
        row = {"keypoints": count, "candidates_per_query": kbar}
        for name, form in (("auto", 0), ("plain", 1), ("banded", 2)):
            mt.set_params(form=form)
            row[f"{name}_ms"] = timed(lambda: mt.match(*args(50.0)))
        mt.set_params(form=0)
        rows.append(row)
    out["scalability"] = {"workload": "one 6048x4032 pair per size, epipole far outside, eps 50 px, u8 128-d",
                          "rows": rows}

    sc = synth.config2("far", 200.0, seed=6)
    d = mt.to_device(sc)
    rows = []
    qi = torch.as_tensor(sc.gt[:, 0], dtype=torch.int32).to(mt.device)
    rj = torch.as_tensor(sc.gt[:, 1], dtype=torch.int32).to(mt.device)
    for level in (0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.3):
        Fn = synth.perturb_pose(sc, level, seed=11) if level > 0 else sc.F
        Ft = torch.as_tensor(np.ascontiguousarray(Fn).reshape(9)).to(mt.device)
        res = mt.residuals(d["xy1"], d["xy2"], Ft, qi, rj).cpu().numpy()
        o = mt.match(*args(200.0, Ft))
        rec, prec = quality(sc, o)
        mt.set_params(form=2)
        ob = mt.match(*args(1e7, Ft))
        mt.set_params(form=0)
        brec, bprec = quality(sc, ob)
        rows.append({"level": level, "candidate_recall": float(np.mean(res <= 200.0)), "matching_recall": rec,
                     "matching_precision": prec, "bf_matching_recall": brec, "bf_matching_precision": bprec,
                     "ms": timed(lambda: mt.match(*args(200.0, Ft)))})
    out["pose_noise"] = {"workload": "one 6048x4032 pair, 16,384 keypoints per image, epipole far outside; F from "
                                     "a perturbed pose (per-axis rotation U[-l, l] deg, translation U[-l/4, l/4] "
                                     "units); eps 200 px vs brute force (eps 1e7 px)",
                         "rows": rows}
    return out


def mlp_leg(mt, torch, stream):
    """Throughput of the learned-tolerance kernels on config-5-like features.

    FLOPs per sample: forward 2 (5*64 + 2*64*64 + 64) = 17 152 in the layer
    products plus ~25 per unit for GELU / softplus; training adds the
    backward pass, twice the forward products.  The forward pass (inference
    and training) runs layers 2 and 3 on the tensor cores (two BF16 products
    per layer: activations split into hi and lo parts), the rest on the FP32
    CUDA cores; the backward pass and Adam run on the CUDA cores.  Both legs
    are bound by CUDA-core issue: the peak is the device's SMs x 128 FP32
    lanes x 2 FLOP x its largest SM clock (nvidia-smi's clocks.max.sm, else
    2070 MHz), each product of the FP32 network counted once."""
    import numpy as np
    import synth

    rng = np.random.default_rng(5)
    n = 1 << 20
    s = np.exp(rng.uniform(0.0, np.log(16.0), n))
    feat = np.stack([s, rng.uniform(0, 2 * np.pi, n), np.exp(rng.normal(0, 0.3, n)) / s,
                     rng.uniform(0, 1, n), rng.uniform(0, 1, n)], axis=1).astype(np.float32)
    resid = np.abs(rng.normal(0, 1, n) * 0.42 * s).astype(np.float32)
    f = torch.as_tensor(feat).to(mt.device)
    r = torch.as_tensor(resid).to(mt.device)
    net = mt.tolnet(synth.mlp_init(0))
    eps = torch.empty(n, dtype=torch.float64, device=mt.device)
    batch = 65536
    fb, rb = f[:batch].contiguous(), r[:batch].contiguous()
    from paper_2603_18401_gb300 import check

    def infer():
        check(mt.lib.egm_mlp_infer(net.handle, f.data_ptr(), n, eps.data_ptr()), "egm_mlp_infer")

    def train():
        check(mt.lib.egm_mlp_train_step(net.handle, fb.data_ptr(), rb.data_ptr(), batch, 1e-3, 0.95, None),
              "egm_mlp_train_step")

    out = {}
    for name, fn, samples, flop in (("inference", infer, n, 17152 + 25 * 193),
                                    ("train_step", train, batch, 3 * 17152 + 75 * 193)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"samples_per_s": samples / (ms * 1e-3), "ms": ms, "samples": samples,
                     "tflops": samples * flop / (ms * 1e-3) / 1e12}
    net.close()
    sms = torch.cuda.get_device_properties(mt.device).multi_processor_count
    mhz = max_sm_mhz(mt.device)
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    src = f"derived: {sms} SMs x 128 FP32 lanes x 2 FLOP x {mhz:g} MHz"
    out["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak, "peak_source": src,
                       "achieved": out["train_step"]["tflops"], "frac": out["train_step"]["tflops"] / peak,
                       "kernel": "mlp_forward_tc_kernel + mlp_backward_kernel + adam_kernel (one training step)"}
    out["roofline_inference"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak, "peak_source": src,
                                 "achieved": out["inference"]["tflops"],
                                 "frac": out["inference"]["tflops"] / peak,
                                 "kernel": "mlp_forward_tc_kernel (FLOPs of the FP32 network, each product once)"}
    out["network"] = "5-64-64-64-1 GELU, softplus + 0.25 px, BF16-rounded weights, FP32 arithmetic"
    out["inference"]["kernel"] = ("mlp_forward_tc_kernel: layers 2 and 3 as tcgen05.mma (M 128, N 64, K 64, BF16 "
                                  "hi + lo activations, FP32 in TMEM); layers 1 and 4, GELU on CUDA cores")
    return out


def _config5_chunk(seed, idx):
    import synth

    return synth.config5(seed=seed, only=idx)


def config5_scenes(seed, npairs):
    """The config-5 pairs, generated on the host cores in parallel (spawned
    workers: safe beside a CUDA context)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    workers = max(1, min(16, os.cpu_count() or 1))
    chunks = [list(range(k, npairs, workers)) for k in range(workers)]
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_config5_chunk, [seed] * len(chunks), chunks))
    out = [None] * npairs
    for idx, scs in zip(chunks, parts):
        for p, sc in zip(idx, scs):
            out[p] = sc
    return out


def learned_tolerance_experiment(mt, torch, stream, args):
    """Config 5 as stated: 512 pairs (4k-16k keypoints per image, keypoint
    scale s ~ logU[1, 16], localisation noise 0.3 s px); the network is
    trained by the library's kernels on the exact residuals of the true
    matches of pairs 0-383 (Adam, lr 1e-3, 20 epochs, pinball loss at
    q = 0.95) and tested on pairs 384-511 against the fixed tolerance of
    2 px and against a fixed tolerance with the same candidate budget (the
    mean learned tolerance).  The oracle judges: its brute-force candidate
    sets at each tolerance give the candidate recall (true match in the
    set) and the candidates per query, and the GPU candidate sets at the
    learned tolerance are compared with them pair by pair.  Matching rates
    are the 128 test pairs in one CUDA-graph launch per step."""
    import numpy as np

    import oracle
    import synth

    t0 = time.perf_counter()
    scenes = config5_scenes(0, args.learned_pairs)
    gen_s = time.perf_counter() - t0
    ntrain = args.learned_pairs * 3 // 4
    train, test = scenes[:ntrain], scenes[ntrain:]
    dev = mt.device
    # training set: features of the image-2 keypoint of every true match and
    # its exact residual (Eq. 3, egm_pair_residuals)
    F, R = [], []
    for sc in train:
        d = mt.to_device(sc)
        F.append(sc.feat2[sc.gt[:, 1]])
        R.append(mt.residuals(d["xy1"], d["xy2"], d["F"], sc.gt[:, 0], sc.gt[:, 1]))
    f = torch.as_tensor(np.concatenate(F).astype(np.float32)).to(dev)
    r = torch.cat(R).float()
    del F, R
    net = mt.tolnet(synth.mlp_init(0))
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    batch, epochs, lr, q = 1024, 20, 1e-3, 0.95
    steps = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(epochs):
        perm = torch.randperm(f.shape[0], device=dev, generator=g)
        fp, rp = f[perm].contiguous(), r[perm].contiguous()
        for b in range(0, f.shape[0] - batch + 1, batch):
            net.train_step(fp[b:b + batch], rp[b:b + batch], lr, q)
            steps += 1
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)

    # held-out pairs: learned tolerance, then the oracle's judgement
    eps_l = [net.infer(sc.feat2).cpu().numpy() for sc in test]
    mean_l = float(np.mean(np.concatenate(eps_l)))
    settings = (("learned", eps_l), ("fixed_2px", [2.0] * len(test)), ("fixed_same_budget", [mean_l] * len(test)))
    rows = {}
    identical = 0
    for name, eps in settings:
        hit = cand = tot = 0
        for k, (sc, e) in enumerate(zip(test, eps)):
            c = oracle.candidates(sc.xy1, sc.xy2, sc.F, e)
            off, idx = c["offsets"], c["idx"]
            rowid = np.repeat(np.arange(sc.m, dtype=np.int64), np.diff(off))
            hit += int(np.isin(sc.gt[:, 0] * sc.n + sc.gt[:, 1], rowid * sc.n + idx).sum())
            cand += int(off[-1])
            tot += len(sc.gt)
            if name == "learned":
                d = mt.to_device(sc)
                o = mt.match(d["xy1"], d["xy2"], d["F"], torch.as_tensor(e).to(dev), d["desc1"], d["desc2"],
                             sc.kind, sc.dim, sc.width, sc.height, csr=True)
                identical += int(np.array_equal(o["cand_offsets"].cpu().numpy(), off) and
                                 np.array_equal(o["cand_idx"].cpu().numpy(), idx))
        rows[name] = {"candidate_recall": hit / tot, "candidates_per_query": cand / sum(s.m for s in test),
                      "mean_eps_px": float(np.mean(np.concatenate([np.broadcast_to(e, (s.n,)) for s, e in
                                                                   zip(test, eps)])))}

    # matching on the GPU: the 128 test pairs in one graph per step
    qn = sum(s.m for s in test)
    feat_all = torch.as_tensor(np.concatenate([s.feat2 for s in test]).astype(np.float32)).to(dev)
    for name, eps in settings:
        items = []
        for sc, e in zip(test, eps):
            d = mt.to_device(sc)
            d["eps"] = torch.as_tensor(e).to(dev) if np.ndim(e) else float(e)
            items.append(d)
        out = mt._alloc_out(qn, False, 0)
        graph = mt.graph_create(items, out)
        for _ in range(3):
            graph.launch()
        torch.cuda.synchronize()
        reps = 10
        e0.record(stream)
        for _ in range(reps):
            graph.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        graph.close()
        best, flags = out["best"].cpu().numpy(), out["flags"].cpu().numpy()
        tp = ngot = ntrue = 0
        q0 = 0
        for sc in test:
            ok = np.nonzero(flags[q0:q0 + sc.m] & 2)[0]
            got = set(zip(ok.tolist(), best[q0:q0 + sc.m][ok].tolist()))
            truth = set(map(tuple, sc.gt.tolist()))
            tp += len(got & truth)
            ngot += len(got)
            ntrue += len(truth)
            q0 += sc.m
        rows[name].update({"match_ms": ms, "queries_per_s": qn / (ms * 1e-3), "matches": ngot,
                           "matches_per_s": ngot / (ms * 1e-3), "matching_recall": tp / max(ntrue, 1),
                           "matching_precision": tp / max(ngot, 1)})
    # inference over every test keypoint
    epsbuf = torch.empty(feat_all.shape[0], dtype=torch.float64, device=dev)
    from paper_2603_18401_gb300 import check

    for _ in range(3):
        check(mt.lib.egm_mlp_infer(net.handle, feat_all.data_ptr(), feat_all.shape[0], epsbuf.data_ptr()), "infer")
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(10):
        check(mt.lib.egm_mlp_infer(net.handle, feat_all.data_ptr(), feat_all.shape[0], epsbuf.data_ptr()), "infer")
    e1.record(stream)
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / 10
    rows["learned"]["infer_ms"] = infer_ms
    rows["learned"]["queries_per_s_with_inference"] = qn / ((rows["learned"]["match_ms"] + infer_ms) * 1e-3)
    net.close()
    return {"workload": f"config 5: {len(scenes)} pairs 6048x4032, 4096-16384 keypoints per image, scale "
                        "logU[1,16], noise 0.3 s px; train on pairs 0-" + str(ntrain - 1) + ", test on " +
                        f"{ntrain}-{len(scenes) - 1}",
            "training": {"samples": int(f.shape[0]), "epochs": epochs, "batch": batch, "lr": lr, "quantile": q,
                         "adam_steps": steps, "ms": train_ms, "generation_s": gen_s},
            "oracle_checked_pairs": len(test), "gpu_candidate_sets_identical_to_oracle": identical,
            "judge": "oracle brute-force candidate sets (recall = true match in the set)",
            "test": rows}


def batched_leg(mt, torch, stream, args, world, local):
    """The batched configuration: 256 pairs with uneven counts in one
    CUDA-graph launch per step, in the requested form and the plain form,
    with the per-stage split; the 64-pair float batch in both forms and both
    tensor-core passes."""
    from paper_2603_18401_gb300 import EgmError

    import synth as _synth

    bsc = _synth.config3(seed=0, npairs=args.batch_pairs)
    bitems = [mt.to_device(s) for s in bsc]
    bM = sum(s.m for s in bsc)

    def time_graph(form, items=bitems, total=bM):
        mt.set_params(form=form)
        bout = mt._alloc_out(total, False, 0)
        graph = mt.graph_create(items, bout)
        for _ in range(3):
            if graph.launch() != 0:
                raise EgmError(mt.sync(), "batched warm-up")
        torch.cuda.synchronize()
        bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.batch_steps)]
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.batch_steps):
            bev[k][0].record(stream)
            graph.launch()
            bev[k][1].record(stream)
        torch.cuda.synchronize()
        st = mt.sync()
        if st != 0:
            raise EgmError(st, "batched timed region")
        graph.close()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in bev), world, local) / args.batch_steps

    bform = {"auto": 0, "plain": 1, "banded": 2}[args.form]
    bms = time_graph(bform)
    # per-stage split of one batch, outside the timed region
    mt.set_timing(True)
    for _ in range(3):
        mt.match_batch(bitems)
    bt = mt.timing()
    mt.set_timing(False)
    bstage = {k[:-3]: round(bt[k] / max(bt["calls"], 1), 4) for k in bt if k.endswith("_ms")}
    in_bytes = sum(s.xy1.nbytes + s.xy2.nbytes + s.desc1.nbytes + s.desc2.nbytes for s in bsc)
    batched = {"workload": f"{len(bsc)} pairs 6048x4032, per-image counts log-uniform in [1024, 32768], "
                           "random poses (rotation up to 30 deg), u8 L2 on even / 256-bit binary on odd pairs",
               "pairs_per_s": world * len(bsc) / (bms * 1e-3),
               "queries_per_s": world * bM / (bms * 1e-3), "ms_per_step": bms, "steps": args.batch_steps,
               "queries_per_step": bM, "refs_per_step": sum(s.n for s in bsc),
               "input_bytes": int(in_bytes), "l2": "inputs larger than L2 (129 MB)",
               "form": f"{args.form} (egm_graph_launch, one CUDA graph per step)",
               "stage_ms": bstage,
               "tuned_regimes": mt.tuner_entries()}
    if bform != 1:
        # the band kernel over the batch, on the method's algorithmic bytes
        # (each pair's inputs read once, its results written once); beside
        # them the kernel's own layout read once: per query its order entry,
        # FP32 record, descriptor row and outputs, per reference its sorted
        # record and descriptor row (re-reads of a row by neighbouring tiles
        # not counted)
        kb = sum(algorithmic_bytes(s) for s in bsc)
        lb = sum(s.m * (4 + 48 + desc_row_bytes(s.kind, s.dim) + 17) + s.n * (16 + desc_row_bytes(s.kind, s.dim))
                 for s in bsc)
        ks = bstage["stab"] * 1e-3
        peak, peak_kind = measured_peaks()
        prof = kernel_profile("band_kernel", "batch")
        traffic = prof.get("dram_bytes_per_launch") if prof else None
        batched["roofline"] = {"kernel": "band_kernel", "bound": "hbm", "achieved": kb / ks / 1e9, "peak": peak,
                               "peak_source": peak_kind, "unit": "GB/s", "frac": kb / ks / 1e9 / peak,
                               "algorithmic_bytes_per_launch": kb, "layout_bytes_per_launch": lb,
                               "avg_launch_us": ks * 1e6, "traffic": traffic,
                               "traffic_over_algorithmic": traffic / kb if traffic else None,
                               "tensor_pipe_active_pct": prof.get("tensor_pipe_active_pct") if prof else None,
                               "whole_batch": {"achieved": kb / (bms * 1e-3) / 1e9,
                                               "frac": kb / (bms * 1e-3) / 1e9 / peak}}
    if bform != 1 and not args.no_compare:
        pms = time_graph(1)
        batched["plain_form"] = {"pairs_per_s": world * len(bsc) / (pms * 1e-3), "ms_per_step": pms}
    del bitems
    # float descriptors: 128-d RootSIFT-like FP32, 16384 keypoints per image
    if not args.no_float:
        fsc = _synth.config4(seed=0, npairs=args.float_pairs)
        fitems = [mt.to_device(s) for s in fsc]
        fM = sum(s.m for s in fsc)
        fms = time_graph(bform, fitems, fM)
        fl = {"workload": f"{len(fsc)} pairs 6048x4032, 16384 keypoints per image, 128-d float L2 "
                          "(RootSIFT-like), random poses",
              "pairs_per_s": world * len(fsc) / (fms * 1e-3), "queries_per_s": world * fM / (fms * 1e-3),
              "ms_per_step": fms, "form": args.form}
        if bform != 1 and not args.no_compare:
            pms = time_graph(1, fitems, fM)
            fl["plain_form"] = {"pairs_per_s": world * len(fsc) / (pms * 1e-3), "ms_per_step": pms}
            # the FP8 (E4M3, per-row scale) tensor-core pass instead of BF16
            mt.set_params(float_pass=1)
            f8 = time_graph(2, fitems, fM)
            mt.set_params(float_pass=0)
            fl["fp8_pass"] = {"pairs_per_s": world * len(fsc) / (f8 * 1e-3), "ms_per_step": f8,
                              "form": "banded, FP8 E4M3 pass with per-row scales, FP32 rerank"}
        fl["pass"] = "BF16 tensor-core pass, FP32 rerank (outputs identical to the plain FP32 form)"
        batched["float_descriptors"] = fl
        del fitems
    mt.set_params(form=bform)
    return batched


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as g

    rank, world, local = dist_setup(args.gpus)
    scs = scenes()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before the first GPU call
        cpu = cpu_oracle_rate(scs, args.cpu_seconds)
        seg = cpu_segtree_rate(scs, max(args.cpu_seconds / 2, 1.0))
    g.build()
    from paper_2603_18401_gb300 import Matcher, EgmError, _egm

    torch.cuda.set_device(local)
    mt = Matcher(local)
    mt.set_params(sync=False, form={"auto": 0, "plain": 1, "banded": 2}[args.form])
    dev = [mt.to_device(s) for s in scs]
    outs = [mt._alloc_out(s.m, False, 0) for s in scs]
    pairs, ostr, keep = [], [], []
    for d, o in zip(dev, outs):
        pairs.append(mt.make_pair(d["xy1"], d["xy2"], d["F"], d["eps"], d["desc1"], d["desc2"], d["kind"],
                                  d["dim"], d["width"], d["height"]))
        keep.append(mt._keep)
        ostr.append(mt._out_struct(o, 0))
    mt.reserve(max(s.m for s in scs), max(s.n for s in scs), 1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=mt.device)
    stream = torch.cuda.current_stream()
    if args.batched_only:
        # the batched configuration alone (for profiling it): its own line
        b = batched_leg(mt, torch, stream, args, world, local)
        if rank == 0:
            print(json.dumps({"metric": "pairs/sec batched", "value": b["pairs_per_s"], "unit": "pairs/s",
                              "n_gpus": world, "higher_is_better": True, "batched": b}), flush=True)
        mt.close()
        return

    def step():
        for p, o in zip(pairs, ostr):
            st = mt.egm_match_pair(p, o)
            if st != 0:
                raise EgmError(st, "egm_match_pair")

    for _ in range(args.warmup):
        flush.zero_()
        step()
    st = mt.sync()
    if st != 0:
        raise EgmError(st, "warm-up")
    # parity of the last warm-up outputs against the oracle happens in the tests;
    # here only sanity: every query got a decision
    assert all(int((o["flags"] & 8).sum()) < s.m for o, s in zip(outs, scs))

    clocks = Clocks(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    clocks.edge()  # the enqueued steps are still running on the device
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    st = mt.sync()
    if st != 0:
        raise EgmError(st, "timed region")
    # per-stage split from the library's stage events, pair by pair, in
    # separate untimed passes (the events add host work to every call); the
    # library also reports which form each call ran
    per_pair = []
    for p, o in zip(pairs, ostr):
        mt.set_timing(True)
        for _ in range(20):
            flush.zero_()
            if mt.egm_match_pair(p, o) != 0:
                raise EgmError(mt.sync(), "timing pass")
        torch.cuda.synchronize()
        t = mt.timing()
        mt.set_timing(False)
        c = max(t["calls"], 1)
        per_pair.append(({k[:-3]: t[k] / c for k in t if k.endswith("_ms")}, 2 * t["banded_calls"] > t["calls"]))
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, world, local)
    q_per_step = sum(s.m for s in scs)
    value = replica_rate(q_per_step * args.steps, world, ms * 1e-3)

    # dominant kernel: the matching kernel ("stab" stage) that takes the most
    # time over the step -- stab_kernel on the pairs run in the plain form,
    # band_kernel on those run in the banded form
    stage_ms = {}
    for st_ms, _ in per_pair:
        for k, v in st_ms.items():
            stage_ms[k] = stage_ms.get(k, 0.0) + v / len(per_pair)
    dom = max(stage_ms, key=stage_ms.get)
    n_banded = sum(1 for _, b in per_pair if b)

    def layout_bytes(sc, band):
        """The kernel's own layout: what it reads and writes per launch."""
        row = sc.desc1.shape[1]
        if band:
            # every query's order entry (4 B), line record (48 B), descriptor
            # and result (17 B) once; every reference's record (16 B) and
            # descriptor once
            return sc.m * (4 + 48 + row + 17) + sc.n * (16 + row)
        # every query's line record (48 B), descriptor and result (17 B) once;
        # every reference's record (16 B) and descriptor once
        return sc.m * (48 + row + 17) + sc.n * (16 + row)

    kt = {False: 0.0, True: 0.0}
    kb = {False: 0.0, True: 0.0}
    kl = {False: 0.0, True: 0.0}
    for (st_ms, b), sc in zip(per_pair, scs):
        kt[b] += st_ms["stab"]
        kb[b] += algorithmic_bytes(sc)
        kl[b] += layout_bytes(sc, b)
    banded = kt[True] > kt[False]
    # the plain form of a single pair with u8 or binary rows runs the warp-per-query variant
    kernel = "band_kernel" if banded else ("stab_pair_kernel" if all(s.kind in (0, 2) for s in scs)
                                           else "stab_kernel")
    npk = n_banded if banded else len(scs) - n_banded
    kbytes = kb[banded] / max(npk, 1)
    lbytes = kl[banded] / max(npk, 1)
    k_s = kt[banded] / max(npk, 1) * 1e-3
    peak, peak_kind = measured_peaks()
    achieved = kbytes / k_s / 1e9
    prof = kernel_profile(kernel)
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    step_bytes = sum(algorithmic_bytes(sc) for sc in scs)
    step_s = ms / args.steps * 1e-3
    roofline = {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "traffic_over_algorithmic": traffic / kbytes if traffic else None,
                "tensor_pipe_active_pct": prof.get("tensor_pipe_active_pct") if prof else None,
                "avg_launch_us": k_s * 1e6, "algorithmic_bytes_per_launch": kbytes,
                "algorithmic_bytes_rule": "per query 16 + D + 17 B, per reference 16 + D (+8 with per-keypoint "
                                          "eps) B, per pair 72 B; D = 128 (u8), 32 (binary), 512 (float)",
                "layout_bytes_per_launch": lbytes,
                "launches_averaged": f"{npk} of the {len(scs)} pairs run this kernel",
                "stage_us_per_pair": {k: round(v * 1e3, 2) for k, v in stage_ms.items()},
                "dominant_stage": dom,
                "pairs_banded": n_banded,
                "whole_step": {"algorithmic_bytes": step_bytes, "achieved": step_bytes / step_s / 1e9,
                               "frac": step_bytes / step_s / 1e9 / peak}}

    # the same step in each forced form (or the other one), for comparison
    other_form = None
    if not args.no_compare:
        other_form = {}
        forms = (1, 2) if args.form == "auto" else ((2,) if args.form == "plain" else (1,))
        for other in forms:
            mt.set_params(form=other)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.compare_steps)]
            for k in range(args.compare_steps):
                flush.zero_()
                pe[k][0].record(stream)
                step()
                pe[k][1].record(stream)
            torch.cuda.synchronize()
            pms = max_over_ranks(sum(a.elapsed_time(b) for a, b in pe), world, local)
            other_form["banded" if other == 2 else "plain"] = {
                "value": world * q_per_step * args.compare_steps / (pms * 1e-3), "unit": "queries/s",
                "ms_per_step": pms / args.compare_steps, "steps": args.compare_steps,
                "form": ("banded: tcgen05 tiles of 128 queries" if other == 2
                         else "plain: windowed stabbing, CUDA-core descriptor distances")}
        mt.set_params(form={"auto": 0, "plain": 1, "banded": 2}[args.form])

    # the same nine pairs as one batch: one CUDA graph (egm_graph_launch) per
    # step, L2 flushed before every step, in the automatic and the plain form;
    # the outputs must equal the one-pair calls'
    same_batch = None
    if not args.no_compare:
        same_batch = {"workload": "the nine pairs above in one call", "api": "egm_graph_launch (one CUDA graph per step)"}
        single = {k: torch.cat([o[k][:s.m] for o, s in zip(outs, scs)]) for k in ("best", "second", "flags")}
        for name, form in (("auto", 0), ("plain", 1)):
            mt.set_params(form=form)
            mt.match_batch(dev)  # the first batch of a size class also tunes the band tile shape
            mt.set_timing(True)
            mt.match_batch(dev)
            banded_calls = mt.timing()["banded_calls"]
            mt.set_timing(False)
            bout = mt._alloc_out(q_per_step, False, 0)
            graph = mt.graph_create(dev, bout)
            for _ in range(3):
                flush.zero_()
                if graph.launch() != 0:
                    raise EgmError(mt.sync(), "nine-pair batch warm-up")
            torch.cuda.synchronize()
            for k in single:
                if not torch.equal(bout[k][:q_per_step], single[k]):
                    raise RuntimeError(f"nine-pair batch ({name}): {k} differs from the one-pair calls")
            pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.compare_steps)]
            for k in range(args.compare_steps):
                flush.zero_()
                pe[k][0].record(stream)
                graph.launch()
                pe[k][1].record(stream)
            torch.cuda.synchronize()
            st = mt.sync()
            if st != 0:
                raise EgmError(st, "nine-pair batch")
            graph.close()
            pms = max_over_ranks(sum(a.elapsed_time(b) for a, b in pe), world, local)
            same_batch[name] = {"value": world * q_per_step * args.compare_steps / (pms * 1e-3),
                                "unit": "queries/s", "ms_per_step": pms / args.compare_steps,
                                "steps": args.compare_steps,
                                "form": "banded" if banded_calls else "plain"}
        mt.set_params(form={"auto": 0, "plain": 1, "banded": 2}[args.form])

    # end to end: host (pinned) buffers through egm_match_pair_host, copies inside
    host = []
    h2d = d2h = 0
    for s in scs:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hs = type(s)(**{**s.__dict__})
        for k in ("xy1", "xy2", "F", "desc1", "desc2"):
            setattr(hs, k, pin(getattr(s, k)))
        host.append(hs)
        h2d += hs.xy1.nbytes + hs.xy2.nbytes + hs.F.nbytes + hs.desc1.nbytes + hs.desc2.nbytes
        d2h += s.m * (4 + 4 + 4 + 4 + 1)
    hbufs = []
    for hs in host:
        m = hs.m
        o = {k: torch.empty(m, dtype=dt).pin_memory().numpy() for k, dt in
             (("best", torch.int32), ("second", torch.int32), ("best_d", torch.float32),
              ("second_d", torch.float32), ("flags", torch.uint8))}
        hbufs.append(o)
    import ctypes as C

    hp = lambda a: a.ctypes.data_as(C.c_void_p)
    hpairs, houts = [], []
    for hs, o in zip(host, hbufs):
        p = _egm.egm_pair()
        p.xy1, p.xy2, p.F, p.eps2, p.eps_scalar = hp(hs.xy1), hp(hs.xy2), hp(hs.F), None, float(hs.eps)
        p.desc1, p.desc2 = hp(hs.desc1), hp(hs.desc2)
        p.m, p.n, p.kind, p.dim, p.width, p.height = hs.m, hs.n, hs.kind, hs.dim, hs.width, hs.height
        s_ = _egm.egm_out()
        s_.best, s_.second, s_.best_d, s_.second_d, s_.flags = (hp(o["best"]), hp(o["second"]),
                                                                hp(o["best_d"]), hp(o["second_d"]),
                                                                hp(o["flags"]))
        hpairs.append(p)
        houts.append(s_)

    def e2e_step():
        # the nine pairs in one call: each matched as by egm_match_pair, the
        # uploads of later pairs overlapping the matching of earlier ones
        st = mt.egm_match_batch_host(hpairs, houts)
        if st != 0:
            raise EgmError(st, "egm_match_batch_host")

    def e2e_step_per_call():
        for p, o in zip(hpairs, houts):
            st = mt.egm_match_pair_host(p, o)
            if st != 0:
                raise EgmError(st, "egm_match_pair_host")

    def time_e2e(fn, steps):
        for _ in range(3):
            fn()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world, local)
        barrier(world)
        for o, ref in zip(hbufs, outs):
            assert np.array_equal(o["best"], ref["best"].cpu().numpy()), "host path disagrees with device path"
            assert np.array_equal(o["flags"], ref["flags"].cpu().numpy()), "host path disagrees with device path"
        return world * q_per_step * steps / el

    e2e_value = time_e2e(e2e_step, args.e2e_steps)
    # the host link's copy rate: one pinned upload of a step's input bytes
    hsrc = torch.empty(int(h2d) // 4, dtype=torch.float32).pin_memory()
    hdst = torch.empty_like(hsrc, device=mt.device)
    for _ in range(3):
        hdst.copy_(hsrc, non_blocking=True)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(10):
        hdst.copy_(hsrc, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 10 * hsrc.numel() * 4 / (c0.elapsed_time(c1) * 1e-3) / 1e9
    del hsrc, hdst
    e2e_per_call = time_e2e(e2e_step_per_call, max(args.e2e_steps // 2, 1))

    # batched: 256 pairs with uneven counts in one CUDA-graph launch per step
    batched = None if args.no_batched else batched_leg(mt, torch, stream, args, world, local)

    # mutual matching and the match list, with recall / precision on the
    # scenes' true pairs (synthetic ground truth)
    matching = None
    if not args.no_matching:
        matching = matching_leg(mt, torch, stream, scs, dev, args.compare_steps)

    # tolerance and pose-noise sweeps
    sweeps = None
    if not args.no_sweeps:
        sweeps = sweeps_leg(mt, torch, stream, 10)

    # learned tolerance: training steps and inference of the 5-64-64-64-1 network
    mlp = None
    if not args.no_mlp:
        mlp = mlp_leg(mt, torch, stream)
        if not args.no_learned_experiment:
            mlp["experiment"] = learned_tolerance_experiment(mt, torch, stream, args)

    # kernels per match call: geometry, prep, bucket count, bucket scan, and
    # either the stab kernel or the query sort, pack and band kernels
    launches = 7 * n_banded + 5 * (len(scs) - n_banded)
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64/f32 geometry; u8 descriptors: int32 distances (plain form) and bf16 tensor-core "
                  "products with f32 sums (banded form), both exact integers"), "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs_per_step": len(scs), "queries_per_step": q_per_step,
                   "form": f"{args.form} one-pair (egm_match_pair)", "l2": "flushed before every step (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "api": "egm_match_batch_host: the nine pairs per call from pinned host memory, each matched as by "
                       "egm_match_pair, uploads on a copy stream overlapping the matching",
                "steps": args.e2e_steps,
                "h2d_gbs_measured": h2d_gbs,
                "h2d_bound_queries_per_s": q_per_step / (h2d / (h2d_gbs * 1e9)),
                "one_pair_per_call": {"value": e2e_per_call, "unit": "queries/s", "api": "egm_match_pair_host"}},
        "roofline": roofline,
        "batched": batched,
        "forced_forms_one_pair": other_form,
        "same_pairs_one_batch": same_batch,
        "learned_tolerance": mlp,
        "matching": matching,
        "sweeps": sweeps,
        "clocks": clk,
        "tuned_regimes": mt.tuner_entries(),
        "gpu_launches": launches * args.steps,
    }
    if cpu is not None:
        rate, cores, npairs, el = cpu
        # the CPU leg: the oracle, and beside it the paper's own data structure on the same cores
        line["cpu_baseline"] = {"value": rate, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                "sample": f"{npairs} config pairs (16384 queries each) cycled, {el:.1f} s",
                                "segment_tree": seg}
    if rank == 0:
        print(json.dumps(line), flush=True)
    mt.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist

        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
