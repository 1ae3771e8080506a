"""Seeded synthetic two-view scenes (inputs only).

This module draws the inputs that both the CUDA library and the CPU oracle
consume: keypoints in two images, the fundamental matrix of the true relative
pose, per-keypoint tolerances, descriptors and the ground-truth pairing known
to the generator.  It contains none of the matching method's arithmetic (no
epipoles, intervals, point-to-line distances or descriptor comparisons).

The fundamental matrix follows the paper's Eq. (F = K2^-T [t]x R K1^-1) with
the convention x2 = R x1 + t between camera frames, so that a true
correspondence satisfies p2^T F p1 = 0 (Sec. 3).

The workloads stand in for the paper's ETH3D experiments (6048x4032 images,
up to 50k SIFT keypoints, Sec. 5.1); no dataset item is reproduced.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DESC_U8_L2 = 0
DESC_F32_L2 = 1
DESC_BIN256 = 2

HIGHRES_W, HIGHRES_H, HIGHRES_F = 6048, 4032, 4800.0


@dataclass
class Scene:
    """One image pair.  Arrays are C-contiguous numpy arrays."""

    xy1: np.ndarray            # (m, 2) float64, image-1 query keypoints (px)
    xy2: np.ndarray            # (n, 2) float64, image-2 reference keypoints (px)
    F: np.ndarray              # (3, 3) float64, p2^T F p1 = 0
    eps: np.ndarray | float    # (n,) float64 per reference keypoint, or a scalar
    desc1: np.ndarray          # (m, row) uint8 / float32
    desc2: np.ndarray          # (n, row)
    kind: int                  # DESC_*
    dim: int                   # elements (u8, f32) or bits (binary)
    width: int
    height: int
    gt: np.ndarray             # (t, 2) int64 true pairs (i in image 1, j in image 2)
    meta: dict = field(default_factory=dict)
    feat2: np.ndarray | None = None   # (n, 5) float64 keypoint features (scale, orientation, response, x/W, y/H)
    feat1: np.ndarray | None = None   # (m, 5) for image-1 keypoints

    @property
    def m(self) -> int:
        return int(self.xy1.shape[0])

    @property
    def n(self) -> int:
        return int(self.xy2.shape[0])

    def eps_array(self) -> np.ndarray:
        if np.isscalar(self.eps) or np.ndim(self.eps) == 0:
            return np.full(self.n, float(self.eps))
        return np.asarray(self.eps, dtype=np.float64)


def intrinsics(f: float, w: int, h: int) -> np.ndarray:
    return np.array([[f, 0.0, w / 2.0], [0.0, f, h / 2.0], [0.0, 0.0, 1.0]])


def rotation(axis, degrees: float) -> np.ndarray:
    """Rodrigues rotation about `axis` by `degrees`."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    th = math.radians(degrees)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(th) * k + (1 - math.cos(th)) * (k @ k)


def skew(t) -> np.ndarray:
    t = np.asarray(t, dtype=np.float64)
    return np.array([[0, -t[2], t[1]], [t[2], 0, -t[0]], [-t[1], t[0], 0]])


def fundamental(K1, K2, R, t) -> np.ndarray:
    """F = K2^-T [t]x R K1^-1 (paper, Eq. F of Sec. 3)."""
    return np.linalg.inv(K2).T @ skew(t) @ R @ np.linalg.inv(K1)


def _project_true_points(rng, n_true, K1, K2, R, t, w, h, depth=(2.0, 10.0)):
    """Draw n_true 3D points visible in both views; return pixel coords."""
    K1i = np.linalg.inv(K1)
    out1 = np.empty((0, 2))
    out2 = np.empty((0, 2))
    tries = 0
    while out1.shape[0] < n_true:
        tries += 1
        if tries > 200:
            raise RuntimeError("pose leaves too few points visible in image 2")
        k = max(1024, 2 * (n_true - out1.shape[0]))
        uv = rng.uniform([0.0, 0.0], [w, h], size=(k, 2))
        z = rng.uniform(depth[0], depth[1], size=k)
        ray = (K1i @ np.vstack([uv.T, np.ones(k)])).T
        X1 = ray * z[:, None]
        X2 = X1 @ R.T + np.asarray(t)[None, :]
        ok = X2[:, 2] > 1e-3
        p = (K2 @ X2.T).T
        with np.errstate(divide="ignore", invalid="ignore"):
            q = p[:, :2] / p[:, 2:3]
        ok &= (q[:, 0] >= 0) & (q[:, 0] < w) & (q[:, 1] >= 0) & (q[:, 1] < h)
        out1 = np.vstack([out1, uv[ok]])
        out2 = np.vstack([out2, q[ok]])
    return out1[:n_true], out2[:n_true]


def _u8_desc(rng, n_true, n_out1, n_out2, dim=128, sigma=8.0):
    base = rng.integers(0, 256, size=(n_true, dim)).astype(np.float64)
    d1 = np.clip(np.rint(base + rng.normal(0, sigma, base.shape)), 0, 255)
    d2 = np.clip(np.rint(base + rng.normal(0, sigma, base.shape)), 0, 255)
    o1 = rng.integers(0, 256, size=(n_out1, dim))
    o2 = rng.integers(0, 256, size=(n_out2, dim))
    return (np.vstack([d1, o1]).astype(np.uint8), np.vstack([d2, o2]).astype(np.uint8))


def _bin_desc(rng, n_true, n_out1, n_out2, bits=256, p_flip=0.08):
    nb = bits // 8
    base = rng.integers(0, 2, size=(n_true, bits), dtype=np.uint8)
    f1 = (rng.random((n_true, bits)) < p_flip).astype(np.uint8)
    f2 = (rng.random((n_true, bits)) < p_flip).astype(np.uint8)
    v1 = np.vstack([base ^ f1, rng.integers(0, 2, size=(n_out1, bits), dtype=np.uint8)])
    v2 = np.vstack([base ^ f2, rng.integers(0, 2, size=(n_out2, bits), dtype=np.uint8)])
    return (np.packbits(v1, axis=1, bitorder="little").reshape(-1, nb),
            np.packbits(v2, axis=1, bitorder="little").reshape(-1, nb))


def _rootsift_like(rng, k, dim):
    g = rng.gamma(0.5, 1.0, size=(k, dim))
    g /= np.maximum(g.sum(axis=1, keepdims=True), 1e-300)
    return np.sqrt(g)


def _f32_desc(rng, n_true, n_out1, n_out2, dim=128, sigma=0.02):
    base = _rootsift_like(rng, n_true, dim)

    def view(b):
        v = b + rng.normal(0, sigma, b.shape)
        return v / np.linalg.norm(v, axis=1, keepdims=True)

    d1 = np.vstack([view(base), _rootsift_like(rng, n_out1, dim)])
    d2 = np.vstack([view(base), _rootsift_like(rng, n_out2, dim)])
    return d1.astype(np.float32), d2.astype(np.float32)


def make_pair(rng, *, w, h, K1, K2, R, t, m, n, n_true, noise=0.5, eps=2.0,
              kind=DESC_U8_L2, dim=128, depth=(2.0, 10.0), scale_model=False,
              meta=None) -> Scene:
    """One scene: n_true true projections plus uniform outliers in each image.

    The order of keypoints is shuffled independently in each image, so index
    order carries no information about the pairing.
    """
    n_true = int(min(n_true, m, n))
    p1, p2 = _project_true_points(rng, n_true, K1, K2, R, t, w, h, depth)
    feat1 = feat2 = None
    if scale_model:
        # per 3D point: scale s ~ logU[1,16], localisation noise 0.3*s in both views
        s = np.exp(rng.uniform(math.log(1.0), math.log(16.0), size=n_true))
        p1 = p1 + rng.normal(0, 1, p1.shape) * (0.3 * s)[:, None]
        p2 = p2 + rng.normal(0, 1, p2.shape) * (0.3 * s)[:, None]
        so1 = np.exp(rng.uniform(0.0, math.log(16.0), size=m - n_true))
        so2 = np.exp(rng.uniform(0.0, math.log(16.0), size=n - n_true))
        s1 = np.concatenate([s, so1])
        s2 = np.concatenate([s, so2])
    else:
        p1 = p1 + rng.normal(0, noise, p1.shape)
        p2 = p2 + rng.normal(0, noise, p2.shape)
    o1 = rng.uniform([0.0, 0.0], [w, h], size=(m - n_true, 2))
    o2 = rng.uniform([0.0, 0.0], [w, h], size=(n - n_true, 2))
    xy1 = np.vstack([p1, o1])
    xy2 = np.vstack([p2, o2])
    if kind == DESC_U8_L2:
        d1, d2 = _u8_desc(rng, n_true, m - n_true, n - n_true, dim)
    elif kind == DESC_BIN256:
        d1, d2 = _bin_desc(rng, n_true, m - n_true, n - n_true, dim)
    elif kind == DESC_F32_L2:
        d1, d2 = _f32_desc(rng, n_true, m - n_true, n - n_true, dim)
    else:
        raise ValueError(kind)
    if scale_model:
        def feats(xy, sc):
            k = xy.shape[0]
            ori = rng.uniform(0, 2 * math.pi, size=k)
            resp = (1.0 / sc) * np.exp(rng.normal(0, 0.3, size=k))
            return np.stack([sc, ori, resp, xy[:, 0] / w, xy[:, 1] / h], axis=1)
        feat1 = feats(xy1, s1)
        feat2 = feats(xy2, s2)
    perm1 = rng.permutation(m)
    perm2 = rng.permutation(n)
    inv1 = np.empty(m, np.int64)
    inv1[perm1] = np.arange(m)
    inv2 = np.empty(n, np.int64)
    inv2[perm2] = np.arange(n)
    gt = np.stack([inv1[:n_true], inv2[:n_true]], axis=1)
    sc = Scene(
        xy1=np.ascontiguousarray(xy1[perm1]), xy2=np.ascontiguousarray(xy2[perm2]),
        F=fundamental(K1, K2, R, t), eps=eps,
        desc1=np.ascontiguousarray(d1[perm1]), desc2=np.ascontiguousarray(d2[perm2]),
        kind=kind, dim=dim, width=w, height=h, gt=gt, meta=dict(meta or {}),
        feat1=None if feat1 is None else np.ascontiguousarray(feat1[perm1]),
        feat2=None if feat2 is None else np.ascontiguousarray(feat2[perm2]))
    sc.meta.update(dict(R=R, t=np.asarray(t, dtype=np.float64), K1=K1, K2=K2))
    return sc


# --------------------------------------------------------------------------
# The five workloads.  `scale` shrinks keypoint counts for quick tests.
# --------------------------------------------------------------------------

def config1(seed: int = 0, scale: float = 1.0) -> Scene:
    """640x480, f=500, R=10 deg about y, |t|=0.3 (mostly sideways), 1500 true + 500 outliers."""
    rng = np.random.default_rng(seed)
    K = intrinsics(500.0, 640, 480)
    R = rotation([0, 1, 0], 10.0)
    t = 0.3 * np.array([1.0, 0.0, 0.1]) / np.linalg.norm([1.0, 0.0, 0.1])
    n_true = max(1, int(round(1500 * scale)))
    cnt = n_true + int(round(500 * scale))
    return make_pair(rng, w=640, h=480, K1=K, K2=K, R=R, t=t, m=cnt, n=cnt,
                     n_true=n_true, noise=0.5, eps=2.0, kind=DESC_U8_L2, dim=128,
                     meta=dict(config=1, seed=seed))


CONFIG2_POSES = {
    "inside": (0.05, 0.03, 1.0),     # forward motion: epipole inside the image
    "far": (1.0, 0.2, 0.01),         # epipole ~5e5 px away
    "infinity": (1.0, 0.3, 0.0),     # pure sideways: epipole at infinity
}


def config2(pose: str = "inside", eps: float = 2.0, seed: int | None = None,
            scale: float = 1.0) -> Scene:
    """6048x4032, f=4800, 16384 keypoints per image (70% true), R=5 deg about a random axis."""
    names = list(CONFIG2_POSES)
    if seed is None:
        seed = names.index(pose)
    rng = np.random.default_rng(seed)
    K = intrinsics(HIGHRES_F, HIGHRES_W, HIGHRES_H)
    axis = rng.normal(size=3)
    R = rotation(axis, 5.0)
    t = np.array(CONFIG2_POSES[pose], dtype=np.float64)
    cnt = max(2, int(round(16384 * scale)))
    n_true = int(round(0.7 * cnt))
    return make_pair(rng, w=HIGHRES_W, h=HIGHRES_H, K1=K, K2=K, R=R, t=t, m=cnt, n=cnt,
                     n_true=n_true, noise=0.5, eps=float(eps), kind=DESC_U8_L2, dim=128,
                     meta=dict(config=2, pose=pose, seed=seed))


def perturb_pose(sc: Scene, level: float, seed: int = 0) -> np.ndarray:
    """F of the scene's true pose with pose noise of the given level: the
    rotation perturbed about each axis by U[-level, level] degrees and each
    translation component by U[-0.25 level, 0.25 level] scene units (the
    paper's noise model, Sec. 5.5; a scene unit plays the metre, depths are
    2 to 10 units)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-level, level, 3)
    dR = rotation([0, 0, 1], a[2]) @ rotation([0, 1, 0], a[1]) @ rotation([1, 0, 0], a[0])
    dt = rng.uniform(-0.25 * level, 0.25 * level, 3)
    m = sc.meta
    return fundamental(m["K1"], m["K2"], dR @ m["R"], np.asarray(m["t"], np.float64) + dt)


def _random_pose(rng, max_deg):
    axis = rng.normal(size=3)
    R = rotation(axis, rng.uniform(0.0, max_deg))
    t = rng.normal(size=3)
    return R, t / np.linalg.norm(t)


def config3(seed: int = 0, npairs: int = 256, scale: float = 1.0,
            lo: int = 1024, hi: int = 32768, only=None) -> list[Scene]:
    """Batched: per-image counts log-uniform in [lo, hi]; u8 L2 on even pairs, 256-bit binary on odd.

    `only`: indices of the pairs to build (the others are drawn and skipped, so
    pair p is the same scene whether or not its neighbours are built)."""
    rng = np.random.default_rng(seed)
    K = intrinsics(HIGHRES_F, HIGHRES_W, HIGHRES_H)
    out = []
    keep = None if only is None else set(int(x) for x in only)
    for p in range(npairs):
        m = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))) * scale)
        n = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))) * scale)
        m, n = max(m, 2), max(n, 2)
        R, t = _random_pose(rng, 30.0)
        if keep is not None and p not in keep:
            continue
        kind = DESC_U8_L2 if p % 2 == 0 else DESC_BIN256
        dim = 128 if kind == DESC_U8_L2 else 256
        sub = np.random.default_rng([seed, p])
        out.append(make_pair(sub, w=HIGHRES_W, h=HIGHRES_H, K1=K, K2=K, R=R, t=t, m=m, n=n,
                             n_true=int(0.7 * min(m, n)), noise=0.5, eps=2.0, kind=kind,
                             dim=dim, meta=dict(config=3, seed=seed, pair=p)))
    return out


def config4(seed: int = 0, npairs: int = 64, scale: float = 1.0) -> list[Scene]:
    """Float descriptors: 128-d RootSIFT-like f32, 16384 keypoints, epipole far outside."""
    K = intrinsics(HIGHRES_F, HIGHRES_W, HIGHRES_H)
    out = []
    for p in range(npairs):
        rng = np.random.default_rng([seed, 4, p])
        R = rotation(rng.normal(size=3), 5.0)
        t = np.array(CONFIG2_POSES["far"])
        cnt = max(2, int(round(16384 * scale)))
        out.append(make_pair(rng, w=HIGHRES_W, h=HIGHRES_H, K1=K, K2=K, R=R, t=t, m=cnt, n=cnt,
                             n_true=int(round(0.7 * cnt)), noise=0.5, eps=2.0,
                             kind=DESC_F32_L2, dim=128, meta=dict(config=4, seed=seed, pair=p)))
    return out


def config5(seed: int = 0, npairs: int = 512, scale: float = 1.0, only=None) -> list[Scene]:
    """Scale-dependent localisation noise (sigma = 0.3 s) for the learned per-keypoint tolerance.

    Pair p draws from its own generator, so `only` (indices of the pairs to
    build) gives the same scenes as the full list."""
    K = intrinsics(HIGHRES_F, HIGHRES_W, HIGHRES_H)
    out = []
    for p in (range(npairs) if only is None else only):
        rng = np.random.default_rng([seed, 5, int(p)])
        m = max(2, int(rng.integers(4096, 16385) * scale))
        n = max(2, int(rng.integers(4096, 16385) * scale))
        R, t = _random_pose(rng, 30.0)
        out.append(make_pair(rng, w=HIGHRES_W, h=HIGHRES_H, K1=K, K2=K, R=R, t=t, m=m, n=n,
                             n_true=int(0.7 * min(m, n)), eps=2.0, kind=DESC_U8_L2, dim=128,
                             scale_model=True, meta=dict(config=5, seed=seed, pair=int(p))))
    return out


def uniform_pair(rng, m, n, F, *, w=640, h=480, eps=2.0, kind=DESC_U8_L2, dim=128,
                 margin=0.0) -> Scene:
    """Keypoints uniform over [-margin, w+margin] x [-margin, h+margin] with random descriptors."""
    xy1 = rng.uniform([-margin, -margin], [w + margin, h + margin], size=(m, 2))
    xy2 = rng.uniform([-margin, -margin], [w + margin, h + margin], size=(n, 2))
    if kind == DESC_U8_L2:
        d1 = rng.integers(0, 256, size=(m, dim), dtype=np.uint8)
        d2 = rng.integers(0, 256, size=(n, dim), dtype=np.uint8)
    elif kind == DESC_BIN256:
        d1 = rng.integers(0, 256, size=(m, dim // 8), dtype=np.uint8)
        d2 = rng.integers(0, 256, size=(n, dim // 8), dtype=np.uint8)
    else:
        d1 = _rootsift_like(rng, m, dim).astype(np.float32)
        d2 = _rootsift_like(rng, n, dim).astype(np.float32)
    return Scene(xy1=xy1, xy2=xy2, F=np.asarray(F, dtype=np.float64), eps=eps, desc1=d1,
                 desc2=d2, kind=kind, dim=dim, width=w, height=h,
                 gt=np.zeros((0, 2), np.int64))


# --------------------------------------------------------------------------
# Initial weights of the tolerance network (random numbers only).
# Flat layout: W1 (64,5), b1 (64), W2 (64,64), b2 (64), W3 (64,64), b3 (64),
# W4 (1,64), b4 (1); rows are output units.
# --------------------------------------------------------------------------
MLP_SIZES = ((64, 5), (64, 64), (64, 64), (1, 64))


def mlp_param_count() -> int:
    return sum(o * i + o for o, i in MLP_SIZES)


def mlp_init(seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and zero biases, float32."""
    rng = np.random.default_rng([seed, 77])
    parts = []
    for o, i in MLP_SIZES:
        bound = 1.0 / math.sqrt(i)
        parts.append(rng.uniform(-bound, bound, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)
