"""Seeded synthetic 3DGS scenes: the inputs both the CUDA path and the CPU oracle consume.

This module only draws random numbers. It holds none of the codec's arithmetic
(no scaling, quantisation, ordering, block coding or SH evaluation), so it can be
shared by the tests, the benchmark and the oracle without coupling them.

What is generated stands in for the trained scenes of the paper's experiments
(Sec. V-A: bicycle, bonsai, garden), which are not available here:

* positions ``p`` in [0, 1]^3, drawn from a mixture of ``clusters`` isotropic
  Gaussians (centres uniform in [0.1, 0.9]^3, sigma 0.05, clipped to the cube);
  each Gaussian's cluster is drawn independently, so storage order is not
  spatially coherent;
* premultiplied SH colour coefficients ``H~ = mu H`` (Sec. II, Eq. premult),
  shape [N, 16, 3] float32, coefficient k = l*l + l + m:
  DC (k = 0) ~ N(0, 0.8), band l >= 1 ~ N(0, 0.15 / (l + 1)) (standard deviations);
  optionally a heavy-tailed fraction whose bands 2-3 are Laplace(0, 0.3);
* view directions uniform on the unit sphere, and camera centres uniform on a
  sphere of radius 2 around (0.5, 0.5, 0.5);
* for rendering (Sec. II), per-Gaussian geometry: scales ``s`` (log-normal around a
  given size, per axis), rotation quaternions ``q`` (normal draws, not normalised)
  and opacity logits ``t`` ~ N(0, 1.5); and pinhole cameras on the same sphere
  looking at (0.5, 0.5, 0.5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SH_COEFFS = 16


def band_of(k: int) -> int:
    """SH band l of coefficient index k = l*l + l + m."""
    l = 0
    while (l + 1) * (l + 1) <= k:
        l += 1
    return l


@dataclass
class Scene:
    pos: np.ndarray  # [N, 3] float32
    sh: np.ndarray   # [N, 16, 3] float32, premultiplied by opacity


def make_scene(n: int, seed: int, clusters: int = 8, heavy_frac: float = 0.0) -> Scene:
    """Draw one synthetic scene of ``n`` Gaussians (see module docstring)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, size=(clusters, 3))
    which = rng.integers(0, clusters, size=n)
    pos = centres[which] + rng.normal(0.0, 0.05, size=(n, 3))
    pos = np.clip(pos, 0.0, 1.0).astype(np.float32)
    std = np.array([0.8] + [0.15 / (band_of(k) + 1) for k in range(1, SH_COEFFS)], dtype=np.float64)
    sh = rng.standard_normal(size=(n, SH_COEFFS, 3)) * std[None, :, None]
    if heavy_frac > 0.0:
        heavy = rng.random(n) < heavy_frac
        idx = np.nonzero(heavy)[0]
        k_hi = np.arange(4, SH_COEFFS)  # bands 2 and 3
        sh[np.ix_(idx, k_hi, np.arange(3))] = rng.laplace(0.0, 0.3, size=(idx.size, k_hi.size, 3))
    return Scene(pos=pos, sh=sh.astype(np.float32))


def make_dirs(v: int, seed: int) -> np.ndarray:
    """``v`` unit view directions, uniform on the sphere, [V, 3] float32."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(size=(v, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


def make_cams(v: int, seed: int, radius: float = 2.0) -> np.ndarray:
    """``v`` camera centres uniform on a sphere of ``radius`` around the cube centre, [V, 3] float32."""
    return (0.5 + radius * make_dirs(v, seed).astype(np.float64)).astype(np.float32)


# The benchmark configurations, by what they are.
TINY = dict(n=4096, seed=1001, clusters=8, heavy_frac=0.0)              # 4,096 Gaussians, BC1, 16 shared dirs
MEDIUM = dict(n=262144, seed=1002, clusters=8, heavy_frac=0.0)          # 262,144 Gaussians, BC1/BC7/rate
SCENE = dict(n=3000000, seed=1003, clusters=64, heavy_frac=0.10)        # 3M Gaussians, 64 clusters, 10% heavy tail


def batch_sizes(n_scenes: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Scene sizes log-uniform in [lo, hi] (batched and served workloads)."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_scenes)).astype(np.int64)


# Batched workload: 64 scenes, sizes log-uniform in [50,000, 2,000,000], the scene-scale
# value distributions; formats cycle BC1, BC7, rate-controlled, the rate targets cycle
# 3, 4, 6, 8 bits per texel (given x4).
BATCH = dict(n_scenes=64, seed=2000, lo=50_000, hi=2_000_000)


def batch_mix(n_scenes: int, seed: int, lo: int, hi: int):
    """[(n, scene seed, format name, rate target x4)] of the batched workload."""
    sizes = batch_sizes(n_scenes, seed, lo, hi)
    out = []
    for i, n in enumerate(sizes):
        fmt = ("bc1", "bc7", "rate")[i % 3]
        out.append((int(n), seed + 1 + i, fmt, (12, 16, 24, 32)[(i // 3) % 4] if fmt == "rate" else 0))
    return out


# Served workload: a pool of scenes of 10,000..4,000,000 Gaussians (log-uniform), half BC1 and
# half BC7, and a Poisson stream of requests (mean 200 per second): a re-encode of a pool scene
# with probability encode_frac, else a decode + SH evaluation of a pool scene for 1..32 camera
# centres (uniform).
SERVE = dict(n_scenes=32, seed=3000, lo=10_000, hi=4_000_000, rate_hz=200.0, encode_frac=0.1)


def serve_trace(n_scenes: int, seed: int, lo: int, hi: int, rate_hz: float, encode_frac: float, seconds: float):
    """(pool [(n, scene seed, format name)], requests [(t_arrival_s, kind, scene, V, cams seed)])."""
    sizes = batch_sizes(n_scenes, seed, lo, hi)
    pool = [(int(n), seed + 1 + i, ("bc1", "bc7")[i % 2]) for i, n in enumerate(sizes)]
    rng = np.random.default_rng(seed + 999)
    reqs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= seconds:
            break
        kind = "encode" if rng.random() < encode_frac else "eval"
        reqs.append((t, kind, int(rng.integers(n_scenes)), int(rng.integers(1, 33)), int(rng.integers(1 << 30))))
    return pool, reqs


@dataclass
class Geometry:
    scale: np.ndarray  # [N, 3] float32, linear axis scales s (Eq. covar)
    rot: np.ndarray    # [N, 4] float32, rotation quaternion (w, x, y, z), not normalised
    logit: np.ndarray  # [N] float32, opacity logits t (Eq. sigmoid)


def make_geometry(n: int, seed: int, scale: float = 0.004) -> Geometry:
    """Per-Gaussian shape and opacity parameters for rendering."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.normal(np.log(scale), 0.35, size=(n, 3)))
    q = rng.standard_normal(size=(n, 4))
    t = rng.normal(0.0, 1.5, size=n)
    return Geometry(scale=s.astype(np.float32), rot=q.astype(np.float32), logit=t.astype(np.float32))


def look_at(eye, target, width: int, height: int, fov_x_deg: float = 50.0, near: float = 0.2) -> dict:
    """A pinhole camera at ``eye`` looking at ``target``: world -> camera rotation R (rows: image
    right, image down, viewing direction) and translation t = -R eye; focal length from the
    horizontal field of view, principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.95 else np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    f = 0.5 * width / np.tan(np.radians(fov_x_deg) / 2)
    return dict(R=R.astype(np.float32).reshape(9), t=t.astype(np.float32), fx=np.float32(f), fy=np.float32(f),
                cx=np.float32(width / 2), cy=np.float32(height / 2), width=int(width), height=int(height),
                near_z=np.float32(near))


def make_views(count: int, seed: int, width: int, height: int, radius: float = 2.0, fov_x_deg: float = 50.0):
    """``count`` cameras on a sphere of ``radius`` around (0.5, 0.5, 0.5), looking at it."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(size=(count, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c = np.array([0.5, 0.5, 0.5])
    return [look_at(c + radius * d[i], c, width, height, fov_x_deg) for i in range(count)]


RENDER = dict(n=3000000, seed=1003, clusters=64, heavy_frac=0.10, geom_seed=1103, scale=0.004,
              width=1920, height=1080, views=4, view_seed=1203)    # the 3M scene rendered at 1080p
