"""Seeded synthetic scenes, cameras and targets for the 3D Gabor splatting rasterizer.

This module only draws random numbers and builds camera poses. It holds none of the
rasterizer's arithmetic (no projection, no splatting, no compositing), so that both the
CUDA path and the FP64 oracle can consume exactly the same inputs without sharing code.

Scene recipes (all attributes are returned already activated, as the rasterizer expects:
positive scales, opacity and Gabor weights in [0, 1)):

* ``tiny``/config 0: n=256, K=2, SH degree 0.  means ~ U[-1,1]^3, log-scale ~ N(-2.5, 0.5),
  quaternions = normalised N(0, I4), opacity = sigmoid(N(0,1)), frequency direction uniform
  on S^2 with magnitude U[0, 8] cycles per world unit, weights ~ U[0, 1], SH ~ N(0, 0.2).
  Camera at distance 4 looking at the origin, 60 deg horizontal field of view, 128x128.
* config 1: n=50k, K=4, SH degree 3; means from a 32-component isotropic Gaussian mixture
  (centres U[-3,3]^3, sigma 0.3); log-scale ~ N(-4, 0.7); the rest as config 0; 800x800.
* config 2: n=1.5M, K=4, SH degree 3; 80% of means from a 64-component mixture (centres
  U[-4,4]^3, sigma 0.3) and 20% on a background shell (radius U[20,40], direction uniform);
  log-scale ~ N(-4, 0.7); 1600x1064; 16 orbit poses of radius 4 at azimuth 22.5 deg * j.
* config 3: eight config-2-style scenes of {100k .. 3M} primitives, BF16 storage.
* config 4: n=3M as config 2 at 1920x1080 with K in {0, 1, 2, 4, 8}.

The paper's datasets (Mip-NeRF 360, Tanks & Temples, Deep Blending) are not available;
these scenes stand in for them with primitive counts that bracket the paper's 2.74M
(Table 3) and a training-view resolution of the same order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CONFIG_SEED_BASE = 1000
SERVE_SEED = 2000


@dataclass
class SceneSpec:
    n: int
    K: int
    sh_degree: int
    layout: str            # "uniform" | "mixture" | "mixture+shell"
    box: float = 1.0       # half-width of the uniform box / mixture centre box
    n_clusters: int = 0
    cluster_sigma: float = 0.3
    shell_frac: float = 0.0
    shell_r: tuple = (20.0, 40.0)
    log_scale: tuple = (-2.5, 0.5)
    freq_max: float = 8.0
    sh_sigma: float = 0.2


@dataclass
class CameraSpec:
    width: int
    height: int
    fov_x_deg: float = 60.0
    radius: float = 4.0
    znear: float = 0.2
    zfar: float = 100.0
    poses: list = field(default_factory=lambda: [(0.0, 0.0)])  # (azimuth, elevation) in degrees


CONFIGS = {
    0: (SceneSpec(n=256, K=2, sh_degree=0, layout="uniform", box=1.0, log_scale=(-2.5, 0.5)),
        CameraSpec(128, 128)),
    1: (SceneSpec(n=50_000, K=4, sh_degree=3, layout="mixture", box=3.0, n_clusters=32,
                  log_scale=(-4.0, 0.7)),
        CameraSpec(800, 800)),
    2: (SceneSpec(n=1_500_000, K=4, sh_degree=3, layout="mixture+shell", box=4.0, n_clusters=64,
                  shell_frac=0.2, log_scale=(-4.0, 0.7)),
        CameraSpec(1600, 1064, poses=[(22.5 * j, 0.0) for j in range(16)])),
    4: (SceneSpec(n=3_000_000, K=4, sh_degree=3, layout="mixture+shell", box=4.0, n_clusters=64,
                  shell_frac=0.2, log_scale=(-4.0, 0.7)),
        CameraSpec(1920, 1080, poses=[(22.5 * j, 0.0) for j in range(16)])),
}
SERVE_SCENE_SIZES = [100_000, 250_000, 500_000, 1_000_000, 1_500_000, 2_000_000, 2_500_000, 3_000_000]
SERVE_RESOLUTIONS = [(400, 400), (800, 800), (1280, 720), (1920, 1080)]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def make_scene(spec: SceneSpec, seed: int, n: int | None = None, K: int | None = None) -> dict:
    """Draw one scene.  Returns float32 arrays:

    means [n,3], scales [n,3] (>0), quats [n,4] (w,x,y,z, unit norm), opacity [n] in (0,1),
    sh [n,(d+1)^2,3], freqs [n,K,3] (world frame, cycles per unit), weights [n,K] in [0,1).
    """
    n = spec.n if n is None else n
    K = spec.K if K is None else K
    rng = _rng(seed)
    if spec.layout == "uniform":
        means = rng.uniform(-spec.box, spec.box, (n, 3))
    else:
        n_shell = int(round(n * spec.shell_frac))
        n_mix = n - n_shell
        centres = rng.uniform(-spec.box, spec.box, (spec.n_clusters, 3))
        comp = rng.integers(0, spec.n_clusters, n_mix)
        mix = centres[comp] + rng.standard_normal((n_mix, 3)) * spec.cluster_sigma
        if n_shell:
            r = rng.uniform(spec.shell_r[0], spec.shell_r[1], n_shell)
            shell = _unit_vectors(rng, n_shell) * r[:, None]
            means = np.concatenate([mix, shell], 0)
            means = means[rng.permutation(n)]
        else:
            means = mix
    log_s = rng.normal(spec.log_scale[0], spec.log_scale[1], (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.standard_normal(n)))
    nsh = (spec.sh_degree + 1) ** 2
    sh = rng.normal(0.0, spec.sh_sigma, (n, nsh, 3))
    fdir = _unit_vectors(rng, n * K).reshape(n, K, 3)
    fmag = rng.uniform(0.0, spec.freq_max, (n, K, 1))
    freqs = fdir * fmag
    weights = rng.uniform(0.0, 1.0, (n, K))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(means=f32(means), scales=f32(np.exp(log_s)), quats=f32(q), opacity=f32(opacity),
                sh=f32(sh), freqs=f32(freqs.reshape(n, K, 3)), weights=f32(weights.reshape(n, K)),
                sh_degree=spec.sh_degree, K=K, n=n)


def look_at(eye, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)):
    """World->camera rotation R (rows = camera x right, y down, z forward) and translation t."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(down, np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    t = -R @ eye
    return R, t


def make_camera(width, height, fov_x_deg=60.0, eye=(0.0, 0.0, -4.0), target=(0.0, 0.0, 0.0),
                znear=0.2, zfar=100.0) -> dict:
    R, t = look_at(eye, target)
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return dict(R=np.ascontiguousarray(R, np.float32), t=np.ascontiguousarray(t, np.float32),
                fx=float(np.float32(fx)), fy=float(np.float32(fx)),
                cx=float(np.float32(0.5 * width)), cy=float(np.float32(0.5 * height)),
                width=int(width), height=int(height), znear=float(np.float32(znear)),
                zfar=float(np.float32(zfar)))


def orbit_camera(width, height, azimuth_deg, elevation_deg=0.0, radius=4.0, fov_x_deg=60.0,
                 znear=0.2, zfar=100.0) -> dict:
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    eye = (radius * math.cos(el) * math.sin(az), -radius * math.sin(el), -radius * math.cos(el) * math.cos(az))
    return make_camera(width, height, fov_x_deg, eye, (0.0, 0.0, 0.0), znear, zfar)


def config_scene(cfg: int, **kw) -> dict:
    spec, _ = CONFIGS[cfg]
    return make_scene(spec, CONFIG_SEED_BASE + cfg, **kw)


def config_cameras(cfg: int, width=None, height=None) -> list:
    _, cs = CONFIGS[cfg]
    w = cs.width if width is None else width
    h = cs.height if height is None else height
    return [orbit_camera(w, h, az, el, cs.radius, cs.fov_x_deg, cs.znear, cs.zfar) for az, el in cs.poses]


def make_target(width, height, seed) -> np.ndarray:
    """Seeded uniform-random target image, [3, H, W] float32 in [0, 1)."""
    return _rng(seed).uniform(0.0, 1.0, (3, height, width)).astype(np.float32)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns float32 values."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """The uint16 bit patterns of bf16_round(x) (for uploading BF16 storage)."""
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def serve_scenes(sizes=None) -> list:
    spec, _ = CONFIGS[2]
    sizes = SERVE_SCENE_SIZES if sizes is None else sizes
    return [make_scene(spec, 3000 + i, n=n) for i, n in enumerate(sizes)]


def serve_requests(n_req=2000, rate=200.0, n_scenes=8, seed=SERVE_SEED, resolutions=None) -> list:
    """Poisson request stream: list of dicts (arrival_s, scene, width, height, azimuth, elevation)."""
    rng = _rng(seed)
    res = SERVE_RESOLUTIONS if resolutions is None else resolutions
    gaps = rng.exponential(1.0 / rate, n_req)
    arrivals = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n_req):
        w, h = res[int(rng.integers(0, len(res)))]
        out.append(dict(arrival_s=float(arrivals[i]), scene=int(rng.integers(0, n_scenes)), width=w, height=h,
                        azimuth=float(rng.uniform(0.0, 360.0)), elevation=float(rng.uniform(-30.0, 30.0))))
    return out
