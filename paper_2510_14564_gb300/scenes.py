"""Seeded synthetic scenes and cameras for the 3DGS training hot path.

This module only draws random numbers and builds camera matrices.  It holds
none of the method's arithmetic (no projection, no blending, no gradients), so
the CUDA path and the CPU oracle can both be fed from it without sharing code.

Workload recipes (the paper trains on Mip-NeRF360, Tanks&Temples and Deep
Blending; those captures are not available, so seeded synthetic scenes with the
same skewed-density structure stand in for them, see Sec. III-A where dense
regions hold up to 100x the Gaussians of sparse ones):

* uniform scene: means ~ U[-1,1]^3, log-scales ~ N(-4, 0.5), rotations are
  normalised N(0, I4) quaternions, opacity logits ~ N(0, 1), all 48 degree-3
  SH coefficients ~ N(0, 0.2).
* skewed scene: 80% of the means fall in 20 tight clusters (centres
  U[-1,1]^3 drawn from their own seed, member offsets N(0, 0.02^2 I)), the
  other 20% are uniform; every other attribute as above.

Cameras are pinhole, 60 degree horizontal field of view, looking at the
origin from distance 3; the image y axis points along world +y.

Seeds: scene 0, target scene 1, cluster centres 2, views 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_COEFFS = 16          # degree 3: (3 + 1)^2 coefficients per colour channel
PARAM_FLOATS = 3 + 3 + 4 + 1 + SH_COEFFS * 3   # 59 floats per Gaussian
TILE = 16


@dataclass
class Camera:
    """Pinhole camera; world->camera is p_cam = R @ p_world + t."""
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray                       # (3, 3) float32, rows = camera axes
    t: np.ndarray                       # (3,) float32
    znear: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)

    @property
    def campos(self) -> np.ndarray:
        """Camera centre in world space, -R^T t, rounded to float32."""
        R = self.R.astype(np.float64)
        return (-(R.T @ self.t.astype(np.float64))).astype(np.float32)

    @property
    def tiles_x(self) -> int:
        return (self.W + TILE - 1) // TILE

    @property
    def tiles_y(self) -> int:
        return (self.H + TILE - 1) // TILE

    @property
    def n_tiles(self) -> int:
        return self.tiles_x * self.tiles_y


def look_at_camera(W: int, H: int, centre, target=(0.0, 0.0, 0.0),
                   fov_x_deg: float = 60.0, znear: float = 0.2) -> Camera:
    """Camera at `centre` looking at `target`; 'down' in the image is world +y."""
    c = np.asarray(centre, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ c)).astype(np.float32)
    focal = (W / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(W=W, H=H, fx=float(np.float32(focal)), fy=float(np.float32(focal)),
                  cx=W / 2.0, cy=H / 2.0, R=R, t=t, znear=znear)


def front_camera(W: int, H: int) -> Camera:
    """The single-view camera: centre (0, 0, -3), looking along +z, R = I."""
    return look_at_camera(W, H, (0.0, 0.0, -3.0))


def ring_cameras(n_views: int, sizes, radius: float = 3.0, seed: int = 3):
    """`n_views` cameras on a circle of `radius` in the xz-plane, looking at
    the origin, with the (W, H) sizes given; the ring is rotated by a seeded
    random phase."""
    rng = np.random.Generator(np.random.PCG64(seed))
    phase = rng.uniform(0.0, 2.0 * math.pi)
    cams = []
    for k in range(n_views):
        a = phase + 2.0 * math.pi * k / n_views
        W, H = sizes[k]
        cams.append(look_at_camera(W, H, (radius * math.sin(a), 0.0, -radius * math.cos(a))))
    return cams


def uneven_sizes(n_views: int, lo=(800, 600), hi=(1920, 1080)):
    """(W, H) per view, linearly spaced from `lo` to `hi` and rounded."""
    out = []
    for k in range(n_views):
        s = k / max(1, n_views - 1)
        out.append((int(round(lo[0] + s * (hi[0] - lo[0]))),
                    int(round(lo[1] + s * (hi[1] - lo[1])))))
    return out


@dataclass
class Scene:
    """Per-Gaussian parameters, float32, C-contiguous."""
    means: np.ndarray          # (N, 3)
    log_scales: np.ndarray     # (N, 3)
    quats: np.ndarray          # (N, 4)  (w, x, y, z), unit length as drawn
    opacity_logits: np.ndarray # (N,)
    sh: np.ndarray             # (N, 16, 3), coefficient-major, RGB innermost
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.means.shape[0]

    def flat(self) -> np.ndarray:
        """The grouped parameter buffer [means | log_scales | quats | logits | sh]
        (59 N floats) that the Adam step updates in one pass."""
        return np.concatenate([self.means.ravel(), self.log_scales.ravel(),
                               self.quats.ravel(), self.opacity_logits.ravel(),
                               self.sh.ravel()]).astype(np.float32)

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), dict(self.meta))


def _attributes(rng, n):
    log_scales = rng.normal(-4.0, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.0, 1.0, size=(n,))
    sh = rng.normal(0.0, 0.2, size=(n, SH_COEFFS, 3))
    return log_scales, q, logits, sh


def uniform_scene(n: int, seed: int = 0) -> Scene:
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    ls, q, lg, sh = _attributes(rng, n)
    return _pack(means, ls, q, lg, sh, dict(kind="uniform", n=n, seed=seed))


def skewed_scene(n: int, seed: int = 0, n_clusters: int = 20, cluster_frac: float = 0.8,
                 cluster_sigma: float = 0.02, centre_seed: int = 2) -> Scene:
    crng = np.random.Generator(np.random.PCG64(centre_seed))
    centres = crng.uniform(-1.0, 1.0, size=(n_clusters, 3))
    rng = np.random.Generator(np.random.PCG64(seed))
    n_cl = int(round(cluster_frac * n))
    which = rng.integers(0, n_clusters, size=n_cl)
    clustered = centres[which] + rng.normal(0.0, cluster_sigma, size=(n_cl, 3))
    uniform = rng.uniform(-1.0, 1.0, size=(n - n_cl, 3))
    means = np.concatenate([clustered, uniform])
    perm = rng.permutation(n)
    means = means[perm]
    ls, q, lg, sh = _attributes(rng, n)
    return _pack(means, ls, q, lg, sh,
                 dict(kind="skewed", n=n, seed=seed, n_clusters=n_clusters,
                      cluster_frac=cluster_frac, cluster_sigma=cluster_sigma))


def _pack(means, ls, q, lg, sh, meta) -> Scene:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f(means), f(ls), f(q), f(lg), f(sh), meta)


def random_image(W: int, H: int, seed: int = 1) -> np.ndarray:
    """A seeded [3, H, W] float32 image in [0, 1) (a stand-in L1 target)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random(size=(3, H, W), dtype=np.float32)


def random_cotangent(shape, seed: int = 7) -> np.ndarray:
    """A seeded float32 upstream gradient of the given shape."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, 1.0, size=shape).astype(np.float32)


def density_draws(n: int, seed: int = 11):
    """Seeded random draws of one density-control round: per point three
    standard normals z and three uniforms u in [0, 1) (float32, [n, 3] each)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.normal(0.0, 1.0, size=(n, 3)).astype(np.float32)
    u = rng.random(size=(n, 3), dtype=np.float32)
    return z, u


# ---------------------------------------------------------------------------
# Named workloads (sizes and structure only).
# ---------------------------------------------------------------------------

WORKLOADS = {
    # plain FP32 single view, L1 against a second seeded scene
    "uniform-10k-256x256": dict(n=10_000, kind="uniform", views=[(256, 256)]),
    # skewed-density training step with Adam
    "skewed-500k-1280x720": dict(n=500_000, kind="skewed", views=[(1280, 720)]),
    # the throughput workload: 3M skewed Gaussians, one 1600x1060 view
    "skewed-3M-1600x1060": dict(n=3_000_000, kind="skewed", views=[(1600, 1060)]),
    # scheduler workload: 1.5M skewed, 16 views from 800x600 to 1920x1080
    "skewed-1.5M-16views": dict(n=1_500_000, kind="skewed", views=uneven_sizes(16), ring=True),
    # dynamic training: 6M skewed, 4 views at 1920x1080, a clone-and-prune
    # after every step (2% clones, opacity < 0.005 dropped)
    "dynamic-6M-4x1920x1080": dict(n=6_000_000, kind="skewed", views=[(1920, 1080)] * 4, ring=True,
                                   dynamic=dict(clone_frac=0.02, min_opacity=0.005)),
}


def make_workload(name: str, seed: int = 0):
    """Return (scene, [cameras]) for a named workload."""
    w = WORKLOADS[name]
    scene = (uniform_scene if w["kind"] == "uniform" else skewed_scene)(w["n"], seed)
    if w.get("ring"):
        cams = ring_cameras(len(w["views"]), w["views"])
    else:
        cams = [front_camera(W, H) for (W, H) in w["views"]]
    return scene, cams
