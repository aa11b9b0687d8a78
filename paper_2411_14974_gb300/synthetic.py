"""Seeded synthetic inputs for the convex rasterizer: scenes of smooth convexes and pinhole cameras.

This module only draws inputs.  It holds none of the renderer's arithmetic (no projection, hull,
indicator or compositing), so both the CUDA path and the CPU oracle can consume the same arrays.

Scene layout (all float32, C-contiguous):
  points  [N][K][3]   the K free 3D points of each convex (Sec. 3.2, "point-based representation")
  delta   [N]         smoothness delta > 0 (Eq. 2), activated unless raw (then log delta)
  sigma   [N]         sharpness sigma > 0 (Eq. 3), activated unless raw (then log sigma)
  opacity [N]         o in (0, 1) (Eq. 5), activated unless raw (then logit o)
  sh      [N][(D+1)^2][3]  spherical-harmonic colour coefficients (Sec. 3.2, colour c_n)

Camera: world-to-camera rotation R (row-major 3x3) and translation t with OpenCV axes
(x right, y down, z forward), intrinsics fx, fy, cx, cy in pixels, image width x height.

The recipes follow the synthetic workloads that stand in for the paper's datasets (Mip-NeRF360,
Tanks&Temples, Deep Blending are not available): uniform blobs (1k convexes, 128x128), surface-
clustered scenes (100k..3M convexes, SH degree 3) and heavily clustered stress scenes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Y_00 of the real spherical-harmonic basis, 1/(2 sqrt(pi)); used only to draw degree-0
# coefficients whose colour is uniform in [0, 1].
_Y00 = 0.28209479177387814


@dataclasses.dataclass
class Scene:
    points: np.ndarray
    delta: np.ndarray
    sigma: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    sh_degree: int
    raw: bool = False  # True: delta, sigma hold log values and opacity its logit (training parameters)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def k(self) -> int:
        return int(self.points.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.points[idx]), np.ascontiguousarray(self.delta[idx]),
                     np.ascontiguousarray(self.sigma[idx]), np.ascontiguousarray(self.opacity[idx]),
                     np.ascontiguousarray(self.sh[idx]), self.sh_degree, self.raw)

    def copy(self) -> "Scene":
        return Scene(self.points.copy(), self.delta.copy(), self.sigma.copy(), self.opacity.copy(),
                     self.sh.copy(), self.sh_degree, self.raw)

    def as_raw(self) -> "Scene":
        """The same draw expressed as training parameters: log delta, log sigma, logit opacity
        (rounded to float32; activating them gives back the drawn values to about an ulp)."""
        assert not self.raw
        o = self.opacity.astype(np.float64)
        f = lambda a: np.ascontiguousarray(a, np.float32)
        return Scene(self.points.copy(), f(np.log(self.delta.astype(np.float64))),
                     f(np.log(self.sigma.astype(np.float64))), f(np.log(o) - np.log1p(-o)), self.sh.copy(),
                     self.sh_degree, True)


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # [3,3] float32, world -> camera
    t: np.ndarray  # [3] float32
    z_near: float = 0.2


def _unit_vectors(rng: np.random.Generator, shape) -> np.ndarray:
    v = rng.standard_normal(tuple(shape) + (3,))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    return v


def look_at(eye, target=(0.0, 0.0, 0.0), down=(0.0, 0.0, -1.0)):
    """World->camera (R, t) for a camera at ``eye`` looking at ``target`` (OpenCV axes).

    ``down`` is the world direction that should point down the image (camera +y)."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    down = np.asarray(down, np.float64)
    if abs(float(np.dot(down, z))) > 0.999:
        down = np.array([0.0, 0.0, 1.0]) if abs(z[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    t = -R @ eye
    return R.astype(np.float32), t.astype(np.float32)


def pinhole(width: int, height: int, fov_x_deg: float, R, t, z_near: float = 0.2) -> Camera:
    """Camera with horizontal field of view ``fov_x_deg``, square pixels, principal point at the centre."""
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(int(width), int(height), float(np.float32(fx)), float(np.float32(fx)),
                  float(width) / 2.0, float(height) / 2.0,
                  np.asarray(R, np.float32).reshape(3, 3).copy(), np.asarray(t, np.float32).reshape(3).copy(),
                  float(z_near))


def _params(rng: np.random.Generator, n: int):
    delta = np.exp(rng.uniform(math.log(0.5), math.log(50.0), n))
    sigma = np.exp(rng.uniform(math.log(0.01), math.log(10.0), n))
    opacity = rng.uniform(0.1, 0.9, n)
    return delta.astype(np.float32), sigma.astype(np.float32), opacity.astype(np.float32)


def blob_scene(seed: int = 0, n: int = 1000, k: int = 6, radius: float = 0.05, sh_degree: int = 0) -> Scene:
    """Oracle-size scene: centres uniform in [-1,1]^3, points = centre + radius * unit vectors.

    delta log-uniform in [0.5, 50], sigma log-uniform in [0.01, 10], opacity uniform in [0.1, 0.9];
    degree-0 colour drawn uniform in [0, 1] per channel.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-1.0, 1.0, (n, 3))
    pts = centres[:, None, :] + radius * _unit_vectors(rng, (n, k))
    delta, sigma, opacity = _params(rng, n)
    nb = (sh_degree + 1) ** 2
    sh = np.zeros((n, nb, 3), np.float64)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (rgb - 0.5) / _Y00
    if nb > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.3, (n, nb - 1, 3))
    return Scene(pts.astype(np.float32), delta, sigma, opacity, sh.astype(np.float32), sh_degree)


def _surface_samples(rng: np.random.Generator, n: int, n_surfaces: int = 8) -> np.ndarray:
    """Samples from 4 random planes (square patches) and 4 random spheres inside [-1,1]^3."""
    which = rng.integers(0, n_surfaces, n)
    out = np.empty((n, 3))
    for s in range(n_surfaces):
        m = which == s
        cnt = int(m.sum())
        srng = np.random.default_rng(rng.integers(1 << 62))
        if s % 2 == 0:  # plane patch
            c = srng.uniform(-0.6, 0.6, 3)
            u = _unit_vectors(srng, (1,))[0]
            w = np.cross(u, _unit_vectors(srng, (1,))[0])
            w /= np.linalg.norm(w)
            half = srng.uniform(0.3, 0.6)
            a = rng.uniform(-half, half, (cnt, 1))
            b = rng.uniform(-half, half, (cnt, 1))
            out[m] = c + a * u + b * w
        else:  # sphere
            c = srng.uniform(-0.5, 0.5, 3)
            r = srng.uniform(0.15, 0.4)
            out[m] = c + r * _unit_vectors(rng, (cnt,))
    return out


def surface_scene(seed: int = 0, n: int = 100_000, k: int = 6, sh_degree: int = 3,
                  clustered_fraction: float = 0.0) -> Scene:
    """Surface-clustered scene: centres on 8 noisy planes/spheres (noise sigma 0.01), log-normal
    per-convex scale (mu = ln 0.01, s = 0.5), SH coefficients N(0, 0.3).

    ``clustered_fraction`` > 0 moves that fraction of centres into a cube of 5% of the [-1,1]^3
    volume (side 2 * 0.05^(1/3)) to make the per-tile load very uneven.
    """
    rng = np.random.default_rng(seed)
    centres = _surface_samples(rng, n) + rng.normal(0.0, 0.01, (n, 3))
    if clustered_fraction > 0:
        m = rng.uniform(0, 1, n) < clustered_fraction
        half = 0.05 ** (1.0 / 3.0)
        centres[m] = rng.uniform(-half, half, (int(m.sum()), 3))
        centres[~m] = rng.uniform(-1.0, 1.0, (int((~m).sum()), 3))
    scale = np.exp(rng.normal(math.log(0.01), 0.5, n))
    pts = centres[:, None, :] + scale[:, None, None] * _unit_vectors(rng, (n, k))
    delta, sigma, opacity = _params(rng, n)
    nb = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, nb, 3))
    return Scene(pts.astype(np.float32), delta, sigma, opacity, sh.astype(np.float32), sh_degree)


def sphere_cameras(n: int, width: int, height: int, radius=4.0, fov_x_deg: float = 50.0,
                   seed: int = 0, hemisphere: bool = False, fibonacci: bool = False):
    """``n`` cameras on a sphere (or the upper hemisphere) of ``radius`` looking at the origin.

    ``radius`` may be a float or a (lo, hi) range drawn uniformly per camera.
    """
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n):
        if fibonacci:
            golden = math.pi * (3.0 - math.sqrt(5.0))
            zf = 1.0 - (i + 0.5) / n if hemisphere else 1.0 - 2.0 * (i + 0.5) / n
            rr = math.sqrt(max(0.0, 1.0 - zf * zf))
            d = np.array([rr * math.cos(golden * i), rr * math.sin(golden * i), zf])
        else:
            d = _unit_vectors(rng, (1,))[0]
            if hemisphere:
                d[2] = abs(d[2])
        rad = float(rng.uniform(radius[0], radius[1])) if isinstance(radius, (tuple, list)) else float(radius)
        # world +z appears up in the image
        R, t = look_at(rad * d, down=(0.0, 0.0, -1.0))
        cams.append(pinhole(width, height, fov_x_deg, R, t))
    return cams


def blob_camera(width: int = 128, height: int = 128, fov_x_deg: float = 50.0) -> Camera:
    """R = I, t = (0, 0, 4): the camera sits at (0, 0, -4) looking down +z at the origin."""
    return pinhole(width, height, fov_x_deg, np.eye(3, dtype=np.float32), np.array([0.0, 0.0, 4.0], np.float32))


def random_target(seed: int, width: int, height: int, n_views: int = 1) -> np.ndarray:
    """Fixed random target image(s) [V][3][H][W], uniform in [0, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (n_views, 3, height, width)).astype(np.float32)


# Workload recipes (sizes, resolutions) used by the tests and the benchmark.
def workload(name: str, seed: int = 0):
    """Return (scene, cameras) for a named workload."""
    if name == "blob1k_128":
        return blob_scene(seed), [blob_camera()]
    if name == "surface100k_1237x822":
        return surface_scene(seed, 100_000), sphere_cameras(1, 1237, 822, 4.0, seed=seed + 1)
    if name == "surface1M_1920x1080":
        return surface_scene(seed, 1_000_000), sphere_cameras(1, 1920, 1080, 4.0, seed=seed + 1)
    if name == "surface1M_1600x1060":
        return surface_scene(seed, 1_000_000), sphere_cameras(100, 1600, 1060, 4.0, seed=seed + 1,
                                                              hemisphere=True, fibonacci=True)
    if name == "clustered3M_3840x2160x16":
        return (surface_scene(seed, 3_000_000, clustered_fraction=0.9),
                sphere_cameras(16, 3840, 2160, 4.0, seed=seed + 1))
    raise KeyError(name)
