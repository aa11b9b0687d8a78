"""Hand-built scenes and cameras for the oracle pins and the GPU parity tests."""
import math

import numpy as np

from paper_2411_14974_gb300 import synthetic as syn

Y00 = 0.5 / math.sqrt(math.pi)


def grey_sh(n, deg=0):
    """All coefficients zero: the colour is exactly 0.5 in every channel and every direction."""
    return np.zeros((n, (deg + 1) ** 2, 3), np.float32)


def rgb_sh(rgb):
    rgb = np.asarray(rgb, np.float64).reshape(-1, 3)
    sh = np.zeros((rgb.shape[0], 1, 3), np.float32)
    sh[:, 0, :] = (rgb - 0.5) / Y00
    return sh


def axis_camera(width=128, height=128, f=128.0, c=63.5):
    """Camera at the world origin looking down +z; the principal point sits on a pixel centre."""
    return syn.Camera(width, height, float(f), float(f), float(c), float(c),
                      np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 0.2)


def square_scene(a_px=8.0, z=4.0, f=128.0, delta=0.5, sigma=0.125, opacity=1.0, rgb=(0.5, 0.5, 0.5)):
    """One convex of K=4 points whose projection is the axis-aligned square of half-width a_px
    centred on the principal point.  With f=128, z=4, a=8 every coordinate is exact in binary32.
    The default colour 0.5 (all SH coefficients zero) is exact as well."""
    h = a_px * z / f
    pts = np.array([[[-h, -h, z], [h, -h, z], [h, h, z], [-h, h, z]]], np.float32)
    return syn.Scene(pts, np.array([delta], np.float32), np.array([sigma], np.float32),
                     np.array([opacity], np.float32), rgb_sh([rgb]), 0)


def square_indicator_closed_form(width, height, c, a, dp, sp):
    """I(q) = 1/(1+exp(sp * log sum_t exp(dp L_t(q)))) for the square [c-a, c+a]^2 (Eq. 2/3 in 2D)."""
    ys, xs = np.meshgrid(np.arange(height) + 0.5, np.arange(width) + 0.5, indexing="ij")
    L = np.stack([xs - (c + a), (c - a) - xs, ys - (c + a), (c - a) - ys], 0)
    m = (dp * L).max(0)
    phi = m + np.log(np.exp(dp * L - m).sum(0))
    return 1.0 / (1.0 + np.exp(sp * phi)), phi


def camera_distance(scene, cam):
    """Distance from the camera centre to each convex's mean point, in binary64."""
    c = scene.points.astype(np.float64).mean(1)
    cc = c @ cam.R.astype(np.float64).T + cam.t.astype(np.float64)
    return np.linalg.norm(cc, axis=1)


def project64(points, cam):
    xc = points.astype(np.float64) @ cam.R.astype(np.float64).T + cam.t.astype(np.float64)
    u = cam.fx * xc[..., 0] / xc[..., 2] + cam.cx
    v = cam.fy * xc[..., 1] / xc[..., 2] + cam.cy
    return np.stack([u, v], -1), xc
