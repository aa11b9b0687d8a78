"""Pins for the oracle's smooth indicator (Eq. 2/3, in 2D as Eq. S1/S2 with the d-scaling).

References: the closed form of the indicator of an axis-aligned square, the LogSumExp bounds,
the hard-polygon limit as delta, sigma grow (Sec. 3.1), and the invariance of the image under
scaling the scene about the camera centre when delta and sigma are divided by d^p.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _cases as C

EXACT = dict(tau=0.0, alpha_max=1.0, t_min=0.0)


def test_square_worked_example_golden():
    """Fixture: the square of half-width 8 px at distance 4 (K=4), delta'=2, sigma'=0.5."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "square_indicator.json")) as f:
        g = json.load(f)
    sc = C.square_scene(a_px=g["a_px"], z=g["z"], f=g["f"], delta=g["delta"], sigma=g["sigma"])
    cam = C.axis_camera(f=g["f"])
    r = oracle.render_pixels(sc, cam, oracle.settings(**EXACT), np.array([g["pixel"]], np.int32))
    assert abs(r["rgb"][0, 0] / 0.5 - g["I_centre"]) < 1e-12
    # the closed form written out here: phi(q0) = -dp*a + ln 4, I = 1/(1+exp(sp*phi))
    dp, sp, a = g["z"] * g["delta"], g["z"] * g["sigma"], g["a_px"]
    phi = -dp * a + math.log(4.0)
    assert abs(phi - g["phi_centre"]) < 1e-12
    assert abs(1.0 / (1.0 + math.exp(sp * phi)) - g["I_centre"]) < 1e-12


@pytest.mark.parametrize("a,delta,sigma", [(8.0, 0.5, 0.125), (8.0, 0.05, 0.5), (4.0, 2.0, 0.02), (16.0, 0.1, 1.0)])
def test_square_matches_closed_form_everywhere(a, delta, sigma):
    f, z = 128.0, 4.0
    sc = C.square_scene(a_px=a, z=z, f=f, delta=delta, sigma=sigma)
    cam = C.axis_camera(f=f)
    img = oracle.render_image(sc, cam, oracle.settings(**EXACT))["image"] / 0.5
    d32, s32 = float(np.float32(delta)), float(np.float32(sigma))  # the parameters are binary32
    I, phi = C.square_indicator_closed_form(128, 128, 63.5, a, z * d32, z * s32)
    assert np.abs(img[0] - I).max() < 1e-12
    # I = 1/2 exactly where phi = 0 (boundary of the smooth convex): the sigmoid's fixed point
    near = np.abs(phi) < 1e-2
    if near.any():
        assert np.allclose(img[0][near], 1.0 / (1.0 + np.exp(z * s32 * phi[near])), atol=1e-14)


def test_indicator_range_and_lse_bounds():
    """0 < I < 1, and d delta max_t L_t <= phi <= d delta max_t L_t + ln T (LogSumExp bounds)."""
    sc, cams = syn.workload("blob1k_128", seed=3)
    cam = cams[0]
    disc = oracle.discrete(sc, cam)
    rng = np.random.default_rng(0)
    ids = rng.choice(np.nonzero(disc["visible"])[0], 12, replace=False)
    for i in ids:
        one = sc.subset([i])
        one.opacity[:] = 1.0
        one.sh = C.grey_sh(1)
        img = oracle.render_image(one, cam, oracle.settings(**EXACT))["image"][0] / 0.5
        assert (img >= 0).all() and (img <= 1).all()
        # lines from an independent binary64 projection of the oracle's hull vertices
        q, xc = C.project64(one.points[0], cam)
        T = disc["hull_t"][i]
        hv = q[disc["hull_idx"][i][:T]]
        ys, xs = np.meshgrid(np.arange(128) + 0.5, np.arange(128) + 0.5, indexing="ij")
        L = []
        for t in range(T):
            v, w = hv[t], hv[(t + 1) % T]
            e = w - v
            n = np.array([e[1], -e[0]]) / np.hypot(*e)
            L.append(n[0] * (xs - v[0]) + n[1] * (ys - v[1]))
        L = np.stack(L)
        d = C.camera_distance(one, cam)[0]
        dp, sp = d * float(one.delta[0]), d * float(one.sigma[0])
        ok = (img > 1e-9) & (img < 1 - 1e-9)
        phi = np.log(1.0 / img[ok] - 1.0) / sp
        lo = dp * L.max(0)[ok]
        tol = 1e-6 * (1 + np.abs(lo))
        assert (phi >= lo - tol).all()
        assert (phi <= lo + math.log(T) + tol).all()


def test_hard_polygon_limit():
    """As delta, sigma grow the indicator tends to the hard mask of the square away from its edge."""
    f, z, a = 128.0, 4.0, 8.0
    cam = C.axis_camera(f=f)
    ys, xs = np.meshgrid(np.arange(128) + 0.5, np.arange(128) + 0.5, indexing="ij")
    dist_out = np.maximum(np.abs(xs - 63.5), np.abs(ys - 63.5)) - a  # Chebyshev distance to the square edge
    mask = (dist_out < 0).astype(np.float64)
    far = np.abs(dist_out) >= 1.0
    errs = []
    for s in (1.0, 10.0, 100.0, 1000.0):
        sc = C.square_scene(a_px=a, z=z, f=f, delta=0.5 * s, sigma=0.05 * s)
        img = oracle.render_image(sc, cam, oracle.settings(**EXACT))["image"][0] / 0.5
        errs.append(np.abs(img - mask)[far].max())
    assert errs[0] > errs[1] > errs[2] >= errs[3]
    assert errs[-1] < 1e-12


@pytest.mark.parametrize("power,mode", [(1.0, 0), (2.0, 0), (0.5, 0), (1.0, 1)])
def test_scale_about_camera_centre_invariance(power, mode):
    """Projection is invariant under scaling the scene by s about the camera centre while d scales
    by s; dividing delta and sigma by s^p must therefore leave the image unchanged."""
    sc, _ = syn.workload("blob1k_128", seed=4)
    cam = C.axis_camera()
    cam.R = syn.blob_camera().R
    sc.points[..., 2] += 4.0  # move the blob in front of a camera at the origin (t = 0)
    s = 4.0  # a power of two: every binary32 coordinate, distance and hull decision scales exactly
    big = sc.copy()
    big.points *= s
    big.delta /= np.float32(s ** power)
    big.sigma /= np.float32(s ** power)
    st = oracle.settings(dist_power=power, dist_mode=mode)
    a = oracle.render_image(sc, cam, st)["image"]
    b = oracle.render_image(big, cam, st)["image"]
    assert a.max() > 0.1
    assert np.abs(a - b).max() < 1e-12
