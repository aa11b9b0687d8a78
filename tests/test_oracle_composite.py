"""Pins for the oracle's front-to-back compositing (Eq. 5) and the depth order (Sec. 3.2).

References: Eq. 5 written out in numpy from single-convex renders and an independently computed
depth order, the energy identity C = c (1 - T) for a constant colour c, monotone transmittance,
invariance under relabelling, and invariance under adding an interior point (Sec. 3.2: the K
points need not be vertices).
"""
import numpy as np

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _cases as C

EXACT = dict(tau=0.0, alpha_max=1.0, t_min=0.0)


def _small_overlapping_scene(seed, n=24):
    """n blobs near the optical axis so that most pixels see several overlapping convexes."""
    sc = syn.blob_scene(seed, n=n, radius=0.12)
    sc.points[..., :2] *= 0.25
    rng = np.random.default_rng(seed + 100)
    sc.sh = C.rgb_sh(rng.uniform(0.1, 1.0, (n, 3)))
    return sc


def test_single_convex_closed_form():
    sc = C.square_scene(opacity=0.7, rgb=(0.5, 0.5, 0.5))
    cam = C.axis_camera()
    for amax in (1.0, 0.6):
        img = oracle.render_image(sc, cam, oracle.settings(tau=0.0, alpha_max=amax, t_min=0.0))["image"]
        I, _ = C.square_indicator_closed_form(128, 128, 63.5, 8.0, 2.0, 0.5)
        want = 0.5 * np.minimum(float(np.float32(amax)), float(np.float32(0.7)) * I)  # settings are binary32
        assert np.abs(img - want[None]).max() < 1e-12


def test_eq5_literal_against_single_convex_renders():
    """tau = t_min = 0, alpha_max = 1: C = sum_n c_n a_n prod_{i<n} (1 - a_i) in increasing distance."""
    cam = syn.blob_camera(64, 64)
    for seed in (0, 1):
        sc = _small_overlapping_scene(seed)
        disc = oracle.discrete(sc, cam)
        vis = np.nonzero(disc["visible"])[0]
        assert len(vis) >= 20
        dist = C.camera_distance(sc, cam)
        order = vis[np.argsort(dist[vis], kind="stable")]
        st = oracle.settings(**EXACT)
        alphas = {}
        rgb = {}
        for i in vis:
            one = sc.subset([i])
            g = one.copy()
            g.sh = C.grey_sh(1)
            alphas[i] = oracle.render_image(g, cam, st)["image"][0] / 0.5
            rgb[i] = oracle.render_image(one, cam, st)["image"] / np.maximum(alphas[i][None], 1e-300)
        Cimg = np.zeros((3, 64, 64))
        T = np.ones((64, 64))
        for i in order:
            a = alphas[i]
            col = (0.5 + C.Y00 * sc.sh[i, 0, :].astype(np.float64))[:, None, None]
            Cimg += col * a[None] * T[None]
            T *= 1.0 - a
        full = oracle.render_image(sc, cam, st)
        assert np.abs(full["image"] - Cimg).max() < 1e-12
        assert np.abs(full["t_final"] - T).max() < 1e-12
        # the reverse order is a different image: the test can see a flipped sort
        Crev = np.zeros((3, 64, 64))
        Tr = np.ones((64, 64))
        for i in order[::-1]:
            col = (0.5 + C.Y00 * sc.sh[i, 0, :].astype(np.float64))[:, None, None]
            Crev += col * alphas[i][None] * Tr[None]
            Tr *= 1.0 - alphas[i]
        assert np.abs(full["image"] - Crev).max() > 1e-3


def test_energy_identity_and_background():
    """Constant colour c, background b: C = c (1 - T_final) + b T_final, under the default cut-offs."""
    sc, cams = syn.workload("blob1k_128", seed=5)
    sc.sh = C.grey_sh(sc.n)
    cam = cams[0]
    r = oracle.render_image(sc, cam, oracle.settings())
    assert np.abs(r["image"] - 0.5 * (1.0 - r["t_final"])[None]).max() < 1e-12
    bg = (0.2, 0.3, 0.4)
    rb = oracle.render_image(sc, cam, oracle.settings(bg=bg))
    want = r["image"] + np.asarray(bg, np.float32).astype(np.float64)[:, None, None] * r["t_final"][None]
    assert np.abs(rb["image"] - want).max() < 1e-12


def test_transmittance_monotone_along_depth_order():
    cam = syn.blob_camera(64, 64)
    sc = _small_overlapping_scene(3)
    disc = oracle.discrete(sc, cam)
    vis = np.nonzero(disc["visible"])[0]
    order = vis[np.lexsort((vis, disc["depth_bits"][vis]))]
    prev = np.ones((64, 64))
    for m in range(1, len(order) + 1):
        T = oracle.render_image(sc.subset(np.sort(order[:m])), cam, oracle.settings(**EXACT))["t_final"]
        assert (T <= prev + 1e-15).all() and (T >= 0).all()
        prev = T
    r = oracle.render_image(sc, cam, oracle.settings())
    assert (r["t_final"] <= 1).all()
    # with the default cut-off, a pixel stops right after its transmittance falls below t_min
    assert (r["t_final"] > 0.99 * 1e-4 * 0.01).all()


def test_relabelling_invariance():
    sc, cams = syn.workload("blob1k_128", seed=6)
    cam = cams[0]
    disc = oracle.discrete(sc, cam)
    assert len(np.unique(disc["depth_bits"])) == sc.n  # distinct depths: the order is unique
    perm = np.random.default_rng(0).permutation(sc.n)
    a = oracle.render_image(sc, cam)
    b = oracle.render_image(sc.subset(perm), cam)
    assert np.abs(a["image"] - b["image"]).max() < 1e-13
    assert (perm[b["last_id"][b["last_id"] >= 0]] == a["last_id"][a["last_id"] >= 0]).all()


def test_interior_point_invariance():
    """Adding a K+1-th point at the centroid leaves hull, centre, distance and image unchanged."""
    sc, cams = syn.workload("blob1k_128", seed=7)
    cam = cams[0]
    sc = sc.subset(np.arange(300))
    cen = sc.points.astype(np.float64).mean(1, keepdims=True)
    big = syn.Scene(np.concatenate([sc.points, cen.astype(np.float32)], 1), sc.delta, sc.sigma, sc.opacity,
                    sc.sh, sc.sh_degree)
    a = oracle.render_image(sc, cam)
    b = oracle.render_image(big, cam)
    da, db = oracle.discrete(sc, cam), oracle.discrete(big, cam)
    assert (da["hull_idx"] == db["hull_idx"]).all()
    assert np.abs(a["image"] - b["image"]).max() < 1e-6


def test_golden_blob_samples():
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "blob1k_seed0_samples.json")) as f:
        g = json.load(f)
    sc, cams = syn.workload(g["workload"], seed=g["seed"])
    r = oracle.render_pixels(sc, cams[0], oracle.settings(), np.asarray(g["pixels"], np.int32))
    assert np.abs(r["rgb"] - np.asarray(g["rgb"])).max() < 1e-12
    assert (r["last_id"] == np.asarray(g["last_id"])).all()
