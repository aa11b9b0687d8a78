"""Pin of the oracle's binary32-vertex mode (q_binary32) to its binary64-projection mode.

The GPU parity tests compare against the mode that builds the hull lines from the binary32
projected points on which the hull is decided.  That mode differs from the finite-difference-
pinned binary64 mode only by the binary32 rounding of the projected points, so wherever the
binary64 mode is insensitive to moving the points by 4 binary32 ulps, the two modes must agree
to within the same small amount, for images and for gradients.
"""
import numpy as np

import oracle
from paper_2411_14974_gb300 import synthetic as syn


def _sens_image(sc, cam, st):
    r0 = oracle.render_image(sc, cam, st)
    d = np.zeros(r0["image"].shape[1:])
    for seed in (1, 2):
        d = np.maximum(d, np.abs(oracle.render_image(sc, cam, st, perturb_seed=seed)["image"] - r0["image"]).max(0))
    return r0, d


def test_binary32_vertices_image_within_envelope():
    """Outside pixels whose first-order sensitivity bound to 4-ulp vertex motion exceeds 2.5e-5
    (or whose cut-off decisions are within their bands), the two modes agree to 2.5e-5."""
    for seed in (0, 1):
        sc, cams = syn.workload("blob1k_128", seed=seed)
        cam = cams[0]
        r64 = oracle.render_image(sc, cam, oracle.settings(perturb_ulps=4.0))
        r32 = oracle.render_image(sc, cam, oracle.settings(q_binary32=True))
        calm = (r64["sens"] <= 2.5e-5) & ((r64["flags"] & 3) == 0)
        assert calm.mean() > 0.2  # the worst-case vertex-motion bound is conservative
        assert np.abs(r32["image"] - r64["image"]).max(0)[calm].max() <= 2.5e-5
        assert np.abs(r32["image"] - r64["image"]).max() > 0  # the modes do differ somewhere


def test_binary32_vertices_gradient_within_envelope():
    sc = syn.blob_scene(2, n=200, radius=0.08, sh_degree=2)
    sc.points[..., :2] *= 0.5
    cam = syn.blob_camera(48, 48)
    G = np.random.default_rng(1).uniform(-1, 1, (3, 48, 48))
    st64 = oracle.settings()
    g64 = oracle.backward_image(sc, cam, st64, G)
    gp = [oracle.backward_image(sc, cam, st64, G, perturb_seed=s) for s in (1, 2)]
    g32 = oracle.backward_image(sc, cam, oracle.settings(q_binary32=True), G)
    for f in ("points", "delta", "sigma", "opacity", "sh"):
        b = g64[f].ravel()
        scale = np.abs(b).max()
        sens = np.max([np.abs(p[f].ravel() - b) for p in gp], 0)
        tol = 1e-3 * np.abs(b) + 1e-4 * scale
        calm = sens <= 0.25 * tol
        assert np.abs(g32[f].ravel() - b)[calm].max() <= tol[calm].max(), f
        assert (np.abs(g32[f].ravel() - b) <= tol)[calm].all(), f
