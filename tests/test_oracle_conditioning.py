"""Pin of the conditioning model that decides which pixels and gradient elements the GPU parity
tests compare.

The parity references build the hull lines in binary64 from the binary32 projected points
(q_binary32).  A binary32 renderer evaluates those lines in binary32 instead: the record form of
the discrete specification (lines scaled by log2(e) d^p delta and anchored at the first hull
vertex, Eq. 1 with Eq. S1/S2), re-based to the origin of the pixel's 8 x 4 block and evaluated
with fused multiply-adds.  The oracle's line_f32 mode evaluates every line value exactly that way
and keeps the rest binary64, so the difference between the two oracle modes is the effect of the
binary32 line evaluation alone.  These tests check, on the scenes the GPU parity tests use, that

  * images: wherever no cut-off decision lies within its band (Eq. 5 with the 3DGS cut-offs), the
    change of every channel stays within the oracle's first-order bound ``sens`` (built from the
    line_rel error model), and the decisions themselves (contributing pairs, last contributor)
    do not change;
  * gradients: on the elements that the two-sign line-error probe does not exclude, the gradient
    moves by at most a tenth of the parity tolerance, and the probe excludes at most 1% of the
    elements.

Both sides are binary32-vs-binary64 statements about the oracle alone; nothing here runs on a GPU.
"""
import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _parity as P

FIELDS = ("points", "delta", "sigma", "opacity", "sh")


def _image_cases():
    cases = []
    for seed in (0, 1):
        sc, cams = syn.workload("blob1k_128", seed=seed)
        cases.append((f"blob1k_128 seed {seed}", sc, cams[0]))
    sc = syn.surface_scene(11, n=10_000, sh_degree=3)
    cases.append(("surface 10k", sc, syn.sphere_cameras(1, 160, 120, 4.0, seed=12)[0]))
    return cases


@pytest.mark.parametrize("case", range(3))
def test_line_model_bounds_the_binary32_record_lines_in_the_image(case):
    name, sc, cam = _image_cases()[case]
    ref = oracle.render_image(sc, cam, P.oracle_settings())
    f32 = oracle.render_image(sc, cam, P.oracle_settings(line_f32=True))
    calm = (ref["flags"] & 3) == 0
    d = np.abs(f32["image"] - ref["image"]).max(0)
    assert d.max() > 0, "the binary32 line evaluation should change some pixel"
    over = d[calm] > ref["sens"][calm]
    assert not over.any(), (name, int(over.sum()), float((d[calm] / ref["sens"][calm]).max()))
    # the decisions (which pairs contribute, where the walk stops) are the same where no cut-off
    # lies within its band
    assert (f32["n_contrib"] == ref["n_contrib"])[calm].all(), name
    assert (f32["last_id"] == ref["last_id"])[calm].all(), name
    # the mask the parity tests apply stays small
    ill = (ref["sens"] > P.COND_TOL) | ~calm
    assert ill.mean() <= 0.04, (name, ill.mean())


def test_line_model_is_what_covers_the_binary32_lines():
    """With the line term of the model switched off (only the fixed allowances for the
    transcendentals left), the binary32 record lines break the bound: the line term carries it."""
    sc, cams = syn.workload("blob1k_128", seed=0)
    cam = cams[0]
    f32 = oracle.render_image(sc, cam, P.oracle_settings(line_f32=True))
    tiny = oracle.render_image(sc, cam, oracle.settings(q_binary32=True, line_rel=2.0 ** -40))
    calm = (tiny["flags"] & 3) == 0
    d = np.abs(f32["image"] - tiny["image"]).max(0)
    assert (d[calm] > tiny["sens"][calm]).any()


def _blob(seed, n=300, deg=0, radius=0.08):
    sc = syn.blob_scene(seed, n=n, radius=radius, sh_degree=deg)
    sc.points[..., :2] *= 0.5
    return sc


def _gradient_cases():
    return [("blob seed 0", _blob(0), syn.blob_camera(64, 64)),
            ("blob seed 1, SH 3", _blob(1, deg=3), syn.blob_camera(64, 64)),
            ("blob seed 2, SH 2", _blob(2, deg=2), syn.blob_camera(48, 40)),
            ("surface 5k, SH 3", syn.surface_scene(21, n=5_000, sh_degree=3),
             syn.sphere_cameras(1, 120, 96, 4.0, seed=22)[0])]


@pytest.mark.parametrize("case", range(4))
def test_gradient_probe_bounds_the_binary32_record_lines(case):
    name, sc, cam = _gradient_cases()[case]
    G = np.random.default_rng(case).uniform(-1, 1, (3, cam.height, cam.width))
    st = P.oracle_settings()
    ref = oracle.backward_image(sc, cam, st, G)
    probes = [oracle.backward_image(sc, cam, st, G, perturb_seed=s) for s in (1, 2)]
    f32 = oracle.backward_image(sc, cam, P.oracle_settings(line_f32=True), G)
    for f in FIELDS:
        b = ref[f].ravel()
        scale = np.abs(b).max()
        tol = P.GRAD_REL * np.abs(b) + P.GRAD_FLOOR * scale
        ill = P.gradient_ill(b, [p[f].ravel() for p in probes], tol)
        nz = np.abs(b) > P.GRAD_FLOOR * scale
        d = np.abs(f32[f].ravel() - b)
        assert (d[~ill] <= 0.1 * tol[~ill]).all(), (name, f, float((d / tol)[~ill].max()))
        assert ill[nz].mean() <= P.GRAD_MAX_EXCLUDED, (name, f, float(ill[nz].mean()))
