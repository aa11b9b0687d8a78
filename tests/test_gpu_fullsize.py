"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

1M surface-clustered convexes (K=6, SH degree 3) at 1920x1080, and 100k at 1237x822: bit-exact
discrete decisions and tile-pair order for every convex; images at sampled pixels the oracle can
compute one by one (binary64 brute force over all convexes); gradients of a loss restricted to
sampled pixels.
"""
import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _parity as P
from tests.test_gpu_backward import FIELDS, compare
from tests._parity import oracle_settings
from tests.test_gpu_forward import check_discrete, check_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["surface100k_1237x822", "surface1M_1920x1080"])
def workload(request):
    sc, cams = syn.workload(request.param, seed=0)
    img, tf, state, t = P.gpu_render(sc, cams[:1])
    yield request.param, sc, cams[0], img, tf, state, t
    state.release()


def test_fullsize_discrete_and_pair_order(workload):
    name, sc, cam, img, tf, state, _ = workload
    disc = check_discrete(state, sc, cam)
    assert disc["visible"].mean() > 0.5
    check_pairs(state, [disc], [cam])


def test_fullsize_sampled_pixels(workload):
    name, sc, cam, img, tf, state, _ = workload
    rng = np.random.default_rng(1)
    pix = np.stack([rng.integers(0, cam.width, 192), rng.integers(0, cam.height, 192)], 1).astype(np.int32)
    ref, ill = P.oracle_pixels_reference(sc, cam, pix)
    got = img[0][:, pix[:, 1], pix[:, 0]].T
    d = np.abs(got - ref["rgb"]).max(1)
    assert ill.mean() <= 0.05
    assert d[~ill].max() <= P.IMAGE_TOL, (d[~ill].max(), np.argmax(np.where(ill, 0, d)))
    assert np.abs(tf[0][pix[:, 1], pix[:, 0]] - ref["t_final"])[~ill].max() <= P.IMAGE_TOL


def test_fullsize_sampled_pixel_gradient(workload):
    import torch
    import paper_2411_14974_gb300 as cs
    name, sc, cam, img, tf, state, t = workload
    rng = np.random.default_rng(2)
    pix = np.stack([rng.integers(0, cam.width, 48), rng.integers(0, cam.height, 48)], 1).astype(np.int32)
    pix = np.unique(pix, axis=0)
    w = rng.uniform(-1, 1, (len(pix), 3))
    G = np.zeros((1, 3, cam.height, cam.width), np.float32)
    G[0, :, pix[:, 1], pix[:, 0]] = w.astype(np.float32)
    g = cs.backward(state, torch.as_tensor(G, device="cuda:0"))
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    st = oracle_settings()
    ref = oracle.backward_pixels(sc, cam, st, pix, w.astype(np.float32).astype(np.float64))
    refp = [oracle.backward_pixels(sc, cam, st, pix, w.astype(np.float32).astype(np.float64), perturb_seed=s)
            for s in (1, 2)]
    compare(got, ref, refp)
