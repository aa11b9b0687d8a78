"""Heavy-tile splitting (cs_settings.tile_split) against the oracle and the unsplit path, through
the C ABI.

A tile with more than N pairs is blended as chunks of N pairs by separate CTAs and merged in depth
order by C = C_a + T_a C_b, T = T_a T_b (3DGS-style binning, Sec. 3.2, with the associative
compositing of Eq. 5); where a pixel's walk stops inside a later chunk, that chunk is walked again
from T_a, so the t_min cut-off is the unsplit walk's.  The oracle has no tiles: the split image and
gradients must match it like the unsplit ones.  Clustered scenes make tiles of thousands of pairs;
the low-opacity variant makes pixels stop only after several chunks (the walk-again path).
"""
import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _parity as P
from tests.test_gpu_backward import compare, gpu_grads
from tests.test_gpu_forward import check_image

pytestmark = pytest.mark.gpu

SPLIT = 256


def _clustered(seed, n, opacity_scale=1.0):
    sc = syn.surface_scene(seed, n=n, sh_degree=1, clustered_fraction=0.9)
    c = sc.points.mean(axis=1, keepdims=True)
    sc.points = (c + 2.0 * (sc.points - c)).astype(np.float32)
    sc.opacity = (sc.opacity * opacity_scale).astype(np.float32)
    return sc


def _heavy_tiles(state, split):
    r = state.array("tile_ranges").reshape(-1, 2).astype(np.int64)
    return int(((r[:, 1] - r[:, 0]) > split).sum()), int((r[:, 1] - r[:, 0]).max())


@pytest.mark.parametrize("opacity_scale", [1.0, 0.15])
def test_split_image_matches_oracle_and_unsplit(opacity_scale):
    sc = _clustered(51, 20_000, opacity_scale)
    cam = syn.sphere_cameras(1, 192, 144, 3.0, seed=52)[0]
    img_s, tf_s, state, _ = P.gpu_render(sc, [cam], tile_split=SPLIT)
    heavy, longest = _heavy_tiles(state, SPLIT)
    state.release()
    assert heavy >= 10 and longest > 4 * SPLIT  # tiles of several chunks
    img_u, tf_u, state, _ = P.gpu_render(sc, [cam])
    state.release()
    ref, ill = P.oracle_reference(sc, cam)
    check_image(img_s[0], ref, ill, max_ill=0.06)
    check_image(img_u[0], ref, ill, max_ill=0.06)
    # split and unsplit differ only by the rounding of the merged transmittance products
    assert np.abs(img_s[0] - img_u[0]).max(0)[~ill].max() <= P.IMAGE_TOL
    assert np.abs(tf_s[0] - tf_u[0])[~ill].max() <= P.IMAGE_TOL
    if opacity_scale < 1.0:
        # faint convexes: many pixels composite more than one chunk's worth of pairs before
        # stopping (or never stop), so merges and walks-again both occur
        assert (tf_s[0] < 1e-3).mean() < 0.9


def test_split_gradient_matches_oracle_and_unsplit():
    sc = _clustered(53, 3_000, 0.3)
    cam = syn.sphere_cameras(1, 96, 80, 3.0, seed=54)[0]
    G = np.random.default_rng(55).uniform(-1, 1, (1, 3, 80, 96))
    got_s, _ = gpu_grads(sc, [cam], G, tile_split=SPLIT)
    got_u, _ = gpu_grads(sc, [cam], G)
    _, _, state, _ = P.gpu_render(sc, [cam], tile_split=SPLIT)
    heavy, _ = _heavy_tiles(state, SPLIT)
    state.release()
    assert heavy >= 3
    st = P.oracle_settings()
    ref = oracle.backward_image(sc, cam, st, G[0])
    refp = [oracle.backward_image(sc, cam, st, G[0], perturb_seed=s) for s in (1, 2)]
    compare(got_s, ref, refp)
    compare(got_u, ref, refp)
    for f in got_s:
        scale = np.abs(got_u[f]).max() + 1e-30
        assert np.abs(got_s[f] - got_u[f]).max() <= 1e-4 * scale, f


def test_split_multi_view_and_settings_check():
    """A batch of views split together equals the views rendered alone unsplit; out-of-range
    chunk sizes are rejected on the host."""
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    sc = _clustered(56, 10_000)
    cams = syn.sphere_cameras(3, 128, 96, 3.0, seed=57)
    img_s, _, state, _ = P.gpu_render(sc, cams, tile_split=SPLIT)
    state.release()
    for v, cam in enumerate(cams):
        one, _, st1, _ = P.gpu_render(sc, [cam])
        st1.release()
        assert np.abs(img_s[v] - one[0]).max() <= 2 * P.IMAGE_TOL
    with pytest.raises(B.CsError, match="tile_split"):
        P.gpu_render(sc, cams[:1], tile_split=100)
