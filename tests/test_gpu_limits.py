"""Size limits of the forward path, through the C ABI: the largest images (an 8K frame and a strip
at the 32768-pixel maximum side), a batch of many views, and the rejections just past each limit.

The discrete specification and the sorted pair list are compared with the oracle bit for bit;
images on sampled pixels (the oracle renders pixels one by one), within the image tolerance on
well-conditioned pixels.
"""
import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _parity as P
from tests.test_gpu_forward import check_discrete, check_pairs

pytestmark = pytest.mark.gpu


def _sampled(sc, cam, img, tf, n=400, seed=0):
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], 1).astype(np.int32)
    ref, ill = P.oracle_pixels_reference(sc, cam, pix)
    got = img[:, pix[:, 1], pix[:, 0]].T
    ok = ~ill
    assert ok.mean() > 0.9
    assert np.abs(got - ref["rgb"])[ok].max() <= P.IMAGE_TOL
    assert np.abs(tf[pix[:, 1], pix[:, 0]] - ref["t_final"])[ok].max() <= P.IMAGE_TOL


def test_8k_frame():
    sc = syn.surface_scene(41, n=60_000, sh_degree=3)
    cam = syn.sphere_cameras(1, 7680, 4320, 3.5, seed=42)[0]
    img, tf, state, _ = P.gpu_render(sc, [cam])
    assert state.sizes()["tiles"] == 480 * 270
    disc = check_discrete(state, sc, cam)
    check_pairs(state, [disc], [cam])
    _sampled(sc, cam, img[0], tf[0])


def test_strip_at_the_maximum_side():
    sc = syn.blob_scene(43, n=3000, radius=0.03)
    sc.points[..., 1] *= 0.02  # a thin horizontal band
    cam = syn.blob_camera(32768, 16)
    cam.fx = cam.fy = 4000.0
    img, tf, state, _ = P.gpu_render(sc, [cam])
    disc = check_discrete(state, sc, cam)
    assert disc["visible"].sum() > 100
    check_pairs(state, [disc], [cam])
    _sampled(sc, cam, img[0], tf[0], seed=1)


def test_many_views_in_one_batch():
    import torch
    import paper_2411_14974_gb300 as cs
    sc = syn.surface_scene(44, n=8_000, sh_degree=1)
    cams = syn.sphere_cameras(96, 64, 48, 4.0, seed=45)
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    img, tf, state = cs.forward(t, cams, cs.Settings(), keep_state=True)
    torch.cuda.synchronize()
    assert state.sizes()["records"] == 96 * sc.n
    for v in (0, 37, 95):  # each view of the batch, bit for bit the view rendered alone
        one, tf1, _ = cs.forward(t, [cams[v]], cs.Settings())
        torch.cuda.synchronize()
        assert torch.equal(one[0], img[v]) and torch.equal(tf1[0], tf[v])
    discs = [oracle.discrete(sc, c) for c in cams[:2]]
    two, _, st2 = cs.forward(t, cams[:2], cs.Settings(), keep_state=True)
    torch.cuda.synchronize()
    check_pairs(st2, discs, cams[:2])


def test_requests_past_the_limits_are_rejected():
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    t = cs.SceneTensors.from_numpy(syn.blob_scene(46, n=10), torch.device("cuda:0"))
    with pytest.raises(B.CsError, match="out of range"):
        cs.forward(t, [syn.blob_camera(32769, 8)], cs.Settings())
    with pytest.raises(B.CsError, match="cameras"):
        cs.forward(t, [syn.blob_camera(8, 8)] * 1025, cs.Settings())
    with pytest.raises(B.CsError):
        cs.forward(t, [syn.blob_camera(8, 8)], cs.Settings(tile_test=2))


def test_pair_keys_without_room_for_block_masks():
    """129 views of 4096 x 4112 (65,792 tiles each: 17 tile bits, 8 view bits) leave a pair key no
    room for the 8-bit block mask, so the blend gathers test the records' pixel boxes instead; each
    view of that batch renders bit for bit as it does alone (with masks).  About 52 GB of views."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc = syn.blob_scene(72, n=2000, radius=0.08)
    cams = syn.sphere_cameras(129, 4096, 4112, 4.0, seed=73)
    tiles = (4096 // 16) * ((4112 + 15) // 16)
    assert (len(cams) - 1).bit_length() + (tiles - 1).bit_length() + 8 > 32  # view + tile + mask bits
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    img, tf, _ = cs.forward(t, cams, cs.Settings())
    torch.cuda.synchronize()
    for v in (0, 64, 128):
        one, tf1, _ = cs.forward(t, [cams[v]], cs.Settings())
        torch.cuda.synchronize()
        assert torch.equal(one[0], img[v]) and torch.equal(tf1[0], tf[v]), v
        del one, tf1
    del img, tf
    torch.cuda.empty_cache()


def test_measured_alu_rates_are_plausible():
    """The per-SM rates used as roofline peaks: the transcendental unit and the FP32 FMA pipe,
    measured with clock64 on the device, within a factor of two of 16-32 and 128 per clock."""
    import paper_2411_14974_gb300 as cs
    r = cs.alu_rates(0)
    assert 8.0 <= r["mufu_per_clk_sm"] <= 64.0, r
    assert 64.0 <= r["fma_per_clk_sm"] <= 256.0, r
    assert 500.0 <= r["sm_mhz"] <= 3000.0, r
    assert r["sms"] >= 1

