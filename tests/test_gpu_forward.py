"""GPU forward parity with the oracle, through the C ABI.

Bit-exact: visibility, hull vertex indices, tile ranges, depth keys and the sorted tile-pair lists
(Sec. 3.2).  Within 1e-4 per channel: the images (Eq. 5), outside a conditioning mask, under two
protocols.  (1) Against the oracle with hull lines built from the binary32 projected points
(q_binary32): pixels whose first-order bound of the change under the binary32 line-evaluation
error model exceeds 2.5e-5, or where a cut-off decision is within its band, are excluded (the
model is checked against the binary32 record-form lines in tests/test_oracle_conditioning.py).
(2) Against the binary64-projection oracle: pixels whose value moves by more than 2.5e-5 when the
projected points move by 4 binary32 ulps (four seeded sign patterns), or where a cut-off decision
is within its band, are excluded.  Every test bounds the excluded fraction.
"""
import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _cases as C
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _pack_rect(r):
    r = r.astype(np.uint64)
    return np.stack([r[:, 0] | (r[:, 2] << 16), r[:, 1] | (r[:, 3] << 16)], 1).astype(np.uint32)


def check_discrete(state, sc, cam, rec_base=0, tile_base=0, **kw):
    disc = oracle.discrete(sc, cam, oracle.settings(**kw))
    n = sc.n
    dk = state.array("depth_keys")[rec_base:rec_base + n]
    cnt = state.array("counts")[rec_base:rec_base + n]
    rects = state.array("rects").reshape(-1, 2)[rec_base:rec_base + n]
    hulls = state.array("hulls")[rec_base:rec_base + n]
    vis = disc["visible"].astype(bool)
    assert ((cnt > 0) == vis).all(), "visibility differs"
    assert (dk[vis] == disc["depth_bits"][vis]).all(), "depth keys differ"
    assert (dk[~vis] == 0xFFFFFFFF).all()
    assert (hulls == oracle.pack_hull(disc)).all(), "hull vertex indices differ"
    assert (rects[vis] == _pack_rect(disc["rect"][vis])).all(), "tile ranges differ"
    assert (cnt[vis] == disc["count"][vis]).all(), "kept-tile counts of the exact tile test differ"
    return disc


def check_pairs(state, discs, cams):
    """Bit-exact sorted pair list: key = view << b | tile index within the view (b = bits of the
    largest view's tile count), stable order (tile, view, depth bits, convex index)."""
    tiles = [((c.width + 15) // 16) * ((c.height + 15) // 16) for c in cams]
    lb = (max(tiles) - 1).bit_length()
    keys, vals = [], []
    rb = 0
    for v, (disc, cam) in enumerate(zip(discs, cams)):
        k, val = oracle.sorted_pairs(disc, cam, 0, rb)
        keys.append((v << lb) | k)
        vals.append(val)
        rb += len(disc["visible"])
    keys = np.concatenate(keys)
    vals = np.concatenate(vals)
    perm = np.argsort(keys & ((1 << lb) - 1), kind="stable")
    keys, vals = keys[perm], vals[perm]
    gk = state.array("pair_keys").astype(np.int64)
    gv = state.array("pair_values").astype(np.int64)
    assert len(gk) == len(keys), f"{len(gk)} pairs, expected {len(keys)}"
    assert (gk == keys).all(), "pair keys differ"
    assert (gv == vals).all(), "pair order differs"
    rng = state.array("tile_ranges").reshape(-1, 2).astype(np.int64)
    base = np.concatenate([[0], np.cumsum(tiles)[:-1]])
    want = np.zeros((sum(tiles), 2), np.int64)
    if len(keys):
        brk = np.nonzero(np.diff(keys))[0] + 1
        starts = np.concatenate([[0], brk])
        ends = np.concatenate([brk, [len(keys)]])
        grp = keys[starts]
        gidx = base[grp >> lb] + (grp & ((1 << lb) - 1))
        want[gidx, 0] = starts
        want[gidx, 1] = ends
    assert (rng == want).all(), "tile ranges differ"
    check_tile_order(state, want)


def check_tile_order(state, ranges):
    """The blend launch order: every tile exactly once, by decreasing floor(log2(pairs + 1))."""
    order = state.array("tile_order").astype(np.int64)
    assert len(order) == len(ranges)
    assert (np.sort(order) == np.arange(len(ranges))).all(), "tile order is not a permutation"
    cls = np.floor(np.log2(ranges[order, 1] - ranges[order, 0] + 1.0))
    assert (np.diff(cls) <= 0).all(), "tile order is not longest class first"


def check_image(img, ref, ill, max_ill=0.02):
    d = np.abs(img - ref["image"]).max(0)
    frac = float(ill.mean())
    assert frac <= max_ill, f"{frac:.4f} of the pixels are ill-conditioned"
    worst = float(d[~ill].max()) if (~ill).any() else 0.0
    assert worst <= P.IMAGE_TOL, f"max |gpu - oracle| = {worst:.3e} on well-conditioned pixels"
    return worst, frac


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_blob1k_128_discrete_and_order(seed):
    sc, cams = syn.workload("blob1k_128", seed=seed)
    img, tf, state, _ = P.gpu_render(sc, cams)
    disc = check_discrete(state, sc, cams[0])
    check_pairs(state, [disc], cams)


@pytest.mark.parametrize("scene", ["blob", "surface", "clustered"])
def test_exact_tile_test_parity(scene):
    """tile_test = 1: the kept tiles of every convex (per thread for small rectangles, per warp for
    large ones, in the preprocess count and again in the emission) equal the oracle's bit for bit,
    and the image is unchanged within the parity bar."""
    if scene == "blob":
        sc, cam = syn.workload("blob1k_128", seed=5)[0], syn.blob_camera()
    elif scene == "surface":
        sc, cam = syn.surface_scene(31, n=30_000, sh_degree=1), syn.sphere_cameras(1, 320, 240, 3.0, seed=32)[0]
    else:
        sc = syn.surface_scene(33, n=30_000, sh_degree=0, clustered_fraction=0.9)
        sc.points = (sc.points.mean(axis=1, keepdims=True) + 3.0 * (sc.points - sc.points.mean(axis=1, keepdims=True))).astype(np.float32)
        cam = syn.sphere_cameras(1, 480, 360, 3.0, seed=34)[0]
    img, tf, state, _ = P.gpu_render(sc, [cam], tile_test=1)
    disc = check_discrete(state, sc, cam, tile_test=1)
    area = (disc["rect"][:, 2] - disc["rect"][:, 0] + 1) * (disc["rect"][:, 3] - disc["rect"][:, 1] + 1)
    vis = disc["visible"] == 1
    assert (disc["count"][vis] < area[vis]).any()  # the test removes tiles here
    if scene == "clustered":
        assert (area[vis] > 8).sum() > 100  # the warp-cooperative path runs
    check_pairs(state, [disc], [cam])
    ref, ill = P.oracle_reference(sc, cam, tile_test=1)
    check_image(img[0], ref, ill, max_ill={"blob": 0.03, "surface": 0.06, "clustered": 0.04}[scene])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_blob1k_128_image(seed):
    sc, cams = syn.workload("blob1k_128", seed=seed)
    ref, ill = P.oracle_reference(sc, cams[0])
    img, tf, state, _ = P.gpu_render(sc, cams)
    check_image(img[0], ref, ill)
    assert np.abs(tf[0] - ref["t_final"])[~ill].max() <= P.IMAGE_TOL


def test_well_conditioned_needs_no_mask():
    sc, cams = syn.workload("blob1k_128", seed=3)
    rng = np.random.default_rng(3)
    sc.sigma = np.exp(rng.uniform(np.log(0.01), np.log(0.3), sc.n)).astype(np.float32)
    sc.delta = np.exp(rng.uniform(np.log(0.5), np.log(5.0), sc.n)).astype(np.float32)
    ref, ill = P.oracle_reference(sc, cams[0])
    img, _, _, _ = P.gpu_render(sc, cams, keep_state=False)
    d = np.abs(img[0] - ref["image"]).max(0)
    flag = (ref["flags"] & 3) != 0  # only cut-off decisions within their band are excluded
    assert flag.mean() < 0.01
    assert d[~flag].max() <= P.IMAGE_TOL


def _fp64_protocol_reference(sc, cam, **kw):
    """The second parity protocol: the oracle's binary64 projection (no binary32 vertices), and a
    mask of the pixels whose binary64 value moves by more than COND_TOL when every projected
    coordinate moves by 4 binary32 ulps (four seeded sign patterns), or where a cut-off decision
    lies within its band."""
    st = oracle.settings(perturb_ulps=4.0, **kw)
    r0 = oracle.render_image(sc, cam, st)
    moved = np.zeros(r0["image"].shape[1:])
    for seed in (1, 2, 3, 4):
        moved = np.maximum(moved, np.abs(oracle.render_image(sc, cam, st, perturb_seed=seed)["image"] -
                                         r0["image"]).max(0))
    flagged = (r0["flags"] & 3) != 0
    return r0, (moved > P.COND_TOL) | flagged, flagged


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_blob1k_128_image_binary64_projection(seed):
    """Against the binary64-projection oracle with the 4-ulp vertex probe as the mask."""
    sc, cams = syn.workload("blob1k_128", seed=seed)
    ref, ill, _ = _fp64_protocol_reference(sc, cams[0])
    img, tf, _, _ = P.gpu_render(sc, cams, keep_state=False)
    check_image(img[0], ref, ill, max_ill=0.02)
    assert np.abs(tf[0] - ref["t_final"])[~ill].max() <= P.IMAGE_TOL


def test_well_conditioned_binary64_projection_needs_no_probe_mask():
    """sigma in [0.01, 0.3], delta in [0.5, 5]: against the binary64-projection oracle with only
    the cut-off decisions within their bands excluded (no vertex-probe mask)."""
    sc, cams = syn.workload("blob1k_128", seed=3)
    rng = np.random.default_rng(3)
    sc.sigma = np.exp(rng.uniform(np.log(0.01), np.log(0.3), sc.n)).astype(np.float32)
    sc.delta = np.exp(rng.uniform(np.log(0.5), np.log(5.0), sc.n)).astype(np.float32)
    ref, _, flagged = _fp64_protocol_reference(sc, cams[0])
    img, _, _, _ = P.gpu_render(sc, cams, keep_state=False)
    assert flagged.mean() < 0.02
    d = np.abs(img[0] - ref["image"]).max(0)
    assert d[~flagged].max() <= P.IMAGE_TOL


@pytest.mark.parametrize("w,h", [(100, 75), (17, 33), (1, 1), (129, 16)])
def test_ragged_sizes(w, h):
    sc, _ = syn.workload("blob1k_128", seed=4)
    cam = syn.blob_camera(w, h)
    ref, ill = P.oracle_reference(sc, cam)
    img, _, state, _ = P.gpu_render(sc, [cam])
    disc = check_discrete(state, sc, cam)
    check_pairs(state, [disc], [cam])
    check_image(img[0], ref, ill, max_ill=0.04 if w * h > 64 else 1.0)


@pytest.mark.parametrize("k,deg", [(3, 1), (4, 2), (5, 3), (7, 0), (8, 3)])
def test_points_per_convex_and_sh_degree(k, deg):
    sc = syn.blob_scene(5 + k, n=600, k=k, radius=0.08, sh_degree=deg)
    cam = syn.blob_camera(96, 80)
    ref, ill = P.oracle_reference(sc, cam)
    img, _, state, _ = P.gpu_render(sc, [cam])
    disc = check_discrete(state, sc, cam)
    check_pairs(state, [disc], [cam])
    # small sharp convexes at 96x80, and projected triangles that are often thin slivers: a larger
    # share of pixels is ill-conditioned than in the 128x128 blob scenes
    check_image(img[0], ref, ill, max_ill={3: 0.04, 4: 0.05, 5: 0.06, 7: 0.04, 8: 0.07}[k])


@pytest.mark.parametrize("kw", [dict(dist_power=0.0), dict(dist_power=0.5), dict(dist_power=2.0),
                                dict(dist_mode=1), dict(tau=0.02, t_min=1e-3, bg=(0.2, 0.5, 1.0)),
                                dict(alpha_max=0.5)])
def test_settings_variants(kw):
    sc, cams = syn.workload("blob1k_128", seed=6)
    if kw.get("dist_power") == 2.0:
        sc.delta /= 4.0
        sc.sigma /= 4.0
    ref, ill = P.oracle_reference(sc, cams[0], **kw)
    img, _, state, _ = P.gpu_render(sc, cams, **kw)
    disc = check_discrete(state, sc, cams[0], **kw)
    check_pairs(state, [disc], cams)
    check_image(img[0], ref, ill, max_ill=0.04)


def test_tau_zero_full_screen_ranges():
    sc = syn.blob_scene(7, n=60, radius=0.1)
    cam = syn.blob_camera(64, 48)
    kw = dict(tau=0.0, t_min=0.0)
    ref, ill = P.oracle_reference(sc, cam, **kw)
    img, _, state, _ = P.gpu_render(sc, [cam], **kw)
    disc = check_discrete(state, sc, cam, **kw)
    assert disc["full"][disc["visible"] == 1].all()
    assert state.sizes()["pairs"] == int(disc["visible"].sum()) * 4 * 3
    check_pairs(state, [disc], [cam])
    check_image(img[0], ref, ill, max_ill=0.05)


def test_empty_and_fully_culled_scenes():
    cam = syn.blob_camera(40, 24)
    empty = syn.Scene(np.zeros((0, 6, 3), np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                      np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0)
    img, tf, state, _ = P.gpu_render(empty, [cam], bg=(0.25, 0.5, 0.75))
    assert np.allclose(img[0], np.array([0.25, 0.5, 0.75], np.float32)[:, None, None].astype(np.float64))
    assert (tf == 1).all() and state.sizes()["pairs"] == 0
    sc = syn.blob_scene(8, n=50)
    sc.points[..., 2] -= 10.0  # everything behind the camera
    img, tf, state, _ = P.gpu_render(sc, [cam])
    assert (img == 0).all() and (tf == 1).all() and state.sizes()["pairs"] == 0
    assert (state.array("counts") == 0).all()


def test_nonfinite_and_invalid_parameters_are_culled():
    sc = syn.blob_scene(9, n=200)
    sc.points[0, 0, 0] = np.nan
    sc.delta[1] = -1.0
    sc.sigma[2] = np.inf
    sc.opacity[3] = 0.0
    cam = syn.blob_camera()
    ref, ill = P.oracle_reference(sc, cam)
    img, _, state, _ = P.gpu_render(sc, [cam])
    disc = check_discrete(state, sc, cam)
    assert not disc["visible"][:4].any()
    check_image(img[0], ref, ill)


def test_raw_parameters_are_activated_in_the_forward():
    """CS_ACT_EXP_SIGMOID: the forward activates log delta, log sigma and logit opacity (Sec. 3.3)
    in the binary32 definition both sides share, so the discrete spec stays bit-exact; raw values
    beyond the exp range make delta/sigma infinite or zero and opacity 0, which culls."""
    raw = syn.workload("blob1k_128", seed=3)[0].as_raw()
    raw.delta[0], raw.sigma[1], raw.delta[2], raw.opacity[3] = 100.0, -100.0, 88.9, -300.0
    cam = syn.blob_camera()
    act = oracle.activate(raw)
    img, tf, state, _ = P.gpu_render(raw, [cam])
    disc = check_discrete(state, act, cam)
    assert not disc["visible"][:4].any()
    check_pairs(state, [disc], [cam])
    ref, ill = P.oracle_reference(act, cam)
    check_image(img[0], ref, ill)


def _widened(sc, dtype):
    """The scene as the 16-bit storage holds it, widened back to float32 (exactly)."""
    import torch
    out = sc.copy()
    for name in ("points", "delta", "sigma", "opacity", "sh"):
        t = torch.as_tensor(getattr(sc, name)).to(dtype).to(torch.float32)
        setattr(out, name, np.ascontiguousarray(t.numpy()))
    return out


@pytest.mark.parametrize("dtype_name", ["float16", "bfloat16"])
def test_light_16bit_storage(dtype_name):
    """16-bit parameter storage (the light model): the kernels widen every value on load, so the
    render equals the oracle's on the widened float32 values, the discrete spec bit for bit."""
    import torch
    import paper_2411_14974_gb300 as cs
    dtype = getattr(torch, dtype_name)
    for sc, cam in ((syn.workload("blob1k_128", seed=4)[0], syn.blob_camera()),
                    (syn.surface_scene(13, n=20_000, sh_degree=3), syn.sphere_cameras(1, 160, 120, 4.0, seed=14)[0])):
        wide = _widened(sc, dtype)
        t = cs.SceneTensors.from_numpy(sc, torch.device("cuda:0"), dtype=dtype)
        assert t.storage == (1 if dtype == torch.float16 else 2)
        img, tf, state = cs.forward(t, [cam], cs.Settings(), keep_state=True)
        torch.cuda.synchronize()
        disc = check_discrete(state, wide, cam)
        check_pairs(state, [disc], [cam])
        ref, ill = P.oracle_reference(wide, cam)
        check_image(img[0].cpu().numpy().astype(np.float64), ref, ill, max_ill=0.06)
        state.release()


def test_each_thread_gets_its_own_context_released_when_the_thread_ends():
    """The binding gives every host thread its own library context (calls on one context must not
    overlap); a thread's context renders like the main thread's and is released when the thread
    ends."""
    import gc
    import threading
    import weakref
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300.rasterizer import Context
    sc, cams = syn.workload("blob1k_128", seed=0)
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    want, _, _ = cs.forward(t, cams)
    torch.cuda.synchronize()
    seen = {}

    def work():
        img, _, _ = cs.forward(t, cams)
        torch.cuda.synchronize()
        seen["img"] = img
        ctx = Context.get(0)
        seen["same"] = ctx is Context.get(0)
        seen["ref"] = weakref.ref(ctx)

    th = threading.Thread(target=work)
    th.start()
    th.join()
    gc.collect()
    assert seen["same"]
    assert seen["ref"]() is None, "the thread's context outlived the thread"
    assert Context.get(0) is not None
    assert torch.equal(seen["img"], want)


def test_multi_view_equals_single_views():
    """Views are binned and sorted together (view index in the tile key); each view's image is the
    same, bit for bit, as rendering it alone."""
    sc = syn.surface_scene(11, n=20_000, sh_degree=3)
    cams = syn.sphere_cameras(3, 160, 120, 4.0, seed=12)
    img, _, state, _ = P.gpu_render(sc, cams)
    discs = [check_discrete(state, sc, c, rec_base=i * sc.n) for i, c in enumerate(cams)]
    check_pairs(state, discs, cams)
    for v, cam in enumerate(cams):
        one, _, _, _ = P.gpu_render(sc, [cam], keep_state=False)
        assert (one[0] == img[v]).all()


def test_surface_scene_image_sh3():
    sc = syn.surface_scene(13, n=30_000, sh_degree=3)
    cam = syn.sphere_cameras(1, 200, 150, 4.0, seed=14)[0]
    ref, ill = P.oracle_reference(sc, cam)
    img, _, state, _ = P.gpu_render(sc, [cam])
    check_discrete(state, sc, cam)
    # sub-pixel, very sharp convexes at this resolution: more alpha ~ tau crossings
    check_image(img[0], ref, ill, max_ill=0.045)


def test_square_worked_example_on_gpu():
    sc = C.square_scene()
    cam = C.axis_camera()
    img, _, _, _ = P.gpu_render(sc, [cam], tau=0.0, alpha_max=1.0, t_min=0.0)
    I, _ = C.square_indicator_closed_form(128, 128, 63.5, 8.0, 2.0, 0.5)
    assert np.abs(img[0, 0] - 0.5 * I).max() < 1e-5


def _unit(rng, shape):
    u = rng.normal(size=shape + (3,))
    return u / np.linalg.norm(u, axis=-1, keepdims=True)


def test_equal_depth_keys_keep_convex_order():
    """Every convex a copy of the same points (one depth key for all; the depth sort then runs no
    pass) with its own smoothness, sharpness, opacity and colour: ties keep convex-index order in
    every tile, as in the oracle, and the image matches."""
    sc = syn.blob_scene(71, n=300, radius=0.3)
    sc.points = np.repeat(sc.points[:1], sc.n, axis=0)
    cam = syn.blob_camera(96, 80)
    img, tf, state, _ = P.gpu_render(sc, [cam])
    disc = check_discrete(state, sc, cam)
    keys = disc["depth_bits"][disc["visible"] == 1]
    assert len(keys) == sc.n and (keys == keys[0]).all()
    check_pairs(state, [disc], [cam])
    ref, ill = P.oracle_reference(sc, cam)
    check_image(img[0], ref, ill)


def test_depth_keys_over_a_wide_range():
    """Camera distances from 0.06 to 90 (binary32 keys that differ in their exponent bits, so the
    depth sort orders more than 24 key bits in four passes): the pair list equals the oracle's bit
    for bit."""
    rng = np.random.default_rng(70)
    n = 2000
    depth = np.exp(rng.uniform(np.log(0.06), np.log(90.0), n))
    ang = rng.uniform(-0.35, 0.35, (n, 2))
    centres = np.stack([depth * np.tan(ang[:, 0]), depth * np.tan(ang[:, 1]), depth - 4.0], 1)
    sc = syn.blob_scene(70, n=n)
    sc.points = (centres[:, None, :] + 0.02 * depth[:, None, None] * _unit(rng, (n, sc.points.shape[1]))).astype(
        np.float32)
    cam = syn.blob_camera(256, 192)
    img, tf, state, _ = P.gpu_render(sc, [cam])
    disc = check_discrete(state, sc, cam)
    keys = disc["depth_bits"][disc["visible"] == 1].astype(np.int64)
    assert len(keys) > n // 2 and (int(keys.max()) ^ int(keys.min())) >> 24
    check_pairs(state, [disc], [cam])


@pytest.mark.parametrize("seed", [0, 1])
def test_work_counts_against_the_oracle(seed):
    """Evaluations counted on the GPU (the instrumented blend kernels) against the oracle on the
    1000-convex 128 x 128 scenes: every pixel is counted once; the backward's contributing pairs
    (alpha >= tau up to each pixel's last contributor, the pairs the forward composited) equal the
    oracle's composited pairs up to the pixels whose cut-off decisions sit within their error
    bands; the forward, which may evaluate a record past a pixel's termination, counts no fewer."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc, cams = syn.workload("blob1k_128", seed=seed)
    cam = cams[0]
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    _, _, st = cs.forward(t, [cam], cs.Settings(), keep_state=True)
    wc = cs.work_counts(st, torch.ones((1, 3, cam.height, cam.width), device=dev))
    torch.cuda.synchronize()
    st.release()
    ref = oracle.render_image(sc, cam, oracle.settings())
    nc = ref["n_contrib"].astype(np.int64)
    flagged = ref["flags"] != 0
    total, slack = int(nc.sum()), int(nc[flagged].sum() + flagged.sum())
    f, b = wc["forward"], wc["backward"]
    assert f["pixels"] == b["pixels"] == cam.width * cam.height
    assert abs(b["contributing"] - total) <= slack, (b["contributing"], total, slack)
    assert f["contributing"] >= b["contributing"]
    assert f["visited"] >= f["passed"] >= f["contributing"] and f["lines_visited"] >= f["lines_passed"]
