"""Serving loop (continuous batching over resident scenes), through the C ABI.

Each result must equal rendering the view alone with cs_forward, whatever batch it lands in;
requests that arrive while batches are on the GPU are admitted as memory frees up; requests
larger than the whole budget, unknown scenes, bad cameras and scenes removed while requests are
queued are reported, not rendered.
"""
import threading
import time

import numpy as np
import pytest

from paper_2411_14974_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _scenes(dev):
    import paper_2411_14974_gb300 as cs
    raw = [syn.surface_scene(31, n=20_000, sh_degree=3), syn.surface_scene(32, n=50_000, sh_degree=1),
           syn.blob_scene(33, n=1000)]
    return raw, [cs.SceneTensors.from_numpy(s, dev) for s in raw]


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    sizes = [(320, 240), (256, 256), (200, 120)]
    out = []
    for i in range(n):
        w, h = sizes[rng.integers(3)]
        cam = syn.sphere_cameras(1, w, h, (3.0, 5.0), seed=int(rng.integers(1 << 30)))[0]
        out.append((int(rng.integers(3)), cam))
    return out


def _alone(scene_t, cam):
    import torch
    import paper_2411_14974_gb300 as cs
    img, _, _ = cs.forward(scene_t, [cam])
    torch.cuda.synchronize()
    return img[0]


@pytest.mark.parametrize("max_batch, n_req", [(8, 24), (40, 64)])
def test_results_alone_equal_results_in_the_mix(max_batch, n_req):
    """Batches of up to 32 views are blended by one persistent launch with a completion flag per
    view; larger ones (max_batch 40) by one launch per view: either way each image equals the view
    rendered alone."""
    import torch
    import paper_2411_14974_gb300 as cs
    dev = torch.device("cuda:0")
    _, scenes = _scenes(dev)
    reqs = _requests(n_req, 1)
    with cs.Server(0, budget_bytes=4 << 30, max_batch=max_batch) as srv:
        sids = [srv.add_scene(s) for s in scenes]
        outs = {}
        for si, cam in reqs:
            img = torch.full((3, cam.height, cam.width), float("nan"), device=dev)
            outs[srv.submit(sids[si], cam, img)] = (si, cam, img)
        done = []
        t0 = time.time()
        while len(done) < len(reqs) and time.time() - t0 < 60:
            done += srv.poll(64, wait_ms=100)
        st = srv.stats()
    assert len(done) == len(reqs) and all(d["status"] == "ok" for d in done)
    assert st["largest_batch"] > 1  # requests were batched
    torch.cuda.synchronize()
    for d in done:
        si, cam, img = outs[d["id"]]
        ref = _alone(scenes[si], cam)
        assert torch.isfinite(img).all()
        assert (img - ref).abs().max().item() <= 1e-4


def test_requests_arriving_while_batches_run_are_admitted():
    import torch
    import paper_2411_14974_gb300 as cs
    dev = torch.device("cuda:0")
    _, scenes = _scenes(dev)
    reqs = _requests(40, 2)
    # a budget for about two 320x240 views of the 50k scene in flight at a time
    with cs.Server(0, budget_bytes=40 << 20, max_batch=4) as srv:
        sids = [srv.add_scene(s) for s in scenes]
        imgs = {}

        def producer():
            for si, cam in reqs:
                img = torch.empty((3, cam.height, cam.width), device=dev)
                imgs[srv.submit(sids[si], cam, img)] = img
                time.sleep(0.002)

        th = threading.Thread(target=producer)
        th.start()
        done = []
        t0 = time.time()
        while len(done) < len(reqs) and time.time() - t0 < 60:
            done += srv.poll(64, wait_ms=50)
        th.join()
        st = srv.stats()
    assert len(done) == len(reqs) and all(d["status"] == "ok" for d in done)
    assert st["batches"] >= 10 and st["largest_batch"] <= 4
    assert st["peak_bytes"] <= 40 << 20
    assert 0 < st["peak_pool_bytes"] <= 40 << 20  # what the pool really held, not only the estimate
    assert all(d["latency_ms"] >= d["queue_ms"] >= 0 for d in done)


def test_budget_bad_requests_and_scene_removal():
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    dev = torch.device("cuda:0")
    _, scenes = _scenes(dev)
    with cs.Server(0, budget_bytes=8 << 20, max_batch=4) as srv:
        sids = [srv.add_scene(s) for s in scenes]
        big = syn.sphere_cameras(1, 1920, 1080, 4.0, seed=5)[0]
        img = torch.empty((3, 1080, 1920), device=dev)
        rid = srv.submit(sids[1], big, img)  # 50k convexes at 1080p: larger than the whole budget
        bad = syn.sphere_cameras(1, 64, 64, 4.0, seed=6)[0]
        bad.fx = float("nan")
        with pytest.raises(B.CsError):
            srv.submit(sids[0], bad, torch.empty((3, 64, 64), device=dev))
        with pytest.raises(B.CsError):
            srv.submit(99, syn.blob_camera(), torch.empty((3, 128, 128), device=dev))
        done = []
        t0 = time.time()
        while not done and time.time() - t0 < 30:
            done += srv.poll(8, wait_ms=50)
        assert done[0]["id"] == rid and done[0]["status"] == "budget"
        srv.remove_scene(sids[2])
        with pytest.raises(B.CsError):
            srv.submit(sids[2], syn.blob_camera(), torch.empty((3, 128, 128), device=dev))
