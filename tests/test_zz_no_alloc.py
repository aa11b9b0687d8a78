"""cs_forward_static, the forward render that allocates nothing, against cs_forward.

Callers that cannot allocate device memory where they render (an engine whose arena owns all
device memory, a real-time loop that must not enter the driver's allocator, a plugin that may
only allocate during set-up) use cs_forward_static: its scratch is a fixed device array inside
the library that every call shares and that keeps the previous call's contents.  Two calls in a
row on different scenes must each give cs_forward's image and transmittance, so nothing left
over from the first call may leak into the second.  Called through the C ABI.
"""
import ctypes

import numpy as np
import pytest

from paper_2411_14974_gb300 import synthetic as syn
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _static_forward(scene_t, cam, settings):
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    H, W = cam.height, cam.width
    img = torch.full((3, H, W), float("nan"), device="cuda:0")
    tf = torch.full((H, W), float("nan"), device="cuda:0")
    sc = scene_t.struct()
    cc = cs.camera_struct(cam)
    st = settings.struct()
    code = B.lib().cs_forward_static(ctypes.byref(sc), ctypes.byref(cc), ctypes.byref(st), img.data_ptr(),
                                     tf.data_ptr(), torch.cuda.current_stream().cuda_stream)
    B.check(code, "cs_forward_static")
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), tf.cpu().numpy().astype(np.float64)


def test_static_forward_matches_cs_forward_on_two_calls_in_a_row():
    import torch
    import paper_2411_14974_gb300 as cs
    dev = torch.device("cuda:0")
    cases = [(syn.workload("blob1k_128", seed=0)[0], syn.blob_camera()),
             (syn.surface_scene(5, n=40_000, sh_degree=3), syn.sphere_cameras(1, 640, 360, 4.0, seed=6)[0])]
    scenes = [cs.SceneTensors.from_numpy(sc, dev) for sc, _ in cases]
    settings = cs.Settings()
    got = [_static_forward(t, cam, settings) for t, (_, cam) in zip(scenes, cases)]  # two calls in a row
    for (img_s, tf_s), t, (_, cam) in zip(got, scenes, cases):
        img, tf, _ = cs.forward(t, [cam], settings)
        torch.cuda.synchronize()
        img = img[0].cpu().numpy().astype(np.float64)
        tf = tf[0].cpu().numpy().astype(np.float64)
        assert np.isfinite(img_s).all() and np.isfinite(tf_s).all()
        assert np.abs(img_s - img).max() <= P.IMAGE_TOL
        assert np.abs(tf_s - tf).max() <= P.IMAGE_TOL


def test_static_forward_rejects_sizes_beyond_its_limits():
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    dev = torch.device("cuda:0")
    big = syn.blob_scene(1, n=65537)
    t = cs.SceneTensors.from_numpy(big, dev)
    with pytest.raises(B.CsError, match="static limit"):
        _static_forward(t, syn.blob_camera(), cs.Settings())
    small = cs.SceneTensors.from_numpy(syn.blob_scene(2, n=100), dev)
    with pytest.raises(B.CsError, match="static limit"):
        _static_forward(small, syn.blob_camera(2048, 1025), cs.Settings())
