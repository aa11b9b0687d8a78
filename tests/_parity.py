"""Helpers shared by the GPU parity tests: oracle references with the conditioning mask, and
calls into the CUDA path through the package's C-ABI binding."""
import numpy as np

import oracle

# A pixel is ill-conditioned when moving the projected points by 4 binary32 ulps (two seeded sign
# patterns) changes the binary64 image by more than this, or when a cut-off decision is within
# its band (alpha near tau, T near t_min).
COND_TOL = 2.5e-5
IMAGE_TOL = 1e-4


def oracle_settings(**kw):
    return oracle.settings(**kw)


def gpu_settings(**kw):
    import paper_2411_14974_gb300 as cs
    return cs.Settings(**kw)


def oracle_reference(sc, cam, **kw):
    st = oracle.settings(**kw)
    r0 = oracle.render_image(sc, cam, st)
    d = np.zeros(r0["image"].shape[1:])
    for seed in (1, 2):
        r = oracle.render_image(sc, cam, st, perturb_seed=seed)
        d = np.maximum(d, np.abs(r["image"] - r0["image"]).max(0))
    ill = (d > COND_TOL) | ((r0["flags"] & 3) != 0)
    return r0, ill


def oracle_pixels_reference(sc, cam, pix, **kw):
    st = oracle.settings(**kw)
    r0 = oracle.render_pixels(sc, cam, st, pix)
    d = np.zeros(len(pix))
    for seed in (1, 2):
        r = oracle.render_pixels(sc, cam, st, pix, perturb_seed=seed)
        d = np.maximum(d, np.abs(r["rgb"] - r0["rgb"]).max(1))
    ill = (d > COND_TOL) | ((r0["flags"] & 3) != 0)
    return r0, ill


def gpu_render(sc, cams, keep_state=True, **kw):
    import torch
    import paper_2411_14974_gb300 as cs
    t = cs.SceneTensors.from_numpy(sc, torch.device("cuda:0"))
    img, tf, state = cs.forward(t, cams, cs.Settings(**kw), keep_state=keep_state)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), tf.cpu().numpy().astype(np.float64), state, t
