"""Helpers shared by the GPU parity tests: oracle references with the conditioning mask, and
calls into the CUDA path through the package's C-ABI binding."""
import numpy as np

import oracle

# The references build the hull lines from the same binary32 projected points on which both
# sides decide the hull (oracle setting q_binary32); the continuous maths is binary64.  What
# remains between the two is the GPU's binary32 evaluation of the lines relative to the anchor
# vertex, modelled as at most LINE_REL x (sum of the magnitudes involved) pixels per line value
# (2^-22: twice one rounding per operation).  A pixel is ill-conditioned when the oracle's
# first-order bound of its change under that error exceeds COND_TOL, or when a cut-off decision
# (alpha vs tau, T vs t_min) lies within that error of its threshold.  The model is checked
# against the binary32 record-form evaluation itself in tests/test_oracle_conditioning.py.
COND_TOL = 2.5e-5
IMAGE_TOL = 1e-4
LINE_REL = 2.0 ** -22
PARITY = dict(q_binary32=True, line_rel=LINE_REL)

# Gradients: 1e-3 relative per element with an absolute floor of 1e-4 x the largest oracle
# gradient of the tensor.  An element is ill-conditioned (excluded, counted) when either of two
# seeded sign patterns of the line error model moves its oracle gradient by more than half of
# its tolerance; on the parity scenes the binary32 record-form lines then move the remaining
# elements by at most a tenth of the tolerance and at most 1% of the elements are excluded.
GRAD_REL = 1e-3
GRAD_FLOOR = 1e-4
GRAD_PROBE_FRAC = 0.5
GRAD_MAX_EXCLUDED = 0.01


def oracle_settings(**kw):
    return oracle.settings(**PARITY, **kw)


def gradient_ill(ref, probes, tol):
    """Elements whose oracle gradient moves by more than GRAD_PROBE_FRAC x tol under a probe."""
    sens = np.zeros_like(ref)
    for p in probes:
        sens = np.maximum(sens, np.abs(p - ref))
    return sens > GRAD_PROBE_FRAC * tol


def oracle_reference(sc, cam, **kw):
    r0 = oracle.render_image(sc, cam, oracle_settings(**kw))
    ill = (r0["sens"] > COND_TOL) | ((r0["flags"] & 3) != 0)
    return r0, ill


def oracle_pixels_reference(sc, cam, pix, **kw):
    r0 = oracle.render_pixels(sc, cam, oracle_settings(**kw), pix)
    ill = (r0["sens"] > COND_TOL) | ((r0["flags"] & 3) != 0)
    return r0, ill


def gpu_render(sc, cams, keep_state=True, **kw):
    import torch
    import paper_2411_14974_gb300 as cs
    t = cs.SceneTensors.from_numpy(sc, torch.device("cuda:0"))
    img, tf, state = cs.forward(t, cams, cs.Settings(**kw), keep_state=keep_state)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), tf.cpu().numpy().astype(np.float64), state, t
