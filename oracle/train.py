"""Oracle for the training step around the rasterizer (Sec. 3.3): the photometric loss
L = (1 - lambda) L1 + lambda L_D-SSIM (Eq. 6 without the mask term) and the Adam update.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: binary64 numpy, written from the
definitions, sharing nothing with the CUDA path.

Readings (the paper names the terms but not their constants):
  * L1 = mean over views, channels and pixels of |image - target|.
  * D-SSIM = 1 - mean SSIM, SSIM per Wang et al. (2004) with an 11 x 11 Gaussian window of
    standard deviation 1.5 (normalised to sum 1), C1 = 0.01^2, C2 = 0.03^2 for a dynamic range of
    1, local statistics by correlation over each channel plane with zero padding outside the image
    ("same" size), as the 3DGS training loss the paper follows does.
  * lambda = 0.2 (Sec. 3.3).
  * Adam per Kingma and Ba (2015), Algorithm 1: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

parity pinned by tests/test_oracle_train.py: SSIM of an image with itself, the closed form on
constant images away from the border, a brute-force 2-D window sum, central finite differences
of the loss, and the first Adam step's closed form plus torch.optim.Adam on the same inputs.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window() -> np.ndarray:
    """The 1-D Gaussian of the separable window (11 taps, sd 1.5, sum 1)."""
    x = np.arange(WINDOW, dtype=np.float64) - WINDOW // 2
    g = np.exp(-(x * x) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def _filter(a: np.ndarray) -> np.ndarray:
    """Correlate the last two axes with the 11 x 11 window, zero outside the image."""
    g = gaussian_window()
    a = ndimage.correlate1d(a, g, axis=-1, mode="constant", cval=0.0)
    return ndimage.correlate1d(a, g, axis=-2, mode="constant", cval=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of two [..., H, W] arrays."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss_l1_dssim(image: np.ndarray, target: np.ndarray, lam: float = 0.2):
    """(L, dL/dimage) for images [V][3][H][W] (or any [..., H, W])."""
    x = np.asarray(image, np.float64)
    y = np.asarray(target, np.float64)
    M = x.size
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
    B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
    D = B1 * B2
    S = A1 * A2 / D
    L = (1.0 - lam) * np.abs(x - y).mean() + lam * (1.0 - S.mean())
    # derivatives of S w.r.t. the local statistics mu_x, s_xx, s_xy ...
    dS_dmx = 2.0 * (my * A2 - S * mx * B2) / D
    dS_dsxx = -S * B1 / D
    dS_dsxy = 2.0 * A1 / D
    # ... and w.r.t. the filtered moments mu_x, E[x^2], E[xy] (s_xx = E[x^2] - mu_x^2, ...)
    a = dS_dmx - 2.0 * mx * dS_dsxx - my * dS_dsxy
    b = dS_dsxx
    c = dS_dsxy
    # the window is symmetric, so the adjoint of the zero-padded correlation is the same filter
    dS_dx = _filter(a) + 2.0 * x * _filter(b) + y * _filter(c)
    grad = (1.0 - lam) * np.sign(x - y) / M - lam * dS_dx / M
    return float(L), grad


def adam_step(p, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step (Algorithm 1 of Kingma and Ba) in binary64; returns new (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
