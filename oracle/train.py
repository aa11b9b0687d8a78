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


# ---- adaptive refinement: K-way split and pruning (Sec. 3.3, supplement Sec. A) ----------------
def _centre32(points32: np.ndarray) -> np.ndarray:
    """Mean of the K points in binary32: sequential sum over k, then divide by K."""
    f32 = np.float32
    s = points32[:, 0, :].copy()
    for k in range(1, points32.shape[1]):
        s = (s + points32[:, k, :]).astype(f32)
    return (s / f32(points32.shape[1])).astype(f32)


def densify_decisions(points, opacity_raw, sigma_grad_abs, window_steps, threshold=4e-6, prune_opacity=0.03,
                      prune_size=np.inf):
    """Per convex 0 = keep, 1 = split, 2 = prune, all decided in binary32.

    Prune (checked first) when the activated opacity is below prune_opacity or the convex's size,
    the largest distance from its centre to one of its points, exceeds prune_size (supplement
    Sec. A: opacity < 0.03, size > 0.3 x scene size).  Otherwise split when the sharpness statistic,
    the mean |dL/dsigma| over the steps since the last refinement, exceeds the threshold (the
    paper's "loss of sigma exceeds 0.000004").  Non-finite values prune."""
    f32 = np.float32
    p = np.ascontiguousarray(points, f32)
    c = _centre32(p)
    d = (p - c[:, None, :]).astype(f32)
    size = np.sqrt(((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]).astype(f32) + d[..., 2] * d[..., 2]).astype(f32))
    size = size.max(axis=1)
    o = _sigmoid_vec(opacity_raw)
    mean = (np.ascontiguousarray(sigma_grad_abs, f32) / f32(window_steps)).astype(f32)
    prune = ~(o >= f32(prune_opacity)) | ~(size <= f32(prune_size))
    split = ~prune & (mean > f32(threshold))
    return np.where(prune, 2, np.where(split, 1, 0)).astype(np.int32)


def _sigmoid_vec(raw32):
    """sigmoid_spec of every value (the oracle's binary32 activation, evaluated in C)."""
    import oracle
    raw32 = np.ascontiguousarray(raw32, np.float32)
    n = raw32.size
    z = np.zeros(n, np.float32)
    d, s, o = (np.empty(n, np.float32) for _ in range(3))
    oracle.lib().orc_activate(n, oracle._p(z), oracle._p(z), oracle._p(raw32), oracle._p(d), oracle._p(s),
                              oracle._p(o))
    return o


def densify(params: dict, m: dict, v: dict, sigma_grad_abs, window_steps, threshold=4e-6, split_scale=0.7,
            split_sigma_scale=1.5, split_opacity_scale=0.5, prune_opacity=0.03, prune_size=np.inf):
    """Refined raw-parameter set (points, delta, sigma, opacity, sh as log/logit values) and Adam
    moments, in binary32.  Output order: for each input convex in order, itself when kept, its K
    children when split, nothing when pruned.  Child j of a convex with points p_k and centre c
    has points p_j + s (p_k - c) (scaled down by s about its new centre p_j), the same delta and
    colour, sigma x split_sigma_scale (raw: + ln scale) and opacity x split_opacity_scale (raw:
    ln(o'/(1 - o'))), ln being the binary32 definition shared with the tile range; its moments
    start at 0.  Returns (params, m, v, decisions)."""
    import oracle
    f32 = np.float32
    P = {k: np.ascontiguousarray(params[k], f32) for k in ("points", "delta", "sigma", "opacity", "sh")}
    dec = densify_decisions(P["points"], P["opacity"], sigma_grad_abs, window_steps, threshold, prune_opacity,
                            prune_size)
    N, K = P["points"].shape[:2]
    c = _centre32(P["points"])
    d = (P["points"] - c[:, None, :]).astype(f32)
    o = _sigmoid_vec(P["opacity"])
    oc = (o * f32(split_opacity_scale)).astype(f32)
    ratio = (oc / (f32(1.0) - oc).astype(f32)).astype(f32)
    child_op = oracle.ln_spec_array(ratio)
    ln_ss = f32(oracle.ln_spec(float(f32(split_sigma_scale))))
    child_sig = (P["sigma"] + ln_ss).astype(f32)
    out = {k: [] for k in P}
    om = {k: [] for k in P}
    ov = {k: [] for k in P}
    for i in range(N):
        if dec[i] == 2:
            continue
        if dec[i] == 0:
            for k in P:
                out[k].append(P[k][i:i + 1])
                om[k].append(np.ascontiguousarray(m[k], f32)[i:i + 1])
                ov[k].append(np.ascontiguousarray(v[k], f32)[i:i + 1])
            continue
        for j in range(K):
            pts = (P["points"][i, j][None, :] + (f32(split_scale) * d[i]).astype(f32)).astype(f32)
            out["points"].append(pts[None])
            out["delta"].append(P["delta"][i:i + 1])
            out["sigma"].append(child_sig[i:i + 1])
            out["opacity"].append(child_op[i:i + 1])
            out["sh"].append(P["sh"][i:i + 1])
            for k in P:
                om[k].append(np.zeros_like(P[k][i:i + 1]))
                ov[k].append(np.zeros_like(P[k][i:i + 1]))

    def cat(lst, k):
        return np.concatenate(lst, 0) if lst else np.zeros((0,) + P[k].shape[1:], f32)
    return ({k: cat(out[k], k) for k in P}, {k: cat(om[k], k) for k in P}, {k: cat(ov[k], k) for k in P}, dec)
