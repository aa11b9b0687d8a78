"""Pins for the training-step oracle (Sec. 3.3: L1 + D-SSIM loss, Adam).

References other than the oracle itself: SSIM's identity and constant-image closed form, a
brute-force 2-D window sum, binary64 central finite differences of the loss, the closed form of
Adam's first step and torch.optim.Adam (float64, CPU) on the same inputs.
"""
import math

import numpy as np
import pytest

from oracle import train as T


def test_window_is_a_normalised_symmetric_gaussian():
    g = T.gaussian_window()
    assert g.shape == (11,)
    assert abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    assert abs(g[6] / g[5] - math.exp(-1.0 / (2 * 1.5 ** 2))) < 1e-14


def test_ssim_of_an_image_with_itself_is_one():
    x = np.random.default_rng(0).uniform(0, 1, (2, 3, 20, 27))
    np.testing.assert_allclose(T.ssim_map(x, x), 1.0, atol=1e-12)
    L, g = T.loss_l1_dssim(x, x)
    assert abs(L) < 1e-12
    # at x = y the D-SSIM term is at its minimum (zero gradient); the L1 subgradient sign(0) = 0
    assert np.abs(g).max() < 1e-12


def test_constant_images_closed_form_away_from_the_border():
    c1, c2 = 0.3, 0.7
    x = np.full((40, 40), c1)
    y = np.full((40, 40), c2)
    s = T.ssim_map(x, y)
    want = (2 * c1 * c2 + T.C1) / (c1 * c1 + c2 * c2 + T.C1)  # variances and covariance vanish
    np.testing.assert_allclose(s[5:-5, 5:-5], want, rtol=1e-12)


def test_separable_filter_matches_a_brute_force_window_sum():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (13, 17))
    y = rng.uniform(0, 1, (13, 17))
    g = T.gaussian_window()
    w2 = np.outer(g, g)
    H, W = x.shape

    def win(a, i, j):
        s = 0.0
        for di in range(-5, 6):
            for dj in range(-5, 6):
                ii, jj = i + di, j + dj
                if 0 <= ii < H and 0 <= jj < W:
                    s += w2[di + 5, dj + 5] * a[ii, jj]
        return s

    got = T.ssim_map(x, y)
    for i, j in [(0, 0), (6, 8), (12, 16), (3, 14), (9, 1)]:
        mx, my = win(x, i, j), win(y, i, j)
        sxx, syy, sxy = win(x * x, i, j) - mx * mx, win(y * y, i, j) - my * my, win(x * y, i, j) - mx * my
        want = ((2 * mx * my + T.C1) * (2 * sxy + T.C2)) / ((mx * mx + my * my + T.C1) * (sxx + syy + T.C2))
        assert abs(got[i, j] - want) < 1e-13


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_loss_gradient_matches_finite_differences(lam):
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (1, 3, 14, 18))
    y = rng.uniform(0, 1, (1, 3, 14, 18))
    L, g = T.loss_l1_dssim(x, y, lam)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 7, 9), (0, 2, 13, 17), (0, 0, 3, 16), (0, 2, 10, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (T.loss_l1_dssim(xp, y, lam)[0] - T.loss_l1_dssim(xm, y, lam)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(g[idx]), 1e-3), (idx, fd, g[idx])


def test_l1_part_alone():
    x = np.array([[[[0.1, 0.9], [0.5, 0.5]]]])
    y = np.array([[[[0.3, 0.2], [0.5, 0.6]]]])
    L, g = T.loss_l1_dssim(x, y, 0.0)
    assert abs(L - (0.2 + 0.7 + 0.0 + 0.1) / 4) < 1e-15
    np.testing.assert_array_equal(g, np.array([[[[-0.25, 0.25], [0.0, -0.25]]]]))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p, g = rng.normal(size=100), rng.normal(size=100)
    z = np.zeros(100)
    p1, m1, v1 = T.adam_step(p, g, z, z, lr=0.01, t=1, eps=1e-8)
    # bias correction makes m_hat = g and v_hat = g^2 at t = 1
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-14)


def test_adam_matches_torch_optim_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=64)
    grads = [rng.normal(size=64) for _ in range(5)]
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.005, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(64), np.zeros(64)
    for t, gr in enumerate(grads, 1):
        tp.grad = torch.tensor(gr, dtype=torch.float64)
        opt.step()
        p, m, v = T.adam_step(p, gr, m, v, lr=0.005, t=t, eps=1e-8)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


# ---- adaptive refinement (split / prune) --------------------------------------------------------
def _raw_params(n, seed=0, k=6, deg=1):
    from paper_2411_14974_gb300 import synthetic as syn
    r = syn.blob_scene(seed, n=n, k=k, sh_degree=deg).as_raw()
    return dict(points=r.points, delta=r.delta, sigma=r.sigma, opacity=r.opacity, sh=r.sh)


def _zeros_like(P):
    return {k: np.zeros_like(v) for k, v in P.items()}


def test_densify_with_nothing_to_do_is_the_identity():
    P = _raw_params(40)
    M = {k: np.random.default_rng(1).normal(size=v.shape).astype(np.float32) for k, v in P.items()}
    out, m, v, dec = T.densify(P, M, M, np.zeros(40, np.float32), 10, threshold=1.0, prune_opacity=0.0)
    assert (dec == 0).all()
    for k in P:
        np.testing.assert_array_equal(out[k], P[k])
        np.testing.assert_array_equal(m[k], M[k])


def test_split_children_follow_the_paper():
    """K children centred at the parent's points, offsets scaled by s, same delta and colour,
    sigma x 1.5 and opacity x 0.5 after activation, zero moments."""
    import oracle
    P = _raw_params(3, seed=2, k=5)
    acc = np.array([0.0, 1.0, 0.0], np.float32)  # only convex 1 splits
    out, m, v, dec = T.densify(P, _zeros_like(P), _zeros_like(P), acc, 1, threshold=0.5, split_scale=0.6,
                               prune_opacity=0.0)
    assert dec.tolist() == [0, 1, 0]
    assert out["points"].shape[0] == 2 + 5
    parent = P["points"][1].astype(np.float64)
    c = parent.mean(axis=0)
    for j in range(5):
        child = out["points"][1 + j].astype(np.float64)
        np.testing.assert_allclose(child.mean(axis=0), parent[j], atol=1e-6)
        np.testing.assert_allclose(child - child.mean(axis=0), 0.6 * (parent - c), atol=1e-6)
        assert out["delta"][1 + j] == P["delta"][1]
        np.testing.assert_array_equal(out["sh"][1 + j], P["sh"][1])
        s_parent = math.exp(float(P["sigma"][1]))
        assert abs(math.exp(float(out["sigma"][1 + j])) - 1.5 * s_parent) <= 1e-6 * s_parent
        o_parent = 1.0 / (1.0 + math.exp(-float(P["opacity"][1])))
        o_child = 1.0 / (1.0 + math.exp(-float(out["opacity"][1 + j])))
        assert abs(o_child - 0.5 * o_parent) <= 1e-6
        for k in P:
            assert not m[k][1 + j].any() and not v[k][1 + j].any()
    np.testing.assert_array_equal(out["points"][0], P["points"][0])
    np.testing.assert_array_equal(out["points"][-1], P["points"][2])


def test_prune_by_opacity_and_size_and_nonfinite():
    P = _raw_params(6, seed=3)
    P["opacity"][0] = -5.0                              # sigmoid ~ 0.0067 < 0.03
    P["opacity"][1] = float(np.log(0.031 / 0.969))      # just above 0.03: kept
    P["points"][2] = P["points"][2] * 0 + np.array([0.0, 0.0, 0.0], np.float32)
    P["points"][2][0] = [1.0, 0.0, 0.0]                 # size about 0.83 > 0.5
    P["points"][3][0, 0] = np.nan
    acc = np.full(6, 1.0, np.float32)                   # everything else would split
    out, m, v, dec = T.densify(P, _zeros_like(P), _zeros_like(P), acc, 1, threshold=0.5, prune_size=0.5)
    assert dec.tolist()[:4] == [2, 1, 2, 2]
    assert out["points"].shape[0] == 6 * int((dec == 1).sum())


def test_split_decision_is_strictly_greater_in_binary32():
    P = _raw_params(3, seed=4)
    thr = np.float32(4e-6)
    acc = np.array([thr * 8, np.nextafter(thr, np.float32(1)) * 8, np.nextafter(thr, np.float32(0)) * 8],
                   np.float32)
    dec = T.densify_decisions(P["points"], P["opacity"], acc, 8, threshold=float(thr), prune_opacity=0.0)
    assert dec.tolist() == [0, 1, 0]
