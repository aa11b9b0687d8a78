"""GPU parity of the training step around the renderer (Sec. 3.3), through the C ABI:
cs_loss_l1_dssim against the oracle's binary64 L1 + D-SSIM loss and gradient, cs_adam_step
against the oracle's Adam update, and the Trainer's composition of forward, loss, backward and
Adam on raw parameters.

Tolerances: the loss to 1e-5 relative (binary32 window sums of a few hundred terms); the loss
gradient per element to 1e-3 relative with a floor of 1e-4 x its largest magnitude (the SSIM
statistics s_xx = E_xx - mu_x^2 lose a few bits to cancellation in binary32); Adam's v to 2e-6
relative (positive terms, three roundings a step), m to 1e-6 relative plus 2e-7 absolute (its
terms cancel), the parameters to 2e-6 absolute (the update divides m's error by sqrt(v)).
"""
import numpy as np
import pytest

import oracle
from oracle import train as OT
from paper_2411_14974_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch.device("cuda:0")


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device=_dev())


@pytest.mark.parametrize("shape,lam,same", [((1, 3, 16, 32), 0.2, False), ((2, 3, 37, 53), 0.2, False),
                                            ((1, 3, 5, 7), 1.0, False), ((1, 3, 70, 41), 0.0, False),
                                            ((1, 3, 33, 45), 0.2, True)])
def test_loss_and_gradient_match_oracle(shape, lam, same):
    import torch
    import paper_2411_14974_gb300 as cs
    rng = np.random.default_rng(sum(shape))
    x = rng.uniform(0, 1, shape).astype(np.float32)
    y = x.copy() if same else rng.uniform(0, 1, shape).astype(np.float32)
    L_ref, g_ref = OT.loss_l1_dssim(x.astype(np.float64), y.astype(np.float64), lam)
    loss, g = cs.loss_l1_dssim(_t(x), _t(y), lam)
    torch.cuda.synchronize()
    L = float(loss.item())
    g = g.cpu().numpy().astype(np.float64)
    assert abs(L - L_ref) <= 1e-5 * max(abs(L_ref), 1e-3), (L, L_ref)
    if same:  # the gradient vanishes; binary32 leaves cancellation noise far below an L1 step 1/M
        tol = np.full_like(g_ref, 1e-3 / x.size)
        scale = 1.0 / x.size
    else:
        scale = np.abs(g_ref).max()
        tol = 1e-3 * np.abs(g_ref) + 1e-4 * scale
    assert (np.abs(g - g_ref) <= tol).all(), np.abs(g - g_ref).max() / scale


def test_loss_only_and_large_image():
    import torch
    import paper_2411_14974_gb300 as cs
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (1, 3, 270, 480)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1).astype(np.float32)
    L_ref, g_ref = OT.loss_l1_dssim(x.astype(np.float64), y.astype(np.float64), 0.2)
    loss, none = cs.loss_l1_dssim(_t(x), _t(y), 0.2, grad=False)
    assert none is None
    assert abs(float(loss.item()) - L_ref) <= 1e-5 * L_ref
    _, g = cs.loss_l1_dssim(_t(x), _t(y), 0.2)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    tol = 1e-3 * np.abs(g_ref) + 1e-4 * np.abs(g_ref).max()
    assert (np.abs(g - g_ref) <= tol).all()


def test_adam_matches_oracle_over_steps():
    import torch
    import paper_2411_14974_gb300 as cs
    rng = np.random.default_rng(3)
    sizes = [1, 3, 4096, 4097, 10_000, 0, 70_001]
    lrs = [0.01, 0.005, 5e-4, 0.0045, 0.025, 0.1, 0.0025]
    # a one-element offset makes the second group's buffers 4-byte aligned only (scalar path)
    P = [rng.normal(size=n).astype(np.float32) for n in sizes]
    dev = _dev()
    params, grads, ms, vs, accs = [], [], [], [], []
    for i, n in enumerate(sizes):
        off = 1 if i == 1 else 0
        buf = torch.zeros(n + off, device=dev)
        buf[off:] = torch.as_tensor(P[i], device=dev)
        params.append(buf[off:])
        mk = lambda: torch.zeros(n + off, device=dev)[off:]
        grads.append(mk()), ms.append(mk()), vs.append(mk()), accs.append(mk())
    ref = [(P[i].astype(np.float64), np.zeros(n), np.zeros(n)) for i, n in enumerate(sizes)]
    acc_ref = [np.zeros(n) for n in sizes]
    for t in range(1, 5):
        G = [rng.normal(size=n).astype(np.float32) for n in sizes]
        for i in range(len(sizes)):
            grads[i].copy_(torch.as_tensor(G[i], device=dev))
        groups = [dict(param=params[i], grad=grads[i], m=ms[i], v=vs[i], lr=lrs[i], grad_abs_sum=accs[i])
                  for i in range(len(sizes))]
        cs.adam_step(groups, t, 0.9, 0.999, 1e-8, zero_grad=True)
        for i in range(len(sizes)):
            p, m, v = ref[i]
            # the ABI takes the betas as binary32 (0.999f differs from 0.999 by 1.3e-8)
            ref[i] = OT.adam_step(p, G[i].astype(np.float64), m, v, float(np.float32(lrs[i])), t,
                                  float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8)))
            acc_ref[i] += np.abs(G[i].astype(np.float64))
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        p, m, v = ref[i]
        gp = params[i].cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(gp, p, rtol=1e-6, atol=2e-6)
        # m = b1 m + (1 - b1) g rounds at 2^-24 of its terms (|0.1 g| <= 0.5 here), not of a result
        # that cancels toward 0: three roundings a step over four steps stay below 2e-7
        np.testing.assert_allclose(ms[i].cpu().numpy(), m, rtol=1e-6, atol=2e-7)
        np.testing.assert_allclose(vs[i].cpu().numpy(), v, rtol=2e-6, atol=1e-12)
        np.testing.assert_allclose(accs[i].cpu().numpy(), acc_ref[i], rtol=1e-6)
        assert (grads[i] == 0).all()


def test_adam_rejects_bad_arguments():
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    p = torch.zeros(10, device=_dev())
    g = dict(param=p, grad=torch.zeros_like(p), m=torch.zeros_like(p), v=torch.zeros_like(p), lr=0.1)
    with pytest.raises(B.CsError, match="step"):
        cs.adam_step([g], 0)
    with pytest.raises(B.CsError, match="beta"):
        cs.adam_step([g], 1, beta1=1.0)


def _raw_blob(seed):
    sc = syn.blob_scene(seed, n=300, radius=0.08, sh_degree=1)
    sc.points[..., :2] *= 0.5
    return sc.as_raw()


def test_trainer_step_is_forward_loss_backward_adam():
    """One Trainer step is the four C-ABI calls made one by one: the same loss, the same gradients
    reaching Adam (m = (1 - beta1) g after step 1; the backward's float atomics may reorder sums),
    and the same parameters wherever the gradient's sign is well determined (Adam's first step is
    lr sign(g))."""
    import torch
    import paper_2411_14974_gb300 as cs
    raw = _raw_blob(1)
    cam = syn.blob_camera(64, 64)
    target = _t(np.random.default_rng(2).uniform(0, 1, (1, 3, 64, 64)))
    a = cs.SceneTensors.from_numpy(raw, _dev())
    b = cs.SceneTensors.from_numpy(raw, _dev())
    tr = cs.Trainer(a)
    loss = tr.step([cam], target)
    img, _, st = cs.forward(b, [cam], keep_state=True)
    l2, dL = cs.loss_l1_dssim(img, target, 0.2)
    grads = {k: torch.zeros_like(getattr(b, k)) for k in cs.PARAMS}
    cs.backward(st, dL, grads)
    st.release()
    c = cs.TrainConfig()
    lr = dict(points=c.points_lr(1), delta=c.lr_delta, sigma=c.lr_sigma, opacity=c.lr_opacity, sh=c.lr_sh)
    groups = [dict(param=getattr(b, k), grad=grads[k], m=torch.zeros_like(grads[k]), v=torch.zeros_like(grads[k]),
                   lr=lr[k]) for k in cs.PARAMS]
    cs.adam_step(groups, 1, c.beta1, c.beta2, c.eps, zero_grad=False)
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - float(l2.item())) <= 1e-6 * float(l2.item())
    for k in cs.PARAMS:
        gb = grads[k].cpu().numpy().astype(np.float64)
        ga = tr.m[k].cpu().numpy().astype(np.float64) / (1.0 - c.beta1)
        big = np.abs(gb).max()
        np.testing.assert_allclose(ga, gb, rtol=1e-4, atol=1e-5 * big)
        well = np.abs(gb) > 1e-3 * big
        np.testing.assert_allclose(getattr(a, k).cpu().numpy()[well], getattr(b, k).cpu().numpy()[well], rtol=0,
                                   atol=1e-6)
        assert (tr.grads[k] == 0).all()
    # the loss of the step is the oracle's loss of the oracle's image of the same parameters
    ref = oracle.render_image(oracle.activate(raw), cam, oracle.settings())
    L_ref, _ = OT.loss_l1_dssim(ref["image"][None], target.cpu().numpy().astype(np.float64), 0.2)
    assert abs(float(loss.item()) - L_ref) <= 1e-3 * L_ref


def test_trainer_fits_a_perturbed_scene():
    """Optimising raw parameters toward the render of a slightly different scene lowers the loss."""
    import torch
    import paper_2411_14974_gb300 as cs
    raw = _raw_blob(3)
    cam = syn.blob_camera(96, 96)
    goal = raw.copy()
    goal.sh[:, 0, :] += np.random.default_rng(4).normal(0, 0.3, goal.sh[:, 0, :].shape).astype(np.float32)
    target, _, _ = cs.forward(cs.SceneTensors.from_numpy(goal, _dev()), [cam])
    scene = cs.SceneTensors.from_numpy(raw, _dev())
    tr = cs.Trainer(scene, config=cs.TrainConfig(lr_sh=0.01))
    losses = [float(tr.step([cam], target).item()) for _ in range(40)]
    assert losses[-1] < 0.6 * losses[0], losses[::8]
    assert float(tr.sigma_grad_abs.sum().item()) > 0
