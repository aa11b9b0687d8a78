"""GPU backward parity, through the C ABI: the hand-written adjoint (reverse compositing that
recomputes the transmittance, warp-reduced atomics, chain to points/delta/sigma/opacity/SH)
against (1) the oracle's analytic binary64 gradient and (2) binary64 central finite differences
of the oracle's forward on sampled parameters.

Tolerance: 1e-3 relative per element, with an absolute floor of 1e-4 x the largest oracle
gradient of that tensor (FP32 accumulation of many cancelling terms).  The oracle builds the hull
lines from the binary32 projected points the hull was decided on; elements whose oracle gradient
moves by more than half of the tolerance when every line value is moved by the binary32
evaluation error model (two seeded sign patterns) are ill-conditioned and excluded (counted, at
most 1%).  tests/test_oracle_conditioning.py checks that rule against the binary32 record-form
line evaluation.
"""
import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests._parity import GRAD_FLOOR as FLOOR
from tests._parity import GRAD_MAX_EXCLUDED, gradient_ill, oracle_settings
from tests._parity import GRAD_REL as REL

pytestmark = pytest.mark.gpu

FIELDS = ("points", "delta", "sigma", "opacity", "sh")


def gpu_grads(sc, cams, G, **kw):
    import torch
    import paper_2411_14974_gb300 as cs
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    img, _, state = cs.forward(t, cams, cs.Settings(**kw), keep_state=True)
    g = cs.backward(state, torch.as_tensor(np.ascontiguousarray(G, np.float32), device=dev))
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    state.release()
    return out, img.cpu().numpy()


def compare(got, ref, refs_perturbed, max_excluded=GRAD_MAX_EXCLUDED):
    report = {}
    for f in FIELDS:
        a, b = got[f].ravel(), ref[f].ravel()
        if b.size == 0:
            continue
        scale = np.abs(b).max()
        tol = REL * np.abs(b) + FLOOR * scale
        ill = gradient_ill(b, [rp[f].ravel() for rp in refs_perturbed], tol)
        bad = (np.abs(a - b) > tol) & ~ill
        nz = np.abs(b) > FLOOR * scale
        report[f] = dict(excluded=float(ill[nz].mean()) if nz.any() else 0.0, bad=int(bad.sum()),
                         worst=float((np.abs(a - b) / np.maximum(tol, 1e-30))[~ill].max()) if (~ill).any() else 0.0)
        assert not bad.any(), (f, report[f], np.nonzero(bad)[0][:10], a[bad][:5], b[bad][:5])
        assert report[f]["excluded"] <= max_excluded, (f, report[f])
    return report


def _blob(seed, n=300, deg=0, radius=0.08):
    sc = syn.blob_scene(seed, n=n, radius=radius, sh_degree=deg)
    sc.points[..., :2] *= 0.5
    return sc


@pytest.mark.parametrize("seed,deg", [(0, 0), (1, 3)])
def test_gradient_matches_oracle_blob(seed, deg):
    sc = _blob(seed, deg=deg)
    cam = syn.blob_camera(64, 64)
    G = np.random.default_rng(seed).uniform(-1, 1, (1, 3, 64, 64))
    st = oracle_settings()
    ref = oracle.backward_image(sc, cam, st, G[0])
    refp = [oracle.backward_image(sc, cam, st, G[0], perturb_seed=s) for s in (1, 2)]
    got, _ = gpu_grads(sc, [cam], G)
    compare(got, ref, refp)


@pytest.mark.parametrize("kw", [dict(dist_power=0.5), dict(dist_power=2.0), dict(dist_mode=1),
                                dict(bg=(0.3, 0.6, 0.9), tau=0.01, alpha_max=0.9)])
def test_gradient_settings_variants(kw):
    sc = _blob(2, deg=2)
    if kw.get("dist_power") == 2.0:
        sc.delta /= 4.0
        sc.sigma /= 4.0
    cam = syn.blob_camera(48, 40)
    G = np.random.default_rng(5).uniform(-1, 1, (1, 3, 40, 48))
    st = oracle_settings(**kw)
    ref = oracle.backward_image(sc, cam, st, G[0])
    refp = [oracle.backward_image(sc, cam, st, G[0], perturb_seed=s) for s in (1, 2)]
    got, _ = gpu_grads(sc, [cam], G, **kw)
    compare(got, ref, refp)


def test_gradient_raw_parameters():
    """With CS_ACT_EXP_SIGMOID the backward returns gradients w.r.t. log delta, log sigma and
    logit opacity: the oracle's activated-scene gradient times exp' = exp and sigmoid' = o (1 - o)."""
    raw = _blob(4, deg=1).as_raw()
    act = oracle.activate(raw)
    cam = syn.blob_camera(64, 64)
    G = np.random.default_rng(4).uniform(-1, 1, (1, 3, 64, 64))
    st = oracle_settings()
    ref = oracle.raw_gradients(raw, oracle.backward_image(act, cam, st, G[0]))
    refp = [oracle.raw_gradients(raw, oracle.backward_image(act, cam, st, G[0], perturb_seed=s)) for s in (1, 2)]
    got, _ = gpu_grads(raw, [cam], G)
    compare(got, ref, refp)


@pytest.mark.parametrize("deg", [2, 3])  # SH staged element by element / in 16-byte chunks
def test_gradient_16bit_storage(deg):
    """Float32 gradients of a float16-stored scene equal the oracle's on the widened values."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc = _blob(6, deg=deg)
    wide = sc.copy()
    for name in FIELDS:
        setattr(wide, name, np.ascontiguousarray(
            torch.as_tensor(getattr(sc, name)).to(torch.float16).to(torch.float32).numpy()))
    cam = syn.blob_camera(64, 64)
    G = np.random.default_rng(6).uniform(-1, 1, (1, 3, 64, 64))
    st = oracle_settings()
    ref = oracle.backward_image(wide, cam, st, G[0])
    refp = [oracle.backward_image(wide, cam, st, G[0], perturb_seed=s) for s in (1, 2)]
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev, dtype=torch.float16)
    _, _, state = cs.forward(t, [cam], cs.Settings(), keep_state=True)
    g = cs.backward(state, torch.as_tensor(np.ascontiguousarray(G, np.float32), device=dev))
    torch.cuda.synchronize()
    assert all(v.dtype == torch.float32 for v in g.values())
    compare({k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}, ref, refp)
    state.release()


def test_gradient_surface_sh3():
    sc = syn.surface_scene(21, n=20_000, sh_degree=3)
    cam = syn.sphere_cameras(1, 120, 96, 4.0, seed=22)[0]
    G = np.random.default_rng(23).uniform(-1, 1, (1, 3, 96, 120))
    st = oracle_settings()
    ref = oracle.backward_image(sc, cam, st, G[0])
    refp = [oracle.backward_image(sc, cam, st, G[0], perturb_seed=s) for s in (1, 2)]
    got, _ = gpu_grads(sc, [cam], G)
    compare(got, ref, refp)


def test_unaligned_sh_array():
    """SH coefficients at an address that is not 16-byte aligned (staged element by element instead
    of in 16-byte chunks): the same image bit for bit, and the same gradients up to the order of
    the blend backward's atomic additions."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc = syn.surface_scene(27, n=6_000, sh_degree=3)
    cam = syn.sphere_cameras(1, 128, 96, 4.0, seed=28)[0]
    dev = torch.device("cuda:0")
    G = torch.as_tensor(np.random.default_rng(29).uniform(-1, 1, (1, 3, 96, 128)).astype(np.float32), device=dev)
    t = cs.SceneTensors.from_numpy(sc, dev)
    buf = torch.empty(t.sh.numel() + 1, dtype=torch.float32, device=dev)
    shifted = buf[1:].view(t.sh.shape)
    shifted.copy_(t.sh)
    assert shifted.data_ptr() % 16 != 0
    u = cs.SceneTensors(t.points, t.delta, t.sigma, t.opacity, shifted)
    out = []
    for scene in (t, u):
        img, tf, state = cs.forward(scene, [cam], cs.Settings(), keep_state=True)
        g = cs.backward(state, G)
        torch.cuda.synchronize()
        out.append((img.clone(), tf.clone(), {k: v.clone() for k, v in g.items()}))
        state.release()
    (ia, ta, ga), (ib, tb, gb) = out
    assert torch.equal(ia, ib) and torch.equal(ta, tb)
    for f in FIELDS:
        scale = float(ga[f].abs().max()) + 1e-30
        assert float((ga[f] - gb[f]).abs().max()) <= 1e-5 * scale, f


def test_multi_view_gradient_is_sum_of_views():
    sc = syn.surface_scene(24, n=5_000, sh_degree=1)
    cams = syn.sphere_cameras(3, 64, 48, 4.0, seed=25)
    G = np.random.default_rng(26).uniform(-1, 1, (3, 3, 48, 64))
    got, _ = gpu_grads(sc, cams, G)
    acc = None
    for v, cam in enumerate(cams):
        one, _ = gpu_grads(sc, [cam], G[v:v + 1])
        acc = one if acc is None else {k: acc[k] + one[k] for k in acc}
    for f in FIELDS:
        scale = np.abs(acc[f]).max() + 1e-30
        assert np.abs(got[f] - acc[f]).max() <= 1e-5 * scale, f


def test_gradient_against_finite_differences():
    """64 sampled parameters of visible convexes: GPU gradient vs binary64 central differences of
    the oracle forward (steps h and h/2 must agree; discrete structure unchanged across the step)."""
    sc = _blob(3, n=120, deg=3, radius=0.1)
    cam = syn.blob_camera(48, 48)
    G = np.random.default_rng(7).uniform(-1, 1, (1, 3, 48, 48))
    got, _ = gpu_grads(sc, [cam], G)
    st = oracle.settings()  # smooth binary64 projection: finite differences need no quantised vertices
    disc = oracle.discrete(sc, cam, st)
    vis = np.nonzero(disc["visible"])[0]
    rng = np.random.default_rng(8)

    def loss(s):
        r = oracle.render_image(s, cam, st)
        return float((r["image"] * G[0]).sum()), r["n_contrib"], r["last_id"]

    def fd(field, idx, h):
        vals, structs = [], []
        for sgn in (1, -1):
            p = sc.copy()
            arr = getattr(p, field)
            arr[idx] = np.float32(arr[idx] + sgn * h)
            L, nc, last = loss(p)
            vals.append((L, float(arr[idx]) - float(getattr(sc, field)[idx])))
            structs.append((nc, last))
        same = (structs[0][0] == structs[1][0]).all() and (structs[0][1] == structs[1][1]).all()
        return (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1]), same

    checked = 0
    for _ in range(64):
        i = int(rng.choice(vis))
        field = ["points", "delta", "sigma", "opacity", "sh"][rng.integers(5)]
        if field == "points":
            idx, h = (i, int(rng.integers(sc.k)), int(rng.integers(3))), 1e-4
        elif field == "sh":
            idx, h = (i, int(rng.integers(sc.sh.shape[1])), int(rng.integers(3))), 1e-3
        elif field == "opacity":
            idx, h = (i,), 1e-3
        else:
            idx, h = (i,), 1e-3 * float(getattr(sc, field)[i])
        d1, s1 = fd(field, idx, h)
        d2, s2 = fd(field, idx, h / 2)
        if not (s1 and s2):
            continue
        scale = max(abs(d2), 1e-6)
        if abs(d1 - d2) > 0.05 * scale:
            continue
        rich = (4 * d2 - d1) / 3
        a = float(got[field][idx])
        gmax = np.abs(got[field]).max()
        assert abs(a - rich) <= REL * abs(rich) + FLOOR * gmax + 0.05 * abs(d1 - d2), (field, idx, a, rich, d1, d2)
        checked += 1
    assert checked >= 40


def test_autograd_render_matches_direct_backward_after_buffers_are_freed():
    """torch.autograd path (render -> loss.backward) equals the direct C-ABI backward, even when the
    forward's image / T_final tensors are released and their memory reused before the backward."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc = _blob(4, deg=1)
    cam = syn.blob_camera(64, 48)
    G = np.random.default_rng(9).uniform(-1, 1, (1, 3, 48, 64))
    want, _ = gpu_grads(sc, [cam], G)
    t = cs.SceneTensors.from_numpy(sc, torch.device("cuda:0"))
    params = [getattr(t, f).clone().requires_grad_(True) for f in FIELDS]
    img = cs.render(*params, [cam])
    loss = (img * torch.as_tensor(G, dtype=torch.float32, device="cuda:0")).sum()
    junk = [torch.full((1 << 20,), float("nan"), device="cuda:0") for _ in range(8)]  # reuse freed memory
    loss.backward()
    del junk
    for f, p in zip(FIELDS, params):
        got = p.grad.detach().cpu().numpy().astype(np.float64)
        scale = np.abs(want[f]).max() + 1e-30
        assert np.abs(got - want[f]).max() <= 1e-5 * scale, f


@pytest.mark.parametrize("n_views, offset", [(1, 0), (2, 0), (1, 1), (2, 3)])
def test_backward_write_equals_accumulate_into_zeros(n_views, offset):
    """cs_backward_write writes the gradients (buffers full of NaN beforehand) and equals
    cs_backward accumulating into zeroed buffers, up to the order of the blend's atomics; with the
    buffers `offset` floats into larger ones (4-byte but not 16-byte aligned), the 16-byte
    write-out and the clears of several views write exactly the buffers (the floats around them
    stay NaN)."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc = syn.surface_scene(61, n=8_000, sh_degree=3)
    cams = syn.sphere_cameras(n_views, 96, 72, 4.0, seed=62)
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    G = torch.as_tensor(np.random.default_rng(63).uniform(-1, 1, (n_views, 3, 72, 96)).astype(np.float32), device=dev)
    _, _, state = cs.forward(t, cams, cs.Settings(), keep_state=True)
    acc = cs.backward(state, G)
    bases = {f: torch.full((getattr(t, f).numel() + offset + 5,), float("nan"), device=dev) for f in FIELDS}
    junk = {f: bases[f][offset:offset + getattr(t, f).numel()].view(tuple(getattr(t, f).shape)) for f in FIELDS}
    wrote = cs.backward(state, G, junk, accumulate=False)
    torch.cuda.synchronize()
    state.release()
    for f in FIELDS:
        a, w = acc[f].cpu().numpy(), wrote[f].cpu().numpy()
        assert np.isfinite(w).all(), f
        assert np.abs(a - w).max() <= 1e-5 * (np.abs(a).max() + 1e-30), f
        around = torch.cat([bases[f][:offset], bases[f][offset + getattr(t, f).numel():]])
        assert torch.isnan(around).all(), f


@pytest.mark.parametrize("pinned,n_views", [(True, 1), (False, 1), (True, 2)])
def test_step_through_host_buffers_equals_device_calls(pinned, n_views):
    """cs_step_host (scene, dL/dimage, image and gradients in host memory; the gradients, image
    and cotangent read and written in place where the GPU can reach them) gives the image of
    cs_forward bit for bit and the gradients of cs_backward up to the order of the atomics."""
    import torch
    import paper_2411_14974_gb300 as cs
    sc = syn.surface_scene(64, n=6_000, sh_degree=2)
    cams = syn.sphere_cameras(n_views, 80, 64, 4.0, seed=65)
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    G = np.random.default_rng(66).uniform(-1, 1, (n_views, 3, 64, 80)).astype(np.float32)
    img, _, state = cs.forward(t, cams, cs.Settings(), keep_state=True)
    want = cs.backward(state, torch.as_tensor(G, device=dev))
    torch.cuda.synchronize()
    state.release()
    host = lambda a: (torch.as_tensor(np.ascontiguousarray(a, np.float32)).pin_memory() if pinned
                      else torch.as_tensor(np.ascontiguousarray(a, np.float32)))
    scene_h = dict(points=host(sc.points), delta=host(sc.delta), sigma=host(sc.sigma), opacity=host(sc.opacity),
                   sh=host(sc.sh))
    img_h = host(np.full((n_views, 3, 64, 80), np.nan))
    g_h = {f: host(np.full(tuple(getattr(t, f).shape), np.nan)) for f in FIELDS}
    cs.step_host(scene_h, sc.sh_degree, cams, cs.Settings(), host(G), img_h, g_h)
    torch.cuda.synchronize()
    assert torch.equal(img_h, img.cpu())
    for f in FIELDS:
        a, b = g_h[f].numpy(), want[f].cpu().numpy()
        assert np.isfinite(a).all(), f
        assert np.abs(a - b).max() <= 1e-5 * (np.abs(b).max() + 1e-30), f


@pytest.mark.parametrize("pinned", [True, False])
def test_pipelined_host_steps_equal_device_calls(pinned):
    """cs_step_host_submit / cs_step_host_wait: seven steps submitted back to back over three
    views (inputs copied in and outputs copied out while other steps compute, the three slots each
    reused) give, step by step, the image of cs_forward bit for bit and the gradients of
    cs_backward up to the order of the atomics, from pinned or pageable host memory; a ticket that
    was never submitted is rejected; a step that fails in the worker thread (a backward with
    alpha_max above 0.999) is reported, with its message, by the next wait, once, and the steps
    after it still run."""
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    sc = syn.surface_scene(67, n=6_000, sh_degree=2)
    cams = syn.sphere_cameras(3, 80, 64, 4.0, seed=68)
    dev = torch.device("cuda:0")
    t = cs.SceneTensors.from_numpy(sc, dev)
    G = np.random.default_rng(69).uniform(-1, 1, (3, 1, 3, 64, 80)).astype(np.float32)
    pin = lambda a: (torch.as_tensor(np.ascontiguousarray(a, np.float32)).pin_memory() if pinned
                     else torch.as_tensor(np.ascontiguousarray(a, np.float32)))
    scene_h = dict(points=pin(sc.points), delta=pin(sc.delta), sigma=pin(sc.sigma), opacity=pin(sc.opacity),
                   sh=pin(sc.sh))
    n_steps = 7
    imgs = [pin(np.full((1, 3, 64, 80), np.nan)) for _ in range(n_steps)]
    gs = [{f: pin(np.full(tuple(getattr(t, f).shape), np.nan)) for f in FIELDS} for _ in range(n_steps)]
    dls = [pin(G[v]) for v in range(3)]
    tickets = [cs.step_host_submit(scene_h, sc.sh_degree, cams[i % 3], cs.Settings(), dls[i % 3], imgs[i], gs[i])
               for i in range(n_steps)]
    assert tickets == sorted(tickets) and len(set(tickets)) == n_steps
    cs.step_host_wait(tickets[-1])
    wants = []
    for v, cam in enumerate(cams):
        img, _, state = cs.forward(t, [cam], cs.Settings(), keep_state=True)
        want = cs.backward(state, torch.as_tensor(G[v], device=dev))
        torch.cuda.synchronize()
        state.release()
        wants.append((img.cpu(), {f: want[f].cpu().numpy() for f in FIELDS}))
    for i in range(n_steps):
        img, want = wants[i % 3]
        assert torch.equal(imgs[i], img), i
        for f in FIELDS:
            a, b = gs[i][f].numpy(), want[f]
            assert np.isfinite(a).all(), (i, f)
            assert np.abs(a - b).max() <= 1e-5 * (np.abs(b).max() + 1e-30), (i, f)
    with pytest.raises(B.CsError):
        cs.step_host_wait(tickets[-1] + 100)
    # a queued step whose backward is refused: the wait reports it once, later steps still run
    bad = cs.Settings(alpha_max=0.9999)
    cs.step_host_submit(scene_h, sc.sh_degree, cams[0], bad, dls[0], imgs[0], gs[0])
    imgs[1].fill_(float("nan"))
    tk = cs.step_host_submit(scene_h, sc.sh_degree, cams[1], cs.Settings(), dls[1], imgs[1], gs[1])
    with pytest.raises(B.CsError, match="alpha_max"):
        cs.step_host_wait(tk)
    cs.step_host_wait(tk)
    assert torch.equal(imgs[1], wants[1][0])
