"""GPU parity of the adaptive refinement (Sec. 3.3, supplement Sec. A) through cs_refine: every
split / prune decision, the output count and every output value (kept parameters and moments,
children's points, raw sigma and raw opacity) equal the oracle's bit for bit, since both sides
evaluate the same binary32 expressions in the same order.
"""
import ctypes

import numpy as np
import pytest

from oracle import train as OT
from paper_2411_14974_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

FIELDS = ("points", "delta", "sigma", "opacity", "sh")


def _case(n, k, deg, seed):
    rng = np.random.default_rng(seed)
    r = syn.blob_scene(seed, n=n, k=k, sh_degree=deg).as_raw()
    P = dict(points=r.points, delta=r.delta, sigma=r.sigma, opacity=r.opacity, sh=r.sh)
    P["opacity"][rng.random(n) < 0.1] = -6.0                      # ~10% fall below the opacity bound
    P["points"][rng.integers(n, size=3), 0, 1] = np.nan            # non-finite points prune
    big = rng.integers(n, size=max(1, n // 50))                  # ~2% blown up 20x about their centre
    c = P["points"][big].mean(axis=1, keepdims=True)
    P["points"][big] = (c + 20.0 * (P["points"][big] - c)).astype(np.float32)
    M = {f: rng.normal(size=P[f].shape).astype(np.float32) for f in FIELDS}
    V = {f: rng.uniform(0, 1, P[f].shape).astype(np.float32) for f in FIELDS}
    stat = rng.uniform(0, 8e-5, n).astype(np.float32)               # window 10: about half split
    return P, M, V, stat


def _gpu(P, M, V, stat, window, **kw):
    import torch
    import paper_2411_14974_gb300 as cs
    dev = torch.device("cuda:0")
    t = lambda d: {f: torch.as_tensor(np.ascontiguousarray(d[f]), device=dev) for f in FIELDS}
    out, om, ov, dec = cs.refine(t(P), torch.as_tensor(stat, device=dev), window, cs.RefineSettings(**kw), t(M),
                                 t(V), decisions=True)
    torch.cuda.synchronize()
    h = lambda d: {f: d[f].cpu().numpy() for f in FIELDS}
    return h(out), h(om), h(ov), dec.cpu().numpy()


@pytest.mark.parametrize("n,k,deg,seed", [(5000, 6, 3, 0), (777, 3, 0, 1), (2049, 8, 1, 2)])
def test_refine_matches_oracle_bit_for_bit(n, k, deg, seed):
    P, M, V, stat = _case(n, k, deg, seed)
    kw = dict(split_threshold=4e-6, split_scale=0.7, split_sigma_scale=1.5, split_opacity_scale=0.5,
              prune_opacity=0.03, prune_size=0.12)
    ref, rm, rv, rdec = OT.densify(P, M, V, stat, 10, threshold=kw["split_threshold"], split_scale=kw["split_scale"],
                                   split_sigma_scale=kw["split_sigma_scale"],
                                   split_opacity_scale=kw["split_opacity_scale"], prune_opacity=kw["prune_opacity"],
                                   prune_size=kw["prune_size"])
    out, om, ov, dec = _gpu(P, M, V, stat, 10, **kw)
    assert (rdec == 0).any() and (rdec == 1).any() and (rdec == 2).any()
    np.testing.assert_array_equal(dec, rdec)
    for f in FIELDS:
        np.testing.assert_array_equal(out[f], ref[f], err_msg=f)
        np.testing.assert_array_equal(om[f], rm[f], err_msg=f)
        np.testing.assert_array_equal(ov[f], rv[f], err_msg=f)


def test_refine_reports_capacity():
    import torch
    import paper_2411_14974_gb300 as cs
    from paper_2411_14974_gb300 import _binding as B
    P, M, V, stat = _case(300, 6, 0, 3)
    dev = torch.device("cuda:0")
    t = {f: torch.as_tensor(np.ascontiguousarray(P[f]), device=dev) for f in FIELDS}
    small = {f: torch.empty((10,) + tuple(t[f].shape[1:]), device=dev) for f in FIELDS}
    n_out = ctypes.c_int64()
    st = cs.RefineSettings().struct()
    a_in, a_out = cs.rasterizer._param_arrays(t), cs.rasterizer._param_arrays(small)
    s = torch.as_tensor(stat, device=dev)
    code = B.lib().cs_refine(cs.Context.get(0).handle, 300, 6, 0, ctypes.byref(a_in), None, None, s.data_ptr(), 10,
                             ctypes.byref(st), 10, ctypes.byref(a_out), None, None, None, ctypes.byref(n_out),
                             torch.cuda.current_stream().cuda_stream)
    assert code == 4  # CS_ERR_BUDGET
    ref_dec = OT.densify_decisions(P["points"], P["opacity"], stat, 10)
    assert n_out.value == int((ref_dec == 0).sum() + 6 * (ref_dec == 1).sum()) > 10


def test_trainer_refines_then_keeps_training():
    import torch
    import paper_2411_14974_gb300 as cs
    raw = syn.blob_scene(5, n=400, radius=0.08, sh_degree=1)
    raw.points[..., :2] *= 0.5
    raw = raw.as_raw()
    cam = syn.blob_camera(64, 64)
    target = torch.as_tensor(np.random.default_rng(6).uniform(0, 1, (1, 3, 64, 64)).astype(np.float32),
                             device="cuda:0")
    tr = cs.Trainer(cs.SceneTensors.from_numpy(raw, "cuda:0"))
    for _ in range(5):
        tr.step([cam], target)
    thr = float(torch.quantile(tr.sigma_grad_abs / 5, 0.8))
    dec = tr.refine(cs.RefineSettings(split_threshold=thr)).cpu().numpy()
    assert set(np.unique(dec)) <= {0, 1, 2} and (dec == 1).any()
    n_new = int((dec == 0).sum() + 6 * (dec == 1).sum())
    assert tr.scene.points.shape[0] == n_new and tr.m["sh"].shape[0] == n_new
    assert float(tr.sigma_grad_abs.abs().sum()) == 0.0
    loss = tr.step([cam], target)
    assert np.isfinite(float(loss.item()))
