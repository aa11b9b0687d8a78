"""Python face of the C ABI: forward/backward calls, the autograd Function and state access.

Only argument marshalling happens here; every step of the rasterizer runs in the CUDA library.
PyTorch provides device memory (tensors) and the current stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import threading
from typing import Optional, Sequence

import numpy as np
import torch

from . import _binding as B

ARRAYS = dict(records=0, depth_keys=1, rects=2, counts=3, pair_keys=4, pair_values=5, tile_ranges=6,
              n_last=7, hulls=8, tile_order=9)
_ARRAY_DTYPES = dict(records=np.float32, depth_keys=np.uint32, rects=np.uint32, counts=np.uint32,
                     pair_keys=np.uint32, pair_values=np.uint32, tile_ranges=np.uint32, n_last=np.uint32,
                     hulls=np.uint32, tile_order=np.uint32)


@dataclasses.dataclass
class Settings:
    """Compositing constants (3DGS-style cut-offs; Eq. 5 has none) and the distance scaling."""
    tau: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    dist_mode: int = 0
    dist_power: float = 1.0
    tile_test: int = 0  # 1: exact tile test against the offset hull (tighter binning)
    tile_split: int = 0  # N > 0: tiles with more than N pairs blended as chunks of N, then merged

    def struct(self) -> B.CsSettings:
        s = B.CsSettings()
        s.tau, s.alpha_max, s.t_min = float(self.tau), float(self.alpha_max), float(self.t_min)
        for i in range(3):
            s.bg[i] = float(self.bg[i])
        s.dist_mode, s.dist_power = int(self.dist_mode), float(self.dist_power)
        s.tile_test = int(self.tile_test)
        s.tile_split = int(self.tile_split)
        return s


def camera_struct(cam) -> B.CsCamera:
    c = B.CsCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.z_near = float(getattr(cam, "z_near", 0.2))
    return c


def cameras_array(cams: Sequence) -> ctypes.Array:
    arr = (B.CsCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


class Context:
    """Library context on one device (owns the stream-ordered memory pool of transient buffers and
    the forward's readback slot).  Calls on one context must not overlap, and ctypes releases the
    interpreter lock during a call, so `get` gives each host thread its own context, kept in the
    thread's local storage: it is released when the thread ends and nothing else (a forward
    state) still refers to it."""
    _local = threading.local()

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        B.check(B.lib().cs_context_create(int(device), ctypes.byref(h)), "cs_context_create")
        self.handle = h
        self.device = int(device)

    @classmethod
    def get(cls, device: int = 0) -> "Context":
        by_device = getattr(cls._local, "by_device", None)
        if by_device is None:
            by_device = cls._local.by_device = {}
        if int(device) not in by_device:
            by_device[int(device)] = Context(device)
        return by_device[int(device)]

    def __del__(self):
        try:
            if self.handle:
                B.lib().cs_context_destroy(self.handle)
        except Exception:
            pass


_STORAGE = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}


@dataclasses.dataclass
class SceneTensors:
    """Device tensors of a scene (float32, contiguous, on one CUDA device)."""
    points: torch.Tensor   # [N][K][3]
    delta: torch.Tensor    # [N]
    sigma: torch.Tensor    # [N]
    opacity: torch.Tensor  # [N]
    sh: torch.Tensor       # [N][(D+1)^2][3]
    raw: bool = False      # delta, sigma, opacity hold log, log, logit (activated inside the forward)

    @property
    def sh_degree(self) -> int:
        nb = int(self.sh.shape[1])
        d = int(round(nb ** 0.5)) - 1
        if (d + 1) ** 2 != nb:
            raise ValueError("sh must be [N][(D+1)^2][3]")
        return d

    @property
    def storage(self) -> int:
        """cs_storage of the parameter tensors (all five share one dtype)."""
        dt = self.points.dtype
        if any(getattr(self, n).dtype != dt for n in ("delta", "sigma", "opacity", "sh")):
            raise ValueError("points, delta, sigma, opacity and sh must share one dtype")
        if dt not in _STORAGE:
            raise ValueError("parameters must be float32, float16 or bfloat16")
        return _STORAGE[dt]

    def struct(self) -> B.CsScene:
        s = B.CsScene()
        storage = self.storage
        for name in ("points", "delta", "sigma", "opacity", "sh"):
            t = getattr(self, name)
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA tensor")
            setattr(s, name, t.data_ptr() if t.numel() else None)
        s.n = int(self.points.shape[0])
        s.k = int(self.points.shape[1])
        s.sh_degree = self.sh_degree
        s.activation = 1 if self.raw else 0
        s.storage = storage
        return s

    @staticmethod
    def from_numpy(scene, device="cuda", dtype=torch.float32) -> "SceneTensors":
        """dtype float16 / bfloat16 stores the parameters in 16 bits (the paper's light model)."""
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device).to(dtype)
        return SceneTensors(f(scene.points), f(scene.delta), f(scene.sigma), f(scene.opacity), f(scene.sh),
                            bool(getattr(scene, "raw", False)))


class State:
    """What a forward keeps for its backward (sorted tile lists, screen records, T_final, ...)."""

    def __init__(self, handle: ctypes.c_void_p, ctx: Context, scene: SceneTensors, n_views: int, hw):
        self.handle = handle
        self.ctx = ctx
        self.scene = scene  # keeps the parameter buffers alive until the backward
        self.n_views = n_views
        self.hw = hw

    def release(self):
        if self.handle:
            B.lib().cs_state_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def sizes(self):
        r, p, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        B.check(B.lib().cs_state_sizes(self.handle, ctypes.byref(r), ctypes.byref(p), ctypes.byref(t)),
                "cs_state_sizes")
        return dict(records=r.value, pairs=p.value, tiles=t.value)

    def array(self, name: str) -> np.ndarray:
        which = ARRAYS[name]
        n = ctypes.c_size_t()
        B.check(B.lib().cs_state_copy(self.handle, which, None, 0, ctypes.byref(n)), "cs_state_copy")
        out = np.empty(n.value // 4, _ARRAY_DTYPES[name])
        if n.value:
            B.check(B.lib().cs_state_copy(self.handle, which, out.ctypes.data_as(ctypes.c_void_p), n.value,
                                          ctypes.byref(n)), "cs_state_copy")
        return out


def _stream_ptr(device) -> Optional[int]:
    return torch.cuda.current_stream(device).cuda_stream


def forward(scene: SceneTensors, cams: Sequence, settings: Optional[Settings] = None, keep_state: bool = False,
            image: Optional[torch.Tensor] = None, t_final: Optional[torch.Tensor] = None):
    """cs_forward: render ``scene`` into len(cams) equal-size views.

    Returns (image [V][3][H][W], t_final [V][H][W], state or None)."""
    settings = settings or Settings()
    dev = scene.points.device
    ctx = Context.get(dev.index if dev.index is not None else torch.cuda.current_device())
    V = len(cams)
    H, W = int(cams[0].height), int(cams[0].width)
    if image is None:
        image = torch.empty((V, 3, H, W), device=dev, dtype=torch.float32)
    if t_final is None:
        t_final = torch.empty((V, H, W), device=dev, dtype=torch.float32)
    st_handle = ctypes.c_void_p()
    sc = scene.struct()
    cams_arr = cameras_array(cams)
    s = settings.struct()
    code = B.lib().cs_forward(ctx.handle, ctypes.byref(sc), cams_arr, V, ctypes.byref(s), image.data_ptr(),
                              t_final.data_ptr(), ctypes.byref(st_handle) if keep_state else None,
                              _stream_ptr(dev))
    B.check(code, "cs_forward")
    state = State(st_handle, ctx, scene, V, (H, W)) if keep_state else None
    return image, t_final, state


def backward(state: State, dL_dimage: torch.Tensor, grads: Optional[dict] = None, accumulate: bool = True) -> dict:
    """cs_backward: accumulate d(loss)/d(points, delta, sigma, opacity, sh) into ``grads``
    (zero tensors are created when not given); accumulate=False writes them instead
    (cs_backward_write: the buffers' contents are not read)."""
    sc = state.scene
    if grads is None:  # gradients are float32 whatever the parameter storage
        z = lambda t: torch.zeros(t.shape, dtype=torch.float32, device=t.device)
        grads = dict(points=z(sc.points), delta=z(sc.delta), sigma=z(sc.sigma), opacity=z(sc.opacity), sh=z(sc.sh))
    g = dL_dimage.contiguous()
    if g.dtype != torch.float32:
        g = g.float()
    ptr = lambda t: t.data_ptr() if (t is not None and t.numel()) else None
    fn = B.lib().cs_backward if accumulate else B.lib().cs_backward_write
    code = fn(state.ctx.handle, state.handle, g.data_ptr(), ptr(grads.get("points")), ptr(grads.get("delta")),
              ptr(grads.get("sigma")), ptr(grads.get("opacity")), ptr(grads.get("sh")), _stream_ptr(sc.points.device))
    B.check(code, "cs_backward" if accumulate else "cs_backward_write")
    return grads


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, delta, sigma, opacity, sh, cams, settings, raw):
        scene = SceneTensors(points.detach().contiguous(), delta.detach().contiguous(), sigma.detach().contiguous(),
                             opacity.detach().contiguous(), sh.detach().contiguous(), raw)
        need = any(ctx.needs_input_grad[:5])
        image, _, state = forward(scene, cams, settings, keep_state=need)
        ctx.state = state
        return image

    @staticmethod
    def backward(ctx, dL_dimage):
        state = ctx.state
        g = backward(state, dL_dimage)
        sc = state.scene
        state.release()
        ctx.state = None
        out = [g[k].to(getattr(sc, k).dtype) for k in PARAMS]  # float32 gradients, in each input's dtype
        return (*out, None, None, None)


def render(points, delta, sigma, opacity, sh, cams, settings: Optional[Settings] = None,
           raw: bool = False) -> torch.Tensor:
    """Differentiable render (Sec. 3.2, Eq. 4, 5, S1, S2): image [V][3][H][W] for len(cams) views.

    delta, sigma, opacity are activated values (> 0, > 0, in (0, 1]), or with raw=True the
    training parameters log delta, log sigma, logit opacity (Sec. 3.3), activated in the forward."""
    return _Render.apply(points, delta, sigma, opacity, sh, list(cams), settings or Settings(), bool(raw))


# ---- training step (Sec. 3.3) -------------------------------------------------------------------
PARAMS = ("points", "delta", "sigma", "opacity", "sh")


def _ctx_of(t: torch.Tensor) -> Context:
    return Context.get(t.device.index if t.device.index is not None else torch.cuda.current_device())


def loss_l1_dssim(image: torch.Tensor, target: torch.Tensor, lam: float = 0.2, grad: bool = True,
                  loss_out: Optional[torch.Tensor] = None, dL_dimage: Optional[torch.Tensor] = None):
    """cs_loss_l1_dssim: (1 - lam) L1 + lam D-SSIM of images [V][3][H][W] (Eq. 6 without the mask
    term).  Returns (loss as a one-element device tensor, dL/dimage or None)."""
    if image.shape != target.shape or image.dim() != 4 or image.shape[1] != 3:
        raise ValueError("image and target must both be [V][3][H][W]")
    for t in (image, target):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("image and target must be contiguous float32 CUDA tensors")
    V, _, H, W = image.shape
    if loss_out is None:
        loss_out = torch.empty(1, device=image.device, dtype=torch.float32)
    if grad and dL_dimage is None:
        dL_dimage = torch.empty_like(image)
    code = B.lib().cs_loss_l1_dssim(_ctx_of(image).handle, image.data_ptr(), target.data_ptr(), V, H, W, float(lam),
                                    loss_out.data_ptr(), dL_dimage.data_ptr() if grad else None,
                                    _stream_ptr(image.device))
    B.check(code, "cs_loss_l1_dssim")
    return loss_out, (dL_dimage if grad else None)


def adam_step(groups: Sequence[dict], step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15,
              zero_grad: bool = True):
    """cs_adam_step over groups of dict(param, grad, m, v, lr[, grad_abs_sum]) (float32 CUDA tensors
    of equal size), all in one launch."""
    if len(groups) > B.ADAM_MAX_GROUPS:
        raise ValueError(f"at most {B.ADAM_MAX_GROUPS} groups")
    arr = (B.CsAdamGroup * max(1, len(groups)))()
    dev = None
    for i, g in enumerate(groups):
        p = g["param"]
        dev = p.device
        for name in ("param", "grad", "m", "v", "grad_abs_sum"):
            t = g.get(name)
            if t is None:
                continue
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() != p.numel():
                raise ValueError(f"group {i}: {name} must be a contiguous float32 CUDA tensor like param")
            setattr(arr[i], name, t.data_ptr() if t.numel() else None)
        arr[i].n = p.numel()
        arr[i].lr = float(g["lr"])
    st = B.CsAdamSettings(float(beta1), float(beta2), float(eps), int(bool(zero_grad)))
    if dev is None:
        return
    code = B.lib().cs_adam_step(_ctx_of(groups[0]["param"]).handle, arr, len(groups), ctypes.byref(st), int(step),
                                _stream_ptr(dev))
    B.check(code, "cs_adam_step")


@dataclasses.dataclass
class RefineSettings:
    """Adaptive refinement settings (supplement Sec. A).  The paper gives the split threshold, the
    scale-down (0.7 indoor, 0.6 outdoor) and the opacity prune level; how much sigma rises and
    opacity falls for split children, and the size bound, are settings."""
    split_threshold: float = 4e-6
    split_scale: float = 0.7
    split_sigma_scale: float = 1.5
    split_opacity_scale: float = 0.5
    prune_opacity: float = 0.03
    prune_size: float = float("inf")

    def struct(self) -> B.CsRefineSettings:
        return B.CsRefineSettings(self.split_threshold, self.split_scale, self.split_sigma_scale,
                                  self.split_opacity_scale, self.prune_opacity, self.prune_size)


def _param_arrays(d: Optional[dict]):
    if d is None:
        return None
    a = B.CsParamArrays()
    for k in PARAMS:
        t = d[k]
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{k} must be a contiguous float32 CUDA tensor")
        setattr(a, k, t.data_ptr() if t.numel() else None)
    return a


def refine(params: dict, sigma_grad_abs: torch.Tensor, window_steps: int, settings: Optional[RefineSettings] = None,
           m: Optional[dict] = None, v: Optional[dict] = None, decisions: bool = False):
    """cs_refine: split / prune raw parameters (dict of PARAMS tensors) and their Adam moments.
    Returns (new params, new m or None, new v or None, decisions tensor or None)."""
    settings = settings or RefineSettings()
    pts = params["points"]
    n, k = int(pts.shape[0]), int(pts.shape[1])
    nb = int(params["sh"].shape[1])
    deg = int(round(nb ** 0.5)) - 1
    dev = pts.device
    cap = n * k
    alloc = lambda: {key: torch.empty((cap,) + tuple(params[key].shape[1:]), device=dev) for key in PARAMS}
    out, om, ov = alloc(), (alloc() if m is not None else None), (alloc() if m is not None else None)
    dec = torch.empty(n, dtype=torch.int32, device=dev) if decisions else None
    n_out = ctypes.c_int64()
    st = settings.struct()
    a_in, a_m, a_v = _param_arrays(params), _param_arrays(m), _param_arrays(v)
    a_out, a_om, a_ov = _param_arrays(out), _param_arrays(om), _param_arrays(ov)
    ref = lambda x: ctypes.byref(x) if x is not None else None
    code = B.lib().cs_refine(_ctx_of(pts).handle, n, k, deg, ref(a_in), ref(a_m), ref(a_v),
                             sigma_grad_abs.data_ptr() if n else None, int(window_steps), ctypes.byref(st), cap,
                             ref(a_out), ref(a_om), ref(a_ov), dec.data_ptr() if dec is not None else None,
                             ctypes.byref(n_out), _stream_ptr(dev))
    B.check(code, "cs_refine")
    cut = lambda d: None if d is None else {key: d[key][:n_out.value].contiguous() for key in PARAMS}
    return cut(out), cut(om), cut(ov), dec


@dataclasses.dataclass
class TrainConfig:
    """Optimiser settings of Sec. 3.3 and the supplementary hyper-parameters.  The paper gives the
    rates for delta, sigma and the points (5e-4 decaying exponentially to 5e-6); opacity and SH
    rates are not given and are settings here."""
    lr_points: float = 5e-4
    lr_points_final: float = 5e-6
    lr_decay_steps: int = 30_000
    lr_delta: float = 0.005
    lr_sigma: float = 0.0045
    lr_opacity: float = 0.025
    lr_sh: float = 0.0025
    lam: float = 0.2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15

    def points_lr(self, step: int) -> float:
        """Log-linear decay from lr_points at step 1 to lr_points_final at lr_decay_steps."""
        s = min(max(step - 1, 0) / max(self.lr_decay_steps - 1, 1), 1.0)
        return math.exp((1.0 - s) * math.log(self.lr_points) + s * math.log(self.lr_points_final))


class Trainer:
    """One optimisation step per call, all on the device: forward on the raw training parameters
    (activations inside the preprocess), L1 + D-SSIM loss against the target, backward into the
    raw-parameter gradients, then one fused Adam launch over the five parameter groups.  The
    sigma group also accumulates |dL/dsigma| per convex (the split statistic)."""

    def __init__(self, scene: SceneTensors, settings: Optional[Settings] = None, config: Optional[TrainConfig] = None):
        if not scene.raw:
            raise ValueError("Trainer optimises raw parameters: SceneTensors(raw=True)")
        if scene.storage != 0:
            raise ValueError("Trainer optimises float32 parameters (16-bit storage is for rendering)")
        self.scene = scene
        self.settings = settings or Settings()
        self.config = config or TrainConfig()
        self.grads = {k: torch.zeros_like(getattr(scene, k)) for k in PARAMS}
        self.m = {k: torch.zeros_like(getattr(scene, k)) for k in PARAMS}
        self.v = {k: torch.zeros_like(getattr(scene, k)) for k in PARAMS}
        self.sigma_grad_abs = torch.zeros_like(scene.sigma)
        self.step_count = 0
        self._last_refine = 0
        self._image = None
        self._dL = None
        self.loss = torch.zeros(1, device=scene.points.device)

    def groups(self, step: int) -> list:
        c = self.config
        lr = dict(points=c.points_lr(step), delta=c.lr_delta, sigma=c.lr_sigma, opacity=c.lr_opacity, sh=c.lr_sh)
        out = []
        for k in PARAMS:
            g = dict(param=getattr(self.scene, k), grad=self.grads[k], m=self.m[k], v=self.v[k], lr=lr[k])
            if k == "sigma":
                g["grad_abs_sum"] = self.sigma_grad_abs
            out.append(g)
        return out

    def refine(self, settings: Optional[RefineSettings] = None, window_steps: Optional[int] = None):
        """Split and prune (cs_refine) with the sigma statistic gathered since the last refinement;
        the scene, moments and gradients are replaced and the statistic restarts."""
        window = window_steps if window_steps is not None else max(self.step_count - self._last_refine, 1)
        params = {k: getattr(self.scene, k) for k in PARAMS}
        out, m, v, dec = refine(params, self.sigma_grad_abs, window, settings, self.m, self.v, decisions=True)
        for k in PARAMS:
            setattr(self.scene, k, out[k])
        self.m, self.v = m, v
        self.grads = {k: torch.zeros_like(out[k]) for k in PARAMS}
        self.sigma_grad_abs = torch.zeros_like(out["sigma"])
        self._last_refine = self.step_count
        return dec

    def step(self, cams: Sequence, target: torch.Tensor) -> torch.Tensor:
        """target: [V][3][H][W] float32 on the scene's device.  Returns the loss (device tensor)."""
        V = len(cams)
        H, W = int(cams[0].height), int(cams[0].width)
        if self._image is None or tuple(self._image.shape) != (V, 3, H, W):
            self._image = torch.empty((V, 3, H, W), device=self.scene.points.device)
            self._dL = torch.empty_like(self._image)
        _, _, st = forward(self.scene, cams, self.settings, keep_state=True, image=self._image)
        loss_l1_dssim(self._image, target, self.config.lam, True, self.loss, self._dL)
        backward(st, self._dL, self.grads)
        st.release()
        self.step_count += 1
        c = self.config
        adam_step(self.groups(self.step_count), self.step_count, c.beta1, c.beta2, c.eps, zero_grad=True)
        return self.loss


# ---- instrumentation and host-buffer entry points ---------------------------------------------
def profile_enable(on: bool = True, device: int = 0):
    """Bracket every stage of every call with CUDA events on the launching stream."""
    B.check(B.lib().cs_profile_enable(Context.get(device).handle, int(bool(on))), "cs_profile_enable")


def profile_read(device: int = 0) -> dict:
    """{stage: (total ms, timed launches)} since the last read."""
    n = len(B.STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    B.check(B.lib().cs_profile_read(Context.get(device).handle, ms, cnt), "cs_profile_read")
    return {name: (ms[i], cnt[i]) for i, name in enumerate(B.STAGES)}


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(B.lib().cs_kernel_launch_count())


def alu_rates(device: int = 0) -> dict:
    """Measured per-SM rates of the transcendental unit (ex2.approx results per clock) and the FP32
    pipe (fused multiply-adds per clock), the SM clock during the measurement and the SM count."""
    out = (ctypes.c_double * 4)()
    B.check(B.lib().cs_measure_alu_rates(int(device), out), "cs_measure_alu_rates")
    return dict(mufu_per_clk_sm=out[0], fma_per_clk_sm=out[1], sm_mhz=out[2], sms=int(out[3]))


WORK_FIELDS = ("visited", "lines_visited", "passed", "lines_passed", "contributing", "pixels")


def work_counts(state: State, dL_dimage: Optional[torch.Tensor] = None) -> dict:
    """Work done by the forward (and backward) blend of a state, from instrumented kernels."""
    out = (ctypes.c_uint64 * 12)()
    g = dL_dimage.contiguous() if dL_dimage is not None else None
    B.check(B.lib().cs_work_counts(state.ctx.handle, state.handle, g.data_ptr() if g is not None else None, out,
                                   _stream_ptr(state.scene.points.device)), "cs_work_counts")
    fwd = {k: int(out[i]) for i, k in enumerate(WORK_FIELDS)}
    bwd = {k: int(out[6 + i]) for i, k in enumerate(WORK_FIELDS)}
    return dict(forward=fwd, backward=bwd)


def step_host(scene_host: dict, sh_degree: int, cams: Sequence, settings: Optional[Settings], dL_host, image_host,
              grads_host: Optional[dict] = None, device: int = 0):
    """cs_step_host: one forward (+ backward when dL_host is given) with every buffer in host memory.

    scene_host: dict of contiguous float32 CPU tensors (points, delta, sigma, opacity, sh), ideally
    pinned; image_host / dL_host / grads_host likewise."""
    ctx = Context.get(device)
    sc = B.CsScene()
    for name in ("points", "delta", "sigma", "opacity", "sh"):
        t = scene_host[name]
        setattr(sc, name, t.data_ptr() if t.numel() else None)
    sc.n = int(scene_host["points"].shape[0])
    sc.k = int(scene_host["points"].shape[1])
    sc.sh_degree = int(sh_degree)
    sc.activation = 1 if scene_host.get("raw", False) else 0
    sc.storage = _STORAGE[scene_host["points"].dtype]
    s = (settings or Settings()).struct()
    g = grads_host or {}
    ptr = lambda t: t.data_ptr() if t is not None else None
    code = B.lib().cs_step_host(ctx.handle, ctypes.byref(sc), cameras_array(cams), len(cams), ctypes.byref(s),
                                ptr(dL_host), image_host.data_ptr(), ptr(g.get("points")), ptr(g.get("delta")),
                                ptr(g.get("sigma")), ptr(g.get("opacity")), ptr(g.get("sh")),
                                _stream_ptr(torch.device("cuda", device)))
    B.check(code, "cs_step_host")


def _host_scene_struct(scene_host: dict, sh_degree: int):
    sc = B.CsScene()
    for name in ("points", "delta", "sigma", "opacity", "sh"):
        t = scene_host[name]
        setattr(sc, name, t.data_ptr() if t.numel() else None)
    sc.n = int(scene_host["points"].shape[0])
    sc.k = int(scene_host["points"].shape[1])
    sc.sh_degree = int(sh_degree)
    sc.activation = 1 if scene_host.get("raw", False) else 0
    sc.storage = _STORAGE[scene_host["points"].dtype]
    return sc


def step_host_submit(scene_host: dict, sh_degree: int, cam, settings: Optional[Settings], dL_host, image_host,
                     grads_host: Optional[dict] = None, device: int = 0) -> int:
    """cs_step_host_submit: enqueue one host-buffer step of one view; returns its ticket.  The host
    tensors (pinned for overlap) must stay untouched until step_host_wait(ticket)."""
    ctx = Context.get(device)
    sc = _host_scene_struct(scene_host, sh_degree)
    s = (settings or Settings()).struct()
    g = grads_host or {}
    ptr = lambda t: t.data_ptr() if t is not None else None
    ticket = ctypes.c_uint64(0)
    code = B.lib().cs_step_host_submit(ctx.handle, ctypes.byref(sc), cameras_array([cam]), ctypes.byref(s),
                                       ptr(dL_host), image_host.data_ptr(), ptr(g.get("points")),
                                       ptr(g.get("delta")), ptr(g.get("sigma")), ptr(g.get("opacity")),
                                       ptr(g.get("sh")), ctypes.byref(ticket))
    B.check(code, "cs_step_host_submit")
    return int(ticket.value)


def step_host_wait(ticket: int, device: int = 0) -> None:
    """cs_step_host_wait: block until the submitted step `ticket` (and every earlier one) is done."""
    B.check(B.lib().cs_step_host_wait(Context.get(device).handle, ctypes.c_uint64(ticket)), "cs_step_host_wait")


# ---- serving -----------------------------------------------------------------------------------
class Server:
    """Continuous-batching view server over resident scenes (cs_server_* in the C ABI).

    Requests are queued with submit(); a worker thread in the library admits them into batches
    by a memory budget and renders each batch with one preprocess, binning and sort and one blend
    launch per view; poll() returns completions with their latencies.  pipelined=False makes the
    worker wait for each batch before admitting the next (with max_batch=1: one view at a time)."""

    STATUS = {0: "ok", 1: "arg", 2: "cuda", 3: "nomem", 4: "budget", 5: "timeout", 6: "device", 7: "state"}

    def __init__(self, device: int = 0, budget_bytes: int = 32 << 30, max_batch: int = 32,
                 settings: Optional[Settings] = None, pipelined: bool = True):
        h = ctypes.c_void_p()
        s = (settings or Settings()).struct()
        B.check(B.lib().cs_server_create(int(device), int(budget_bytes), int(max_batch), ctypes.byref(s),
                                         ctypes.byref(h)), "cs_server_create")
        self.handle = h
        if not pipelined:
            B.check(B.lib().cs_server_set_pipelining(h, 0), "cs_server_set_pipelining")
        self.device = device
        self._scenes = {}
        self._outputs = {}

    def add_scene(self, scene: SceneTensors) -> int:
        sid = ctypes.c_int32()
        sc = scene.struct()
        B.check(B.lib().cs_server_add_scene(self.handle, ctypes.byref(sc), ctypes.byref(sid)), "cs_server_add_scene")
        self._scenes[sid.value] = scene
        return sid.value

    def remove_scene(self, sid: int):
        B.check(B.lib().cs_server_remove_scene(self.handle, int(sid)), "cs_server_remove_scene")
        self._scenes.pop(sid, None)

    def submit(self, sid: int, cam, image: torch.Tensor) -> int:
        """Queue a view; image: contiguous float32 CUDA tensor [3][H][W], kept alive until polled."""
        rid = ctypes.c_uint64()
        c = camera_struct(cam)
        B.check(B.lib().cs_server_submit(self.handle, int(sid), ctypes.byref(c), image.data_ptr(), ctypes.byref(rid)),
                "cs_server_submit")
        self._outputs[rid.value] = image
        return rid.value

    def poll(self, max_n: int = 256, wait_ms: int = 0) -> list:
        buf = (B.CsCompletion * max_n)()
        n = ctypes.c_int32()
        B.check(B.lib().cs_server_poll(self.handle, buf, max_n, ctypes.byref(n), int(wait_ms)), "cs_server_poll")
        out = []
        for i in range(n.value):
            c = buf[i]
            self._outputs.pop(c.id, None)
            out.append(dict(id=c.id, status=self.STATUS.get(c.status, str(c.status)), batch_size=c.batch_size,
                            queue_ms=c.queue_ms, latency_ms=c.latency_ms))
        return out

    def stats(self) -> dict:
        a = (ctypes.c_uint64 * 7)()
        B.check(B.lib().cs_server_stats(self.handle, a), "cs_server_stats")
        return dict(completed=a[0], batches=a[1], largest_batch=a[2], peak_bytes=a[3], queued=a[4], on_gpu=a[5],
                    peak_pool_bytes=a[6])

    def close(self):
        if self.handle:
            B.lib().cs_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
