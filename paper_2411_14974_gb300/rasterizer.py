"""Python face of the C ABI: forward/backward calls, the autograd Function and state access.

Only argument marshalling happens here; every step of the rasterizer runs in the CUDA library.
PyTorch provides device memory (tensors) and the current stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _binding as B

ARRAYS = dict(records=0, depth_keys=1, rects=2, counts=3, pair_keys=4, pair_values=5, tile_ranges=6,
              n_last=7, hulls=8)
_ARRAY_DTYPES = dict(records=np.float32, depth_keys=np.uint32, rects=np.uint32, counts=np.uint32,
                     pair_keys=np.uint32, pair_values=np.uint32, tile_ranges=np.uint32, n_last=np.uint32,
                     hulls=np.uint32)


@dataclasses.dataclass
class Settings:
    """Compositing constants (3DGS-style cut-offs; Eq. 5 has none) and the distance scaling."""
    tau: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    dist_mode: int = 0
    dist_power: float = 1.0

    def struct(self) -> B.CsSettings:
        s = B.CsSettings()
        s.tau, s.alpha_max, s.t_min = float(self.tau), float(self.alpha_max), float(self.t_min)
        for i in range(3):
            s.bg[i] = float(self.bg[i])
        s.dist_mode, s.dist_power = int(self.dist_mode), float(self.dist_power)
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
    """Per-device library context (owns the stream-ordered memory pool of transient buffers)."""
    _by_device: dict = {}

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        B.check(B.lib().cs_context_create(int(device), ctypes.byref(h)), "cs_context_create")
        self.handle = h
        self.device = int(device)

    @classmethod
    def get(cls, device: int = 0) -> "Context":
        if device not in cls._by_device:
            cls._by_device[device] = Context(device)
        return cls._by_device[device]

    def __del__(self):
        try:
            if self.handle:
                B.lib().cs_context_destroy(self.handle)
        except Exception:
            pass


@dataclasses.dataclass
class SceneTensors:
    """Device tensors of a scene (float32, contiguous, on one CUDA device)."""
    points: torch.Tensor   # [N][K][3]
    delta: torch.Tensor    # [N]
    sigma: torch.Tensor    # [N]
    opacity: torch.Tensor  # [N]
    sh: torch.Tensor       # [N][(D+1)^2][3]

    @property
    def sh_degree(self) -> int:
        nb = int(self.sh.shape[1])
        d = int(round(nb ** 0.5)) - 1
        if (d + 1) ** 2 != nb:
            raise ValueError("sh must be [N][(D+1)^2][3]")
        return d

    def struct(self) -> B.CsScene:
        s = B.CsScene()
        for name in ("points", "delta", "sigma", "opacity", "sh"):
            t = getattr(self, name)
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
            setattr(s, name, t.data_ptr() if t.numel() else None)
        s.n = int(self.points.shape[0])
        s.k = int(self.points.shape[1])
        s.sh_degree = self.sh_degree
        return s

    @staticmethod
    def from_numpy(scene, device="cuda") -> "SceneTensors":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)
        return SceneTensors(f(scene.points), f(scene.delta), f(scene.sigma), f(scene.opacity), f(scene.sh))


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


def backward(state: State, dL_dimage: torch.Tensor, grads: Optional[dict] = None) -> dict:
    """cs_backward: accumulate d(loss)/d(points, delta, sigma, opacity, sh) into ``grads``
    (zero tensors are created when not given)."""
    sc = state.scene
    if grads is None:
        grads = dict(points=torch.zeros_like(sc.points), delta=torch.zeros_like(sc.delta),
                     sigma=torch.zeros_like(sc.sigma), opacity=torch.zeros_like(sc.opacity),
                     sh=torch.zeros_like(sc.sh))
    g = dL_dimage.contiguous()
    if g.dtype != torch.float32:
        g = g.float()
    ptr = lambda t: t.data_ptr() if (t is not None and t.numel()) else None
    code = B.lib().cs_backward(state.ctx.handle, state.handle, g.data_ptr(), ptr(grads.get("points")),
                               ptr(grads.get("delta")), ptr(grads.get("sigma")), ptr(grads.get("opacity")),
                               ptr(grads.get("sh")), _stream_ptr(sc.points.device))
    B.check(code, "cs_backward")
    return grads


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, delta, sigma, opacity, sh, cams, settings):
        scene = SceneTensors(points.detach().contiguous(), delta.detach().contiguous(), sigma.detach().contiguous(),
                             opacity.detach().contiguous(), sh.detach().contiguous())
        need = any(ctx.needs_input_grad[:5])
        image, _, state = forward(scene, cams, settings, keep_state=need)
        ctx.state = state
        return image

    @staticmethod
    def backward(ctx, dL_dimage):
        state = ctx.state
        g = backward(state, dL_dimage)
        state.release()
        ctx.state = None
        return g["points"], g["delta"], g["sigma"], g["opacity"], g["sh"], None, None


def render(points, delta, sigma, opacity, sh, cams, settings: Optional[Settings] = None) -> torch.Tensor:
    """Differentiable render (Sec. 3.2, Eq. 4, 5, S1, S2): image [V][3][H][W] for len(cams) views.

    delta, sigma, opacity are activated values (> 0, > 0, in (0, 1])."""
    return _Render.apply(points, delta, sigma, opacity, sh, list(cams), settings or Settings())


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
    s = (settings or Settings()).struct()
    g = grads_host or {}
    ptr = lambda t: t.data_ptr() if t is not None else None
    code = B.lib().cs_step_host(ctx.handle, ctypes.byref(sc), cameras_array(cams), len(cams), ctypes.byref(s),
                                ptr(dL_host), image_host.data_ptr(), ptr(g.get("points")), ptr(g.get("delta")),
                                ptr(g.get("sigma")), ptr(g.get("opacity")), ptr(g.get("sh")),
                                _stream_ptr(torch.device("cuda", device)))
    B.check(code, "cs_step_host")


# ---- serving -----------------------------------------------------------------------------------
class Server:
    """Continuous-batching view server over resident scenes (cs_server_* in the C ABI).

    Requests are queued with submit(); a worker thread in the library admits them into batches
    by an estimated memory budget and renders each batch with one binning/sort and one blend
    launch; poll() returns completions with their latencies."""

    STATUS = {0: "ok", 1: "arg", 2: "cuda", 3: "nomem", 4: "budget", 5: "timeout", 6: "device", 7: "state"}

    def __init__(self, device: int = 0, budget_bytes: int = 32 << 30, max_batch: int = 32,
                 settings: Optional[Settings] = None):
        h = ctypes.c_void_p()
        s = (settings or Settings()).struct()
        B.check(B.lib().cs_server_create(int(device), int(budget_bytes), int(max_batch), ctypes.byref(s),
                                         ctypes.byref(h)), "cs_server_create")
        self.handle = h
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
        a = (ctypes.c_uint64 * 6)()
        B.check(B.lib().cs_server_stats(self.handle, a), "cs_server_stats")
        return dict(completed=a[0], batches=a[1], largest_batch=a[2], peak_bytes=a[3], queued=a[4], on_gpu=a[5])

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
