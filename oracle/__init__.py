"""CPU oracle for the convex tile rasterizer of 3D Convex Splatting (arXiv 2411.14974).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product package never does.  It wraps ``cs_oracle.c``
(plain C, binary64 continuous maths, binary32 discrete specification) through ctypes and shares
no code with the CUDA path.

Functions take the scene/camera objects produced by ``paper_2411_14974_gb300.synthetic`` (plain
numpy arrays; that module draws inputs and holds none of the method's arithmetic).

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force or library routines.  The one unpinned quantity is the absolute agreement
with the authors' own rasterizer, for which no code, numbers or figures exist ("parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, f"libcs_oracle_{platform.machine()}.so")

KMAX = 8


def build(force: bool = False) -> str:
    """Compile ``cs_oracle.c`` (gcc, -O2, no FMA contraction, OpenMP) if it is missing or stale."""
    if (not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-Wno-unknown-pragmas", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("z_near", ctypes.c_float)]


class OrcSettings(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("dist_mode", ctypes.c_int32), ("dist_power", ctypes.c_float),
                ("q_binary32", ctypes.c_int32), ("perturb_ulps", ctypes.c_float), ("line_rel", ctypes.c_float),
                ("tile_test", ctypes.c_int32), ("line_f32", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        _lib.orc_orient.restype = ctypes.c_int
        _lib.orc_orient.argtypes = [ctypes.c_float] * 6
        _lib.orc_hull2d.restype = ctypes.c_int
        _lib.orc_hull2d.argtypes = [P, i32, P]
        _lib.orc_ln_spec.restype = ctypes.c_float
        _lib.orc_ln_spec.argtypes = [ctypes.c_float]
        _lib.orc_exp_spec.restype = ctypes.c_float
        _lib.orc_exp_spec.argtypes = [ctypes.c_float]
        _lib.orc_sigmoid_spec.restype = ctypes.c_float
        _lib.orc_sigmoid_spec.argtypes = [ctypes.c_float]
        _lib.orc_ln_array.restype = None
        _lib.orc_ln_array.argtypes = [i64, P, P]
        _lib.orc_activate.restype = None
        _lib.orc_activate.argtypes = [i64, P, P, P, P, P, P]
        _lib.orc_discrete.restype = ctypes.c_int
        _lib.orc_discrete.argtypes = [P, i64, i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_tiles.restype = ctypes.c_int
        _lib.orc_tiles.argtypes = [P, i64, i32, P, P, P, P, P, P, P]
        _lib.orc_render_pixels.restype = ctypes.c_int
        _lib.orc_render_pixels.argtypes = [P, i64, i32, P, P, P, P, i32, P, P, P, i64, u64, P, P, P, P, P, P]
        _lib.orc_backward_pixels.restype = ctypes.c_int
        _lib.orc_backward_pixels.argtypes = [P, i64, i32, P, P, P, P, i32, P, P, P, i64, P, u64, P, P, P, P, P]
        _lib.orc_alpha_support.restype = ctypes.c_int
        _lib.orc_alpha_support.argtypes = [P, i64, i32, P, P, P, P, i32, P, P, P]
        _lib.orc_alpha_tile_mask.restype = ctypes.c_int
        _lib.orc_alpha_tile_mask.argtypes = [P, i64, i32, P, P, P, P, i32, P, P, P]
        _lib.orc_sh_basis.restype = None
        _lib.orc_sh_basis.argtypes = [i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P]
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def camera(cam) -> OrcCamera:
    c = OrcCamera()
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


def settings(tau=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, bg=(0.0, 0.0, 0.0), dist_mode=0,
             dist_power=1.0, q_binary32=False, perturb_ulps=4.0, line_rel=0.0, tile_test=0,
             line_f32=False) -> OrcSettings:
    """Method settings plus oracle-only knobs (no counterpart in the method).

    q_binary32: build the hull lines from the binary32 projected points the hull was decided on
    (the discrete specification) rather than from a binary64 re-projection; the continuous maths
    stays binary64.
    Error model for the conditioning bound ``sens``, the decision bands and the probes:
      line_rel > 0: every line value may be off by line_rel (|q - a|_1 + |a - v_t|_1 + 32 + |L_t|)
                    pixels (binary32 evaluation relative to the anchor vertex a);
      otherwise:    every hull vertex may move by perturb_ulps binary32 ulps.
    line_f32: evaluate every line value in binary32 from the record form of the discrete
    specification (anchored lines scaled by log2(e) d^p delta, re-based to the pixel's 8 x 4 block
    origin, fused multiply-adds), the rest in binary64; used only to check the line_rel model."""
    s = OrcSettings()
    s.tau, s.alpha_max, s.t_min = float(tau), float(alpha_max), float(t_min)
    for i in range(3):
        s.bg[i] = float(bg[i])
    s.dist_mode, s.dist_power = int(dist_mode), float(dist_power)
    s.q_binary32, s.perturb_ulps, s.line_rel = int(bool(q_binary32)), float(perturb_ulps), float(line_rel)
    s.tile_test = int(tile_test)
    s.line_f32 = int(bool(line_f32))
    return s


def _scene_arrays(scene):
    if getattr(scene, "raw", False):
        raise ValueError("raw-parameter scene: pass activate(scene) to the oracle")
    pts = np.ascontiguousarray(scene.points, np.float32)
    n, k = pts.shape[0], pts.shape[1]
    arr = dict(points=pts,
               delta=np.ascontiguousarray(scene.delta, np.float32),
               sigma=np.ascontiguousarray(scene.sigma, np.float32),
               opacity=np.ascontiguousarray(scene.opacity, np.float32),
               sh=np.ascontiguousarray(scene.sh, np.float32))
    return arr, n, k, int(scene.sh_degree)


def orient(a, b, c) -> int:
    """Exact sign of (b-a) x (c-a) for binary32 points."""
    f = np.float32
    return lib().orc_orient(f(a[0]), f(a[1]), f(b[0]), f(b[1]), f(c[0]), f(c[1]))


def hull2d(uv) -> list:
    """Hull vertex indices (pivot first, increasing polar angle) of K <= 8 binary32 points."""
    uv = np.ascontiguousarray(uv, np.float32).reshape(-1, 2)
    idx = np.zeros(KMAX, np.int32)
    T = lib().orc_hull2d(_p(uv), uv.shape[0], _p(idx))
    return [int(i) for i in idx[:T]]


def ln_spec(x: float) -> float:
    return float(np.float32(lib().orc_ln_spec(np.float32(x))))


def ln_spec_array(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32).ravel()
    out = np.empty_like(x)
    lib().orc_ln_array(x.size, _p(x), _p(out))
    return out


def exp_spec(x: float) -> float:
    """The binary32 exp of the parameter activations (Cody-Waite reduction, degree-7 Taylor)."""
    return float(np.float32(lib().orc_exp_spec(np.float32(x))))


def sigmoid_spec(x: float) -> float:
    return float(np.float32(lib().orc_sigmoid_spec(np.float32(x))))


def activate(scene):
    """Copy of a raw-parameter scene with delta = exp, sigma = exp, opacity = sigmoid of the raw
    values (Sec. 3.3), each in the binary32 definition both sides share."""
    n = scene.points.shape[0]
    rd, rs, ro = (np.ascontiguousarray(getattr(scene, a), np.float32) for a in ("delta", "sigma", "opacity"))
    d, s, o = np.empty(n, np.float32), np.empty(n, np.float32), np.empty(n, np.float32)
    lib().orc_activate(n, _p(rd), _p(rs), _p(ro), _p(d), _p(s), _p(o))
    out = scene.copy()
    out.delta, out.sigma, out.opacity, out.raw = d, s, o, False
    return out


def raw_gradients(scene_raw, grads: dict) -> dict:
    """Chain rule from gradients w.r.t. the activated (delta, sigma, opacity) to the raw values:
    d exp(x)/dx = exp(x), d sigmoid(x)/dx = sigmoid(x) (1 - sigmoid(x)); binary64."""
    act = activate(scene_raw)
    out = dict(grads)
    out["delta"] = grads["delta"] * act.delta.astype(np.float64)
    out["sigma"] = grads["sigma"] * act.sigma.astype(np.float64)
    o = act.opacity.astype(np.float64)
    out["opacity"] = grads["opacity"] * o * (1.0 - o)
    return out


def discrete(scene, cam, st=None) -> dict:
    """Discrete specification per convex: visibility, hull, tile rectangle, kept-tile count and
    list (the exact tile test), depth key, binary32 uv.  tiles[tile_offsets[i]:][:count[i]] are
    convex i's tiles in row-major order."""
    st = st or settings()
    a, n, k, _ = _scene_arrays(scene)
    out = dict(visible=np.zeros(n, np.int32), reason=np.zeros(n, np.int32), hull_t=np.zeros(n, np.int32),
               hull_idx=np.zeros((n, KMAX), np.int32), rect=np.zeros((n, 4), np.int32),
               full=np.zeros(n, np.int32), depth_bits=np.zeros(n, np.uint32), uv=np.zeros((n, k, 2), np.float32),
               count=np.zeros(n, np.int32))
    c = camera(cam)
    rc = lib().orc_discrete(_p(a["points"]), n, k, _p(a["delta"]), _p(a["sigma"]), _p(a["opacity"]),
                            ctypes.byref(c), ctypes.byref(st), _p(out["visible"]), _p(out["reason"]),
                            _p(out["hull_t"]), _p(out["hull_idx"]), _p(out["rect"]), _p(out["full"]),
                            _p(out["depth_bits"]), _p(out["uv"]), _p(out["count"]))
    if rc:
        raise ValueError(f"orc_discrete failed ({rc})")
    cnt = out["count"].astype(np.int64)
    offsets = np.ascontiguousarray(np.cumsum(cnt) - cnt)
    tiles = np.zeros(int(cnt.sum()), np.int32)
    rc = lib().orc_tiles(_p(a["points"]), n, k, _p(a["delta"]), _p(a["sigma"]), _p(a["opacity"]), ctypes.byref(c),
                         ctypes.byref(st), _p(offsets), _p(tiles))
    if rc:
        raise ValueError(f"orc_tiles failed ({rc})")
    out["tiles"], out["tile_offsets"] = tiles, offsets
    return out


def all_pixels(width: int, height: int) -> np.ndarray:
    ys, xs = np.meshgrid(np.arange(height, dtype=np.int32), np.arange(width, dtype=np.int32), indexing="ij")
    return np.ascontiguousarray(np.stack([xs.ravel(), ys.ravel()], 1))


def render_pixels(scene, cam, st=None, pix=None, perturb_seed: int = 0) -> dict:
    """Eq. 5 at the listed pixels ([npix][2] = (x, y)), brute force over all convexes, binary64."""
    st = st or settings()
    a, n, k, deg = _scene_arrays(scene)
    if pix is None:
        pix = all_pixels(cam.width, cam.height)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    m = pix.shape[0]
    out = dict(rgb=np.zeros((m, 3)), t_final=np.zeros(m), last_id=np.zeros(m, np.int64),
               n_contrib=np.zeros(m, np.int32), flags=np.zeros(m, np.uint32), sens=np.zeros(m))
    c = camera(cam)
    rc = lib().orc_render_pixels(_p(a["points"]), n, k, _p(a["delta"]), _p(a["sigma"]), _p(a["opacity"]),
                                 _p(a["sh"]), deg, ctypes.byref(c), ctypes.byref(st), _p(pix), m,
                                 int(perturb_seed), _p(out["rgb"]), _p(out["t_final"]), _p(out["last_id"]),
                                 _p(out["n_contrib"]), _p(out["flags"]), _p(out["sens"]))
    if rc:
        raise ValueError(f"orc_render_pixels failed ({rc})")
    return out


def render_image(scene, cam, st=None, perturb_seed: int = 0) -> dict:
    """Full image: rgb [3][H][W], t_final [H][W], last_id, n_contrib, flags, sens [H][W].

    sens is a first-order bound on how much any channel can change when every hull vertex moves
    by perturb_ulps binary32 ulps; flags mark cut-off decisions within their bands."""
    r = render_pixels(scene, cam, st, None, perturb_seed)
    H, W = cam.height, cam.width
    return dict(image=np.ascontiguousarray(r["rgb"].reshape(H, W, 3).transpose(2, 0, 1)),
                t_final=r["t_final"].reshape(H, W), last_id=r["last_id"].reshape(H, W),
                n_contrib=r["n_contrib"].reshape(H, W), flags=r["flags"].reshape(H, W),
                sens=r["sens"].reshape(H, W))


def backward_pixels(scene, cam, st, pix, dL_dC, perturb_seed: int = 0) -> dict:
    """Analytic binary64 gradient of sum_i dL_dC[i] . C(pix[i]) w.r.t. points, delta, sigma, opacity, SH.

    perturb_seed != 0 moves the projected points by 4 binary32 ulps in the per-pixel part (a
    conditioning probe, as in render_pixels)."""
    st = st or settings()
    a, n, k, deg = _scene_arrays(scene)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    g = np.ascontiguousarray(dL_dC, np.float64).reshape(-1, 3)
    assert g.shape[0] == pix.shape[0]
    nb = (deg + 1) ** 2
    out = dict(points=np.zeros((n, k, 3)), delta=np.zeros(n), sigma=np.zeros(n), opacity=np.zeros(n),
               sh=np.zeros((n, nb, 3)))
    c = camera(cam)
    rc = lib().orc_backward_pixels(_p(a["points"]), n, k, _p(a["delta"]), _p(a["sigma"]), _p(a["opacity"]),
                                   _p(a["sh"]), deg, ctypes.byref(c), ctypes.byref(st), _p(pix), pix.shape[0],
                                   _p(g), int(perturb_seed), _p(out["points"]), _p(out["delta"]), _p(out["sigma"]),
                                   _p(out["opacity"]), _p(out["sh"]))
    if rc:
        raise ValueError(f"orc_backward_pixels failed ({rc})")
    return out


def backward_image(scene, cam, st, dL_dimage, perturb_seed: int = 0) -> dict:
    """Gradient for a full-image cotangent dL_dimage [3][H][W]."""
    H, W = cam.height, cam.width
    g = np.asarray(dL_dimage, np.float64).reshape(3, H, W).transpose(1, 2, 0).reshape(-1, 3)
    return backward_pixels(scene, cam, st, all_pixels(W, H), g, perturb_seed)


def alpha_support(scene, cam, st=None) -> np.ndarray:
    """Per convex, the pixel bbox (x0, y0, x1, y1) of {alpha >= tau}, or -1s."""
    st = st or settings()
    a, n, k, deg = _scene_arrays(scene)
    bbox = np.zeros((n, 4), np.int32)
    c = camera(cam)
    rc = lib().orc_alpha_support(_p(a["points"]), n, k, _p(a["delta"]), _p(a["sigma"]), _p(a["opacity"]),
                                 _p(a["sh"]), deg, ctypes.byref(c), ctypes.byref(st), _p(bbox))
    if rc:
        raise ValueError(f"orc_alpha_support failed ({rc})")
    return bbox


def alpha_tile_mask(scene, cam, st=None) -> np.ndarray:
    """[n][tiles] mask: 1 where some pixel of the tile has binary64 alpha >= tau."""
    st = st or settings()
    a, n, k, deg = _scene_arrays(scene)
    nt = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    out = np.zeros((n, nt), np.uint8)
    c = camera(cam)
    rc = lib().orc_alpha_tile_mask(_p(a["points"]), n, k, _p(a["delta"]), _p(a["sigma"]), _p(a["opacity"]),
                                   _p(a["sh"]), deg, ctypes.byref(c), ctypes.byref(st), _p(out))
    if rc:
        raise ValueError(f"orc_alpha_tile_mask failed ({rc})")
    return out


def sh_basis(deg: int, d) -> tuple:
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().orc_sh_basis(int(deg), float(d[0]), float(d[1]), float(d[2]), _p(Y), _p(dY))
    return Y, dY


def tile_lists(disc: dict, cam) -> dict:
    """Expected per-tile convex lists in (depth bits, id) order from the discrete specification.

    Returns dict(tile -> np.ndarray of convex ids).  Uses numpy's sort as the ordering primitive.
    """
    vis = np.nonzero(disc["visible"])[0]
    order = vis[np.lexsort((vis, disc["depth_bits"][vis]))]
    lists = {}
    for cid in order:
        o, c = disc["tile_offsets"][cid], disc["count"][cid]
        for t in disc["tiles"][o:o + c]:
            lists.setdefault(int(t), []).append(int(cid))
    return {t: np.asarray(v, np.int64) for t, v in lists.items()}


def num_threads() -> int:
    return int(lib().orc_num_threads())


def sorted_pairs(disc: dict, cam, tile_base: int = 0, rec_base: int = 0):
    """Expected sorted (tile, record) pairs of one view: visible convexes in (depth bits, id) order
    each list their kept tiles in row-major order, then a stable sort by tile index.
    Returns (keys = tile_base + tile index, values = rec_base + convex id)."""
    vis = np.nonzero(disc["visible"])[0]
    order = vis[np.lexsort((vis, disc["depth_bits"][vis]))]
    cnt = disc["count"][order].astype(np.int64)
    rep = np.repeat(np.arange(len(order)), cnt)
    within = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    keys = disc["tiles"][disc["tile_offsets"][order][rep] + within].astype(np.int64)
    vals = order[rep]
    perm = np.argsort(keys, kind="stable")
    return (keys[perm] + tile_base).astype(np.int64), (vals[perm] + rec_base).astype(np.int64)


def pack_hull(disc: dict) -> np.ndarray:
    """Hull of every convex in the packed form T | idx_i << (4 + 3 i); 0 when not drawn."""
    out = np.zeros(len(disc["visible"]), np.uint32)
    for i in np.nonzero(disc["visible"])[0]:
        T = int(disc["hull_t"][i])
        w = T
        for j in range(T):
            w |= int(disc["hull_idx"][i][j]) << (4 + 3 * j)
        out[i] = w
    return out
