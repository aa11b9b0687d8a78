"""Pins for the oracle's binary32 discrete specification (projection, depth key, culling, the
spec logarithm and the conservative tile range) and for its spherical-harmonic basis.

References: math.log, closed-form pinhole projection (Eq. 4 with the perspective divide), the
binary64 distance to the centre, and the definition of the tile range: every pixel whose
binary64 alpha reaches tau must lie in a tile of its convex's range.  SH: orthonormality by
exact quadrature on the sphere and finite differences of the basis.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn
from tests import _cases as C


def test_ln_spec_matches_log():
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.exp(rng.uniform(math.log(1e-30), math.log(1e30), 4000)),
                         rng.uniform(1e-3, 260.0, 4000), [1.0, 2.0, 0.5, 254.0, 1e-38, 3e38]]).astype(np.float32)
    for x in xs:
        got = oracle.ln_spec(x)
        want = math.log(float(x))
        assert abs(got - want) <= 4e-7 * max(1.0, abs(want)), (x, got, want)


def test_projection_closed_form():
    cam = syn.blob_camera()  # R = I, t = (0, 0, 4), 128x128, 50 degrees
    assert abs(cam.fx - 64.0 / math.tan(math.radians(25.0))) < 1e-4
    pts = np.array([[[0, 0, 0], [0.5, -0.25, 1.0], [-0.7, 0.3, -1.0], [0.1, 0.9, 0.5], [0.0, 0.0, 2.0],
                     [0.2, 0.2, 0.2]]], np.float32)
    sc = syn.Scene(pts, np.ones(1, np.float32), np.ones(1, np.float32), np.full(1, 0.5, np.float32),
                   np.zeros((1, 1, 3), np.float32), 0)
    d = oracle.discrete(sc, cam)
    uv = d["uv"][0].astype(np.float64)
    z = pts[0, :, 2].astype(np.float64) + 4.0
    want_u = cam.fx * pts[0, :, 0] / z + cam.cx
    want_v = cam.fy * pts[0, :, 1] / z + cam.cy
    assert uv[0, 0] == cam.cx and uv[0, 1] == cam.cy  # on the optical axis
    assert np.abs(uv[:, 0] - want_u).max() < 2e-5 and np.abs(uv[:, 1] - want_v).max() < 2e-5


def test_depth_key_is_binary32_distance():
    sc, cams = syn.workload("blob1k_128", seed=1)
    d = oracle.discrete(sc, cams[0])
    f = d["depth_bits"].view(np.float32).astype(np.float64)
    want = C.camera_distance(sc, cams[0])
    assert (np.abs(f - want) <= 4 * np.spacing(want.astype(np.float32)).astype(np.float64)).all()
    # the unsigned key orders like the float (positive distances)
    o1 = np.argsort(d["depth_bits"], kind="stable")
    o2 = np.argsort(f, kind="stable")
    assert (o1 == o2).all()


def test_culling_rules():
    cam = syn.blob_camera()
    base = syn.blob_scene(0, n=8)
    sc = base.copy()
    sc.points[0, 0, 2] = -3.9        # z = 0.1 < z_near
    sc.opacity[1] = 1.0 / 255.0      # o <= tau
    sc.points[2, :, :] = sc.points[2, 0, :]  # all points coincide: no hull
    sc.delta[3] = 0.0                # delta must be > 0
    sc.sigma[4] = np.nan             # non-finite
    sc.points[5, :, 0] = 40.0        # projects off screen (far right)
    d = oracle.discrete(sc, cam)
    assert list(d["visible"]) == [0, 0, 0, 0, 0, 0, 1, 1]
    assert list(d["reason"][:6]) == [3, 6, 7, 2, 1, 9]


def _conservative(sc, cam, st=None):
    """Every pixel with binary64 alpha >= tau lies in the rectangle and in a tile the exact tile
    test keeps; returns (convexes reaching tau, tiles the test removed from the rectangles)."""
    st = st or oracle.settings()
    d = oracle.discrete(sc, cam, st)
    bb = oracle.alpha_support(sc, cam, st)
    has = bb[:, 0] >= 0
    assert (d["visible"][has] == 1).all(), "a culled convex reaches tau"
    r = d["rect"][has]
    b = bb[has]
    assert (b[:, 0] // 16 >= r[:, 0]).all() and (b[:, 2] // 16 <= r[:, 2]).all()
    assert (b[:, 1] // 16 >= r[:, 1]).all() and (b[:, 3] // 16 <= r[:, 3]).all()
    mask = oracle.alpha_tile_mask(sc, cam, st)
    for i in np.nonzero(has)[0]:
        kept = set(d["tiles"][d["tile_offsets"][i]:][:d["count"][i]].tolist())
        need = set(np.nonzero(mask[i])[0].tolist())
        assert need <= kept, (i, sorted(need - kept))
    vis = d["visible"] == 1
    area = (d["rect"][vis, 2] - d["rect"][vis, 0] + 1) * (d["rect"][vis, 3] - d["rect"][vis, 1] + 1)
    return has.sum(), int(area.sum() - d["count"][vis].sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tile_range_conservative_blob(seed):
    sc, cams = syn.workload("blob1k_128", seed=seed)
    assert _conservative(sc, cams[0])[0] > 500
    assert _conservative(sc, cams[0], oracle.settings(tile_test=1))[0] > 500


def test_tile_range_conservative_soft_and_sharp():
    """Very diffuse (long tails) and very hard convexes, several opacities and cut-offs."""
    cam = syn.blob_camera(96, 80)
    sc = syn.blob_scene(9, n=300)
    rng = np.random.default_rng(1)
    sc.delta = np.exp(rng.uniform(math.log(0.02), math.log(200.0), sc.n)).astype(np.float32)
    sc.sigma = np.exp(rng.uniform(math.log(0.001), math.log(20.0), sc.n)).astype(np.float32)
    sc.opacity = rng.uniform(0.005, 1.0, sc.n).astype(np.float32)
    removed = 0
    for st in (oracle.settings(), oracle.settings(tau=0.05), oracle.settings(dist_power=2.0),
               oracle.settings(dist_mode=1, dist_power=0.5)):
        n, rm = _conservative(sc, cam, st)
        assert n > 50 and rm == 0  # without the tile test every tile of the rectangle is kept
    for st in (oracle.settings(tile_test=1), oracle.settings(tau=0.05, tile_test=1),
               oracle.settings(dist_power=2.0, tile_test=1), oracle.settings(dist_mode=1, dist_power=0.5, tile_test=1)):
        n, rm = _conservative(sc, cam, st)
        assert n > 50
        removed += rm
    assert removed > 0  # the exact tile test is not vacuous on these shapes


def test_exact_tile_test_drops_tiles_a_thin_diagonal_convex_misses():
    """A thin sharp convex along the image diagonal: its rectangle spans many tiles, most of which
    lie off the diagonal and are dropped; the tiles along it are kept."""
    cam = syn.blob_camera(160, 160)
    z, f = 4.0, cam.fx
    # a sliver from pixel (8, 8) to (152, 152), about 1 px wide
    a = np.array([8.0, 8.0]) - 80.0
    b = np.array([152.0, 152.0]) - 80.0
    w = np.array([0.7, -0.7])
    quad = [a, b, b + w, a + w]
    pts = np.array([[q[0] * z / f, q[1] * z / f, z] for q in quad] + [[a[0] * z / f, a[1] * z / f, z]] * 2)
    sc = syn.Scene(pts[None].astype(np.float32) - np.array([0, 0, 4.0], np.float32),
                   np.array([5.0], np.float32), np.array([5.0], np.float32), np.array([0.9], np.float32),
                   np.zeros((1, 1, 3), np.float32), 0)
    st = oracle.settings(tile_test=1)
    d = oracle.discrete(sc, cam, st)
    assert d["visible"][0] == 1
    x0, y0, x1, y1 = d["rect"][0]
    area = (x1 - x0 + 1) * (y1 - y0 + 1)
    assert area >= 80 and d["count"][0] <= 0.4 * area
    kept = set(d["tiles"][:d["count"][0]].tolist())
    assert all((t * 10 + t) in kept for t in range(1, 9))  # the diagonal tiles (ty = tx)
    _conservative(sc, cam, st)
    assert oracle.discrete(sc, cam)["count"][0] == area  # without the test: the whole rectangle


def test_sh_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform in phi integrates these degree <= 6 products exactly."""
    xg, wg = np.polynomial.legendre.leggauss(8)
    nphi = 16
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            Y, _ = oracle.sh_basis(3, (st * math.cos(ph), st * math.sin(ph), ct))
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_gradient_finite_differences_and_degree0():
    rng = np.random.default_rng(2)
    for _ in range(20):
        d = rng.standard_normal(3)
        Y, dY = oracle.sh_basis(3, d)
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1e-6
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / 2e-6
            assert np.abs(fd - dY[:, a]).max() < 1e-7
        Y0, _ = oracle.sh_basis(0, d / np.linalg.norm(d))
        assert Y0[0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-16) and not Y0[1:].any()
