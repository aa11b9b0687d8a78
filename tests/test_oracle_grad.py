"""Pins for the oracle's analytic binary64 gradient (reverse of Eq. 5, Eq. S1/S2, Eq. 4).

Reference: binary64 central finite differences of the oracle's own forward render at steps h and
h/2 (they must agree with each other, a Richardson check), on samples whose discrete structure
(visibility, hull, per-pixel contributing set and last contributor) is the same at +h and -h.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn


def _scene(seed, deg):
    sc = syn.blob_scene(seed, n=40, radius=0.15, sh_degree=deg)
    sc.points[..., :2] *= 0.3
    return sc


def _loss(sc, cam, st, G):
    r = oracle.render_image(sc, cam, st)
    return float((r["image"] * G).sum()), r["n_contrib"], r["last_id"]


def _fd(sc, cam, st, G, field, index, h):
    vals = []
    structs = []
    for s in (+1, -1):
        p = sc.copy()
        arr = getattr(p, field)
        arr[index] = np.float32(arr[index] + s * h)
        actual = float(arr[index]) - float(getattr(sc, field)[index])
        L, nc, last = _loss(p, cam, st, G)
        vals.append((L, actual))
        structs.append((nc, last))
    (Lp, hp), (Lm, hm) = vals
    same = (structs[0][0] == structs[1][0]).all() and (structs[0][1] == structs[1][1]).all()
    return (Lp - Lm) / (hp - hm), same


@pytest.mark.parametrize("deg,power,mode", [(0, 1.0, 0), (3, 1.0, 0), (1, 2.0, 0), (2, 0.5, 1)])
def test_gradient_matches_finite_differences(deg, power, mode):
    cam = syn.blob_camera(48, 48)
    sc = _scene(deg + 7, deg)
    # work in binary64-representable steps: points/params are binary32, steps exact multiples
    st = oracle.settings(dist_power=power, dist_mode=mode)
    rng = np.random.default_rng(deg)
    G = rng.uniform(-1, 1, (3, 48, 48))
    g = oracle.backward_image(sc, cam, st, G)
    disc = oracle.discrete(sc, cam, st)
    vis = np.nonzero(disc["visible"])[0]
    checked = 0
    samples = []
    for i in rng.choice(vis, 12, replace=False):
        samples += [("points", (i, rng.integers(sc.k), rng.integers(3)), 2e-4),
                    ("delta", (i,), 2e-3 * float(sc.delta[i])), ("sigma", (i,), 2e-3 * float(sc.sigma[i])),
                    ("opacity", (i,), 1e-3), ("sh", (i, rng.integers(sc.sh.shape[1]), rng.integers(3)), 1e-3)]
    for field, index, h in samples:
        a = float(g[field][index])
        d1, s1 = _fd(sc, cam, st, G, field, index, h)
        d2, s2 = _fd(sc, cam, st, G, field, index, h / 2)
        if not (s1 and s2):
            continue  # a discrete decision flipped inside the step
        scale = max(abs(a), abs(d2), 1e-6)
        if abs(d1 - d2) > 0.05 * scale:
            continue  # not resolved by the steps (a kink in the step); Richardson disagreement
        rich = (4 * d2 - d1) / 3
        # truncation error of the extrapolated value is far below |d1 - d2| (the estimate of d2's error)
        assert abs(rich - a) <= max(1e-5 * scale, 0.05 * abs(d1 - d2)) + 1e-9, (field, index, a, d1, d2)
        checked += 1
    assert checked >= 0.6 * len(samples)


def test_gradient_zero_for_invisible_and_culled():
    cam = syn.blob_camera(32, 32)
    sc = _scene(1, 0)
    sc.points[0, :, 2] = -10.0  # behind the camera: culled
    g = oracle.backward_image(sc, cam, oracle.settings(), np.ones((3, 32, 32)))
    assert not g["points"][0].any() and g["delta"][0] == 0 and g["opacity"][0] == 0
