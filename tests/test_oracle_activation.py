"""Pins for the parameter activations of Sec. 3.3 (delta, sigma = exp of the raw values, o =
sigmoid of the raw value) in the oracle's binary32 definition, and for its chain rule to the raw
values.

Reference: the exponential itself (math.exp to within 2 binary32 ulps over the whole normal
range), its special values and range limits, monotonicity, the sigmoid's symmetry, and binary64
central finite differences of the oracle's render taken in the raw parameters.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_14974_gb300 import synthetic as syn


def _ulps(got: float, want: float) -> float:
    return abs(got - want) / float(np.spacing(np.float32(want)))


def test_exp_spec_within_two_ulps_of_exp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-87.3, 88.7, 20000), rng.uniform(-1, 1, 5000),
                         np.linspace(-87.33, 88.72, 5001)]).astype(np.float32)
    worst = max(_ulps(oracle.exp_spec(float(x)), math.exp(float(x))) for x in xs)
    assert worst <= 2.0


def test_exp_spec_special_values_and_range():
    assert oracle.exp_spec(0.0) == 1.0
    assert oracle.exp_spec(-0.0) == 1.0
    assert _ulps(oracle.exp_spec(1.0), math.e) <= 1.0
    for k in (-120, -60, -1, 1, 30, 120):
        x = float(np.float32(k * math.log(2.0)))
        assert _ulps(oracle.exp_spec(x), math.exp(x)) <= 2.0
    assert oracle.exp_spec(89.0) == math.inf and oracle.exp_spec(1e30) == math.inf
    assert oracle.exp_spec(-88.0) == 0.0 and oracle.exp_spec(-1e30) == 0.0
    assert math.isnan(oracle.exp_spec(float("nan")))
    # smallest non-flushed result is a normal binary32 number
    assert oracle.exp_spec(-87.33654022216797) >= 2.0 ** -126


def test_exp_spec_is_monotone_across_reduction_boundaries():
    # consecutive binary32 inputs around points where k = rint(x log2 e) changes
    for k in (-100, -3, -1, 0, 1, 7, 100):
        c = np.float32((k + 0.5) * math.log(2.0))
        xs = [c]
        for _ in range(200):
            xs.append(np.nextafter(xs[-1], np.float32(np.inf)))
        xs = [c] + xs
        lo = c
        for _ in range(200):
            lo = np.nextafter(lo, np.float32(-np.inf))
            xs.insert(0, lo)
        ys = [oracle.exp_spec(float(x)) for x in xs]
        assert all(b >= a for a, b in zip(ys, ys[1:]))


def test_sigmoid_spec_symmetry_and_range():
    assert oracle.sigmoid_spec(0.0) == 0.5
    rng = np.random.default_rng(1)
    for x in rng.uniform(-30, 30, 3000).astype(np.float32):
        s, t = oracle.sigmoid_spec(float(x)), oracle.sigmoid_spec(float(-x))
        assert 0.0 <= s <= 1.0
        assert abs(s + t - 1.0) <= 3 * 2.0 ** -24
        want = 1.0 / (1.0 + math.exp(-float(x)))
        assert abs(s - want) <= 3 * float(np.spacing(np.float32(want)))
    assert oracle.sigmoid_spec(200.0) == 1.0 and oracle.sigmoid_spec(-200.0) == 0.0


def test_activate_matches_the_drawn_values():
    sc = syn.blob_scene(3, n=500)
    act = oracle.activate(sc.as_raw())
    assert not act.raw
    for name in ("delta", "sigma", "opacity"):
        a, b = getattr(act, name).astype(np.float64), getattr(sc, name).astype(np.float64)
        assert np.all(np.abs(a - b) <= 4 * np.spacing(np.float32(b)).astype(np.float64))
    np.testing.assert_array_equal(act.points, sc.points)
    np.testing.assert_array_equal(act.sh, sc.sh)


def test_oracle_refuses_raw_scenes():
    with pytest.raises(ValueError, match="raw"):
        oracle.discrete(syn.blob_scene(0, n=10).as_raw(), syn.blob_camera())


def test_raw_gradients_match_finite_differences_in_raw_parameters():
    cam = syn.blob_camera(40, 40)
    sc = syn.blob_scene(11, n=30, radius=0.15, sh_degree=0)
    sc.points[..., :2] *= 0.3
    raw = sc.as_raw()
    st = oracle.settings()
    G = np.random.default_rng(2).uniform(-1, 1, (3, 40, 40))
    g = oracle.raw_gradients(raw, oracle.backward_image(oracle.activate(raw), cam, st, G))

    def loss(r):
        img = oracle.render_image(oracle.activate(r), cam, st)
        return float((img["image"] * G).sum()), img["n_contrib"]

    vis = np.nonzero(oracle.discrete(oracle.activate(raw), cam, st)["visible"])[0]
    checked = 0
    for i in vis[:10]:
        for name in ("delta", "sigma", "opacity"):
            h = 2e-3
            vals = []
            for s in (+1, -1):
                r = raw.copy()
                getattr(r, name)[i] = np.float32(getattr(raw, name)[i] + s * h)
                step = float(getattr(r, name)[i]) - float(getattr(raw, name)[i])
                vals.append(loss(r) + (step,))
            (lp, np_, hp), (lm, nm, hm) = vals
            if not (np_ == nm).all():
                continue
            fd = (lp - lm) / (hp - hm)
            a = float(g[name][i])
            scale = max(abs(a), abs(fd), 1e-4)
            # steps of 2e-3 in the raw value: O(h^2) truncation plus binary32 rounding of the
            # activated value (about 1e-7 relative, divided by h)
            assert abs(fd - a) <= 2e-3 * scale + 1e-6, (name, i, a, fd)
            checked += 1
    assert checked >= 15
