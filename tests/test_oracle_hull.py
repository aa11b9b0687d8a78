"""Pins for the oracle's exact orientation predicate and Graham-scan hull (Sec. 3.2).

The references here are independent of the oracle: Python's exact rational arithmetic
(fractions.Fraction) for the orientation, and a brute-force O(K^3) hull (an edge i->j belongs to
the strictly convex hull iff every other point is strictly to its left or strictly inside the
segment).
"""
import itertools
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle


def orient_exact(a, b, c):
    ax, ay, bx, by, cx, cy = (Fraction(float(v)) for v in (*a, *b, *c))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def brute_hull(pts):
    """Canonical strictly convex hull: pivot (least v, then least u) first, increasing angle."""
    pts = [(float(np.float32(x)), float(np.float32(y))) for x, y in pts]
    keep = []
    for i, p in enumerate(pts):
        if all(pts[j] != p for j in range(i)):
            keep.append(i)
    if len(keep) < 3:
        return None
    F = {i: (Fraction(pts[i][0]), Fraction(pts[i][1])) for i in keep}

    def orient(i, j, m):
        (ax, ay), (bx, by), (cx, cy) = F[i], F[j], F[m]
        d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
        return (d > 0) - (d < 0)

    def strictly_inside(i, j, m):
        (ax, ay), (bx, by), (cx, cy) = F[i], F[j], F[m]
        t = (cx - ax) * (bx - ax) + (cy - ay) * (by - ay)
        return 0 < t < (bx - ax) ** 2 + (by - ay) ** 2

    nxt = {}
    for i, j in itertools.permutations(keep, 2):
        ok = True
        for m in keep:
            if m in (i, j):
                continue
            o = orient(i, j, m)
            if o < 0 or (o == 0 and not strictly_inside(i, j, m)):
                ok = False
                break
        if ok:
            nxt[i] = j
    if len(nxt) < 3:
        return None
    piv = min(nxt.keys(), key=lambda i: (pts[i][1], pts[i][0], i))
    cyc = [piv]
    while True:
        j = nxt[cyc[-1]]
        if j == piv:
            break
        cyc.append(j)
        assert len(cyc) <= len(keep)
    return cyc


def check(pts):
    got = oracle.hull2d(np.asarray(pts, np.float32))
    want = brute_hull(pts)
    if want is None:
        assert len(got) < 3, (pts, got)
    else:
        assert got == want, (pts, got, want)


def test_orient_matches_rationals_random():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        p = rng.uniform(-2000, 2000, 6).astype(np.float32)
        assert oracle.orient(p[0:2], p[2:4], p[4:6]) == orient_exact(p[0:2], p[2:4], p[4:6])


def test_orient_matches_rationals_near_degenerate():
    rng = np.random.default_rng(2)
    for _ in range(3000):
        a = rng.uniform(-1000, 1000, 2)
        b = rng.uniform(-1000, 1000, 2)
        t = rng.uniform(-2, 3)
        c = a + t * (b - a)  # collinear in reals, perturbed by float32 rounding
        a, b, c = (np.asarray(v, np.float32) for v in (a, b, c))
        if rng.uniform() < 0.3:
            c = np.nextafter(c, np.float32(np.inf) * np.sign(rng.uniform(-1, 1, 2)).astype(np.float32))
        assert oracle.orient(a, b, c) == orient_exact(a, b, c)


def test_orient_extreme_magnitudes():
    vals = [np.float32(v) for v in (1e-38, 1e-45, 3e38, -3e38, 1.0, 1 + 2 ** -23, 2 ** 20, -2 ** 20, 0.0, -0.0)]
    rng = random.Random(3)
    for _ in range(2000):
        p = [rng.choice(vals) for _ in range(6)]
        assert oracle.orient(p[0:2], p[2:4], p[4:6]) == orient_exact(p[0:2], p[2:4], p[4:6])


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8])
def test_hull_random_float_sets(k):
    rng = np.random.default_rng(10 + k)
    for _ in range(300):
        check(rng.uniform(-50, 50, (k, 2)).astype(np.float32))


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8])
def test_hull_integer_grid_degenerate_sets(k):
    """Points on a 4x4 integer grid: many collinear triples, duplicates and coincident pivots."""
    rng = np.random.default_rng(20 + k)
    for _ in range(400):
        check(rng.integers(0, 4, (k, 2)).astype(np.float32))


def test_hull_special_cases():
    # square with an interior point: the interior point never appears (points need not be vertices)
    sq = [(0, 0), (4, 0), (4, 4), (0, 4), (2, 2)]
    h = oracle.hull2d(np.asarray(sq, np.float32))
    assert sorted(h) == [0, 1, 2, 3] and 4 not in h
    # a point in the middle of an edge is dropped (strictly convex vertices only)
    h = oracle.hull2d(np.asarray([(0, 0), (2, 0), (4, 0), (2, 3)], np.float32))
    assert h == [0, 2, 3]
    # exact duplicates: the lowest index is kept
    h = oracle.hull2d(np.asarray([(1, 1), (0, 0), (3, 0), (0, 0), (1, 1), (1, 3)], np.float32))
    assert h == [1, 2, 5]  # (1, 1) is inside the triangle; its duplicate and the pivot's are dropped
    h = oracle.hull2d(np.asarray([(3, 0), (0, 0), (1, 3), (0, 0)], np.float32))
    assert h == [1, 0, 2]  # the pivot (0, 0) keeps its lowest index
    # all on a line: degenerate
    assert len(oracle.hull2d(np.asarray([(0, 0), (1, 1), (2, 2), (3, 3)], np.float32))) < 3
    # all coincident
    assert len(oracle.hull2d(np.asarray([(5, 5)] * 4, np.float32))) < 3
    # orientation: consecutive hull triples turn the same (positive) way
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = rng.uniform(0, 10, (6, 2)).astype(np.float32)
        h = oracle.hull2d(p)
        for i in range(len(h)):
            a, b, c = p[h[i]], p[h[(i + 1) % len(h)]], p[h[(i + 2) % len(h)]]
            assert orient_exact(a, b, c) > 0
