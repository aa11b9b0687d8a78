"""Writes the stored expected values under tests/golden/ by calling only the oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2411_14974_gb300 import synthetic as syn  # noqa: E402
from tests import _cases as C  # noqa: E402


def square():
    g = dict(a_px=8.0, z=4.0, f=128.0, delta=0.5, sigma=0.125, pixel=[63, 63])
    sc = C.square_scene(a_px=g["a_px"], z=g["z"], f=g["f"], delta=g["delta"], sigma=g["sigma"])
    cam = C.axis_camera(f=g["f"])
    st = oracle.settings(tau=0.0, alpha_max=1.0, t_min=0.0)
    r = oracle.render_pixels(sc, cam, st, np.array([g["pixel"]], np.int32))
    I = float(r["rgb"][0, 0]) / 0.5  # colour 0.5 (SH coefficients zero)
    g["I_centre"] = I
    g["phi_centre"] = float(np.log(1.0 / I - 1.0) / (g["z"] * g["sigma"]))
    g["source"] = ("Eq. 2 (LogSumExp of the scaled edge distances) and Eq. 3 (I = Sigmoid(-sigma phi)) "
                   "in their 2D form with the distance scaling of Eq. S1/S2; a square of half-width a "
                   "seen at its centre has L_t = -a for its 4 edges, so phi = -d delta a + ln 4.")
    return g


def blob_samples():
    sc, cams = syn.workload("blob1k_128", seed=0)
    rng = np.random.default_rng(123)
    pix = np.stack([rng.integers(0, 128, 64), rng.integers(0, 128, 64)], 1).astype(np.int32)
    r = oracle.render_pixels(sc, cams[0], oracle.settings(), pix)
    return dict(workload="blob1k_128", seed=0, pixels=pix.tolist(), rgb=r["rgb"].tolist(),
                t_final=r["t_final"].tolist(), last_id=r["last_id"].tolist(),
                source="oracle regression fixture (binary64 brute force, default settings)")


if __name__ == "__main__":
    with open(os.path.join(HERE, "square_indicator.json"), "w") as f:
        json.dump(square(), f, indent=1)
    with open(os.path.join(HERE, "blob1k_seed0_samples.json"), "w") as f:
        json.dump(blob_samples(), f)
    print("written")
