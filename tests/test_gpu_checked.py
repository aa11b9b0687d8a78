"""The bounds-checked build (CS_CHECKED=1) through the C ABI.

That build tests, inside the kernels, every index an inconsistent upstream value could send out of
its buffer, skips the access, and reports the failed test through a device status word as
CS_ERR_DEVICE (no trap); it also hands out every transient buffer filled with 0xff bytes (NaN as
float).  (1) On consistent inputs it reports nothing and renders exactly what the production build
renders, so no buffer is read before it is written.  (2) A pair list made inconsistent on purpose
(one pair pointing past the records) makes the backward return CS_ERR_DEVICE, and the library
stays usable afterwards.  The checked library runs in a child process (one library per process).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2411_14974_gb300 import build as B
from paper_2411_14974_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2411_14974_gb300 import _binding, build
_binding.LIB = build.CHECKED_LIB
import paper_2411_14974_gb300 as cs
from paper_2411_14974_gb300 import synthetic as syn
from tests.test_gpu_checked import cases, run_case
out = {}
for name, sc, cams in cases():
    img, g = run_case(sc, cams)
    np.savez(sys.argv[2] + "_" + name + ".npz", img=img, **g)
# an inconsistent pair list: the last contributing pair of a covered pixel points past the records
sc, cams = cases()[0][1:]
t = cs.SceneTensors.from_numpy(sc, torch.device("cuda:0"))
_, _, state = cs.forward(t, cams, cs.Settings(), keep_state=True)
last = state.array("n_last").astype(np.int64)
i = int(last[last > 0][0]) - 1
n_rec = state.sizes()["records"]
_binding.check(_binding.lib().cs_debug_set_pair_value(state.handle, i, n_rec + 5), "cs_debug_set_pair_value")
G = torch.ones((len(cams), 3, cams[0].height, cams[0].width), device="cuda:0")
try:
    cs.backward(state, G)
    out["corrupt"] = "no error"
except _binding.CsError as e:
    out["corrupt"] = str(e)
state.release()
img, g = run_case(sc, cams)  # usable again, status cleared
out["after"] = bool(np.isfinite(img).all())
print(json.dumps(out))
'''


def cases():
    blob, cams = syn.workload("blob1k_128", seed=0)
    surf = syn.surface_scene(41, n=20_000, sh_degree=3)
    return [("blob", blob, cams), ("surface2", surf, syn.sphere_cameras(2, 160, 120, 4.0, seed=42))]


def run_case(sc, cams):
    import torch
    import paper_2411_14974_gb300 as cs
    t = cs.SceneTensors.from_numpy(sc, torch.device("cuda:0"))
    img, _, state = cs.forward(t, cams, cs.Settings(), keep_state=True)
    G = torch.as_tensor(np.random.default_rng(3).uniform(-1, 1, tuple(img.shape)).astype(np.float32), device="cuda:0")
    g = cs.backward(state, G)
    torch.cuda.synchronize()
    out = img.cpu().numpy(), {k: v.cpu().numpy() for k, v in g.items()}
    state.release()
    return out


@pytest.fixture(scope="module")
def checked_run(tmp_path_factory):
    B.build(checked=True)
    base = str(tmp_path_factory.mktemp("checked") / "out")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, base], capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return base, json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_is_silent_and_renders_like_production(checked_run):
    base, _ = checked_run
    for name, sc, cams in cases():
        img, g = run_case(sc, cams)
        got = np.load(base + "_" + name + ".npz")
        assert np.isfinite(got["img"]).all()
        assert np.abs(got["img"] - img).max() <= 1e-6, name
        for f, v in g.items():
            scale = np.abs(v).max() + 1e-30
            assert np.isfinite(got[f]).all(), (name, f)
            assert np.abs(got[f] - v).max() <= 1e-5 * scale, (name, f)  # atomics add in another order


def test_checked_build_reports_an_inconsistent_pair_list(checked_run):
    _, out = checked_run
    assert "status 6" in out["corrupt"] and "device status 0x2" in out["corrupt"], out["corrupt"]
    assert out["after"]
