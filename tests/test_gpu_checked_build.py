"""The bounds-checked build (-DCTS_BOUNDS_CHECK) on the GPU: on valid inputs its
index checks never fire, so every launch path gives exactly what the default
build gives.  The checked library runs in a child process (CTS_CHECKED=1
selects it when the package loads); no case here plants an out-of-range
index on the device."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    # (preset, events, first id, mode, field, keep_induced)
    ("plain_3keV_100um", 4, 500, cts.CTS_MODE_BATCHED, None, 3),
    ("plain_3keV_100um", 2, 510, cts.CTS_MODE_PLAIN, None, 3),
    ("plain_3keV_100um", 2, 520, cts.CTS_MODE_BATCHED, dict(spherical=1), 3),
    ("batch_20keV_320um", 2, 530, cts.CTS_MODE_BATCHED, None, 0),
    ("mip_50um", 1, 540, cts.CTS_MODE_SERVE, None, 1),
]

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_2506_09712_gb300 as cts
import workloads as W
from tests.test_gpu_checked_build import CASES, run_case
assert cts.sim_build_flags() == cts.SIM_BUILD_BOUNDS_CHECK
print(json.dumps([run_case(*c) for c in CASES]))
"""


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09712_gb300 import build
    build.build()
    build.build(checked=True)
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_case(name, n, first, mode, field, flags):
    p = W.preset(name)
    fld = W.field_switches(**field) if field else None
    evs = W.make_events(name, n=n, first_id=first)
    with cts.Simulator(p["sensor"], p["mobility"], fld, mode=mode, keep_induced=flags) as sim:
        got = sim.run(evs, induced_capacity=8192 if flags else 0)
    out = []
    for d in got:
        out.append(dict(status=int(d["status"]), n_steps=int(d["n_steps"]),
                        pixels=d["pixels"].tolist(), n_lost=int(d["n_lost"]),
                        induced=None if d["induced"] is None else d["induced"][-1:].tolist(),
                        induced_px=(None if d["induced_px"] is None
                                    else d["induced_px"][-1].ravel().tolist())))
    return out


def test_checked_build_matches_the_default_build():
    assert cts.sim_build_flags() == 0
    env = dict(os.environ, CTS_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-4000:]
    checked = json.loads(r.stdout.strip().splitlines()[-1])
    for case, got in zip(CASES, checked):
        ref = run_case(*case)
        assert len(got) == len(ref)
        for a, b in zip(got, ref):
            assert a["status"] == b["status"] == 0, case
            assert a["n_steps"] == b["n_steps"], case
            assert a["pixels"] == b["pixels"], case
            assert a["n_lost"] == b["n_lost"], case
            for key in ("induced", "induced_px"):
                if b[key] is not None:
                    assert np.allclose(a[key], b[key], rtol=1e-9, atol=1e-9), (case, key)
