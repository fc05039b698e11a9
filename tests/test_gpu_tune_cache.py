"""The tuner's cache file (HPS_TUNE_CACHE): a process that measured the
kernel choices of a problem writes them, and another process reading the
same file measures nothing and builds with the same launch count (the same
choices); the solution is the same either way."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1812_07167_gb300 import hps
from paper_1812_07167_gb300 import workloads as W
pr = hps.Problem(8, 12, 30.0, 30.0, leaf_form=hps.HPS_LEAF_INVERSE)
c, s, t = W.random_data(8, 12, 30.0, 30.0, seed=5, nrhs=1)
st = torch.cuda.current_stream()
n = hps.hps_tune([pr], st)
h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
u = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), u, 1, st)
torch.cuda.synchronize()
print(json.dumps({{"tuned": n, "launches": h.info().build_launches, "u0": float(abs(u.cpu().numpy()).max())}}))
h.free()
"""


def _run(cache):
    env = dict(os.environ, HPS_TUNE_CACHE=cache)
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    import json
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_cached_choices_are_taken_by_another_process(tmp_path):
    cache = str(tmp_path / "tune.txt")
    first = _run(cache)
    assert first["tuned"] > 0
    lines = open(cache).read().split("\n")
    assert all(len(ln.split()) == 7 for ln in lines if ln.strip())
    second = _run(cache)
    assert second["tuned"] == 0
    assert second["launches"] == first["launches"]
    assert abs(second["u0"] - first["u0"]) <= 1e-12 * first["u0"]
