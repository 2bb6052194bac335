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
    assert e["grain"] in (1, 2, 4, 8) and e["ccap"] in (16, 24, 64) and e["variant"] in range(10)
    # a second process loads the file and reuses it (and still computes the same table)
    out2 = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True)
    assert out2.returncode == 0, out2.stderr


def test_pipe_peaks_probe():
    """The pipe probe reports rates a GB300-class part can reach: FP64 FMAs per
    clock per SM at most the nominal 2, FP32 at most the nominal 128, and the SM
    clock it ran at."""
    pk = gbs.pipe_peaks()
    assert 0.5 <= pk["fp64_fma_per_clk_per_sm"] <= 2.05
    assert 32 <= pk["fp32_fma_per_clk_per_sm"] <= 130
    assert 500 <= pk["sm_mhz_fp64_probe"] <= 2200 and 500 <= pk["sm_mhz_fp32_probe"] <= 2200
    assert pk["fp32_flops"] > 10 * pk["fp64_flops"]


PINNED = r"""
import sys, hashlib, json, torch
sys.path.insert(0, {root!r})
import synthetic, paper_2511_14923_gb300 as gbs
inst = synthetic.random_instance(40, 5, seed=12, r_range=(0.5, 1.4), eta_range=(0.3, 0.5))
t = gbs.cumulants(torch.from_numpy(inst.V).cuda(), 5, {prec!r})
print(hashlib.sha256(t.cpu().numpy().tobytes()).hexdigest())
print(json.dumps(gbs.schedule(40, 5, {prec!r})))
"""


@pytest.mark.parametrize("prec,variants", [("fp64", (0, 1)), ("fp32r", (0, 1, 2, 3, 4, 5, 6, 7, 8, 9))])
def test_every_cta_shape_gives_identical_table(tmp_path, prec, variants):
    """Each CTA shape, pinned through the cache file, fills the same table bit for bit."""
    digests = set()
    for v in variants:
        for grain, ccap in ((1, 16), (8, 64)):
            cache = tmp_path / f"pin_{prec}_{v}_{grain}.json"
            maj, mnr = torch.cuda.get_device_capability(0)
            cache.write_text(json.dumps([{"cc": 10 * maj + mnr, "sms": torch.cuda.get_device_properties(0).multi_processor_count,
                                          "M": 40, "kmax": 5, "precision": gbs.PRECISIONS[prec], "grain": grain,
                                          "ccap": ccap, "variant": v}]))
            env = dict(os.environ, GBS_AUTOTUNE_CACHE=str(cache))
            out = subprocess.run([sys.executable, "-c", PINNED.format(root=ROOT, prec=prec)], env=env,
                                 capture_output=True, text=True)
            assert out.returncode == 0, out.stderr
            digest, sched = out.stdout.strip().splitlines()
            digests.add(digest)
            # gbs_schedule reports the pinned schedule (the slot-free shape has room for 24 children)
            assert json.loads(sched) == {"variant": v, "grain": grain, "ccap": min(ccap, 24) if v == 9 else ccap}
    assert len(digests) == 1
