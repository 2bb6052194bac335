"""Ragged batches in one persistent launch: every instance's table equals the
single-instance call (identical arithmetic, so exactly equal) under the default
and the autotuned schedules, small instances match the oracle, the launch
replays from a CUDA graph after V changes in place, and the full 256-instance
workload (M up to 144, kmax up to 5) is checked the same way."""
import ctypes
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    gbs.build()


def ragged(n, seed, m_range=(5, 60)):
    rng = np.random.default_rng(seed)
    insts = []
    for i in range(n):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        k = int(min(rng.integers(1, 6), M))
        insts.append(synthetic.random_instance(M, k, seed=seed * 1000 + i, r_range=(0.4, 1.4), eta_range=(0.2, 0.6),
                                               n_squeezed=max(1, M // 2)))
    return insts


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("tuned", [False, True])
def test_batch_equals_single_instance_calls(precision, tuned):
    insts = ragged(24, 3)
    Vs = [torch.from_numpy(x.V).cuda() for x in insts]
    b = gbs.Batch(Vs, [x.kmax for x in insts], precision, autotune=tuned)
    sch = b.schedule()
    assert sch["ctas"] >= 152 and sch["grain"] in (1, 2, 4, 8) and sch["children_per_batch"] in (16, 64)
    if tuned:
        assert b.tune_ms > 0
        for o in b.outputs:
            o.fill_(float("nan"))  # the tuning runs wrote the tables already
    outs = b.run(check=True)
    for x, V, o in zip(insts, Vs, outs):
        ref = gbs.cumulants(V, x.kmax, precision)
        assert torch.equal(o, ref), (x.M, x.kmax, (o - ref).abs().max().item())


def test_batch_small_instances_match_oracle():
    insts = ragged(6, 5, m_range=(5, 14))
    b = gbs.Batch([torch.from_numpy(x.V).cuda() for x in insts], [x.kmax for x in insts], "fp32r")
    outs = b.run(check=True)
    for x, o in zip(insts, outs):
        ref = oracle.tables(x.V, x.kmax)[2]
        assert np.abs(o.cpu().numpy() - ref).max() <= 1e-12


def test_batch_graph_replay_tracks_inputs():
    insts = ragged(10, 7)
    Vs = [torch.from_numpy(x.V).cuda() for x in insts]
    b = gbs.Batch(Vs, [x.kmax for x in insts], "fp32r")
    b.capture()
    outs = [o.clone() for o in b.replay()]
    torch.cuda.synchronize()
    for x, V, o in zip(insts, Vs, outs):
        assert torch.equal(o, gbs.cumulants(V, x.kmax, "fp32r"))
    # new inputs written in place, same shapes: replay picks them up
    other = [synthetic.random_instance(x.M, x.kmax, seed=99 + i) for i, x in enumerate(insts)]
    for V, y in zip(Vs, other):
        V.copy_(torch.from_numpy(y.V))
    outs2 = b.replay()
    assert b.status() == 0
    for y, V, o in zip(other, Vs, outs2):
        assert torch.equal(o, gbs.cumulants(V, y.kmax, "fp32r"))


def test_batch_plan_rejects_bad_instances():
    V = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError):
        gbs.Batch([V], [6])


def test_batch_launch_needs_a_plan():
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    rc = gbs.lib().gbs_cumulants_batched(1, ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    assert rc == 1 and b"gbs_batched_plan" in gbs.lib().gbs_last_error()


def test_batch_autotune_is_recorded(tmp_path):
    """The batch schedule lands in the JSON cache and a new plan of the same
    batch shape (other covariances, instances in another order) picks it up."""
    path = tmp_path / "tune.json"
    os.environ["GBS_AUTOTUNE_CACHE"] = str(path)
    try:
        insts = ragged(8, 11, m_range=(20, 40))
        b = gbs.Batch([torch.from_numpy(x.V).cuda() for x in insts], [x.kmax for x in insts], "fp32r",
                      autotune=True)
        entries = json.loads(path.read_text())
        mine = [e for e in entries if "batch" in e and e["n"] == 8 and e["precision"] == 1]
        assert len(mine) == 1 and mine[0]["ms"] > 0
        other = [synthetic.random_instance(x.M, x.kmax, seed=500 + i) for i, x in enumerate(insts)][::-1]
        b2 = gbs.Batch([torch.from_numpy(x.V).cuda() for x in other], [x.kmax for x in other], "fp32r")
        for x, o in zip(other, b2.run(check=True)):
            assert torch.equal(o, gbs.cumulants(torch.from_numpy(x.V).cuda(), x.kmax, "fp32r"))
        del b, b2
    finally:
        del os.environ["GBS_AUTOTUNE_CACHE"]


@pytest.mark.parametrize("precision", ["fp32r", "fp64"])
def test_full_ragged_workload(precision):
    """The 256-instance workload (M~U{16..144}, kmax~U{2..5}, 5.4e9 subsets, 43 GB
    of tables): autotuned batch (refined) or default schedule (FP64) equal to the
    single-instance calls bit for bit, and every instance with M <= 20 equal to the
    oracle within the stated bounds."""
    insts = synthetic.batch_instances(256)
    assert max(x.M for x in insts) == 144 and max(x.kmax for x in insts) == 5
    Vs = [torch.from_numpy(x.V).cuda() for x in insts]
    b = gbs.Batch(Vs, [x.kmax for x in insts], precision, autotune=precision == "fp32r")
    outs = b.run(check=True)
    torch.cuda.synchronize()
    ws = {}
    small = 0
    for x, V, o in zip(insts, Vs, outs):
        key = (x.M, x.kmax)
        if key not in ws:
            ws[key] = gbs.Workspace(x.M, x.kmax, precision)
        ref = gbs.cumulants(V, x.kmax, precision, workspace=ws[key])
        assert torch.equal(o, ref), (x.M, x.kmax)
        if x.M <= 20:
            small += 1
            kt = oracle.tables(x.V, x.kmax)[2]
            assert np.abs(o.cpu().numpy() - kt).max() <= 1e-12, (x.M, x.kmax)
    assert small >= 3
    del b, outs
    torch.cuda.empty_cache()
