"""Ragged batches in one persistent launch: every instance's table equals the
single-instance call (identical arithmetic, so exactly equal), small instances
match the oracle, and the launch replays from a CUDA graph after V changes in
place."""
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
def test_batch_equals_single_instance_calls(precision):
    insts = ragged(24, 3)
    Vs = [torch.from_numpy(x.V).cuda() for x in insts]
    b = gbs.Batch(Vs, [x.kmax for x in insts], precision)
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
