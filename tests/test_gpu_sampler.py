"""Chain-rule sampler on the GPU (gbs_sample) against the oracle (oracle/sampler.c),
on the same seeded uniforms.

FP64: the kernels sum in another order than the oracle, so probabilities agree
to rounding (log-probabilities within 1e-11) and every drawn bit is the oracle's (a
decision could only differ when u falls within ~1e-13 of q0). FP32 (the
precision the paper stores its tables in): each GPU decision is checked against
the oracle's q0 for the GPU's own bitstring (scored with forced bits) -- a bit
may differ from u < q0 only when |u - q0| < 2e-4 -- and the GPU's q0 and
log-probability agree with the oracle's within 2e-4 and 1e-3 absolute,
a bound from the FP32 unit roundoff (6e-8) times the few thousand terms of the
longest sums at these sizes."""
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


def kappa_of(inst, K):
    return gbs.spin_cumulants(torch.from_numpy(inst.V).cuda(), K, "fp64")


def uniforms(n, M, seed):
    return np.random.default_rng(seed).random((n, M))


@pytest.mark.parametrize("K,M,orders,n,batch", [(3, 12, None, 300, 128), (5, 14, None, 200, 128),
                                                (5, 13, (2, 2, 1), 130, 128), (5, 9, (3, 2, 1), 64, 128),
                                                (3, 3, None, 64, 128), (5, 5, None, 260, 128),
                                                (4, 12, None, 200, 128), (4, 10, (3, 3, 2), 128, 128),
                                                (4, 4, None, 64, 128)])
def test_fp64_draws_match_oracle(K, M, orders, n, batch):
    inst = synthetic.random_instance(M, K, seed=500 + M + K, r_range=(0.5, 1.3))
    kap = kappa_of(inst, K)
    u = uniforms(n, M, seed=M * 7 + K)
    bits, logp, q0 = gbs.sample(kap, M, K, u=torch.from_numpy(u).cuda(), orders=orders, batch=batch,
                                precision="fp64", want_q0=True)
    rb, rp, rq = oracle.sample(kap.cpu().numpy(), M, K, u=u, orders=orders)
    assert np.array_equal(bits.cpu().numpy(), rb)
    np.testing.assert_allclose(logp.cpu().numpy(), np.log(rp), rtol=0, atol=1e-11)
    assert np.abs(q0.cpu().numpy() - rq).max() <= 1e-12


@pytest.mark.parametrize("K", [3, 4, 5])
def test_fp64_scores_all_bitstrings(K):
    M = 9
    inst = synthetic.random_instance(M, K, seed=90 + K)
    kap = kappa_of(inst, K)
    allb = ((np.arange(1 << M)[:, None] >> np.arange(M)) & 1).astype(np.uint8)
    _, logp, _ = gbs.sample(kap, M, K, force=torch.from_numpy(allb).cuda(), batch=128, precision="fp64")
    _, rp, _ = oracle.sample(kap.cpu().numpy(), M, K, force=allb)
    p = np.exp(logp.cpu().numpy())
    np.testing.assert_allclose(p, rp, rtol=1e-11, atol=1e-17)
    assert abs(p.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("K,M", [(3, 24), (4, 22), (5, 20)])
def test_fp32_decisions_consistent_with_oracle(K, M):
    inst = synthetic.random_instance(M, K, seed=3200 + M, r_range=(0.6, 1.4), eta_range=(0.3, 0.5))
    kap = kappa_of(inst, K)
    n = 256
    u = uniforms(n, M, seed=11)
    bits, logp, q0 = gbs.sample(kap, M, K, u=torch.from_numpy(u).cuda(), batch=256, precision="fp32",
                                want_q0=True)
    b = bits.cpu().numpy()
    _, rp, rq = oracle.sample(kap.cpu().numpy(), M, K, force=b)
    tau = 2e-4
    assert np.abs(q0.cpu().numpy() - rq).max() <= tau
    np.testing.assert_allclose(logp.cpu().numpy(), np.log(rp), rtol=0, atol=1e-3)
    drawn_zero = b == 0
    assert np.all(np.where(drawn_zero, u < rq + tau, u >= rq - tau))


def test_fp32_m144_k5_consistent_on_a_few_samples():
    """The benchmark's M = 144 state: a handful of FP32 samples scored by the oracle."""
    inst = synthetic.config(2)
    kap = kappa_of(inst, 5)
    n = 64
    u = uniforms(n, 144, seed=144)
    bits, logp, q0 = gbs.sample(kap, 144, 5, u=torch.from_numpy(u).cuda(), batch=256, precision="fp32",
                                want_q0=True)
    assert bool(torch.isfinite(logp).all())
    b = bits.cpu().numpy()[:2]
    _, rp, rq = oracle.sample(kap.cpu().numpy(), 144, 5, force=b)
    tau = 2e-4
    assert np.abs(q0.cpu().numpy()[:2] - rq).max() <= tau
    np.testing.assert_allclose(logp.cpu().numpy()[:2], np.log(rp), rtol=0, atol=1e-3)
    assert np.all(np.where(b == 0, u[:2] < rq + tau, u[:2] >= rq - tau))


def test_fp32_k3_1152_modes():
    """K = 3 at the 1152-mode size of a 144-mode interferometer read out through 8
    time bins (a lossy 1152-mode instance of the same model): finite
    probabilities, and one sample scored by the oracle."""
    M = 1152
    inst = synthetic.random_instance(M, 3, seed=1152, r_range=(0.3, 0.9), eta_range=(0.2, 0.4), n_squeezed=576)
    kap = kappa_of(inst, 3)
    u = uniforms(128, M, seed=1152)
    bits, logp, q0 = gbs.sample(kap, M, 3, u=torch.from_numpy(u).cuda(), batch=256, precision="fp32",
                                want_q0=True)
    assert bool(torch.isfinite(logp).all())
    b = bits.cpu().numpy()[:1]
    _, rp, rq = oracle.sample(kap.cpu().numpy(), M, 3, force=b)
    tau = 2e-4
    assert np.abs(q0.cpu().numpy()[:1] - rq).max() <= tau
    np.testing.assert_allclose(logp.cpu().numpy()[:1], np.log(rp), rtol=0, atol=5e-3)
    assert np.all(np.where(b == 0, u[:1] < rq + tau, u[:1] >= rq - tau))


def test_invalid_arguments():
    inst = synthetic.random_instance(8, 5, seed=1)
    kap = kappa_of(inst, 5)
    u = torch.rand(4, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError):
        gbs.sample(kap, 8, 5, u=u, batch=64)
    with pytest.raises(gbs.GbsError):
        gbs.sample(kap, 8, 5, u=u, orders=(4, 3, 2))
    assert gbs.sampler_workspace_bytes(8, 6, 128) == 0
    assert gbs.sampler_workspace_bytes(4, 5, 128) == 0
    assert gbs.sampler_workspace_bytes(1025, 5, 128) == 0 and gbs.sampler_workspace_bytes(1152, 3, 128) > 0
    assert gbs.sampler_workspace_bytes(8, 5, 64) == 0
    assert gbs.sampler_workspace_bytes(8, 5, (1 << 21) + 128) == 0 and gbs.sampler_workspace_bytes(8, 5, 1 << 21) > 0


def test_fp32_tensor_core_product_matches_simt(monkeypatch):
    """FP32 calls run the step product on the tensor cores (tcgen05, 3-term TF32
    split); GBS_SAMPLER_SIMT=1 selects the CUDA-core product. Same uniforms: the
    log-probabilities agree to FP32 rounding and the decisions agree except within
    the q0 tolerance of the FP32 tests."""
    M, K = 40, 5
    inst = synthetic.random_instance(M, K, seed=4040, r_range=(0.6, 1.4), eta_range=(0.3, 0.5))
    kap = kappa_of(inst, K)
    u = torch.from_numpy(uniforms(256, M, seed=5)).cuda()
    b_tc, l_tc, q_tc = gbs.sample(kap, M, K, u=u, batch=256, precision="fp32", want_q0=True)
    monkeypatch.setenv("GBS_SAMPLER_SIMT", "1")
    b_s, l_s, q_s = gbs.sample(kap, M, K, u=u, batch=256, precision="fp32", want_q0=True)
    same = (b_tc == b_s).all(dim=1)
    assert float(same.float().mean()) > 0.9
    assert torch.abs(l_tc[same] - l_s[same]).max().item() <= 1e-3
    assert torch.abs(q_tc[same] - q_s[same]).max().item() <= 2e-4


def test_status_word_read_after_a_call(monkeypatch):
    """check=True reads the status word the sampler keeps in its workspace: GBS_OK
    after a normal call; GBS_ERR_TIMEOUT when the tensor-core step product's
    first wait runs out (host-side injection: the product issues no copies, so
    nothing is in flight when it gives up); afterwards the context is intact and
    a normal call reproduces the first call's bits."""
    inst = synthetic.random_instance(24, 5, seed=44)
    kap = kappa_of(inst, 5)
    u = torch.from_numpy(uniforms(256, 24, 9)).cuda()
    bits, logp, _ = gbs.sample(kap, 24, 5, u=u, batch=256, precision="fp32", check=True)
    monkeypatch.setenv("GBS_FAULT_INJECT", "sampler_no_loads")
    with pytest.raises(gbs.GbsError) as err:
        gbs.sample(kap, 24, 5, u=u, batch=256, precision="fp32", check=True)
    assert err.value.code == 4
    monkeypatch.delenv("GBS_FAULT_INJECT")
    bits2, logp2, _ = gbs.sample(kap, 24, 5, u=u, batch=256, precision="fp32", check=True)
    assert torch.equal(bits, bits2) and torch.equal(logp, logp2)
