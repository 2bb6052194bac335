"""Gradients: the adjoint kernel (gbs_cumulants_backward) against the oracle's
gradient and central finite differences, the covariance model and its adjoint
against the numpy model and the oracle chain, and the autograd path used for
fitting r and eta to target cumulants. Tolerances: adjoint vs oracle gradient
relative 1e-10 (max abs difference over max abs entry); vs central differences
(step 1e-6) relative 1e-6."""
from math import comb

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


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("M,kmax,seed", [(5, 5, 1), (7, 5, 2), (10, 4, 3), (12, 3, 4), (9, 2, 5), (4, 1, 6),
                                         (23, 5, 7)])
def test_adjoint_matches_oracle_gradient(M, kmax, seed):
    inst = synthetic.random_instance(M, kmax, seed=seed, r_range=(0.3, 1.3), eta_range=(0.2, 0.7))
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(gbs.table_size(M, kmax))
    G = gbs.cumulants_backward(cuda(inst.V), kmax, cuda(g)).cpu().numpy()
    R = oracle.grad(inst.V, kmax, g)
    assert np.abs(G - G.T).max() <= 1e-12 * np.abs(R).max()
    assert np.abs(G - R).max() <= 1e-10 * np.abs(R).max()


def fit_problem():
    inst = synthetic.config(3)
    tgt = synthetic.fit_target(inst)
    return inst, tgt


def fit_loss_grad_kappa(kt, kt_target, M, kmax):
    w = gbs.fit_weights(M, kmax, device=kt.device)
    return 2.0 * w * (kt - kt_target)


def test_fit_gradient_m100_matches_oracle():
    """M=100, kmax=4: loss = sum_d C(M,d)^-1 sum_S (kt - kt*)^2; dL/dV from the
    adjoint against the oracle's gradient."""
    inst, tgt = fit_problem()
    M, K = inst.M, inst.kmax
    kt = gbs.cumulants(cuda(inst.V), K)
    kt_t = gbs.cumulants(cuda(tgt.V), K)
    g = fit_loss_grad_kappa(kt, kt_t, M, K)
    G = gbs.cumulants_backward(cuda(inst.V), K, g).cpu().numpy()
    R = oracle.grad(inst.V, K, g.cpu().numpy())
    assert np.abs(G - R).max() <= 1e-10 * np.abs(R).max()


def test_covariance_kernel_matches_model():
    inst = synthetic.config(3)
    U = torch.from_numpy(inst.U).cuda()
    V = gbs.covariance(U, cuda(inst.r), cuda(inst.eta)).cpu().numpy()
    assert np.abs(V - inst.V).max() <= 1e-12 * np.abs(inst.V).max()


@pytest.mark.parametrize("M,seed", [(20, 11), (3, 12), (37, 13)])
def test_covariance_adjoint_matches_oracle_chain(M, seed):
    inst = synthetic.random_instance(M, 3, seed=seed)
    rng = np.random.default_rng(seed - 9)
    G = rng.standard_normal((2 * M, 2 * M)); G = G + G.T
    U = torch.from_numpy(inst.U).cuda()
    dr, de = gbs.covariance_backward(U, cuda(inst.r), cuda(inst.eta), cuda(inst.V), cuda(G))
    rr, re = oracle.chain_to_params(G, inst.r, inst.eta, inst.U)
    np.testing.assert_allclose(dr.cpu().numpy(), rr, rtol=1e-10, atol=1e-10 * np.abs(rr).max())
    np.testing.assert_allclose(de.cpu().numpy(), re, rtol=1e-10, atol=1e-10 * np.abs(re).max())


def test_fit_gradient_wrt_parameters_matches_central_differences():
    """Full path r, eta -> V -> kt -> loss on M=100, kmax=4 through the autograd
    Functions; dL/dr_i and dL/deta_i against central differences of the forward."""
    inst, tgt = fit_problem()
    M, K = inst.M, inst.kmax
    U = torch.from_numpy(inst.U).cuda()
    kt_t = gbs.cumulants(cuda(tgt.V), K)
    w = gbs.fit_weights(M, K, device="cuda")

    def loss(r, eta):
        V = gbs.CovarianceFn.apply(r, eta, U)
        kt = gbs.CumulantFn.apply(V, K)
        return (w * (kt - kt_t) ** 2).sum()

    r = cuda(inst.r).requires_grad_(True)
    eta = cuda(inst.eta).requires_grad_(True)
    L = loss(r, eta)
    dr, de = torch.autograd.grad(L, (r, eta))
    h = 1e-6
    with torch.no_grad():
        for i in (0, 7, 49, 50, 99):
            for which, grad in (("r", dr), ("eta", de)):
                rp, rm = cuda(inst.r), cuda(inst.r)
                ep, em = cuda(inst.eta), cuda(inst.eta)
                if which == "r":
                    rp[i] += h; rm[i] -= h
                else:
                    ep[i] += h; em[i] -= h
                fd = (loss(rp, ep) - loss(rm, em)).item() / (2 * h)
                an = grad[i].item()
                assert an == pytest.approx(fd, rel=1e-6, abs=1e-6 * max(abs(fd), 1e-12) + 1e-14), (which, i, an, fd)


def test_adjoint_closed_form_single_squeezer():
    """L = P0({0}) of a squeezed vacuum: dL/dr = -tanh r / cosh r through both adjoints."""
    r0 = 0.7
    U = torch.eye(1, dtype=torch.complex128, device="cuda")
    r = torch.tensor([r0], dtype=torch.float64, device="cuda", requires_grad=True)
    eta = torch.tensor([1.0], dtype=torch.float64, device="cuda", requires_grad=True)
    V = gbs.CovarianceFn.apply(r, eta, U)
    kt = gbs.CumulantFn.apply(V, 1)
    (1.0 - kt[0]).backward()   # P0 = 1 - kt({0})
    assert r.grad.item() == pytest.approx(-np.tanh(r0) / np.cosh(r0), rel=1e-12)


@pytest.mark.parametrize("M,seed", [(1, 21), (7, 22), (16, 23), (37, 24)])
def test_covariance_kernel_ragged_tiles(M, seed):
    """The covariance kernel's 32 x 32 tiles: one partial tile, an exact fit
    (2M = 32) and a ragged edge over several tiles."""
    inst = synthetic.random_instance(M, 1, seed=seed, r_range=(0.2, 1.1), eta_range=(0.3, 0.9))
    U = torch.from_numpy(inst.U).cuda()
    V = gbs.covariance(U, cuda(inst.r), cuda(inst.eta)).cpu().numpy()
    assert np.abs(V - inst.V).max() <= 1e-12 * np.abs(inst.V).max()


def test_autograd_functions_defer_device_errors():
    """CumulantFn queues its device status instead of synchronising: a reduced
    covariance that is not positive definite gives NaN entries at once and a
    GbsError (not positive definite) from check_pending; a clean call after it
    leaves nothing pending."""
    inst = synthetic.random_instance(12, 3, seed=41)
    bad = cuda(inst.V).clone()
    bad[2, 2] = -5.0
    kt = gbs.CumulantFn.apply(bad, 3)  # no exception here
    assert torch.isnan(kt).any()
    with pytest.raises(gbs.GbsError) as err:
        gbs.check_pending()
    assert err.value.code == 2
    V = cuda(inst.V).requires_grad_(True)
    kt = gbs.CumulantFn.apply(V, 3)
    (g,) = torch.autograd.grad(kt.sum(), (V,))
    gbs.check_pending()
    assert torch.isfinite(g).all()
