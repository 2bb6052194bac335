"""Spin-correlator and spin-cumulant tables (the paper's stage-1 outputs,
Eq. correlator_sum_cov and Eq. cumulant_corr_main) against the oracle. Both are
2^d-scaled relatives of the click tables (Eq. cumulant_exponential), so the
absolute bound for order d is 2^d x 1e-12; the spin-cumulant table must equal
(-2)^d times the click-cumulant table exactly for d >= 2."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu


def order_of(M, kmax):
    return np.concatenate([np.full(gbs.table_size(M, d) - gbs.table_size(M, d - 1) if d > 1 else M, d)
                           for d in range(1, kmax + 1)])


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("which", ["cfg0", "m12k5", "cfg1"])
def test_spin_tables_match_oracle(which, precision):
    inst = {"cfg0": lambda: synthetic.config(0), "cfg1": lambda: synthetic.config(1),
            "m12k5": lambda: synthetic.random_instance(12, 5, seed=1212, r_range=(0.5, 1.5))}[which]()
    V = torch.from_numpy(inst.V).cuda()
    c = gbs.spin_correlators(V, inst.kmax, precision).cpu().numpy()
    k = gbs.spin_cumulants(V, inst.kmax, precision).cpu().numpy()
    rc, rk = oracle.spin_tables(inst.V, inst.kmax)
    bound = 2.0 ** order_of(inst.M, inst.kmax) * 1e-12
    assert np.all(np.abs(c - rc) <= bound)
    assert np.all(np.abs(k - rk) <= bound)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_spin_cumulants_are_scaled_click_cumulants(precision):
    inst = synthetic.random_instance(40, 5, seed=4040, r_range=(0.6, 1.5), eta_range=(0.3, 0.5))
    V = torch.from_numpy(inst.V).cuda()
    k = gbs.spin_cumulants(V, 5, precision)
    kt = gbs.cumulants(V, 5, precision)
    for d in range(2, 6):
        lo, hi = gbs.order_offset(40, d), gbs.table_size(40, d)
        assert torch.equal(k[lo:hi], (-2.0) ** d * kt[lo:hi])
    assert torch.allclose(k[:40], 1.0 - 2.0 * kt[:40], rtol=0, atol=1e-15)


def test_spin_tables_m144_sampled():
    inst = synthetic.config(2)
    V = torch.from_numpy(inst.V).cuda()
    c = gbs.spin_correlators(V, 5, "fp32r")
    k = gbs.spin_cumulants(V, 5, "fp32r")
    for d in (3, 4, 5):
        sets = synthetic.random_subsets(144, d, 150, seed=500 + d)
        idx = torch.tensor([gbs.order_offset(144, d) + gbs.rank(S) for S in sets], device="cuda")
        gc, gk = c[idx].cpu().numpy(), k[idx].cpu().numpy()
        rc = np.array([oracle.spin_correlator(inst.V, S) for S in sets])
        rk = np.array([oracle.spin_cumulant(inst.V, S) for S in sets])
        assert np.abs(gc - rc).max() <= 2.0 ** d * 1e-12
        assert np.abs(gk - rk).max() <= 2.0 ** d * 1e-12
