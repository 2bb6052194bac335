"""Displaced Gaussian states (Eq. vacuum_gaussian_prob with first moments) through
gbs_displaced_tables, against the oracle's from-scratch entries.

Inputs: the generic lossy-interferometer instances with coherent displacements on
the inputs (synthetic.displaced_mean). Tolerances as for the zero-mean FP64 path:
P0 relative 1e-12, click moments and cumulants absolute 1e-12, spin tables
absolute 2^d x 1e-12. With zero mean the tables must equal the zero-mean entry
points bit for bit (the exponential factor is exactly exp(-0) = 1)."""
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


def order_of(M, kmax):
    return np.concatenate([np.full(gbs.table_size(M, d) - (gbs.table_size(M, d - 1) if d > 1 else 0), d)
                           for d in range(1, kmax + 1)])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("M,kmax,scale", [(12, 5, 0.6), (9, 4, 1.5), (6, 3, 0.3), (5, 5, 1.0)])
def test_all_tables_match_oracle(M, kmax, scale):
    inst = synthetic.random_instance(M, kmax, seed=700 + M)
    mean = synthetic.displaced_mean(inst, seed=900 + M, alpha_scale=scale)
    V, m = dev(inst.V), dev(mean)
    got = {t: gbs.displaced_tables(V, m, kmax, t).cpu().numpy() for t in gbs.TABLES}
    p0, mu, kt = oracle.tables_displaced(inst.V, mean, kmax)
    c, k = oracle.spin_tables_displaced(inst.V, mean, kmax)
    rel = np.abs(got["p0"] - p0) / np.abs(p0)
    assert rel.max() <= 1e-12, rel.max()
    assert np.abs(got["mu"] - mu).max() <= 1e-12
    assert np.abs(got["kappa"] - kt).max() <= 1e-12
    bound = 2.0 ** order_of(M, kmax) * 1e-12
    assert np.all(np.abs(got["spin_c"] - c) <= bound)
    assert np.all(np.abs(got["spin_kappa"] - k) <= bound)
    # the displacement matters: P0 differs from the zero-mean table
    p0_zero = gbs.vacuum_probs(V, kmax, "fp64").cpu().numpy()
    assert np.abs(got["p0"] - p0_zero).max() > 1e-3


def test_zero_mean_is_bit_identical_to_zero_mean_path():
    inst = synthetic.random_instance(30, 5, seed=31)
    V = dev(inst.V)
    z = torch.zeros(60, dtype=torch.float64, device="cuda")
    for t, f in (("p0", gbs.vacuum_probs), ("mu", gbs.click_moments), ("kappa", gbs.cumulants),
                 ("spin_c", gbs.spin_correlators), ("spin_kappa", gbs.spin_cumulants)):
        assert torch.equal(gbs.displaced_tables(V, z, 5, t), f(V, 5, "fp64")), t


@pytest.mark.parametrize("M", [40, 144])
def test_sampled_entries_several_tiles(M):
    """Orders 4 and 5 run on the prefix-tree kernels over many CTAs and batches:
    sampled entries against the oracle, every entry finite."""
    inst = synthetic.random_instance(M, 5, seed=4000 + M) if M != 144 else synthetic.config(2)
    mean = synthetic.displaced_mean(inst, seed=17 + M, alpha_scale=0.7)
    V, m = dev(inst.V), dev(mean)
    p0 = gbs.displaced_tables(V, m, 5, "p0")
    kt = gbs.displaced_tables(V, m, 5, "kappa")
    assert bool(torch.isfinite(p0).all()) and bool(torch.isfinite(kt).all())
    n = 2000 if M == 40 else 300
    for d in range(1, 6):
        sets = synthetic.random_subsets(M, d, n, seed=60 + d)
        idx = torch.tensor([gbs.order_offset(M, d) + gbs.rank(S) for S in sets], device="cuda")
        ref = oracle.entries_displaced(inst.V, mean, sets, want=("p0", "kappa"))
        g0, gk = p0[idx].cpu().numpy(), kt[idx].cpu().numpy()
        assert (np.abs(g0 - ref["p0"]) / ref["p0"]).max() <= 1e-12, d
        assert np.abs(gk - ref["kappa"]).max() <= 1e-12, d


def test_product_state_with_displacement():
    """No interferometer: displaced squeezed modes are independent, so every joint
    cumulant of order >= 2 vanishes and P0 factorises."""
    M, kmax = 10, 5
    rng = np.random.default_rng(5)
    inst = synthetic.make_instance(M, kmax, rng.uniform(0.2, 0.9, M), rng.uniform(0.3, 0.8, M), np.eye(M))
    mean = rng.normal(0, 0.8, 2 * M)
    V, m = dev(inst.V), dev(mean)
    p0 = gbs.displaced_tables(V, m, kmax, "p0").cpu().numpy()
    kt = gbs.displaced_tables(V, m, kmax, "kappa").cpu().numpy()
    assert np.abs(kt[M:]).max() <= 1e-13
    for d in range(2, kmax + 1):
        sets = oracle.enumerate_subsets(M, d)
        lo = gbs.order_offset(M, d)
        np.testing.assert_allclose(p0[lo:lo + len(sets)], np.prod(p0[:M][sets], axis=1), rtol=1e-13)


def test_invalid_arguments():
    inst = synthetic.random_instance(6, 3, seed=1)
    V = dev(inst.V)
    with pytest.raises(ValueError):
        gbs.displaced_tables(V, torch.zeros(11, dtype=torch.float64, device="cuda"), 3)
    with pytest.raises(ValueError):
        gbs.displaced_tables(V, torch.zeros(12, dtype=torch.float64, device="cuda"), 3, table="bogus")
    L = gbs.lib()
    ws = gbs.Workspace(6, 3)
    out = torch.empty(gbs.table_size(6, 3), dtype=torch.float64, device="cuda")
    import ctypes
    rc = L.gbs_displaced_tables(ctypes.c_void_p(V.data_ptr()), None, 6, 3, 2, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(ws.ptr), ws.nbytes, None)
    assert rc == 1 and b"mean" in L.gbs_last_error()
    m = torch.zeros(12, dtype=torch.float64, device="cuda")
    rc = L.gbs_displaced_tables(ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(m.data_ptr()), 6, 3, 7,
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.ptr), ws.nbytes, None)
    assert rc == 1 and b"table" in L.gbs_last_error()
