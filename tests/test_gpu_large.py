"""Edge sizes: tables with more than 2^31 entries (64-bit indices), large M for
the prefix-tree kernel, and the largest M the ABI accepts (1024 modes with
kmax >= 4; 4096 with kmax <= 3). Each table stays on
the device; a seeded sample of entries (including entries above index 2^31) is
gathered there and compared with entries the oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu
TOL = {"fp64": (1e-12, 1e-12), "fp32r": (1e-11, 1e-12)}


def check_sample(V_np, table, M, d, n, seed, which, precision, min_rank=0):
    rng = np.random.default_rng(seed)
    sets = synthetic.random_subsets(M, d, n, seed)
    ranks = np.array([gbs.rank(S) for S in sets], dtype=np.int64)
    if min_rank:
        # also entries with ranks above min_rank
        assert min_rank < gbs.table_size(M, d) - gbs.order_offset(M, d), "no entry of that order has such a rank"
        hi = []
        while len(hi) < n // 2:
            S = np.sort(rng.choice(M, d, replace=False))
            if gbs.rank(S) >= min_rank:
                hi.append(S)
        sets = np.concatenate([sets, np.array(hi, dtype=np.int32)])
        ranks = np.array([gbs.rank(S) for S in sets], dtype=np.int64)
    idx = torch.from_numpy(gbs.order_offset(M, d) + ranks).cuda()
    got = table[idx].cpu().numpy()
    ref = oracle.entries(V_np, sets, want=(which,))[which]
    rel, ab = TOL[precision]
    if which == "p0":
        assert np.abs(got / ref - 1).max() <= rel
    else:
        assert np.abs(got - ref).max() <= ab
    return idx.max().item()


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_table_beyond_2_31_entries(precision):
    M, K = 200, 5
    inst = synthetic.random_instance(M, K, seed=2001, r_range=(0.6, 1.4), eta_range=(0.3, 0.5), n_squeezed=100)
    V = torch.from_numpy(inst.V).cuda()
    N = gbs.table_size(M, K)
    assert N > 2**31
    kt = gbs.cumulants(V, K, precision)
    top = check_sample(inst.V, kt, M, 5, 4000, 7, "kappa", precision, min_rank=2**31 - gbs.order_offset(M, 5))
    assert top >= 2**31
    check_sample(inst.V, kt, M, 4, 2000, 8, "kappa", precision)
    del kt
    p0 = gbs.vacuum_probs(V, K, precision)
    check_sample(inst.V, p0, M, 5, 2000, 9, "p0", precision, min_rank=2**31 - gbs.order_offset(M, 5))


def test_large_modes_prefix_tree():
    M, K = 600, 4
    inst = synthetic.random_instance(M, K, seed=6001, r_range=(0.4, 1.2), eta_range=(0.2, 0.5), n_squeezed=300)
    V = torch.from_numpy(inst.V).cuda()
    kt = gbs.cumulants(V, K, "fp32r")
    check_sample(inst.V, kt, M, 4, 3000, 11, "kappa", "fp32r")
    check_sample(inst.V, kt, M, 3, 1000, 12, "kappa", "fp32r")
    del kt
    mu = gbs.click_moments(V, K, "fp64")
    check_sample(inst.V, mu, M, 4, 2000, 13, "mu", "fp64")


def test_maximum_modes_prefix_tree_orders():
    """kmax >= 4 (prefix-tree kernels) accepts up to 1024 modes."""
    with pytest.raises(gbs.GbsError):
        gbs.cumulants(torch.eye(2 * 1025, dtype=torch.float64, device="cuda"), 4)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_thousands_of_modes_low_orders(precision):
    """kmax <= 3 runs without the prefix-tree kernels and accepts up to 4096
    modes: M = 2048 with kmax = 3 (1.43e9 entries)."""
    M, K = 2048, 3
    inst = synthetic.random_instance(M, K, seed=2048, r_range=(0.3, 1.0), eta_range=(0.2, 0.5), n_squeezed=1024)
    V = torch.from_numpy(inst.V).cuda()
    kt = gbs.cumulants(V, K, precision)
    check_sample(inst.V, kt, M, 3, 3000, 21, "kappa", precision)
    check_sample(inst.V, kt, M, 2, 1000, 22, "kappa", precision)
    check_sample(inst.V, kt, M, 1, 200, 23, "kappa", precision)


def test_maximum_modes_low_orders():
    """M = 4096, kmax = 2 (the largest M accepted): a state of independent
    8-mode blocks, sampled entries within and across blocks; 4097 modes are
    rejected."""
    M, b = 4096, 8
    blocks = [synthetic.random_instance(b, 2, seed=40 + k % 16).V for k in range(M // b)]
    V = np.zeros((2 * M, 2 * M))
    for k, B in enumerate(blocks):
        o = k * b
        for r0 in (0, 1):
            for c0 in (0, 1):
                V[r0 * M + o:r0 * M + o + b, c0 * M + o:c0 * M + o + b] = B[r0 * b:(r0 + 1) * b, c0 * b:(c0 + 1) * b]
    Vd = torch.from_numpy(V).cuda()
    p0 = gbs.vacuum_probs(Vd, 2, "fp64")
    check_sample(V, p0, M, 2, 2000, 31, "p0", "fp64")
    check_sample(V, p0, M, 1, 500, 32, "p0", "fp64")
    sets = np.array([[8 * k, 8 * k + 3] for k in range(0, 512, 7)], dtype=np.int32)  # pairs within a block
    idx = torch.tensor([gbs.order_offset(M, 2) + gbs.rank(S) for S in sets], device="cuda")
    ref = oracle.entries(V, sets, want=("p0",))["p0"]
    assert np.abs(p0[idx].cpu().numpy() / ref - 1).max() <= 1e-12
    del p0, Vd
    with pytest.raises(gbs.GbsError):
        gbs.cumulants(torch.eye(2 * 4097, dtype=torch.float64, device="cuda"), 2)
