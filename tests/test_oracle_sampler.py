"""Pins of the stage-2 sampler oracle (oracle/sampler.c) against results fixed by
the paper's expansion and by exact distributions, independent of the oracle:

* Eq. probs_corr_cumulants_3 is exact when no cumulant is truncated and every
  marginal it uses is exact: the K = 3 single-elision sampler reproduces the
  Torontonian click distribution for M <= 3, the double-elision sampler for
  M <= K at K = 4 (orders 2, 2, 1) and K = 5 (orders 3, 3, 2);
* for a state made of independent blocks of consecutive modes, every cumulant
  that spans two blocks vanishes and the approximated marginals factorise:
  blocks of <= K modes give the exact product distribution at any M;
* the terms beyond the first are odd in the drawn bit, so the estimated
  probabilities of all 2^M bitstrings sum to 1;
* drawing with seeded uniforms reproduces the exact distribution's frequencies;
* the same exactness holds for displaced states, whose exact click distribution
  follows from their vacuum probabilities by inclusion-exclusion.
"""
import itertools

import numpy as np
import pytest

import oracle
import synthetic


def kappa_table(V, K):
    return oracle.spin_tables(V, K)[1]


def all_bits(M):
    return np.array(list(itertools.product([0, 1], repeat=M)), dtype=np.uint8)[:, ::-1].copy()


def tor_probs_of(bits, V):
    """Exact probabilities of bit rows (bit k = mode k) from the Torontonian route."""
    probs = oracle.torontonian_click_probs(V)
    idx = (bits.astype(np.int64) << np.arange(bits.shape[1])).sum(axis=1)
    return probs[idx]


def block_covariance(blocks):
    """xxpp covariance of independent blocks of consecutive modes."""
    M = sum(b.shape[0] // 2 for b in blocks)
    V = np.zeros((2 * M, 2 * M))
    o = 0
    for b in blocks:
        m = b.shape[0] // 2
        for (r0, r1), (c0, c1) in itertools.product([(0, m), (m, 2 * m)], repeat=2):
            R = slice(o + (M if r0 else 0), o + (M if r0 else 0) + m)
            C = slice(o + (M if c0 else 0), o + (M if c0 else 0) + m)
            V[R, C] = b[r0:r1, c0:c1]
        o += m
    return V


def sub_table(kap, M, K, n):
    """Spin-cumulant table of the first n modes: in colex order the subsets of
    {0..n-1} open every order group."""
    from math import comb
    parts, o = [], 0
    for d in range(1, K + 1):
        parts.append(kap[o:o + comb(n, d)])
        o += comb(M, d)
    return np.concatenate(parts)


@pytest.mark.parametrize("K", [3, 4, 5])
def test_exact_for_small_M(K):
    """M = K: nothing is truncated and every marginal the rules reach is exact."""
    inst = synthetic.random_instance(K, K, seed=300 + K, r_range=(0.5, 1.3))
    bits = all_bits(K)
    _, p, _ = oracle.sample(kappa_table(inst.V, K), K, K, force=bits)
    np.testing.assert_allclose(p, tor_probs_of(bits, inst.V), rtol=1e-10, atol=1e-14)


def exact_click_probs_displaced(V, mean, M):
    """All 2^M click probabilities of a displaced state by inclusion-exclusion over
    its vacuum probabilities: with Z the silent modes of x and C the clicking ones,
    p(x) = sum_{T subset of C} (-1)^{|T|} P0(Z + T), P0(empty) = 1."""
    cache = {}

    def P0(S):
        S = tuple(sorted(S))
        if not S:
            return 1.0
        if S not in cache:
            cache[S] = oracle.p0_displaced(V, mean, np.array(S))
        return cache[S]

    bits = all_bits(M)
    out = np.empty(len(bits))
    for r, x in enumerate(bits):
        Z = [k for k in range(M) if not x[k]]
        C = [k for k in range(M) if x[k]]
        out[r] = sum((-1) ** j * P0(Z + list(T)) for j in range(len(C) + 1) for T in itertools.combinations(C, j))
    return bits, out


@pytest.mark.parametrize("K", [3, 4, 5])
def test_exact_for_small_M_displaced(K):
    """A displaced state (first moments from coherent inputs): at M = K the sampler
    fed with the spin cumulants of its displaced tables reproduces the exact click
    distribution of the state."""
    inst = synthetic.random_instance(K, K, seed=400 + K, r_range=(0.5, 1.2))
    mean = synthetic.displaced_mean(inst, seed=40 + K, alpha_scale=0.8)
    kap = oracle.spin_tables_displaced(inst.V, mean, K)[1]
    bits, want = exact_click_probs_displaced(inst.V, mean, K)
    assert abs(want.sum() - 1.0) < 1e-12 and want.min() > -1e-15
    _, p, _ = oracle.sample(kap, K, K, force=bits)
    np.testing.assert_allclose(p, want, rtol=1e-10, atol=1e-14)


def test_exact_for_independent_displaced_blocks():
    """Independent displaced blocks of <= K consecutive modes: the K = 5 sampler
    gives the product of the blocks' exact click distributions."""
    rng = np.random.default_rng(515)
    sizes = (4, 5, 2)
    insts = [synthetic.random_instance(m, 1, seed=int(rng.integers(1 << 30)), r_range=(0.5, 1.2)) for m in sizes]
    means = [synthetic.displaced_mean(x, seed=int(rng.integers(1 << 30)), alpha_scale=0.7) for x in insts]
    V = block_covariance([x.V for x in insts])
    M = V.shape[0] // 2
    mean = np.concatenate([np.concatenate([m[:x.M] for m, x in zip(means, insts)]),
                           np.concatenate([m[x.M:] for m, x in zip(means, insts)])])
    kap = oracle.spin_tables_displaced(V, mean, 5)[1]
    bits = rng.integers(0, 2, (48, M)).astype(np.uint8)
    _, p, _ = oracle.sample(kap, M, 5, force=bits)
    want = np.ones(len(bits))
    o = 0
    for x, m in zip(insts, means):
        bb, pb = exact_click_probs_displaced(x.V, m, x.M)
        idx = (bits[:, o:o + x.M].astype(np.int64) << np.arange(x.M)).sum(axis=1)
        lookup = dict(zip((bb.astype(np.int64) << np.arange(x.M)).sum(axis=1), pb))
        want *= np.array([lookup[i] for i in idx])
        o += x.M
    np.testing.assert_allclose(p, want, rtol=1e-9)


@pytest.mark.parametrize("K,sizes", [(3, (3, 2, 3, 1)), (4, (4, 3, 4)), (5, (5, 2, 4))])
def test_exact_for_independent_blocks(K, sizes):
    rng = np.random.default_rng(sum(sizes) + K)
    blocks = [synthetic.random_instance(m, 1, seed=int(rng.integers(1 << 30)), r_range=(0.5, 1.3)).V for m in sizes]
    V = block_covariance(blocks)
    M = V.shape[0] // 2
    kap = kappa_table(V, K)
    bits = rng.integers(0, 2, (64, M)).astype(np.uint8)
    _, p, _ = oracle.sample(kap, M, K, force=bits)
    want = np.ones(len(bits))
    o = 0
    for b, m in zip(blocks, sizes):
        want *= tor_probs_of(np.ascontiguousarray(bits[:, o:o + m]), b)
        o += m
    np.testing.assert_allclose(p, want, rtol=1e-9)


@pytest.mark.parametrize("K,orders", [(3, None), (4, None), (5, None), (5, (2, 2, 1))])
def test_probabilities_sum_to_one(K, orders):
    inst = synthetic.random_instance(8, K, seed=81, r_range=(0.6, 1.4))
    bits = all_bits(8)
    _, p, q0 = oracle.sample(kappa_table(inst.V, K), 8, K, force=bits, orders=orders)
    assert abs(p.sum() - 1.0) < 1e-12
    assert np.all((q0 >= 0) & (q0 <= 1))


def test_draws_follow_exact_distribution_three_modes():
    inst = synthetic.random_instance(3, 3, seed=33, r_range=(0.6, 1.2))
    rng = np.random.default_rng(7)
    n = 60000
    bits, p, _ = oracle.sample(kappa_table(inst.V, 3), 3, 3, u=rng.random((n, 3)))
    freq = np.bincount((bits.astype(np.int64) << np.arange(3)).sum(axis=1), minlength=8) / n
    probs = oracle.torontonian_click_probs(inst.V)
    sigma = np.sqrt(probs * (1 - probs) / n)
    assert np.all(np.abs(freq - probs) <= 5 * sigma + 1e-12)
    # each drawn bitstring carries its exact probability
    np.testing.assert_allclose(p, tor_probs_of(bits, inst.V), rtol=1e-10)


def test_q0_is_the_conditional_of_the_scored_prefix():
    """The sampler's first n bits only see the first n modes: scoring the drawn
    prefix on the n-mode sub-table gives P[n], and q0 of bit n + 1 is
    P(prefix, 0) / P(prefix) whenever neither branch was clipped."""
    M, K = 9, 5
    inst = synthetic.random_instance(M, K, seed=71)
    kap = kappa_table(inst.V, K)
    rng = np.random.default_rng(1)
    bits, _, q0 = oracle.sample(kap, M, K, u=rng.random((3, M)))
    for s in range(3):
        for n in range(K, M):
            _, pre, _ = oracle.sample(sub_table(kap, M, K, n), n, K, force=bits[s:s + 1, :n])
            z = np.append(bits[s, :n], 0)[None, :].astype(np.uint8)
            _, pre0, _ = oracle.sample(sub_table(kap, M, K, n + 1), n + 1, K, force=z)
            if pre[0] > 0 and 0 < pre0[0] < pre[0]:
                assert q0[s, n] == pytest.approx(pre0[0] / pre[0], rel=1e-12)


def test_truncation_error_is_small_for_a_lossy_state():
    """Lossy eight-mode state: the estimated distribution stays close to the exact
    one (total-variation distance), closer at K = 5 than at K = 3."""
    inst = synthetic.random_instance(8, 5, seed=808, r_range=(0.5, 1.0), eta_range=(0.3, 0.5))
    bits = all_bits(8)
    exact = tor_probs_of(bits, inst.V)
    tv = {}
    for K in (3, 4, 5):
        _, p, _ = oracle.sample(kappa_table(inst.V, K), 8, K, force=bits)
        tv[K] = 0.5 * np.abs(p - exact).sum()
    assert tv[5] < 0.02 and tv[3] < 0.05
    assert tv[5] < tv[4] < tv[3]
