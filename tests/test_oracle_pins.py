"""Pins for the CPU oracle: each test checks it against something other than
itself -- closed forms, textbook special cases, an independent formulation
(Torontonians, log of the moment generating polynomial), brute force on tiny
inputs, and invariants the paper states. CPU only."""
import itertools
from math import comb, cosh, exp, factorial, tanh

import numpy as np
import pytest

import oracle
import synthetic


# ------------------------------------------------------------------ helpers

def xxpp_from_blocks(blocks):
    """Direct sum of single-mode 2x2 covariances (x, p) laid out xxpp."""
    M = len(blocks)
    V = np.zeros((2 * M, 2 * M))
    for k, b in enumerate(blocks):
        idx = [k, k + M]
        V[np.ix_(idx, idx)] = b
    return V


def squeezed(r, phi=0.0):
    """Single-mode squeezed vacuum, hbar = 2, squeezing axis rotated by phi."""
    c, s = np.cos(phi), np.sin(phi)
    Rm = np.array([[c, -s], [s, c]])
    return Rm @ np.diag([exp(-2 * r), exp(2 * r)]) @ Rm.T


def thermal(nbar):
    return (2 * nbar + 1) * np.eye(2)


def tmsv(r):
    """Two-mode squeezed vacuum on modes (0, 1), xxpp, hbar = 2."""
    ch, sh = cosh(2 * r), np.sinh(2 * r)
    V = np.zeros((4, 4))
    V[np.ix_([0, 1], [0, 1])] = [[ch, sh], [sh, ch]]
    V[np.ix_([2, 3], [2, 3])] = [[ch, -sh], [-sh, ch]]
    return V


def moments_by_mask(V, S):
    d = len(S)
    mom = np.zeros(1 << d)
    mom[0] = 1.0
    for mask in range(1, 1 << d):
        mom[mask] = oracle.mu(V, [S[i] for i in range(d) if mask >> i & 1])
    return mom


# ------------------------------------------------------------------ determinants

def leibniz_det(a):
    n = a.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        p = 1.0
        for i in range(n):
            p *= a[i, perm[i]]
        tot += (-1) ** inv * p
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_det_matches_leibniz(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        a = rng.standard_normal((n, n))
        assert oracle.det(a) == pytest.approx(leibniz_det(a), rel=1e-11, abs=1e-12)


def test_det_needs_pivoting():
    # zero leading entry: fails without row exchanges
    a = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    assert oracle.det(a) == pytest.approx(leibniz_det(a), rel=1e-14)


# ------------------------------------------------------------------ closed forms (Eq. vacuum_gaussian_prob)

@pytest.mark.parametrize("r", [0.0, 0.3, 0.8, 1.6])
@pytest.mark.parametrize("phi", [0.0, 0.7])
def test_squeezed_vacuum_probability(r, phi):
    V = xxpp_from_blocks([squeezed(r, phi)])
    assert oracle.p0(V, [0]) == pytest.approx(1.0 / cosh(r), rel=1e-14)
    assert oracle.mu(V, [0]) == pytest.approx(1.0 - 1.0 / cosh(r), abs=1e-15)


@pytest.mark.parametrize("nbar", [0.0, 0.2, 1.5, 7.0])
def test_thermal_vacuum_probability(nbar):
    V = xxpp_from_blocks([thermal(nbar)])
    assert oracle.p0(V, [0]) == pytest.approx(1.0 / (1.0 + nbar), rel=1e-14)


@pytest.mark.parametrize("r", [0.2, 0.9])
def test_two_mode_squeezed_vacuum(r):
    """TMSV: perfectly correlated photon numbers, so P0({0}) = P0({1}) = P0({0,1})
    = 1/cosh^2 r, mu({0,1}) = tanh^2 r. Also pins the xxpp row selection."""
    V = tmsv(r)
    p = 1.0 / cosh(r) ** 2
    assert oracle.p0(V, [0]) == pytest.approx(p, rel=1e-14)
    assert oracle.p0(V, [1]) == pytest.approx(p, rel=1e-14)
    assert oracle.p0(V, [0, 1]) == pytest.approx(p, rel=1e-13)
    assert oracle.mu(V, [0, 1]) == pytest.approx(tanh(r) ** 2, rel=1e-13)
    t2 = tanh(r) ** 2
    assert oracle.kappa(V, [0, 1]) == pytest.approx(t2 - t2 * t2, rel=1e-12)


def test_vacuum_state():
    V = np.eye(8)
    for S in ([0], [1, 2], [0, 1, 3]):
        assert oracle.p0(V, S) == pytest.approx(1.0, abs=1e-15)
        assert oracle.mu(V, S) == pytest.approx(0.0, abs=1e-15)
        assert oracle.kappa(V, S) == pytest.approx(0.0, abs=1e-15)


def test_product_state_factorises():
    """Independent modes: P0 and mu factorise, cumulants of order >= 2 vanish."""
    rng = np.random.default_rng(5)
    blocks = []
    for k in range(5):
        b = squeezed(rng.uniform(0.2, 1.0), rng.uniform(0, 3))
        b = 0.6 * b + 0.4 * np.eye(2)  # loss keeps the state Gaussian and physical
        blocks.append(b)
    V = xxpp_from_blocks(blocks)
    singles_p0 = [oracle.p0(V, [k]) for k in range(5)]
    singles_mu = [oracle.mu(V, [k]) for k in range(5)]
    for d in range(2, 6):
        for S in itertools.combinations(range(5), d):
            assert oracle.p0(V, S) == pytest.approx(np.prod([singles_p0[k] for k in S]), rel=1e-13)
            assert oracle.mu(V, S) == pytest.approx(np.prod([singles_mu[k] for k in S]), rel=1e-11, abs=1e-15)
            assert abs(oracle.kappa(V, S)) < 1e-14


# ------------------------------------------------------------------ set partitions and the cumulant map

def test_bell_numbers_and_valid_partitions():
    for d, bell in zip(range(1, 7), [1, 2, 5, 15, 52, 203]):
        parts = oracle.set_partitions(d)
        assert parts.shape == (bell, d)
        canon = set()
        for lab in parts:
            # restricted growth string: first label 0, each new label at most one above the max so far
            assert lab[0] == 0
            for i in range(1, d):
                assert lab[i] <= lab[:i].max() + 1
            canon.add(tuple(lab))
        assert len(canon) == bell


@pytest.mark.parametrize("p", [0.1, 0.37, 0.5, 0.9])
def test_bernoulli_cumulants(p):
    """d copies of one Bernoulli(p) variable: every joint moment is p, and the joint
    cumulant is the d-th cumulant of Bernoulli(p) (textbook closed forms)."""
    closed = {
        1: p,
        2: p * (1 - p),
        3: p * (1 - p) * (1 - 2 * p),
        4: p * (1 - p) * (1 - 6 * p + 6 * p * p),
        5: p * (1 - p) * (1 - 2 * p) * (1 - 12 * p + 12 * p * p),
    }
    for d, want in closed.items():
        mom = np.full(1 << d, p)
        mom[0] = 1.0
        assert oracle.cumulant_from_moments(mom) == pytest.approx(want, abs=1e-15)


def _subset_conv(a, b, d):
    out = np.zeros(1 << d)
    for m in range(1 << d):
        s = m
        while True:
            out[m] += a[s] * b[m ^ s]
            if s == 0:
                break
            s = (s - 1) & m
    return out


def cumulant_via_log(mom, d):
    """kappa(S) = multilinear coefficient of u^S in log(sum_B mu(B) u^B): the
    log of the moment generating polynomial in the ring with u_i^2 = 0."""
    G = mom.copy()
    G[0] = 0.0
    acc = np.zeros(1 << d)
    P = np.zeros(1 << d); P[0] = 1.0
    for k in range(1, d + 1):
        P = _subset_conv(P, G, d)
        acc += ((-1) ** (k + 1) / k) * P
    return acc[(1 << d) - 1]


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_partition_sum_equals_log_generating_polynomial(d):
    rng = np.random.default_rng(100 + d)
    # a random joint distribution over d bits -> its moments
    p = rng.random(1 << d); p /= p.sum()
    mom = np.zeros(1 << d)
    for mask in range(1 << d):
        mom[mask] = sum(p[x] for x in range(1 << d) if (x & mask) == mask)
    assert oracle.cumulant_from_moments(mom) == pytest.approx(cumulant_via_log(mom, d), abs=1e-15)


def test_moments_from_cumulants_roundtrip():
    """Inverse relation (Eq. moments_cumulants_rel): mu(S) = sum_pi prod_b kappa(b)."""
    inst = synthetic.random_instance(7, 5, seed=11)
    S = [0, 2, 3, 5, 6]
    d = len(S)
    kap = np.zeros(1 << d)
    for mask in range(1, 1 << d):
        kap[mask] = oracle.kappa(inst.V, [S[i] for i in range(d) if mask >> i & 1])
    for mask in range(1, 1 << d):
        sub = [i for i in range(d) if mask >> i & 1]
        tot = 0.0
        for lab in oracle.set_partitions(len(sub)):
            prod = 1.0
            for b in range(lab.max() + 1):
                bm = 0
                for pos, l in enumerate(lab):
                    if l == b:
                        bm |= 1 << sub[pos]
                prod *= kap[bm]
            tot += prod
        assert tot == pytest.approx(oracle.mu(inst.V, [S[i] for i in sub]), rel=1e-12, abs=1e-15)


def test_spin_cumulant_identity():
    """Eq. cumulant_exponential: kappa(S) = (-2)^{|S|} kt(S) for |S| > 1 and
    1 - 2 mu for |S| = 1, with kappa from the correlators of Eq. correlator_sum_cov."""
    inst = synthetic.random_instance(6, 5, seed=12)
    V = inst.V
    assert oracle.spin_cumulant(V, [3]) == pytest.approx(1 - 2 * oracle.mu(V, [3]), abs=1e-15)
    for S in ([0, 4], [1, 2, 5], [0, 1, 3, 4], [0, 1, 2, 4, 5]):
        d = len(S)
        assert oracle.spin_cumulant(V, S) == pytest.approx((-2) ** d * oracle.kappa(V, S), rel=1e-10, abs=1e-14)


# ------------------------------------------------------------------ Torontonian brute force

@pytest.mark.parametrize("which", ["config0", "random6"])
def test_marginals_match_torontonian_distribution(which):
    """Full click distribution from Torontonians (independent of the xxpp
    determinant route): P0 and mu of every subset up to order 3 agree."""
    inst = synthetic.config(0) if which == "config0" else synthetic.random_instance(6, 3, seed=21)
    M = inst.M
    probs = oracle.torontonian_click_probs(inst.V)
    assert probs.sum() == pytest.approx(1.0, abs=1e-12)
    assert probs.min() > -1e-13
    p0t, mut, kt = oracle.tables(inst.V, 3)
    pos = 0
    for d in range(1, 4):
        for S in oracle.enumerate_subsets(M, d):
            a, b = oracle.marginals_from_probs(probs, M, S)
            assert p0t[pos] == pytest.approx(a, rel=1e-11)
            assert mut[pos] == pytest.approx(b, rel=1e-9, abs=1e-13)
            pos += 1


def test_cumulants_match_distribution_log_route():
    """Cumulants of the Torontonian distribution via the log of the moment
    generating polynomial agree with the oracle's partition sums."""
    inst = synthetic.random_instance(6, 4, seed=22)
    probs = oracle.torontonian_click_probs(inst.V)
    for S in ([0, 3], [1, 2, 4], [0, 2, 3, 5]):
        d = len(S)
        mom = np.zeros(1 << d)
        for mask in range(1 << d):
            sub = [S[i] for i in range(d) if mask >> i & 1]
            mom[mask] = oracle.marginals_from_probs(probs, inst.M, sub)[1] if sub else 1.0
        assert oracle.kappa(inst.V, S) == pytest.approx(cumulant_via_log(mom, d), abs=1e-12)


# ------------------------------------------------------------------ enumeration and ranks

@pytest.mark.parametrize("M", [1, 5, 9, 13])
def test_enumeration_is_colex(M):
    for d in range(1, min(M, 5) + 1):
        sets = oracle.enumerate_subsets(M, d)
        assert sets.shape == (comb(M, d), d)
        ref = sorted(itertools.combinations(range(M), d), key=lambda c: tuple(reversed(c)))
        assert [tuple(s) for s in sets] == ref
        for i, S in enumerate(sets):
            assert oracle.colex_rank(S) == i


# ------------------------------------------------------------------ table and entry routes agree

def test_tables_match_entries_from_scratch():
    inst = synthetic.random_instance(9, 4, seed=31)
    p0t, mut, kt = oracle.tables(inst.V, 4)
    pos = 0
    for d in range(1, 5):
        sets = oracle.enumerate_subsets(9, d)
        e = oracle.entries(inst.V, sets)
        n = len(sets)
        np.testing.assert_allclose(p0t[pos:pos + n], e["p0"], rtol=1e-14)
        np.testing.assert_allclose(mut[pos:pos + n], e["mu"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(kt[pos:pos + n], e["kappa"], rtol=0, atol=1e-15)
        pos += n


def test_order_one_entries():
    inst = synthetic.config(0)
    p0t, mut, kt = oracle.tables(inst.V, 1)
    np.testing.assert_allclose(mut, 1.0 - p0t, atol=1e-16)
    np.testing.assert_allclose(kt, mut, atol=1e-16)


def test_mode_permutation_covariance():
    inst = synthetic.random_instance(7, 3, seed=41)
    rng = np.random.default_rng(0)
    perm = rng.permutation(7)              # new mode i is old mode perm[i]
    idx = np.concatenate([perm, perm + 7])
    Vp = inst.V[np.ix_(idx, idx)]
    for S in ([0, 1], [2, 4, 6], [1, 3, 5]):
        old = sorted(perm[list(S)])
        assert oracle.kappa(Vp, S) == pytest.approx(oracle.kappa(inst.V, old), abs=1e-15)
        assert oracle.p0(Vp, S) == pytest.approx(oracle.p0(inst.V, old), rel=1e-14)


def test_moment_bounds_and_monotonicity():
    inst = synthetic.random_instance(8, 4, seed=51)
    for S in ([0, 1, 2, 3], [2, 5, 6, 7]):
        for d in range(1, 5):
            for sub in itertools.combinations(S, d):
                m = oracle.mu(inst.V, sub)
                assert -1e-15 <= m <= 1.0
                if d > 1:
                    assert m <= oracle.mu(inst.V, sub[:-1]) + 1e-15


# ------------------------------------------------------------------ gradients

def test_gradient_closed_form_single_squeezer():
    """L = P0({0}) of a squeezed mode: dL/dr = -tanh r / cosh r."""
    r = 0.7
    U = np.eye(1, dtype=complex)
    inst = synthetic.make_instance(1, 1, np.array([r]), np.array([1.0]), U)
    G = oracle.grad(inst.V, 1, np.array([-1.0]))   # kt({0}) = 1 - P0 -> dL/dkt = -1
    dr, _ = oracle.chain_to_params(G, inst.r, inst.eta, inst.U)
    assert dr[0] == pytest.approx(-tanh(r) / cosh(r), rel=1e-12)


def test_gradient_matches_central_differences():
    inst = synthetic.random_instance(5, 4, seed=61)
    M, k = 5, 4
    rng = np.random.default_rng(3)
    g = rng.standard_normal(oracle.table_size(M, k))
    G = oracle.grad(inst.V, k, g)
    assert np.allclose(G, G.T, atol=1e-13)
    h = 1e-6
    for (a, b) in [(0, 0), (1, 6), (3, 8), (7, 7), (2, 4)]:
        E = np.zeros_like(inst.V); E[a, b] += 1.0
        if a != b:
            E[b, a] += 1.0
        lp = g @ oracle.tables(inst.V + h * E, k)[2]
        lm = g @ oracle.tables(inst.V - h * E, k)[2]
        fd = (lp - lm) / (2 * h)
        an = G[a, b] + (G[b, a] if a != b else 0.0)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_parameter_chain_matches_central_differences():
    inst = synthetic.random_instance(4, 3, seed=71)
    rng = np.random.default_rng(4)
    G = rng.standard_normal(inst.V.shape); G = G + G.T
    dr, de = oracle.chain_to_params(G, inst.r, inst.eta, inst.U)
    h = 1e-6
    for i in range(4):
        e = np.zeros(4); e[i] = h
        fd_r = ((synthetic.covariance(inst.r + e, inst.eta, inst.U) - synthetic.covariance(inst.r - e, inst.eta, inst.U)) * G).sum() / (2 * h)
        fd_e = ((synthetic.covariance(inst.r, inst.eta + e, inst.U) - synthetic.covariance(inst.r, inst.eta - e, inst.U)) * G).sum() / (2 * h)
        assert dr[i] == pytest.approx(fd_r, rel=1e-6, abs=1e-8)
        assert de[i] == pytest.approx(fd_e, rel=1e-6, abs=1e-8)


# ------------------------------------------------------------------ stored values

def test_golden_config0_tables():
    """Regression anchor: tables for the M=8, kmax=3 workload written by
    tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "config0_tables.txt")
    data = np.loadtxt(path)
    inst = synthetic.config(0)
    p0t, mut, kt = oracle.tables(inst.V, 3)
    np.testing.assert_allclose(data[:, 0], p0t, rtol=1e-13)
    np.testing.assert_allclose(data[:, 1], mut, rtol=0, atol=1e-15)
    np.testing.assert_allclose(data[:, 2], kt, rtol=0, atol=1e-15)


def test_spin_tables_match_entries_and_identity():
    """Spin tables (lookup route) equal the from-scratch entries, and satisfy
    Eq. cumulant_exponential against the click tables: kappa = (-2)^d kt for
    d >= 2 and 1 - 2 mu for d = 1."""
    inst = synthetic.random_instance(8, 4, seed=91)
    c, k = oracle.spin_tables(inst.V, 4)
    _, mu, kt = oracle.tables(inst.V, 4)
    pos = 0
    for d in range(1, 5):
        sets = oracle.enumerate_subsets(8, d)
        for i, S in enumerate(sets):
            assert c[pos + i] == pytest.approx(oracle.spin_correlator(inst.V, S), abs=1e-14)
            assert k[pos + i] == pytest.approx(oracle.spin_cumulant(inst.V, S), abs=1e-13)
            want = 1 - 2 * mu[pos + i] if d == 1 else (-2) ** d * kt[pos + i]
            assert k[pos + i] == pytest.approx(want, abs=1e-12)
        pos += len(sets)
    # single mode: c({0}) = E[(-1)^x] = 2 P0 - 1
    V = xxpp_from_blocks([squeezed(0.6)])
    assert oracle.spin_tables(V, 1)[0][0] == pytest.approx(2.0 / cosh(0.6) - 1.0, abs=1e-15)


# ------------------------------------------------------------------ displaced states (Eq. vacuum_gaussian_prob, mu != 0)

@pytest.mark.parametrize("alpha", [0.0, 0.4 + 0.3j, -1.1j, 1.7])
def test_coherent_state_vacuum_probability(alpha):
    """Coherent state |alpha>: V = I, first moments (2 Re alpha, 2 Im alpha) for
    hbar = 2, vacuum probability exp(-|alpha|^2)."""
    V = np.eye(2)
    m = np.array([2 * alpha.real if isinstance(alpha, complex) else 2 * alpha,
                  2 * alpha.imag if isinstance(alpha, complex) else 0.0])
    assert oracle.p0_displaced(V, m, [0]) == pytest.approx(np.exp(-abs(alpha) ** 2), rel=1e-14)


def test_displaced_product_state_factorises_and_zero_mean_reduces():
    rng = np.random.default_rng(8)
    blocks = [0.7 * squeezed(rng.uniform(0.2, 1.0), rng.uniform(0, 3)) + 0.3 * np.eye(2) for _ in range(4)]
    V = xxpp_from_blocks(blocks)
    m = rng.normal(0, 0.8, 8)
    singles = [oracle.p0_displaced(V, m, [k]) for k in range(4)]
    for S in ([0, 1], [1, 2, 3], [0, 1, 2, 3]):
        assert oracle.p0_displaced(V, m, S) == pytest.approx(np.prod([singles[k] for k in S]), rel=1e-13)
    inst = synthetic.random_instance(6, 3, seed=17)
    for S in ([0], [1, 4], [0, 2, 5]):
        assert oracle.p0_displaced(inst.V, np.zeros(12), S) == pytest.approx(oracle.p0(inst.V, S), rel=1e-13)
    e = oracle.entries_displaced(V, m, np.array([[0, 1, 2]]))
    assert abs(e["kappa"][0]) < 1e-14  # independent modes: no joint cumulant


def test_displaced_thermal_closed_form():
    """Displaced thermal state: V = (2 nbar + 1) I, mean (x, p): the vacuum probability
    is exp(-(x^2 + p^2) / (4 (nbar + 1))) / (nbar + 1)."""
    for nbar, x, p in ((0.5, 1.0, -0.3), (2.0, -2.2, 0.7)):
        V = (2 * nbar + 1) * np.eye(2)
        want = np.exp(-(x * x + p * p) / (4 * (nbar + 1))) / (nbar + 1)
        assert oracle.p0_displaced(V, np.array([x, p]), [0]) == pytest.approx(want, rel=1e-14)


def _fock_two_mode_state(cut, r1, a1, r2, a2, theta, phi):
    """Two displaced squeezed vacua mixed on a beam splitter, built in a truncated
    Fock space by matrix exponentials of the ladder operators (no Gaussian
    formalism involved). Returns the state and the ladder operators."""
    from scipy.linalg import expm
    a = np.diag(np.sqrt(np.arange(1, cut)), 1).astype(complex)
    one = np.eye(cut)

    def mode(r, alpha):
        sq = expm(0.5 * r * (a @ a - a.conj().T @ a.conj().T))
        disp = expm(alpha * a.conj().T - np.conj(alpha) * a)
        v = np.zeros(cut, complex); v[0] = 1
        return disp @ sq @ v

    A, B = np.kron(a, one), np.kron(one, a)
    bs = expm(theta * (np.exp(1j * phi) * A.conj().T @ B - np.exp(-1j * phi) * A @ B.conj().T))
    psi = bs @ np.kron(mode(r1, a1), mode(r2, a2))
    return psi.reshape(cut, cut), (A, B)


def test_displaced_two_mode_state_matches_fock_space():
    """Eq. vacuum_gaussian_prob with first moments, against a state vector in Fock
    space: mean and covariance are measured from the state (x = a + a^dag,
    p = -i(a - a^dag), hbar = 2), vacuum probabilities are the squared amplitudes."""
    cut = 34
    psi, (A, B) = _fock_two_mode_state(cut, 0.35, 0.5 - 0.3j, 0.2, -0.4 + 0.2j, 0.7, 0.4)
    vec = psi.reshape(-1)
    quads = [A + A.conj().T, B + B.conj().T, -1j * (A - A.conj().T), -1j * (B - B.conj().T)]
    ev = lambda op: np.vdot(vec, op @ vec)
    m = np.array([ev(q).real for q in quads])
    V = np.array([[(0.5 * ev(qa @ qb + qb @ qa)).real - m[i] * m[j] for j, qb in enumerate(quads)]
                  for i, qa in enumerate(quads)])
    prob = np.abs(psi) ** 2
    assert oracle.p0_displaced(V, m, [0]) == pytest.approx(prob[0, :].sum(), rel=1e-9)
    assert oracle.p0_displaced(V, m, [1]) == pytest.approx(prob[:, 0].sum(), rel=1e-9)
    assert oracle.p0_displaced(V, m, [0, 1]) == pytest.approx(prob[0, 0], rel=1e-9)
    e = oracle.entries_displaced(V, m, np.array([[0, 1]]))
    click_both = prob.sum() - prob[0, :].sum() - prob[:, 0].sum() + prob[0, 0]
    assert e["mu"][0] == pytest.approx(click_both, rel=1e-9)
    q0, q1 = 1 - prob[0, :].sum(), 1 - prob[:, 0].sum()
    assert e["kappa"][0] == pytest.approx(click_both - q0 * q1, abs=1e-10)


def test_displaced_squeezed_single_mode_closed_form():
    """D(alpha) S(r)|0> with x squeezed (V = diag(e^{-2r}, e^{2r})): the Fock-basis
    overlap gives |<0|D S|0>|^2 = exp(-|alpha|^2 - tanh r Re(conj(alpha)^2)) / cosh r."""
    for r, alpha in ((0.4, 0.6 + 0.2j), (1.1, -0.3 + 0.9j), (0.0, 1.2j)):
        V = np.diag([np.exp(-2 * r), np.exp(2 * r)])
        m = np.array([2 * alpha.real, 2 * alpha.imag])
        want = np.exp(-abs(alpha) ** 2 - tanh(r) * (np.conj(alpha) ** 2).real) / cosh(r)
        assert oracle.p0_displaced(V, m, [0]) == pytest.approx(want, rel=1e-13)


def test_displaced_tables_consistent_with_fock_space_and_spin_identity():
    """Displaced tables: the spin correlator of the two-mode Fock-space state is
    E[(-1)^{x_0 + x_1}] summed from its photon-number distribution, and the spin
    cumulants of order >= 2 are (-2)^{|S|} times the click cumulants
    (Eq. cumulant_exponential)."""
    psi, _ = _fock_two_mode_state(34, 0.3, 0.2 + 0.4j, 0.25, -0.5, 0.9, -0.2)
    vec = psi.reshape(-1)
    cut = psi.shape[0]
    a = np.diag(np.sqrt(np.arange(1, cut)), 1).astype(complex)
    A, B = np.kron(a, np.eye(cut)), np.kron(np.eye(cut), a)
    quads = [A + A.conj().T, B + B.conj().T, -1j * (A - A.conj().T), -1j * (B - B.conj().T)]
    ev = lambda op: np.vdot(vec, op @ vec)
    m = np.array([ev(q).real for q in quads])
    V = np.array([[(0.5 * ev(qa @ qb + qb @ qa)).real - m[i] * m[j] for j, qb in enumerate(quads)]
                  for i, qa in enumerate(quads)])
    prob = np.abs(psi) ** 2
    click0 = np.ones(cut); click0[0] = 0
    s0 = 1 - 2 * click0  # (-1)^{x}: +1 for no click, -1 for a click
    c, k = oracle.spin_tables_displaced(V, m, 2)
    assert c[2] == pytest.approx(float(s0 @ prob @ s0), rel=1e-8)
    assert c[0] == pytest.approx(float(s0 @ prob.sum(axis=1)), rel=1e-8)
    inst = synthetic.random_instance(7, 3, seed=23)
    mean = np.random.default_rng(3).normal(0, 0.6, 14)
    _, _, kt = oracle.tables_displaced(inst.V, mean, 4)
    _, kk = oracle.spin_tables_displaced(inst.V, mean, 4)
    for d in range(2, 5):
        o, n = oracle.table_size(7, d) - comb(7, d), comb(7, d)
        np.testing.assert_allclose(kk[o:o + n], (-2.0) ** d * kt[o:o + n], rtol=1e-12, atol=1e-13)
