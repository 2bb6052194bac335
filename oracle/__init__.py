"""CPU FP64 oracle for stage 1 of the emulator (arXiv:2511.14923).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use it; the library never does. It shares no code with
the CUDA path. The C part (``oracle.c``) computes the plain definitions
(LU determinants, inclusion-exclusion, explicit set partitions); this module
wraps it and adds two numpy pieces:

* ``torontonian_click_probs`` -- the full threshold-detection distribution of an
  M <= 10 mode state from Torontonians (App. "Benchmarking theory and
  implementation", Eq. ground_truth_prob_tor and Eq. torontonian_def), an
  independent route to the same marginals.
* ``chain_to_params`` -- dL/dV pulled back to squeezing r and transmissions eta
  through V = D S Q S^T D + I - D^2 (Eq. ground_truth_cov with per-mode loss).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "sampler.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c and sampler.c into liboracle.so with gcc (OpenMP if available)."""
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *_SRCS, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    lib.orc_det.argtypes = [D, ctypes.c_int]; lib.orc_det.restype = ctypes.c_double
    for f in ("orc_p0", "orc_mu", "orc_kappa", "orc_spin_correlator", "orc_spin_cumulant"):
        getattr(lib, f).argtypes = [D, ctypes.c_int, I, ctypes.c_int]
        getattr(lib, f).restype = ctypes.c_double
    lib.orc_set_partitions.argtypes = [ctypes.c_int, I, ctypes.c_int]; lib.orc_set_partitions.restype = ctypes.c_int
    lib.orc_cumulant_from_moments.argtypes = [D, ctypes.c_int]; lib.orc_cumulant_from_moments.restype = ctypes.c_double
    lib.orc_binom.argtypes = [ctypes.c_int, ctypes.c_int]; lib.orc_binom.restype = ctypes.c_uint64
    lib.orc_colex_rank.argtypes = [I, ctypes.c_int]; lib.orc_colex_rank.restype = ctypes.c_uint64
    lib.orc_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, I]; lib.orc_enumerate.restype = ctypes.c_int64
    lib.orc_entries.argtypes = [D, ctypes.c_int, ctypes.c_int, I, ctypes.c_int64, D, D, D]
    lib.orc_entries.restype = None
    lib.orc_tables.argtypes = [D, ctypes.c_int, ctypes.c_int, D, D, D]; lib.orc_tables.restype = ctypes.c_int
    lib.orc_grad.argtypes = [D, ctypes.c_int, ctypes.c_int, D, D]; lib.orc_grad.restype = ctypes.c_int
    lib.orc_spin_tables.argtypes = [D, ctypes.c_int, ctypes.c_int, D, D]; lib.orc_spin_tables.restype = ctypes.c_int
    lib.orc_spin_tables_from_p0.argtypes = [D, ctypes.c_int, ctypes.c_int, D, D]
    lib.orc_spin_tables_from_p0.restype = ctypes.c_int
    lib.orc_p0_displaced.argtypes = [D, D, ctypes.c_int, I, ctypes.c_int]; lib.orc_p0_displaced.restype = ctypes.c_double
    lib.orc_entries_displaced.argtypes = [D, D, ctypes.c_int, ctypes.c_int, I, ctypes.c_int64, D, D, D]
    lib.orc_entries_displaced.restype = None
    lib.orc_num_threads.argtypes = []; lib.orc_num_threads.restype = ctypes.c_int
    U8 = ctypes.POINTER(ctypes.c_uint8)
    lib.orc_sample_batch.argtypes = [D, ctypes.c_int, ctypes.c_int, I, ctypes.c_int64, D, U8, U8, D, D]
    lib.orc_sample_batch.restype = ctypes.c_int
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _V(V) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    assert V.ndim == 2 and V.shape[0] == V.shape[1] and V.shape[0] % 2 == 0
    return V


def _S(S) -> np.ndarray:
    return np.ascontiguousarray(S, dtype=np.int32)


def num_threads() -> int:
    return _load().orc_num_threads()


def table_size(M: int, kmax: int) -> int:
    return sum(comb(M, d) for d in range(1, kmax + 1))


def det(a) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return _load().orc_det(_dp(a), a.shape[0])


def p0(V, S) -> float:
    V = _V(V); S = _S(S)
    return _load().orc_p0(_dp(V), V.shape[0] // 2, _ip(S), S.size)


def mu(V, S) -> float:
    V = _V(V); S = _S(S)
    return _load().orc_mu(_dp(V), V.shape[0] // 2, _ip(S), S.size)


def kappa(V, S) -> float:
    V = _V(V); S = _S(S)
    return _load().orc_kappa(_dp(V), V.shape[0] // 2, _ip(S), S.size)


def spin_correlator(V, S) -> float:
    V = _V(V); S = _S(S)
    return _load().orc_spin_correlator(_dp(V), V.shape[0] // 2, _ip(S), S.size)


def spin_cumulant(V, S) -> float:
    V = _V(V); S = _S(S)
    return _load().orc_spin_cumulant(_dp(V), V.shape[0] // 2, _ip(S), S.size)


def set_partitions(d: int) -> np.ndarray:
    cap = 4140
    out = np.zeros(cap * max(d, 1), dtype=np.int32)
    n = _load().orc_set_partitions(d, _ip(out), cap)
    return out[: n * d].reshape(n, d)


def cumulant_from_moments(mom_by_mask) -> float:
    """mom_by_mask[mask] = joint moment of the variables in mask (index 0 unused)."""
    m = np.ascontiguousarray(mom_by_mask, dtype=np.float64)
    d = int(round(np.log2(m.size)))
    assert m.size == 1 << d
    return _load().orc_cumulant_from_moments(_dp(m), d)


def binom(n: int, k: int) -> int:
    return int(_load().orc_binom(n, k))


def colex_rank(S) -> int:
    S = _S(S)
    return int(_load().orc_colex_rank(_ip(S), S.size))


def enumerate_subsets(M: int, d: int) -> np.ndarray:
    n = comb(M, d)
    out = np.zeros(n * d, dtype=np.int32)
    got = _load().orc_enumerate(M, d, _ip(out))
    assert got == n
    return out.reshape(n, d)


def entries(V, sets, want=("p0", "mu", "kappa")):
    """Entries for each row of sets (sorted d-subsets), each from scratch."""
    V = _V(V); sets = _S(sets)
    n, d = sets.shape
    outs = {k: np.empty(n) for k in want}
    null = ctypes.POINTER(ctypes.c_double)()
    _load().orc_entries(_dp(V), V.shape[0] // 2, d, _ip(sets), n,
                        _dp(outs["p0"]) if "p0" in outs else null,
                        _dp(outs["mu"]) if "mu" in outs else null,
                        _dp(outs["kappa"]) if "kappa" in outs else null)
    return outs


def p0_displaced(V, mean, S) -> float:
    V = _V(V); S = _S(S)
    m = np.ascontiguousarray(mean, dtype=np.float64)
    return _load().orc_p0_displaced(_dp(V), _dp(m), V.shape[0] // 2, _ip(S), S.size)


def entries_displaced(V, mean, sets, want=("p0", "mu", "kappa")):
    """Displaced-state entries (Eq. vacuum_gaussian_prob with first moments) for each
    row of sets, each from scratch."""
    V = _V(V); sets = _S(sets)
    m = np.ascontiguousarray(mean, dtype=np.float64)
    n, d = sets.shape
    outs = {k: np.empty(n) for k in want}
    null = ctypes.POINTER(ctypes.c_double)()
    _load().orc_entries_displaced(_dp(V), _dp(m), V.shape[0] // 2, d, _ip(sets), n,
                                  _dp(outs["p0"]) if "p0" in outs else null,
                                  _dp(outs["mu"]) if "mu" in outs else null,
                                  _dp(outs["kappa"]) if "kappa" in outs else null)
    return outs


def tables_displaced(V, mean, kmax: int):
    """(P0, mu, kappa) tables of a displaced state, every entry from scratch."""
    M = _V(V).shape[0] // 2
    outs = [entries_displaced(V, mean, enumerate_subsets(M, d)) for d in range(1, kmax + 1)]
    return tuple(np.concatenate([o[k] for o in outs]) for k in ("p0", "mu", "kappa"))


def tables(V, kmax: int):
    """(P0, mu, kappa) tables over all subsets of order 1..kmax, colex order per order."""
    V = _V(V)
    M = V.shape[0] // 2
    N = table_size(M, kmax)
    a, b, c = np.empty(N), np.empty(N), np.empty(N)
    rc = _load().orc_tables(_dp(V), M, kmax, _dp(a), _dp(b), _dp(c))
    if rc != 0:
        raise ValueError("orc_tables rejected its arguments")
    return a, b, c


def spin_tables(V, kmax: int):
    """(c, kappa): spin-correlator table (Eq. correlator_sum_cov) and spin-cumulant
    table (Eq. cumulant_corr_main), orders 1..kmax, colex order per order."""
    V = _V(V)
    M = V.shape[0] // 2
    N = table_size(M, kmax)
    c, k = np.empty(N), np.empty(N)
    if _load().orc_spin_tables(_dp(V), M, kmax, _dp(c), _dp(k)) != 0:
        raise ValueError("orc_spin_tables rejected its arguments")
    return c, k


def spin_tables_displaced(V, mean, kmax: int):
    """(c, kappa) of a displaced state: the spin tables over its P0 table."""
    V = _V(V)
    M = V.shape[0] // 2
    p0 = tables_displaced(V, mean, kmax)[0]
    N = table_size(M, kmax)
    c, k = np.empty(N), np.empty(N)
    if _load().orc_spin_tables_from_p0(_dp(np.ascontiguousarray(p0)), M, kmax, _dp(c), _dp(k)) != 0:
        raise ValueError("orc_spin_tables_from_p0 rejected its arguments")
    return c, k


def grad(V, kmax: int, g_kappa) -> np.ndarray:
    """dL/dV (2M x 2M) for dL/dkappa = g_kappa (table layout)."""
    V = _V(V)
    M = V.shape[0] // 2
    g = np.ascontiguousarray(g_kappa, dtype=np.float64)
    assert g.size == table_size(M, kmax)
    out = np.empty((2 * M, 2 * M))
    rc = _load().orc_grad(_dp(V), M, kmax, _dp(g), _dp(out))
    if rc != 0:
        raise ValueError("orc_grad rejected its arguments")
    return out


# ------------------------------------------------------------------ Torontonian route

def torontonian(O: np.ndarray) -> complex:
    """tor(O) for a 2n x 2n matrix in (a, a^dagger) ordering: sum over R subset [n] of
    (-1)^{n-|R|} / sqrt(det(I - O_R)), where O_R keeps rows/cols k and k+n for k in R.
    The sign (-1)^{n-|R|} is the standard Torontonian (Quesada et al. 2018); the
    printed (-1)^{|R|} differs from it by (-1)^n and would make odd-click
    probabilities negative."""
    n = O.shape[0] // 2
    acc = 0.0 + 0.0j
    for mask in range(1 << n):
        R = [k for k in range(n) if mask >> k & 1]
        idx = R + [k + n for k in R]
        sub = O[np.ix_(idx, idx)] if idx else np.zeros((0, 0))
        dt = np.linalg.det(np.eye(len(idx)) - sub) if idx else 1.0
        acc += (-1) ** (n - len(R)) / np.sqrt(dt + 0j)
    return acc


def torontonian_click_probs(V) -> np.ndarray:
    """p(x) for every click pattern x in {0,1}^M (index = sum_k x_k 2^k), from
    p(x) = tor(O_(x)) / sqrt(det Sigma), Sigma = I/2 + R V R^dagger / 2 (hbar = 2),
    R = [[I, iI], [I, -iI]] / sqrt(2), O = I - Sigma^{-1}."""
    V = _V(V)
    M = V.shape[0] // 2
    I = np.eye(M)
    R = np.block([[I, 1j * I], [I, -1j * I]]) / np.sqrt(2.0)
    Sigma = 0.5 * np.eye(2 * M) + 0.5 * (R @ V @ R.conj().T)
    O = np.eye(2 * M) - np.linalg.inv(Sigma)
    norm = np.sqrt(np.linalg.det(Sigma) + 0j)
    probs = np.empty(1 << M)
    for mask in range(1 << M):
        C = [k for k in range(M) if mask >> k & 1]
        idx = C + [k + M for k in C]
        t = torontonian(O[np.ix_(idx, idx)]) if C else 1.0
        probs[mask] = (t / norm).real
    return probs


def marginals_from_probs(probs: np.ndarray, M: int, S):
    """(P0(S), mu(S)) from a full click distribution: probability that no mode
    of S clicks, and that every mode of S clicks."""
    m = 0
    for k in S:
        m |= 1 << int(k)
    idx = np.arange(1 << M)
    none = (idx & m) == 0
    allc = (idx & m) == m
    return float(probs[none].sum()), float(probs[allc].sum())


# ------------------------------------------------------------------ parameter chain

def chain_to_params(G: np.ndarray, r: np.ndarray, eta: np.ndarray, U: np.ndarray):
    """(dL/dr, dL/deta) from G = dL/dV through V = D W D + I - D^2,
    W = S Q S^T, Q = diag(e^{-2r}, e^{2r}), D = diag(sqrt(eta), sqrt(eta)).
      dV/dr_i   = D S (dQ/dr_i) S^T D,  dQ/dr_i = -2 e^{-2r_i} at (i,i), +2 e^{2r_i} at (i+M,i+M)
      dV/deta_m = W_ab (dD_a D_b + D_a dD_b) - delta_ab 2 D_a dD_a,  dD_a = [mode(a)=m] / (2 sqrt(eta_m))
    """
    M = U.shape[0]
    S = np.block([[U.real, -U.imag], [U.imag, U.real]])
    q = np.concatenate([np.exp(-2.0 * r), np.exp(2.0 * r)])
    dd = np.sqrt(np.concatenate([eta, eta]))
    W = (S * q[None, :]) @ S.T
    Gs = dd[:, None] * G * dd[None, :]
    H = S.T @ Gs @ S                      # H_kk = sum_ab G_ab D_a D_b S_ak S_bk
    dr = np.empty(M)
    for i in range(M):
        dr[i] = -2.0 * np.exp(-2.0 * r[i]) * H[i, i] + 2.0 * np.exp(2.0 * r[i]) * H[i + M, i + M]
    deta = np.empty(M)
    Gsym = G + G.T
    for m in range(M):
        tot = 0.0
        for a in (m, m + M):
            tot += (Gsym[a, :] * W[a, :] * dd).sum() / (2.0 * np.sqrt(eta[m]))
            tot -= G[a, a]
        deta[m] = tot
    return dr, deta


# ------------------------------------------------------------------ stage 2: chain-rule sampler

def sample(kappa, M: int, K: int, u=None, force=None, orders=None):
    """Chain-rule sampler (sampler.c): K = 3 single elision or K = 5 double
    elision, reading the spin-cumulant table kappa (orders 1..K, table layout).
    u: (ns, M) uniforms, or force: (ns, M) bits to score instead of drawing.
    orders: (p+, p1, p2) expansion orders for K = 5 (default the paper's 3, 3, 2).
    Returns (bits (ns, M) uint8, p (ns,) = estimated probability of each
    bitstring, q0 (ns, M) = probability of a 0 each bit was drawn with)."""
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    assert kappa.size == table_size(M, K)
    src = u if force is None else force
    ns = np.asarray(src).reshape(-1, M).shape[0]
    uu = None if u is None else np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(ns, M))
    ff = None if force is None else np.ascontiguousarray(np.asarray(force, dtype=np.uint8).reshape(ns, M))
    bits = np.empty((ns, M), dtype=np.uint8)
    p = np.empty(ns)
    q0 = np.empty((ns, M))
    U8 = ctypes.POINTER(ctypes.c_uint8)
    ordv = None if orders is None else np.ascontiguousarray(orders, dtype=np.int32)
    bad = _load().orc_sample_batch(_dp(kappa), M, K, None if ordv is None else _ip(ordv), ns,
                                   None if uu is None else _dp(uu),
                                   None if ff is None else ff.ctypes.data_as(U8),
                                   bits.ctypes.data_as(U8), _dp(p), _dp(q0))
    if bad:
        raise ValueError("orc_sample rejected its arguments")
    return bits, p, q0
