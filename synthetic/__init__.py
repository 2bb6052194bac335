"""Seeded synthetic inputs: zero-mean Gaussian covariances of lossy squeezed-light
interferometers (hbar = 2, xxpp ordering).

This module only draws random parameters and assembles the input covariance
V = D S Q S^T D + I - D^2 of the ground-truth model (App. "Benchmarking theory and
implementation", Eq. ground_truth_cov with a per-mode loss T = diag(sqrt(eta)) U);
it contains none of the stage-1 arithmetic (vacuum probabilities, moments,
cumulants). Both the CPU oracle and the CUDA library consume the arrays it returns.

Workload recipes (seed s_i = 20251114 + i, numpy PCG64):
  0: M=8,   kmax=3, r~U[0.3,0.8] on modes 0-3 (vacuum 4-7), Haar U, eta=0.5
  1: M=50,  kmax=4, r~U[0.5,1.2] on all modes, Haar U, eta=0.3
  2: M=144, kmax=5, r~U[0.8,1.6] on modes 0-71, Haar U, eta_i~U[0.3,0.5]
  3: M=100, kmax=4, r~U[0.5,1.2] on modes 0-49, Haar U, eta_i~U[0.3,0.6]
     (the fitting target uses the same U and r*, eta* drawn from seed s_3 + 1)
  4: 256 instances, M~U{16..144}, kmax~U{2..5}, r~U[0.5,1.5] on the first M//2
     modes, Haar U, eta_i~U[0.2,0.6]
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 20251114


@dataclass
class Instance:
    M: int
    kmax: int
    r: np.ndarray       # squeezing per input mode (0 = vacuum), length M
    eta: np.ndarray     # transmission per output mode, length M
    U: np.ndarray       # M x M complex unitary
    V: np.ndarray       # 2M x 2M float64 covariance, xxpp, hbar = 2

    @property
    def n_subsets(self) -> int:
        from math import comb
        return sum(comb(self.M, d) for d in range(1, self.kmax + 1))


def haar_unitary(M: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / np.sqrt(2.0)
    q, rr = np.linalg.qr(z)
    ph = np.diag(rr) / np.abs(np.diag(rr))
    return q * ph[None, :]


def covariance(r: np.ndarray, eta: np.ndarray, U: np.ndarray) -> np.ndarray:
    """V = D S Q S^T D + I - D^2 with S = [[Re U, -Im U], [Im U, Re U]],
    Q = diag(e^{-2r}, e^{+2r}) (x block then p block), D = diag(sqrt(eta), sqrt(eta))."""
    M = U.shape[0]
    S = np.block([[U.real, -U.imag], [U.imag, U.real]])
    q = np.concatenate([np.exp(-2.0 * r), np.exp(2.0 * r)])
    dd = np.sqrt(np.concatenate([eta, eta]))
    W = (S * q[None, :]) @ S.T
    V = dd[:, None] * W * dd[None, :] + np.diag(1.0 - dd * dd)
    return 0.5 * (V + V.T)


def make_instance(M: int, kmax: int, r: np.ndarray, eta: np.ndarray, U: np.ndarray) -> Instance:
    return Instance(M=M, kmax=kmax, r=r, eta=eta, U=U, V=covariance(r, eta, U))


def config(i: int) -> Instance:
    """Workload i (0..3) as listed in the module docstring."""
    rng = np.random.default_rng(BASE_SEED + i)
    if i == 0:
        M, kmax = 8, 3
        r = np.zeros(M); r[:4] = rng.uniform(0.3, 0.8, 4)
        U = haar_unitary(M, rng)
        eta = np.full(M, 0.5)
    elif i == 1:
        M, kmax = 50, 4
        r = rng.uniform(0.5, 1.2, M)
        U = haar_unitary(M, rng)
        eta = np.full(M, 0.3)
    elif i == 2:
        M, kmax = 144, 5
        r = np.zeros(M); r[:72] = rng.uniform(0.8, 1.6, 72)
        U = haar_unitary(M, rng)
        eta = rng.uniform(0.3, 0.5, M)
    elif i == 3:
        M, kmax = 100, 4
        r = np.zeros(M); r[:50] = rng.uniform(0.5, 1.2, 50)
        U = haar_unitary(M, rng)
        eta = rng.uniform(0.3, 0.6, M)
    else:
        raise ValueError("config index must be 0..3; use batch_instances() for the ragged batch")
    return make_instance(M, kmax, r, eta, U)


def fit_target(inst: Instance) -> Instance:
    """Target for the fitting workload: same interferometer, r* and eta* drawn
    from seed s_3 + 1 with the same ranges as workload 3."""
    rng = np.random.default_rng(BASE_SEED + 3 + 1)
    M = inst.M
    r = np.zeros(M); r[:50] = rng.uniform(0.5, 1.2, 50)
    eta = rng.uniform(0.3, 0.6, M)
    return make_instance(M, inst.kmax, r, eta, inst.U)


def batch_instances(n: int = 256, seed_offset: int = 4, m_range=(16, 144), k_range=(2, 5)) -> list[Instance]:
    """Ragged batch: M~U{m_range}, kmax~U{k_range}, r~U[0.5,1.5] on the first
    M//2 modes, Haar U, eta_i~U[0.2,0.6]."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    out = []
    for _ in range(n):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        kmax = int(rng.integers(k_range[0], k_range[1] + 1))
        kmax = min(kmax, M)
        r = np.zeros(M); r[: M // 2] = rng.uniform(0.5, 1.5, M // 2)
        U = haar_unitary(M, rng)
        eta = rng.uniform(0.2, 0.6, M)
        out.append(make_instance(M, kmax, r, eta, U))
    return out


def random_instance(M: int, kmax: int, seed: int, r_range=(0.3, 1.2), eta_range=(0.2, 0.7),
                    n_squeezed: int | None = None) -> Instance:
    """Small generic instance for tests (same model, arbitrary sizes)."""
    rng = np.random.default_rng(seed)
    ns = M if n_squeezed is None else n_squeezed
    r = np.zeros(M); r[:ns] = rng.uniform(*r_range, ns)
    U = haar_unitary(M, rng)
    eta = rng.uniform(*eta_range, M)
    return make_instance(M, kmax, r, eta, U)


def random_subsets(M: int, d: int, n: int, seed: int) -> np.ndarray:
    """n sorted d-subsets of {0..M-1}, each drawn uniformly (rows are independent).
    Vectorised rejection sampling: draw d modes, keep rows whose modes are distinct."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, d), dtype=np.int32)
    todo = np.arange(n)
    while todo.size:
        draw = np.sort(rng.integers(0, M, size=(todo.size, d)), axis=1)
        ok = np.all(np.diff(draw, axis=1) > 0, axis=1) if d > 1 else np.ones(todo.size, bool)
        out[todo[ok]] = draw[ok]
        todo = todo[~ok]
    return out


def displaced_mean(inst: Instance, seed: int, alpha_scale: float = 0.5) -> np.ndarray:
    """First moments (2M, xxpp, hbar = 2) of the instance's network fed with coherent
    displacements alpha_k ~ alpha_scale * (N(0,1) + i N(0,1)) / sqrt(2) on its inputs:
    the output amplitudes are sqrt(eta) * (U alpha), and mean = 2 (Re, Im) of them."""
    rng = np.random.default_rng(seed)
    alpha = alpha_scale * (rng.standard_normal(inst.M) + 1j * rng.standard_normal(inst.M)) / np.sqrt(2.0)
    beta = np.sqrt(inst.eta) * (inst.U @ alpha)
    return np.concatenate([2.0 * beta.real, 2.0 * beta.imag])
