/*
 * CPU FP64 oracle for stage 1 of the Gaussian boson sampling emulator
 * (arXiv:2511.14923): vacuum probabilities, click moments and click cumulants
 * of a zero-mean Gaussian state over every mode subset of size <= kmax.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library calls this file: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it. It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (the paper keeps hbar general; here hbar = 2):
 *   V       2M x 2M covariance, row-major, xxpp: mode k owns rows/cols k and k+M.
 *   V_T     keep rows/cols k and k+M for k in T  (reduction rule, App. "Correlators
 *           of GBS with binary outcomes", text before Eq. vacuum_gaussian_prob).
 *   P0(T)   <0_T|rho_T|0_T> = det[(V_T + I)/2]^{-1/2}  (Eq. vacuum_gaussian_prob with
 *           zero mean and hbar = 2); P0(empty) = 1.
 *   mu(S)   p(x_k = 1 for all k in S)  (Eq. joint_moments_def, Eq.
 *           joint_moments_threshold) = Tr[rho prod_{k in S}(I - |0_k><0_k|)]
 *           = sum_{T subset S} (-1)^{|T|} P0(T)  (expanding the product the same way
 *           as Eq. corr_oper_reexpressed).
 *   kt(S)   click cumulant, sum over set partitions pi of S of
 *           (-1)^{|pi|-1} (|pi|-1)! prod_{b in pi} mu(b)  (Eq. joint_cumulants_def).
 *   c(S)    spin correlator (-1)^{|S|} sum_{R subset S} (-2)^{|R|} P0(R)
 *           (Eq. correlator_sum_cov); kappa(S) its cumulant (Eq. cumulant_corr_main).
 *   Tables  ordered by order d = 1..kmax, and within an order by colex rank,
 *           generated here by nested loops (largest element outermost).
 *
 * Every routine computes the plain definition: determinants by LU with partial
 * pivoting, inclusion-exclusion by looping over subsets, cumulants by explicitly
 * enumerating set partitions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 8          /* largest subset order the oracle handles */
#define ORC_MAXN (2 * ORC_MAXD)

/* ---------------------------------------------------------------- linear algebra */

/* det(a) for an n x n row-major matrix by LU with partial pivoting; a is destroyed. */
static double det_lu(double *a, int n) {
    double det = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
        if (best == 0.0) return 0.0;
        if (p != k) {
            for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
            det = -det;
        }
        double piv = a[k * n + k];
        det *= piv;
        for (int i = k + 1; i < n; ++i) {
            double f = a[i * n + k] / piv;
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
        }
    }
    return det;
}

/* inv = a^{-1} by Gauss-Jordan elimination with partial pivoting; a is destroyed.
   Returns 0 on success, -1 if a is singular. */
static int inv_gj(double *a, double *inv, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
        if (best == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t;
                t = inv[k * n + j]; inv[k * n + j] = inv[p * n + j]; inv[p * n + j] = t;
            }
        double piv = a[k * n + k];
        for (int j = 0; j < n; ++j) { a[k * n + j] /= piv; inv[k * n + j] /= piv; }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            double f = a[i * n + k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) { a[i * n + j] -= f * a[k * n + j]; inv[i * n + j] -= f * inv[k * n + j]; }
        }
    }
    return 0;
}

double orc_det(const double *a_in, int n) {
    double a[ORC_MAXN * ORC_MAXN * 4];
    if (n > 2 * ORC_MAXN) return NAN;
    memcpy(a, a_in, sizeof(double) * n * n);
    return det_lu(a, n);
}

/* (V_T + I)/2 for mode set T (t modes): rows T[0..t-1] then T[0..t-1] + M. */
static void reduced_A(const double *V, int M, const int *T, int t, double *a) {
    int n = 2 * t;
    for (int i = 0; i < n; ++i) {
        int gi = (i < t) ? T[i] : T[i - t] + M;
        for (int j = 0; j < n; ++j) {
            int gj = (j < t) ? T[j] : T[j - t] + M;
            a[i * n + j] = 0.5 * (V[(size_t)gi * 2 * M + gj] + (i == j ? 1.0 : 0.0));
        }
    }
}

/* 1 if every mode of T lies in [0, M). */
static int modes_in_range(const int *T, int t, int M) {
    for (int i = 0; i < t; ++i)
        if (T[i] < 0 || T[i] >= M) return 0;
    return 1;
}

/* ---------------------------------------------------------------- Eq. vacuum_gaussian_prob */

double orc_p0(const double *V, int M, const int *T, int t) {
    double a[ORC_MAXN * ORC_MAXN];
    if (t == 0) return 1.0;
    if (t > ORC_MAXD || !modes_in_range(T, t, M)) return NAN;
    reduced_A(V, M, T, t, a);
    double det = det_lu(a, 2 * t);
    if (!(det > 0.0)) return NAN;
    return 1.0 / sqrt(det);
}

double orc_cumulant_from_moments(const double *mom, int d);

/* Displaced state (first moments mean[2M], xxpp, hbar = 2): the full Eq.
   vacuum_gaussian_prob, P0(T) = exp(-1/2 m_T^T (V_T + I)^{-1} m_T) / sqrt(det((V_T + I)/2)),
   with (V_T + I)^{-1} m_T from Gauss-Jordan elimination. */
double orc_p0_displaced(const double *V, const double *mean, int M, const int *T, int t) {
    double a[ORC_MAXN * ORC_MAXN], b[ORC_MAXN * ORC_MAXN], inv[ORC_MAXN * ORC_MAXN];
    if (t == 0) return 1.0;
    if (t > ORC_MAXD || !modes_in_range(T, t, M)) return NAN;
    int n = 2 * t;
    reduced_A(V, M, T, t, a);
    memcpy(b, a, sizeof(double) * n * n);
    double det = det_lu(b, n);
    if (!(det > 0.0)) return NAN;
    for (int q = 0; q < n * n; ++q) a[q] *= 2.0; /* V_T + I */
    if (inv_gj(a, inv, n) != 0) return NAN;
    double m[ORC_MAXN], quad = 0.0;
    for (int i = 0; i < n; ++i) m[i] = mean[(i < t) ? T[i] : T[i - t] + M];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) quad += m[i] * inv[i * n + j] * m[j];
    return exp(-0.5 * quad) / sqrt(det);
}

/* Entries of a displaced state for n sorted d-subsets, from scratch: P0 by the
   formula above, mu by inclusion-exclusion over subsets, the click cumulant by
   the partition sum over the moments of the blocks. Any output may be NULL. */
void orc_entries_displaced(const double *V, const double *mean, int M, int d, const int *sets, int64_t n,
                           double *p0, double *mu, double *kt) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const int *S = sets + (size_t)i * d;
        double pm[1u << ORC_MAXD], mom[1u << ORC_MAXD];
        int T[ORC_MAXD];
        for (unsigned mask = 0; mask < (1u << d); ++mask) {
            int t = 0;
            for (int k = 0; k < d; ++k)
                if (mask >> k & 1u) T[t++] = S[k];
            pm[mask] = orc_p0_displaced(V, mean, M, T, t);
        }
        for (unsigned mask = 0; mask < (1u << d); ++mask) {
            double acc = 0.0;
            for (unsigned sub = mask;; sub = (sub - 1) & mask) {
                acc += ((__builtin_popcount(sub) & 1) ? -1.0 : 1.0) * pm[sub];
                if (sub == 0) break;
            }
            mom[mask] = acc;
        }
        if (p0) p0[i] = pm[(1u << d) - 1];
        if (mu) mu[i] = mom[(1u << d) - 1];
        if (kt) kt[i] = orc_cumulant_from_moments(mom, d);
    }
}

/* ---------------------------------------------------------------- click moments */

/* mu(S) = sum_{T subset S} (-1)^{|T|} P0(T), each P0 from its own determinant. */
double orc_mu(const double *V, int M, const int *S, int d) {
    double acc = 0.0;
    int T[ORC_MAXD];
    for (unsigned mask = 0; mask < (1u << d); ++mask) {
        int t = 0;
        for (int i = 0; i < d; ++i)
            if (mask >> i & 1u) T[t++] = S[i];
        double sgn = (t & 1) ? -1.0 : 1.0;
        acc += sgn * orc_p0(V, M, T, t);
    }
    return acc;
}

/* ---------------------------------------------------------------- set partitions */

/* All set partitions of {0..d-1} as restricted growth strings: label[0] = 0 and
   label[i] <= 1 + max(label[0..i-1]). Writes count*d labels into out (capacity
   cap partitions); returns the count (the Bell number B_d). */
int orc_set_partitions(int d, int *out, int cap) {
    int lab[ORC_MAXD], mx[ORC_MAXD];
    int count = 0;
    if (d <= 0 || d > ORC_MAXD) return 0;
    for (int i = 0; i < d; ++i) { lab[i] = 0; mx[i] = 0; }
    for (;;) {
        if (count < cap) memcpy(out + (size_t)count * d, lab, sizeof(int) * d);
        ++count;
        /* next restricted growth string: bump the last position that can grow */
        int i = d - 1;
        while (i > 0 && lab[i] == mx[i - 1] + 1) --i;
        if (i == 0) break;
        lab[i] += 1;
        mx[i] = lab[i] > mx[i - 1] ? lab[i] : mx[i - 1];
        for (int j = i + 1; j < d; ++j) { lab[j] = 0; mx[j] = mx[i]; }
    }
    return count;
}

/* Partition-lattice weight (-1)^{|pi|-1} (|pi|-1)!. */
static double partition_weight(int nblocks) {
    double f = 1.0;
    for (int k = 2; k <= nblocks - 1; ++k) f *= (double)k;
    return ((nblocks - 1) & 1) ? -f : f;
}

/* Cumulant of the d variables from their joint moments: mom[mask] is the moment of
   the variables whose local positions are set in mask (mask 1..2^d-1). Sum over all
   set partitions of (-1)^{|pi|-1}(|pi|-1)! prod_{b in pi} mom[b]  (Eq.
   joint_cumulants_def; the same map takes correlators to spin cumulants,
   Eq. cumulant_corr_main). */
double orc_cumulant_from_moments(const double *mom, int d) {
    static const int bell[ORC_MAXD + 1] = {1, 1, 2, 5, 15, 52, 203, 877, 4140};
    if (d <= 0 || d > ORC_MAXD) return NAN;
    const int cap = bell[d];
    int *parts = (int *)malloc(sizeof(int) * cap * d);
    int np = orc_set_partitions(d, parts, cap);
    double acc = 0.0;
    for (int p = 0; p < np; ++p) {
        const int *lab = parts + (size_t)p * d;
        unsigned bm[ORC_MAXD] = {0};
        int nb = 0;
        for (int i = 0; i < d; ++i) {
            bm[lab[i]] |= 1u << i;
            if (lab[i] + 1 > nb) nb = lab[i] + 1;
        }
        double prod = partition_weight(nb);
        for (int b = 0; b < nb; ++b) prod *= mom[bm[b]];
        acc += prod;
    }
    free(parts);
    return acc;
}

/* Click cumulant of S from scratch: moments of every sub-block, then the partition sum. */
double orc_kappa(const double *V, int M, const int *S, int d) {
    double mom[1u << ORC_MAXD];
    int B[ORC_MAXD];
    mom[0] = 1.0;
    for (unsigned mask = 1; mask < (1u << d); ++mask) {
        int b = 0;
        for (int i = 0; i < d; ++i)
            if (mask >> i & 1u) B[b++] = S[i];
        mom[mask] = orc_mu(V, M, B, b);
    }
    return orc_cumulant_from_moments(mom, d);
}

/* Spin correlator c(S) (Eq. correlator_sum_cov, hbar = 2). */
double orc_spin_correlator(const double *V, int M, const int *S, int d) {
    double acc = 0.0;
    int R[ORC_MAXD];
    for (unsigned mask = 0; mask < (1u << d); ++mask) {
        int t = 0;
        for (int i = 0; i < d; ++i)
            if (mask >> i & 1u) R[t++] = S[i];
        acc += pow(-2.0, t) * orc_p0(V, M, R, t);
    }
    return ((d & 1) ? -1.0 : 1.0) * acc;
}

/* Spin cumulant kappa(S) from the correlators of its sub-blocks (Eq. cumulant_corr_main). */
double orc_spin_cumulant(const double *V, int M, const int *S, int d) {
    double c[1u << ORC_MAXD];
    int B[ORC_MAXD];
    c[0] = 1.0;
    for (unsigned mask = 1; mask < (1u << d); ++mask) {
        int b = 0;
        for (int i = 0; i < d; ++i)
            if (mask >> i & 1u) B[b++] = S[i];
        c[mask] = orc_spin_correlator(V, M, B, b);
    }
    return orc_cumulant_from_moments(c, d);
}

/* ---------------------------------------------------------------- enumeration */

/* Binomial coefficient by a plain product loop (exact for the sizes used here). */
uint64_t orc_binom(int n, int k) {
    if (k < 0 || n < k) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

/* Position of the sorted set S (S[0] < ... < S[d-1]) among the d-subsets in
   colex order: sum_i C(S[i], i+1). Pinned against the nested-loop order below. */
uint64_t orc_colex_rank(const int *S, int d) {
    uint64_t r = 0;
    for (int i = 0; i < d; ++i) r += orc_binom(S[i], i + 1);
    return r;
}

static void enum_rec(int M, int d, int level, int upper, int *cur, int *out, int64_t *count) {
    /* level counts down from d-1 (largest element) to 0 (smallest element) */
    for (int c = level; c < upper; ++c) {
        cur[level] = c;
        if (level == 0) {
            memcpy(out + (size_t)(*count) * d, cur, sizeof(int) * d);
            ++*count;
        } else {
            enum_rec(M, d, level - 1, c, cur, out, count);
        }
    }
}

/* All d-subsets of {0..M-1} in colex order (largest element outermost loop, each
   row sorted ascending). out must hold C(M,d)*d ints. Returns the count. */
int64_t orc_enumerate(int M, int d, int *out) {
    int cur[ORC_MAXD];
    int64_t count = 0;
    if (d <= 0 || d > ORC_MAXD || d > M) return 0;
    enum_rec(M, d, d - 1, M, cur, out, &count);
    return count;
}

/* ---------------------------------------------------------------- entries from scratch */

/* For n sorted d-subsets (rows of sets), each entry computed from its own
   determinants and partitions. Any output pointer may be NULL. */
void orc_entries(const double *V, int M, int d, const int *sets, int64_t n,
                 double *p0, double *mu, double *kt) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const int *S = sets + (size_t)i * d;
        if (p0) p0[i] = orc_p0(V, M, S, d);
        if (mu) mu[i] = orc_mu(V, M, S, d);
        if (kt) kt[i] = orc_kappa(V, M, S, d);
    }
}

/* ---------------------------------------------------------------- full tables */

static uint64_t table_offset(int M, int d) {
    uint64_t off = 0;
    for (int e = 1; e < d; ++e) off += orc_binom(M, e);
    return off;
}

static uint64_t index_of(int M, const int *S, int d) {
    return table_offset(M, d) + orc_colex_rank(S, d);
}

/* Tables of P0, mu and the click cumulant over all subsets of order 1..kmax.
   The P0 entries come from determinants; mu from inclusion-exclusion over the
   P0 entries of the subsets; the cumulants from the partition sum over the mu
   entries of the blocks. Any output may be NULL. Returns 0, or -1 on bad args. */
int orc_tables(const double *V, int M, int kmax, double *p0_out, double *mu_out, double *kt_out) {
    if (M <= 0 || kmax <= 0 || kmax > M || kmax > ORC_MAXD) return -1;
    uint64_t N = table_offset(M, kmax + 1);
    double *p0 = p0_out ? p0_out : (double *)malloc(sizeof(double) * N);
    double *mu = mu_out ? mu_out : (double *)malloc(sizeof(double) * N);
    for (int d = 1; d <= kmax; ++d) {
        int64_t cnt = (int64_t)orc_binom(M, d);
        int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
        orc_enumerate(M, d, sets);
        uint64_t off = table_offset(M, d);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < cnt; ++i) p0[off + i] = orc_p0(V, M, sets + (size_t)i * d, d);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < cnt; ++i) {
            const int *S = sets + (size_t)i * d;
            int T[ORC_MAXD];
            double acc = 1.0; /* T = empty */
            for (unsigned mask = 1; mask < (1u << d); ++mask) {
                int t = 0;
                for (int k = 0; k < d; ++k)
                    if (mask >> k & 1u) T[t++] = S[k];
                acc += ((t & 1) ? -1.0 : 1.0) * p0[index_of(M, T, t)];
            }
            mu[off + i] = acc;
        }
        free(sets);
    }
    if (kt_out) {
        for (int d = 1; d <= kmax; ++d) {
            int64_t cnt = (int64_t)orc_binom(M, d);
            int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
            orc_enumerate(M, d, sets);
            uint64_t off = table_offset(M, d);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < cnt; ++i) {
                const int *S = sets + (size_t)i * d;
                double mom[1u << ORC_MAXD];
                int B[ORC_MAXD];
                mom[0] = 1.0;
                for (unsigned mask = 1; mask < (1u << d); ++mask) {
                    int b = 0;
                    for (int k = 0; k < d; ++k)
                        if (mask >> k & 1u) B[b++] = S[k];
                    mom[mask] = mu[index_of(M, B, b)];
                }
                kt_out[off + i] = orc_cumulant_from_moments(mom, d);
            }
            free(sets);
        }
    }
    if (!p0_out) free(p0);
    if (!mu_out) free(mu);
    return 0;
}

/* ---------------------------------------------------------------- spin tables */

/* Spin-correlator and spin-cumulant tables (orders 1..kmax): c(S) by Eq.
   correlator_sum_cov over the P0 entries of the subsets of S, kappa(S) by Eq.
   cumulant_corr_main over the c entries of the blocks of S. Either output may be
   NULL. Returns 0, or -1 on bad args. */
int orc_spin_tables_from_p0(const double *p0, int M, int kmax, double *c_out, double *k_out);

int orc_spin_tables(const double *V, int M, int kmax, double *c_out, double *k_out) {
    if (M <= 0 || kmax <= 0 || kmax > M || kmax > ORC_MAXD) return -1;
    uint64_t N = table_offset(M, kmax + 1);
    double *p0 = (double *)malloc(sizeof(double) * N);
    orc_tables(V, M, kmax, p0, NULL, NULL);
    int rc = orc_spin_tables_from_p0(p0, M, kmax, c_out, k_out);
    free(p0);
    return rc;
}

/* The same two tables from a given P0 table. Expanding prod_k (-1)^{x_k} =
   prod_k (2 y_k - 1) over the no-click indicators y_k, whose joint moments are
   the P0 entries, gives Eq. correlator_sum_cov for any state, displaced or not. */
int orc_spin_tables_from_p0(const double *p0, int M, int kmax, double *c_out, double *k_out) {
    if (M <= 0 || kmax <= 0 || kmax > M || kmax > ORC_MAXD) return -1;
    uint64_t N = table_offset(M, kmax + 1);
    double *c = c_out ? c_out : (double *)malloc(sizeof(double) * N);
    for (int d = 1; d <= kmax; ++d) {
        int64_t cnt = (int64_t)orc_binom(M, d);
        int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
        orc_enumerate(M, d, sets);
        uint64_t off = table_offset(M, d);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < cnt; ++i) {
            const int *S = sets + (size_t)i * d;
            int R[ORC_MAXD];
            double acc = 0.0;
            for (unsigned mask = 0; mask < (1u << d); ++mask) {
                int t = 0;
                for (int k = 0; k < d; ++k)
                    if (mask >> k & 1u) R[t++] = S[k];
                acc += pow(-2.0, t) * (t ? p0[index_of(M, R, t)] : 1.0);
            }
            c[off + i] = ((d & 1) ? -1.0 : 1.0) * acc;
        }
        free(sets);
    }
    if (k_out) {
        for (int d = 1; d <= kmax; ++d) {
            int64_t cnt = (int64_t)orc_binom(M, d);
            int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
            orc_enumerate(M, d, sets);
            uint64_t off = table_offset(M, d);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < cnt; ++i) {
                const int *S = sets + (size_t)i * d;
                double cor[1u << ORC_MAXD];
                int B[ORC_MAXD];
                cor[0] = 1.0;
                for (unsigned mask = 1; mask < (1u << d); ++mask) {
                    int b = 0;
                    for (int k = 0; k < d; ++k)
                        if (mask >> k & 1u) B[b++] = S[k];
                    cor[mask] = c[index_of(M, B, b)];
                }
                k_out[off + i] = orc_cumulant_from_moments(cor, d);
            }
            free(sets);
        }
    }
    if (!c_out) free(c);
    return 0;
}

/* ---------------------------------------------------------------- gradient */

/* dL/dV for L with dL/dkt(S) = gk[index(S)] over the whole table (orders 1..kmax).
   Chain rule in the order the quantities are defined:
     gmu(B)  = sum_{S >= B} gk(S) * sum_{pi of S, B in pi} w(pi) prod_{B' in pi, B' != B} mu(B')
     gP0(T)  = (-1)^{|T|} sum_{S >= T} gmu(S)
     dV_T   += gP0(T) * dP0(T)/dV_T,  dP0(T)/dV_T = -1/2 P0(T) (V_T + I)^{-1}
   (from d det(X)^{-1/2} = -1/2 det(X)^{-1/2} tr(X^{-1} dX) with X = (V_T+I)/2).
   dV is the gradient with respect to every entry V_ab taken as independent
   (2M x 2M, symmetric). Returns 0, or -1 on bad args. */
int orc_grad(const double *V, int M, int kmax, const double *gk, double *dV) {
    if (M <= 0 || kmax <= 0 || kmax > M || kmax > ORC_MAXD) return -1;
    uint64_t N = table_offset(M, kmax + 1);
    int n2 = 2 * M;
    double *p0 = (double *)malloc(sizeof(double) * N);
    double *mu = (double *)malloc(sizeof(double) * N);
    double *gmu = (double *)calloc(N, sizeof(double));
    double *gp0 = (double *)calloc(N, sizeof(double));
    orc_tables(V, M, kmax, p0, mu, NULL);
    int *parts = (int *)malloc(sizeof(int) * 4140 * ORC_MAXD);

    for (int d = 1; d <= kmax; ++d) {
        int64_t cnt = (int64_t)orc_binom(M, d);
        int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
        orc_enumerate(M, d, sets);
        uint64_t off = table_offset(M, d);
        int np = orc_set_partitions(d, parts, 4140);
        for (int64_t i = 0; i < cnt; ++i) {
            double g = gk[off + i];
            if (g == 0.0) continue;
            const int *S = sets + (size_t)i * d;
            double mom[1u << ORC_MAXD];
            uint64_t idx[1u << ORC_MAXD];
            int B[ORC_MAXD];
            for (unsigned mask = 1; mask < (1u << d); ++mask) {
                int b = 0;
                for (int k = 0; k < d; ++k)
                    if (mask >> k & 1u) B[b++] = S[k];
                idx[mask] = index_of(M, B, b);
                mom[mask] = mu[idx[mask]];
            }
            for (int p = 0; p < np; ++p) {
                const int *lab = parts + (size_t)p * d;
                unsigned bm[ORC_MAXD] = {0};
                int nb = 0;
                for (int k = 0; k < d; ++k) {
                    bm[lab[k]] |= 1u << k;
                    if (lab[k] + 1 > nb) nb = lab[k] + 1;
                }
                double w = partition_weight(nb);
                for (int b = 0; b < nb; ++b) {
                    double prod = w;
                    for (int o = 0; o < nb; ++o)
                        if (o != b) prod *= mom[bm[o]];
                    gmu[idx[bm[b]]] += g * prod;
                }
            }
        }
        free(sets);
    }
    for (int d = 1; d <= kmax; ++d) {
        int64_t cnt = (int64_t)orc_binom(M, d);
        int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
        orc_enumerate(M, d, sets);
        uint64_t off = table_offset(M, d);
        for (int64_t i = 0; i < cnt; ++i) {
            double g = gmu[off + i];
            if (g == 0.0) continue;
            const int *S = sets + (size_t)i * d;
            int T[ORC_MAXD];
            for (unsigned mask = 1; mask < (1u << d); ++mask) {
                int t = 0;
                for (int k = 0; k < d; ++k)
                    if (mask >> k & 1u) T[t++] = S[k];
                gp0[index_of(M, T, t)] += ((t & 1) ? -1.0 : 1.0) * g;
            }
        }
        free(sets);
    }
    memset(dV, 0, sizeof(double) * (size_t)n2 * n2);
    for (int d = 1; d <= kmax; ++d) {
        int64_t cnt = (int64_t)orc_binom(M, d);
        int *sets = (int *)malloc(sizeof(int) * (size_t)cnt * d);
        orc_enumerate(M, d, sets);
        uint64_t off = table_offset(M, d);
#pragma omp parallel
        {
            double *loc = (double *)calloc((size_t)n2 * n2, sizeof(double));
#pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < cnt; ++i) {
                double g = gp0[off + i];
                if (g == 0.0) continue;
                const int *S = sets + (size_t)i * d;
                int n = 2 * d;
                double a[ORC_MAXN * ORC_MAXN], inv[ORC_MAXN * ORC_MAXN];
                /* a = V_S + I */
                reduced_A(V, M, S, d, a);
                for (int q = 0; q < n * n; ++q) a[q] *= 2.0;
                if (inv_gj(a, inv, n) != 0) continue;
                double coef = -0.5 * g * p0[off + i];
                for (int r = 0; r < n; ++r) {
                    int gr = (r < d) ? S[r] : S[r - d] + M;
                    for (int c = 0; c < n; ++c) {
                        int gc = (c < d) ? S[c] : S[c - d] + M;
                        loc[(size_t)gr * n2 + gc] += coef * inv[c * n + r];
                    }
                }
            }
#pragma omp critical
            for (size_t q = 0; q < (size_t)n2 * n2; ++q) dV[q] += loc[q];
            free(loc);
        }
        free(sets);
    }
    free(parts); free(p0); free(mu); free(gmu); free(gp0);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
