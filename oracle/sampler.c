/*
 * CPU FP64 oracle for stage 2 of the emulator (arXiv:2511.14923): the chain-rule
 * sampler that draws threshold-detector bitstrings from the spin cumulants
 * kappa(S) of orders 1..K.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it; the library never does.
 *
 * The exact chain rule (Eq. probs_corr_cumulants_3, with bit n the newest):
 *   p(x_n..x_1) = 1/2 p(x_{n-1}..x_1)
 *               + sum_{R subset [n-1]} 2^{-(|R|+1)} chi_{R+n}(x) kappa(R + {n}) p(x_{[n-1] - R}),
 * chi_A(x) = prod_{k in A} (-1)^{x_k}. Truncating at |R| + 1 <= K and replacing
 * the marginals p(x_{[n-1] - R}) by tables that are themselves filled by truncated
 * forms of the same rule gives the two samplers of the paper:
 *
 *   single elision, K = 3 (Sec. Methods: Eq. methprob, Eq. b, Eq. a):
 *     P[a]      = p(x_a..x_1)
 *     P1[a][e]  = p1(x_a..~x_e..x_1)  (all of 1..a but e)
 *     Pp[a][b]  = p+(x_a..x_b)        (all of b..a)
 *   double elision, K = 5 (App. "Approximating marginals efficiently with a chain
 *   rule": Eq. probade, Eq. probpartialade, Eq. probelidedade, Eq.
 *   probdoubleelidedade; K = 4 drops the |R| = 4 term), which adds
 *     P2[a][e][d] = p2(x_a..~x_e..~x_d..x_1)  (all of 1..a but e > d).
 *
 * Conventions for the boundary cases the update rules reach:
 *   P[0] = 1; Pp[a][b] = 1 for an empty range (b > a);
 *   P1[a][a] = P[a-1] (eliding the newest variable leaves the chain below it);
 *   P2[a][a][d] = P1[a-1][d] for the same reason.
 *
 * Variables are 1-based here; variable n is mode n - 1, and kappa(S) is read from
 * the spin-cumulant table laid out as gbs.h describes (orders 1..K, colex ranks).
 *
 * Drawing bit n: the expansion gives p(x_n = 0, ..) = P[n-1]/2 + B and
 * p(x_n = 1, ..) = P[n-1]/2 - B (every term but the first is odd in x_n). The bit
 * is 0 when u_n < q0 = max(p0, 0) / (max(p0, 0) + max(p1, 0)) (q0 = 1/2 if both
 * are <= 0), and P[n] keeps the unclipped value of the chosen branch.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SMP_MAXK 5

static uint64_t smp_binom(int n, int k) {
    if (k < 0 || n < k) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

/* kappa of the variable set vars[0..d) (1-based, any order) from the table. */
static double kap(const double *kappa, int M, const int *vars, int d) {
    int s[SMP_MAXK];
    for (int i = 0; i < d; ++i) s[i] = vars[i] - 1;
    for (int i = 1; i < d; ++i)
        for (int j = i; j > 0 && s[j - 1] > s[j]; --j) {
            int t = s[j]; s[j] = s[j - 1]; s[j - 1] = t;
        }
    uint64_t idx = 0;
    for (int e = 1; e < d; ++e) idx += smp_binom(M, e);
    for (int i = 0; i < d; ++i) idx += smp_binom(s[i], i + 1);
    return kappa[idx];
}

/* gamma_A = kappa(A) chi_A(x) for the variable set A = vars[0..d). */
static double gam(const double *kappa, int M, const double *chi, const int *vars, int d) {
    double g = kap(kappa, M, vars, d);
    for (int i = 0; i < d; ++i) g *= chi[vars[i]];
    return g;
}

typedef struct {
    int M;
    double *P;   /* [M+1] */
    double *P1;  /* [(M+1)^2], P1[a*(M+1)+e] */
    double *Pp;  /* [(M+1)^2], Pp[a*(M+1)+b] */
    double *P2;  /* [(M+1)^3] or NULL */
} Tables;

static double tP(const Tables *t, int a) { return t->P[a]; }
static double tPp(const Tables *t, int a, int b) { return b > a ? 1.0 : t->Pp[(size_t)a * (t->M + 1) + b]; }
static double tP1(const Tables *t, int a, int e) { return e == a ? t->P[a - 1] : t->P1[(size_t)a * (t->M + 1) + e]; }
static double tP2(const Tables *t, int a, int e, int d) {
    /* e > d */
    if (e == a) return tP1(t, a - 1, d);
    return t->P2[((size_t)a * (t->M + 1) + e) * (t->M + 1) + d];
}

/* (a, b, c) = the arguments in decreasing order */
static void ord3(int x, int y, int z, int *a, int *b, int *c) {
    int v[3] = {x, y, z};
    for (int i = 1; i < 3; ++i)
        for (int j = i; j > 0 && v[j - 1] < v[j]; --j) {
            int t = v[j]; v[j] = v[j - 1]; v[j - 1] = t;
        }
    *a = v[0]; *b = v[1]; *c = v[2];
}

/* The odd part B of p(x_n..x_1) (the value with x_n = 0 is P[n-1]/2 + B) for
   K = 3 single elision, Eq. methprob; chi[n] is set to +1 while this runs. */
static double bias_k3(const Tables *t, const double *kappa, int M, const double *chi, int n) {
    int v[3];
    v[0] = n;
    double B = 0.5 * gam(kappa, M, chi, v, 1) * tP(t, n - 1);
    for (int i = 1; i <= n - 1; ++i) {
        v[0] = i; v[1] = n;
        B += 0.25 * gam(kappa, M, chi, v, 2) * tP1(t, n - 1, i);
    }
    for (int i = 2; i <= n - 1; ++i)
        for (int j = 1; j <= i - 1; ++j) {
            v[0] = i; v[1] = j; v[2] = n;
            B += 0.125 * gam(kappa, M, chi, v, 3) * tPp(t, n - 1, i + 1) * tP1(t, i - 1, j);
        }
    return B;
}

/* The same for double elision, Eq. probade, truncated at |R| + 1 <= K (K = 4
   or 5). The |R| = 2 term uses the double-elided table p2 (the printed equation
   omits the symbol; the text states that |R| = 1 and 2 use p1 and p2). */
static double bias_k5(const Tables *t, const double *kappa, int M, const double *chi, int n, int K) {
    int v[5];
    v[0] = n;
    double B = 0.5 * gam(kappa, M, chi, v, 1) * tP(t, n - 1);
    for (int i = 1; i <= n - 1; ++i) {
        v[0] = i; v[1] = n;
        B += 0.25 * gam(kappa, M, chi, v, 2) * tP1(t, n - 1, i);
    }
    for (int i = 2; i <= n - 1; ++i)
        for (int j = 1; j <= i - 1; ++j) {
            v[0] = i; v[1] = j; v[2] = n;
            B += 0.125 * gam(kappa, M, chi, v, 3) * tP2(t, n - 1, i, j);
        }
    for (int i = 3; i <= n - 1; ++i)
        for (int j = 2; j <= i - 1; ++j)
            for (int k = 1; k <= j - 1; ++k) {
                v[0] = i; v[1] = j; v[2] = k; v[3] = n;
                B += 0.0625 * gam(kappa, M, chi, v, 4) * tPp(t, n - 1, i + 1) * tP2(t, i - 1, j, k);
            }
    for (int i = 4; K >= 5 && i <= n - 1; ++i)
        for (int j = 3; j <= i - 1; ++j)
            for (int k = 2; k <= j - 1; ++k)
                for (int l = 1; l <= k - 1; ++l) {
                    v[0] = i; v[1] = j; v[2] = k; v[3] = l; v[4] = n;
                    B += 0.03125 * gam(kappa, M, chi, v, 5) * tPp(t, n - 1, i + 1) * tPp(t, i - 1, j + 1) *
                         tP2(t, j - 1, k, l);
                }
    return B;
}

/* Table updates after bit n is fixed (chi[n] = its spin).
   K = 3: Eq. b (P1) and Eq. a (Pp), both of order 2.
   K = 5: Eq. probpartialade (Pp, order opp), Eq. probelidedade (P1, order op1),
   Eq. probdoubleelidedade (P2, order op2); the paper's forms are orders 3, 3, 2,
   and it reports running one order lower (2, 2, 1) in practice. */
static void update_tables(Tables *t, const double *kappa, int M, const double *chi, int n, int K, int opp, int op1,
                          int op2) {
    const size_t W = (size_t)M + 1;
    int v[3];
    v[0] = n;
    const double h = 0.5 * (1.0 + gam(kappa, M, chi, v, 1));
    /* p+ (x_n .. x_l), l = 1..n */
    for (int l = 1; l <= n; ++l) {
        double s = h * tPp(t, n - 1, l);
        if (opp >= 2)
            for (int i = l; i <= n - 1; ++i) {
                v[0] = i; v[1] = n;
                s += 0.25 * gam(kappa, M, chi, v, 2) * tPp(t, n - 1, i + 1) * tPp(t, i - 1, l);
            }
        if (opp >= 3)
            for (int i = l + 1; i <= n - 1; ++i)
                for (int j = l; j <= i - 1; ++j) {
                    v[0] = i; v[1] = j; v[2] = n;
                    s += 0.125 * gam(kappa, M, chi, v, 3) * tPp(t, n - 1, i + 1) * tPp(t, i - 1, j + 1) *
                         tPp(t, j - 1, l);
                }
        t->Pp[n * W + l] = s;
    }
    /* p1 (x_n .. ~x_e .. x_1), e = 1..n-1 */
    for (int e = 1; e <= n - 1; ++e) {
        double s = h * tP1(t, n - 1, e);
        if (op1 >= 2)
            for (int i = 1; i <= n - 1; ++i) {
                if (i == e) continue;
                const int a = i > e ? i : e, b = i > e ? e : i;  /* a > b */
                v[0] = i; v[1] = n;
                const double g = gam(kappa, M, chi, v, 2);
                if (K == 3) s += 0.25 * g * tPp(t, n - 1, a + 1) * tP1(t, a - 1, b);  /* Eq. b */
                else s += 0.25 * g * tP2(t, n - 1, a, b);
            }
        if (op1 >= 3)
            for (int i = 2; i <= n - 1; ++i)
                for (int j = 1; j <= i - 1; ++j) {
                    if (i == e || j == e) continue;
                    int a, b, c;
                    ord3(i, j, e, &a, &b, &c);
                    v[0] = i; v[1] = j; v[2] = n;
                    s += 0.125 * gam(kappa, M, chi, v, 3) * tPp(t, n - 1, a + 1) * tP2(t, a - 1, b, c);
                }
        t->P1[n * W + e] = s;
    }
    if (K == 3) return;
    /* p2 (x_n .. ~x_e .. ~x_d .. x_1), n-1 >= e > d >= 1 */
    for (int e = 2; e <= n - 1; ++e)
        for (int d = 1; d <= e - 1; ++d) {
            double s = h * tP2(t, n - 1, e, d);
            if (op2 >= 2)
                for (int i = 1; i <= n - 1; ++i) {
                    if (i == e || i == d) continue;
                    int a, b, c;
                    ord3(i, e, d, &a, &b, &c);
                    v[0] = i; v[1] = n;
                    s += 0.25 * gam(kappa, M, chi, v, 2) * tPp(t, n - 1, a + 1) * tP2(t, a - 1, b, c);
                }
            t->P2[(n * W + e) * W + d] = s;
        }
}

/* One sample. K = 3 (single elision), 4 or 5 (double elision); orders = {opp,
   op1, op2} for K = 4, 5 (1..3, 1..3, 1..2; NULL = the defaults above; ignored
   for K = 3). u[M]: uniforms; force (may be NULL): bits to
   score instead of drawing. Outputs (any may be NULL): bits[M], p_out = P[M],
   q0[M] = the probability of a 0 each bit was drawn with. Returns 0, or -1 on bad
   arguments or allocation failure. */
int orc_sample(const double *kappa, int M, int K, const int *orders, const double *u, const uint8_t *force,
               uint8_t *bits, double *p_out, double *q0) {
    if (M < K || K < 3 || K > 5 || !kappa) return -1;
    if (orders && (orders[0] < 1 || orders[0] > 3 || orders[1] < 1 || orders[1] > 3 || orders[2] < 1 || orders[2] > 2))
        return -1;
    const size_t W = (size_t)M + 1;
    Tables t;
    t.M = M;
    t.P = (double *)calloc(W, sizeof(double));
    t.P1 = (double *)calloc(W * W, sizeof(double));
    t.Pp = (double *)calloc(W * W, sizeof(double));
    t.P2 = K >= 4 ? (double *)calloc(W * W * W, sizeof(double)) : NULL;
    double *chi = (double *)calloc(W, sizeof(double));
    if (!t.P || !t.P1 || !t.Pp || (K >= 4 && !t.P2) || !chi) {
        free(t.P); free(t.P1); free(t.Pp); free(t.P2); free(chi);
        return -1;
    }
    /* K = 3: Eq. a and Eq. b are both of order 2 (there is no p2 table). K = 5:
       the paper's orders 3, 3, 2. K = 4: the same rule (one order below the
       minimum that keeps O(M^K) time) gives 2, 2, 1. */
    const int dpp = K == 5 ? 3 : 2, dp1 = K == 5 ? 3 : 2, dp2 = K == 5 ? 2 : 1;
    const int opp = K == 3 ? 2 : (orders ? orders[0] : dpp), op1 = K == 3 ? 2 : (orders ? orders[1] : dp1);
    const int op2 = orders ? orders[2] : dp2;
    t.P[0] = 1.0;
    for (int n = 1; n <= M; ++n) {
        chi[n] = 1.0;
        const double B = K == 3 ? bias_k3(&t, kappa, M, chi, n) : bias_k5(&t, kappa, M, chi, n, K);
        const double p0 = 0.5 * t.P[n - 1] + B, p1 = 0.5 * t.P[n - 1] - B;
        const double c0 = p0 > 0.0 ? p0 : 0.0, c1 = p1 > 0.0 ? p1 : 0.0;
        const double qz = (c0 + c1 > 0.0) ? c0 / (c0 + c1) : 0.5;
        int x;
        if (force) x = force[n - 1] ? 1 : 0;
        else x = (u[n - 1] < qz) ? 0 : 1;
        chi[n] = x ? -1.0 : 1.0;
        t.P[n] = x ? p1 : p0;
        if (bits) bits[n - 1] = (uint8_t)x;
        if (q0) q0[n - 1] = qz;
        update_tables(&t, kappa, M, chi, n, K, opp, op1, op2);
    }
    if (p_out) *p_out = t.P[M];
    free(t.P); free(t.P1); free(t.Pp); free(t.P2); free(chi);
    return 0;
}

/* ns samples in parallel: u is ns x M, force (may be NULL) ns x M, bits ns x M,
   p_out ns, q0 ns x M (each output may be NULL). Returns the number of failures. */
int orc_sample_batch(const double *kappa, int M, int K, const int *orders, int64_t ns, const double *u,
                     const uint8_t *force, uint8_t *bits, double *p_out, double *q0) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int64_t s = 0; s < ns; ++s) {
        const size_t o = (size_t)s * M;
        bad += orc_sample(kappa, M, K, orders, u ? u + o : NULL, force ? force + o : NULL, bits ? bits + o : NULL,
                          p_out ? p_out + s : NULL, q0 ? q0 + o : NULL) != 0;
    }
    return bad;
}
