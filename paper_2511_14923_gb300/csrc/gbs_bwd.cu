// Adjoint of the click-cumulant table (gbs_cumulants_backward) and the
// covariance model of squeezers and a lossy interferometer (gbs_covariance and
// its adjoint), for fitting r and eta to target cumulants.
//
// Chain rule, in the order the forward quantities are defined:
//   * kt(S) = (-1)^{|S|} ky(S), where ky is the cumulant of the no-click
//     indicators y = 1 - x, whose joint moments are the P0 values (for |S| = 1,
//     kt = 1 - P0 = -ky + 1). So g_y(S) = (-1)^{|S|} dL/dkt(S).
//   * ky(S) is the multilinear coefficient of u^S in log F(u), F(u) =
//     sum_B P0(B) u^B (the partition sum of Eq. joint_cumulants_def, written as a
//     logarithm). Hence d ky(S) / d P0(B) = [u^{S-B}] (1/F) =: h(S - B) for
//     B subset S, and h obeys F * h = 1:  h(empty) = 1,
//     h(R) = -sum_{empty != T subset R} P0(T) h(R - T).
//     gP0(B) = sum_{S >= B, |S| <= kmax} g_y(S) h(S - B).
//   * P0(T) = det(A_T)^{-1/2}, A_T = (V_T + I)/2 (Eq. vacuum_gaussian_prob):
//     dP0(T)/dV_T = -1/2 P0(T) (V_T + I)^{-1} = -1/4 P0(T) A_T^{-1}; A_T^{-1} comes
//     from A_{T'}^{-1} (T' = T minus its smallest mode) by the block inverse.
// grad_V is the symmetric gradient: for every symmetric perturbation dV,
// dL = sum_ab grad_V[a][b] dV[a][b].
#include <cstdio>

#include "gbs.h"
#include "gbs_bwd.cuh"
#include "gbs_common.cuh"
#include "gbs_refined.cuh"

namespace gbs {

constexpr int BWD_THREADS = 256;

// Table index of the subset of the sorted set s[0..d) selected by mask.
__device__ __forceinline__ uint64_t sub_index(const int *s, int d, unsigned mask, const uint64_t *off) {
    uint64_t r = 0;
    int i = 0;
    for (int e = 0; e < d; ++e)
        if (mask >> e & 1u) r += binom(s[e], ++i);
    return off[i] + r;
}

struct Offsets {
    uint64_t off[GBS_MAX_ORDER + 2];  // off[m] = index of the first order-m entry (off[0] unused)
};

__host__ __device__ inline Offsets make_offsets(int M) {
    Offsets o{};
    o.off[0] = 0;
    for (int m = 1; m <= GBS_MAX_ORDER + 1; ++m) o.off[m] = order_offset(M, m);
    return o;
}

// h table, order r (all lower orders done): h(R) = -sum_{T nonempty subset R} P0(T) h(R - T).
__global__ void h_kernel(int M, int r, Offsets o, const double *__restrict__ p0, double *__restrict__ h) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= binom(M, r)) return;
    int s[GBS_MAX_ORDER];
    colex_unrank(i, r, s);
    const unsigned full = (1u << r) - 1;
    double acc = 0.0;
    for (unsigned t = 1; t <= full; ++t) {
        const unsigned rest = full ^ t;
        const double hr = rest ? h[sub_index(s, r, rest, o.off)] : 1.0;
        acc = fma(-p0[sub_index(s, r, t, o.off)], hr, acc);
    }
    h[o.off[r] + i] = acc;
}

// grad_V scatter, order d (used for d = 1): -1/4 gP0(T) P0(T) A_T^{-1} into the rows/cols of T,
// optionally privatised in shared memory (lower triangle of the 2M x 2M gradient).
template <int D>
__global__ void gv_kernel(int M, Offsets o, const double *__restrict__ A, const double *__restrict__ p0,
                          const double *__restrict__ gp0, double *__restrict__ gV, bool private_smem,
                          unsigned *status) {
    constexpr int N = 2 * D;
    extern __shared__ double sgv[];
    const int n2 = 2 * M;
    const size_t ntri = (size_t)n2 * (n2 + 1) / 2;
    if (private_smem) {
        for (size_t q = threadIdx.x; q < ntri; q += blockDim.x) sgv[q] = 0.0;
        __syncthreads();
    }
    const uint64_t cnt = binom(M, D);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
        const double g = gp0[o.off[D] + i];
        if (g == 0.0) continue;
        int s[D];
        colex_unrank(i, D, s);
        // A_T with rows ordered (x of s[0..D), p of s[0..D))
        double a[N][N];
#pragma unroll
        for (int u = 0; u < D; ++u)
#pragma unroll
            for (int v = 0; v < D; ++v) {
                const Blk b = ablk(A, M, s[u], s[v]);
                a[u][v] = b.a00;
                a[u][v + D] = b.a01;
                a[u + D][v] = b.a10;
                a[u + D][v + D] = b.a11;
            }
        // Cholesky (lower, in place) and the inverse of L
        bool ok = true;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double dkk = a[k][k];
#pragma unroll
            for (int m = 0; m < k; ++m) dkk = fma(-a[k][m], a[k][m], dkk);
            ok = ok && dkk > 0.0;
            const double inv = rsqrt(dkk);
            a[k][k] = inv;  // store 1 / L_kk
#pragma unroll
            for (int r = k + 1; r < N; ++r) {
                double v = a[r][k];
#pragma unroll
                for (int m = 0; m < k; ++m) v = fma(-a[r][m], a[k][m], v);
                a[r][k] = v * inv;
            }
        }
        if (!ok) {
            flag_status(status, ST_NOT_POSDEF);
            continue;
        }
        // W = L^{-1} (lower), column by column, into the upper triangle's mirror storage
        double w[N][N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
#pragma unroll
            for (int r = 0; r < N; ++r) {
                if (r < c) {
                    w[r][c] = 0.0;
                    continue;
                }
                double v = (r == c) ? 1.0 : 0.0;
#pragma unroll
                for (int m = c; m < r; ++m) v = fma(-a[r][m], w[m][c], v);
                w[r][c] = v * a[r][r];
            }
        }
        const double coef = -0.25 * g * p0[o.off[D] + i];
        // A^{-1} = W^T W ; scatter the lower triangle (and the mirror for off-diagonal pairs)
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const int gr = (r < D) ? s[r] : s[r - D] + M;
#pragma unroll
            for (int c = 0; c <= r; ++c) {
                const int gc = (c < D) ? s[c] : s[c - D] + M;
                double v = 0.0;
#pragma unroll
                for (int m = (r > c ? r : c); m < N; ++m) v = fma(w[m][r], w[m][c], v);
                v *= coef;
                const int hi = gr > gc ? gr : gc, lo = gr > gc ? gc : gr;
                if (private_smem) {
                    atomicAdd(sgv + (size_t)hi * (hi + 1) / 2 + lo, v);
                } else {
                    atomicAdd(gV + (size_t)hi * n2 + lo, v);  // lower triangle; mirrored at the end
                }
            }
        }
    }
    if (private_smem) {
        __syncthreads();
        for (size_t q = threadIdx.x; q < ntri; q += blockDim.x) {
            const double v = sgv[q];
            if (v == 0.0) continue;
            // q = hi*(hi+1)/2 + lo
            int hi = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
            while ((size_t)hi * (hi + 1) / 2 > q) --hi;
            while ((size_t)(hi + 1) * (hi + 2) / 2 <= q) ++hi;
            const int lo = (int)(q - (size_t)hi * (hi + 1) / 2);
            atomicAdd(gV + (size_t)hi * n2 + lo, v);
        }
    }
}

// gP0 by gathering: for the order-b subset B,
//   gP0(B) = sum over R disjoint from B, |R| <= kmax - b, of g_y(B + R) h(R),
// with g_y(S) = (-1)^{|S|} g(S) and h(empty) = 1.
//
// Each nonempty R is split as R' + {z} with z = max R, and the work unit is the
// pair (B, R'): its thread walks z upward from max R' + 1 through the gaps of B.
// With g elements of B below z and r = |R| = |R'| + 1, the colex ranks are
//   rank(R' + {z})     = rank(R') + C(z, r),
//   rank(B + R' + {z}) = c_g + C(z, r + g),
// where c_g sums C(e, position + 1) over the other elements e of B + R'. When z
// passes B[g], that element moves from position g + r to g + r - 1, so c_g gains
// C(B[g], g + r) and loses C(B[g], g + r + 1). The column C(z, 0..b+r) follows z
// by Pascal's rule, so each term costs two loads, one FMA and b + r integer adds.
//
// A team of T threads (a power of two) owns one B: lane l takes the units
// l, l + T, ... of the U = sum_{s < kmax - b} C(M - b, s) sets R' (all s-subsets
// of the modes outside B, s = |R'|, ordered by size then colex rank), and the
// team adds its lanes in a fixed order, so the result does not depend on timing.

// Sum over z of g_y(B + R' + {z}) h(R' + {z}) for one unit with |R'| = R - 1.
template <int BB, int R>
__device__ __forceinline__ double gather_walk(int M, const Offsets &o, const int *B, const int *Rp,
                                              const double *__restrict__ gk, const double *__restrict__ h) {
    const int z0 = R > 1 ? Rp[R - 2] + 1 : 0;
    int g0 = 0;
#pragma unroll
    for (int k = 0; k < BB; ++k) g0 += B[k] < z0;
    uint64_t rank_rp = 0, low = 0, high = 0;
#pragma unroll
    for (int i = 0; i < R - 1; ++i) {
        int below = 0;  // elements of B below Rp[i]
#pragma unroll
        for (int k = 0; k < BB; ++k) below += B[k] < Rp[i];
        rank_rp += binom(Rp[i], i + 1);
        low += binom(Rp[i], i + below + 1);
    }
#pragma unroll
    for (int k = 0; k < BB; ++k) {
        if (k < g0) {
            int below = 0;  // elements of R' below B[k]
#pragma unroll
            for (int i = 0; i < R - 1; ++i) below += Rp[i] < B[k];
            low += binom(B[k], k + below + 1);
        } else {
            high += binom(B[k], k + R + 1);
        }
    }
    uint64_t cc[BB + R + 1];  // cc[j] = C(z, j)
#pragma unroll
    for (int j = 0; j <= BB + R; ++j) cc[j] = binom(z0, j);
    const double *hr = h + o.off[R] + rank_rp;
    double t = 0.0;
    int z = z0;
#pragma unroll
    for (int g = 0; g <= BB; ++g) {
        if (g < g0) continue;
        const int zend = g < BB ? B[g] : M;
        const double *gs = gk + o.off[BB + R] + low + high;
#pragma unroll 4
        for (; z < zend; ++z) {  // unrolled: four independent gathers in flight
            t = fma(gs[cc[R + g]], hr[cc[R]], t);
#pragma unroll
            for (int j = BB + R; j > 0; --j) cc[j] += cc[j - 1];
        }
        if (g < BB) {  // z = B[g]: step over it into the next gap
            low += cc[g + R];
            high -= cc[g + R + 1];
#pragma unroll
            for (int j = BB + R; j > 0; --j) cc[j] += cc[j - 1];
            ++z;
        }
    }
    return ((BB + R) & 1) ? -t : t;
}

template <int BB>
__global__ void __launch_bounds__(1024) gp0_gather_kernel(int M, int kmax, Offsets o, const double *__restrict__ gk,
                                                          const double *__restrict__ h, double *__restrict__ gp0,
                                                          int team) {
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t unit_b = gt / team;
    const int lane = (int)(gt % team);
    const bool live = unit_b < binom(M, BB);
    int B[BB];
    double acc = 0.0;
    if (live) {
        colex_unrank(unit_b, BB, B);
        const int rm = kmax - BB;  // largest |R|
        uint64_t cum[GBS_MAX_ORDER + 1];
        cum[0] = 0;
        for (int q = 0; q < rm; ++q) cum[q + 1] = cum[q] + binom(M - BB, q);
        const uint64_t U = cum[rm];
        for (uint64_t u = lane; u < U; u += team) {
            int sz = 0;
            while (cum[sz + 1] <= u) ++sz;
            int Rp[GBS_MAX_ORDER];
            if (sz > 0) colex_unrank(u - cum[sz], sz, Rp);
            for (int i = 0; i < sz; ++i) {  // index among the modes outside B -> mode
                int m = Rp[i];
#pragma unroll
                for (int k = 0; k < BB; ++k) m += B[k] <= m;
                Rp[i] = m;
            }
            switch (sz + 1) {
                case 1: acc += gather_walk<BB, 1>(M, o, B, Rp, gk, h); break;
                case 2: if constexpr (BB + 2 <= GBS_MAX_ORDER) acc += gather_walk<BB, 2>(M, o, B, Rp, gk, h); break;
                case 3: if constexpr (BB + 3 <= GBS_MAX_ORDER) acc += gather_walk<BB, 3>(M, o, B, Rp, gk, h); break;
                case 4: if constexpr (BB + 4 <= GBS_MAX_ORDER) acc += gather_walk<BB, 4>(M, o, B, Rp, gk, h); break;
                default: break;
            }
        }
        if (lane == 0) acc += (BB & 1) ? -gk[o.off[BB] + unit_b] : gk[o.off[BB] + unit_b];  // R empty
    }
    // team sum in a fixed order
    const int w = team < 32 ? team : 32;
    for (int off = w / 2; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, w);
    if (team <= 32) {
        if (live && lane == 0) gp0[o.off[BB] + unit_b] = acc;
    } else {  // one team per block
        __shared__ double red[32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0 && live) {
            double tot = 0.0;
            for (int k = 0; k < team / 32; ++k) tot += red[k];
            gp0[o.off[BB] + unit_b] = tot;
        }
    }
}

// gP0 for the top order: only R = empty contributes, gP0(B) = g_y(B).
__global__ void gp0_top_kernel(uint64_t n, double sign, const double *__restrict__ gk, double *__restrict__ gp0) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) gp0[i] = sign * gk[i];
}

// A_{T'}^{-1} for every order-DP subset T' (rows x of T', then p of T'), packed
// lower triangle (row-major) per T'. One thread per T'.
template <int DP>
__global__ void ainv_kernel(int M, const double *__restrict__ A, double *__restrict__ inv, unsigned *status) {
    constexpr int N = 2 * DP, NT = N * (N + 1) / 2;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= binom(M, DP)) return;
    int s[DP];
    colex_unrank(i, DP, s);
    double a[N][N];
#pragma unroll
    for (int u = 0; u < DP; ++u)
#pragma unroll
        for (int v = 0; v < DP; ++v) {
            const Blk bl = ablk(A, M, s[u], s[v]);
            a[u][v] = bl.a00;
            a[u][v + DP] = bl.a01;
            a[u + DP][v] = bl.a10;
            a[u + DP][v + DP] = bl.a11;
        }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double dkk = a[k][k];
#pragma unroll
        for (int m = 0; m < k; ++m) dkk = fma(-a[k][m], a[k][m], dkk);
        ok = ok && dkk > 0.0;
        const double ik = rsqrt(dkk);
        a[k][k] = ik;
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            double v = a[r][k];
#pragma unroll
            for (int m = 0; m < k; ++m) v = fma(-a[r][m], a[k][m], v);
            a[r][k] = v * ik;
        }
    }
    if (!ok) flag_status(status, ST_NOT_POSDEF);
    // W = L^{-1} (lower), stored transposed in the upper triangle: W[r][c] at a[c][r]
    // for r > c; the diagonal a[k][k] = 1 / L_kk is W[k][k].
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            double v = 0.0;
#pragma unroll
            for (int m = c; m < r; ++m) v = fma(-a[r][m], a[c][m], v);  // L[r][m] W[m][c]
            a[c][r] = v * a[r][r];
        }
    double *out = inv + (size_t)i * NT;
    int q = 0;
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) {
            double v = 0.0;
#pragma unroll
            for (int m = r; m < N; ++m) v = fma(a[r][m], a[c][m], v);  // (W^T W)_{rc} = sum_m W_mr W_mc
            out[q++] = v;
        }
}

// dL/dV for the order-D subsets T = {j} + T' (j < s0 = min T'), one thread per
// prefix T' (order DP = D - 1) looping over its s0 leaves. With A' = A_{T'},
// b = A[T', j], a = A_jj, u = A'^{-1} b, S = a - b^T u (the Schur complement)
// and v = u S^{-1}:
//   A_T^{-1} = [[A'^{-1} + v u^T, -v], [-v^T, S^{-1}]].
// Each contribution is C(T) A_T^{-1}, C(T) = -1/4 gP0(T) P0(T). The thread keeps
// A'^{-1} and the T' x T' block's running sum (sum_j C) A'^{-1} + sum_j C v u^T
// in registers and adds the block once; the j rows go straight to dV.
// The low orders, whose few prefixes would leave most of the GPU idle, split
// each prefix's leaves: thread x of grid row y takes leaves [y L, y L + L) of the
// prefix of colex rank x and adds its part of the T' x T' block on its own. The
// higher orders (one thread per prefix walking all its leaves) run the same
// update in double-float arithmetic (gv2df_kernel).
template <int DP, int L>
__global__ void __launch_bounds__(128) gv2_kernel(int M, Offsets o, const double *__restrict__ A,
                                                  const double *__restrict__ p0, const double *__restrict__ gp0,
                                                  const double *__restrict__ inv, double *__restrict__ gV,
                                                  unsigned *status) {
    constexpr int N = 2 * DP, NT = N * (N + 1) / 2, D = DP + 1;
    int s[DP];
    int j0, j1;
    static_assert(L > 0, "chunked leaves only");
    {
        const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (w >= binom(M, DP)) return;
        colex_unrank(w, DP, s);
        j0 = (int)blockIdx.y * L;
        j1 = j0 + L < s[0] ? j0 + L : s[0];
        if (j0 >= j1) return;
    }
    const int s0 = s[0];
    const int n2 = 2 * M;
    // A'^{-1} (packed lower triangle) of T', whose colex rank among the order-DP subsets is w
    uint64_t w = 0;
#pragma unroll
    for (int u = 0; u < DP; ++u) w += binom(s[u], u + 1);
    double ai[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) ai[q] = inv[w * NT + q];
    auto AI = [&](int r, int c) { return r >= c ? ai[r * (r + 1) / 2 + c] : ai[c * (c + 1) / 2 + r]; };
    int gr[N];
#pragma unroll
    for (int u = 0; u < N; ++u) gr[u] = u < DP ? s[u] : s[u - DP] + M;
    // rank of T = {j} + T' is baseT + j
    uint64_t baseT = o.off[D];
#pragma unroll
    for (int u = 0; u < DP; ++u) baseT += binom(s[u], u + 2);
    double sumC = 0.0, acc[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) acc[q] = 0.0;
    (void)s0;
    for (int j = j0; j < j1; ++j) {
        const double g = gp0[baseT + j];
        if (g == 0.0) continue;
        const double C = -0.25 * g * p0[baseT + j];
        double b[N][2];
#pragma unroll
        for (int u = 0; u < DP; ++u) {
            const Blk bl = ablk(A, M, s[u], j);
            b[u][0] = bl.a00;
            b[u][1] = bl.a01;
            b[u + DP][0] = bl.a10;
            b[u + DP][1] = bl.a11;
        }
        double uu[N][2];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            double x0 = 0.0, x1 = 0.0;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const double aic = AI(r, c);
                x0 = fma(aic, b[c][0], x0);
                x1 = fma(aic, b[c][1], x1);
            }
            uu[r][0] = x0;
            uu[r][1] = x1;
        }
        const Sym ajj = blk_sym(ablk(A, M, j, j));
        double S00 = ajj.s00, S01 = ajj.s01, S11 = ajj.s11;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            S00 = fma(-b[r][0], uu[r][0], S00);
            S01 = fma(-b[r][0], uu[r][1], S01);
            S11 = fma(-b[r][1], uu[r][1], S11);
        }
        const double det = fma(-S01, S01, S00 * S11);
        if (!(det > 0.0) || !(S00 > 0.0)) {
            flag_status(status, ST_NOT_POSDEF);
            continue;
        }
        const double Cd = C / det;
        const double i00 = S11 * Cd, i01 = -S01 * Cd, i11 = S00 * Cd;  // C S^{-1}
        sumC += C;
        double cv[N][2];  // C v = u (C S^{-1})
#pragma unroll
        for (int r = 0; r < N; ++r) {
            cv[r][0] = fma(uu[r][0], i00, uu[r][1] * i01);
            cv[r][1] = fma(uu[r][0], i01, uu[r][1] * i11);
        }
        int q = 0;
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c, ++q) acc[q] = fma(cv[r][0], uu[c][0], fma(cv[r][1], uu[c][1], acc[q]));
        // j rows: -C v against T', C S^{-1} on the j block; lower triangle only
        // (row >= column), mirrored at the end
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const int g0 = gr[r];
            atomicAdd(gV + (size_t)g0 * n2 + j, -cv[r][0]);  // g0 > j
            const int jm = j + M;
            if (g0 >= jm) atomicAdd(gV + (size_t)g0 * n2 + jm, -cv[r][1]);
            else atomicAdd(gV + (size_t)jm * n2 + g0, -cv[r][1]);
        }
        atomicAdd(gV + (size_t)j * n2 + j, i00);
        atomicAdd(gV + (size_t)(j + M) * n2 + j, i01);
        atomicAdd(gV + (size_t)(j + M) * n2 + j + M, i11);
    }
    if (sumC != 0.0) {
        int q = 0;
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c, ++q) {
                const double v = fma(sumC, ai[q], acc[q]);
                const int hi2 = gr[r] > gr[c] ? gr[r] : gr[c], lo2 = gr[r] > gr[c] ? gr[c] : gr[r];
                atomicAdd(gV + (size_t)hi2 * n2 + lo2, v);
            }
    }
}

// ---------------------------------------------------------------- double-float scatter
// The dL/dV scatter of the orders whose prefixes are numerous (one thread per
// prefix, gv2_kernel<DP, 0>) in double-float arithmetic on the FP32 pipe: the
// same block-inverse update, each FP64 product replaced by an unevaluated FP32
// pair (about 2^-44 relative per operation; GB300's FP32 pipe issues 62 times the
// FP64 pipe's FMAs). Inputs come from the float-pair copy of A and from FP64
// tables (A_{T'}^{-1} split once per prefix); each result is rounded to FP64
// once, for its atomic add.

// s + t, not normalised: a dot product's running sum (t gathers the rounding
// errors of the two-sums and the low parts of the products).
struct DFAcc {
    float s, t;
};

__device__ __forceinline__ void dfa_fma(DFAcc &acc, DF a, DF b) {  // acc += a b
    const float p = a.h * b.h;
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    const float s = __fadd_rn(acc.s, p);
    const float bb = __fsub_rn(s, acc.s);
    const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.s = s;
    acc.t = __fadd_rn(acc.t, __fadd_rn(err, e));
}

__device__ __forceinline__ DF dfa_val(DFAcc a) {  // two-sum s + t
    const float r = __fadd_rn(a.s, a.t);
    const float bb = __fsub_rn(r, a.s);
    return DF{r, __fadd_rn(__fsub_rn(a.s, __fsub_rn(r, bb)), __fsub_rn(a.t, bb))};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }

__device__ __forceinline__ DF df_prod(DF a, DF b) {
    DFAcc z{0.f, 0.f};
    dfa_fma(z, a, b);
    return dfa_val(z);
}

// a / b for b > 0: an FP32 quotient, corrected once by the exact residual a - q b.
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float rb = __frcp_rn(b.h);
    const float q1 = a.h * rb;
    DFAcc r{a.h, a.l};
    dfa_fma(r, DF{-q1, 0.f}, b);
    const float q2 = __fadd_rn(r.s, r.t) * rb;
    const float q = __fadd_rn(q1, q2);
    return DF{q, __fsub_rn(q2, __fsub_rn(q, q1))};
}

__device__ __forceinline__ DF df_of(double x) {
    DF r;
    split_df(x, r.h, r.l);
    return r;
}

__device__ __forceinline__ double df_to_double(DF a) { return f2d_bits(a.h) + f2d_bits(a.l); }

// One thread per prefix T' walking all its leaves j < s0 = min T' (the block
// inverse update of gv2_kernel). Prefixes are numbered by their smallest element
// s0 (the C(M-1-s0, DP-1) of them with smallest element s0 follow the
// C(M-1, DP) - C(M-s0, DP) with a smaller one, s0 >= 1), so the threads of a warp
// share s0 and the trip count; the largest s0 come first (thread gi takes prefix
// n - 1 - gi).
template <int DP>
__global__ void __launch_bounds__(128) gv2df_kernel(int M, Offsets o, const float *__restrict__ Af,
                                                    const double *__restrict__ p0, const double *__restrict__ gp0,
                                                    const double *__restrict__ inv, double *__restrict__ gV,
                                                    unsigned *status) {
    constexpr int N = 2 * DP, NT = N * (N + 1) / 2, D = DP + 1;
    int s[DP];
    const uint64_t nthr = binom(M - 1, DP);
    const uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= nthr) return;
    const uint64_t i = nthr - 1 - gi;
    int lo = 1, hi = M - DP + 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (nthr - binom(M - mid, DP) <= i) lo = mid;
        else hi = mid;
    }
    s[0] = lo;
    if constexpr (DP > 1) {
        int e[DP - 1];
        colex_unrank(i - (nthr - binom(M - lo, DP)), DP - 1, e);
#pragma unroll
        for (int k = 0; k < DP - 1; ++k) s[k + 1] = lo + 1 + e[k];
    }
    const int s0 = s[0];
    const int n2 = 2 * M;
    uint64_t w = 0;
#pragma unroll
    for (int u = 0; u < DP; ++u) w += binom(s[u], u + 1);
    const double *invw = inv + w * NT;
    DF ai[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) ai[q] = df_of(invw[q]);
    auto AI = [&](int r, int c) { return r >= c ? ai[r * (r + 1) / 2 + c] : ai[c * (c + 1) / 2 + r]; };
    int gr[N];
#pragma unroll
    for (int u = 0; u < N; ++u) gr[u] = u < DP ? s[u] : s[u - DP] + M;
    uint64_t baseT = o.off[D];
#pragma unroll
    for (int u = 0; u < DP; ++u) baseT += binom(s[u], u + 2);
    const float4 *A4 = reinterpret_cast<const float4 *>(Af);
    double sumC = 0.0;
    DFAcc acc[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) acc[q] = DFAcc{0.f, 0.f};
    // The lanes of a warp share s0 (and so their trip count). Each starts its walk
    // over the leaves at its own j, so that their atomic adds to row s0 and to the
    // j diagonal block go to different addresses instead of one.
    int j = (int)(threadIdx.x & 31u) % s0;
    for (int t = 0; t < s0; ++t, j = (j + 1 == s0) ? 0 : j + 1) {
        const double g = gp0[baseT + j];
        if (g == 0.0) continue;
        const double C64 = -0.25 * g * p0[baseT + j];
        const DF C = df_of(C64);
        DF b[N][2];
#pragma unroll
        for (int u = 0; u < DP; ++u) {
            const size_t bi = 2 * ((size_t)s[u] * M + j);
            const float4 bh = A4[bi], bl = A4[bi + 1];
            b[u][0] = DF{bh.x, bl.x};
            b[u][1] = DF{bh.y, bl.y};
            b[u + DP][0] = DF{bh.z, bl.z};
            b[u + DP][1] = DF{bh.w, bl.w};
        }
        DF uu[N][2];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            DFAcc x0{0.f, 0.f}, x1{0.f, 0.f};
#pragma unroll
            for (int c = 0; c < N; ++c) {
                dfa_fma(x0, AI(r, c), b[c][0]);
                dfa_fma(x1, AI(r, c), b[c][1]);
            }
            uu[r][0] = dfa_val(x0);
            uu[r][1] = dfa_val(x1);
        }
        const size_t di = 2 * ((size_t)j * M + j);
        const float4 dh = A4[di], dl = A4[di + 1];
        DFAcc S00{dh.x, dl.x}, S11{dh.w, dl.w};
        // the symmetric part of the off-diagonal pair, (a01 + a10) / 2, as for blk_sym
        DFAcc S01{dh.y, dl.y};
        dfa_fma(S01, DF{dh.z, dl.z}, DF{1.f, 0.f});
        S01.s *= 0.5f;
        S01.t *= 0.5f;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            dfa_fma(S00, df_neg(b[r][0]), uu[r][0]);
            dfa_fma(S01, df_neg(b[r][0]), uu[r][1]);
            dfa_fma(S11, df_neg(b[r][1]), uu[r][1]);
        }
        const DF s00 = dfa_val(S00), s01 = dfa_val(S01), s11 = dfa_val(S11);
        DFAcc dt{0.f, 0.f};
        dfa_fma(dt, s00, s11);
        dfa_fma(dt, df_neg(s01), s01);
        const DF det = dfa_val(dt);
        if (!(det.h > 0.f) || !(s00.h > 0.f)) {
            flag_status(status, ST_NOT_POSDEF);
            continue;
        }
        sumC += C64;
        const DF Cd = df_div(C, det);
        const DF i00 = df_prod(s11, Cd), i01 = df_neg(df_prod(s01, Cd)), i11 = df_prod(s00, Cd);  // C S^{-1}
        DF cv[N][2];  // C v = u (C S^{-1})
#pragma unroll
        for (int r = 0; r < N; ++r) {
            DFAcc c0{0.f, 0.f}, c1{0.f, 0.f};
            dfa_fma(c0, uu[r][0], i00);
            dfa_fma(c0, uu[r][1], i01);
            dfa_fma(c1, uu[r][0], i01);
            dfa_fma(c1, uu[r][1], i11);
            cv[r][0] = dfa_val(c0);
            cv[r][1] = dfa_val(c1);
        }
        int q = 0;
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c, ++q) {
                dfa_fma(acc[q], cv[r][0], uu[c][0]);
                dfa_fma(acc[q], cv[r][1], uu[c][1]);
            }
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const int g0 = gr[r];
            atomicAdd(gV + (size_t)g0 * n2 + j, -df_to_double(cv[r][0]));  // g0 > j
            const int jm = j + M;
            const double v1 = -df_to_double(cv[r][1]);
            if (g0 >= jm) atomicAdd(gV + (size_t)g0 * n2 + jm, v1);
            else atomicAdd(gV + (size_t)jm * n2 + g0, v1);
        }
        atomicAdd(gV + (size_t)j * n2 + j, df_to_double(i00));
        atomicAdd(gV + (size_t)(j + M) * n2 + j, df_to_double(i01));
        atomicAdd(gV + (size_t)(j + M) * n2 + j + M, df_to_double(i11));
    }
    if (sumC != 0.0) {
        int q = 0;
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c, ++q) {
                const double v = fma(sumC, invw[q], df_to_double(dfa_val(acc[q])));
                const int hi2 = gr[r] > gr[c] ? gr[r] : gr[c], lo2 = gr[r] > gr[c] ? gr[c] : gr[r];
                atomicAdd(gV + (size_t)hi2 * n2 + lo2, v);
            }
    }
}

// Mirror the accumulated lower triangle of dV into the upper triangle.
__global__ void mirror_kernel(int n2, double *__restrict__ gV) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n2 * n2) return;
    const int r = (int)(idx / n2), c = (int)(idx % n2);
    if (r < c) gV[idx] = gV[(size_t)c * n2 + r];
}

BwdLayout bwd_layout(int M, int kmax, int sms) {
    BwdLayout b{};
    b.fwd = ws_layout(M, kmax, sms);  // packing, status, scratch slots
    const uint64_t N = order_offset(M, kmax + 1);
    size_t off = b.fwd.total;
    b.p0_off = off;
    off += ((sizeof(double) * N + 255) & ~(size_t)255);
    b.h_off = off;
    off += ((sizeof(double) * order_offset(M, kmax) + 255) & ~(size_t)255);
    b.gp0_off = off;
    off += ((sizeof(double) * N + 255) & ~(size_t)255);
    // inverses of A_{T'} for one prefix order at a time (orders 1..kmax-1 reuse the
    // region), sized for the order that needs the most: C(M, dp) packed
    // 2dp x 2dp lower triangles, which for small M is not always dp = kmax - 1
    size_t inv_doubles = 0;
    for (int dp = 1; dp < kmax; ++dp) {
        const size_t n = (size_t)binom(M, dp) * (size_t)(dp * (2 * dp + 1));
        if (n > inv_doubles) inv_doubles = n;
    }
    b.inv_off = off;
    off += ((sizeof(double) * inv_doubles + 255) & ~(size_t)255);
    b.total = off;
    return b;
}

cudaError_t launch_backward(const BwdArgs &a, cudaStream_t st) {
    const int M = a.M, K = a.kmax;
    const Offsets o = make_offsets(M);
    cudaError_t e;
    auto mark = [&](int i) {
        if (a.ev) cudaEventRecord(a.ev[i], st);
    };
    mark(0);
    // 1. P0 table of every order (forward kernels, refined FP32: relative error
    //    about 1e-13, well inside what the double-float scatter keeps; its packing
    //    also leaves the float-pair copy of A that the scatter reads)
    FwdArgs f = a.fwd;
    f.mode = MODE_P0;
    f.precision = GBS_FP32_REFINED;
    f.p0 = f.out = a.p0;
    if ((e = launch_forward(f, st)) != cudaSuccess) return e;
    mark(1);
    // 2. h table, orders 1..kmax-1
    for (int r = 1; r < K; ++r) {
        const uint64_t n = binom(M, r);
        h_kernel<<<(unsigned)((n + BWD_THREADS - 1) / BWD_THREADS), BWD_THREADS, 0, st>>>(M, r, o, a.p0, a.h);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(2);
    // 3. gP0 by gathering over supersets (one team of threads per subset B)
    for (int b = 1; b <= K; ++b) {
        const uint64_t n = binom(M, b);
        if (b == K) {
            gp0_top_kernel<<<(unsigned)((n + BWD_THREADS - 1) / BWD_THREADS), BWD_THREADS, 0, st>>>(
                n, (K & 1) ? -1.0 : 1.0, a.gk + o.off[K], a.gp0 + o.off[K]);
        } else {
            // team size: about four units per lane, at most one block per B
            uint64_t units = 0;
            for (int q = 0; q < K - b; ++q) units += binom(M - b, q);
            int team = 1;
            while (team < 1024 && 4 * (uint64_t)team < units) team *= 2;
            const int nt = team > 32 ? team : 256;  // a team wider than a warp fills its block
            const unsigned gl = (unsigned)((n * team + nt - 1) / nt);
            if (b == 1) gp0_gather_kernel<1><<<gl, nt, 0, st>>>(M, K, o, a.gk, a.h, a.gp0, team);
            else if (b == 2) gp0_gather_kernel<2><<<gl, nt, 0, st>>>(M, K, o, a.gk, a.h, a.gp0, team);
            else if (b == 3) gp0_gather_kernel<3><<<gl, nt, 0, st>>>(M, K, o, a.gk, a.h, a.gp0, team);
            else gp0_gather_kernel<4><<<gl, nt, 0, st>>>(M, K, o, a.gk, a.h, a.gp0, team);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(3);
    // 4. grad_V: order 1 directly, higher orders per prefix T'
    const size_t n2 = 2 * (size_t)M;
    if ((e = cudaMemsetAsync(a.gV, 0, sizeof(double) * n2 * n2, st)) != cudaSuccess) return e;
    gv_kernel<1><<<(unsigned)((M + BWD_THREADS - 1) / BWD_THREADS), BWD_THREADS, 0, st>>>(M, o, f.A, a.p0, a.gp0,
                                                                                       a.gV, false, f.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int d = 2; d <= K; ++d) {
        const uint64_t nt = binom(M, d - 1);
        const unsigned gi = (unsigned)((nt + BWD_THREADS - 1) / BWD_THREADS);
        const unsigned gw = (unsigned)((binom(M - 1, d - 1) + 127) / 128);
        // orders 2 and 3: (prefix, 4 leaves) per thread
        const dim3 gc((unsigned)((nt + 127) / 128), (unsigned)((M + 3) / 4));
        switch (d) {
#define GV2_CASE(DD)                                                                                        \
    case DD:                                                                                                \
        ainv_kernel<DD - 1><<<gi, BWD_THREADS, 0, st>>>(M, f.A, a.inv, f.status);                          \
        if ((e = cudaGetLastError()) != cudaSuccess) return e;                                             \
        if (DD <= 3) gv2_kernel<DD - 1, 4><<<gc, 128, 0, st>>>(M, o, f.A, a.p0, a.gp0, a.inv, a.gV, f.status); \
        else if (gw) gv2df_kernel<DD - 1><<<gw, 128, 0, st>>>(M, o, f.Af, a.p0, a.gp0, a.inv, a.gV, f.status); \
        break;
            GV2_CASE(2)
            GV2_CASE(3)
            GV2_CASE(4)
            GV2_CASE(5)
#undef GV2_CASE
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mirror_kernel<<<(unsigned)((n2 * n2 + BWD_THREADS - 1) / BWD_THREADS), BWD_THREADS, 0, st>>>((int)n2, a.gV);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(4);
    return cudaSuccess;
}

// ---------------------------------------------------------------- covariance model

// V = D W D + I - D^2, W = S Q S^T, S = [[Re U, -Im U], [Im U, Re U]],
// Q = diag(e^{-2r}, e^{2r}), D = diag(sqrt(eta), sqrt(eta))  (Eq. ground_truth_cov
// with hbar = 2 and the per-mode loss T = diag(sqrt(eta)) U).
__device__ __forceinline__ double smat(const double *Ur, const double *Ui, int M, int a, int k) {
    // S[a][k] for a, k in [0, 2M)
    const int ar = a < M ? a : a - M, kc = k < M ? k : k - M;
    const double re = Ur[(size_t)ar * M + kc], im = Ui[(size_t)ar * M + kc];
    if (a < M) return k < M ? re : -im;
    return k < M ? im : re;
}

__device__ __forceinline__ double qdiag(const double *r, int M, int k) {
    return k < M ? exp(-2.0 * r[k]) : exp(2.0 * r[k - M]);
}

// V = D (S Q S^T) D + I - D^2 with D = diag(sqrt(eta)) (eta repeated for the
// x and p blocks), Q = diag(e^{-2r}, e^{2r}): a 2M x 2M symmetric product, tiled
// 32 x 32. Each block computes one tile on or below the diagonal (256 threads,
// four rows each) and writes it and its mirror; the k dimension advances 32 at
// a time through shared memory, with the 32 entries of Q of that step computed
// once per block.
constexpr int COV_TILE = 32;

__global__ void __launch_bounds__(256) covariance_kernel(const double *Ur, const double *Ui, const double *r,
                                                         const double *eta, int M, double *V) {
    __shared__ double As[COV_TILE][COV_TILE + 1], Bs[COV_TILE][COV_TILE + 1];
    const int n2 = 2 * M;
    // block -> tile (ta, tb) with tb <= ta
    int ta = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) * 0.5);
    while ((ta + 1) * (ta + 2) / 2 <= (int)blockIdx.x) ++ta;
    while (ta * (ta + 1) / 2 > (int)blockIdx.x) --ta;
    const int tb = (int)blockIdx.x - ta * (ta + 1) / 2;
    const int a0 = ta * COV_TILE, b0 = tb * COV_TILE;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = 0; k0 < n2; k0 += COV_TILE) {
        const int k = k0 + tx;
        const double q = k < n2 ? qdiag(r, M, k) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = ty + 8 * u;
            As[row][tx] = (a0 + row < n2 && k < n2) ? smat(Ur, Ui, M, a0 + row, k) * q : 0.0;
            Bs[row][tx] = (b0 + row < n2 && k < n2) ? smat(Ur, Ui, M, b0 + row, k) : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < COV_TILE; ++kk) {
            const double bv = Bs[tx][kk];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(As[ty + 8 * u][kk], bv, acc[u]);
        }
        __syncthreads();
    }
    const int b = b0 + tx;
    if (b >= n2) return;
    const double db = sqrt(eta[b < M ? b : b - M]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int a = a0 + ty + 8 * u;
        if (a >= n2 || b > a) continue;
        const double da = sqrt(eta[a < M ? a : a - M]);
        double v = da * acc[u] * db;
        if (a == b) v += 1.0 - da * da;
        V[(size_t)a * n2 + b] = v;
        V[(size_t)b * n2 + a] = v;
    }
}

// One block per mode i, threads over rows a (and columns b for eta):
//   dL/dr_i   = -2 e^{-2 r_i} H_ii + 2 e^{2 r_i} H_{i+M,i+M},  H = S^T (D G D) S
//   dL/deta_i = sum_{a in {i, i+M}} [ sum_b (G_ab + G_ba)(V_ab - delta_ab (1 - eta_i)) / (2 eta_i) - G_aa ]
// (the second uses W_ab D_b = (V_ab - delta_ab (1 - D_a^2)) / D_a).
__global__ void covariance_bwd_kernel(const double *Ur, const double *Ui, const double *r, const double *eta, int M,
                                      const double *V, const double *G, double *dr, double *deta) {
    extern __shared__ double cov_sh[];  // columns i and i + M of D S: 2 x 2M doubles
    const int n2 = 2 * M;
    const int i = blockIdx.x;
    double *ds0 = cov_sh, *ds1 = cov_sh + n2;
    for (int b = threadIdx.x; b < n2; b += blockDim.x) {
        const double db = sqrt(eta[b < M ? b : b - M]);
        ds0[b] = db * smat(Ur, Ui, M, b, i);
        ds1[b] = db * smat(Ur, Ui, M, b, i + M);
    }
    __syncthreads();
    double hx = 0.0, hp = 0.0, te = 0.0;
    for (int a = threadIdx.x; a < n2; a += blockDim.x) {
        double tx = 0.0, tp = 0.0;
        const double *Ga = G + (size_t)a * n2;
        for (int b = 0; b < n2; ++b) {
            const double gab = Ga[b];
            tx = fma(gab, ds0[b], tx);
            tp = fma(gab, ds1[b], tp);
        }
        hx = fma(ds0[a], tx, hx);
        hp = fma(ds1[a], tp, hp);
        // eta term, thread a plays the column b
        for (int q = 0; q < 2; ++q) {
            const int ra = i + q * M;
            const double vab = V[(size_t)ra * n2 + a] - (ra == a ? 1.0 - eta[i] : 0.0);
            te = fma(G[(size_t)ra * n2 + a] + G[(size_t)a * n2 + ra], vab, te);
        }
    }
    __shared__ double red[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        hx += __shfl_down_sync(0xffffffffu, hx, o);
        hp += __shfl_down_sync(0xffffffffu, hp, o);
        te += __shfl_down_sync(0xffffffffu, te, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = hx;
        red[1][w] = hp;
        red[2][w] = te;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sx = 0.0, sp = 0.0, se = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sx += red[0][k];
            sp += red[1][k];
            se += red[2][k];
        }
        dr[i] = -2.0 * exp(-2.0 * r[i]) * sx + 2.0 * exp(2.0 * r[i]) * sp;
        deta[i] = se / (2.0 * eta[i]) - G[(size_t)i * n2 + i] - G[(size_t)(i + M) * n2 + i + M];
    }
}

cudaError_t launch_covariance(const double *Ur, const double *Ui, const double *r, const double *eta, int M, double *V,
                              cudaStream_t st) {
    const int nt = (2 * M + COV_TILE - 1) / COV_TILE;
    covariance_kernel<<<nt * (nt + 1) / 2, 256, 0, st>>>(Ur, Ui, r, eta, M, V);
    return cudaGetLastError();
}

cudaError_t launch_covariance_bwd(const double *Ur, const double *Ui, const double *r, const double *eta, int M,
                                  const double *V, const double *G, double *dr, double *deta, cudaStream_t st) {
    const size_t smem = sizeof(double) * 4 * (size_t)M;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(covariance_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    covariance_bwd_kernel<<<M, 256, smem, st>>>(Ur, Ui, r, eta, M, V, G, dr, deta);
    return cudaGetLastError();
}

}  // namespace gbs
