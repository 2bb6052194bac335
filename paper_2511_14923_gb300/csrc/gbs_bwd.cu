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
//     dP0(T)/dV_T = -1/2 P0(T) (V_T + I)^{-1} = -1/4 P0(T) A_T^{-1}.
// grad_V is the symmetric gradient: for every symmetric perturbation dV,
// dL = sum_ab grad_V[a][b] dV[a][b].
#include <cstdio>

#include "gbs.h"
#include "gbs_bwd.cuh"
#include "gbs_common.cuh"

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

// gP0 scatter, order d: every nonempty B subset S receives g_y(S) h(S - B).
__global__ void gp0_kernel(int M, int d, Offsets o, const double *__restrict__ gk, const double *__restrict__ h,
                           double *__restrict__ gp0) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= binom(M, d)) return;
    const double gy = ((d & 1) ? -1.0 : 1.0) * gk[o.off[d] + i];
    if (gy == 0.0) return;
    int s[GBS_MAX_ORDER];
    colex_unrank(i, d, s);
    const unsigned full = (1u << d) - 1;
    for (unsigned b = 1; b <= full; ++b) {
        const unsigned rest = full ^ b;
        const double hr = rest ? h[sub_index(s, d, rest, o.off)] : 1.0;
        atomicAdd(gp0 + sub_index(s, d, b, o.off), gy * hr);
    }
}

// grad_V scatter, order d: -1/4 gP0(T) P0(T) A_T^{-1} into the rows/cols of T.
// Privatised in shared memory (lower triangle of the 2M x 2M gradient) when it fits.
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
                    atomicAdd(gV + (size_t)hi * n2 + lo, v);
                    if (hi != lo) atomicAdd(gV + (size_t)lo * n2 + hi, v);
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
            if (hi != lo) atomicAdd(gV + (size_t)lo * n2 + hi, v);
        }
    }
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
    b.total = off;
    return b;
}

cudaError_t launch_backward(const BwdArgs &a, cudaStream_t st) {
    const int M = a.M, K = a.kmax;
    const Offsets o = make_offsets(M);
    cudaError_t e;
    // 1. P0 table of every order (forward kernels, FP64)
    FwdArgs f = a.fwd;
    f.mode = MODE_P0;
    f.precision = GBS_FP64;
    f.p0 = f.out = a.p0;
    if ((e = launch_forward(f, st)) != cudaSuccess) return e;
    // 2. h table, orders 1..kmax-1
    for (int r = 1; r < K; ++r) {
        const uint64_t n = binom(M, r);
        h_kernel<<<(unsigned)((n + BWD_THREADS - 1) / BWD_THREADS), BWD_THREADS, 0, st>>>(M, r, o, a.p0, a.h);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 3. gP0 = sum over supersets
    const uint64_t N = order_offset(M, K + 1);
    if ((e = cudaMemsetAsync(a.gp0, 0, sizeof(double) * N, st)) != cudaSuccess) return e;
    for (int d = 1; d <= K; ++d) {
        const uint64_t n = binom(M, d);
        gp0_kernel<<<(unsigned)((n + BWD_THREADS - 1) / BWD_THREADS), BWD_THREADS, 0, st>>>(M, d, o, a.gk, a.h,
                                                                                           a.gp0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 4. grad_V
    const size_t n2 = 2 * (size_t)M;
    if ((e = cudaMemsetAsync(a.gV, 0, sizeof(double) * n2 * n2, st)) != cudaSuccess) return e;
    const size_t tri_bytes = sizeof(double) * n2 * (n2 + 1) / 2;
    const bool priv = tri_bytes <= 200 * 1024;
    const size_t smem = priv ? tri_bytes : 0;
    for (int d = 1; d <= K; ++d) {
        const uint64_t n = binom(M, d);
        uint64_t blocks = (n + BWD_THREADS - 1) / BWD_THREADS;
        const uint64_t cap = priv ? (uint64_t)a.fwd.sms : (uint64_t)a.fwd.sms * 8;
        if (blocks > cap) blocks = cap;
        switch (d) {
#define GV_CASE(DD)                                                                                           \
    case DD:                                                                                                  \
        if (priv && (e = cudaFuncSetAttribute(gv_kernel<DD>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                              (int)smem)) != cudaSuccess)                                      \
            return e;                                                                                         \
        gv_kernel<DD><<<(unsigned)blocks, BWD_THREADS, smem, st>>>(M, o, f.A, a.p0, a.gp0, a.gV, priv, f.status); \
        break;
            GV_CASE(1)
            GV_CASE(2)
            GV_CASE(3)
            GV_CASE(4)
            GV_CASE(5)
#undef GV_CASE
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
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

__device__ __forceinline__ double wmat(const double *Ur, const double *Ui, const double *r, int M, int a, int b) {
    double acc = 0.0;
    for (int k = 0; k < 2 * M; ++k) acc = fma(smat(Ur, Ui, M, a, k) * qdiag(r, M, k), smat(Ur, Ui, M, b, k), acc);
    return acc;
}

__global__ void covariance_kernel(const double *Ur, const double *Ui, const double *r, const double *eta, int M,
                                  double *V) {
    const int n2 = 2 * M;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n2 * n2) return;
    const int a = idx / n2, b = idx - a * n2;
    if (b > a) return;  // lower triangle computes, mirror writes
    const double da = sqrt(eta[a < M ? a : a - M]), db = sqrt(eta[b < M ? b : b - M]);
    double v = da * wmat(Ur, Ui, r, M, a, b) * db;
    if (a == b) v += 1.0 - da * da;
    V[(size_t)a * n2 + b] = v;
    V[(size_t)b * n2 + a] = v;
}

// One block per mode i, threads over rows a (and columns b for eta):
//   dL/dr_i   = -2 e^{-2 r_i} H_ii + 2 e^{2 r_i} H_{i+M,i+M},  H = S^T (D G D) S
//   dL/deta_i = sum_{a in {i, i+M}} [ sum_b (G_ab + G_ba)(V_ab - delta_ab (1 - eta_i)) / (2 eta_i) - G_aa ]
// (the second uses W_ab D_b = (V_ab - delta_ab (1 - D_a^2)) / D_a).
__global__ void covariance_bwd_kernel(const double *Ur, const double *Ui, const double *r, const double *eta, int M,
                                      const double *V, const double *G, double *dr, double *deta) {
    const int n2 = 2 * M;
    const int i = blockIdx.x;
    double hx = 0.0, hp = 0.0, te = 0.0;
    for (int a = threadIdx.x; a < n2; a += blockDim.x) {
        double tx = 0.0, tp = 0.0;
        for (int b = 0; b < n2; ++b) {
            const double gab = G[(size_t)a * n2 + b] * sqrt(eta[b < M ? b : b - M]);
            tx = fma(gab, smat(Ur, Ui, M, b, i), tx);
            tp = fma(gab, smat(Ur, Ui, M, b, i + M), tp);
        }
        const double da = sqrt(eta[a < M ? a : a - M]);
        hx = fma(smat(Ur, Ui, M, a, i) * da, tx, hx);
        hp = fma(smat(Ur, Ui, M, a, i + M) * da, tp, hp);
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
    const int n = 4 * M * M;
    covariance_kernel<<<(n + 255) / 256, 256, 0, st>>>(Ur, Ui, r, eta, M, V);
    return cudaGetLastError();
}

cudaError_t launch_covariance_bwd(const double *Ur, const double *Ui, const double *r, const double *eta, int M,
                                  const double *V, const double *G, double *dr, double *deta, cudaStream_t st) {
    covariance_bwd_kernel<<<M, 256, 0, st>>>(Ur, Ui, r, eta, M, V, G, dr, deta);
    return cudaGetLastError();
}

}  // namespace gbs
