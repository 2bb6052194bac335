// Device-side helpers shared by the libgbs kernels: colex combinatorics, the
// packed 2x2-block view of A = (V + I)/2, and 2x2 Cholesky/Schur steps in FP64.
#pragma once
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

namespace gbs {

// ---------------------------------------------------------------- status word
// Bits OR-ed into the workspace status word by kernels; host maps them to gbs_status.
enum : unsigned {
    ST_NOT_POSDEF = 1u << 0,
    ST_TIMEOUT = 1u << 1,
    ST_BAD_INDEX = 1u << 2,
};

// ---------------------------------------------------------------- combinatorics
// C(n, k) for 0 <= k <= 6; 0 if n < k or k < 0. Each step r <- r (n - i) / (i + 1)
// keeps r = C(n, i + 1) exact, and the divisors are constants, so no runtime
// 64-bit division is emitted. The largest intermediate, C(n, k-1) (n - k + 1),
// stays below 2^64 for k <= 5 up to n = 4096 and for k = 6 up to n = 1030.
__host__ __device__ __forceinline__ uint64_t binom(int n, int k) {
    if (n < k || k < 0) return 0;
    const uint64_t N = (uint64_t)n;
    uint64_t r = 1;
    if (k >= 1) r = N;
    if (k >= 2) r = r * (N - 1) / 2;
    if (k >= 3) r = r * (N - 2) / 3;
    if (k >= 4) r = r * (N - 3) / 4;
    if (k >= 5) r = r * (N - 4) / 5;
    if (k >= 6) r = r * (N - 5) / 6;
    return r;
}

__host__ __device__ __forceinline__ uint64_t binom2(int n) { return n < 2 ? 0 : (uint64_t)n * (n - 1) / 2; }

// Largest c >= k-1 with C(c, k) <= r (the top element when unranking r in colex
// order at level k). Starts from a floating-point root estimate and corrects it.
__device__ __forceinline__ int colex_top(uint64_t r, int k) {
    if (k == 1) return (int)r;
    float fr = (float)r;
    float est;
    // C(c, k) ~ (c - (k-1)/2)^k / k!, so c ~ (k! r)^(1/k) + (k-1)/2; the loops
    // below correct the estimate exactly
    if (k == 2) est = 0.5f * (1.f + sqrtf(1.f + 8.f * fr));
    else if (k == 3) est = cbrtf(6.f * fr) + 1.f;
    else if (k == 4) est = sqrtf(sqrtf(24.f * fr)) + 1.5f;
    else {
        float kf = 1.f;
        for (int i = 2; i <= k; ++i) kf *= (float)i;
        est = powf(fr * kf, 1.f / (float)k) + 0.5f * (float)(k - 1);
    }
    int c = (int)est;
    if (c < k - 1) c = k - 1;
    while (binom(c, k) > r) --c;
    while (binom(c + 1, k) <= r) ++c;
    return c;
}

// Sorted modes (ascending) of colex rank r among d-subsets.
__device__ __forceinline__ void colex_unrank(uint64_t r, int d, int *modes) {
    for (int k = d; k >= 1; --k) {
        int c = colex_top(r, k);
        modes[k - 1] = c;
        r -= binom(c, k);
    }
}

// Pair index t = C(c2, 2) + j  ->  (c2, j) with j < c2.
__device__ __forceinline__ void pair_decode(uint32_t t, int &c2, int &j) {
    int c = (int)(0.5f * (1.f + sqrtf(1.f + 8.f * (float)t)));
    while ((uint32_t)binom2(c) > t) --c;
    while ((uint32_t)binom2(c + 1) <= t) ++c;
    c2 = c;
    j = (int)(t - (uint32_t)binom2(c));
}

// Offset of the order-d group: sum_{e=1}^{d-1} C(M, e).
__host__ __device__ __forceinline__ uint64_t order_offset(int M, int d) {
    uint64_t off = 0;
    for (int e = 1; e < d; ++e) off += binom(M, e);
    return off;
}

// ---------------------------------------------------------------- 2x2 blocks
// A 2x2 block of a (Schur-complemented) A = (V+I)/2 between modes x (rows x, x+M)
// and y (cols y, y+M): {a00, a01, a10, a11} = {A[x][y], A[x][y+M], A[x+M][y], A[x+M][y+M]}.
struct Blk {
    double a00, a01, a10, a11;
};
// Symmetric 2x2 block (diagonal blocks): {s00, s01, s11}.
struct Sym {
    double s00, s01, s11;
};
// Inverse of the lower Cholesky factor of a 2x2 SPD block: [[m00, 0], [m10, m11]].
struct LInv {
    double m00, m10, m11;
};

__device__ __forceinline__ Blk load_blk(const double *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 u = q[0], v = q[1];
    return Blk{u.x, u.y, v.x, v.y};
}
__device__ __forceinline__ void store_blk(double *p, const Blk &b) {
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(b.a00, b.a01);
    q[1] = make_double2(b.a10, b.a11);
}

// Lower Cholesky factor inverse of [[s00, s01], [s01, s11]]; ok = false unless
// both pivots are positive. det = s00 * (s11 - s01^2/s00).
__device__ __forceinline__ LInv chol2_inv(const Sym &s, bool &ok, double &det) {
    double ia = rsqrt(s.s00);             // 1 / l00
    double l10 = s.s01 * ia;
    double p2 = fma(-l10, l10, s.s11);     // l11^2
    double ib = rsqrt(p2);                 // 1 / l11
    ok = (s.s00 > 0.0) && (p2 > 0.0);
    det = s.s00 * p2;
    return LInv{ia, -l10 * ia * ib, ib};
}

// W = Linv * X for a 2x2 block X (rows = pivot components).
__device__ __forceinline__ Blk lmul(const LInv &m, const Blk &x) {
    Blk w;
    w.a00 = m.m00 * x.a00;
    w.a01 = m.m00 * x.a01;
    w.a10 = fma(m.m10, x.a00, m.m11 * x.a10);
    w.a11 = fma(m.m10, x.a01, m.m11 * x.a11);
    return w;
}

// d - W^T W for a symmetric block d.
__device__ __forceinline__ Sym sym_sub_gram(const Sym &d, const Blk &w) {
    Sym s;
    s.s00 = fma(-w.a10, w.a10, fma(-w.a00, w.a00, d.s00));
    s.s01 = fma(-w.a10, w.a11, fma(-w.a00, w.a01, d.s01));
    s.s11 = fma(-w.a11, w.a11, fma(-w.a01, w.a01, d.s11));
    return s;
}

// X - Za^T Zb for 2x2 blocks.
__device__ __forceinline__ Blk blk_sub_cross(const Blk &x, const Blk &za, const Blk &zb) {
    Blk r;
    r.a00 = fma(-za.a10, zb.a10, fma(-za.a00, zb.a00, x.a00));
    r.a01 = fma(-za.a10, zb.a11, fma(-za.a00, zb.a01, x.a01));
    r.a10 = fma(-za.a11, zb.a10, fma(-za.a01, zb.a00, x.a10));
    r.a11 = fma(-za.a11, zb.a11, fma(-za.a01, zb.a01, x.a11));
    return r;
}

__device__ __forceinline__ double det_sym(const Sym &s) { return fma(-s.s01, s.s01, s.s00 * s.s11); }

__device__ __forceinline__ Sym blk_sym(const Blk &b) { return Sym{b.a00, 0.5 * (b.a01 + b.a10), b.a11}; }

// Packed A: block (x, y) at ablk + 4*(x*M + y).
__device__ __forceinline__ Blk ablk(const double *A, int M, int x, int y) {
    return load_blk(A + 4 * ((size_t)x * M + y));
}

// ---------------------------------------------------------------- first moments
// Displaced states: with b = mean / 2 per mode (b_k = (mean[k], mean[k+M]) / 2),
// the exponent of Eq. vacuum_gaussian_prob (hbar = 2) is
// -1/2 mean^T (V + I)^{-1} mean = -b^T A^{-1} b. Under the elimination of a pivot
// p with inverse factor m_p, a mode x's reduced half-mean becomes
// b(x) - y(x)^T g_p, y(x) = m_p A[p, x], g_p = m_p b(p); the leaf j left after
// eliminating S' contributes r^T Sch_j^{-1} r with r its reduced half-mean.
struct Vec2 {
    double v0, v1;
};

__device__ __forceinline__ Vec2 half_mean(const double *mean, int M, int k) {
    return Vec2{0.5 * mean[k], 0.5 * mean[k + M]};
}

// m * b for an inverse Cholesky factor m.
__device__ __forceinline__ Vec2 lvec(const LInv &m, const Vec2 &b) {
    return Vec2{m.m00 * b.v0, fma(m.m10, b.v0, m.m11 * b.v1)};
}

// r - w^T g for a 2x2 block w (rows = pivot components).
__device__ __forceinline__ Vec2 sub_wtg(const Vec2 &r, const Blk &w, const Vec2 &g) {
    return Vec2{fma(-w.a10, g.v1, fma(-w.a00, g.v0, r.v0)), fma(-w.a11, g.v1, fma(-w.a01, g.v0, r.v1))};
}

// r^T S^{-1} r for a 2x2 SPD block S, given 1 / det S.
__device__ __forceinline__ double quad_inv(const Sym &s, double idet, const Vec2 &r) {
    return idet * fma(s.s11 * r.v0, r.v0, fma(-2.0 * s.s01 * r.v0, r.v1, s.s00 * r.v1 * r.v1));
}

__device__ __forceinline__ void flag_status(unsigned *status, unsigned bits) {
    if (status) atomicOr(status, bits);
}

// Host-side fault injection, for tests of the error paths: true when the
// environment variable GBS_FAULT_INJECT lists `site` (comma-separated names).
// Sites: "forward_memset" (the forward calls' first runtime call is treated as
// failed, GBS_ERR_CUDA), "sampler_no_loads" (the sampler's tensor-core step
// product issues no copies and gives up its first wait quickly, so the call
// reports GBS_ERR_TIMEOUT with nothing in flight). Nothing faults on the GPU.
inline bool fault_injected(const char *site) {
    const char *env = getenv("GBS_FAULT_INJECT");
    if (!env || !*env) return false;
    const size_t n = strlen(site);
    for (const char *p = env; (p = strstr(p, site)) != nullptr; p += n)
        if ((p == env || p[-1] == ',') && (p[n] == '\0' || p[n] == ',')) return true;
    return false;
}

}  // namespace gbs
