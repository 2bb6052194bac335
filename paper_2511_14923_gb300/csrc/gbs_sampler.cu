// Stage 2 of the emulator: the chain-rule sampler (arXiv:2511.14923, Sec. "The
// sampling algorithm", Sec. Methods and App. "Approximating marginals efficiently
// with a chain rule"), for a batch of S samples drawn in lockstep.
//
// The rule. For bits x_1..x_M (bit n = mode n-1), Eq. probs_corr_cumulants_3
// truncated at order K expands p(x_n..x_1) over the spin cumulants kappa(R+{n}),
// |R| < K, times marginals p(x_{[n-1]-R}) that are approximated by tables:
//   P[a] = p(x_a..x_1),  Pp[a][b] = p+(x_a..x_b),  P1[a][e] = p1(x_a..~x_e..x_1),
//   P2[a][e][d] = p2(x_a..~x_e..~x_d..x_1)  (K = 5 only),
// filled by truncated forms of the same rule: K = 3 single elision (Eq. methprob,
// Eq. b, Eq. a), K = 5 double elision (Eq. probade, Eq. probpartialade,
// Eq. probelidedade, Eq. probdoubleelidedade; orders 3, 3, 2 for p+, p1, p2 unless
// the caller lowers them), K = 4 the same without the |R| = 4 term (orders
// 2, 2, 1 by default). Boundary cases: P[0] = 1, an empty p+ range is 1,
// P1[a][a] = P[a-1], P2[a][a][d] = P1[a-1][d].
//
// Scaling. Each table entry over a variable set A is stored times prod_{v in A}
// s_v, with s_v = exp(H_v) and H_v the click entropy of mode v - 1 (from
// kappa({v})), so that a typical sample's values stay near 1 instead of
// decaying like e^{-sum H}. Writing hs_v = s_v / 2 and kappa'(S) = kappa(S)
// prod_{v in S} hs_v, every rule keeps its form with the factors 2^{-(|R|+1)}
// absorbed: the term of R becomes chi kappa'(R + {n}) times the scaled
// marginal, and the leading 1/2 (1 + gamma_n) becomes hs_n + chi_n kappa'_n.
// Then p(x_n = 0) and p(x_n = 1) are proportional to hs_n P~[n-1] +- B~, with B~
// the scaled odd part, and the probability of a bitstring is
// P~[M] exp(-sum_v H_v).
//
// Factorisation of the expensive terms. The terms of the bias B that reach back
// to a table row j - 1 through P2[j-1] (or P1[j-1] for K = 3) are sums over
// pairs (or single indices) below j of kappa(.., j, i, m) W_j, with
// W_j(e, d) = chi_e chi_d P2~[j-1][e][d] (K = 3: W_j(d) = chi_d P1~[j-1][d]).
// W_j only involves bits below j, so right after bit j - 1 is drawn one matrix
// product per step,
//   Z_j[row][s] = sum_r kappa[base(row) + r] W_j[r][s],
// evaluates those sums for every later (i, m) at once; in colex order the
// kappa entries of one row are contiguous, so each row is a segment of the
// table. The rows at step j are (K = 5) the order-3 set {., ., j} (used at this
// step), the order-4 sets {., ., j, n}, the order-5 sets {., ., j, i, m} and the
// pairs below j of the order-3 sets {., ., n} (X_j(n), the part of the p1 update
// whose largest index is the elided one);
// (K = 3) the order-2 set {., j} and the order-3 sets {., j, n}. At step n the
// bias then only combines stored Z values with p+ factors:
//   K = 5: B~ = kappa'_n P~[n-1] + sum_i kappa'(i,n) chi_i P1~[n-1][i] + G3
//             + sum_{i<n} chi_i Pp~[n-1][i+1] (Z3_i(n) + sum_{j<i} chi_j Pp~[i-1][j+1] Z5_j(i,n))
//   K = 3: B~ = kappa'_n P~[n-1] + G2 + sum_{i<n} chi_i Pp~[n-1][i+1] Z_i(n)
// (chi_n taken as +1: every term but hs_n P~[n-1] is odd in x_n; kappa' in every
// product row).
//
// Drawing. x_n = 0 when u_n < q0 = max(p0, 0) / (max(p0, 0) + max(p1, 0))
// (1/2 if both are <= 0); P[n] keeps the chosen branch unclipped.
//
// Layout. Every per-sample array is [entry][S] (sample index fastest), so a warp
// always touches consecutive samples of one entry: 32 with one sample per lane,
// 128 in the FP32 table updates, whose lanes hold 4 samples each (16-byte loads)
// and whose warps take one entry of one 128-sample group, the groups along the
// slow grid axis (all entries of a group in flight together share its rows in L2).
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "gbs.h"
#include "gbs_common.cuh"
#include "gbs_sampler.cuh"

namespace gbs {
namespace smp {


__host__ __device__ __forceinline__ uint64_t cb(int n, int k) { return binom(n, k); }

// Entry indices (variables 1-based).
__host__ __device__ __forceinline__ uint64_t i_pp(int a, int b) { return cb(a, 2) + (uint64_t)(b - 1); }       // 1<=b<=a
__host__ __device__ __forceinline__ uint64_t i_p1(int a, int e) { return cb(a - 1, 2) + (uint64_t)(e - 1); }   // 1<=e<a
__host__ __device__ __forceinline__ uint64_t i_p2(int a, int e, int d) {                                          // d<e<a
    return cb(a - 1, 3) + cb(e - 1, 2) + (uint64_t)(d - 1);
}
__host__ __device__ __forceinline__ uint64_t i_z(int t, int n) { return cb(n - 1, 2) + (uint64_t)(t - 1); }     // t<n
__host__ __device__ __forceinline__ uint64_t i_z5(int t, int i, int m) {                                         // t<i<m
    return cb(m - 1, 3) + cb(i - 1, 2) + (uint64_t)(t - 1);
}

template <class R>
struct Args {
    const R *kap;          // spin cumulants, orders 1..K, gbs.h layout
    uint64_t off[6];       // order offsets of the cumulant table
    int M, K, S, opp, op1, op2;
    R *chi, *P, *Pp, *P1, *P2, *Z, *Z5, *G, *Y, *X, *W;
    R *CA, *CB, *CC;       // per-step coefficients [i][S]: chi_i Pp~[n-1][i+1], kappa(i,n) chi_i, kappa(i,n) chi_i Pp~[n-1][i+1]
    R *T;                  // [C(M,2)][2][S] per-pair parts of the p1 order-3 term (see p2_kernel)
    float *At;             // tensor-core product: the step's rows, split and tiled (atc_kernel)
    const R *hs;           // per-variable half scale s_v / 2, hs[v], v = 1..M
    const R *lead;         // per-variable pairs (kappa'({v}), hs[v]) at lead[2v], lead[2v+1]
    const double *H;       // per-variable log scale ln s_v (the click entropy of mode v - 1)
    unsigned *status;      // status word (ST_* bits), first bytes of the workspace
    int use_tc;            // FP32: step product on the tensor cores
    int wait_limit;        // polls of an mbarrier before a wait gives up (ST_TIMEOUT)
    int no_loads;          // test hook: the step product issues no copies (its first wait runs out)
    uint32_t *bw;          // spins as bits: word w of sample s at bw[w * S + s], bit v & 31 = x_v
    const double *u;       // [n_samples][M] uniforms (chunk base)
    const uint8_t *force;  // [n_samples][M] or null
    uint8_t *bits;         // [n_samples][M]
    double *q0;            // [n_samples][M] or null
    int n_valid;           // samples of this chunk that are real
};

template <class R>
__device__ __forceinline__ R pp(const Args<R> &a, int x, int b, int s) {
    return b > x ? R(1) : a.Pp[i_pp(x, b) * a.S + s];
}
template <class R>
__device__ __forceinline__ R p1(const Args<R> &a, int x, int e, int s) {
    return e == x ? a.P[(size_t)(x - 1) * a.S + s] : a.P1[i_p1(x, e) * a.S + s];
}
template <class R>
__device__ __forceinline__ R p2(const Args<R> &a, int x, int e, int d, int s) {
    return e == x ? p1(a, x - 1, d, s) : a.P2[i_p2(x, e, d) * a.S + s];
}
template <class R>
__device__ __forceinline__ R chi(const Args<R> &a, int v, int s) {
    return a.chi[(size_t)v * a.S + s];
}
// Spins of one sample read from its packed bits; the current 32-bit word is
// cached, so a loop over ascending variables loads one word per 32 of them.
template <class R>
struct Spins {
    const uint32_t *bw;
    int S, s, w;
    uint32_t cur;
    __device__ Spins(const Args<R> &a, int s_) : bw(a.bw), S(a.S), s(s_), w(-1), cur(0) {}
    __device__ __forceinline__ R operator()(int v) {
        if ((v >> 5) != w) {
            w = v >> 5;
            cur = bw[(size_t)w * S + s];
        }
        return (cur >> (v & 31)) & 1u ? R(-1) : R(1);
    }
};

// (kappa'({n}), hs_n) in one vector load: the leading coefficient of every rule
// at step n is hs_n + chi_n kappa'({n}).
template <class R>
struct Pair2;
template <>
struct Pair2<float> {
    using T = float2;
};
template <>
struct Pair2<double> {
    using T = double2;
};
template <class R>
__device__ __forceinline__ typename Pair2<R>::T lead(const Args<R> &a, int n) {
    return reinterpret_cast<const typename Pair2<R>::T *>(a.lead)[n];
}

// kappa of the sorted variable set (v_1 < .. < v_d), 1-based.
template <class R>
__device__ __forceinline__ R k1(const Args<R> &a, int n) { return a.kap[a.off[1] + (n - 1)]; }
template <class R>
__device__ __forceinline__ R k2(const Args<R> &a, int i, int n) { return a.kap[a.off[2] + cb(n - 1, 2) + (i - 1)]; }
template <class R>
__device__ __forceinline__ R k3(const Args<R> &a, int j, int i, int n) {
    return a.kap[a.off[3] + cb(n - 1, 3) + cb(i - 1, 2) + (j - 1)];
}

// (x, y, z) -> decreasing order
__device__ __forceinline__ void ord3(int x, int y, int z, int &p, int &q, int &r) {
    if (x < y) { int t = x; x = y; y = t; }
    if (y < z) { int t = y; y = z; z = t; }
    if (x < y) { int t = x; x = y; y = t; }
    p = x; q = y; r = z;
}

// Pair rank -> (hi, lo), hi > lo >= 0 (colex: rank = C(hi, 2) + lo). The root
// estimate is taken in FP32 (GB300's FP64 pipe is narrow and every lane of the
// table kernels decodes its pair) and corrected exactly by the loops.
__device__ __forceinline__ void pair_of(uint64_t r, int &hi, int &lo) {
    int c = (int)(0.5f * (1.f + sqrtf(1.f + 8.f * (float)r)));
    if (c < 1) c = 1;
    while (cb(c, 2) > r) --c;
    while (cb(c + 1, 2) <= r) ++c;
    hi = c;
    lo = (int)(r - cb(c, 2));
}

// ---------------------------------------------------------------- step t: Z rows

// Rows of the product at step t and where each result goes. kbase = offset of the
// row's segment in the cumulant table; dst = its output entry (or -1 for G).
__device__ __forceinline__ void zrow(int K, int M, int t, uint64_t q, const uint64_t *off, uint64_t &kbase,
                                     int &kind, uint64_t &dst) {
    if (K == 3) {
        if (q == 0) {
            kbase = off[2] + cb(t - 1, 2);
            kind = 0;
            dst = 0;
        } else {
            const int n = t + (int)q;
            kbase = off[3] + cb(n - 1, 3) + cb(t - 1, 2);
            kind = 1;
            dst = i_z(t, n);
        }
        return;
    }
    if (q == 0) {
        kbase = off[3] + cb(t - 1, 3);
        kind = 0;
        dst = 0;
    } else if (q <= (uint64_t)(M - t)) {
        const int n = t + (int)q;
        kbase = off[4] + cb(n - 1, 4) + cb(t - 1, 3);
        kind = 1;
        dst = i_z(t, n);
    } else if (q <= 2 * (uint64_t)(M - t)) {
        // the pairs below t of the order-3 set {., ., n}: X_t(n) for the p1 update
        const int n = t + (int)(q - (uint64_t)(M - t));
        kbase = off[3] + cb(n - 1, 3);
        kind = 3;
        dst = i_z(t, n);
    } else {  // K = 5 only
        int hi, lo;
        pair_of(q - 1 - 2 * (uint64_t)(M - t), hi, lo);
        const int i = t + 1 + lo, m = t + 1 + hi;
        kbase = off[5] + cb(m - 1, 5) + cb(i - 1, 4) + cb(t - 1, 3);
        kind = 2;
        dst = i_z5(t, i, m);
    }
}

// W_t[r][s], the inner operand of the step-t product: K = 5, pair r = (e, d) of
// bits below t, chi_e chi_d P2~[t-1][e][d]; K = 3, d = r + 1, chi_d P1~[t-1][d].
// Grid: (samples / ETB, entries); the entry index is uniform in a block.
constexpr int ETB = 64;  // threads per block of the per-(entry, sample) kernels

template <class R, int K>
__global__ void __launch_bounds__(ETB) w_kernel(Args<R> a, int t, int D) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    const size_t S = (size_t)a.S;
    // this block's share of r = 0 .. D-1, walked in order
    const int per = (D + (int)gridDim.y - 1) / (int)gridDim.y;
    const int r0 = blockIdx.y * per, r1 = r0 + per < D ? r0 + per : D;
    if (r0 >= r1) return;
    Spins<R> sp(a, s);
    R *W = a.W + s;
    if (K == 3) {
        // W_t(d) = chi_d P1~[t-1][d], d = r + 1; d = t - 1 -> P~[t-2]
        const R *q = a.P1 + (t >= 3 ? i_p1(t - 1, 1) : 0) * S + s;
        for (int r = r0; r < r1; ++r) {
            const int d = r + 1;
            const R v = d == t - 1 ? a.P[(size_t)(t - 2) * S + s] : q[(size_t)r * S];
            W[(size_t)r * S] = v * sp(d);
        }
        return;
    }
    // K = 5: pair r = (e, d); for e < t - 1 the p2 row t - 1 holds the same pairs in
    // the same order (offset C(t-2, 3)); e = t - 1 comes from P1~[t-2][d] (P~[t-3]
    // when d = t - 2)
    int hi, lo;
    pair_of((uint64_t)r0, hi, lo);
    int e = hi + 1, d = lo + 1;
    Spins<R> sd(a, s);
    const uint64_t rowlen = cb(t - 2, 2);
    const R *q2 = a.P2 + (t >= 4 ? cb(t - 2, 3) : 0) * S + s;
    for (int r = r0; r < r1; ++r) {
        R v;
        if ((uint64_t)r < rowlen) v = q2[(size_t)r * S];
        else v = d == t - 2 ? a.P[(size_t)(t - 3) * S + s] : a.P1[i_p1(t - 2, d) * S + s];
        W[(size_t)r * S] = v * sp(e) * sd(d);
        if (++d == e) {
            ++e;
            d = 1;
        }
    }
}

// Z[row][s] = sum_{r < D} kappa[kbase(row) + r] W_t[r][s] for rows [0, rows) and
// all samples. 256 threads, (16 TM) x (16 TN) results per CTA, TM x TN per
// thread (two 4-wide halves each way when 8), 8 inner entries per stage with
// the next stage prefetched into registers.
template <class R, int K, int TM, int TN>
__global__ void __launch_bounds__(256) zgemm_kernel(Args<R> a, int t, uint64_t rows, int D) {
    constexpr int BMt = 16 * TM, BNt = 16 * TN, BKt = 8;
    constexpr int AE = BMt * BKt / 256, BE = BNt * BKt / 256;  // elements per thread per stage
    __shared__ __align__(16) R As[2][BKt][BMt];
    __shared__ __align__(16) R Bs[2][BKt][BNt];
    __shared__ uint64_t kb[BMt];
    __shared__ uint64_t dst[BMt];
    __shared__ int kind[BMt];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const uint64_t m0 = (uint64_t)blockIdx.x * BMt;
    const int s0 = blockIdx.y * BNt;
    for (int m = tid; m < BMt; m += 256) {
        const uint64_t q = m0 + m;
        if (q < rows) zrow(K, a.M, t, q, a.off, kb[m], kind[m], dst[m]);
        else kind[m] = -1;
    }
    __syncthreads();
    // stage loaders: A element e = tid + 256 q -> (row e / 8, inner e % 8);
    // B: BE consecutive samples of inner row tid / (BNt / BE)
    const int bk = tid / (BNt / BE), bs = (tid % (BNt / BE)) * BE;
    R ra[AE], rb[BE];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < AE; ++q) {
            const int e = tid + 256 * q, m = e / BKt, k = e % BKt;
            ra[q] = (kind[m] >= 0 && k0 + k < D) ? a.kap[kb[m] + k0 + k] : R(0);
        }
        const R *w = a.W + (size_t)(k0 + bk) * a.S + s0 + bs;
#pragma unroll
        for (int q = 0; q < BE; ++q) rb[q] = (k0 + bk < D) ? w[q] : R(0);
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < AE; ++q) {
            const int e = tid + 256 * q;
            As[buf][e % BKt][e / BKt] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) Bs[buf][bk][bs + q] = rb[q];
    };
    R acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = R(0);
    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < D; k0 += BKt) {
        const bool more = k0 + BKt < D;
        if (more) load(k0 + BKt);
#pragma unroll
        for (int k = 0; k < BKt; ++k) {
            R av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[buf][k][(i < 4 ? 0 : BMt / 2) + ty * 4 + (i & 3)];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][k][(j < 4 ? 0 : BNt / 2) + tx * 4 + (j & 3)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = (i < 4 ? 0 : BMt / 2) + ty * 4 + (i & 3);
        if (kind[m] < 0) continue;
        R *out = kind[m] == 0 ? a.G
               : kind[m] == 1 ? a.Z + dst[m] * a.S
               : kind[m] == 2 ? a.Z5 + dst[m] * a.S
                              : a.X + dst[m] * a.S;
#pragma unroll
        for (int j = 0; j < TN; ++j) out[s0 + (j < 4 ? 0 : BNt / 2) + tx * 4 + (j & 3)] = acc[i][j];
    }
}

// ---------------------------------------------------------------- step product on the tensor cores
// FP32 calls with a batch that is a multiple of 256 run the step product on the
// 5th-generation tensor cores: tcgen05.mma kind::tf32 with the 3-term split
// x = hi + lo (hi, lo TF32), Z = Ahi Bhi + Ahi Blo + Alo Bhi accumulated in FP32
// in tensor memory (the dropped Alo Blo term is ~2^-22 relative). A CTA of 128
// threads owns 128 rows x 256 samples. W arrives from wtc_kernel already split
// and laid out as the MMA's K-major core matrices (8 rows x 16 bytes, no
// swizzle), one contiguous block per TC_KC-wide K chunk and sample tile, and
// is brought in by one TMA bulk copy per chunk; the rows (cumulant segments)
// arrive the same way from atc_kernel. One elected thread issues the MMAs. A
// ring of TC_NS stages, each with a "full" mbarrier (the bulk copies' bytes) and
// an "empty" one (the MMAs' commit), keeps TC_NS - 1 chunks loading while the
// MMAs of one run; the ring takes 96 KB of shared memory, so two CTAs share a
// multiprocessor (and its 512 tensor-memory columns) and one's epilogue
// overlaps the other's MMAs. Every wait is bounded; one that runs out sets ST_TIMEOUT in the status
// word.
constexpr int TC_M = 128, TC_N = 256, TC_KC = 8, TC_NS = 4;  // TC_NS stages of TC_KC-wide chunks
constexpr int TC_ACH = TC_M * TC_KC;            // floats of one A copy (hi or lo) of one chunk
constexpr int TC_BCH = TC_N * TC_KC;            // floats of one B copy of one chunk
constexpr int TC_AB = TC_M * TC_KC * 4;         // bytes of one A copy per stage (4 KB)
constexpr int TC_BB = TC_N * TC_KC * 4;         // bytes of one B copy per stage (8 KB)
constexpr int TC_STAGE = 2 * TC_AB + 2 * TC_BB;  // A hi, A lo, B hi, B lo
constexpr int TC_SMEM = TC_NS * TC_STAGE + 256;  // stages, then 2 x TC_NS mbarriers, TMEM slot, flag
// instruction descriptor: D f32, A and B tf32, both K-major, N = 256, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row r, inner k) of an operand copy with 32-wide K
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
    const int core = (r >> 3) * (TC_KC / 4) + (k >> 2);  // core matrix: 8-row group, then 4-wide K slice
    return (uint32_t)((core * 8 + (r & 7)) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: K-major, no swizzle; leading byte offset 128
// (next core matrix along K), stride byte offset 32 TC_KC (next group of 8 rows)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((32 * TC_KC) >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

// Bounded wait for phase `parity` of the mbarrier: at most `limit` polls
// (try_wait may itself suspend the thread briefly); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// TMA bulk copies global -> shared that complete their bytes on an mbarrier;
// the expected byte count is announced once per phase.
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// W_t split into TF32 hi / lo in the tensor-core tile layout: element (r, s),
// r < KC ceil(D / KC) (zero beyond D; KC = TC_KC inner entries per chunk), at
// float offset ((c nsb + sb) 2 + part) 256 KC + tc_off(s % 256, r % KC) / 4,
// c = r / KC, sb = s / 256, nsb = S / 256. A thread forms four consecutive r (one 16-byte
// row of a core matrix) of one sample, so 8 consecutive samples write one
// 128-byte line. Grid: (samples / ETB, quads of r).
template <int K>
__global__ void __launch_bounds__(ETB) wtc_kernel(Args<float> a, int t, int D) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    const int Dp = (D + TC_KC - 1) / TC_KC * TC_KC;
    const int nsb = a.S / TC_N, sb = s / TC_N, sl = s % TC_N;
    Spins<float> sp(a, s), sd(a, s);
    // K = 4, 5: pair r = (e, d) with e < t - 1 is entry C(t-2, 3) + r of the p2
    // table (row t - 1 lists its pairs in colex order); e = t - 1 reads P1~[t-2][d]
    const size_t S = (size_t)a.S;
    const uint64_t rowlen = K == 3 ? 0 : cb(t - 2, 2);
    const float *q2 = a.P2 + (K != 3 && t >= 4 ? cb(t - 2, 3) : 0) * S + s;
    for (int qd = blockIdx.y; qd < Dp / 4; qd += gridDim.y) {
        const int r0 = 4 * qd;
        float v[4];
        int e = 0, d = 0;
        if (K != 3 && r0 < D) {
            int hi, lo;
            pair_of((uint64_t)r0, hi, lo);
            e = hi + 1;
            d = lo + 1;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + j;
            v[j] = 0.f;
            if (r < D) {
                if (K == 3) {
                    v[j] = p1(a, t - 1, r + 1, s) * sp(r + 1);
                } else {
                    const float p = (uint64_t)r < rowlen ? q2[(size_t)r * S]
                                    : d == t - 2         ? a.P[(size_t)(t - 3) * S + s]
                                                         : a.P1[i_p1(t - 2, d) * S + s];
                    v[j] = p * sp(e) * sd(d);
                    if (++d == e) {  // next pair in colex order
                        ++e;
                        d = 1;
                    }
                }
            }
        }
        float4 h, l;
        h.x = to_tf32(v[0]); l.x = to_tf32(v[0] - h.x);
        h.y = to_tf32(v[1]); l.y = to_tf32(v[1] - h.y);
        h.z = to_tf32(v[2]); l.z = to_tf32(v[2] - h.z);
        h.w = to_tf32(v[3]); l.w = to_tf32(v[3] - h.w);
        const size_t blk = ((size_t)(r0 / TC_KC) * nsb + sb) * 2 * TC_BCH;
        const uint32_t o = tc_off(sl, r0 % TC_KC) / 4;
        *reinterpret_cast<float4 *>(a.W + blk + o) = h;
        *reinterpret_cast<float4 *>(a.W + blk + TC_BCH + o) = l;
    }
}

// The rows of the step product (cumulant segments) split into TF32 hi / lo and
// laid out like W: row tile rt (128 rows), chunk c (TC_KC inner entries) at
// float offset (rt nk + c) 2 128 TC_KC, hi then lo, each in the core-matrix layout.
// Rows beyond `rows` and entries beyond D are zero. Grid: (row tiles, chunks),
// 128 threads, thread i = row i of the tile.
template <int K>
__global__ void __launch_bounds__(128) atc_kernel(Args<float> a, int t, uint64_t rows, int D) {
    const int tid = threadIdx.x, rt = blockIdx.x, c = blockIdx.y, nk = gridDim.y;
    const uint64_t q = (uint64_t)rt * TC_M + tid;
    uint64_t kb = 0, dst = 0;
    int kind = -1;
    if (q < rows) zrow(K, a.M, t, q, a.off, kb, kind, dst);
    float *blk = a.At + ((size_t)rt * nk + c) * 2 * TC_ACH;
    const float *kp = a.kap + kb;
#pragma unroll 2
    for (int j = 0; j < TC_KC; j += 4) {
        const int k = c * TC_KC + j;
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (kind >= 0 && k + i < D) ? kp[k + i] : 0.f;
        float4 h, l;
        h.x = to_tf32(v[0]); l.x = to_tf32(v[0] - h.x);
        h.y = to_tf32(v[1]); l.y = to_tf32(v[1] - h.y);
        h.z = to_tf32(v[2]); l.z = to_tf32(v[2] - h.z);
        h.w = to_tf32(v[3]); l.w = to_tf32(v[3] - h.w);
        const uint32_t o = tc_off(tid, j) / 4;
        *reinterpret_cast<float4 *>(blk + o) = h;
        *reinterpret_cast<float4 *>(blk + TC_ACH + o) = l;
    }
}

// Z rows of one 128-row tile x 256 samples. Thread 0 streams both operands by
// TMA bulk copies (A: 128 rows, W: 256 samples, hi and lo, per TC_KC-wide
// chunk) into a ring of TC_NS stages and issues the MMAs; chunk c-1+TC_NS is
// loaded into the stage of chunk c-1 once the MMAs of chunk c-1 have completed,
// while those of chunk c run. All threads then read
// the accumulator (thread i = row i) and write the rows out.
template <int K>
__global__ void __launch_bounds__(128, 2) ztc_kernel(Args<float> a, int t, uint64_t rows, int D) {
    extern __shared__ __align__(1024) unsigned char smem[];
    static_assert(TC_NS <= 8, "barrier area");
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + TC_NS * TC_STAGE);
    uint64_t *empty = full + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + TC_NS * TC_STAGE + 128);
    int *flag = reinterpret_cast<int *>(smem + TC_NS * TC_STAGE + 192);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint64_t m0 = (uint64_t)blockIdx.x * TC_M;
    const int rt = blockIdx.x, sb = blockIdx.y, s0 = sb * TC_N, nsb = a.S / TC_N;
    const int nk = (D + TC_KC - 1) / TC_KC;
    if (tid == 0) {
        for (int i = 0; i < TC_NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        *flag = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t sbase = smem_u32(smem);
        const float *Ab = a.At + (size_t)rt * nk * 2 * TC_ACH;
        const float *Wb = a.W + (size_t)sb * 2 * TC_BCH;
        auto load = [&](int c) {
            const int st = c % TC_NS;
            unsigned char *sp = smem + st * TC_STAGE;
            mbar_expect(&full[st], 2 * TC_AB + 2 * TC_BB);
            tma_bulk(sp, Ab + (size_t)c * 2 * TC_ACH, 2 * TC_AB, &full[st]);
            tma_bulk(sp + 2 * TC_AB, Wb + (size_t)c * nsb * 2 * TC_BCH, 2 * TC_BB, &full[st]);
        };
        // chunk c uses stage c % TC_NS and completes phase (c / TC_NS) & 1 of its
        // barriers; nl chunks loaded, nf of them waited for (full), nc committed,
        // ne of those waited for (empty)
        int nl = 0, nf = 0, nc = 0, ne = 0;
        const int lim = a.wait_limit;
        auto wait_full = [&](int c) { return mbar_wait(&full[c % TC_NS], (uint32_t)(c / TC_NS) & 1u, lim); };
        auto wait_empty = [&](int c) { return mbar_wait(&empty[c % TC_NS], (uint32_t)(c / TC_NS) & 1u, lim); };
        bool ok = true;
        if (!a.no_loads)
            for (int c = 0; c < TC_NS && c < nk; ++c) {
                load(c);
                ++nl;
            }
        for (int c = 0; c < nk && ok; ++c) {
            const int st = c % TC_NS;
            ok = wait_full(c);
            if (!ok) break;
            ++nf;
            tc_fence_after();
            const uint32_t sbs = sbase + st * TC_STAGE;
#pragma unroll
            for (int j = 0; j < TC_KC / 8; ++j) {
                const uint32_t o = j * 256;  // two core matrices per 8-wide slice of K
                const uint64_t ahi = tc_desc(sbs + o), alo = tc_desc(sbs + TC_AB + o);
                const uint64_t bhi = tc_desc(sbs + 2 * TC_AB + o), blo = tc_desc(sbs + 2 * TC_AB + TC_BB + o);
                tc_mma(tmem, ahi, bhi, (c > 0 || j > 0) ? 1u : 0u);
                tc_mma(tmem, ahi, blo, 1u);
                tc_mma(tmem, alo, bhi, 1u);
            }
            tc_commit(&empty[st]);
            ++nc;
            // refill the stage of chunk c-1 with chunk c-1+TC_NS once its MMAs are
            // done (those of chunk c are queued behind them meanwhile)
            if (c >= 1 && c - 1 + TC_NS < nk) {
                ok = wait_empty(c - 1);
                if (ok) {
                    ++ne;
                    load(c - 1 + TC_NS);
                    ++nl;
                }
            }
        }
        // the loop waited for chunks 0 .. nk-1-TC_NS; wait for the rest
        while (ok && ne < nc) {
            ok = wait_empty(ne);
            if (ok) ++ne;
        }
        if (!ok) {
            *flag = 0;
            if (a.status) atomicOr(a.status, ST_TIMEOUT);
            // drain what this thread issued before leaving: copies not yet waited
            // for, then committed MMAs, each wait bounded again; what is still
            // outstanding after that is abandoned (the kernel has already failed)
            for (int c = nf; c < nl; ++c) wait_full(c);
            for (int c = ne; c < nc; ++c) wait_empty(c);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*flag) {
        uint64_t kb = 0, dst = 0;
        int kind = -1;
        if (m0 + tid < rows) zrow(K, a.M, t, m0 + tid, a.off, kb, kind, dst);
        float *out = kind < 0    ? nullptr
                   : kind == 0 ? a.G
                   : kind == 1 ? a.Z + dst * a.S
                   : kind == 2 ? a.Z5 + dst * a.S
                               : a.X + dst * a.S;
        // The warp's 32 rows leave through shared memory (the ring is idle now):
        // a lane holds 32 columns of its own row after tcgen05.ld; the warp
        // writes them to a 32 x 36-float tile and reads them back as 8 lanes per
        // row, so every store instruction writes four whole 128-byte row pieces.
        const int lane = tid & 31, rsub = lane >> 3, c4 = (lane & 7) * 4;
        float *tile = reinterpret_cast<float *>(smem) + warp * 32 * 36;
        float *optr[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int src = 4 * i + rsub;  // row of the tile this lane stores in round i
            const unsigned long long p = __shfl_sync(0xffffffffu, (unsigned long long)out, src);
            optr[i] = reinterpret_cast<float *>(p);
        }
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cc = 0; cc < TC_N / 32; ++cc) {
            uint32_t v[32];
            tc_ld32(lane_base + (uint32_t)(cc * 32), v);
            float4 *row = reinterpret_cast<float4 *>(tile + lane * 36);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                row[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                     __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 w = *reinterpret_cast<const float4 *>(tile + (4 * i + rsub) * 36 + c4);
                if (optr[i]) *reinterpret_cast<float4 *>(optr[i] + s0 + cc * 32 + c4) = w;
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
}

// ---------------------------------------------------------------- step n: bias and draw

// K = 5: Y[i][s] = Z3_i(n) + sum_{3 <= j < i} chi_j Pp~[i-1][j+1] Z5_j(i, n), 3 <= i < n.
template <class R>
__global__ void __launch_bounds__(ETB) y_kernel(Args<R> a, int n) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    for (int i = 3 + blockIdx.y; i < n; i += gridDim.y) {
        Spins<R> sp(a, s);
        R y = a.Z[i_z(i, n) * a.S + s];
        for (int j = 3; j < i; ++j) y = fma(sp(j) * pp(a, i - 1, j + 1, s), a.Z5[i_z5(j, i, n) * a.S + s], y);
        a.Y[(size_t)i * a.S + s] = y;
    }
}

template <class R, int K>
__global__ void bias_kernel(Args<R> a, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    Spins<R> sp(a, s);
    const R Pm = a.P[(size_t)(n - 1) * a.S + s];
    R B = k1(a, n) * Pm;
    if (K == 3) {
        if (n >= 2) B += a.G[s];
        for (int i = 2; i < n; ++i) B = fma(sp(i) * pp(a, n - 1, i + 1, s), a.Z[i_z(i, n) * a.S + s], B);
    } else {
        for (int i = 1; i < n; ++i) B = fma(k2(a, i, n) * sp(i), p1(a, n - 1, i, s), B);
        if (n >= 3) B += a.G[s];
        // K = 5: Y = Z3 + the order-5 part (y_kernel); K = 4: Z3 alone
        const R *Yv = K == 5 ? a.Y : nullptr;
        for (int i = 3; i < n; ++i)
            B = fma(sp(i) * pp(a, n - 1, i + 1, s), K == 5 ? Yv[(size_t)i * a.S + s] : a.Z[i_z(i, n) * a.S + s], B);
    }
    const R hn = lead(a, n).y;
    const R p0 = fma(hn, Pm, B), p1v = fma(hn, Pm, -B);
    const R c0 = p0 > R(0) ? p0 : R(0), c1 = p1v > R(0) ? p1v : R(0);
    const R q = (c0 + c1 > R(0)) ? c0 / (c0 + c1) : R(0.5);
    int x = 0;
    const bool real = s < a.n_valid;
    if (real) {
        const size_t o = (size_t)s * a.M + (n - 1);
        if (a.force) x = a.force[o] ? 1 : 0;
        else x = (a.u[o] < (double)q) ? 0 : 1;
        a.bits[o] = (uint8_t)x;
        if (a.q0) a.q0[o] = (double)q;
    }
    a.chi[(size_t)n * a.S + s] = x ? R(-1) : R(1);
    if (x) a.bw[(size_t)(n >> 5) * a.S + s] |= 1u << (n & 31);
    a.P[(size_t)n * a.S + s] = x ? p1v : p0;
}

// ---------------------------------------------------------------- step n: table rows
// Thread per (entry, sample); the entry comes from blockIdx.y, so every index
// below is uniform across a warp. These grids serve the FP64 calls (a few
// hundred samples); FP32 runs the grouped forms further down (p2_kernel for
// both, ppv/pvv/yv/p1v for FP32).

// Order-3 part of the p+ update, factored: the term
//   sum_{i > j >= l} kappa(j,i,n) chi_i chi_j chi_n Pp~[n-1][i+1] Pp~[i-1][j+1] Pp~[j-1][l]
// equals chi_n sum_{j >= l} Pp~[j-1][l] v(j) with
//   v(j) = chi_j sum_{i > j} kappa(j,i,n) chi_i Pp~[n-1][i+1] Pp~[i-1][j+1],
// which does not depend on l. v goes to Y (free after the bias).
template <class R>
__global__ void __launch_bounds__(ETB) pv_kernel(Args<R> a, int n) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    for (int j = 1 + blockIdx.y; j < n; j += gridDim.y) {
        Spins<R> sp(a, s);
        R v = R(0);
        for (int i = j + 1; i < n; ++i)
            v = fma(k3(a, j, i, n) * sp(i) * pp(a, n - 1, i + 1, s), pp(a, i - 1, j + 1, s), v);
        a.Y[(size_t)j * a.S + s] = v * sp(j);
    }
}

// Pp~[n][l], l = 1..n (Eq. a / Eq. probpartialade).
template <class R>
__global__ void __launch_bounds__(ETB) pp_kernel(Args<R> a, int n) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    for (int l = 1 + blockIdx.y; l <= n; l += gridDim.y) {
        Spins<R> sp(a, s);
        const R cn = sp(n);
        R acc = R(0);
        if (a.opp >= 2)
            for (int i = l; i < n; ++i)
                acc = fma(k2(a, i, n) * sp(i) * pp(a, n - 1, i + 1, s), pp(a, i - 1, l, s), acc);
        if (a.opp >= 3)
            for (int j = l; j < n - 1; ++j) acc = fma(a.Y[(size_t)j * a.S + s], pp(a, j - 1, l, s), acc);
        const auto ld = lead(a, n);
        a.Pp[i_pp(n, l) * a.S + s] = fma(cn, acc, fma(ld.x, cn, ld.y) * pp(a, n - 1, l, s));
    }
}

// Per-step coefficients of the table updates, one per (i < n, sample):
//   CA = chi_i Pp~[n-1][i+1],  CB = kappa(i,n) chi_i,  CC = kappa(i,n) chi_i Pp~[n-1][i+1].
template <class R>
__global__ void __launch_bounds__(ETB) coef_kernel(Args<R> a, int n) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    for (int i = 1 + blockIdx.y; i < n; i += gridDim.y) {
        Spins<R> sp(a, s);
        const R ppv = pp(a, n - 1, i + 1, s), cbv = k2(a, i, n) * sp(i);
        const size_t o = (size_t)i * a.S + s;
        a.CA[o] = sp(i) * ppv;
        a.CB[o] = cbv;
        a.CC[o] = cbv * ppv;
    }
}

// P1~[n][e], e = 1..n-1 (Eq. b / Eq. probelidedade).
// K = 5, order 3: with (a, b, c) the decreasing order of (i, j, e), the terms with
// a = e come from the product rows (X_e(n), times Pp~[n-1][e+1]); the others
// (a = i > e) from the per-pair sums p2_kernel leaves in T.
template <class R, int K>
__global__ void __launch_bounds__(ETB) p1_kernel(Args<R> a, int n) {
    const int s = blockIdx.x * ETB + threadIdx.x;
    const size_t S = (size_t)a.S;
    for (int e = 1 + blockIdx.y; e < n; e += gridDim.y) {
        Spins<R> sp(a, s);
        const R cn = sp(n);
        R acc = R(0);
        if (a.op1 >= 2)
            for (int i = 1; i < n; ++i) {
                if (i == e) continue;
                const int hi = i > e ? i : e, lo = i > e ? e : i;
                const R g2 = k2(a, i, n) * sp(i);
                if (K == 3) acc = fma(g2 * pp(a, n - 1, hi + 1, s), p1(a, hi - 1, lo, s), acc);
                else acc = fma(g2, p2(a, n - 1, hi, lo, s), acc);
            }
        if (K >= 4 && a.op1 >= 3) {
            if (e >= 3) acc = fma(pp(a, n - 1, e + 1, s), a.X[i_z(e, n) * S + s], acc);
            // pairs (e, d), d < e, carry chi_d-weighted parts for e; pairs (j, e), j > e, for e
            const R *T = a.T + s;
            Spins<R> sd(a, s);
            for (int d = 1; d < e; ++d) acc = fma(sd(d), T[(2 * (cb(e - 1, 2) + (uint64_t)(d - 1))) * S], acc);
            for (int j = e + 1; j < n; ++j) acc = fma(sd(j), T[(2 * (cb(j - 1, 2) + (uint64_t)(e - 1)) + 1) * S], acc);
        }
        const auto ld = lead(a, n);
        a.P1[i_p1(n, e) * S + s] = fma(cn, acc, fma(ld.x, cn, ld.y) * p1(a, n - 1, e, s));
    }
}

// VW consecutive samples of one lane, loaded and stored as one vector.
template <class R, int VW>
struct Lanes {
    R v[VW];
};
template <class R, int VW>
__device__ __forceinline__ Lanes<R, VW> ldl(const R *p) {
    Lanes<R, VW> r;
    if constexpr (VW == 1) {
        r.v[0] = *p;
    } else if constexpr (VW == 2) {
        const auto q = *reinterpret_cast<const typename Pair2<R>::T *>(p);
        r.v[0] = q.x;
        r.v[1] = q.y;
    } else {
        static_assert(VW % 4 == 0 && sizeof(R) == 4, "four or more lanes: float only");
#pragma unroll
        for (int h = 0; h < VW / 4; ++h) {
            const float4 q = reinterpret_cast<const float4 *>(p)[h];
            r.v[4 * h] = q.x;
            r.v[4 * h + 1] = q.y;
            r.v[4 * h + 2] = q.z;
            r.v[4 * h + 3] = q.w;
        }
    }
    return r;
}
template <class R, int VW>
__device__ __forceinline__ void stl(R *p, const R (&x)[VW]) {
    if constexpr (VW == 1) {
        *p = x[0];
    } else if constexpr (VW == 2) {
        typename Pair2<R>::T q;
        q.x = x[0];
        q.y = x[1];
        *reinterpret_cast<typename Pair2<R>::T *>(p) = q;
    } else {
#pragma unroll
        for (int h = 0; h < VW / 4; ++h)
            reinterpret_cast<float4 *>(p)[h] = make_float4(x[4 * h], x[4 * h + 1], x[4 * h + 2], x[4 * h + 3]);
    }
}
// Sample-independent part of the address of P2~[x][e][d] (with its boundary
// cases P2~[x][x][d] = P1~[x-1][d], P1~[y][y] = P~[y-1]).
template <class R>
__device__ __forceinline__ const R *p2_row(const Args<R> &a, int x, int e, int d) {
    const size_t S = (size_t)a.S;
    if (e != x) return a.P2 + i_p2(x, e, d) * S;
    return d == x - 1 ? a.P + (size_t)(x - 2) * S : a.P1 + i_p1(x - 1, d) * S;
}

// P2~[n][e][d], n-1 >= e > d >= 1 (Eq. probdoubleelidedade).
// Order 2: i > e reaches P2~[i-1][e][d] (factor Pp~[n-1][i+1]); i < e reaches
// P2~[e-1][max(i,d)][min(i,d)] (common factor Pp~[n-1][e+1]). The loops walk the
// p2 rows by running offsets; the boundary entries (P2~[i-1][i-1][.] =
// P1~[i-2][.], P1~[i-2][i-2] = P~[i-3]) are taken apart.
// The same values P2~[i-1][e][d], i > e, are every term of the p1 order-3 sums
// whose largest index is i (Eq. probelidedade with (a, b, c) = (i, e, d)): they
// enter P1~[n][e] with weight CA[i] kappa(d,i,n) chi_d and P1~[n][d] with weight
// CA[i] kappa(e,i,n) chi_e. Both sums are formed here, without chi_d / chi_e, and
// left in T for p1_kernel, so each value is read once per step.
// Schedule: one warp (one block) per pair (e, d) and 32 VW consecutive samples,
// VW per lane (vector loads), the samples along the slow grid axis, so that the
// pairs of one sample group run together and the three reads of each p2 value
// (two in the row sums over i < e, one in the column sum over i > e) fall close
// in time and are mostly served by L2. The kernel is bound by load latency: the
// bounds cap it at 64 registers, so that 32 one-warp blocks (the per-SM block
// limit) stay resident.
template <class R, int VW>
__global__ void __launch_bounds__(32, 32) p2_kernel(Args<R> a, int n) {
    const int s = (int)blockIdx.y * (32 * VW) + (int)threadIdx.x * VW;
    const size_t S = (size_t)a.S;
    const uint64_t nr = cb(n - 1, 2);
    const R *P1 = a.P1 + s, *P2 = a.P2 + s, *P = a.P + s;
    const R *CA = a.CA + s, *CB = a.CB + s, *CC = a.CC + s;
    R cn[VW];
    {
        const uint32_t *bw = a.bw + (size_t)(n >> 5) * S + s;
#pragma unroll
        for (int k = 0; k < VW; ++k) cn[k] = (bw[k] >> (n & 31)) & 1u ? R(-1) : R(1);
    }
    const auto ld = lead(a, n);
    for (uint64_t r = blockIdx.x; r < nr; r += gridDim.x) {
        int hi, lo;
        pair_of(r, hi, lo);
        const int e = hi + 1, d = lo + 1;
        R acc[VW], tE[VW], tD[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = tE[k] = tD[k] = R(0);
        if (a.op2 >= 2) {
            R t[VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) t[k] = R(0);
            // i < d: P2~[e-1][d][i]
            if (d < e - 1) {
                const R *q = P2 + i_p2(e - 1, d, 1) * S;
#pragma unroll 4
                for (int i = 1; i < d; ++i, q += S) {
                    const auto c = ldl<R, VW>(CB + i * S), v = ldl<R, VW>(q);
#pragma unroll
                    for (int k = 0; k < VW; ++k) t[k] = fma(c.v[k], v.v[k], t[k]);
                }
            } else {
                const R *q = P1 + (e >= 3 ? i_p1(e - 2, 1) : 0) * S;
                for (int i = 1; i < d; ++i, q += S) {
                    const auto c = ldl<R, VW>(CB + i * S), v = ldl<R, VW>(i == e - 2 ? P + (size_t)(e - 3) * S : q);
#pragma unroll
                    for (int k = 0; k < VW; ++k) t[k] = fma(c.v[k], v.v[k], t[k]);
                }
            }
            // d < i < e: P2~[e-1][i][d]
            if (d + 1 <= e - 2) {
                uint64_t idx = i_p2(e - 1, d + 1, d);
#pragma unroll 4
                for (int i = d + 1; i < e - 1; ++i) {
                    const auto c = ldl<R, VW>(CB + i * S), v = ldl<R, VW>(P2 + idx * S);
#pragma unroll
                    for (int k = 0; k < VW; ++k) t[k] = fma(c.v[k], v.v[k], t[k]);
                    idx += (uint64_t)(i - 1);
                }
            }
            if (d < e - 1) {
                const auto c = ldl<R, VW>(CB + (e - 1) * S);
                const auto v = ldl<R, VW>(d == e - 2 ? P + (size_t)(e - 3) * S : P1 + i_p1(e - 2, d) * S);
#pragma unroll
                for (int k = 0; k < VW; ++k) t[k] = fma(c.v[k], v.v[k], t[k]);
            }
            if (e + 1 > n - 1) {
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] = t[k];
            } else {
                const auto w = ldl<R, VW>(a.Pp + i_pp(n - 1, e + 1) * S + s);
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] = w.v[k] * t[k];
            }
        }
        if ((a.op2 >= 2 || a.op1 >= 3) && e + 1 < n) {
            const R *k3n = a.kap + a.off[3] + cb(n - 1, 3) - 1;  // k3n[C(i-1,2) + j] = kappa(j, i, n)
            R a2[VW];
            // i = e + 1: P1~[e-1][d], or P~[e-2] when d = e - 1
            {
                const auto v = ldl<R, VW>(d == e - 1 ? P + (size_t)(e - 2) * S : P1 + i_p1(e - 1, d) * S);
                const R *kp = k3n + cb(e, 2);
                const R kd = kp[d], ke = kp[e];
                const auto ca = ldl<R, VW>(CA + (e + 1) * S), cc = ldl<R, VW>(CC + (e + 1) * S);
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    a2[k] = cc.v[k] * v.v[k];
                    tE[k] = ca.v[k] * kd * v.v[k];
                    tD[k] = ca.v[k] * ke * v.v[k];
                }
            }
            uint64_t idx = i_p2(e + 1, e, d);
#pragma unroll 4
            for (int i = e + 2; i < n; ++i) {
                const auto v = ldl<R, VW>(P2 + idx * S);
                const R *kp = k3n + cb(i - 1, 2);
                const R kd = kp[d], ke = kp[e];
                const auto ca = ldl<R, VW>(CA + i * S), cc = ldl<R, VW>(CC + i * S);
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    a2[k] = fma(cc.v[k], v.v[k], a2[k]);
                    tE[k] = fma(ca.v[k] * kd, v.v[k], tE[k]);
                    tD[k] = fma(ca.v[k] * ke, v.v[k], tD[k]);
                }
                idx += cb(i - 2, 2);
            }
            if (a.op2 >= 2) {
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] += a2[k];
            }
        }
        if (a.op1 >= 3) {
            const uint64_t o = 2 * r;
            stl<R, VW>(a.T + o * S + s, tE);
            stl<R, VW>(a.T + (o + 1) * S + s, tD);
        }
        const auto pv = ldl<R, VW>(p2_row(a, n - 1, e, d) + s);
        R out[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) out[k] = fma(cn[k], acc[k], fma(ld.x, cn[k], ld.y) * pv.v[k]);
        stl<R, VW>(a.P2 + i_p2(n, e, d) * S + s, out);
    }
}

// Spins of VW consecutive samples from their packed bits (vector loads); the
// current 32-bit words are cached as in Spins.
template <class R, int VW>
struct SpinsV {
    const uint32_t *bw;
    size_t S;
    int s, w;
    uint32_t cur[VW];
    __device__ SpinsV(const Args<R> &a, int s_) : bw(a.bw), S((size_t)a.S), s(s_), w(-1) {}
    __device__ __forceinline__ void operator()(int v, R (&x)[VW]) {
        if ((v >> 5) != w) {
            w = v >> 5;
            const uint32_t *p = bw + (size_t)w * S + s;
            if constexpr (VW == 4) {
                const uint4 q = *reinterpret_cast<const uint4 *>(p);
                cur[0] = q.x;
                cur[1] = q.y;
                cur[2] = q.z;
                cur[3] = q.w;
            } else if constexpr (VW == 2) {
                const uint2 q = *reinterpret_cast<const uint2 *>(p);
                cur[0] = q.x;
                cur[1] = q.y;
            } else {
                cur[0] = *p;
            }
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) x[k] = (cur[k] >> (v & 31)) & 1u ? R(-1) : R(1);
    }
};

// P1~[n][e] (Eq. probelidedade; K = 3: Eq. b), the same sums as p1_kernel, one
// warp per elided variable e and 32 VW consecutive samples (VW per lane), the
// sample groups on the slow grid axis as in p2_kernel: each p2 value of row
// n - 1 is read by the warps of e = hi and e = lo of the same group.
template <class R, int K, int VW>
__global__ void __launch_bounds__(32, 32) p1v_kernel(Args<R> a, int n) {
    const int s = (int)blockIdx.y * (32 * VW) + (int)threadIdx.x * VW;
    const size_t S = (size_t)a.S;
    R cn[VW];
    {
        SpinsV<R, VW> sn(a, s);
        sn(n, cn);
    }
    const auto ld = lead(a, n);
    for (int e = 1 + (int)blockIdx.x; e < n; e += (int)gridDim.x) {
        R acc[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = R(0);
        if (a.op1 >= 2) {
            SpinsV<R, VW> sp(a, s);
            for (int i = 1; i < n; ++i) {
                if (i == e) continue;
                const int hi = i > e ? i : e, lo = i > e ? e : i;
                R c[VW];
                sp(i, c);
                const R k2v = k2(a, i, n);
                if (K == 3) {
                    const auto q = ldl<R, VW>((lo == hi - 1 ? a.P + (size_t)(hi - 2) * S : a.P1 + i_p1(hi - 1, lo) * S) + s);
                    if (hi + 1 > n - 1) {
#pragma unroll
                        for (int k = 0; k < VW; ++k) acc[k] = fma(k2v * c[k] * R(1), q.v[k], acc[k]);
                    } else {
                        const auto w = ldl<R, VW>(a.Pp + i_pp(n - 1, hi + 1) * S + s);
#pragma unroll
                        for (int k = 0; k < VW; ++k) acc[k] = fma(k2v * c[k] * w.v[k], q.v[k], acc[k]);
                    }
                } else {
                    const auto q = ldl<R, VW>(p2_row(a, n - 1, hi, lo) + s);
#pragma unroll
                    for (int k = 0; k < VW; ++k) acc[k] = fma(k2v * c[k], q.v[k], acc[k]);
                }
            }
        }
        if (K >= 4 && a.op1 >= 3) {
            if (e >= 3) {
                const auto x = ldl<R, VW>(a.X + i_z(e, n) * S + s);
                if (e + 1 > n - 1) {
#pragma unroll
                    for (int k = 0; k < VW; ++k) acc[k] = fma(R(1), x.v[k], acc[k]);
                } else {
                    const auto w = ldl<R, VW>(a.Pp + i_pp(n - 1, e + 1) * S + s);
#pragma unroll
                    for (int k = 0; k < VW; ++k) acc[k] = fma(w.v[k], x.v[k], acc[k]);
                }
            }
            // pairs (e, d), d < e, carry chi_d-weighted parts for e; pairs (j, e), j > e, for e
            const R *T = a.T + s;
            SpinsV<R, VW> sd(a, s);
            for (int d = 1; d < e; ++d) {
                R c[VW];
                sd(d, c);
                const auto t = ldl<R, VW>(T + (2 * (cb(e - 1, 2) + (uint64_t)(d - 1))) * S);
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] = fma(c[k], t.v[k], acc[k]);
            }
            for (int j = e + 1; j < n; ++j) {
                R c[VW];
                sd(j, c);
                const auto t = ldl<R, VW>(T + (2 * (cb(j - 1, 2) + (uint64_t)(e - 1)) + 1) * S);
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] = fma(c[k], t.v[k], acc[k]);
            }
        }
        const auto pv = ldl<R, VW>((e == n - 1 ? a.P + (size_t)(n - 2) * S : a.P1 + i_p1(n - 1, e) * S) + s);
        R out[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) out[k] = fma(cn[k], acc[k], fma(ld.x, cn[k], ld.y) * pv.v[k]);
        stl<R, VW>(a.P1 + i_p1(n, e) * S + s, out);
    }
}

// Pp~[x][b] of VW consecutive samples (1 when the range is empty, b > x).
template <class R, int VW>
__device__ __forceinline__ Lanes<R, VW> ppl(const Args<R> &a, int x, int b, int s) {
    if (b > x) {
        Lanes<R, VW> r;
#pragma unroll
        for (int k = 0; k < VW; ++k) r.v[k] = R(1);
        return r;
    }
    return ldl<R, VW>(a.Pp + i_pp(x, b) * (size_t)a.S + s);
}

// FP32 forms of y_kernel, pv_kernel and pp_kernel with the schedule of p2_kernel:
// one warp per entry and 32 VW consecutive samples (VW per lane), the sample
// groups on the slow grid axis; the same terms in the same order per sample.
template <class R, int VW>
__global__ void __launch_bounds__(32, 32) yv_kernel(Args<R> a, int n) {
    const int s = (int)blockIdx.y * (32 * VW) + (int)threadIdx.x * VW;
    const size_t S = (size_t)a.S;
    for (int i = 3 + (int)blockIdx.x; i < n; i += (int)gridDim.x) {
        SpinsV<R, VW> sp(a, s);
        const auto z = ldl<R, VW>(a.Z + i_z(i, n) * S + s);
        R y[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) y[k] = z.v[k];
        for (int j = 3; j < i; ++j) {
            R c[VW];
            sp(j, c);
            const auto w = ppl<R, VW>(a, i - 1, j + 1, s);
            const auto z5 = ldl<R, VW>(a.Z5 + i_z5(j, i, n) * S + s);
#pragma unroll
            for (int k = 0; k < VW; ++k) y[k] = fma(c[k] * w.v[k], z5.v[k], y[k]);
        }
        stl<R, VW>(a.Y + (size_t)i * S + s, y);
    }
}

template <class R, int VW>
__global__ void __launch_bounds__(32, 32) pvv_kernel(Args<R> a, int n) {
    const int s = (int)blockIdx.y * (32 * VW) + (int)threadIdx.x * VW;
    const size_t S = (size_t)a.S;
    for (int j = 1 + (int)blockIdx.x; j < n; j += (int)gridDim.x) {
        SpinsV<R, VW> sp(a, s);
        R v[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] = R(0);
        for (int i = j + 1; i < n; ++i) {
            R c[VW];
            sp(i, c);
            const R k3v = k3(a, j, i, n);
            const auto w = ppl<R, VW>(a, n - 1, i + 1, s), q = ppl<R, VW>(a, i - 1, j + 1, s);
#pragma unroll
            for (int k = 0; k < VW; ++k) v[k] = fma(k3v * c[k] * w.v[k], q.v[k], v[k]);
        }
        R cj[VW];
        sp(j, cj);
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] = v[k] * cj[k];
        stl<R, VW>(a.Y + (size_t)j * S + s, v);
    }
}

template <class R, int VW>
__global__ void __launch_bounds__(32, 32) ppv_kernel(Args<R> a, int n) {
    const int s = (int)blockIdx.y * (32 * VW) + (int)threadIdx.x * VW;
    const size_t S = (size_t)a.S;
    R cn[VW];
    {
        SpinsV<R, VW> sn(a, s);
        sn(n, cn);
    }
    const auto ld = lead(a, n);
    for (int l = 1 + (int)blockIdx.x; l <= n; l += (int)gridDim.x) {
        R acc[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = R(0);
        if (a.opp >= 2) {
            SpinsV<R, VW> sp(a, s);
            for (int i = l; i < n; ++i) {
                R c[VW];
                sp(i, c);
                const R k2v = k2(a, i, n);
                const auto w = ppl<R, VW>(a, n - 1, i + 1, s), q = ppl<R, VW>(a, i - 1, l, s);
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] = fma(k2v * c[k] * w.v[k], q.v[k], acc[k]);
            }
        }
        if (a.opp >= 3)
            for (int j = l; j < n - 1; ++j) {
                const auto y = ldl<R, VW>(a.Y + (size_t)j * S + s), q = ppl<R, VW>(a, j - 1, l, s);
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] = fma(y.v[k], q.v[k], acc[k]);
            }
        const auto w = ppl<R, VW>(a, n - 1, l, s);
        R out[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) out[k] = fma(cn[k], acc[k], fma(ld.x, cn[k], ld.y) * w.v[k]);
        stl<R, VW>(a.Pp + i_pp(n, l) * S + s, out);
    }
}

template <class R>
__global__ void init_kernel(Args<R> a) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < a.S) {
        a.P[s] = R(1);
        a.chi[s] = R(1);
        for (int w = 0; w <= a.M / 32; ++w) a.bw[(size_t)w * a.S + s] = 0u;
    }
}

// ln of the estimated probability: ln P~[M] - sum_v ln s_v (NaN if P~[M] <= 0).
template <class R>
__global__ void logp_kernel(Args<R> a, double *logp) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_valid) return;
    double h = 0.0;
    for (int v = 1; v <= a.M; ++v) h += a.H[v];
    const double P = (double)a.P[(size_t)a.M * a.S + s];
    logp[s] = P > 0.0 ? log(P) - h : __longlong_as_double(0x7ff8000000000000ULL);
}

// Per-variable scales from the order-1 cumulants: kappa({v}) = c_v = <(-1)^{x_v}>,
// so mode v - 1 is silent with probability (1 + c_v) / 2; s_v = exp(H_v) with H_v
// that binary entropy in nats (s_v in [1, 2]).
template <class R>
__global__ void scale_kernel(const double *__restrict__ kap, int M, R *hs, R *lead, double *H) {
    const int v = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (v > M) return;
    double p0 = 0.5 * (1.0 + kap[v - 1]);
    p0 = p0 < 0.0 ? 0.0 : (p0 > 1.0 ? 1.0 : p0);
    const double p1 = 1.0 - p0;
    const double h = (p0 > 0.0 ? -p0 * log(p0) : 0.0) + (p1 > 0.0 ? -p1 * log(p1) : 0.0);
    const double half = 0.5 * exp(h);
    H[v] = h;
    hs[v] = (R)half;
    lead[2 * v] = (R)(kap[v - 1] * half);
    lead[2 * v + 1] = (R)half;
}

// kappa'(S) = kappa(S) prod_{v in S} s_v / 2 for every table entry, in the
// arithmetic precision R. A thread takes KS_CHUNK consecutive entries of one
// order: it unranks the first and steps through the rest by colex successor.
constexpr int KS_CHUNK = 64;

template <class R>
__global__ void kscale_kernel(const double *__restrict__ kap, int M, int d, uint64_t off, uint64_t n,
                              const R *__restrict__ hs, R *__restrict__ out) {
    const uint64_t r0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * KS_CHUNK;
    if (r0 >= n) return;
    const uint64_t r1 = r0 + KS_CHUNK < n ? r0 + KS_CHUNK : n;
    int c[6];
    colex_unrank(r0, d, c);
    c[d] = M;  // sentinel
    // product of the scales of c[1..d-1], formed again only when one of them moves
    // (GB300's FP64 pipe is narrow: most successors move c[0] alone)
    auto upper = [&]() {
        double f = 1.0;
        for (int i = d - 1; i >= 1; --i) f *= (double)hs[c[i] + 1];
        return f;
    };
    double fu = upper();
    for (uint64_t r = r0; r < r1; ++r) {
        out[off + r] = (R)(kap[off + r] * (fu * (double)hs[c[0] + 1]));
        // successor: the first element that can move up moves up, the ones below reset
        int i = 0;
        while (i < d - 1 && c[i] + 1 == c[i + 1]) ++i;
        ++c[i];
        for (int j = 0; j < i; ++j) c[j] = j;
        if (i > 0 && r + 1 < r1) fu = upper();
    }
}

// ---------------------------------------------------------------- host side

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

SamplerLayout sampler_layout(int M, int K, int S, int precision) {
    SamplerLayout L{};
    const size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    const size_t Ss = (size_t)S;
    size_t off = 256;  // status word first (read by gbs_stream_status)
    auto take = [&](size_t &field, size_t entries) {
        field = off;
        off = a256(off + entries * Ss * es);
    };
    take(L.chi, (size_t)M + 1);
    take(L.P, (size_t)M + 1);
    take(L.Pp, cb(M, 2) + (size_t)M);
    take(L.P1, cb(M, 2));
    take(L.P2, K >= 4 ? cb(M, 3) : 0);
    take(L.Z, cb(M, 2));
    take(L.Z5, K == 5 ? cb(M, 3) : 0);
    take(L.G, 1);
    take(L.Y, K >= 4 ? (size_t)M + 1 : 0);
    take(L.X, K >= 4 ? cb(M, 2) : 0);
    // W: plain [r][S], or for the tensor-core product hi / lo copies of 32-padded chunks
    take(L.W, 2 * ((K >= 4 ? cb(M - 1, 2) : (size_t)M) + 32));
    // tensor-core product rows: max over the steps of (row tiles x chunks) x 8192 floats
    size_t at = 0;
    if (precision != 0)
        for (int t = 1; t <= M; ++t) {
            const uint64_t D = K == 3 ? (uint64_t)(t - 1) : cb(t - 1, 2);
            const uint64_t rows = K == 3   ? 1 + (uint64_t)(M - t)
                                  : K == 4 ? 1 + 2 * (uint64_t)(M - t)
                                           : 1 + 2 * (uint64_t)(M - t) + cb(M - t, 2);
            const size_t n = (size_t)((rows + TC_M - 1) / TC_M) * ((D + TC_KC - 1) / TC_KC) * 2 * TC_ACH;
            if (n > at) at = n;
        }
    L.At = off;
    off = a256(off + at * sizeof(float));
    take(L.CA, K >= 4 ? 3 * ((size_t)M + 1) : 0);
    take(L.T, K >= 4 ? 2 * cb(M - 1, 2) : 0);
    L.bw = off;
    off = a256(off + (size_t)(M / 32 + 1) * Ss * sizeof(uint32_t));
    L.kap = off;  // the rescaled cumulants kappa', in the arithmetic precision
    uint64_t nk = 0;
    for (int d = 1; d <= K; ++d) nk += cb(M, d);
    off = a256(off + nk * es);
    L.hs = off;
    off = a256(off + ((size_t)M + 1) * es);
    L.H = off;
    off = a256(off + ((size_t)M + 1) * sizeof(double));
    L.lead = off;
    off = a256(off + 2 * ((size_t)M + 1) * es);
    L.total = off;
    return L;
}

// Grid of a per-(entry, sample) kernel: samples along x, entries along y, about
// 10^4 blocks in all (each block loops over its share of the entries).
static dim3 egrid(int S, uint64_t entries) {
    const uint64_t bx = (uint64_t)(S / ETB);
    uint64_t cap = 10000 / bx;
    if (cap < 16) cap = 16;
    uint64_t by = entries < cap ? entries : cap;
    if (by < 1) by = 1;
    return dim3((unsigned)bx, (unsigned)by);
}

template <class R, int K>
static cudaError_t run_chunk(Args<R> a, double *prob, cudaStream_t st) {
    const int S = a.S, M = a.M;
    const int TB = 256;
    constexpr int TM = sizeof(R) == 4 ? 8 : 4, TN = TM;
    init_kernel<R><<<(S + TB - 1) / TB, TB, 0, st>>>(a);
    for (int t = 1; t <= M; ++t) {
        // products for this step and later ones (inputs: rows < t of the tables)
        const int D = K == 3 ? t - 1 : (int)cb(t - 1, 2);  // K = 4, 5: pairs below t
        if (D > 0) {
            bool tc = false;
            if constexpr (sizeof(R) == 4) tc = a.use_tc != 0;
            if constexpr (sizeof(R) == 4) {
                if (tc) wtc_kernel<K><<<egrid(S, (uint64_t)((D + TC_KC - 1) / TC_KC * TC_KC / 4)), ETB, 0, st>>>(a, t, D);
            }
            if (!tc) w_kernel<R, K><<<egrid(S, (uint64_t)D), ETB, 0, st>>>(a, t, D);
            const uint64_t rows = K == 3   ? 1 + (uint64_t)(M - t)
                                  : K == 4 ? 1 + 2 * (uint64_t)(M - t)
                                           : 1 + 2 * (uint64_t)(M - t) + cb(M - t, 2);
            if constexpr (sizeof(R) == 4) {
                if (tc) {
                    const unsigned nrt = (unsigned)((rows + TC_M - 1) / TC_M), nk = (unsigned)((D + TC_KC - 1) / TC_KC);
                    atc_kernel<K><<<dim3(nrt, nk), 128, 0, st>>>(a, t, rows, D);
                    ztc_kernel<K><<<dim3(nrt, (unsigned)(S / TC_N)), 128, TC_SMEM, st>>>(a, t, rows, D);
                } else {
                    dim3 grid((unsigned)((rows + 16 * TM - 1) / (16 * TM)), (unsigned)(S / (16 * TN)));
                    zgemm_kernel<R, K, TM, TN><<<grid, 256, 0, st>>>(a, t, rows, D);
                }
            } else {
                dim3 grid((unsigned)((rows + 16 * TM - 1) / (16 * TM)), (unsigned)(S / (16 * TN)));
                zgemm_kernel<R, K, TM, TN><<<grid, 256, 0, st>>>(a, t, rows, D);
            }
        }
        // FP32 (large batches): warp-per-entry kernels over 128-sample groups; FP64
        // calls, a few hundred samples, keep the (samples, entries) grids
        constexpr bool grouped = sizeof(R) == 4;
        const unsigned gy = (unsigned)(S / 128);
        if (K == 5 && t > 3) {
            if constexpr (grouped) yv_kernel<R, 4><<<dim3((unsigned)(t - 3), gy), 32, 0, st>>>(a, t);
            else y_kernel<R><<<egrid(S, (uint64_t)(t - 3)), ETB, 0, st>>>(a, t);
        }
        bias_kernel<R, K><<<(S + TB - 1) / TB, TB, 0, st>>>(a, t);
        if (K >= 4 && a.opp >= 3 && t > 1) {
            if constexpr (grouped) pvv_kernel<R, 4><<<dim3((unsigned)(t - 1), gy), 32, 0, st>>>(a, t);
            else pv_kernel<R><<<egrid(S, (uint64_t)(t - 1)), ETB, 0, st>>>(a, t);
        }
        if constexpr (grouped) ppv_kernel<R, 4><<<dim3((unsigned)t, gy), 32, 0, st>>>(a, t);
        else pp_kernel<R><<<egrid(S, (uint64_t)t), ETB, 0, st>>>(a, t);
        if (K >= 4 && t > 1) coef_kernel<R><<<egrid(S, (uint64_t)(t - 1)), ETB, 0, st>>>(a, t);
        if (K >= 4 && t > 2) {  // before p1: fills T
            constexpr int VW = sizeof(R) == 4 ? 4 : 2;  // samples per lane (batch: a multiple of 128)
            const uint64_t nr = cb(t - 1, 2);
            p2_kernel<R, VW><<<dim3((unsigned)(nr < (1u << 30) ? nr : (1u << 30)), (unsigned)(S / (32 * VW))), 32, 0, st>>>(a, t);
        }
        if (t > 1) {
            if constexpr (grouped) p1v_kernel<R, K, 4><<<dim3((unsigned)(t - 1), gy), 32, 0, st>>>(a, t);
            else p1_kernel<R, K><<<egrid(S, (uint64_t)(t - 1)), ETB, 0, st>>>(a, t);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (prob) logp_kernel<R><<<(S + TB - 1) / TB, TB, 0, st>>>(a, prob);
    return cudaGetLastError();
}

template <class R>
static cudaError_t run_all(const SamplerCall &c, cudaStream_t st) {
    const SamplerLayout L = sampler_layout(c.M, c.K, c.S, c.precision);
    char *w = static_cast<char *>(c.ws);
    Args<R> a{};
    a.M = c.M;
    a.K = c.K;
    a.S = c.S;
    a.opp = c.K == 3 ? 2 : c.orders[0];
    a.op1 = c.K == 3 ? 2 : c.orders[1];
    a.op2 = c.orders[2];  // the caller resolves the defaults per K
    a.off[0] = 0;
    for (int d = 1; d <= 5; ++d) a.off[d] = order_offset(c.M, d);
    a.chi = reinterpret_cast<R *>(w + L.chi);
    a.P = reinterpret_cast<R *>(w + L.P);
    a.Pp = reinterpret_cast<R *>(w + L.Pp);
    a.P1 = reinterpret_cast<R *>(w + L.P1);
    a.P2 = reinterpret_cast<R *>(w + L.P2);
    a.Z = reinterpret_cast<R *>(w + L.Z);
    a.Z5 = reinterpret_cast<R *>(w + L.Z5);
    a.G = reinterpret_cast<R *>(w + L.G);
    a.Y = reinterpret_cast<R *>(w + L.Y);
    a.X = reinterpret_cast<R *>(w + L.X);
    a.W = reinterpret_cast<R *>(w + L.W);
    a.CA = reinterpret_cast<R *>(w + L.CA);
    a.CB = a.CA + ((size_t)c.M + 1) * c.S;
    a.CC = a.CB + ((size_t)c.M + 1) * c.S;
    a.T = reinterpret_cast<R *>(w + L.T);
    a.At = reinterpret_cast<float *>(w + L.At);
    a.bw = reinterpret_cast<uint32_t *>(w + L.bw);
    a.status = reinterpret_cast<unsigned *>(w);
    {
        cudaError_t e = cudaMemsetAsync(w, 0, 256, st);
        if (e != cudaSuccess) return e;
    }
    a.use_tc = 0;
    a.wait_limit = 1 << 22;
    a.no_loads = 0;
    if (fault_injected("sampler_no_loads")) {
        a.no_loads = 1;
        a.wait_limit = 1 << 10;
    }
    if (sizeof(R) == 4) {
        const char *env = getenv("GBS_SAMPLER_SIMT");
        a.use_tc = (env && *env && *env != '0') || c.S % TC_N != 0 ? 0 : 1;
        if (a.use_tc) {
            cudaError_t e = cudaSuccess;
            if (c.K == 3) e = cudaFuncSetAttribute(ztc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
            if (c.K == 4) e = cudaFuncSetAttribute(ztc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
            if (c.K == 5) e = cudaFuncSetAttribute(ztc_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
            if (e != cudaSuccess) return e;
        }
    }
    {
        R *hs = reinterpret_cast<R *>(w + L.hs);
        double *H = reinterpret_cast<double *>(w + L.H);
        R *ldp = reinterpret_cast<R *>(w + L.lead);
        R *kf = reinterpret_cast<R *>(w + L.kap);
        scale_kernel<R><<<(c.M + 255) / 256, 256, 0, st>>>(c.kappa, c.M, hs, ldp, H);
        uint64_t off = 0;
        for (int d = 1; d <= c.K; ++d) {
            const uint64_t n = cb(c.M, d), threads = (n + KS_CHUNK - 1) / KS_CHUNK;
            kscale_kernel<R><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(c.kappa, c.M, d, off, n, hs, kf);
            off += n;
        }
        a.kap = kf;
        a.hs = hs;
        a.lead = ldp;
        a.H = H;
    }
    for (int s0 = 0; s0 < c.n_samples; s0 += c.S) {
        a.n_valid = c.n_samples - s0 < c.S ? c.n_samples - s0 : c.S;
        const size_t o = (size_t)s0 * c.M;
        a.u = c.u ? c.u + o : nullptr;
        a.force = c.force ? c.force + o : nullptr;
        a.bits = c.bits + o;
        a.q0 = c.q0 ? c.q0 + o : nullptr;
        double *pr = c.prob ? c.prob + s0 : nullptr;
        cudaError_t e = c.K == 3 ? run_chunk<R, 3>(a, pr, st) : c.K == 4 ? run_chunk<R, 4>(a, pr, st) : run_chunk<R, 5>(a, pr, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sampler(const SamplerCall &c, cudaStream_t st) {
    return c.precision == 0 ? run_all<double>(c, st) : run_all<float>(c, st);
}

}  // namespace smp
}  // namespace gbs

// ---------------------------------------------------------------- C ABI

namespace gbs {
int record_error(int code, const char *msg);
}

namespace {

bool dev_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool valid_shape(int M, int K, int batch, int precision) {
    return K >= 3 && K <= 5 && M >= K && M <= (K == 3 ? GBS_MAX_MODES_K3 : GBS_MAX_MODES) && batch >= 128 &&
           batch <= GBS_MAX_SAMPLE_BATCH && batch % 128 == 0 &&
           (precision == GBS_SAMPLE_FP64 || precision == GBS_SAMPLE_FP32);
}

}  // namespace

extern "C" {

size_t gbs_sampler_workspace_bytes(int M, int K, int batch, int precision) {
    if (!valid_shape(M, K, batch, precision)) return 0;
    return gbs::smp::sampler_layout(M, K, batch, precision).total;
}

int gbs_sample(const double *kappa, int M, int K, const int *orders, int n_samples, const double *u,
               const uint8_t *force, uint8_t *bits_out, double *logp_out, double *q0_out, int batch, int precision,
               void *workspace, size_t ws_bytes, void *cuda_stream) {
    using gbs::record_error;
    if (!valid_shape(M, K, batch, precision))
        return record_error(GBS_ERR_INVALID_ARG,
                            "need K in {3, 4, 5}, K <= M <= 1024 (4096 for K = 3), batch a multiple of 128 in "
                            "[128, GBS_MAX_SAMPLE_BATCH] and precision GBS_SAMPLE_FP64 or GBS_SAMPLE_FP32");
    if (n_samples < 0) return record_error(GBS_ERR_INVALID_ARG, "n_samples must be >= 0");
    int ord[3] = {3, 3, 2};  // K = 5; K = 4: one order lower, as the paper's rule gives
    if (K == 4) ord[0] = ord[1] = 2, ord[2] = 1;
    if (orders) {
        for (int i = 0; i < 3; ++i) ord[i] = orders[i];
        if (ord[0] < 1 || ord[0] > 3 || ord[1] < 1 || ord[1] > 3 || ord[2] < 1 || ord[2] > 2)
            return record_error(GBS_ERR_INVALID_ARG, "orders must be {1..3, 1..3, 1..2}");
    }
    if (!kappa || !bits_out || !workspace || (!u && !force))
        return record_error(GBS_ERR_INVALID_ARG, "kappa, bits_out, workspace and one of u / force must be non-NULL");
    if (((uintptr_t)kappa & 7) || (u && ((uintptr_t)u & 7)) || (logp_out && ((uintptr_t)logp_out & 7)) ||
        (q0_out && ((uintptr_t)q0_out & 7)) || ((uintptr_t)workspace & 255))
        return record_error(GBS_ERR_INVALID_ARG, "double arrays must be 8-byte aligned, the workspace 256-byte aligned");
    if (!dev_ptr(kappa) || !dev_ptr(bits_out) || !dev_ptr(workspace) || (u && !dev_ptr(u)) ||
        (force && !dev_ptr(force)) || (logp_out && !dev_ptr(logp_out)) || (q0_out && !dev_ptr(q0_out)))
        return record_error(GBS_ERR_INVALID_ARG, "all arrays must be CUDA device (or managed) memory");
    const gbs::smp::SamplerLayout L = gbs::smp::sampler_layout(M, K, batch, precision);
    if (ws_bytes < L.total) return record_error(GBS_ERR_WORKSPACE, "workspace smaller than gbs_sampler_workspace_bytes()");
    if (n_samples == 0) return record_error(GBS_OK, "");
    gbs::smp::SamplerCall c{};
    c.kappa = kappa;
    c.M = M;
    c.K = K;
    c.S = batch;
    c.precision = precision;
    c.n_samples = n_samples;
    for (int i = 0; i < 3; ++i) c.orders[i] = ord[i];
    c.u = u;
    c.force = force;
    c.bits = bits_out;
    c.prob = logp_out;
    c.q0 = q0_out;
    c.ws = workspace;
    cudaError_t e = gbs::smp::launch_sampler(c, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return record_error(GBS_ERR_CUDA, cudaGetErrorString(e));
    return record_error(GBS_OK, "");
}

}  // extern "C"
