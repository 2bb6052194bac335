// Device code shared by the single-instance forward kernels (gbs_fwd.cu) and the
// batched kernel (gbs_batch.cu): the combine step, the per-order entry
// functions and one work item of the prefix-tree elimination. See gbs_fwd.cu
// for the formulas.
#pragma once
#include <cooperative_groups.h>

#include "gbs.h"
#include "gbs_common.cuh"
#include "gbs_fwd.cuh"
#include "gbs_refined.cuh"

namespace gbs {

constexpr int FLAT_THREADS = 256;
constexpr int TREE_THREADS = 512;
constexpr int XCAP = 1152;  // per-batch x-entries in shared memory (>= GBS_MAX_MODES)
constexpr int CCAP = kMaxChildren;  // per-batch children

// ---------------------------------------------------------------- shared combine step

// Per-child constants of the gathers. P = {c_3, .., c_D} ascending, NP = D-2
// elements, subsets of P by bitmask over P's positions.
//   baseJ[Q]: table index of {x} + Q is baseJ[Q] + x   (x < min P)
//   baseT[Q]: table index of {j, c2} + Q is baseT[Q] + t, t = C(c2,2) + j
//   idxQ[Q] : table index of Q (Q nonempty)
template <int NP>
__device__ __forceinline__ void child_bases(const int *P, int M, uint64_t *baseJ, uint64_t *baseT, uint64_t *idxQ) {
    uint64_t off[GBS_MAX_ORDER + 2];
    off[0] = 0;
    off[1] = 0;
    for (int m = 2; m <= NP + 2; ++m) off[m] = off[m - 1] + binom(M, m - 1);
#pragma unroll
    for (int q = 0; q < (1 << NP); ++q) {
        int m = __popc(q);
        uint64_t sJ = off[m + 1], sT = off[m + 2], sQ = off[m];
        int i = 0;
#pragma unroll
        for (int e = 0; e < NP; ++e)
            if (q >> e & 1) {
                ++i;
                sJ += binom(P[e], i + 1);
                sT += binom(P[e], i + 2);
                sQ += binom(P[e], i);
            }
        baseJ[q] = sJ;
        baseT[q] = sT;
        idxQ[q] = sQ;
    }
}

template <int NP, int MODE>
__host__ __device__ constexpr double lead_sign();
template <int NP, int MODE>
__device__ __forceinline__ double combine_tail(double acc, int j, int c2, uint32_t t, const uint64_t *baseJ,
                                               const uint64_t *baseT, const double *p0R,
                                               const double *__restrict__ p0tab, const double *__restrict__ outtab);

// Mode-specific value of the leaf S = {j, c2} + P (|P| = NP) given P0(S).
// p0R[R] = P0(R) for nonempty R subset of P.
template <int NP, int MODE>
__device__ __forceinline__ double combine(double P0S, int j, int c2, uint32_t t, const uint64_t *baseJ,
                                          const uint64_t *baseT, const double *p0R, const double *__restrict__ p0tab,
                                          const double *__restrict__ outtab) {
    constexpr int PALL = (1 << NP) - 1;
    if (MODE == MODE_P0) return P0S;
    if (MODE == MODE_MU) {
        double acc = outtab[baseJ[PALL] + c2];  // mu(S')
#pragma unroll
        for (int q = 0; q <= PALL; ++q) {
            const double sg = (__popc(q) & 1) ? -1.0 : 1.0;
            acc = fma(-sg, p0tab[baseJ[q] + j], acc);
            const double t2 = (q == PALL) ? P0S : p0tab[baseT[q] + t];
            acc = fma(sg, t2, acc);
        }
        return acc;
    }
    if (MODE == MODE_SPINC) {
        // c(S) = -c(S') - 2 (-1)^d sum_{R' subset S'} (-2)^{|R'|} P0({j} + R'), d = |S|
        // (the sum of Eq. correlator_sum_cov split by whether R contains j)
        constexpr double lead = ((NP + 2) & 1) ? 2.0 : -2.0;  // -2 (-1)^d
        double acc = -outtab[baseJ[PALL] + c2];                // -c(S')
#pragma unroll
        for (int q = 0; q <= PALL; ++q) {
            const double w = lead * ((__popc(q) & 1) ? -1.0 : 1.0) * (double)(1 << __popc(q));  // (-2)^{|q|}
            acc = fma(w, p0tab[baseJ[q] + j], acc);
            const double t2 = (q == PALL) ? P0S : p0tab[baseT[q] + t];
            acc = fma(-2.0 * w, t2, acc);                      // R' = Q + {c2}
        }
        return acc;
    }
    // MODE_KAPPA: kt(S) = (-1)^d [bracket];  MODE_SPINK: kappa(S) = (-2)^d kt(S) = 2^d [bracket],
    // with the lower-order table holding kappa = (-2)^{|Q|} kt (exact power-of-two scalings).
    // The bracket is accumulated already multiplied by lead_sign (the sign of the
    // order for MODE_KAPPA), which every FMA absorbs as an operand negation.
    constexpr double sd = lead_sign<NP, MODE>();
    return combine_tail<NP, MODE>(fma(-sd * p0tab[j], p0tab[baseJ[PALL] + c2], sd * P0S), j, c2, t, baseJ, baseT,
                                  p0R, p0tab, outtab);
}

// Sign carried by the accumulator of the cumulant recursion: (-1)^d for the
// click cumulant (d = NP + 2), + for the spin cumulant.
template <int NP, int MODE>
__host__ __device__ constexpr double lead_sign() {
    return (MODE == MODE_KAPPA && ((NP + 2) & 1)) ? -1.0 : 1.0;
}

// The cumulant recursion (MODE_KAPPA, MODE_SPINK) after its leading term
// acc = lead_sign (P0(S) - P0({j}) P0(S')): the 2^{d-1} - 2 products with
// lower-order cumulants (signs folded into each FMA), then, for the spin
// cumulant, the power of two.
template <int NP, int MODE>
__device__ __forceinline__ double combine_tail(double acc, int j, int c2, uint32_t t, const uint64_t *baseJ,
                                               const uint64_t *baseT, const double *p0R,
                                               const double *__restrict__ p0tab, const double *__restrict__ outtab) {
    constexpr int PALL = (1 << NP) - 1;
    constexpr double sd = lead_sign<NP, MODE>();
#pragma unroll
    for (int q = 1; q <= PALL; ++q) {
        const double sg = (MODE == MODE_KAPPA) ? ((__popc(q) & 1) ? -sd : sd)
                                               : -1.0 / (double)(2 << __popc(q));  // -2^{-(|R|+1)}, R = Q
        acc = fma(sg * outtab[baseJ[q] + j], p0tab[baseJ[PALL ^ q] + c2], acc);
    }
#pragma unroll
    for (int q = 0; q < PALL; ++q) {
        const double sg = (MODE == MODE_KAPPA) ? ((__popc(q) & 1) ? sd : -sd)
                                               : -1.0 / (double)(4 << __popc(q));  // R = Q + {c2}
        acc = fma(sg * outtab[baseT[q] + t], p0R[PALL ^ q], acc);
    }
    if (MODE == MODE_SPINK) return acc * (double)(1 << (NP + 2));
    return acc;
}

template <int MODE>
__device__ __forceinline__ void store_entry(const FwdArgs &a, int d, uint64_t idx, double P0, double v, bool write_p0);

// ---------------------------------------------------------------- small kernels

// Writes block idx = x*M + y of A = (V+I)/2 as 4 doubles, and (if Af is not
// null) as 4 hi floats then 4 lo floats for the refined path.
__device__ __forceinline__ void pack_entry(const double *__restrict__ V, int M, double *__restrict__ A,
                                           float *__restrict__ Af, int idx) {
    const int x = idx / M, y = idx - x * M;
    const size_t n2 = 2 * (size_t)M;
    double a00 = V[x * n2 + y], a01 = V[x * n2 + y + M];
    double a10 = V[(x + M) * n2 + y], a11 = V[(x + M) * n2 + y + M];
    if (x == y) {
        a00 += 1.0;
        a11 += 1.0;
    }
    const Blk b{0.5 * a00, 0.5 * a01, 0.5 * a10, 0.5 * a11};
    store_blk(A + 4 * (size_t)idx, b);
    if (Af) {
        float4 h, l;
        split_df(b.a00, h.x, l.x);
        split_df(b.a01, h.y, l.y);
        split_df(b.a10, h.z, l.z);
        split_df(b.a11, h.w, l.w);
        float4 *f = reinterpret_cast<float4 *>(Af) + 2 * (size_t)idx;
        f[0] = h;
        f[1] = l;
    }
}


template <int MODE, bool DISP = false>
__device__ __forceinline__ void order1_entry(const FwdArgs &a, int j, bool write_p0) {
    const Sym s = blk_sym(ablk(a.A, a.M, j, j));
    const double det = det_sym(s);
    const double rs = rsqrt(det);
    double P0 = rs;
    if (DISP) P0 *= exp(-quad_inv(s, rs * rs, half_mean(a.mean, a.M, j)));
    if (!(det > 0.0) || !(s.s00 > 0.0)) {
        flag_status(a.status, ST_NOT_POSDEF);
        P0 = __longlong_as_double(0x7ff8000000000000ULL);
    }
    if (a.p0f && a.precision == 1) split_df(P0, a.p0f[2 * j], a.p0f[2 * j + 1]);
    // mu({j}) = kt({j}) = 1 - P0({j});  c({j}) = kappa({j}) = 2 P0({j}) - 1
    const double v = (MODE == MODE_MU || MODE == MODE_KAPPA) ? 1.0 - P0
                   : (MODE == MODE_SPINC || MODE == MODE_SPINK) ? fma(2.0, P0, -1.0) : P0;
    store_entry<MODE>(a, 1, (uint64_t)j, P0, v, write_p0);
}


template <int MODE, bool DISP = false>
__device__ __forceinline__ void order2_entry(const FwdArgs &a, uint32_t t, bool write_p0) {
    const int M = a.M;
    int c2, j;
    pair_decode(t, c2, j);
    bool ok;
    double detp;
    const LInv m2 = chol2_inv(blk_sym(ablk(a.A, M, c2, c2)), ok, detp);
    const Blk w = lmul(m2, ablk(a.A, M, c2, j));
    const Sym sch = sym_sub_gram(blk_sym(ablk(a.A, M, j, j)), w);
    const double det2 = det_sym(sch);
    const double rs = rsqrt(det2);
    double P0 = a.p0[c2] * rs;
    if (DISP) {
        const Vec2 r = sub_wtg(half_mean(a.mean, M, j), w, lvec(m2, half_mean(a.mean, M, c2)));
        P0 *= exp(-quad_inv(sch, rs * rs, r));
    }
    if (!(det2 > 0.0) || !ok) {
        flag_status(a.status, ST_NOT_POSDEF);
        P0 = __longlong_as_double(0x7ff8000000000000ULL);
    }
    const uint64_t idx = (uint64_t)M + t;
    double v = P0;
    if (MODE == MODE_MU) v = a.out[c2] - a.p0[j] + P0;
    if (MODE == MODE_KAPPA) v = fma(-a.p0[j], a.p0[c2], P0);
    // c({j,c2}) = -c({c2}) - 2 (P0({j}) - 2 P0(S));  kappa(S) = 4 (P0(S) - P0({j}) P0({c2}))
    if (MODE == MODE_SPINC) v = fma(4.0, P0, fma(-2.0, a.p0[j], -a.out[c2]));
    if (MODE == MODE_SPINK) v = 4.0 * fma(-a.p0[j], a.p0[c2], P0);
    store_entry<MODE>(a, 2, idx, P0, v, write_p0);
}


template <int MODE, bool DISP = false>
__device__ __forceinline__ void order3_entry(const FwdArgs &a, uint64_t r, bool write_p0) {
    const int M = a.M;
    int s[3];
    colex_unrank(r, 3, s);
    const int j = s[0], c2 = s[1], c3 = s[2];
    const uint32_t t = (uint32_t)binom2(c2) + j;
    bool ok3, ok2;
    double dd;
    const LInv m3 = chol2_inv(blk_sym(ablk(a.A, M, c3, c3)), ok3, dd);
    const Blk z2 = lmul(m3, ablk(a.A, M, c3, c2));
    const Blk zj = lmul(m3, ablk(a.A, M, c3, j));
    const LInv m2 = chol2_inv(sym_sub_gram(blk_sym(ablk(a.A, M, c2, c2)), z2), ok2, dd);
    const Sym dj = sym_sub_gram(blk_sym(ablk(a.A, M, j, j)), zj);
    const Blk X = blk_sub_cross(ablk(a.A, M, c2, j), z2, zj);
    const Blk w = lmul(m2, X);
    const Sym sch = sym_sub_gram(dj, w);
    const double det2 = det_sym(sch);
    uint64_t baseJ[2], baseT[2], idxQ[2];
    const int P[1] = {c3};
    child_bases<1>(P, M, baseJ, baseT, idxQ);
    const double rs = rsqrt(det2);
    double P0 = a.p0[baseJ[1] + c2] * rs;
    if (DISP) {
        const Vec2 g3 = lvec(m3, half_mean(a.mean, M, c3));
        const Vec2 r2 = sub_wtg(half_mean(a.mean, M, c2), z2, g3);
        const Vec2 rj = sub_wtg(half_mean(a.mean, M, j), zj, g3);
        P0 *= exp(-quad_inv(sch, rs * rs, sub_wtg(rj, w, lvec(m2, r2))));
    }
    if (!(det2 > 0.0) || !ok3 || !ok2) {
        flag_status(a.status, ST_NOT_POSDEF);
        P0 = __longlong_as_double(0x7ff8000000000000ULL);
    }
    const double p0R[2] = {0.0, a.p0[idxQ[1]]};
    const double v = combine<1, MODE>(P0, j, c2, t, baseJ, baseT, p0R, a.p0, a.out);
    store_entry<MODE>(a, 3, baseT[1] + t, P0, v, write_p0);
}


// ---------------------------------------------------------------- tree kernel

// CC: children per batch it has room for. YC > 0: the slot-free form of the
// refined path, which keeps the item's elimination rows Y(x) (x < c4 <= YC) in
// yq for the whole item and forms every Schur-complement block it needs from
// them instead of reading a slot.
template <int D, int XC = XCAP, bool DISP = false, int CC = CCAP, int YC = 0>
struct TreeShared {
    static constexpr int NP = D - 2;       // |P|
    static constexpr int NQ = 1 << NP;     // subsets of P
    // item decode: K + 1 <= M - 2 prefix entries, M <= XC + 1 for the shapes whose
    // x-entry area is smaller than GBS_MAX_MODES
    uint32_t c4pref[XC < GBS_MAX_MODES ? XC + 3 : GBS_MAX_MODES + 2];
    uint32_t item;
    // uniform pivots of the item's U (and, displaced, their whitened half-means)
    double upiv[DISP ? 10 : 8];
    // children of the current batch
    int c3[CC];
    int xoff[CC + 1];
    uint32_t lpref[CC + 1];
    uint64_t baseJ[CC][NQ];
    uint64_t baseT[CC][NQ];
    double p0R[CC][NQ];
    double m3[CC][3];
    float m3f[CC][6];  // refined path: m3 as float pairs (h, l) x 3
    double g3[DISP ? CC : 1][2];  // displaced: whitened half-mean of each child's c3 pivot
    // Per x-entry data, structure of arrays. FP64 path (10 double rows):
    // z(x) = m3 * S_U[c3, x] (rows 0-3), d(x) = S_U[x,x] - z^T z (rows 4-6),
    // inverse c2-pivot factor m2(x) (rows 7-9). Refined-FP32 path (6 float4
    // rows, so that a leaf loads its x-entries with 9 vector loads, consecutive
    // entries in consecutive 16-byte words): z hi (0), z lo (1), (d hi 00 01 11,
    // d lo 00) (2), (d lo 01 11, c2 pivot FP32 factor l00 l10) (3), (l11, its
    // inverse m00 m10 m11) (4), residual d - l l^T (e00 e01 e11, 0) (5).
    // Displaced states add 4 double rows: the reduced half-mean r(x) after
    // eliminating U and c3 (rows 10-11) and its whitened form g2(x) = m2(x) r(x)
    // as a c2 pivot (rows 12-13).
    // Before the batches of an item start, the same storage holds Y(x) of the
    // elimination of U (8 doubles per mode x < c4).
    static constexpr int XROWS = DISP ? 14 : 10;
    static constexpr int XBYTES = (6 * 16 > XROWS * 8 ? 6 * 16 : XROWS * 8) * XC;
    alignas(16) unsigned char xraw[XBYTES];
    // slot-free form: Y(x) as 16 floats (hi, lo of y5 00 01 10 11, then of y4) in
    // four float4 rows, row r holding floats 4r..4r+3 of every x
    alignas(16) float4 yq[YC > 0 ? 4 : 1][YC > 0 ? YC : 1];
    __device__ double (*xe())[XC] { return reinterpret_cast<double(*)[XC]>(xraw); }
    __device__ float (*xf())[XC] { return reinterpret_cast<float(*)[XC]>(xraw); }
    __device__ float4 (*xq())[XC] { return reinterpret_cast<float4(*)[XC]>(xraw); }
};

// Schur-complement slot access. FP64 path: 2x2 blocks as 4 doubles. Refined
// path: the same 32 bytes hold 4 hi floats then 4 lo floats (value = hi + lo).
template <int PREC>
__device__ __forceinline__ Blk slot_pair_f64(const double *slot, size_t q) {
    if (PREC == 0) return load_blk(slot + 4 * q);
    const float4 *f = reinterpret_cast<const float4 *>(slot) + 2 * q;
    const float4 h = f[0], l = f[1];
    return Blk{join_df(h.x, l.x), join_df(h.y, l.y), join_df(h.z, l.z), join_df(h.w, l.w)};
}
template <int PREC>
__device__ __forceinline__ Sym slot_diag_f64(const double *sdiag, int x) {
    if (PREC == 0) return Sym{sdiag[4 * x], sdiag[4 * x + 1], sdiag[4 * x + 2]};
    const float *f = reinterpret_cast<const float *>(sdiag) + 8 * x;
    return Sym{join_df(f[0], f[3]), join_df(f[1], f[4]), join_df(f[2], f[5])};
}
template <int PREC>
__device__ __forceinline__ void slot_store_pair(double *slot, size_t q, const Blk &b) {
    if (PREC == 0) {
        store_blk(slot + 4 * q, b);
        return;
    }
    float4 h, l;
    split_df(b.a00, h.x, l.x);
    split_df(b.a01, h.y, l.y);
    split_df(b.a10, h.z, l.z);
    split_df(b.a11, h.w, l.w);
    float4 *f = reinterpret_cast<float4 *>(slot) + 2 * q;
    f[0] = h;
    f[1] = l;
}
template <int PREC>
__device__ __forceinline__ void slot_store_diag(double *sdiag, int x, const Sym &d) {
    if (PREC == 0) {
        store_blk(sdiag + 4 * (size_t)x, Blk{d.s00, d.s01, d.s11, 0.0});
        return;
    }
    float4 h, l;
    split_df(d.s00, h.x, h.w);
    split_df(d.s01, h.y, l.x);
    split_df(d.s11, h.z, l.y);
    l.z = l.w = 0.f;
    // layout: h00 h01 h11 l00 | l01 l11 _ _
    float4 *f = reinterpret_cast<float4 *>(sdiag) + 2 * (size_t)x;
    f[0] = h;
    f[1] = l;
}

// Schur-complement block S_U[x][y] (x >= y) of the refined path formed from A's
// float-pair block and the rows Y(x), Y(y) of the eliminated modes U:
// b_uv -= sum_k y(x)_ku y(y)_kv over the pivot rows k of c5 (D = 5) and c4, in
// float pairs on the FP32 pipe. The same operations in the same order as the
// slot build, so both forms give the same bits.
template <int D, int YC>
__device__ __forceinline__ void su_block(const float *__restrict__ Af, int M, const float4 (*yq)[YC], int x, int y,
                                         DF (&b)[4]) {
    const float4 a0 = reinterpret_cast<const float4 *>(Af)[2 * ((size_t)x * M + y)];
    const float4 a1 = reinterpret_cast<const float4 *>(Af)[2 * ((size_t)x * M + y) + 1];
    b[0] = DF{a0.x, a1.x};
    b[1] = DF{a0.y, a1.y};
    b[2] = DF{a0.z, a1.z};
    b[3] = DF{a0.w, a1.w};
    // one pivot row k of one eliminated mode at a time: x's elements (k, 0), (k, 1)
    // and y's in one float4 each; every element still takes its four updates in
    // the build's order (c5 row 0, c5 row 1, c4 row 0, c4 row 1)
#pragma unroll
    for (int blk = (D == 5 ? 0 : 1); blk < 2; ++blk)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float4 xr = yq[2 * blk + k][x], yr = yq[2 * blk + k][y];
            const DF x0{xr.x, xr.y}, x1{xr.z, xr.w}, y0{yr.x, yr.y}, y1{yr.z, yr.w};
            b[0] = df_sub_mul(b[0], x0, y0);
            b[1] = df_sub_mul(b[1], x0, y1);
            b[2] = df_sub_mul(b[2], x1, y0);
            b[3] = df_sub_mul(b[3], x1, y1);
        }
}

// Number of stride classes the children c3 in [2, c4) of one U are split into.
__host__ __device__ __forceinline__ int n_classes(int c4, uint64_t target) {
    const uint64_t leaves = binom(c4, 3);
    uint64_t n = (leaves + target - 1) / target;
    if (n < 1) n = 1;
    if (n > (uint64_t)(c4 - 2)) n = (uint64_t)(c4 - 2);
    return (int)n;
}

// Items of the order-D prefix tree whose top element (c5 for D = 5, c4 for
// D = 4) lies in [lo, hi): the largest c4 that has any, and the items of one c4.
template <int D>
__host__ __device__ __forceinline__ int c4_max(int M, int hi) {
    const int top = hi < M ? hi : M;
    return D == 5 ? top - 2 : top - 1;
}
template <int D>
__host__ __device__ __forceinline__ int c4_max(int M) {
    return c4_max<D>(M, M);
}

// First top element c5 of the items of one c4 (D = 5).
__host__ __device__ __forceinline__ int c5_first(int c4, int lo) { return c4 + 1 > lo ? c4 + 1 : lo; }

template <int D>
__host__ __device__ __forceinline__ uint32_t items_for_c4(int M, int c4, uint64_t target, int lo, int hi) {
    int nU;
    if (D == 5) {
        const int first = c5_first(c4, lo), last = hi < M ? hi : M;
        nU = last > first ? last - first : 0;
    } else {
        nU = (c4 >= lo && c4 < hi) ? 1 : 0;
    }
    return (uint32_t)nU * (uint32_t)n_classes(c4, target);
}
template <int D>
__host__ __device__ __forceinline__ uint32_t items_for_c4(int M, int c4, uint64_t target) {
    return items_for_c4<D>(M, c4, target, 0, M);
}

// Stores entry idx (table layout) of order d: into the caller's slice of order
// kmax during a range call, else into the P0 table (write_p0) and the mode's table.
template <int MODE>
__device__ __forceinline__ void store_entry(const FwdArgs &a, int d, uint64_t idx, double P0, double v, bool write_p0) {
    if (a.top && d == a.kmax) {
        a.top[idx - a.top_base] = (MODE == MODE_P0) ? P0 : v;
        return;
    }
    if (write_p0) a.p0[idx] = P0;
    if (MODE != MODE_P0) a.out[idx] = v;
}

// One work item of the prefix-tree kernel: U = {c4, c5} (D = 5) or {c4} (D = 4),
// children c3 = c4-1-s, c4-1-s-nc, ... >= 2 (stride class s of nc). Called by all
// threads of the block; sh is the block's shared memory, slot its scratch slot.
//
// Displaced states (DISP, FP64 only) carry the reduced half-means along: the
// slot holds r_U(x) after the Schur blocks, the x-entries r(x) and g2(x), and
// each leaf multiplies its P0 by exp(-r^T Sch^{-1} r).
//
// CL: the CTAs of a thread-block cluster share one slot and one U. CTA `part` of
// `nparts` writes every nparts-th chunk of NT Schur blocks, and a cluster-wide
// barrier (release / acquire, so the other CTAs' global writes are visible)
// replaces the block barrier after the build; the caller passes s = part,
// nc = nparts, so each CTA then takes one stride class of the children.
//
// YC > 0 (refined path only): no slot. Y(x) stays in shared memory for the
// whole item and each Schur-complement block is formed where it is used
// (su_block): the c3 pivots, z(x) and d(x) of the batch setup, and one block per
// leaf pair and batch. That trades FP32 work (about 60 more FP32 instructions
// per order-5 leaf with a 384-entry x area) for the slot's DRAM writes and
// re-reads.
template <int D, int MODE, int PREC, int NT = TREE_THREADS, int XC = XCAP, bool DISP = false, bool CL = false,
          int CC = CCAP, int YC = 0>
__device__ __forceinline__ void tree_item(const FwdArgs &a, TreeShared<D, XC, DISP, CC, YC> &sh, double *const slot,
                                          const int c4, const int c5, const int s, const int nc, const bool write_p0,
                                          const int ccap_in = CCAP, const int part = 0, const int nparts = 1) {
    static_assert(!DISP || PREC == 0, "displaced states run in FP64");
    static_assert(!(DISP && CL), "displaced states run without clusters");
    constexpr bool NOSLOT = YC > 0;
    static_assert(!NOSLOT || (PREC == 1 && !CL), "the slot-free form is the refined path's, without clusters");
    const int ccap = ccap_in < CC ? ccap_in : CC;
    using SH = TreeShared<D, XC, DISP, CC, YC>;
    constexpr int NP = SH::NP;
    constexpr int NQ = SH::NQ;
    constexpr int PALL = NQ - 1;
    double(*const xe)[XC] = sh.xe();
    float(*const xf)[XC] = sh.xf();
    float4(*const xq)[XC] = sh.xq();
    const int tid = threadIdx.x;
    const int M = a.M;
    double *const sdiag = slot + 4 * binom2(M);
    double *const rU = sdiag + 4 * (size_t)M;  // displaced: reduced half-means, 2 per mode
    const double *__restrict__ A = a.A;

    if constexpr (NOSLOT) {
        if (c4 > YC) {  // Y rows beyond the shared area (the launcher bounds M): reject, block-uniformly
            if (tid == 0) flag_status(a.status, ST_BAD_INDEX);
            return;
        }
    }
    // ---- Schur complement of A after eliminating U, modes < c4 -> slot
    // uniform pivots: m5 = chol(A[c5,c5])^{-1}, y5(c4), m4 = chol(Pi4)^{-1}
    if (tid == 0) {
        bool ok = true, ok2 = true;
        double dd;
        LInv m5{0, 0, 0};
        Blk y5c4{0, 0, 0, 0};
        Sym pi4 = blk_sym(ablk(A, M, c4, c4));
        if (D == 5) {
            m5 = chol2_inv(blk_sym(ablk(A, M, c5, c5)), ok, dd);
            y5c4 = lmul(m5, ablk(A, M, c5, c4));
            pi4 = sym_sub_gram(pi4, y5c4);
        }
        const LInv m4 = chol2_inv(pi4, ok2, dd);
        if (!ok || !ok2) flag_status(a.status, ST_NOT_POSDEF);
        sh.upiv[0] = m5.m00; sh.upiv[1] = m5.m10; sh.upiv[2] = m5.m11;
        sh.upiv[3] = m4.m00; sh.upiv[4] = m4.m10; sh.upiv[5] = m4.m11;
        if constexpr (DISP) {
            Vec2 g5{0, 0}, r4 = half_mean(a.mean, M, c4);
            if (D == 5) {
                g5 = lvec(m5, half_mean(a.mean, M, c5));
                r4 = sub_wtg(r4, y5c4, g5);
            }
            const Vec2 g4 = lvec(m4, r4);
            sh.upiv[6] = g5.v0; sh.upiv[7] = g5.v1; sh.upiv[8] = g4.v0; sh.upiv[9] = g4.v1;
        }
    }
    __syncthreads();
    {
        // Y(x) = [y5(x); y4(x)] into the x-entry area (it is free until the batches start):
        // 8 doubles per x (FP64 path) or 8 float pairs per x (refined path); x < c4 <= 1023
        double *Y = &xe[0][0];
        float *Yf = &xf[0][0];
        const LInv m5{sh.upiv[0], sh.upiv[1], sh.upiv[2]};
        const LInv m4{sh.upiv[3], sh.upiv[4], sh.upiv[5]};
        Blk y5c4{0, 0, 0, 0};
        if (D == 5) y5c4 = lmul(m5, ablk(A, M, c5, c4));
        for (int x = tid; x < c4; x += NT) {
            Blk y5{0, 0, 0, 0};
            Blk r4 = ablk(A, M, c4, x);
            if (D == 5) {
                y5 = lmul(m5, ablk(A, M, c5, x));
                r4 = blk_sub_cross(r4, y5c4, y5);
            }
            const Blk y4 = lmul(m4, r4);
            if constexpr (DISP) {
                Vec2 r = half_mean(a.mean, M, x);
                if (D == 5) r = sub_wtg(r, y5, Vec2{sh.upiv[6], sh.upiv[7]});
                r = sub_wtg(r, y4, Vec2{sh.upiv[8], sh.upiv[9]});
                rU[2 * x] = r.v0;
                rU[2 * x + 1] = r.v1;
            }
            const double v[8] = {y5.a00, y5.a01, y5.a10, y5.a11, y4.a00, y4.a01, y4.a10, y4.a11};
            if constexpr (NOSLOT) {
                float f[16];
#pragma unroll
                for (int k = 0; k < 8; ++k) split_df(v[k], f[2 * k], f[2 * k + 1]);
#pragma unroll
                for (int r = 0; r < 4; ++r) sh.yq[r][x] = make_float4(f[4 * r], f[4 * r + 1], f[4 * r + 2], f[4 * r + 3]);
            } else if (PREC == 0) {
#pragma unroll
                for (int k = 0; k < 8; ++k) Y[8 * x + k] = v[k];
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) split_df(v[k], Yf[16 * x + 2 * k], Yf[16 * x + 2 * k + 1]);
            }
        }
        __syncthreads();
        // the slot build (the slot-free form has nothing more to do: Y is in place)
        if constexpr (!NOSLOT) {
        const uint32_t npairs = (uint32_t)binom2(c4);
        for (uint32_t qi = (uint32_t)(part * NT + tid); qi < npairs + (uint32_t)c4; qi += (uint32_t)(nparts * NT)) {
            int x, y;
            if (qi < npairs) pair_decode(qi, x, y);
            else x = y = (int)(qi - npairs);
            if (PREC == 0) {
                const double *px = Y + 8 * x, *py = Y + 8 * y;
                Blk b = ablk(A, M, x, y);
                const Blk y5x{px[0], px[1], px[2], px[3]}, y5y{py[0], py[1], py[2], py[3]};
                const Blk y4x{px[4], px[5], px[6], px[7]}, y4y{py[4], py[5], py[6], py[7]};
                if (D == 5) b = blk_sub_cross(b, y5x, y5y);
                b = blk_sub_cross(b, y4x, y4y);
                if (qi < npairs) slot_store_pair<PREC>(slot, qi, b);
                else slot_store_diag<PREC>(sdiag, x, Sym{b.a00, 0.5 * (b.a01 + b.a10), b.a11});
            } else {
                // the same elimination in float pairs: b_uv -= sum_k y(x)_ku y(y)_kv over the
                // pivot rows k of each eliminated mode (y as a 2x2 block {00, 01, 10, 11})
                const float *af = a.Af + 8 * ((size_t)x * M + y);
                DF b[4] = {{af[0], af[4]}, {af[1], af[5]}, {af[2], af[6]}, {af[3], af[7]}};
                const float *px = Yf + 16 * x, *py = Yf + 16 * y;
#pragma unroll
                for (int blk = (D == 5 ? 0 : 1); blk < 2; ++blk) {
                    const float *qx = px + 8 * blk, *qy = py + 8 * blk;
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int v = 0; v < 2; ++v)
#pragma unroll
                            for (int k = 0; k < 2; ++k)
                                b[2 * u + v] = df_sub_mul(b[2 * u + v], DF{qx[2 * (2 * k + u)], qx[2 * (2 * k + u) + 1]},
                                                          DF{qy[2 * (2 * k + v)], qy[2 * (2 * k + v) + 1]});
                }
                if (qi < npairs) {
                    float4 *f = reinterpret_cast<float4 *>(slot) + 2 * (size_t)qi;
                    f[0] = make_float4(b[0].h, b[1].h, b[2].h, b[3].h);
                    f[1] = make_float4(b[0].l, b[1].l, b[2].l, b[3].l);
                } else {
                    // layout: h00 h01 h11 l00 | l01 l11 _ _
                    float4 *f = reinterpret_cast<float4 *>(sdiag) + 2 * (size_t)x;
                    f[0] = make_float4(b[0].h, b[1].h, b[3].h, b[0].l);
                    f[1] = make_float4(b[1].l, b[3].l, 0.f, 0.f);
                }
            }
        }
        if constexpr (CL) cooperative_groups::this_cluster().sync();
        else __syncthreads();
        }
    }

    // ---- children c3 = c4-1-s, c4-1-s-nc, ... >= 2, processed in batches
    const int cfirst = c4 - 1 - s;
    const int nchild = (cfirst >= 2) ? (cfirst - 2) / nc + 1 : 0;
    int k0 = 0;
    while (k0 < nchild) {
        // batch [k0, k0+nb): identical arithmetic in every thread
        int nb = 0, xs = 0;
        while (k0 + nb < nchild && nb < ccap) {
            const int c3 = cfirst - (k0 + nb) * nc;
            if (xs + c3 > XC) break;
            xs += c3;
            ++nb;
        }
        if (nb == 0) {  // a child wider than the x-entry area: reject instead of spinning
            if (tid == 0) flag_status(a.status, ST_BAD_INDEX);
            break;
        }
        // pre-setup: one thread per child
        if (tid < nb) {
            const int b = tid;
            const int c3 = cfirst - (k0 + b) * nc;
            int xo = 0;
            uint32_t lp = 0;
            for (int q = 0; q < b; ++q) {
                const int cq = cfirst - (k0 + q) * nc;
                xo += cq;
                lp += (uint32_t)binom2(cq);
            }
            sh.c3[b] = c3;
            sh.xoff[b] = xo;
            sh.lpref[b] = lp;
            if (b == nb - 1) {
                sh.xoff[nb] = xo + c3;
                sh.lpref[nb] = lp + (uint32_t)binom2(c3);
            }
            int P[3] = {c3, c4, c5};
            uint64_t idxQ[NQ];
            child_bases<NP>(P, M, sh.baseJ[b], sh.baseT[b], idxQ);
            sh.p0R[b][0] = 0.0;
#pragma unroll
            for (int q = 1; q < NQ; ++q) sh.p0R[b][q] = a.p0[idxQ[q]];
            bool ok;
            double dd;
            Sym p3;
            if constexpr (NOSLOT) {
                DF b[4];
                su_block<D, YC>(a.Af, M, sh.yq, c3, c3, b);
                p3 = Sym{join_df(b[0].h, b[0].l), join_df(b[1].h, b[1].l), join_df(b[3].h, b[3].l)};
            } else {
                p3 = slot_diag_f64<PREC>(sdiag, c3);
            }
            const LInv m3 = chol2_inv(p3, ok, dd);
            if (!ok) flag_status(a.status, ST_NOT_POSDEF);
            sh.m3[b][0] = m3.m00; sh.m3[b][1] = m3.m10; sh.m3[b][2] = m3.m11;
            if constexpr (DISP) {
                const Vec2 g3 = lvec(m3, Vec2{rU[2 * c3], rU[2 * c3 + 1]});
                sh.g3[b][0] = g3.v0;
                sh.g3[b][1] = g3.v1;
            }
            if (PREC == 1) {
                split_df(m3.m00, sh.m3f[b][0], sh.m3f[b][1]);
                split_df(m3.m10, sh.m3f[b][2], sh.m3f[b][3]);
                split_df(m3.m11, sh.m3f[b][4], sh.m3f[b][5]);
            }
        }
        __syncthreads();
        // setup: eliminate c3 for every x < c3 of every child in the batch
        for (int e = tid; e < xs; e += NT) {
            int lo2 = 0, hi2 = nb;
            while (hi2 - lo2 > 1) {
                const int mid = (lo2 + hi2) >> 1;
                if (sh.xoff[mid] <= e) lo2 = mid;
                else hi2 = mid;
            }
            const int b = lo2;
            const int c3 = sh.c3[b];
            const int x = e - sh.xoff[b];
            if (PREC == 0) {
                const LInv m3{sh.m3[b][0], sh.m3[b][1], sh.m3[b][2]};
                const Blk z = lmul(m3, slot_pair_f64<PREC>(slot, binom2(c3) + x));
                const Sym dx = sym_sub_gram(slot_diag_f64<PREC>(sdiag, x), z);
                xe[0][e] = z.a00; xe[1][e] = z.a01; xe[2][e] = z.a10; xe[3][e] = z.a11;
                xe[4][e] = dx.s00; xe[5][e] = dx.s01; xe[6][e] = dx.s11;
                Vec2 r3{0, 0};
                if constexpr (DISP) {
                    r3 = sub_wtg(Vec2{rU[2 * x], rU[2 * x + 1]}, z, Vec2{sh.g3[b][0], sh.g3[b][1]});
                    xe[10][e] = r3.v0; xe[11][e] = r3.v1;
                }
                if (x >= 1) {
                    bool ok;
                    double dd;
                    const LInv m2 = chol2_inv(dx, ok, dd);
                    if (!ok) flag_status(a.status, ST_NOT_POSDEF);
                    xe[7][e] = m2.m00; xe[8][e] = m2.m10; xe[9][e] = m2.m11;
                    if constexpr (DISP) {
                        const Vec2 g2 = lvec(m2, r3);
                        xe[12][e] = g2.v0; xe[13][e] = g2.v1;
                    }
                }
            } else {
                // z(x) = m3 S_U[c3, x] and d(x) = S_U[x, x] - z^T z in float pairs (FP32 pipe)
                DF S00, S01, S10, S11, D00, D01, D11;
                if constexpr (NOSLOT) {
                    DF b[4];
                    su_block<D, YC>(a.Af, M, sh.yq, c3, x, b);
                    S00 = b[0]; S01 = b[1]; S10 = b[2]; S11 = b[3];
                    su_block<D, YC>(a.Af, M, sh.yq, x, x, b);
                    D00 = b[0]; D01 = b[1]; D11 = b[3];
                } else {
                    const float *fs = reinterpret_cast<const float *>(slot) + 8 * (binom2(c3) + x);
                    const float *fd = reinterpret_cast<const float *>(sdiag) + 8 * x;
                    S00 = DF{fs[0], fs[4]}; S01 = DF{fs[1], fs[5]}; S10 = DF{fs[2], fs[6]}; S11 = DF{fs[3], fs[7]};
                    D00 = DF{fd[0], fd[3]}; D01 = DF{fd[1], fd[4]}; D11 = DF{fd[2], fd[5]};
                }
                const DF m00{sh.m3f[b][0], sh.m3f[b][1]}, m10{sh.m3f[b][2], sh.m3f[b][3]}, m11{sh.m3f[b][4], sh.m3f[b][5]};
                const DF z00 = df_mul(m00, S00), z01 = df_mul(m00, S01);
                const DF z10 = df_add_mul(df_mul(m10, S00), m11, S10);
                const DF z11 = df_add_mul(df_mul(m10, S01), m11, S11);
                const DF d00 = df_sub_mul(df_sub_mul(D00, z00, z00), z10, z10);
                const DF d01 = df_sub_mul(df_sub_mul(D01, z00, z01), z10, z11);
                const DF d11 = df_sub_mul(df_sub_mul(D11, z01, z01), z11, z11);
                xq[0][e] = make_float4(z00.h, z01.h, z10.h, z11.h);
                xq[1][e] = make_float4(z00.l, z01.l, z10.l, z11.l);
                xq[2][e] = make_float4(d00.h, d01.h, d11.h, d00.l);
                float4 q3 = make_float4(d01.l, d11.l, 0.f, 0.f), q4 = make_float4(0.f, 0.f, 0.f, 0.f),
                       q5 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (x >= 1) {
                    // FP32 Cholesky factor of the c2 pivot d(x), its inverse, and the residual
                    // d - l l^T formed exactly (two-product, two-sum)
                    const float pa = d00.h, pb = d01.h, pc = d11.h;
                    const float i0 = rsqrtf(pa);
                    const float l00 = pa * i0, l10 = pb * i0;
                    const float pq = __fmaf_rn(-l10, l10, pc);
                    const float i1 = rsqrtf(pq);
                    const float l11 = pq * i1;
                    if (!(pa > 0.f) || !(pq > 0.f)) flag_status(a.status, ST_NOT_POSDEF);
                    q3.z = l00;
                    q3.w = l10;
                    q4 = make_float4(l11, i0, -l10 * i0 * i1, i1);
                    EftAcc r00{d00.h, d00.l}, r01{d01.h, d01.l}, r11{d11.h, d11.l};
                    eft_sub_prod(r00, l00, l00);
                    eft_sub_prod(r01, l00, l10);
                    eft_sub_prod(r11, l10, l10);
                    eft_sub_prod(r11, l11, l11);
                    q5 = make_float4(eft_val(r00), eft_val(r01), eft_val(r11), 0.f);
                }
                xq[3][e] = q3;
                xq[4][e] = q4;
                xq[5][e] = q5;
            }
        }
        __syncthreads();
        // leaves (c2, j), j < c2 < c3: pairs t = C(c2, 2) + j on the outer loop and
        // the batch's children (c3 decreasing with b) inside, so each 2x2 block of
        // the slot is read once per batch instead of once per child
        const uint32_t L0 = (uint32_t)binom2(sh.c3[0]);
        for (uint32_t t = tid; t < L0; t += NT) {
            int c2, j;
            pair_decode(t, c2, j);
            Blk S64{0, 0, 0, 0};
            DFBlk Sdf{};
            if constexpr (PREC == 0) {
                S64 = load_blk(slot + 4 * (size_t)t);
            } else if constexpr (NOSLOT) {
                DF b[4];
                su_block<D, YC>(a.Af, M, sh.yq, c2, j, b);
                Sdf = DFBlk{b[0].h, b[1].h, b[2].h, b[3].h, b[0].l, b[1].l, b[2].l, b[3].l};
            } else {
                const float4 *fs = reinterpret_cast<const float4 *>(slot) + 2 * (size_t)t;
                const float4 sh4 = fs[0], sl4 = fs[1];
                Sdf = DFBlk{sh4.x, sh4.y, sh4.z, sh4.w, sl4.x, sl4.y, sl4.z, sl4.w};
            }
            for (int b = 0; b < nb && c2 < sh.c3[b]; ++b) {
                const int xo = sh.xoff[b];
                const int e2 = xo + c2, ej = xo + j;
                const uint64_t *bJ = sh.baseJ[b];
                const uint64_t *bT = sh.baseT[b];
                const double P0Sp = a.p0[bJ[PALL] + c2];
                double P0;
                bool ok;
                if constexpr (PREC == 0) {
                    const Blk z2{xe[0][e2], xe[1][e2], xe[2][e2], xe[3][e2]};
                    const Blk zj{xe[0][ej], xe[1][ej], xe[2][ej], xe[3][ej]};
                    const LInv m2{xe[7][e2], xe[8][e2], xe[9][e2]};
                    const Sym dj{xe[4][ej], xe[5][ej], xe[6][ej]};
                    const Blk X = blk_sub_cross(S64, z2, zj);
                    const Blk w = lmul(m2, X);
                    const Sym sch = sym_sub_gram(dj, w);
                    const double det2 = det_sym(sch);
                    const double rs = rsqrt(det2);
                    P0 = P0Sp * rs;
                    if constexpr (DISP) {
                        const Vec2 r = sub_wtg(Vec2{xe[10][ej], xe[11][ej]}, w, Vec2{xe[12][e2], xe[13][e2]});
                        P0 *= exp(-quad_inv(sch, rs * rs, r));
                    }
                    ok = det2 > 0.0;
                } else {
                    const float4 zh2 = xq[0][e2], zl2 = xq[1][e2], zhj = xq[0][ej], zlj = xq[1][ej];
                    const float4 dj0 = xq[2][ej], dj1 = xq[3][ej];
                    const float4 p3 = xq[3][e2], p4 = xq[4][e2], p5 = xq[5][e2];
                    const DFBlk z2{zh2.x, zh2.y, zh2.z, zh2.w, zl2.x, zl2.y, zl2.z, zl2.w};
                    const DFBlk zj{zhj.x, zhj.y, zhj.z, zhj.w, zlj.x, zlj.y, zlj.z, zlj.w};
                    const DFSym dj{dj0.x, dj0.y, dj0.z, dj0.w, dj1.x, dj1.y};
                    const F32Piv pv{p3.z, p3.w, p4.x, p4.y, p4.z, p4.w, p5.x, p5.y, p5.z};
                    if constexpr (MODE == MODE_KAPPA || MODE == MODE_SPINK) {
                        if (!write_p0 && a.p0f) {
                            // P0(S) is not stored: its product with P0(S') folds into the
                            // recursion's leading term (15 FP64 instructions per entry)
                            float r0, eta;
                            refined_leaf_factor(Sdf, z2, zj, dj, pv, r0, eta, ok);
                            const float2 pj = reinterpret_cast<const float2 *>(a.p0f)[j];
                            double v = combine_tail<NP, MODE>(
                                refined_lead_term<(lead_sign<NP, MODE>() < 0)>(P0Sp, r0, eta, pj.x, pj.y), j, c2, t,
                                bJ, bT, sh.p0R[b], a.p0, a.out);
                            if (!ok) {
                                flag_status(a.status, ST_NOT_POSDEF);
                                v = __longlong_as_double(0x7ff8000000000000ULL);
                            }
                            store_entry<MODE>(a, NP + 2, bT[PALL] + t, 0.0, v, false);
                            continue;
                        }
                    }
                    P0 = refined_leaf_p0(P0Sp, Sdf, z2, zj, dj, pv, ok);
                }
                if (!ok) {
                    flag_status(a.status, ST_NOT_POSDEF);
                    P0 = __longlong_as_double(0x7ff8000000000000ULL);
                }
                const double v = combine<NP, MODE>(P0, j, c2, t, bJ, bT, sh.p0R[b], a.p0, a.out);
                store_entry<MODE>(a, NP + 2, bT[PALL] + t, P0, v, write_p0);
            }
        }
        __syncthreads();
        k0 += nb;
    }
}

}  // namespace gbs
