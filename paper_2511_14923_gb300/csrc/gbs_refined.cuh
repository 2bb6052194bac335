// Refined-FP32 determinant step (GBS_FP32_REFINED).
//
// The leaf determinant ratio det(Sch_j) = det(A4) / det(Pi2), where
//   A4 = [[Pi2, X], [X^T, D]]   (the c2 and j blocks of the Schur complement
//                                after eliminating the prefix, 4x4 SPD)
// is computed as
//   1. an FP32 Cholesky factorisation A4 ~ L L^T, L = [[l2, 0], [w^T, s]],
//      with l2 (the c2 pivot factor) shared by every leaf of one c2;
//   2. one refinement: the residual E = A4 - L L^T formed to FP64 accuracy with
//      error-free FP32 transformations (each product of two FP32 numbers split
//      exactly into p + q by an FMA, sums tracked with Knuth's two-sum), then
//        log det A4 = 2 log det L + log det(I + G),  G = L^{-1} E L^{-T},
//      truncated after the second-order term of log det(I + G). The c2 block
//      G11 cancels against the same expansion of log det Pi2, leaving
//        log det(Sch_j) = 2 log(s00 s11) + tr G22 - ||G12||_F^2 - tr(G22^2)/2.
//   3. P0(S) = P0(S') / (s00 s11) * exp(-delta/2), assembled from an FP32
//      reciprocal with one correction term; the final two products run in FP64.
// Inputs that carry FP64 information (the Schur-complement blocks S, z(x),
// d(x)) arrive as unevaluated FP32 pairs hi + lo (about 48 significant bits).
#pragma once
#include <cuda_runtime.h>

namespace gbs {

// FP32 pair value h + l.
struct DFBlk {
    float h00, h01, h10, h11, l00, l01, l10, l11;
};
struct DFSym {
    float h00, h01, h11, l00, l01, l11;
};
// FP32 Cholesky factor of the c2 pivot, its approximate inverse and the exact
// residual Pi2 - l l^T (rounded to FP32).
struct F32Piv {
    float l00, l10, l11, m00, m10, m11, e00, e01, e11;
};

// FP32 value as FP64, assembled from its bits on the integer pipe (GB300 runs
// FP32<->FP64 conversions on its narrow FP64 pipe). Zero and subnormal inputs
// give a signed zero; inputs here are finite.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long r =
        sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)(e == 0u ? sign : r));
}

// FP64 value truncated to FP32 (toward zero: relative error below 2^-23),
// assembled from its bits on the integer pipe. Finite inputs in FP32's normal
// range only; any other input (zero, below 2^-126, at or above 2^128, inf, NaN)
// gives 0.
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned r = (hi & 0x80000000u) | ((unsigned)e << 23) | m;
    return (e > 0 && e < 255) ? __uint_as_float(r) : 0.f;
}

// Double-float (unevaluated FP32 pair) arithmetic on the FP32 pipe, after Dekker
// and Knuth: products split exactly by an FMA, sums by two-sum. Relative
// accuracy about 2^-47 per operation.
struct DF {
    float h, l;
};
__device__ __forceinline__ DF df_norm(float s, float t) {  // fast two-sum, |s| >= |t|
    const float r = __fadd_rn(s, t);
    return DF{r, __fsub_rn(t, __fsub_rn(r, s))};
}
// a * b
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.h * b.h;
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return df_norm(p, e);
}
// c - a * b
__device__ __forceinline__ DF df_sub_mul(DF c, DF a, DF b) {
    const float p = a.h * b.h;
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    const float s = __fadd_rn(c.h, -p);
    const float bb = __fsub_rn(s, c.h);
    float t = __fadd_rn(__fsub_rn(c.h, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    t = __fadd_rn(t, __fsub_rn(c.l, e));
    return df_norm(s, t);
}
// c + a * b
__device__ __forceinline__ DF df_add_mul(DF c, DF a, DF b) {
    return df_sub_mul(c, DF{-a.h, -a.l}, b);
}

__device__ __forceinline__ void split_df(double x, float &h, float &l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}
__device__ __forceinline__ double join_df(float h, float l) { return (double)h + (double)l; }

// Running value s + e of (A - sum of products), A given as an FP32 pair.
struct EftAcc {
    float s, e;
};

// acc -= x * y, exactly up to the final rounding of e (two-product by FMA, two-sum).
__device__ __forceinline__ void eft_sub_prod(EftAcc &a, float x, float y) {
    const float p = x * y;
    const float q = __fmaf_rn(x, y, -p);
    const float s = __fadd_rn(a.s, -p);
    const float bb = __fsub_rn(s, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    a.s = s;
    a.e = __fadd_rn(a.e, __fsub_rn(err, q));
}

// acc -= (xh + xl)(yh + yl), dropping xl*yl (below 2^-48 of the product).
__device__ __forceinline__ void eft_sub_dfprod(EftAcc &a, float xh, float xl, float yh, float yl) {
    eft_sub_prod(a, xh, yh);
    a.e = __fmaf_rn(-xh, yl, __fmaf_rn(-xl, yh, a.e));
}

__device__ __forceinline__ float eft_val(const EftAcc &a) { return __fadd_rn(a.s, a.e); }

// Refined det(Sch_j)^{-1/2} = r0 (1 + eta), r0 an FP32 reciprocal and eta its
// correction (refinement and reciprocal residual); ok = false if the FP32
// factorisation meets a non-positive pivot.
__device__ __forceinline__ void refined_leaf_factor(const DFBlk &S, const DFBlk &z2, const DFBlk &zj, const DFSym &D,
                                                    const F32Piv &pv, float &r0_out, float &eta_out, bool &ok) {
    // X ~ S - z2^T zj in FP32 (only feeds the FP32 factorisation)
    const float x00 = __fmaf_rn(-z2.h10, zj.h10, __fmaf_rn(-z2.h00, zj.h00, S.h00));
    const float x01 = __fmaf_rn(-z2.h10, zj.h11, __fmaf_rn(-z2.h00, zj.h01, S.h01));
    const float x10 = __fmaf_rn(-z2.h11, zj.h10, __fmaf_rn(-z2.h01, zj.h00, S.h10));
    const float x11 = __fmaf_rn(-z2.h11, zj.h11, __fmaf_rn(-z2.h01, zj.h01, S.h11));
    // w = l2^{-1} X
    const float w00 = pv.m00 * x00, w01 = pv.m00 * x01;
    const float w10 = __fmaf_rn(pv.m10, x00, pv.m11 * x10);
    const float w11 = __fmaf_rn(pv.m10, x01, pv.m11 * x11);
    // Schur block D - w^T w and its Cholesky factor s = [[t00, 0], [t10, t11]]
    const float s00 = __fmaf_rn(-w10, w10, __fmaf_rn(-w00, w00, D.h00));
    const float s01 = __fmaf_rn(-w10, w11, __fmaf_rn(-w00, w01, D.h01));
    const float s11 = __fmaf_rn(-w11, w11, __fmaf_rn(-w01, w01, D.h11));
    const float i0 = rsqrtf(s00);
    const float t00 = s00 * i0, t10 = s01 * i0;
    const float pp = __fmaf_rn(-t10, t10, s11);
    const float i1 = rsqrtf(pp);
    const float t11 = pp * i1;
    ok = (s00 > 0.f) && (pp > 0.f);
    // s^{-1} = [[v00, 0], [v10, v11]]
    const float v00 = i0, v11 = i1, v10 = -t10 * v00 * v11;

    // residual E12 = X - l2 w, with X = S - z2^T zj carried exactly
    EftAcc a00{S.h00, S.l00}, a01{S.h01, S.l01}, a10{S.h10, S.l10}, a11{S.h11, S.l11};
    eft_sub_dfprod(a00, z2.h00, z2.l00, zj.h00, zj.l00);
    eft_sub_dfprod(a00, z2.h10, z2.l10, zj.h10, zj.l10);
    eft_sub_prod(a00, pv.l00, w00);
    eft_sub_dfprod(a01, z2.h00, z2.l00, zj.h01, zj.l01);
    eft_sub_dfprod(a01, z2.h10, z2.l10, zj.h11, zj.l11);
    eft_sub_prod(a01, pv.l00, w01);
    eft_sub_dfprod(a10, z2.h01, z2.l01, zj.h00, zj.l00);
    eft_sub_dfprod(a10, z2.h11, z2.l11, zj.h10, zj.l10);
    eft_sub_prod(a10, pv.l10, w00);
    eft_sub_prod(a10, pv.l11, w10);
    eft_sub_dfprod(a11, z2.h01, z2.l01, zj.h01, zj.l01);
    eft_sub_dfprod(a11, z2.h11, z2.l11, zj.h11, zj.l11);
    eft_sub_prod(a11, pv.l10, w01);
    eft_sub_prod(a11, pv.l11, w11);
    const float e00 = eft_val(a00), e01 = eft_val(a01), e10 = eft_val(a10), e11 = eft_val(a11);
    // residual E22 = D - w^T w - s s^T
    EftAcc b00{D.h00, D.l00}, b01{D.h01, D.l01}, b11{D.h11, D.l11};
    eft_sub_prod(b00, w00, w00);
    eft_sub_prod(b00, w10, w10);
    eft_sub_prod(b00, t00, t00);
    eft_sub_prod(b01, w00, w01);
    eft_sub_prod(b01, w10, w11);
    eft_sub_prod(b01, t00, t10);
    eft_sub_prod(b11, w01, w01);
    eft_sub_prod(b11, w11, w11);
    eft_sub_prod(b11, t10, t10);
    eft_sub_prod(b11, t11, t11);
    const float f00 = eft_val(b00), f01 = eft_val(b01), f11 = eft_val(b11);

    // L^{-1} = [[m2, 0], [K, v]], K = -v w^T m2
    const float y00 = __fmaf_rn(w00, pv.m00, w10 * pv.m10), y01 = w10 * pv.m11;
    const float y10 = __fmaf_rn(w01, pv.m00, w11 * pv.m10), y11 = w11 * pv.m11;
    const float k00 = -v00 * y00, k01 = -v00 * y01;
    const float k10 = -__fmaf_rn(v10, y00, v11 * y10), k11 = -__fmaf_rn(v10, y01, v11 * y11);
    // F = E11 K^T + E12 v^T   (E11 = the c2 pivot residual, symmetric)
    const float F00 = __fmaf_rn(pv.e00, k00, __fmaf_rn(pv.e01, k01, e00 * v00));
    const float F01 = __fmaf_rn(pv.e00, k10, __fmaf_rn(pv.e01, k11, __fmaf_rn(e00, v10, e01 * v11)));
    const float F10 = __fmaf_rn(pv.e01, k00, __fmaf_rn(pv.e11, k01, e10 * v00));
    const float F11 = __fmaf_rn(pv.e01, k10, __fmaf_rn(pv.e11, k11, __fmaf_rn(e10, v10, e11 * v11)));
    // G12 = m2 F
    const float g00 = pv.m00 * F00, g01 = pv.m00 * F01;
    const float g10 = __fmaf_rn(pv.m10, F00, pv.m11 * F10), g11 = __fmaf_rn(pv.m10, F01, pv.m11 * F11);
    const float g12sq = __fmaf_rn(g00, g00, __fmaf_rn(g01, g01, __fmaf_rn(g10, g10, g11 * g11)));
    // H = E12^T K^T + E22 v^T
    const float H00 = __fmaf_rn(e00, k00, __fmaf_rn(e10, k01, f00 * v00));
    const float H01 = __fmaf_rn(e00, k10, __fmaf_rn(e10, k11, __fmaf_rn(f00, v10, f01 * v11)));
    const float H10 = __fmaf_rn(e01, k00, __fmaf_rn(e11, k01, f01 * v00));
    const float H11 = __fmaf_rn(e01, k10, __fmaf_rn(e11, k11, __fmaf_rn(f01, v10, f11 * v11)));
    // G22 = K F + v H
    const float G00 = __fmaf_rn(k00, F00, __fmaf_rn(k01, F10, v00 * H00));
    const float G01 = __fmaf_rn(k00, F01, __fmaf_rn(k01, F11, v00 * H01));
    const float G10 = __fmaf_rn(k10, F00, __fmaf_rn(k11, F10, __fmaf_rn(v10, H00, v11 * H10)));
    const float G11 = __fmaf_rn(k10, F01, __fmaf_rn(k11, F11, __fmaf_rn(v10, H01, v11 * H11)));
    const float Gs = 0.5f * (G01 + G10);
    const float tr = G00 + G11;
    const float tr2 = __fmaf_rn(G00, G00, __fmaf_rn(2.f * Gs, Gs, G11 * G11));
    const float delta = tr - g12sq - 0.5f * tr2;

    // 1 / (t00 t11) from an FP32 reciprocal and its exact residual
    const float qh = t00 * t11;
    const float ql = __fmaf_rn(t00, t11, -qh);
    const float r0 = __frcp_rn(qh);
    const float eps = -__fmaf_rn(ql, r0, __fmaf_rn(qh, r0, -1.f));
    const float eta = __fmaf_rn(eps, eps, eps) + delta * __fmaf_rn(0.125f, delta, __fmaf_rn(-0.5f, eps, -0.5f));
    r0_out = r0;
    eta_out = eta;
}

// P0(S) = P0(S') r0 (1 + eta): two FP64 operations.
__device__ __forceinline__ double refined_leaf_p0(double P0Sp, const DFBlk &S, const DFBlk &z2, const DFBlk &zj,
                                                  const DFSym &D, const F32Piv &pv, bool &ok) {
    float r0, eta;
    refined_leaf_factor(S, z2, zj, D, pv, r0, eta, ok);
    const double u = P0Sp * f2d_bits(r0);
    return fma(u, f2d_bits(eta), u);
}

// +-(P0(S) - P0({j}) P0(S')) = +-P0(S') (r0 (1 + eta) - p) (minus when NEG), the
// leading term of the cumulant recursion when P0(S) itself is not stored, with
// p = P0({j}) given as an FP32 pair (ph + pl). The difference
// w = r0 - ph + r0 eta - pl is formed on the FP32 pipe as an unevaluated pair
// s + lo (two-sum of r0 - ph, which is exact when they are close, plus the exact
// product r0 eta). Then P0(S') w = P0(S') s + P0(S') lo takes one FP64 FMA: the
// second product is a correction about 2^-24 below the first, so it is formed
// in FP32 from P0(S') truncated to FP32 (relative error below 2^-23 on a term
// of relative size 2^-24) and enters as the FMA's addend. P0(S') below FP32's
// normal range drops the correction (an absolute error under 1e-45). The sign
// goes into the FP32 bits.
template <bool NEG>
__device__ __forceinline__ double refined_lead_term(double P0Sp, float r0, float eta, float ph, float pl) {
    const float s = __fadd_rn(r0, -ph);
    const float bb = __fsub_rn(s, r0);
    const float e1 = __fadd_rn(__fsub_rn(r0, __fsub_rn(s, bb)), __fsub_rn(-ph, bb));
    const float pr = r0 * eta;
    const float qr = __fmaf_rn(r0, eta, -pr);
    const float lo = __fadd_rn(__fadd_rn(e1, -pl), __fadd_rn(pr, qr));
    const float c = d2f_bits(P0Sp) * lo;
    const unsigned flip = NEG ? 0x80000000u : 0u;
    return fma(P0Sp, f2d_bits(__uint_as_float(__float_as_uint(s) ^ flip)),
               f2d_bits(__uint_as_float(__float_as_uint(c) ^ flip)));
}

}  // namespace gbs
