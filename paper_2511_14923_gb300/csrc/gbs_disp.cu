// Forward tables of a displaced Gaussian state: Eq. vacuum_gaussian_prob with
// nonzero first moments, P0(T) = exp(-1/2 mean_T^T (V_T + I)^{-1} mean_T) /
// sqrt(det((V_T + I)/2)) (hbar = 2), and every table derived from P0 (click
// moments, click cumulants, spin correlators and cumulants) by the same
// inclusion-exclusion and cumulant recursions as the zero-mean path.
//
// The elimination is the zero-mean one; each mode also carries its reduced
// half-mean, which the Schur step updates like one more column of A. Splitting
// T = {j} + S' gives
//   b_T^T A_T^{-1} b_T = b_{S'}^T A_{S'}^{-1} b_{S'} + r_j^T Sch_j^{-1} r_j,
// with b = mean / 2 and r_j the half-mean of j conditioned on S', so
//   P0(T) = P0(S') det(Sch_j)^{-1/2} exp(-r_j^T Sch_j^{-1} r_j).
// Kernels are compiled in this separate translation unit (FP64, one CTA shape)
// so that the zero-mean kernels stay as they are.
#include "gbs_launch.cuh"

namespace gbs {

cudaError_t launch_forward_displaced(const FwdArgs &a_in, cudaStream_t st) {
    FwdArgs a = a_in;
    a.precision = 0;
    a.variant = 0;
    if (a.ev) cudaEventRecord(a.ev[0], st);
    cudaError_t e = launch_pack(a, st);
    if (e != cudaSuccess) return e;
    if (a.ev) cudaEventRecord(a.ev[1], st);
    return launch_orders<true>(a, st);
}

}  // namespace gbs
