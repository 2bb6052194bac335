// Forward kernels of libgbs: vacuum probabilities P0(S), click moments mu(S) and
// click cumulants kt(S) over all subsets of order 1..kmax (arXiv:2511.14923,
// Eq. vacuum_gaussian_prob, Eq. joint_moments_def, Eq. joint_cumulants_def).
//
// Order d is computed after orders < d, whose tables it reads.
//
//   Determinant (every order). For S = {j} + S' with j = min S, the Schur
//   complement step det A_S = det A_{S'} * det(Sch_j) gives
//   P0(S) = P0(S') * det(Sch_j)^{-1/2}, with P0(S') read from the order-(d-1)
//   table. Sch_j is the 2x2 block of j after Gaussian elimination of the modes
//   of S' from A = (V+I)/2.
//
//   Click moment. Splitting the subsets T of S by whether they contain j:
//     mu(S) = mu(S') - sum_{T' subset S'} (-1)^{|T'|} P0({j} + T').
//
//   Click cumulant. With y_k = 1 - x_k the no-click indicators, the joint
//   moments of y are the P0 values and, by translation invariance and
//   homogeneity of cumulants (the argument of Eq. cumulant_exponential),
//   kt(S) = (-1)^{|S|} ky(S) for |S| >= 2, where ky is the cumulant of y. The
//   block-containing-j recursion of Eq. correlators_expanded_2, applied to y,
//   ky(S) = P0(S) - sum_{R proper subset of S'} ky(R + {j}) P0(S' - R),
//   then gives, with ky({j}) = P0({j}) and ky(Q) = (-1)^{|Q|} kt(Q) otherwise,
//     kt(S) = (-1)^{|S|} [ P0(S) - P0({j}) P0(S')
//                          + sum_{empty != R proper subset S'} (-1)^{|R|} kt(R + {j}) P0(S' - R) ].
//   This is the partition sum of Eq. joint_cumulants_def organised by the block
//   that holds j: 2^{d-1} - 1 products per entry instead of one per partition.
//
// Kernels
//   pack_kernel     A = (V+I)/2 as M x M packed 2x2 blocks (xxpp rows k, k+M).
//   order1/2/3      one thread per subset; the elimination is redone per thread.
//   tree_kernel<D>  D = 4, 5: persistent CTAs walk the colex prefix tree. A CTA
//                   owns U = {c_4, .., c_D} and stores the Schur complement of
//                   A after eliminating U (modes below c_4) in its scratch slot.
//                   For each child P = {c_3} + U it eliminates c_3 once per
//                   mode x < c_3 (z(x), d(x), the c_2 pivots) into shared
//                   memory; each leaf (c_2, j) then costs one 2x2 cross update,
//                   one 2x2 triangular solve and one 2x2 Schur step.
#include <cstdio>

#include "gbs_launch.cuh"

namespace gbs {

__global__ void pack_kernel(const double *__restrict__ V, int M, double *__restrict__ A, float *__restrict__ Af) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < M * M) pack_entry(V, M, A, Af, idx);
}

// ---------------------------------------------------------------- host side

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(int M, int kmax, int sms, int slots_per_sm) {
    WsLayout w{};
    size_t off = 0;
    w.status_off = off;
    off = align256(off + 256);
    w.A_off = off;  // FP64 blocks, then the float-pair copy
    off = align256(off + 2 * sizeof(double) * 4 * (size_t)M * M);
    w.p0f_off = off;  // P0({x}) as float pairs
    off = align256(off + 2 * sizeof(float) * (size_t)M);
    w.p0_off = off;
    const uint64_t np0 = kmax > 1 ? order_offset(M, kmax) : 0;  // orders 1..kmax-1
    off = align256(off + sizeof(double) * (size_t)np0);
    w.scratch_off = off;
    w.slots = (slots_per_sm > 0 ? slots_per_sm : slots_per_sm_for(M)) * (sms > 0 ? sms : 1);
    // 2x2 blocks below the diagonal, diagonal blocks, then 2 doubles per mode for
    // the reduced half-means of a displaced state
    w.slot_doubles = 4 * ((size_t)binom2(M) + (size_t)M) + 2 * (size_t)M;
    if (kmax >= 4) off = align256(off + sizeof(double) * w.slot_doubles * w.slots);
    w.total = off;
    return w;
}

cudaError_t launch_pack(const FwdArgs &a, cudaStream_t st) {
    const int M = a.M;
    pack_kernel<<<(M * M + FLAT_THREADS - 1) / FLAT_THREADS, FLAT_THREADS, 0, st>>>(
        a.V, M, a.A, a.precision == 1 ? a.Af : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_forward(const FwdArgs &a, cudaStream_t st) {
    if (a.ev) cudaEventRecord(a.ev[0], st);
    cudaError_t e = launch_pack(a, st);
    if (e != cudaSuccess) return e;
    if (a.ev) cudaEventRecord(a.ev[1], st);
    return launch_orders<false>(a, st);
}

}  // namespace gbs
