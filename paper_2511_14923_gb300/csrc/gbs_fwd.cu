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

#include "gbs_tree.cuh"

namespace gbs {

__global__ void pack_kernel(const double *__restrict__ V, int M, double *__restrict__ A, float *__restrict__ Af) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < M * M) pack_entry(V, M, A, Af, idx);
}

template <int MODE>
__global__ void order1_kernel(FwdArgs a, bool write_p0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < a.M) order1_entry<MODE>(a, j, write_p0);
}

template <int MODE>
__global__ void order2_kernel(FwdArgs a, bool write_p0) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < binom2(a.M)) order2_entry<MODE>(a, t, write_p0);
}

template <int MODE>
__global__ void order3_kernel(FwdArgs a, bool write_p0) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < binom(a.M, 3)) order3_entry<MODE>(a, r, write_p0);
}

template <int D, int MODE, int PREC, int NT, int XC, int MINB>
__global__ void __launch_bounds__(NT, MINB) tree_kernel(FwdArgs a, uint64_t target, bool write_p0) {
    using SH = TreeShared<D, XC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = *reinterpret_cast<SH *>(smem_raw);
    const int tid = threadIdx.x;
    const int M = a.M;
    const int c4hi = c4_max<D>(M);
    const int K = c4hi - 2;  // c4 runs c4hi, c4hi-1, .., 3
    double *const slot = a.scratch + (size_t)blockIdx.x * a.slot_doubles;

    // prefix of item counts over c4 in descending order (warp 0, chunked scan)
    if (tid < 32) {
        const int per = (K + 31) / 32;
        const int lo = tid * per, hi = min(K, lo + per);
        uint32_t sum = 0;
        for (int k = lo; k < hi; ++k) sum += items_for_c4<D>(M, c4hi - k, target);
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += v;
        }
        uint32_t run = incl - sum;
        for (int k = lo; k < hi; ++k) {
            sh.c4pref[k] = run;
            run += items_for_c4<D>(M, c4hi - k, target);
        }
        if (tid == 31) sh.c4pref[K] = incl;
    }
    __syncthreads();
    const uint32_t total_items = sh.c4pref[K];

    for (;;) {
        if (tid == 0) sh.item = atomicAdd(a.counters + D, 1u);
        __syncthreads();
        const uint32_t item = sh.item;
        if (item >= total_items) break;
        // decode item -> (c4, c5, class s of nc)
        int lo = 0, hi = K;  // find k with c4pref[k] <= item < c4pref[k+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sh.c4pref[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int c4 = c4hi - lo;
        const int nc = n_classes(c4, target);
        const uint32_t rr = item - sh.c4pref[lo];
        const int u = (int)(rr / nc), s = (int)(rr % nc);
        const int c5 = (D == 5) ? c4 + 1 + u : M;
        tree_item<D, MODE, PREC, NT, XC>(a, sh, slot, c4, c5, s, nc, write_p0, a.ccap);
    }
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
    w.p0_off = off;
    const uint64_t np0 = kmax > 1 ? order_offset(M, kmax) : 0;  // orders 1..kmax-1
    off = align256(off + sizeof(double) * (size_t)np0);
    w.scratch_off = off;
    w.slots = (slots_per_sm > 0 ? slots_per_sm : 1) * (sms > 0 ? sms : 1);
    w.slot_doubles = 4 * ((size_t)binom2(M) + (size_t)M);
    if (kmax >= 4) off = align256(off + sizeof(double) * w.slot_doubles * w.slots);
    w.total = off;
    return w;
}

template <int D, int MODE, int PREC, int NT, int XC, int MINB>
static cudaError_t launch_tree_v(const FwdArgs &a, bool write_p0, cudaStream_t st) {
    const int M = a.M;
    const uint64_t leaves = binom(M, D);
    if (leaves == 0) return cudaSuccess;
    const size_t smem = sizeof(TreeShared<D, XC>);
    auto fn = tree_kernel<D, MODE, PREC, NT, XC, MINB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid_max = a.sms * per_sm;
    if (grid_max > a.slots) grid_max = a.slots;
    const int grain = a.grain > 0 ? a.grain : kDefaultCfg.grain;
    uint64_t target = leaves / ((uint64_t)grain * (uint64_t)grid_max);
    if (target < 256) target = 256;
    uint64_t items = 0;
    for (int c4 = c4_max<D>(M); c4 >= 3; --c4) items += items_for_c4<D>(M, c4, target);
    if (items == 0) return cudaSuccess;
    const int grid = (int)(items < (uint64_t)grid_max ? items : (uint64_t)grid_max);
    fn<<<grid, NT, smem, st>>>(a, target, write_p0);
    return cudaGetLastError();
}

template <int D, int MODE, int PREC>
static cudaError_t launch_tree(const FwdArgs &a_in, bool write_p0, cudaStream_t st) {
    FwdArgs a = a_in;  // unset (zero) schedule fields take the defaults
    if (a.grain <= 0) a.grain = kDefaultCfg.grain;
    if (a.ccap <= 0 || a.ccap > CCAP) a.ccap = kDefaultCfg.ccap;
    if (a.variant == 1 && a.M <= kVariant1MaxM) return launch_tree_v<D, MODE, PREC, 256, 576, 2>(a, write_p0, st);
    if constexpr (PREC == 1) {
        // register-lean refined kernels: 20 warps in one CTA, or 3 CTAs of 8 warps
        if (a.variant == 2) return launch_tree_v<D, MODE, PREC, 640, XCAP, 1>(a, write_p0, st);
        if (a.variant == 3 && a.M <= kVariant1MaxM) return launch_tree_v<D, MODE, PREC, 256, 576, 3>(a, write_p0, st);
    }
    return launch_tree_v<D, MODE, PREC, TREE_THREADS, XCAP, 1>(a, write_p0, st);
}

template <int MODE>
static cudaError_t launch_mode(const FwdArgs &a, cudaStream_t st) {
    const int M = a.M;
    auto wp = [&](int d) { return MODE == MODE_P0 || d < a.kmax; };
    auto mark = [&](int i) {
        if (a.ev) cudaEventRecord(a.ev[i], st);
    };
    cudaError_t e = cudaSuccess;
    order1_kernel<MODE><<<(M + FLAT_THREADS - 1) / FLAT_THREADS, FLAT_THREADS, 0, st>>>(a, wp(1));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(2);
    if (a.kmax >= 2) {
        const uint64_t n2 = binom2(M);
        order2_kernel<MODE><<<(unsigned)((n2 + FLAT_THREADS - 1) / FLAT_THREADS), FLAT_THREADS, 0, st>>>(a, wp(2));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(3);
    if (a.kmax >= 3) {
        const uint64_t n3 = binom(M, 3);
        order3_kernel<MODE><<<(unsigned)((n3 + FLAT_THREADS - 1) / FLAT_THREADS), FLAT_THREADS, 0, st>>>(a, wp(3));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(4);
    if (a.kmax >= 4) {
        e = a.precision == 0 ? launch_tree<4, MODE, 0>(a, wp(4), st) : launch_tree<4, MODE, 1>(a, wp(4), st);
        if (e != cudaSuccess) return e;
    }
    mark(5);
    if (a.kmax >= 5) {
        e = a.precision == 0 ? launch_tree<5, MODE, 0>(a, wp(5), st) : launch_tree<5, MODE, 1>(a, wp(5), st);
        if (e != cudaSuccess) return e;
    }
    mark(6);
    return cudaSuccess;
}

cudaError_t launch_forward(const FwdArgs &a, cudaStream_t st) {
    const int M = a.M;
    if (a.ev) cudaEventRecord(a.ev[0], st);
    pack_kernel<<<(M * M + FLAT_THREADS - 1) / FLAT_THREADS, FLAT_THREADS, 0, st>>>(
        a.V, M, a.A, a.precision == 1 ? a.Af : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.ev) cudaEventRecord(a.ev[1], st);
    switch (a.mode) {
        case MODE_P0: return launch_mode<MODE_P0>(a, st);
        case MODE_MU: return launch_mode<MODE_MU>(a, st);
        case MODE_SPINC: return launch_mode<MODE_SPINC>(a, st);
        case MODE_SPINK: return launch_mode<MODE_SPINK>(a, st);
        default: return launch_mode<MODE_KAPPA>(a, st);
    }
}

}  // namespace gbs
