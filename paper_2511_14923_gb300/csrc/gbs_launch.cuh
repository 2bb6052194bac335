// Launch plumbing of the forward kernels, shared by the zero-mean translation
// unit (gbs_fwd.cu) and the displaced-state one (gbs_disp.cu): the per-order
// kernels, the persistent prefix-tree kernel and its launcher, each templated on
// DISP (first moments carried through the elimination, FP64 only).
#pragma once
#include "gbs_tree.cuh"

namespace gbs {

// Flat kernels of orders 1-3: one thread per subset of colex rank first + i,
// i < count (the whole order, or the rank range of a range call's top order).
template <int MODE, bool DISP>
__global__ void order1_kernel(FwdArgs a, bool write_p0, uint64_t first, uint64_t count) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) order1_entry<MODE, DISP>(a, (int)(first + i), write_p0);
}

template <int MODE, bool DISP>
__global__ void order2_kernel(FwdArgs a, bool write_p0, uint64_t first, uint64_t count) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) order2_entry<MODE, DISP>(a, (uint32_t)(first + i), write_p0);
}

template <int MODE, bool DISP>
__global__ void order3_kernel(FwdArgs a, bool write_p0, uint64_t first, uint64_t count) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) order3_entry<MODE, DISP>(a, first + i, write_p0);
}

template <int D, int MODE, int PREC, int NT, int XC, int MINB, bool DISP, int CC = CCAP, int YC = 0>
__global__ void __launch_bounds__(NT, MINB) tree_kernel(FwdArgs a, uint64_t target, bool write_p0) {
    using SH = TreeShared<D, XC, DISP, CC, YC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = *reinterpret_cast<SH *>(smem_raw);
    const int tid = threadIdx.x;
    const int M = a.M;
    // top elements covered: all, or [c_lo, c_hi) for the top order of a range call
    const bool ranged = a.top != nullptr && D == a.kmax;
    const int tlo = ranged ? a.c_lo : 0, thi = ranged ? a.c_hi : M;
    const int c4hi = c4_max<D>(M, thi);
    const int K = c4hi - 2 > 0 ? c4hi - 2 : 0;  // c4 runs c4hi, c4hi-1, .., 3
    double *const slot = a.scratch + (size_t)blockIdx.x * a.slot_doubles;

    // prefix of item counts over c4 in descending order (warp 0, chunked scan)
    if (tid < 32) {
        const int per = (K + 31) / 32;
        const int lo = tid * per, hi = min(K, lo + per);
        uint32_t sum = 0;
        for (int k = lo; k < hi; ++k) sum += items_for_c4<D>(M, c4hi - k, target, tlo, thi);
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += v;
        }
        uint32_t run = incl - sum;
        for (int k = lo; k < hi; ++k) {
            sh.c4pref[k] = run;
            run += items_for_c4<D>(M, c4hi - k, target, tlo, thi);
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
        const int c5 = (D == 5) ? c5_first(c4, tlo) + u : M;
        tree_item<D, MODE, PREC, NT, XC, DISP, false, CC, YC>(a, sh, slot, c4, c5, s, nc, write_p0, a.ccap);
    }
}

// The same walk with thread-block clusters of CS CTAs: a cluster takes one U at a
// time (its item), its CTAs build the Schur complement into the cluster's one
// slot together and then take one stride class of the children each. Rank 0
// draws the item and the others read it from its shared memory; three cluster
// barriers per item (item drawn, slot built, slot released) keep every CTA of a
// cluster on the same item sequence. One slot per cluster instead of one per
// CTA: the slots' L2 footprint and the build work both shrink by CS.
template <int D, int MODE, int PREC, int NT, int XC, int MINB, int CS>
__global__ void __launch_bounds__(NT, MINB) tree_kernel_cl(FwdArgs a, bool write_p0) {
    using SH = TreeShared<D, XC, false>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = *reinterpret_cast<SH *>(smem_raw);
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int M = a.M;
    const bool ranged = a.top != nullptr && D == a.kmax;
    const int tlo = ranged ? a.c_lo : 0, thi = ranged ? a.c_hi : M;
    const int c4hi = c4_max<D>(M, thi);
    const int K = c4hi - 2 > 0 ? c4hi - 2 : 0;
    constexpr uint64_t kWhole = 1ull << 62;  // leaves per item: one item per U
    double *const slot = a.scratch + (size_t)(blockIdx.x / CS) * a.slot_doubles;
    if (tid < 32) {
        const int per = (K + 31) / 32;
        const int lo = tid * per, hi = min(K, lo + per);
        uint32_t sum = 0;
        for (int k = lo; k < hi; ++k) sum += items_for_c4<D>(M, c4hi - k, kWhole, tlo, thi);
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += v;
        }
        uint32_t run = incl - sum;
        for (int k = lo; k < hi; ++k) {
            sh.c4pref[k] = run;
            run += items_for_c4<D>(M, c4hi - k, kWhole, tlo, thi);
        }
        if (tid == 31) sh.c4pref[K] = incl;
    }
    __syncthreads();
    const uint32_t total_items = sh.c4pref[K];
    uint32_t *item0 = cluster.map_shared_rank(&sh.item, 0);
    __shared__ uint32_t s_item;
    for (;;) {
        if (rank == 0 && tid == 0) sh.item = atomicAdd(a.counters + D, 1u);
        cluster.sync();  // the item is in rank 0's shared memory
        if (tid == 0) s_item = *item0;
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= total_items) {
            // every CTA of the cluster reads the same item, so all arrive here; no CTA
            // leaves while another may still read rank 0's item word
            cluster.sync();
            break;
        }
        int lo = 0, hi = K;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sh.c4pref[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int c4 = c4hi - lo;
        const int u = (int)(item - sh.c4pref[lo]);
        const int c5 = (D == 5) ? c5_first(c4, tlo) + u : M;
        tree_item<D, MODE, PREC, NT, XC, false, true>(a, sh, slot, c4, c5, rank, CS, write_p0, a.ccap, rank, CS);
        cluster.sync();  // every CTA is done with the slot (and with rank 0's item word)
    }
}

// ---------------------------------------------------------------- launchers

template <int D, int MODE, int PREC, int NT, int XC, int MINB, int CS>
static cudaError_t launch_tree_cl(const FwdArgs &a, bool write_p0, cudaStream_t st) {
    const int M = a.M;
    const bool ranged = a.top != nullptr && D == a.kmax;
    const int tlo = ranged ? a.c_lo : 0, thi = ranged ? a.c_hi : M;
    if (binom(thi, D) - binom(tlo, D) == 0) return cudaSuccess;
    const size_t smem = sizeof(TreeShared<D, XC, false>);
    auto fn = tree_kernel_cl<D, MODE, PREC, NT, XC, MINB, CS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(CS * a.sms);
    int clusters = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, (void *)fn, &cfg)) != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    if (clusters > a.slots) clusters = a.slots;
    uint64_t items = 0;
    for (int c4 = c4_max<D>(M, thi); c4 >= 3; --c4) items += items_for_c4<D>(M, c4, 1ull << 62, tlo, thi);
    if (items == 0) return cudaSuccess;
    if ((uint64_t)clusters > items) clusters = (int)items;
    cfg.gridDim = dim3(CS * clusters);
    e = cudaLaunchKernelEx(&cfg, fn, a, write_p0);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int D, int MODE, int PREC, int NT, int XC, int MINB, bool DISP, int CC = CCAP, int YC = 0>
static cudaError_t launch_tree_v(const FwdArgs &a, bool write_p0, cudaStream_t st) {
    const int M = a.M;
    const bool ranged = a.top != nullptr && D == a.kmax;
    const int tlo = ranged ? a.c_lo : 0, thi = ranged ? a.c_hi : M;
    const uint64_t leaves = binom(thi, D) - binom(tlo, D);
    if (leaves == 0) return cudaSuccess;
    const size_t smem = sizeof(TreeShared<D, XC, DISP, CC, YC>);
    auto fn = tree_kernel<D, MODE, PREC, NT, XC, MINB, DISP, CC, YC>;
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
    for (int c4 = c4_max<D>(M, thi); c4 >= 3; --c4) items += items_for_c4<D>(M, c4, target, tlo, thi);
    if (items == 0) return cudaSuccess;
    const int grid = (int)(items < (uint64_t)grid_max ? items : (uint64_t)grid_max);
    fn<<<grid, NT, smem, st>>>(a, target, write_p0);
    return cudaGetLastError();
}

template <int D, int MODE, int PREC, bool DISP>
static cudaError_t launch_tree(const FwdArgs &a_in, bool write_p0, cudaStream_t st) {
    FwdArgs a = a_in;  // unset (zero) schedule fields take the defaults
    if (a.grain <= 0) a.grain = kDefaultCfg.grain;
    if (a.ccap <= 0 || a.ccap > CCAP) a.ccap = kDefaultCfg.ccap;
    if constexpr (DISP) {
        // displaced states: FP64, one 512-thread CTA per multiprocessor
        return launch_tree_v<D, MODE, 0, TREE_THREADS, XCAP, 1, true>(a, write_p0, st);
    } else {
        const int v = effective_variant(a.variant, a.M, PREC);
        if (v == 1) return launch_tree_v<D, MODE, PREC, 256, 576, 2, false>(a, write_p0, st);
        if constexpr (PREC == 1) {
            // register-lean refined kernels: 20 warps in one CTA, 3 CTAs of 8 warps,
            // 24 warps in one CTA with room for about 3.5x more children per batch,
            // 2 CTAs of 12 warps with room for about 1.7x more, or 4 CTAs of 8 warps
            // (64 registers) with room for a third fewer
            if (v == 2) return launch_tree_v<D, MODE, PREC, 640, XCAP, 1, false>(a, write_p0, st);
            if (v == 3) return launch_tree_v<D, MODE, PREC, 256, 576, 3, false>(a, write_p0, st);
            if (v == 4) return launch_tree_v<D, MODE, PREC, 768, kWideXC, 1, false>(a, write_p0, st);
            if (v == 5) return launch_tree_v<D, MODE, PREC, 384, kPairXC, 2, false>(a, write_p0, st);
            if (v == 6) {
                // order 4 of the 256 x 4 shape runs without slots where it can: its items
                // are small (one U = {c4} split into many stride classes), so rebuilding
                // the slot per item cost more than forming the blocks in place (same bits)
                if (D == 4 && a.M <= kVariant9MaxM)
                    return launch_tree_v<D, MODE, PREC, 256, kQuadXC, 4, false, kNoSlotCC, kNoSlotYC>(a, write_p0, st);
                return launch_tree_v<D, MODE, PREC, 256, kQuadXC, 4, false>(a, write_p0, st);
            }
            // the 256 x 4 and 256 x 3 shapes in clusters that share one slot per U
            if (v == 7) return launch_tree_cl<D, MODE, PREC, 256, kQuadXC, 4, 4>(a, write_p0, st);
            if (v == 8) return launch_tree_cl<D, MODE, PREC, 256, 576, 3, 3>(a, write_p0, st);
            // 256 x 4 without slots: Schur-complement blocks formed from Y where used
            if (v == 9) return launch_tree_v<D, MODE, PREC, 256, kQuadXC, 4, false, kNoSlotCC, kNoSlotYC>(a, write_p0, st);
        }
        return launch_tree_v<D, MODE, PREC, TREE_THREADS, XCAP, 1, false>(a, write_p0, st);
    }
}

template <int MODE, bool DISP>
static cudaError_t launch_mode(const FwdArgs &a, cudaStream_t st) {
    const int M = a.M;
    auto wp = [&](int d) { return MODE == MODE_P0 || d < a.kmax; };
    auto mark = [&](int i) {
        if (a.ev) cudaEventRecord(a.ev[i], st);
    };
    // ranks of order d to fill: all, or those with top element in [c_lo, c_hi)
    // for the top order of a range call
    auto span = [&](int d, uint64_t &first, uint64_t &count) {
        if (a.top && d == a.kmax) {
            first = binom(a.c_lo, d);
            count = binom(a.c_hi, d) - first;
        } else {
            first = 0;
            count = binom(M, d);
        }
    };
    auto grid = [](uint64_t n) { return (unsigned)((n + FLAT_THREADS - 1) / FLAT_THREADS); };
    cudaError_t e = cudaSuccess;
    uint64_t f = 0, n = 0;
    span(1, f, n);
    if (n) order1_kernel<MODE, DISP><<<grid(n), FLAT_THREADS, 0, st>>>(a, wp(1), f, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(2);
    if (a.kmax >= 2) {
        span(2, f, n);
        if (n) order2_kernel<MODE, DISP><<<grid(n), FLAT_THREADS, 0, st>>>(a, wp(2), f, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(3);
    if (a.kmax >= 3) {
        span(3, f, n);
        if (n) order3_kernel<MODE, DISP><<<grid(n), FLAT_THREADS, 0, st>>>(a, wp(3), f, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(4);
    if (a.kmax >= 4) {
        e = a.precision == 0 ? launch_tree<4, MODE, 0, DISP>(a, wp(4), st) : launch_tree<4, MODE, 1, DISP>(a, wp(4), st);
        if (e != cudaSuccess) return e;
    }
    mark(5);
    if (a.kmax >= 5) {
        e = a.precision == 0 ? launch_tree<5, MODE, 0, DISP>(a, wp(5), st) : launch_tree<5, MODE, 1, DISP>(a, wp(5), st);
        if (e != cudaSuccess) return e;
    }
    mark(6);
    return cudaSuccess;
}

// Queues the per-order kernels (orders 1..kmax) of one forward call after packing.
template <bool DISP>
cudaError_t launch_orders(const FwdArgs &a, cudaStream_t st) {
    switch (a.mode) {
        case MODE_P0: return launch_mode<MODE_P0, DISP>(a, st);
        case MODE_MU: return launch_mode<MODE_MU, DISP>(a, st);
        case MODE_SPINC: return launch_mode<MODE_SPINC, DISP>(a, st);
        case MODE_SPINK: return launch_mode<MODE_SPINK, DISP>(a, st);
        default: return launch_mode<MODE_KAPPA, DISP>(a, st);
    }
}

}  // namespace gbs
