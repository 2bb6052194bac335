// Ragged batches: click-cumulant tables of many instances (different M and kmax)
// in one persistent cooperative launch.
//
// gbs_batched_plan() lays the batch out in the caller's workspace from host-side
// descriptors (instance order sorted by decreasing M, per-phase prefix sums of
// work units, per-instance packed blocks and lower-order P0 tables, the c4
// prefix tables of the tree phases). gbs_cumulants_batched() then queues a single
// kernel that runs six phases separated by grid-wide barriers:
//   0 packing of every instance's (V + I)/2 into 2x2 blocks,
//   1-3 orders 1..3, one work unit per subset (grid-stride over all instances),
//   4-5 orders 4 and 5, prefix-tree items of all instances pulled from one
//       atomic queue per order (largest instances first).
// The launch reads everything from the workspace, so it can be captured in a
// CUDA graph once the plan is written, and replayed after V changes in place.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gbs_batch.cuh"
#include "gbs_tree.cuh"

namespace cg = cooperative_groups;

namespace gbs {

namespace {

constexpr int NPHASE = 6;
constexpr unsigned PLAN_MAGIC = 0x67627331u;

struct InstDev {
    const double *V;
    double *out;
    double *A;
    double *p0;
    int M, kmax;
    uint32_t c4off[2];   // offsets into the c4-prefix pool for orders 4 and 5
    uint64_t target[2];  // leaves per tree item for orders 4 and 5
};

struct PlanHdr {
    unsigned magic;
    int n, precision, maxM;
    size_t slot_doubles;
    size_t inst_off, pref_off, pool_off;  // byte offsets from the workspace base
    uint64_t total[NPHASE];
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct HostPlan {
    PlanHdr hdr{};
    std::vector<InstDev> inst;
    std::vector<uint64_t> pref;  // NPHASE x (n + 1)
    std::vector<uint32_t> pool;
    size_t A_off = 0, p0_off = 0, scratch_off = 0, total = 0;
};

template <int D>
uint32_t items_d(int M, int c4, uint64_t target) {
    return items_for_c4<D>(M, c4, target);
}

// Builds the plan; pointers inside InstDev are relative to base (nullptr base = sizes only).
int build_plan(const gbs_instance *in, int n, int precision, int grid, char *base, HostPlan &hp) {
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return in[x].M > in[y].M; });
    int maxM = 1;
    for (int i = 0; i < n; ++i) maxM = std::max(maxM, in[i].M);
    hp.hdr.magic = PLAN_MAGIC;
    hp.hdr.n = n;
    hp.hdr.precision = precision;
    hp.hdr.maxM = maxM;
    hp.hdr.slot_doubles = 4 * ((size_t)binom2(maxM) + (size_t)maxM);
    // per-phase units and targets
    uint64_t leaves[2] = {0, 0};
    for (int i = 0; i < n; ++i)
        for (int d = 4; d <= 5; ++d)
            if (in[i].kmax >= d) leaves[d - 4] += binom(in[i].M, d);
    uint64_t target[2];
    for (int q = 0; q < 2; ++q) {
        target[q] = leaves[q] / (2 * (uint64_t)grid);
        if (target[q] < 256) target[q] = 256;
    }
    hp.inst.resize(n);
    hp.pref.assign((size_t)NPHASE * (n + 1), 0);
    hp.pool.clear();
    // memory: header+plan, then A, p0, scratch
    size_t off = 256;  // status word and counters
    const size_t hdr_off = off;
    off = a256(off + sizeof(PlanHdr));
    hp.hdr.inst_off = off;
    off = a256(off + sizeof(InstDev) * n);
    hp.hdr.pref_off = off;
    off = a256(off + sizeof(uint64_t) * NPHASE * (n + 1));
    // pool size: per instance and tree order, K + 1 entries
    size_t pool_n = 0;
    for (int i = 0; i < n; ++i)
        for (int d = 4; d <= 5; ++d)
            if (in[i].kmax >= d) pool_n += (size_t)(in[i].M + 1);
    hp.hdr.pool_off = off;
    off = a256(off + sizeof(uint32_t) * pool_n);
    (void)hdr_off;
    for (int r = 0; r < n; ++r) {
        const gbs_instance &x = in[order[r]];
        InstDev &I = hp.inst[r];
        I.V = x.V;
        I.out = x.kappa_out;
        I.M = x.M;
        I.kmax = x.kmax;
        I.A = reinterpret_cast<double *>(base + off);  // FP64 blocks, then the float-pair copy
        off = a256(off + 2 * sizeof(double) * 4 * (size_t)x.M * x.M);
        I.p0 = reinterpret_cast<double *>(base + off);
        off = a256(off + sizeof(double) * (x.kmax > 1 ? order_offset(x.M, x.kmax) : 0));
        for (int d = 4; d <= 5; ++d) {
            I.target[d - 4] = target[d - 4];
            I.c4off[d - 4] = (uint32_t)hp.pool.size();
            if (x.kmax < d) continue;
            const int c4hi = d == 5 ? x.M - 2 : x.M - 1;
            const int K = std::max(c4hi - 2, 0);
            uint32_t run = 0;
            for (int k = 0; k < K; ++k) {
                hp.pool.push_back(run);
                run += d == 5 ? items_d<5>(x.M, c4hi - k, target[1]) : items_d<4>(x.M, c4hi - k, target[0]);
            }
            hp.pool.push_back(run);
            // pad to M + 1 entries so offsets stay predictable
            while (hp.pool.size() < I.c4off[d - 4] + (size_t)(x.M + 1)) hp.pool.push_back(run);
        }
        uint64_t units[NPHASE] = {(uint64_t)x.M * x.M, binom(x.M, 1), x.kmax >= 2 ? binom2(x.M) : 0,
                                  x.kmax >= 3 ? binom(x.M, 3) : 0, 0, 0};
        for (int d = 4; d <= 5; ++d)
            if (x.kmax >= d) units[d] = hp.pool[I.c4off[d - 4] + std::max((d == 5 ? x.M - 2 : x.M - 1) - 2, 0)];
        for (int ph = 0; ph < NPHASE; ++ph) hp.pref[(size_t)ph * (n + 1) + r + 1] = hp.pref[(size_t)ph * (n + 1) + r] + units[ph];
    }
    for (int ph = 0; ph < NPHASE; ++ph) hp.hdr.total[ph] = hp.pref[(size_t)ph * (n + 1) + n];
    hp.scratch_off = off;
    off = a256(off + sizeof(double) * hp.hdr.slot_doubles * grid);
    hp.total = off;
    return GBS_OK;
}

__device__ __forceinline__ int find_inst(const uint64_t *pref, int n, uint64_t u) {
    int lo = 0, hi = n;  // pref[lo] <= u < pref[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pref[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ FwdArgs inst_args(const InstDev &I, unsigned *status, double *scratch, size_t slot_doubles,
                                             int precision) {
    FwdArgs a{};
    a.V = I.V;
    a.M = I.M;
    a.kmax = I.kmax;
    a.mode = MODE_KAPPA;
    a.precision = precision;
    a.A = I.A;
    a.Af = reinterpret_cast<float *>(I.A + 4 * (size_t)I.M * I.M);
    a.p0 = I.p0;
    a.out = I.out;
    a.status = status;
    a.scratch = scratch;
    a.slot_doubles = slot_doubles;
    return a;
}

template <int D, int PREC>
__device__ void tree_phase(char *ws, const PlanHdr &h, const InstDev *inst, const uint64_t *pref, const uint32_t *pool,
                           unsigned *status, unsigned *counters, double *slot, unsigned char *smem) {
    TreeShared<D> &sh = *reinterpret_cast<TreeShared<D> *>(smem);
    __shared__ int s_dec[6];
    const int n = h.n;
    const uint64_t *pf = pref + (size_t)D * (n + 1);
    const uint64_t total = h.total[D];
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t item = atomicAdd(counters + D, 1u);
            s_dec[0] = -1;
            if (item < total) {
                const int i = find_inst(pf, n, item);
                const InstDev &I = inst[i];
                const uint32_t local = (uint32_t)(item - pf[i]);
                const uint32_t *c4p = pool + I.c4off[D - 4];
                const int c4hi = D == 5 ? I.M - 2 : I.M - 1;
                const int K = c4hi - 2;
                int lo = 0, hi = K;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (c4p[mid] <= local) lo = mid;
                    else hi = mid;
                }
                const int c4 = c4hi - lo;
                const int nc = n_classes(c4, I.target[D - 4]);
                const uint32_t rr = local - c4p[lo];
                s_dec[0] = i;
                s_dec[1] = c4;
                s_dec[2] = D == 5 ? c4 + 1 + (int)(rr / nc) : I.M;
                s_dec[3] = (int)(rr % nc);
                s_dec[4] = nc;
            }
        }
        __syncthreads();
        const int i = s_dec[0];
        const int c4 = s_dec[1], c5 = s_dec[2], s = s_dec[3], nc = s_dec[4];
        __syncthreads();
        if (i < 0) break;
        const InstDev &I = inst[i];
        const FwdArgs a = inst_args(I, status, nullptr, h.slot_doubles, PREC);
        tree_item<D, MODE_KAPPA, PREC, TREE_THREADS, XCAP>(a, sh, slot, c4, c5, s, nc, D < I.kmax, CCAP);
    }
}

template <int PREC>
__global__ void __launch_bounds__(TREE_THREADS, 1) batched_kernel(char *ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::grid_group grid = cg::this_grid();
    unsigned *status = reinterpret_cast<unsigned *>(ws);
    unsigned *counters = status + 8;
    const PlanHdr &h = *reinterpret_cast<const PlanHdr *>(ws + 256);
    if (h.magic != PLAN_MAGIC || h.precision != PREC) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(status, ST_BAD_INDEX);
        return;  // uniform across the grid: no barrier is reached
    }
    const int n = h.n;
    const InstDev *inst = reinterpret_cast<const InstDev *>(ws + h.inst_off);
    const uint64_t *pref = reinterpret_cast<const uint64_t *>(ws + h.pref_off);
    const uint32_t *pool = reinterpret_cast<const uint32_t *>(ws + h.pool_off);
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;

    // phase 0: packing
    for (uint64_t u = gtid; u < h.total[0]; u += nthr) {
        const int i = find_inst(pref, n, u);
        pack_entry(inst[i].V, inst[i].M, inst[i].A,
                   PREC == 1 ? reinterpret_cast<float *>(inst[i].A + 4 * (size_t)inst[i].M * inst[i].M) : nullptr,
                   (int)(u - pref[i]));
    }
    grid.sync();
    // phases 1-3: orders 1..3
    for (uint64_t u = gtid; u < h.total[1]; u += nthr) {
        const int i = find_inst(pref + (n + 1), n, u);
        const FwdArgs a = inst_args(inst[i], status, nullptr, 0, PREC);
        order1_entry<MODE_KAPPA>(a, (int)(u - pref[(n + 1) + i]), 1 < a.kmax);
    }
    grid.sync();
    for (uint64_t u = gtid; u < h.total[2]; u += nthr) {
        const int i = find_inst(pref + 2 * (n + 1), n, u);
        const FwdArgs a = inst_args(inst[i], status, nullptr, 0, PREC);
        order2_entry<MODE_KAPPA>(a, (uint32_t)(u - pref[2 * (n + 1) + i]), 2 < a.kmax);
    }
    grid.sync();
    for (uint64_t u = gtid; u < h.total[3]; u += nthr) {
        const int i = find_inst(pref + 3 * (n + 1), n, u);
        const FwdArgs a = inst_args(inst[i], status, nullptr, 0, PREC);
        order3_entry<MODE_KAPPA>(a, u - pref[3 * (n + 1) + i], 3 < a.kmax);
    }
    grid.sync();
    double *slot = reinterpret_cast<double *>(ws + *reinterpret_cast<const size_t *>(ws + 128)) +
                   (size_t)blockIdx.x * h.slot_doubles;
    tree_phase<4, PREC>(ws, h, inst, pref, pool, status, counters, slot, smem_raw);
    grid.sync();
    tree_phase<5, PREC>(ws, h, inst, pref, pool, status, counters, slot, smem_raw);
}

}  // namespace

size_t batched_workspace_bytes(const gbs_instance *inst, int n, int precision, int sms) {
    HostPlan hp;
    build_plan(inst, n, precision, sms, nullptr, hp);
    return hp.total;
}

int batched_plan(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms,
                 cudaStream_t st, size_t &needed) {
    HostPlan hp;
    build_plan(inst, n, precision, sms, ws, hp);
    needed = hp.total;
    if (ws_bytes < hp.total) return GBS_ERR_WORKSPACE;
    // one contiguous host image of [0, pool end): status/counters zero, scratch offset at 128
    const size_t img = hp.hdr.pool_off + sizeof(uint32_t) * hp.pool.size();
    std::vector<char> buf(img, 0);
    const size_t scratch_off = hp.scratch_off;
    memcpy(buf.data() + 128, &scratch_off, sizeof scratch_off);
    memcpy(buf.data() + 256, &hp.hdr, sizeof hp.hdr);
    memcpy(buf.data() + hp.hdr.inst_off, hp.inst.data(), sizeof(InstDev) * hp.inst.size());
    memcpy(buf.data() + hp.hdr.pref_off, hp.pref.data(), sizeof(uint64_t) * hp.pref.size());
    if (!hp.pool.empty()) memcpy(buf.data() + hp.hdr.pool_off, hp.pool.data(), sizeof(uint32_t) * hp.pool.size());
    cudaError_t e = cudaMemcpyAsync(ws, buf.data(), img, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // buf is released on return
    return e == cudaSuccess ? GBS_OK : GBS_ERR_CUDA;
}

cudaError_t launch_batched(char *ws, int precision, int sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ws, 0, 128, st);  // status word and counters; keeps the scratch offset
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(TreeShared<5>);
    void *fn = precision == 0 ? (void *)batched_kernel<0> : (void *)batched_kernel<1>;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TREE_THREADS, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    void *args[] = {&ws};
    return cudaLaunchCooperativeKernel(fn, dim3(sms), dim3(TREE_THREADS), args, smem, st);
}

}  // namespace gbs
