// Ragged batches: click-cumulant tables of many instances (different M and kmax)
// in one persistent cooperative launch.
//
// gbs_batched_plan() lays the batch out in the caller's workspace from host-side
// descriptors (instance order sorted by decreasing M, per-phase prefix sums of
// work units, per-instance packed blocks and lower-order P0 tables, the c4
// prefix tables of the tree phases) for one schedule: CTA shape, items per CTA
// slot (grain) and children per shared-memory batch. The schedule comes from the
// batch autotuner's table when this batch shape has been tuned
// (gbs_batched_autotune), else from a default. gbs_cumulants_batched() then
// queues a single kernel that runs six phases separated by grid-wide barriers:
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
#include <map>
#include <mutex>
#include <vector>

#include "gbs_batch.cuh"
#include "gbs_tree.cuh"
#include "gbs_tune.cuh"

namespace cg = cooperative_groups;

namespace gbs {

namespace {

constexpr int NPHASE = 6;
constexpr unsigned PLAN_MAGIC = 0x67627332u;

struct InstDev {
    const double *V;
    double *out;
    double *A;
    float *p0f;  // P0({x}) as float pairs (refined path)
    double *p0;
    int M, kmax;
    uint32_t c4off[2];   // offsets into the c4-prefix pool for orders 4 and 5
    uint64_t target[2];  // leaves per tree item for orders 4 and 5
};

struct PlanHdr {
    unsigned magic;
    int n, precision, maxM;
    int nt, xc, grid, ccap;  // schedule: threads per CTA, x-entry capacity, CTAs, children per batch
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
    size_t scratch_off = 0, total = 0;
};

template <int D>
uint32_t items_d(int M, int c4, uint64_t target) {
    return items_for_c4<D>(M, c4, target);
}

int max_m(const gbs_instance *in, int n) {
    int maxM = 1;
    for (int i = 0; i < n; ++i) maxM = std::max(maxM, in[i].M);
    return maxM;
}

// Builds the plan for a schedule (grain, ccap) and a launch of grid CTAs of the
// shape (nt, xc); pointers inside InstDev are relative to base (nullptr base =
// sizes only). The scratch area holds slots_per_sm_for(maxM) slots per
// multiprocessor, enough for every CTA shape the batch allows.
void build_plan(const gbs_instance *in, int n, int precision, int sms, int grid, int nt, int xc, int grain, int ccap,
                char *base, HostPlan &hp) {
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return in[x].M > in[y].M; });
    const int maxM = max_m(in, n);
    hp.hdr.magic = PLAN_MAGIC;
    hp.hdr.n = n;
    hp.hdr.precision = precision;
    hp.hdr.maxM = maxM;
    hp.hdr.nt = nt;
    hp.hdr.xc = xc;
    hp.hdr.grid = grid;
    hp.hdr.ccap = ccap;
    hp.hdr.slot_doubles = 4 * ((size_t)binom2(maxM) + (size_t)maxM);
    // per-phase units and targets: leaves per item so that each CTA gets about
    // grain items of each tree order
    uint64_t leaves[2] = {0, 0};
    for (int i = 0; i < n; ++i)
        for (int d = 4; d <= 5; ++d)
            if (in[i].kmax >= d) leaves[d - 4] += binom(in[i].M, d);
    uint64_t target[2];
    for (int q = 0; q < 2; ++q) {
        target[q] = leaves[q] / ((uint64_t)(grain > 0 ? grain : 1) * (uint64_t)(grid > 0 ? grid : 1));
        if (target[q] < 256) target[q] = 256;
    }
    hp.inst.resize(n);
    hp.pref.assign((size_t)NPHASE * (n + 1), 0);
    hp.pool.clear();
    // memory: status/counters (256 B), header, then instances, prefix sums, pool, A, p0, scratch
    size_t off = 256;
    off = a256(off + sizeof(PlanHdr));
    hp.hdr.inst_off = off;
    off = a256(off + sizeof(InstDev) * n);
    hp.hdr.pref_off = off;
    off = a256(off + sizeof(uint64_t) * NPHASE * (n + 1));
    // pool size: per instance and tree order, M + 1 entries
    size_t pool_n = 0;
    for (int i = 0; i < n; ++i)
        for (int d = 4; d <= 5; ++d)
            if (in[i].kmax >= d) pool_n += (size_t)(in[i].M + 1);
    hp.hdr.pool_off = off;
    off = a256(off + sizeof(uint32_t) * pool_n);
    for (int r = 0; r < n; ++r) {
        const gbs_instance &x = in[order[r]];
        InstDev &I = hp.inst[r];
        I.V = x.V;
        I.out = x.kappa_out;
        I.M = x.M;
        I.kmax = x.kmax;
        I.A = reinterpret_cast<double *>(base + off);  // FP64 blocks, then the float-pair copy
        off = a256(off + 2 * sizeof(double) * 4 * (size_t)x.M * x.M);
        I.p0f = reinterpret_cast<float *>(base + off);
        off = a256(off + 2 * sizeof(float) * (size_t)x.M);
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
    off = a256(off + sizeof(double) * hp.hdr.slot_doubles * (size_t)slots_per_sm_for(maxM) * (size_t)(sms > 0 ? sms : 1));
    hp.total = off;
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
    a.p0f = I.p0f;
    a.p0 = I.p0;
    a.out = I.out;
    a.status = status;
    a.scratch = scratch;
    a.slot_doubles = slot_doubles;
    return a;
}

template <int D, int PREC, int NT, int XC>
__device__ void tree_phase(const PlanHdr &h, const InstDev *inst, const uint64_t *pref, const uint32_t *pool,
                           unsigned *status, unsigned *counters, double *slot, unsigned char *smem) {
    TreeShared<D, XC> &sh = *reinterpret_cast<TreeShared<D, XC> *>(smem);
    __shared__ int s_dec[6];
    __shared__ FwdArgs s_args;
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
                s_args = inst_args(I, status, nullptr, h.slot_doubles, PREC);
            }
        }
        __syncthreads();
        const int i = s_dec[0];
        const int c4 = s_dec[1], c5 = s_dec[2], s = s_dec[3], nc = s_dec[4];
        __syncthreads();
        if (i < 0) break;
        tree_item<D, MODE_KAPPA, PREC, NT, XC>(s_args, sh, slot, c4, c5, s, nc, D < GBS_MAX_ORDER && D < s_args.kmax,
                                               h.ccap);
    }
}

// The batched kernel for one CTA shape: NT threads, XC x-entries of shared
// memory, at least MINB resident CTAs per multiprocessor.
template <int PREC, int NT, int XC, int MINB>
__global__ void __launch_bounds__(NT, MINB) batched_kernel(char *ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::grid_group grid = cg::this_grid();
    unsigned *status = reinterpret_cast<unsigned *>(ws);
    unsigned *counters = status + 8;
    const PlanHdr &h = *reinterpret_cast<const PlanHdr *>(ws + 256);
    // a plan made for another kernel or grid is refused before any barrier (the
    // test is uniform across the grid, so every CTA returns)
    if (h.magic != PLAN_MAGIC || h.precision != PREC || h.nt != NT || h.xc != XC || h.grid != (int)gridDim.x ||
        h.maxM > (XC < GBS_MAX_MODES ? XC + 1 : GBS_MAX_MODES) || h.ccap < 1 || h.ccap > CCAP) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(status, ST_BAD_INDEX);
        return;
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
    tree_phase<4, PREC, NT, XC>(h, inst, pref, pool, status, counters, slot, smem_raw);
    grid.sync();
    tree_phase<5, PREC, NT, XC>(h, inst, pref, pool, status, counters, slot, smem_raw);
}

// Kernel of one CTA shape (variant numbering as for the single-instance
// schedules: 0 = 512 x 1, 1 = 256 x 2, refined only 2 = 640 x 1, 3 = 256 x 3,
// 4 = 768 x 1 with a 2048-entry x area, 5 = 384 x 2 with a 960-entry x area,
// 6 = 256 x 4 with a 384-entry x area).
struct KernelInfo {
    void *fn;
    int nt, xc;
    size_t smem;
};

template <int PREC, int NT, int XC, int MINB>
KernelInfo kinfo() {
    return KernelInfo{(void *)batched_kernel<PREC, NT, XC, MINB>, NT, XC, sizeof(TreeShared<5, XC>)};
}

bool variant_ok(int precision, int variant, int maxM) {
    if (variant < 0 || variant >= kNumVariants || variant_clustered(variant) || variant == 9) return false;
    if (precision == 0 && variant >= 2) return false;
    if ((variant == 1 || variant == 3) && maxM > kVariant1MaxM) return false;
    if (variant == 5 && maxM > kVariant5MaxM) return false;
    if (variant == 6 && maxM > kVariant6MaxM) return false;
    return true;
}

KernelInfo kernel_for(int precision, int variant) {
    if (precision == 0) return variant == 1 ? kinfo<0, 256, 576, 2>() : kinfo<0, TREE_THREADS, XCAP, 1>();
    switch (variant) {
        case 1: return kinfo<1, 256, 576, 2>();
        case 2: return kinfo<1, 640, XCAP, 1>();
        case 3: return kinfo<1, 256, 576, 3>();
        case 4: return kinfo<1, 768, kWideXC, 1>();
        case 5: return kinfo<1, 384, kPairXC, 2>();
        case 6: return kinfo<1, 256, kQuadXC, 4>();
        default: return kinfo<1, TREE_THREADS, XCAP, 1>();
    }
}

// Co-resident CTAs of a shape on this device (cooperative launch), at most
// slots_per_sm per multiprocessor.
cudaError_t grid_for(const KernelInfo &k, int sms, int slots_per_sm, int &grid) {
    cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.nt, k.smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    grid = sms * std::min(per_sm, slots_per_sm);
    return cudaSuccess;
}

// Schedule each planned workspace was written for (the launch needs the shape
// and grid on the host; the kernel checks them against the plan's header).
struct Launch {
    int precision, variant, grid, grain, ccap;
};
std::mutex g_mu;
std::map<const void *, Launch> g_launch;

// Default schedule of an untuned batch: the CTA shape the single-instance
// autotuner picks for large tables on GB300 (256 x 3 refined, 256 x 2 FP64)
// where every instance fits it.
TreeCfg default_cfg(int precision, int maxM) {
    TreeCfg c = kDefaultCfg;
    if (maxM <= kVariant1MaxM) c.variant = precision == 1 ? 3 : 1;
    return c;
}

int write_plan(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms, const TreeCfg &cfg,
               cudaStream_t st, size_t &needed) {
    const KernelInfo k = kernel_for(precision, cfg.variant);
    int grid = 0;
    if (grid_for(k, sms, slots_per_sm_for(max_m(inst, n)), grid) != cudaSuccess) return GBS_ERR_CUDA;
    HostPlan hp;
    build_plan(inst, n, precision, sms, grid, k.nt, k.xc, cfg.grain, cfg.ccap, ws, hp);
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
    if (e != cudaSuccess) return GBS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    g_launch[ws] = Launch{precision, cfg.variant, grid, cfg.grain, cfg.ccap};
    return GBS_OK;
}

}  // namespace

size_t batched_workspace_bytes(const gbs_instance *inst, int n, int precision, int sms) {
    HostPlan hp;
    build_plan(inst, n, precision, sms, sms * slots_per_sm_for(max_m(inst, n)), TREE_THREADS, XCAP, kDefaultCfg.grain,
               kDefaultCfg.ccap,
               nullptr, hp);
    return hp.total;
}

int batched_plan(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms,
                 cudaStream_t st, size_t &needed) {
    const int maxM = max_m(inst, n);
    TreeCfg cfg = default_cfg(precision, maxM);
    TreeCfg tuned;
    if (tuned_batch_cfg(sms, inst, n, precision, tuned) && variant_ok(precision, tuned.variant, maxM)) cfg = tuned;
    return write_plan(inst, n, precision, ws, ws_bytes, sms, cfg, st, needed);
}

cudaError_t launch_batched(char *ws, int precision, cudaStream_t st, bool &planned) {
    Launch L{};
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_launch.find(ws);
        planned = it != g_launch.end() && it->second.precision == precision;
        if (!planned) return cudaSuccess;
        L = it->second;
    }
    cudaError_t e = cudaMemsetAsync(ws, 0, 128, st);  // status word and counters; keeps the scratch offset
    if (e != cudaSuccess) return e;
    const KernelInfo k = kernel_for(precision, L.variant);
    if ((e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem)) != cudaSuccess)
        return e;
    void *args[] = {&ws};
    return cudaLaunchCooperativeKernel(k.fn, dim3(L.grid), dim3(k.nt), args, k.smem, st);
}

bool batched_schedule(const void *ws, int *out5) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_launch.find(ws);
    if (it == g_launch.end()) return false;
    const Launch &L = it->second;
    const KernelInfo k = kernel_for(L.precision, L.variant);
    out5[0] = L.variant;
    out5[1] = k.nt;
    out5[2] = L.grid;
    out5[3] = L.grain;
    out5[4] = L.ccap;
    return true;
}

int batched_autotune(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms,
                     cudaStream_t st, TreeCfg &best, float &best_ms, int &tried) {
    const int maxM = max_m(inst, n);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GBS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GBS_ERR_CUDA;
    }
    best_ms = 1e30f;
    best = default_cfg(precision, maxM);
    tried = 0;
    int rc = GBS_OK;
    // times one schedule: plan, one untimed launch, one timed launch
    auto time_cfg = [&](const TreeCfg &c) {
        size_t needed = 0;
        rc = write_plan(inst, n, precision, ws, ws_bytes, sms, c, st, needed);
        if (rc != GBS_OK) return;
        bool planned = false;
        for (int rep = 0; rep < 2 && rc == GBS_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            if (launch_batched(ws, precision, st, planned) != cudaSuccess || !planned) rc = GBS_ERR_CUDA;
            if (rep == 1) cudaEventRecord(e1, st);
        }
        if (rc != GBS_OK) return;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = GBS_ERR_CUDA;
            return;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ++tried;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    // coordinate search: the CTA shape at the default grain and batch size, then
    // grain x children per batch for the fastest shape
    for (int v = 0; v < kNumVariants && rc == GBS_OK; ++v)
        if (variant_ok(precision, v, maxM)) time_cfg(TreeCfg{kDefaultCfg.grain, kDefaultCfg.ccap, v});
    const int vbest = best.variant;
    for (int grain : {1, 2, 4, 8})
        for (int ccap : {16, 64}) {
            if (rc != GBS_OK) break;
            if (grain == kDefaultCfg.grain && ccap == kDefaultCfg.ccap) continue;
            time_cfg(TreeCfg{grain, ccap, vbest});
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GBS_OK) return rc;
    record_batch_cfg(sms, inst, n, precision, best, best_ms);
    size_t needed = 0;
    return write_plan(inst, n, precision, ws, ws_bytes, sms, best, st, needed);
}

}  // namespace gbs
