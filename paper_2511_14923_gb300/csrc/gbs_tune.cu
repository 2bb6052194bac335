// Autotuner for the prefix-tree schedule.
//
// For one problem shape (device, M, kmax, precision) it times the cumulant
// forward pass under every candidate schedule and keeps the fastest:
//   grain   items per CTA slot (subtree granularity: 1, 2, 4, 8),
//   ccap    children per shared-memory batch (16 or 64),
//   variant CTA shape: 512 threads x 1 per SM; 256 x 2 per SM (M <= 577); and for
//           the refined path 640 x 1, 256 x 3 (M <= 577), 768 x 1 with room
//           for more children per batch, 384 x 2 (M <= 961), 256 x 4 (M <= 385),
//           256 x 4 / 256 x 3 in thread-block clusters sharing one slot, or
//           256 x 4 without slots (M <= 162).
// Results live in a process-wide table consulted by every forward call; if the
// environment variable GBS_AUTOTUNE_CACHE names a file, the table is loaded from
// it on first use and rewritten after each tuning run (a JSON array of objects).
// Ragged batches (gbs_batched_autotune) have a second table keyed by the batch's
// multiset of (M, kmax), hashed; its entries share the JSON file and carry a
// "batch" key instead of "M".
// The schedule changes only the order in which entries are computed, never their
// arithmetic, so tuned and untuned calls return identical tables.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gbs.h"
#include "gbs_common.cuh"
#include "gbs_fwd.cuh"
#include "gbs_tune.cuh"

namespace gbs {

namespace {

using Key = std::tuple<int, int, int, int, int>;  // cc, sms, M, kmax, precision
struct Entry {
    TreeCfg cfg;
    float ms;
};

using BKey = std::tuple<int, int, int, uint64_t>;  // cc, sms, precision, batch signature
struct BEntry {
    TreeCfg cfg;
    float ms;
    int n;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;
std::map<BKey, BEntry> g_btable;
bool g_loaded = false;

// FNV-1a over the (M, kmax) pairs in sorted order, then n: the batch's shape
// regardless of instance order.
uint64_t batch_signature(const gbs_instance *inst, int n) {
    std::vector<std::pair<int, int>> mk(n);
    for (int i = 0; i < n; ++i) mk[i] = {inst[i].M, inst[i].kmax};
    std::sort(mk.begin(), mk.end());
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint32_t v) {
        for (int b = 0; b < 4; ++b) {
            h ^= (v >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    for (const auto &p : mk) {
        mix((uint32_t)p.first);
        mix((uint32_t)p.second);
    }
    mix((uint32_t)n);
    return h;
}

int read_hex(const char *obj, const char *end, const char *key, uint64_t &out) {
    char pat[32];
    snprintf(pat, sizeof pat, "\"%s\"", key);
    const char *p = strstr(obj, pat);
    if (!p || p > end) return 0;
    p = strchr(p + strlen(pat), '"');
    if (!p || p > end) return 0;
    out = strtoull(p + 1, nullptr, 16);
    return 1;
}

int read_int(const char *obj, const char *end, const char *key, int &out) {
    char pat[32];
    snprintf(pat, sizeof pat, "\"%s\"", key);
    const char *p = strstr(obj, pat);
    if (!p || p > end) return 0;
    p = strchr(p + strlen(pat), ':');
    if (!p || p > end) return 0;
    out = (int)strtol(p + 1, nullptr, 10);
    return 1;
}

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("GBS_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "rb");
    if (!f) return;
    std::string txt;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, got);
    fclose(f);
    const char *p = txt.c_str();
    while ((p = strchr(p, '{')) != nullptr) {
        const char *end = strchr(p, '}');
        if (!end) break;
        int cc, sms, M, kmax, prec, grain, ccap, variant, nb;
        uint64_t sig;
        if (read_hex(p, end, "batch", sig)) {
            if (read_int(p, end, "cc", cc) && read_int(p, end, "sms", sms) && read_int(p, end, "precision", prec) &&
                read_int(p, end, "n", nb) && read_int(p, end, "grain", grain) && read_int(p, end, "ccap", ccap) &&
                read_int(p, end, "variant", variant) && grain >= 1 && grain <= 64 && ccap >= 1 && ccap <= 64 &&
                variant >= 0 && variant < kNumVariants)
                g_btable[BKey{cc, sms, prec, sig}] = BEntry{TreeCfg{grain, ccap, variant}, -1.f, nb};
        } else if (read_int(p, end, "cc", cc) && read_int(p, end, "sms", sms) && read_int(p, end, "M", M) &&
            read_int(p, end, "kmax", kmax) && read_int(p, end, "precision", prec) &&
            read_int(p, end, "grain", grain) && read_int(p, end, "ccap", ccap) &&
            read_int(p, end, "variant", variant) && grain >= 1 && grain <= 64 && ccap >= 1 && ccap <= 64 &&
            variant >= 0 && variant < kNumVariants) {
            g_table[Key{cc, sms, M, kmax, prec}] = Entry{TreeCfg{grain, ccap, variant}, -1.f};
        }
        p = end + 1;
    }
}

void save_locked() {
    const char *path = getenv("GBS_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    fprintf(f, "[\n");
    size_t i = 0;
    const size_t count = g_table.size() + g_btable.size();
    for (const auto &kv : g_btable) {
        const BKey &k = kv.first;
        const BEntry &e = kv.second;
        fprintf(f,
                "  {\"cc\": %d, \"sms\": %d, \"precision\": %d, \"batch\": \"%016llx\", \"n\": %d, \"grain\": %d, "
                "\"ccap\": %d, \"variant\": %d, \"ms\": %.4f}%s\n",
                std::get<0>(k), std::get<1>(k), std::get<2>(k), (unsigned long long)std::get<3>(k), e.n, e.cfg.grain,
                e.cfg.ccap, e.cfg.variant, e.ms, ++i < count ? "," : "");
    }
    for (const auto &kv : g_table) {
        const Key &k = kv.first;
        const Entry &e = kv.second;
        fprintf(f,
                "  {\"cc\": %d, \"sms\": %d, \"M\": %d, \"kmax\": %d, \"precision\": %d, \"grain\": %d, "
                "\"ccap\": %d, \"variant\": %d, \"ms\": %.4f}%s\n",
                std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), e.cfg.grain,
                e.cfg.ccap, e.cfg.variant, e.ms, ++i < count ? "," : "");
    }
    fprintf(f, "]\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

int device_cc() {
    int dev = 0, mj = 0, mn = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&mj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mn, cudaDevAttrComputeCapabilityMinor, dev);
    return 10 * mj + mn;
}

}  // namespace

TreeCfg tuned_cfg(int sms, int M, int kmax, int precision) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    auto it = g_table.find(Key{device_cc(), sms, M, kmax, precision});
    return it == g_table.end() ? kDefaultCfg : it->second.cfg;
}

bool tuned_batch_cfg(int sms, const gbs_instance *inst, int n, int precision, TreeCfg &cfg) {
    const uint64_t sig = batch_signature(inst, n);
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    auto it = g_btable.find(BKey{device_cc(), sms, precision, sig});
    if (it == g_btable.end()) return false;
    cfg = it->second.cfg;
    return true;
}

void record_batch_cfg(int sms, const gbs_instance *inst, int n, int precision, const TreeCfg &cfg, float ms) {
    const uint64_t sig = batch_signature(inst, n);
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    g_btable[BKey{device_cc(), sms, precision, sig}] = BEntry{cfg, ms, n};
    save_locked();
}

int autotune(FwdArgs a, cudaStream_t st, TreeCfg &best, float &best_ms, int &tried) {
    std::vector<TreeCfg> cand;
    for (int variant = 0; variant <= (a.precision == 1 ? kNumVariants - 1 : 1); ++variant) {
        if ((variant == 1 || variant == 3) && a.M > kVariant1MaxM) continue;
        if (variant == 5 && a.M > kVariant5MaxM) continue;
        if ((variant == 6 || variant == 7) && a.M > kVariant6MaxM) continue;
        if (variant == 8 && a.M > kVariant1MaxM) continue;
        if (variant == 9 && a.M > kVariant9MaxM) continue;
        for (int grain : {1, 2, 4, 8})
            for (int ccap : {16, 64}) cand.push_back(TreeCfg{grain, variant == 9 && ccap > kNoSlotCC ? kNoSlotCC : ccap, variant});
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GBS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GBS_ERR_CUDA;
    }
    best_ms = 1e30f;
    best = kDefaultCfg;
    tried = 0;
    int rc = GBS_OK;
    for (size_t c = 0; c < cand.size() && rc == GBS_OK; ++c) {
        a.grain = cand[c].grain;
        a.ccap = cand[c].ccap;
        a.variant = cand[c].variant;
        // one untimed run per candidate, then one timed run
        for (int rep = 0; rep < 2 && rc == GBS_OK; ++rep) {
            if (cudaMemsetAsync(a.status, 0, 64, st) != cudaSuccess) rc = GBS_ERR_CUDA;
            if (rep == 1) cudaEventRecord(e0, st);
            if (rc == GBS_OK && launch_forward(a, st) != cudaSuccess) rc = GBS_ERR_CUDA;
            if (rep == 1) cudaEventRecord(e1, st);
        }
        if (rc != GBS_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = GBS_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ++tried;
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GBS_OK) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    g_table[Key{device_cc(), a.sms, a.M, a.kmax, a.precision}] = Entry{best, best_ms};
    save_locked();
    return GBS_OK;
}

}  // namespace gbs
