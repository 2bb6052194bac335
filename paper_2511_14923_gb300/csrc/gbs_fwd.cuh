// Forward-table kernels and their launch plumbing (internal to libgbs).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace gbs {

// Table a forward call fills: vacuum probabilities, click moments, click
// cumulants, spin correlators c(S) (Eq. correlator_sum_cov), spin cumulants
// kappa(S) (Eq. cumulant_corr_main).
enum Mode : int { MODE_P0 = 0, MODE_MU = 1, MODE_KAPPA = 2, MODE_SPINC = 3, MODE_SPINK = 4 };

// Everything one forward call needs on the device. Tables use the layout of
// gbs.h (order groups, colex ranks within an order).
struct FwdArgs {
    const double *V;      // 2M x 2M covariance (row-major, xxpp)
    const double *mean;   // first moments (2M, xxpp) of a displaced state; nullptr = zero mean
    int M, kmax, mode, precision;
    double *A;            // packed 2x2 blocks of (V+I)/2, M*M*4 doubles (workspace)
    float *Af;            // the same blocks as float pairs (hi x4, lo x4), refined path (workspace)
    float *p0f;           // P0({x}) as float pairs (hi, lo) per mode, refined path (workspace; may be null)
    double *p0;           // P0 table: the output for MODE_P0, a workspace table (orders < kmax) otherwise
    double *out;          // mu or kappa table (MODE_MU / MODE_KAPPA); equals p0 for MODE_P0
    unsigned *status;     // status word (workspace)
    unsigned *counters;   // per-order work counters (workspace, zeroed per call)
    double *scratch;      // per-CTA Schur-complement slots (workspace)
    size_t slot_doubles;  // doubles per slot
    int slots;            // number of slots = max persistent CTAs
    int sms;              // multiprocessors on the device
    cudaEvent_t *ev;      // GBS_MAX_ORDER + 2 timing events, or nullptr
    // range call (gbs_table_range): order kmax is filled only for top elements in
    // [c_lo, c_hi), into top[idx - top_base]; top = nullptr fills whole tables
    double *top;
    uint64_t top_base;
    int c_lo, c_hi;
    // prefix-tree schedule (autotuned): items per CTA slot, children per shared-
    // memory batch, CTA shape (0: 512 threads x 1 per SM; 1: 256 x 2; refined path
    // only: 2: 640 x 1, 3: 256 x 3, 4: 768 x 1 with a 2048-entry x area, 5: 384 x 2
    // with a 960-entry x area, 6: 256 x 4 with a 384-entry x area, 7: 6 in clusters
    // of 4, 8: 3 in clusters of 3, 9: 6 without Schur-complement slots)
    int grain, ccap, variant;
};

// Valid (M, kmax) of a forward table: orders 4 and 5 run the prefix-tree kernels
// (shared-memory x-entries sized for GBS_MAX_MODES); tables with kmax <= 3 run
// one thread per subset and take up to GBS_MAX_MODES_K3 modes.
inline bool valid_mk(int M, int kmax) {
    return M >= 1 && kmax >= 1 && kmax <= 5 && kmax <= M && M <= (kmax <= 3 ? 4096 : 1024);
}

// Message for an (M, kmax) that valid_mk rejects (defined in gbs_api.cu).
std::string shape_message(int M, int kmax);

// Schedule of the prefix-tree kernels for one problem shape.
struct TreeCfg {
    int grain, ccap, variant;
};
constexpr TreeCfg kDefaultCfg{2, 64, 0};
// Most children per shared-memory batch any CTA shape has room for.
constexpr int kMaxChildren = 64;
// Largest M the 256-thread variant accepts (its shared x-entry area holds 576 modes).
constexpr int kVariant1MaxM = 577;
// x-entries per batch of the 768-thread refined variant (one CTA per SM).
constexpr int kWideXC = 2048;
// x-entries per batch of the 384-thread x 2 refined variant, and its largest M.
constexpr int kPairXC = 960;
constexpr int kVariant5MaxM = kPairXC + 1;
// x-entries per batch of the 256-thread x 4 refined variant, and its largest M.
constexpr int kQuadXC = 384;
constexpr int kVariant6MaxM = kQuadXC + 1;
// The slot-free 256-thread x 4 refined variant: children per batch it has room
// for, and the elimination rows Y(x), x < c4 <= M - 2, it keeps in shared memory.
constexpr int kNoSlotCC = 24;
constexpr int kNoSlotYC = 160;
constexpr int kVariant9MaxM = kNoSlotYC + 1;  // order 4 reaches c4 = M - 1
// Number of CTA shapes (variants 0..kNumVariants-1); 7 and 8 are the 256 x 4 and
// 256 x 3 shapes in thread-block clusters of 4 and 3 CTAs sharing one slot, 9 the
// 256 x 4 shape without slots.
constexpr int kNumVariants = 10;
// CTA shape a forward call of (M, precision) runs for a recorded variant: the
// shapes that do not admit M (or the precision) fall back to 512 x 1.
inline int effective_variant(int variant, int M, int precision) {
    if (variant == 1 || variant == 3 || variant == 8) return M <= kVariant1MaxM && (variant == 1 || precision == 1) ? variant : 0;
    if (precision != 1) return 0;
    if (variant == 2 || variant == 4) return variant;
    if (variant == 5) return M <= kVariant5MaxM ? 5 : 0;
    if (variant == 6 || variant == 7) return M <= kVariant6MaxM ? variant : 0;
    if (variant == 9) return M <= kVariant9MaxM ? 9 : 0;
    return 0;
}
// Whether a variant runs in clusters (the batched kernel has no clustered form).
inline bool variant_clustered(int v) { return v == 7 || v == 8; }

// Workspace layout, shared by the size query and the launcher.
struct WsLayout {
    size_t status_off, A_off, p0f_off, p0_off, scratch_off, total;
    size_t slot_doubles;
    int slots;
};
// Scratch slots per multiprocessor that cover every CTA shape allowed for M:
// four when the 256 x 4 shape can run (M <= 385), else three.
inline int slots_per_sm_for(int M) { return M <= 385 ? 4 : 3; }
// Reserves slots_per_sm scratch slots per multiprocessor (0 = slots_per_sm_for(M);
// with one, only one CTA per multiprocessor runs).
WsLayout ws_layout(int M, int kmax, int sms, int slots_per_sm = 0);

// Queues the packing of A = (V+I)/2 into 2x2 blocks.
cudaError_t launch_pack(const FwdArgs &a, cudaStream_t stream);
// Queues every kernel of one forward call on stream; returns a cudaError_t.
cudaError_t launch_forward(const FwdArgs &a, cudaStream_t stream);
// The same for a displaced state (a.mean set, a.precision = 0).
cudaError_t launch_forward_displaced(const FwdArgs &a, cudaStream_t stream);

}  // namespace gbs
