// Forward-table kernels and their launch plumbing (internal to libgbs).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gbs {

enum Mode : int { MODE_P0 = 0, MODE_MU = 1, MODE_KAPPA = 2 };

// Everything one forward call needs on the device. Tables use the layout of
// gbs.h (order groups, colex ranks within an order).
struct FwdArgs {
    const double *V;      // 2M x 2M covariance (row-major, xxpp)
    int M, kmax, mode, precision;
    double *A;            // packed 2x2 blocks of (V+I)/2, M*M*4 doubles (workspace)
    double *p0;           // P0 table: the output for MODE_P0, a workspace table (orders < kmax) otherwise
    double *out;          // mu or kappa table (MODE_MU / MODE_KAPPA); equals p0 for MODE_P0
    unsigned *status;     // status word (workspace)
    unsigned *counters;   // per-order work counters (workspace, zeroed per call)
    double *scratch;      // per-CTA Schur-complement slots (workspace)
    size_t slot_doubles;  // doubles per slot
    int slots;            // number of slots = max persistent CTAs
    int sms;              // multiprocessors on the device
    cudaEvent_t *ev;      // GBS_MAX_ORDER + 2 timing events, or nullptr
};

// Workspace layout, shared by the size query and the launcher.
struct WsLayout {
    size_t status_off, A_off, p0_off, scratch_off, total;
    size_t slot_doubles;
    int slots;
};
WsLayout ws_layout(int M, int kmax, int sms);

// Queues every kernel of one forward call on stream; returns a cudaError_t.
cudaError_t launch_forward(const FwdArgs &a, cudaStream_t stream);

}  // namespace gbs
