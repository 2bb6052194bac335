// Backward (adjoint) kernels and the covariance model (internal to libgbs).
#pragma once
#include "gbs_fwd.cuh"

namespace gbs {

struct BwdLayout {
    WsLayout fwd;                     // packing, status, lower-order P0 slots, scratch slots
    size_t p0_off, h_off, gp0_off, inv_off, total;
};
BwdLayout bwd_layout(int M, int kmax, int sms);

struct BwdArgs {
    int M, kmax;
    FwdArgs fwd;        // V, packing buffer, status, counters, scratch slots
    const double *gk;   // dL/dkt, table layout
    double *gV;         // 2M x 2M output
    double *p0;         // P0 table, all orders (workspace)
    double *h;          // inverse-moment table, orders < kmax (workspace)
    double *gp0;        // dL/dP0 table (workspace)
    double *inv;        // inverses of A_{T'} for one prefix order (workspace)
    cudaEvent_t *ev;    // 5 timing events around the phases (P0, h, dL/dP0, dL/dV), or nullptr
};

cudaError_t launch_backward(const BwdArgs &a, cudaStream_t st);
cudaError_t launch_covariance(const double *Ur, const double *Ui, const double *r, const double *eta, int M, double *V,
                              cudaStream_t st);
cudaError_t launch_covariance_bwd(const double *Ur, const double *Ui, const double *r, const double *eta, int M,
                                  const double *V, const double *G, double *dr, double *deta, cudaStream_t st);

}  // namespace gbs
