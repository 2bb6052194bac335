// Chain-rule sampler (internal to libgbs): workspace layout and launcher.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gbs {
namespace smp {

// Byte offsets of the per-sample arrays ([entries][S]) in the workspace.
struct SamplerLayout {
    size_t chi, P, Pp, P1, P2, Z, Z5, G, Y, X, W, CA, T, bw, kap, hs, H, lead, At, total;
};
SamplerLayout sampler_layout(int M, int K, int S, int precision);

struct SamplerCall {
    const double *kappa;   // spin-cumulant table, orders 1..K (device)
    int M, K, S, precision, n_samples;
    int orders[3];         // expansion orders of p+, p1, p2 (K = 5)
    const double *u;       // [n_samples][M] uniforms, or null when force is given
    const uint8_t *force;  // [n_samples][M] bits to score, or null
    uint8_t *bits;         // [n_samples][M]
    double *prob;          // [n_samples] ln of the estimated probability, or null
    double *q0;            // [n_samples][M] or null
    void *ws;
};
cudaError_t launch_sampler(const SamplerCall &c, cudaStream_t stream);

}  // namespace smp
}  // namespace gbs
