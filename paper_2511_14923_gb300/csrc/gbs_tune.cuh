// Prefix-tree schedule autotuner (internal to libgbs).
#pragma once
#include "gbs_fwd.cuh"

namespace gbs {
// Tuned schedule for this shape on the current device, or kDefaultCfg.
TreeCfg tuned_cfg(int sms, int M, int kmax, int precision);
// Times every candidate schedule (cumulant mode, a fully prepared) and records the best.
int autotune(FwdArgs a, cudaStream_t st, TreeCfg &best, float &best_ms, int &tried);
}  // namespace gbs
