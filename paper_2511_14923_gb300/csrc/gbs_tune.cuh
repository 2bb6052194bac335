// Prefix-tree schedule autotuner (internal to libgbs).
#pragma once
#include "gbs.h"
#include "gbs_fwd.cuh"

namespace gbs {
// Tuned schedule for this shape on the current device, or kDefaultCfg.
TreeCfg tuned_cfg(int sms, int M, int kmax, int precision);
// Times every candidate schedule (cumulant mode, a fully prepared) and records the best.
int autotune(FwdArgs a, cudaStream_t st, TreeCfg &best, float &best_ms, int &tried);
// Tuned schedule of a ragged batch with this multiset of (M, kmax) on the current
// device: true and cfg set if one is recorded.
bool tuned_batch_cfg(int sms, const gbs_instance *inst, int n, int precision, TreeCfg &cfg);
// Records a batch schedule (and rewrites the JSON cache if one is configured).
void record_batch_cfg(int sms, const gbs_instance *inst, int n, int precision, const TreeCfg &cfg, float ms);
}  // namespace gbs
