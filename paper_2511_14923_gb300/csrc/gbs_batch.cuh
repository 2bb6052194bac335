// Ragged batched launch (internal to libgbs).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "gbs.h"
#include "gbs_fwd.cuh"

namespace gbs {
size_t batched_workspace_bytes(const gbs_instance *inst, int n, int precision, int sms);
// Writes the plan (schedule from the batch autotuner's table, else the default).
int batched_plan(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms, cudaStream_t st,
                 size_t &needed);
// Queues the batched kernel for the plan last written into ws; planned = false
// (nothing queued) if ws holds no plan of this precision from this process.
cudaError_t launch_batched(char *ws, int precision, cudaStream_t st, bool &planned);
// Schedule of the plan last written into ws: {variant, threads per CTA, CTAs,
// grain, children per batch}; false if ws holds no plan.
bool batched_schedule(const void *ws, int *out5);
// Times the candidate schedules on the batch (outputs are overwritten), records
// the fastest and leaves its plan in ws.
int batched_autotune(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms,
                     cudaStream_t st, TreeCfg &best, float &best_ms, int &tried);
}  // namespace gbs
