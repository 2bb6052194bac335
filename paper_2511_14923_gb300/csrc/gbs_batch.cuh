// Ragged batched launch (internal to libgbs).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "gbs.h"

namespace gbs {
size_t batched_workspace_bytes(const gbs_instance *inst, int n, int precision, int sms);
int batched_plan(const gbs_instance *inst, int n, int precision, char *ws, size_t ws_bytes, int sms, cudaStream_t st,
                 size_t &needed);
cudaError_t launch_batched(char *ws, int precision, int sms, cudaStream_t st);
}  // namespace gbs
