// Entry points of topk.cu shared with other translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace vpet {

// Bytes of workspace the discrepancy + top-k path needs for these sizes.
size_t topk_workspace_bytes(int64_t J, int64_t N, int L, int k, int precision);

// abc_discrepancy_topk on a caller-chosen workspace (validated arguments).
int topk_on_workspace(const float* y, int64_t J, int ldy, const float* x, int64_t N, int ldx, int L, const float* w,
                      int k, int precision, void* ws, size_t ws_bytes, int32_t* idx, float* dist, cudaStream_t s);

}  // namespace vpet
