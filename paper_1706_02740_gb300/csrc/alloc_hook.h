// The library's device and pinned-host allocations go through these wrappers, so that a test can
// make chosen ones fail (sft_debug_fail_allocations) and check each caller's error path and
// rollback on the host, with no GPU fault involved.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace sft {

cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
cudaError_t host_alloc(void** p, size_t bytes);

}  // namespace sft
