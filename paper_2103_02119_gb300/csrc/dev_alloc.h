// dev_alloc.h -- the one route by which the library allocates device memory
// (internal), so that a test hook can make an allocation fail on the host.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace lbm {

// cudaMalloc, unless the allocation countdown set by lbm_debug_fail_alloc
// reaches this call: then *p = nullptr and cudaErrorMemoryAllocation,
// without any CUDA call.
cudaError_t dev_malloc(void** p, size_t bytes);

template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace lbm
