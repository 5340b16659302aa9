// mfs_alloc.h -- the one device allocator of every handle (solver, batch, shared-A, MLP).
// It forwards to cudaMalloc unless a failure has been armed with mfs_debug_fail_alloc_after,
// which lets tests take every allocation-failure path without exhausting device memory.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace mfs {
cudaError_t device_malloc(void** p, size_t bytes);
// The bounds-checked build's record for mfs_row_residuals_static (mfs_static.cu); 0 otherwise.
unsigned long long static_bounds_record(bool reset);
}
