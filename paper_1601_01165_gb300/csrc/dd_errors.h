// Status and thread-local error detail for the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "dd.h"

namespace dd {

// Record a formatted detail for dd_last_error() and return `s`.
dd_status set_error(dd_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
// Record a CUDA error (the last one if `e` is cudaSuccess) and return DD_ERR_CUDA.
dd_status set_cuda_error(const char* where, cudaError_t e = cudaSuccess);
void clear_error();

}  // namespace dd
