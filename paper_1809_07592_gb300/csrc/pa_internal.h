// pa_internal.h -- helpers shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Records "what: cuda error string" as the calling thread's last CUDA error and returns PA_ECUDA.
int pa_internal_cuda_fail(cudaError_t e, const char *what);

// Device twiddle tables hi/lo of the length-2^lgL transform for a pa_dtype_t (cudaMalloc'd; caller frees).
int pa_internal_twiddles(int lgL, int dtype, void **hi, void **lo, uint32_t *B);
