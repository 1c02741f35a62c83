// Internal helpers shared by libddh's host translation units.
#pragma once

#include <cuda_runtime.h>

// Record `e` as the library's last CUDA error and map it to DDH_ENOMEM / DDH_ECUDA.
int ddh_internal_cuda_fail(cudaError_t e);
