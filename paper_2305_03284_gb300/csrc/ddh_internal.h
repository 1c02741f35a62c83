// Internal helpers shared by libddh's host translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

// NVTX range over one host-side library call (header-only NVTX3; a no-op unless a profiler
// such as Nsight Compute or Nsight Systems is attached), so that traces show which API call
// enqueued which kernels.
struct DdhNvtxRange {
  explicit DdhNvtxRange(const char* name) { nvtxRangePushA(name); }
  ~DdhNvtxRange() { nvtxRangePop(); }
  DdhNvtxRange(const DdhNvtxRange&) = delete;
  DdhNvtxRange& operator=(const DdhNvtxRange&) = delete;
};

// Makes `dev` the calling thread's current device for the guard's lifetime and restores the
// caller's current device when the guard goes out of scope, so that no library call changes
// which device the caller's thread has current.
class DdhDeviceGuard {
 public:
  explicit DdhDeviceGuard(int dev) {
    err_ = cudaGetDevice(&prev_);
    if (err_ == cudaSuccess && prev_ != dev) {
      err_ = cudaSetDevice(dev);
      switched_ = err_ == cudaSuccess;
    }
  }
  ~DdhDeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  cudaError_t error() const { return err_; }
  DdhDeviceGuard(const DdhDeviceGuard&) = delete;
  DdhDeviceGuard& operator=(const DdhDeviceGuard&) = delete;

 private:
  int prev_ = 0;
  bool switched_ = false;
  cudaError_t err_ = cudaSuccess;
};

// Record `e` as the library's last CUDA error and map it to DDH_ENOMEM / DDH_ECUDA.
int ddh_internal_cuda_fail(cudaError_t e);

struct ddh_params;
// Enqueue the adjoint kernels of one frame step on `stream` (arguments as ddh_step_backward).
int ddh_internal_step_backward(int n, const ddh_params* prm, const void* twiddle, void* stream, const void* y,
                               const float* r_prev, const float* phi_prev, const float* trace, const float* r_new,
                               const float* r_bar, const float* phi_bar, float* r_prev_bar, float* phi_prev_bar,
                               float* grads, void* workspace);

struct ddh_state;
// Read-only view of a state's parameters, twiddle table, stream and device.
int ddh_internal_state_info(const ddh_state* s, const ddh_params** prm, const void** twiddle, void** stream,
                            int* device);
// Set the library's last error message (returned by ddh_last_cuda_error).
void ddh_internal_set_error(const char* msg);
// The state and argument checks shared by every frame-step adjoint entry point: DDH_OK, or
// DDH_EINVAL with the reason set as the library's last error message.
int ddh_internal_backward_check(const ddh_state* s, const void* y, const float* trace);
// Device bytes a state with parameters `p` holds (its path's working images included); 0 if
// the grid size is unsupported.
size_t ddh_internal_state_bytes(const ddh_params* p);
