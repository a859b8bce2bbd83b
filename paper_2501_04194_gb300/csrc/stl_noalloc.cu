// stl_noalloc.cu -- backward entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc at all once they are running: a host application that
// hands this library a fixed pool and forbids further device allocation, a real-time control
// loop whose memory is frozen after start-up, or a plugin whose framework owns every device
// byte.  For them, stl_robustness_backward_noalloc takes the same inputs and outputs as
// stl_robustness_backward but keeps its scratch (the per-thread arrays of the smooth Until
// adjoint and any node buffers that do not fit in shared memory) in the file-scope array
// below, so the caller passes no workspace.
//
// The array is a static __device__ object of STL_NOALLOC_SCRATCH_BYTES: every GPU that loads
// the library holds it until the process exits.  In host code its name is only a host-side
// stand-in, so its device address is obtained with cudaGetSymbolAddress, with the call's device
// current, on every call: after a device reset the module is loaded again and the array may
// sit at another address, so a cached address could point at freed memory.
#include <cuda_runtime.h>

#include "../../include/stl.h"
#include "stl_internal.cuh"

stl_status stl_internal_plan_backward_capped(stl_handle h, const float *sig, int64_t B, int64_t T,
                                             const float *bounds, const stl_params *p, size_t capacity_bytes,
                                             KProgram *prog, int *grid, int *threads, size_t *ws_bytes);
stl_status stl_internal_fail(stl_status st, const char *msg);

namespace {

constexpr size_t kScratchWords = STL_NOALLOC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_noalloc_scratch[kScratchWords];

// device address of the static scratch in the current device's context (looked up per call)
stl_status scratch_address(void **out) {
  void *ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString(e));
  *out = ptr;
  return STL_OK;
}

}  // namespace

extern "C" {

stl_status stl_robustness_backward_noalloc(stl_handle h, const float *sig, int64_t B, int64_t T,
                                           const float *bounds, const stl_params *p, const float *grad_out,
                                           float *grad_sig, float *grad_bounds, void *stream) {
  if (B > 0 && (!grad_out || !grad_sig)) return stl_internal_fail(STL_ERR_INVALID_ARG, "grad_out / grad_sig is NULL");
  KProgram prog;
  int grid = 0, threads = 0;
  size_t ws_bytes = 0;
  stl_status s = stl_internal_plan_backward_capped(h, sig, B, T, bounds, p, STL_NOALLOC_SCRATCH_BYTES, &prog, &grid,
                                                   &threads, &ws_bytes);
  if (s) return s;
  if (B == 0) return STL_OK;   // checked, nothing to launch (the planner stops before planning)
  void *scratch = nullptr;
  s = scratch_address(&scratch);
  if (s) return s;
  // the kernels write every scratch word before reading it, so nothing needs clearing here
  if (grad_bounds && prog.n_slots > 0) {
    cudaError_t e = cudaMemsetAsync(grad_bounds, 0, (size_t)B * prog.n_slots * 2 * sizeof(float),
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString(e));
  }
  LaunchArgs A{};
  int e0 = stl_status_ptr(&A.status);
  if (e0) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString((cudaError_t)e0));
  A.sig = sig;
  A.bounds = prog.n_slots ? bounds : nullptr;
  A.gout = grad_out;
  A.gsig = grad_sig;
  A.gbounds = prog.n_slots ? grad_bounds : nullptr;
  A.ws = ws_bytes > 0 ? (float *)scratch : nullptr;
  A.grid = grid;
  A.threads = threads;
  A.stream = stream;
  int e = stl_launch_main(prog, A);
  if (e) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString((cudaError_t)e));
  return STL_OK;
}

}  // extern "C"
