// stl_kernels.cu -- launch dispatch, device properties and the sticky device status word.
#include <cuda_runtime.h>

#include "stl_internal.cuh"

int stl_launch_nt128(const KProgram &P, const LaunchArgs &A);
int stl_launch_nt256(const KProgram &P, const LaunchArgs &A);
int stl_launch_nt512(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_nt128(int smem_bytes, int *blocks);
int stl_occupancy_nt256(int smem_bytes, int *blocks);
int stl_occupancy_nt512(int smem_bytes, int *blocks);

namespace {
__device__ int g_device_status;   // sticky per-device status word (0 = OK)
}

int stl_status_ptr(int **ptr) {
  return (int)cudaGetSymbolAddress((void **)ptr, g_device_status);
}

int stl_launch_main(const KProgram &P, const LaunchArgs &A) {
  switch (A.threads) {
    case 128: return stl_launch_nt128(P, A);
    case 256: return stl_launch_nt256(P, A);
    case 512: return stl_launch_nt512(P, A);
    default: return (int)cudaErrorInvalidValue;
  }
}

int stl_blocks_per_sm(int threads, int smem_bytes, int *blocks) {
  switch (threads) {
    case 128: return stl_occupancy_nt128(smem_bytes, blocks);
    case 256: return stl_occupancy_nt256(smem_bytes, blocks);
    case 512: return stl_occupancy_nt512(smem_bytes, blocks);
    default: return (int)cudaErrorInvalidValue;
  }
}

int stl_max_smem_optin(int *bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceGetAttribute(bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
}

int stl_num_sms(int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
}

int stl_read_clear_status(void *stream, int *status) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return (int)e;
  int zero = 0;
  e = cudaMemcpyFromSymbol(status, g_device_status, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  return (int)cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
}
