// stl_kernels.cu -- launch dispatch, device properties and the sticky device status word.
#include <cuda_runtime.h>

#include "stl_internal.cuh"

int stl_launch_512_fh(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_512_fh(int smem_bytes, int *blocks);
int stl_launch_512_fs(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_512_fs(int smem_bytes, int *blocks);
int stl_launch_512_bh(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_512_bh(int smem_bytes, int *blocks);
int stl_launch_512_bs(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_512_bs(int smem_bytes, int *blocks);
int stl_launch_256_fh(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_256_fh(int smem_bytes, int *blocks);
int stl_launch_256_fs(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_256_fs(int smem_bytes, int *blocks);
int stl_launch_256_bh(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_256_bh(int smem_bytes, int *blocks);
int stl_launch_256_bs(const KProgram &P, const LaunchArgs &A);
int stl_occupancy_256_bs(int smem_bytes, int *blocks);

namespace {
__device__ int g_device_status;   // sticky per-device status word (0 = OK)
}

int stl_status_ptr(int **ptr) {
  return (int)cudaGetSymbolAddress((void **)ptr, g_device_status);
}

int stl_launch_main(const KProgram &P, const LaunchArgs &A) {
  const int v = (A.threads == 256 ? 4 : 0) + (P.bwd ? 2 : 0) + (P.mode == 1 ? 1 : 0);
  if (A.threads != 512 && A.threads != 256) return (int)cudaErrorInvalidValue;
  switch (v) {
    case 0: return stl_launch_512_fh(P, A);
    case 1: return stl_launch_512_fs(P, A);
    case 2: return stl_launch_512_bh(P, A);
    case 3: return stl_launch_512_bs(P, A);
    case 4: return stl_launch_256_fh(P, A);
    case 5: return stl_launch_256_fs(P, A);
    case 6: return stl_launch_256_bh(P, A);
    default: return stl_launch_256_bs(P, A);
  }
}

int stl_blocks_per_sm(int threads, int bwd, int smooth, int smem_bytes, int *blocks) {
  const int v = (threads == 256 ? 4 : 0) + (bwd ? 2 : 0) + (smooth ? 1 : 0);
  if (threads != 512 && threads != 256) return (int)cudaErrorInvalidValue;
  switch (v) {
    case 0: return stl_occupancy_512_fh(smem_bytes, blocks);
    case 1: return stl_occupancy_512_fs(smem_bytes, blocks);
    case 2: return stl_occupancy_512_bh(smem_bytes, blocks);
    case 3: return stl_occupancy_512_bs(smem_bytes, blocks);
    case 4: return stl_occupancy_256_fh(smem_bytes, blocks);
    case 5: return stl_occupancy_256_fs(smem_bytes, blocks);
    case 6: return stl_occupancy_256_bh(smem_bytes, blocks);
    default: return stl_occupancy_256_bs(smem_bytes, blocks);
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
