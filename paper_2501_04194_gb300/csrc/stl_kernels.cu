// stl_kernels.cu -- launch dispatch, device properties and the sticky device status word.
#include <cuda_runtime.h>

#include "stl_internal.cuh"

#define STL_DECLARE_VARIANT(NAME)                                 \
  int stl_launch_##NAME(const KProgram &P, const LaunchArgs &A); \
  int stl_occupancy_##NAME(int smem_bytes, int *blocks);
STL_DECLARE_VARIANT(512_fh) STL_DECLARE_VARIANT(512_fs) STL_DECLARE_VARIANT(512_bh) STL_DECLARE_VARIANT(512_bs)
STL_DECLARE_VARIANT(256_fh) STL_DECLARE_VARIANT(256_fs) STL_DECLARE_VARIANT(256_bh) STL_DECLARE_VARIANT(256_bs)
STL_DECLARE_VARIANT(512_fh_r) STL_DECLARE_VARIANT(512_fs_r) STL_DECLARE_VARIANT(512_bh_r) STL_DECLARE_VARIANT(512_bs_r)
STL_DECLARE_VARIANT(256_fh_r) STL_DECLARE_VARIANT(256_fs_r) STL_DECLARE_VARIANT(256_bh_r) STL_DECLARE_VARIANT(256_bs_r)

namespace {
__device__ int g_device_status;   // sticky per-device status word (0 = OK)
}

int stl_status_ptr(int **ptr) {
  return (int)cudaGetSymbolAddress((void **)ptr, g_device_status);
}

namespace {
using LaunchFn = int (*)(const KProgram &, const LaunchArgs &);
using OccFn = int (*)(int, int *);
// index: ragged * 8 + (threads == 256) * 4 + backward * 2 + smooth
const LaunchFn k_launch[16] = {
    stl_launch_512_fh,   stl_launch_512_fs,   stl_launch_512_bh,   stl_launch_512_bs,
    stl_launch_256_fh,   stl_launch_256_fs,   stl_launch_256_bh,   stl_launch_256_bs,
    stl_launch_512_fh_r, stl_launch_512_fs_r, stl_launch_512_bh_r, stl_launch_512_bs_r,
    stl_launch_256_fh_r, stl_launch_256_fs_r, stl_launch_256_bh_r, stl_launch_256_bs_r};
const OccFn k_occupancy[16] = {
    stl_occupancy_512_fh,   stl_occupancy_512_fs,   stl_occupancy_512_bh,   stl_occupancy_512_bs,
    stl_occupancy_256_fh,   stl_occupancy_256_fs,   stl_occupancy_256_bh,   stl_occupancy_256_bs,
    stl_occupancy_512_fh_r, stl_occupancy_512_fs_r, stl_occupancy_512_bh_r, stl_occupancy_512_bs_r,
    stl_occupancy_256_fh_r, stl_occupancy_256_fs_r, stl_occupancy_256_bh_r, stl_occupancy_256_bs_r};

int variant(int threads, int bwd, int smooth, int ragged) {
  if (threads != 512 && threads != 256) return -1;
  return (ragged ? 8 : 0) + (threads == 256 ? 4 : 0) + (bwd ? 2 : 0) + (smooth ? 1 : 0);
}
}  // namespace

int stl_launch_main(const KProgram &P, const LaunchArgs &A) {
  const int v = variant(A.threads, P.bwd, P.mode == 1, A.table != nullptr);
  if (v < 0) return (int)cudaErrorInvalidValue;
  return k_launch[v](P, A);
}

int stl_blocks_per_sm(int threads, int bwd, int smooth, int ragged, int smem_bytes, int *blocks) {
  const int v = variant(threads, bwd, smooth, ragged);
  if (v < 0) return (int)cudaErrorInvalidValue;
  return k_occupancy[v](smem_bytes, blocks);
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
