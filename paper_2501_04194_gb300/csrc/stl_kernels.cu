// stl_kernels.cu -- launch dispatch, device properties and the sticky device status word.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "stl_internal.cuh"

#define STL_DECLARE_VARIANT(NAME)                                                 \
  int stl_launch_##NAME(const KProgram &P, const LaunchArgs &A, bool set_smem_attr); \
  int stl_occupancy_##NAME(int smem_bytes, int *blocks);
STL_DECLARE_VARIANT(512_fh) STL_DECLARE_VARIANT(512_fs) STL_DECLARE_VARIANT(512_bh) STL_DECLARE_VARIANT(512_bs)
STL_DECLARE_VARIANT(256_fh) STL_DECLARE_VARIANT(256_fs) STL_DECLARE_VARIANT(256_bh) STL_DECLARE_VARIANT(256_bs)
STL_DECLARE_VARIANT(64_fh) STL_DECLARE_VARIANT(64_fs) STL_DECLARE_VARIANT(64_bh) STL_DECLARE_VARIANT(64_bs)
STL_DECLARE_VARIANT(512_fh_r) STL_DECLARE_VARIANT(512_fs_r) STL_DECLARE_VARIANT(512_bh_r) STL_DECLARE_VARIANT(512_bs_r)
STL_DECLARE_VARIANT(256_fh_r) STL_DECLARE_VARIANT(256_fs_r) STL_DECLARE_VARIANT(256_bh_r) STL_DECLARE_VARIANT(256_bs_r)
STL_DECLARE_VARIANT(64_fh_r) STL_DECLARE_VARIANT(64_fs_r) STL_DECLARE_VARIANT(64_bh_r) STL_DECLARE_VARIANT(64_bs_r)

namespace {
__device__ int g_device_status;   // sticky per-device status word (0 = OK)
}

int stl_status_ptr(int **ptr) {
  return (int)cudaGetSymbolAddress((void **)ptr, g_device_status);
}

namespace {
using LaunchFn = int (*)(const KProgram &, const LaunchArgs &, bool);
using OccFn = int (*)(int, int *);
// index: ragged * 12 + size * 4 + backward * 2 + smooth, size 0 / 1 / 2 = 512 / 256 / 64 threads
const LaunchFn k_launch[24] = {
    stl_launch_512_fh,   stl_launch_512_fs,   stl_launch_512_bh,   stl_launch_512_bs,
    stl_launch_256_fh,   stl_launch_256_fs,   stl_launch_256_bh,   stl_launch_256_bs,
    stl_launch_64_fh,    stl_launch_64_fs,    stl_launch_64_bh,    stl_launch_64_bs,
    stl_launch_512_fh_r, stl_launch_512_fs_r, stl_launch_512_bh_r, stl_launch_512_bs_r,
    stl_launch_256_fh_r, stl_launch_256_fs_r, stl_launch_256_bh_r, stl_launch_256_bs_r,
    stl_launch_64_fh_r,  stl_launch_64_fs_r,  stl_launch_64_bh_r,  stl_launch_64_bs_r};
const OccFn k_occupancy[24] = {
    stl_occupancy_512_fh,   stl_occupancy_512_fs,   stl_occupancy_512_bh,   stl_occupancy_512_bs,
    stl_occupancy_256_fh,   stl_occupancy_256_fs,   stl_occupancy_256_bh,   stl_occupancy_256_bs,
    stl_occupancy_64_fh,    stl_occupancy_64_fs,    stl_occupancy_64_bh,    stl_occupancy_64_bs,
    stl_occupancy_512_fh_r, stl_occupancy_512_fs_r, stl_occupancy_512_bh_r, stl_occupancy_512_bs_r,
    stl_occupancy_256_fh_r, stl_occupancy_256_fs_r, stl_occupancy_256_bh_r, stl_occupancy_256_bs_r,
    stl_occupancy_64_fh_r,  stl_occupancy_64_fs_r,  stl_occupancy_64_bh_r,  stl_occupancy_64_bs_r};

int variant(int threads, int bwd, int smooth, int ragged) {
  const int size = threads == 512 ? 0 : threads == 256 ? 1 : threads == 64 ? 2 : -1;
  if (size < 0) return -1;
  return (ragged ? 12 : 0) + size * 4 + (bwd ? 2 : 0) + (smooth ? 1 : 0);
}
}  // namespace

// Host-side caches (per device) of what every launch plan asks the runtime: the SM count,
// the opt-in shared memory limit, occupancy per (variant, shared bytes), and the dynamic
// shared memory attribute last set on each variant (a launch sets it only when it needs
// more).  Small calls are dominated by these queries otherwise.
namespace {
constexpr int kMaxDev = 64;
std::mutex g_cache_mu;
int g_sms[kMaxDev], g_smem_optin[kMaxDev];
int g_smem_set[kMaxDev][24];
std::map<std::tuple<int, int, int>, int> g_occ;

int current_device(int *dev) { return (int)cudaGetDevice(dev); }
}  // namespace

int stl_launch_main(const KProgram &P, const LaunchArgs &A) {
  const int v = variant(A.threads, P.bwd, P.mode != 0, A.table != nullptr);   // smooth kernels serve both smooth modes
  if (v < 0) return (int)cudaErrorInvalidValue;
  int dev = 0;
  int e = current_device(&dev);
  if (e) return e;
  const int smem = P.smem_words * 4;
  bool need_attr = true;
  if (dev < kMaxDev) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    need_attr = g_smem_set[dev][v] < smem;
  }
  e = k_launch[v](P, A, need_attr);
  if (!e && need_attr && dev < kMaxDev) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_smem_set[dev][v] = smem;   // the attribute now holds exactly this value
  }
  return e;
}

int stl_blocks_per_sm(int threads, int bwd, int smooth, int ragged, int smem_bytes, int *blocks) {
  const int v = variant(threads, bwd, smooth, ragged);
  if (v < 0) return (int)cudaErrorInvalidValue;
  int dev = 0;
  int e = current_device(&dev);
  if (e) return e;
  const auto key = std::make_tuple(dev, v, smem_bytes);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) { *blocks = it->second; return 0; }
  }
  e = k_occupancy[v](smem_bytes, blocks);
  if (!e) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_occ[key] = *blocks;
    if (dev < kMaxDev) g_smem_set[dev][v] = smem_bytes;   // the occupancy query set the attribute
  }
  return e;
}

static int device_attr(int (&cache)[kMaxDev], cudaDeviceAttr attr, int *out) {
  int dev = 0;
  int e = current_device(&dev);
  if (e) return e;
  if (dev < kMaxDev) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (cache[dev] > 0) { *out = cache[dev]; return 0; }
  }
  e = (int)cudaDeviceGetAttribute(out, attr, dev);
  if (!e && dev < kMaxDev) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache[dev] = *out;
  }
  return e;
}

int stl_max_smem_optin(int *bytes) { return device_attr(g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, bytes); }

int stl_num_sms(int *sms) { return device_attr(g_sms, cudaDevAttrMultiProcessorCount, sms); }

int stl_read_clear_status(void *stream, int *status) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return (int)e;
  int zero = 0;
  e = cudaMemcpyFromSymbol(status, g_device_status, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  return (int)cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
}
