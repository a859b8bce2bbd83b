// stl_mining.cu -- time-interval mining steps (include/stl_mining.h): the loss seed of the
// robustness backward and the descent step on the sigmoid-parametrised interval.
#include <cuda_runtime.h>
#include <stdint.h>

#include "stl_mining.h"

stl_status stl_internal_fail(stl_status st, const char *msg);

namespace {

__global__ void mining_seed_kernel(const float *__restrict__ rho, long long N, int T, float *__restrict__ gout,
                                   float *loss) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (n < N) {
    const float r = rho[n * T];
    gout[n * T] = r < 0.f ? -1.f / (float)N : 0.f;
    l = r < 0.f ? -r / (float)N : 0.f;
  }
  if (loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
  }
}

constexpr int UT = 256;

__global__ void __launch_bounds__(UT) mining_update_kernel(float *theta, const float *__restrict__ gb, long long N,
                                                           int n_slots, int slot, int T, float lr, float gamma,
                                                           float *__restrict__ bounds) {
  __shared__ float sa[UT], sb[UT];
  __shared__ float nb[2];
  float ga = 0.f, gbv = 0.f;
  for (long long n = threadIdx.x; n < N; n += UT) {
    ga += gb[(n * n_slots + slot) * 2];
    gbv += gb[(n * n_slots + slot) * 2 + 1];
  }
  sa[threadIdx.x] = ga;
  sb[threadIdx.x] = gbv;
  __syncthreads();
  for (int s = UT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float al = theta[0], be = theta[1];
    const float a = 1.f / (1.f + expf(-al)), b = 1.f / (1.f + expf(-be));
    const float da = ((float)T * sa[0] + gamma) * a * (1.f - a);
    const float db = ((float)T * sb[0] - gamma) * b * (1.f - b);
    const float al2 = al - lr * da, be2 = be - lr * db;
    theta[0] = al2;
    theta[1] = be2;
    nb[0] = (float)T / (1.f + expf(-al2));
    nb[1] = (float)T / (1.f + expf(-be2));
  }
  __syncthreads();
  for (long long n = threadIdx.x; n < N; n += UT) {
    bounds[(n * n_slots + slot) * 2] = nb[0];
    bounds[(n * n_slots + slot) * 2 + 1] = nb[1];
  }
}

// per-trace descent: every trace n owns its interval (a_n, b_n) in steps
__global__ void mining_update_traces_kernel(float *__restrict__ bounds, const float *__restrict__ gb, long long N,
                                            int n_slots, int slot, float lr, float gamma, float scale, float a_cap,
                                            float b_cap, float min_width) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float *bp = bounds + (n * n_slots + slot) * 2;
  const float *g = gb + (n * n_slots + slot) * 2;
  float a = bp[0] - lr * (scale * g[0] + gamma);
  float b = bp[1] - lr * (scale * g[1] - gamma);
  a = fminf(fmaxf(a, 0.f), a_cap);
  b = fminf(fmaxf(b, a + min_width), b_cap);
  a = fminf(a, b - min_width);
  a = fmaxf(a, 0.f);
  bp[0] = a;
  bp[1] = b;
}

}  // namespace

extern "C" {

stl_status stl_mining_update_traces(float *bounds, const float *gbounds, int64_t N, int32_t n_slots, int32_t slot,
                                    float lr, float gamma, float scale, float a_cap, float b_cap, float min_width,
                                    void *stream) {
  if (N < 0 || n_slots < 1 || slot < 0 || slot >= n_slots)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need N >= 0 and 0 <= slot < n_slots");
  if (!(a_cap >= 0.f) || !(b_cap >= min_width) || !(min_width > 0.f))
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need a_cap >= 0, min_width > 0 and b_cap >= min_width");
  if (N == 0) return STL_OK;
  if (!bounds || !gbounds) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  mining_update_traces_kernel<<<(unsigned)((N + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      bounds, gbounds, N, n_slots, slot, lr, gamma, scale, a_cap, b_cap, min_width);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STL_OK : stl_internal_fail(STL_ERR_CUDA, "mining update launch failed");
}


stl_status stl_mining_seed(const float *rho, int64_t N, int32_t T, float *grad_out, float *loss, void *stream) {
  if (N < 0 || T < 1) return stl_internal_fail(STL_ERR_INVALID_ARG, "need N >= 0 and T >= 1");
  if (N == 0) return STL_OK;
  if (!rho || !grad_out) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  mining_seed_kernel<<<(unsigned)((N + 255) / 256), 256, 0, (cudaStream_t)stream>>>(rho, N, T, grad_out, loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STL_OK : stl_internal_fail(STL_ERR_CUDA, "mining seed launch failed");
}

stl_status stl_mining_update(float *theta, const float *gbounds, int64_t N, int32_t n_slots, int32_t slot, int32_t T,
                             float lr, float gamma, float *bounds, void *stream) {
  if (N < 1 || T < 1 || n_slots < 1 || slot < 0 || slot >= n_slots)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need N >= 1, T >= 1 and 0 <= slot < n_slots");
  if (!theta || !gbounds || !bounds) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  mining_update_kernel<<<1, UT, 0, (cudaStream_t)stream>>>(theta, gbounds, N, n_slots, slot, T, lr, gamma, bounds);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STL_OK : stl_internal_fail(STL_ERR_CUDA, "mining update launch failed");
}

}  // extern "C"
