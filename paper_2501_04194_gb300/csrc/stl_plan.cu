// stl_plan.cu -- trajectory-optimisation helpers (include/stl_plan.h): the rollout of the
// saturated single integrator and its adjoint fused with Adam, the solved/active bookkeeping,
// and the elementwise steps of the warm-start MLP (its matrix products: stl_gemm.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "stl_internal.cuh"
#include "stl_plan.h"

stl_status stl_internal_fail(stl_status st, const char *msg);

namespace {

constexpr unsigned FULL = 0xffffffffu;

stl_status cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return STL_OK;
  return stl_internal_fail(STL_ERR_CUDA, what);
}

// exclusive prefix sum over the lanes of a warp (lane order)
__device__ __forceinline__ float warp_excl_prefix(float v) {
  const int lane = threadIdx.x & 31;
  float inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float n = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += n;
  }
  return inc - v;
}

// exclusive suffix sum over the lanes of a warp (reverse lane order)
__device__ __forceinline__ float warp_excl_suffix(float v) {
  const int lane = threadIdx.x & 31;
  float inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float n = __shfl_down_sync(FULL, inc, o);
    if (lane + o < 32) inc += n;
  }
  return inc - v;
}

// x_t = sum_{s<=t} dt tanh(u_s) for one problem, by one warp: each lane owns a chunk of
// consecutive steps (local sums, a warp scan of the chunk totals, then the running sums)
__device__ __forceinline__ void rollout_warp(const float *u, float *x, int T, float dt) {
  const int lane = threadIdx.x & 31;
  const int c = (T + 31) / 32;
  const int t0 = min(lane * c, T), t1 = min(t0 + c, T);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    float s = 0.f;
    for (int t = t0; t < t1; ++t) s += dt * tanhf(u[2 * t + d]);
    float run = warp_excl_prefix(s);
    for (int t = t0; t < t1; ++t) {
      run += dt * tanhf(u[2 * t + d]);
      x[2 * t + d] = run;
    }
  }
}

__global__ void rollout_kernel(const float *__restrict__ u, long long B, int T, float dt, float *__restrict__ x) {
  const long long b = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (b >= B) return;   // whole warps exit together
  rollout_warp(u + b * T * 2, x + b * T * 2, T, dt);
}

__global__ void plan_adam_kernel(float *__restrict__ u, float *__restrict__ m, float *__restrict__ v,
                                 const float *__restrict__ xbar, const int *__restrict__ active, long long B, int T,
                                 float dt, float lr, float b1, float b2, float eps, float c1, float c2,
                                 float *__restrict__ x) {
  const long long b = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (b >= B || !active[b]) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int c = (T + 31) / 32;
  const int t0 = min(lane * c, T), t1 = min(t0 + c, T);
  const long long base = b * T * 2;
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    // suffix sums of xbar: S_t = sum_{s >= t} xbar_s
    float s = 0.f;
    for (int t = t0; t < t1; ++t) s += xbar[base + 2 * t + d];
    float run = warp_excl_suffix(s);   // sum over the later chunks
    for (int t = t1 - 1; t >= t0; --t) {
      const long long i = base + 2 * t + d;
      run += xbar[i];
      const float th = tanhf(u[i]);
      const float g = dt * (1.f - th * th) * run;
      const float mi = b1 * m[i] + (1.f - b1) * g;
      const float vi = b2 * v[i] + (1.f - b2) * g * g;
      m[i] = mi;
      v[i] = vi;
      u[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
  }
  __syncwarp();
  rollout_warp(u + base, x + base, T, dt);
}

__global__ void plan_check_kernel(const float *__restrict__ rho, int *__restrict__ active, int *__restrict__ solved,
                                  int iter, float *__restrict__ gout, long long B, int T, int *n_active) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int still = 0;
  if (b < B) {
    int a = active[b];
    if (a && rho[b * T] >= 0.f) {
      solved[b] = iter;
      active[b] = 0;
      a = 0;
    }
    gout[b * T] = a ? -1.f : 0.f;
    still = a;
  }
  if (n_active) {
    const unsigned bal = __ballot_sync(FULL, still);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(n_active, __popc(bal));
  }
}

// ------------------------------------------------------------------ trajectory optimisation
// with a learnable interval: one warp per problem (suffix scans of xbar, Adam on u, prefix
// scan of the new trajectory), lane 0 updates the problem's interval parameters.
__global__ void trajopt_seed_kernel(const float *__restrict__ rho, const float *__restrict__ gam, long long B, int T,
                                    float *__restrict__ gout) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) gout[b * T] = rho[b * T] < 0.f ? -gam[b * 4] : 0.f;
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

__global__ void trajopt_step_kernel(float *__restrict__ u, float *__restrict__ mu, float *__restrict__ vu,
                                    float *__restrict__ theta, float *__restrict__ mth, float *__restrict__ vth,
                                    const float *__restrict__ xbar, const float *__restrict__ gb,
                                    const float *__restrict__ gam, long long B, int T, int n_slots, int slot, float dt,
                                    float sx, float sy, float umax, float inom, float lr_u, float lr_th, float b1,
                                    float b2, float eps, float c1, float c2, float *__restrict__ x,
                                    float *__restrict__ bounds) {
  const long long b = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (b >= B) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int c = (T + 31) / 32;
  const int t0 = min(lane * c, T), t1 = min(t0 + c, T);
  const long long base = b * T * 2;
  const float g3 = gam[b * 4 + 2] / (float)T, g4 = gam[b * 4 + 3] / (float)T;
  // controls: ubar_t = dt sum_{s >= t} xbar_s + g3 [|u_t| > umax] u_t / |u_t| + 2 g4 u_t
  float s0 = 0.f, s1 = 0.f;
  for (int t = t0; t < t1; ++t) {
    s0 += xbar[base + 2 * t];
    s1 += xbar[base + 2 * t + 1];
  }
  float r0 = warp_excl_suffix(s0), r1 = warp_excl_suffix(s1);
  for (int t = t1 - 1; t >= t0; --t) {
    const long long i = base + 2 * t;
    r0 += xbar[i];
    r1 += xbar[i + 1];
    const float u0 = u[i], u1 = u[i + 1];
    const float nrm = sqrtf(u0 * u0 + u1 * u1);
    const float lim = nrm > umax ? g3 / nrm : 0.f;
    const float g[2] = {dt * r0 + lim * u0 + 2.f * g4 * u0, dt * r1 + lim * u1 + 2.f * g4 * u1};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float mi = b1 * mu[i + d] + (1.f - b1) * g[d];
      const float vi = b2 * vu[i + d] + (1.f - b2) * g[d] * g[d];
      mu[i + d] = mi;
      vu[i + d] = vi;
      u[i + d] -= lr_u * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
  }
  __syncwarp();
  // new trajectory x_t = start + dt sum_{s <= t} u_s
  float p0 = 0.f, p1 = 0.f;
  for (int t = t0; t < t1; ++t) {
    p0 += dt * u[base + 2 * t];
    p1 += dt * u[base + 2 * t + 1];
  }
  float q0 = sx + warp_excl_prefix(p0), q1 = sy + warp_excl_prefix(p1);
  for (int t = t0; t < t1; ++t) {
    q0 += dt * u[base + 2 * t];
    q1 += dt * u[base + 2 * t + 1];
    x[base + 2 * t] = q0;
    x[base + 2 * t + 1] = q1;
  }
  if (lane == 0) {
    // interval: a = sigmoid(alpha), b = sigmoid(beta); dJ/da = T gA + 2 g2 e, dJ/db = T gB - 2 g2 e
    const float al = theta[b * 2], be = theta[b * 2 + 1];
    const float a = sigmoidf_(al), bb = sigmoidf_(be);
    const float e = expf(2.f * (inom - bb + a));
    const float g2 = gam[b * 4 + 1];
    const long long gi = (b * n_slots + slot) * 2;
    const float ga = ((float)T * gb[gi] + 2.f * g2 * e) * a * (1.f - a);
    const float gbt = ((float)T * gb[gi + 1] - 2.f * g2 * e) * bb * (1.f - bb);
    const float gth[2] = {ga, gbt};
    float nth[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float mi = b1 * mth[b * 2 + d] + (1.f - b1) * gth[d];
      const float vi = b2 * vth[b * 2 + d] + (1.f - b2) * gth[d] * gth[d];
      mth[b * 2 + d] = mi;
      vth[b * 2 + d] = vi;
      nth[d] = theta[b * 2 + d] - lr_th * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
    // keep a below b (the masked window needs a < b)
    float na = sigmoidf_(nth[0]);
    const float nb = sigmoidf_(nth[1]);
    if (na > nb - 1e-3f) {
      na = fmaxf(nb - 1e-3f, 1e-6f);
      nth[0] = logf(na / (1.f - na));
    }
    theta[b * 2] = nth[0];
    theta[b * 2 + 1] = nth[1];
    bounds[gi] = (float)T * na;
    bounds[gi + 1] = (float)T * nb;
  }
}

__global__ void mse_grad_kernel(const float *__restrict__ z, const float *__restrict__ y, long long n, float scale,
                                __nv_bfloat16 *__restrict__ dz, float *loss) {
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = z[i] - y[i];
    dz[i] = __float2bfloat16_rn(scale * d);
    s += d * d;
  }
  if (loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
  }
}

__global__ void relu_bwd_kernel(const float *__restrict__ da, const __nv_bfloat16 *__restrict__ act, long long n,
                                __nv_bfloat16 *__restrict__ dz) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dz[i] = __float2bfloat16_rn(__bfloat162float(act[i]) > 0.f ? da[i] : 0.f);
}

// one thread per column, rows walked in order (deterministic)
__global__ void colsum_kernel(const __nv_bfloat16 *__restrict__ dz, int M, int N, float *__restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += __bfloat162float(dz[(long long)m * N + n]);
  db[n] = s;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16 *__restrict__ pb) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(const float *__restrict__ x, long long n, __nv_bfloat16 *__restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void gather_rows_kernel(const float *__restrict__ src, long long n_src, const long long *__restrict__ idx,
                                   long long n_rows, int cols, float *__restrict__ dst) {
  const long long total = n_rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cols;
    const long long s = idx[r];
    dst[i] = (s >= 0 && s < n_src) ? src[s * cols + (i - r * cols)] : 0.f;
  }
}

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

float powi(float b, int e) {
  float r = 1.f;
  for (int i = 0; i < e && r > 0.f; ++i) r *= b;
  return r;
}

}  // namespace

extern "C" {

stl_status stl_rollout(const float *u, int64_t B, int32_t T, float dt, float *x, void *stream) {
  if (B < 0 || T < 1 || T > 65536) return stl_internal_fail(STL_ERR_INVALID_ARG, "need B >= 0 and T in [1, 65536]");
  if (B == 0) return STL_OK;
  if (!u || !x) return stl_internal_fail(STL_ERR_INVALID_ARG, "u / x is NULL");
  const int wpb = 4;
  rollout_kernel<<<(unsigned)((B + wpb - 1) / wpb), 32 * wpb, 0, (cudaStream_t)stream>>>(u, B, T, dt, x);
  return cuda_status(cudaGetLastError(), "rollout launch failed");
}

stl_status stl_plan_adam_step(float *u, float *m, float *v, const float *xbar, const int32_t *active, int64_t B,
                              int32_t T, float dt, float lr, float beta1, float beta2, float eps, int32_t step,
                              float *x, void *stream) {
  if (B < 0 || T < 1 || T > 65536) return stl_internal_fail(STL_ERR_INVALID_ARG, "need B >= 0 and T in [1, 65536]");
  if (step < 1) return stl_internal_fail(STL_ERR_INVALID_ARG, "step must be >= 1");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need 0 <= beta < 1 and eps > 0");
  if (B == 0) return STL_OK;
  if (!u || !m || !v || !xbar || !active || !x) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  const float c1 = 1.f / (1.f - powi(beta1, step)), c2 = 1.f / (1.f - powi(beta2, step));
  const int wpb = 4;
  plan_adam_kernel<<<(unsigned)((B + wpb - 1) / wpb), 32 * wpb, 0, (cudaStream_t)stream>>>(
      u, m, v, xbar, active, B, T, dt, lr, beta1, beta2, eps, c1, c2, x);
  return cuda_status(cudaGetLastError(), "plan Adam launch failed");
}

stl_status stl_plan_check(const float *rho_hard, int32_t *active, int32_t *solved_iter, int32_t iter, float *grad_out,
                          int64_t B, int32_t T, int32_t *n_active, void *stream) {
  if (B < 0 || T < 1) return stl_internal_fail(STL_ERR_INVALID_ARG, "need B >= 0 and T >= 1");
  if (B == 0) return STL_OK;
  if (!rho_hard || !active || !solved_iter || !grad_out) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  plan_check_kernel<<<(unsigned)((B + 255) / 256), 256, 0, (cudaStream_t)stream>>>(rho_hard, active, solved_iter, iter,
                                                                                  grad_out, B, T, n_active);
  return cuda_status(cudaGetLastError(), "plan check launch failed");
}

stl_status stl_trajopt_seed(const float *rho, const float *gam, int64_t B, int32_t T, float *grad_out, void *stream) {
  if (B < 0 || T < 1) return stl_internal_fail(STL_ERR_INVALID_ARG, "need B >= 0 and T >= 1");
  if (B == 0) return STL_OK;
  if (!rho || !gam || !grad_out) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  trajopt_seed_kernel<<<(unsigned)((B + 255) / 256), 256, 0, (cudaStream_t)stream>>>(rho, gam, B, T, grad_out);
  return cuda_status(cudaGetLastError(), "trajopt seed launch failed");
}

stl_status stl_trajopt_step(float *u, float *mu, float *vu, float *theta, float *mth, float *vth, const float *xbar,
                            const float *gbounds, const float *gam, int64_t B, int32_t T, int32_t n_slots, int32_t slot,
                            float dt, float start_x, float start_y, float u_max, float i_nom, float lr_u,
                            float lr_theta, int32_t step, float *x, float *bounds, void *stream) {
  if (B < 0 || T < 1 || T > 65536) return stl_internal_fail(STL_ERR_INVALID_ARG, "need B >= 0 and T in [1, 65536]");
  if (n_slots < 1 || slot < 0 || slot >= n_slots || step < 1)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need 0 <= slot < n_slots and step >= 1");
  if (B == 0) return STL_OK;
  if (!u || !mu || !vu || !theta || !mth || !vth || !xbar || !gbounds || !gam || !x || !bounds)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f / (1.f - powi(b1, step)), c2 = 1.f / (1.f - powi(b2, step));
  const int wpb = 4;
  trajopt_step_kernel<<<(unsigned)((B + wpb - 1) / wpb), 32 * wpb, 0, (cudaStream_t)stream>>>(
      u, mu, vu, theta, mth, vth, xbar, gbounds, gam, B, T, n_slots, slot, dt, start_x, start_y, u_max, i_nom, lr_u,
      lr_theta, b1, b2, 1e-8f, c1, c2, x, bounds);
  return cuda_status(cudaGetLastError(), "trajopt step launch failed");
}

stl_status stl_mse_grad(const float *z, const float *y, int64_t n, float scale, uint16_t *dz, float *loss,
                        void *stream) {
  if (n < 0) return stl_internal_fail(STL_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return STL_OK;
  if (!z || !y || !dz) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  mse_grad_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(z, y, n, scale,
                                                                      reinterpret_cast<__nv_bfloat16 *>(dz), loss);
  return cuda_status(cudaGetLastError(), "mse launch failed");
}

stl_status stl_relu_backward(const float *da, const uint16_t *act, int64_t n, uint16_t *dz, void *stream) {
  if (n < 0) return stl_internal_fail(STL_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return STL_OK;
  if (!da || !act || !dz) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  relu_bwd_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
      da, reinterpret_cast<const __nv_bfloat16 *>(act), n, reinterpret_cast<__nv_bfloat16 *>(dz));
  return cuda_status(cudaGetLastError(), "relu backward launch failed");
}

stl_status stl_colsum_bf16(const uint16_t *dz, int32_t M, int32_t N, float *db, void *stream) {
  if (M < 0 || N < 1) return stl_internal_fail(STL_ERR_INVALID_ARG, "need M >= 0 and N >= 1");
  if (!dz || !db) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  colsum_kernel<<<(unsigned)((N + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16 *>(dz), M, N, db);
  return cuda_status(cudaGetLastError(), "colsum launch failed");
}

stl_status stl_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2,
                    float eps, int32_t step, uint16_t *p_bf16, void *stream) {
  if (n < 0 || step < 1) return stl_internal_fail(STL_ERR_INVALID_ARG, "need n >= 0 and step >= 1");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need 0 <= beta < 1 and eps > 0");
  if (n == 0) return STL_OK;
  if (!p || !g || !m || !v) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  const float c1 = 1.f / (1.f - powi(beta1, step)), c2 = 1.f / (1.f - powi(beta2, step));
  adam_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2,
                                                                  reinterpret_cast<__nv_bfloat16 *>(p_bf16));
  return cuda_status(cudaGetLastError(), "adam launch failed");
}

stl_status stl_to_bf16(const float *x, int64_t n, uint16_t *y, void *stream) {
  if (n < 0) return stl_internal_fail(STL_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return STL_OK;
  if (!x || !y) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  to_bf16_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(x, n, reinterpret_cast<__nv_bfloat16 *>(y));
  return cuda_status(cudaGetLastError(), "bf16 conversion launch failed");
}

stl_status stl_gather_rows(const float *src, int64_t n_src, const int64_t *idx, int64_t n_rows, int32_t cols,
                           float *dst, void *stream) {
  if (n_rows < 0 || n_src < 0 || cols < 1)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "need n_rows, n_src >= 0 and cols >= 1");
  if (n_rows == 0) return STL_OK;
  if (!src || !idx || !dst) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  gather_rows_kernel<<<grid_for(n_rows * cols, 256), 256, 0, (cudaStream_t)stream>>>(
      src, n_src, reinterpret_cast<const long long *>(idx), n_rows, cols, dst);
  return cuda_status(cudaGetLastError(), "gather launch failed");
}

}  // extern "C"
