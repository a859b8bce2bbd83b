// stl_gemm.cu -- the BF16 matrix product of the warm-start MLP on the 5th-generation tensor
// cores of sm_103a: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in tensor
// memory), one CTA per 128 x 128 output tile (cta_group::1, no clusters, no multicast).
//
// Data path of one CTA (128 threads = 4 warps):
//   1. warp 0 allocates 128 tensor-memory columns (the 128 x 128 FP32 accumulator);
//   2. per K block of 64: all threads stage op(A)[m0.., k..] and op(B)^T[n0.., k..] into
//      shared memory as K-major tiles in the 128-byte swizzled layout (row r, 16-byte chunk c
//      at r*128 + ((c ^ (r & 7)) * 16); 8-row atoms of 1024 bytes), make the stores visible
//      to the tensor core's (async) proxy, and one thread issues four 128x128x16 MMAs whose
//      completion it commits to that stage's mbarrier.  Two stages: staging block k+1
//      overlaps the MMAs of block k;
//   3. after the last commit, each warp reads its 32 accumulator rows (tensor-memory lanes
//      32w..32w+31) with tcgen05.ld, adds the bias, applies ReLU and stores FP32 and/or BF16.
// Every mbarrier wait is bounded: on a timeout the kernel records STL_ERR_TIMEOUT in the
// device status word, skips the accumulator reads, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "stl_internal.cuh"
#include "stl_plan.h"

stl_status stl_internal_fail(stl_status st, const char *msg);

namespace {

constexpr int TM = 128, TN = 128;   // output tile
constexpr int TKB = 64;             // K block: 64 bf16 = one 128-byte swizzle row
constexpr int UK = 16;              // K of one kind::f16 MMA
constexpr int TILE_BYTES = TM * TKB * 2;   // 16 KB per operand tile (TN == TM)
constexpr int SMEM_BYTES = 4 * TILE_BYTES + 1024;   // two stages of A and B, 1024-byte alignment
constexpr unsigned kWaitPolls = 1u << 26;          // bounded mbarrier waits (far beyond any MMA)

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a K-major tile in the 128-byte swizzled layout: start
// address (>> 4) in bits 0-13, leading byte offset 16 B (unused by this layout) in bits 16-29,
// stride byte offset 1024 B (between 8-row atoms) in bits 32-45, descriptor version 1 in bits
// 46-47, layout "128-byte swizzle" (2) in bits 61-63.  A K step of 16 elements (32 bytes)
// advances the start address by 2 units.
__device__ __forceinline__ uint64_t sw128_desc(unsigned addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// wait until phase `parity` of the barrier has completed; false after kWaitPolls polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (unsigned i = 0; i < kWaitPolls; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's row (lane) from tensor memory
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage rows [row0, row0 + 128) x K block [k0, k0 + 64) of a matrix X read as X(r, k) into a
// K-major swizzled tile.  kcontig: X(r, k) = X[r * ld + k] (16-byte chunks load as one vector
// when aligned and in bounds); otherwise X(r, k) = X[k * ld + r], read as 16-byte vectors along
// r (16 threads cover 256 contiguous bytes of one k) and transposed on the way into the tile.
// Out-of-range entries are 0.  vec_ok: ld is a multiple of 8 and X 16-byte aligned.
__device__ __forceinline__ void stage_tile(uint8_t *tile, const __nv_bfloat16 *__restrict__ X, int ld, bool kcontig,
                                           int row0, int R, int k0, int K, bool vec_ok) {
  const unsigned short *Xs = reinterpret_cast<const unsigned short *>(X);
  if (!kcontig) {
#pragma unroll
    for (int i = 0; i < (TM * TKB / 8) / 128; ++i) {
      const int idx = threadIdx.x + i * 128;
      const int c8 = idx & 15, k = idx >> 4;   // rows 8 c8 .. 8 c8 + 7, column k of the block
      const int gk = k0 + k, gr = row0 + 8 * c8;
      unsigned short e[8];
      if (gk < K && vec_ok && gr + 8 <= R) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(Xs + (long long)gk * ld + gr));
        e[0] = v.x & 0xffffu; e[1] = v.x >> 16; e[2] = v.y & 0xffffu; e[3] = v.y >> 16;
        e[4] = v.z & 0xffffu; e[5] = v.z >> 16; e[6] = v.w & 0xffffu; e[7] = v.w >> 16;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          e[j] = (gk < K && gr + j < R) ? Xs[(long long)gk * ld + gr + j] : (unsigned short)0;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = 8 * c8 + j;
        *reinterpret_cast<unsigned short *>(tile + r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + (k & 7) * 2) = e[j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < (TM * TKB / 8) / 128; ++i) {
    const int idx = threadIdx.x + i * 128;
    const int r = idx >> 3, c = idx & 7;
    const int gr = row0 + r, gk = k0 + 8 * c;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < R && gk < K) {
      if (vec_ok && gk + 8 <= K) {
        v = __ldg(reinterpret_cast<const uint4 *>(Xs + (long long)gr * ld + gk));
      } else {
        unsigned short e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int kk = gk + j;
          e[j] = kk < K ? Xs[(long long)gr * ld + kk] : (unsigned short)0;
        }
        v.x = e[0] | ((unsigned)e[1] << 16);
        v.y = e[2] | ((unsigned)e[3] << 16);
        v.z = e[4] | ((unsigned)e[5] << 16);
        v.w = e[6] | ((unsigned)e[7] << 16);
      }
    }
    *reinterpret_cast<uint4 *>(tile + r * 128 + ((c ^ (r & 7)) << 4)) = v;
  }
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(const __nv_bfloat16 *__restrict__ A, int lda, int ta,
                                                      const __nv_bfloat16 *__restrict__ Bm, int ldb, int tb, int M,
                                                      int N, int K, const float *__restrict__ bias, int relu,
                                                      float *__restrict__ Cf, __nv_bfloat16 *__restrict__ Cb, int ldc,
                                                      int a_vec, int b_vec, int *status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ unsigned tmem_slot;
  __shared__ int s_fail;
  // 1024-byte aligned in the shared address space (the swizzle pattern follows address bits 4-9)
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sA[2] = {smem, smem + TILE_BYTES};
  uint8_t *sB[2] = {smem + 2 * TILE_BYTES, smem + 3 * TILE_BYTES};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;

  const int nk = (K + TKB - 1) / TKB;
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb & 1;
    if (kb >= 2 && !mbar_wait(&bar[s], ((kb - 2) >> 1) & 1)) s_fail = 1;   // stage s free again
    const int k0 = kb * TKB;
    stage_tile(sA[s], A, lda, !ta, m0, M, k0, K, a_vec != 0);
    stage_tile(sB[s], Bm, ldb, tb != 0, n0, N, k0, K, b_vec != 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor core reads
    __syncthreads();
    if (tid == 0 && !s_fail) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = sw128_desc(smem_u32(sA[s])), db = sw128_desc(smem_u32(sB[s]));
#pragma unroll
      for (int k = 0; k < TKB / UK; ++k)   // +32 bytes per K step of 16 = +2 in the address field
        mma_bf16(tmem, da + 2 * k, db + 2 * k, (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(&bar[s]);
    }
  }
  bool ok = true;
  if (nk > 0) ok = mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1);   // the last commit covers all MMAs
  if (!ok) s_fail = 1;
  __syncthreads();
  const bool failed = s_fail != 0;
  if (failed && tid == 0 && status) atomicExch(status, 2);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w holds accumulator rows 32w..32w+31 (tensor-memory lanes), one per lane
  const int row = m0 + warp * 32 + lane;
  const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
  for (int cb = 0; cb < TN; cb += 16) {
    float v[16];
    if (nk > 0 && !failed) {
      tmem_ld16(trow + cb, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
    if (row >= M || failed) continue;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int col = n0 + cb + i;
      if (col >= N) break;
      float val = v[i];
      if (bias) val += bias[col];
      if (relu) val = fmaxf(val, 0.f);
      if (Cf) Cf[(long long)row * ldc + col] = val;
      if (Cb) Cb[(long long)row * ldc + col] = __float2bfloat16_rn(val);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

}  // namespace

extern "C" {

stl_status stl_gemm_bf16(const uint16_t *a, int32_t lda, int32_t trans_a, const uint16_t *b, int32_t ldb,
                         int32_t trans_b, int32_t M, int32_t N, int32_t K, const float *bias, int32_t relu, float *c_f32,
                         uint16_t *c_bf16, int32_t ldc, void *stream) {
  const int lim = 1 << 20;
  if (M < 1 || N < 1 || K < 1 || M > lim || N > lim || K > lim)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "M, N, K must be in [1, 2^20]");
  if (!a || !b || (!c_f32 && !c_bf16)) return stl_internal_fail(STL_ERR_INVALID_ARG, "NULL argument");
  if (lda < (trans_a ? M : K) || ldb < (trans_b ? K : N) || ldc < N)
    return stl_internal_fail(STL_ERR_INVALID_ARG, "leading dimension too small");
  int *status = nullptr;
  int e = stl_status_ptr(&status);
  if (e) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString((cudaError_t)e));
  cudaError_t ce = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (ce != cudaSuccess) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString(ce));
  // 16-byte vector loads (along K or along the rows) need 16-byte aligned rows
  const int a_vec = (lda % 8 == 0) && ((reinterpret_cast<uintptr_t>(a) & 15) == 0);
  const int b_vec = (ldb % 8 == 0) && ((reinterpret_cast<uintptr_t>(b) & 15) == 0);
  dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM));
  gemm_tc_kernel<<<grid, 128, SMEM_BYTES, (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16 *>(a), lda, trans_a ? 1 : 0, reinterpret_cast<const __nv_bfloat16 *>(b), ldb,
      trans_b ? 1 : 0, M, N, K, bias, relu ? 1 : 0, c_f32, reinterpret_cast<__nv_bfloat16 *>(c_bf16), ldc, a_vec, b_vec,
      status);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return stl_internal_fail(STL_ERR_CUDA, cudaGetErrorString(ce));
  return STL_OK;
}

}  // extern "C"
