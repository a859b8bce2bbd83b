// stl_fk_dev.cuh -- building blocks of the formula-compiled kernels (hard semantics).
//
// For a hard-mode formula whose intervals are static, the library generates one CUDA kernel
// per formula and direction in which every node, window length, buffer offset and loop bound
// is a compile-time constant, and compiles it at run time for sm_103a (NVRTC).  This file is
// the device code those kernels instantiate; it is compiled only as part of the generated
// source and needs no header.
//
// The streaming scheme is that of the interpreter (stl_interp.cuh): one CTA walks a work item
// (trace, segment) in steps of TILE root samples; node n keeps its trace for the live range
// [t0 + LO, t1 + HI) of the step in a linear shared-memory buffer (sample p at p - (t0 + LO)),
// and the part that stays live is moved down by TILE after each step.  Reads past the end of
// the trace see pad-filled buffer words (Sec. IV-B: the last sample, or a constant), so no
// read is clamped or tested.  Windows use the thread-run decomposition (a thread owns R
// consecutive outputs: suffix of its first run, NF whole runs, prefix of a trailing run).
// Hard Until uses the composition of clamp functions
//   rho_t = min( min_{k<=a} phi_{t+k}, (f_{t+a} o ... o f_{t+b})(-inf) ),
//   f_j(v) = min(phi_j, max(psi_j, v)),
// which follows from min distributing over max in the Until of Sec. IV-C.
//
// Ties follow the oracle: windows select the earliest sample, and / or the left operand,
// Until the earliest maximising offset, phi winning min(phi, psi) ties, then the earliest
// minimiser inside the phi prefix.  Backward launches recompute every node's trace with the
// selected sample (stored as an offset from the output sample, 16 bits) and walk each root
// sample's selections down to one predicate sample, where its gradient is deposited as a
// 64-bit fixed-point integer: integer sums do not depend on the order of the deposits.

typedef unsigned long long fk_u64;
typedef long long fk_i64;
typedef unsigned short fk_u16;

#define FK_FULL 0xffffffffu

// Buffers.  In the bounds-checked build (FK_CHECK 1) every shared-memory buffer is a view that
// compares each index with the buffer's length; an index outside it is not performed (the
// access goes to element 0) and sets the library's device status word to -6
// (STL_ERR_DEVICE_CHECK).  The normal build uses plain pointers.
template <class T> struct FkChk {
  T *p;
  int cap, id;
  int *st;
  __device__ __forceinline__ T &operator[](int i) const {
    if ((unsigned)i >= (unsigned)cap) {
      if (st) atomicExch(st, -6);
      return p[0];
    }
    return p[i];
  }
};
#if FK_CHECK
#define FK_BUF(T) const FkChk<T>
#define FK_MAKE(T, ptr, cap, id) FkChk<T>{reinterpret_cast<T *>(ptr), (cap), (id), fk_status}
#define FK_PTR(b) ((b).p)
#else
#define FK_BUF(T) T *const
#define FK_MAKE(T, ptr, cap, id) reinterpret_cast<T *>(ptr)
#define FK_PTR(b) (b)
#endif

__device__ __forceinline__ float fk_inf() { return __int_as_float(0x7f800000); }

// ------------------------------------------------------------------ combine monoids
struct FkMax {
  typedef float T;
  static __device__ __forceinline__ float comb(float a, float b) { return b > a ? b : a; }
};
struct FkMin {
  typedef float T;
  static __device__ __forceinline__ float comb(float a, float b) { return b < a ? b : a; }
};
// value with the sample that supplies it; ties keep the left (earlier) operand
struct FkVP { float v; int p; };
struct FkMaxP {
  typedef FkVP T;
  static __device__ __forceinline__ FkVP comb(FkVP a, FkVP b) { return b.v > a.v ? b : a; }
};
struct FkMinP {
  typedef FkVP T;
  static __device__ __forceinline__ FkVP comb(FkVP a, FkVP b) { return b.v < a.v ? b : a; }
};
// clamp function v -> min(d, max(c, v)); comb(L, R) = L o R with L the earlier samples
struct FkC2 { float c, d; };
struct FkClamp {
  typedef FkC2 T;
  static __device__ __forceinline__ FkC2 comb(FkC2 L, FkC2 R) {
    FkC2 o;
    o.c = fminf(L.d, fmaxf(L.c, R.c));
    o.d = fminf(L.d, fmaxf(L.c, R.d));
    return o;
  }
};
// the same with the sources (2 * sample + child) of c and d; ties: the max keeps L's bound,
// the min keeps d
struct FkCC { float c, d; int cs, ds; };
struct FkClampP {
  typedef FkCC T;
  static __device__ __forceinline__ FkCC comb(FkCC L, FkCC R) {
    FkCC o;
    const bool rc = R.c > L.c;
    const float m = rc ? R.c : L.c;
    const int ms = rc ? R.cs : L.cs;
    const bool dl = L.d <= m;
    o.c = dl ? L.d : m;
    o.cs = dl ? L.ds : ms;
    const bool rd = R.d > L.c;
    const float m2 = rd ? R.d : L.c;
    const int ms2 = rd ? R.ds : L.cs;
    const bool dl2 = L.d <= m2;
    o.d = dl2 ? L.d : m2;
    o.ds = dl2 ? L.ds : ms2;
    return o;
  }
};

template <class M> struct FkIdem { static constexpr bool value = false; };
template <> struct FkIdem<FkMax> { static constexpr bool value = true; };
template <> struct FkIdem<FkMin> { static constexpr bool value = true; };
template <> struct FkIdem<FkMaxP> { static constexpr bool value = true; };
template <> struct FkIdem<FkMinP> { static constexpr bool value = true; };

// ------------------------------------------------------------------ windows
// Scratch entries needed by fk_window: run aggregates and their level-2 blocks.
template <int NT, int K, int R> struct FkScratch {
  static constexpr int NF = K / R - 1;
  static constexpr int entries = 2 * (NT + NF + 16);
};

// out(q, reduce_{i in [IA, IB]} elem(q + i)) for q in [q0, q1), combined in sample order.
// Long windows (K >= 2R): a thread owns R consecutive outputs u..u+R-1 of a pass of NT * R
// outputs; output u+k = suffix of the run at u+IA (hv[k]) (+) runs 1..NF of the following
// threads (+) a prefix of the samples after them.  With NF >= 24 whole runs the middle reads
// blocks of 8 runs: sliding (overlapping) blocks for the idempotent max / min, aligned ones
// for the clamp composition.  Threads whose runs no output uses read nothing; a pass reads
// at most R - 2 samples past the last child sample a live output needs (buffer slack).
// The caller synchronises after the call.
template <class M, int NT, int R, int IA, int IB, class Elem, class Out>
__device__ __forceinline__ void fk_window(int q0, int q1, const Elem &elem, const Out &out, void *scratch) {
  typedef typename M::T T;
  constexpr int K = IB - IA + 1;
  const int tid = threadIdx.x;
  if (q1 <= q0) return;
  if constexpr (K < 2 * R) {
    for (int q = q0 + tid; q < q1; q += NT) {
      T acc = elem(q + IA);
#pragma unroll
      for (int i = IA + 1; i <= IB; ++i) acc = M::comb(acc, elem(q + i));
      out(q, acc);
    }
  } else {
    constexpr int NF = K / R - 1;             // whole runs strictly inside every window
    constexpr int RHO = K - (NF + 1) * R;     // lead of the trailing prefix (0 <= RHO < R)
    constexpr int L2 = 8;
    constexpr bool TWO = NF >= 3 * L2;
    constexpr bool SLIDE = TWO && FkIdem<M>::value;
    T *ra = reinterpret_cast<T *>(scratch);
    T *a2 = ra + NT + NF + 8;
    for (int p0 = q0; p0 < q1; p0 += NT * R) {
      const int u = p0 + tid * R;
      const int nv = min(NT, (q1 - p0 + R - 1) / R);   // threads owning outputs in this pass
      const int nr = nv + NF;                          // run aggregates those outputs use
      T hv[R];
      if (tid < nr) {
        hv[R - 1] = elem(u + IA + R - 1);
#pragma unroll
        for (int k = R - 2; k >= 0; --k) hv[k] = M::comb(elem(u + IA + k), hv[k + 1]);
        ra[tid] = hv[0];
      }
      for (int e = NT + tid; e < nr; e += NT) {
        const int s = p0 + IA + e * R;
        T acc = elem(s);
#pragma unroll
        for (int k = 1; k < R; ++k) acc = M::comb(acc, elem(s + k));
        ra[e] = acc;
      }
      __syncthreads();
      if constexpr (SLIDE) {
        // a2[e] = runs e .. e+7
        for (int e = tid; e + L2 <= nr; e += NT) {
          T acc = ra[e];
#pragma unroll
          for (int k = 1; k < L2; ++k) acc = M::comb(acc, ra[e + k]);
          a2[e] = acc;
        }
        __syncthreads();
      } else if constexpr (TWO) {
        // a2[m] = runs 8m .. 8m+7
        for (int m = tid; (m + 1) * L2 <= nr; m += NT) {
          T acc = ra[m * L2];
#pragma unroll
          for (int k = 1; k < L2; ++k) acc = M::comb(acc, ra[m * L2 + k]);
          a2[m] = acc;
        }
        __syncthreads();
      }
      if (tid < nv) {
        // middle: runs tid+1 .. tid+NF
        T mid;
        if constexpr (SLIDE) {
          constexpr int NB = (NF + L2 - 1) / L2;   // blocks at tid+1, +9, ...; the last ends at tid+NF
          mid = a2[tid + 1];
#pragma unroll
          for (int i = 1; i < NB - 1; ++i) mid = M::comb(mid, a2[tid + 1 + i * L2]);
          mid = M::comb(mid, a2[tid + NF - L2 + 1]);
        } else if constexpr (TWO) {
          const int l = tid + 1, r = tid + NF;
          const int ml = (l + L2 - 1) / L2, mr = (r + 1) / L2 - 1;
          int j = l;
          if (j < ml * L2) {
            mid = ra[j++];
            for (; j < ml * L2; ++j) mid = M::comb(mid, ra[j]);
            mid = M::comb(mid, a2[ml]);
          } else {
            mid = a2[ml];
          }
          for (int m = ml + 1; m <= mr; ++m) mid = M::comb(mid, a2[m]);
          for (j = (mr + 1) * L2; j <= r; ++j) mid = M::comb(mid, ra[j]);
        } else {
          mid = ra[tid + 1];
#pragma unroll
          for (int i = 2; i <= NF; ++i) mid = M::comb(mid, ra[tid + i]);
        }
        // ma = middle (+) the trailing prefix of output u+k, extended by one sample per output
        const int gs = u + IA + (NF + 1) * R;
        T ma = mid;
#pragma unroll
        for (int e = 0; e < RHO; ++e) ma = M::comb(ma, elem(gs + e));
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (u + k < q1) out(u + k, M::comb(hv[k], ma));
          if (k + 1 < R) ma = M::comb(ma, elem(gs + RHO + k));
        }
      }
      if (p0 + NT * R < q1) __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ hard Until in one pass
// rho_q = min(A_q, X_q): A_q = min of phi over [q, q+IA] (MA, with its sample in backward
// launches), X_q = the clamp composition over offsets [IA, IB] (MC).  A thread's outputs
// u..u+R-1 take A from a sliding minimum over its own phi samples u..u+R+IA-1 held in
// registers (van Herk blocks of W = IA+1: suffix within the block of q, prefix within the
// next), so A needs no pass, buffer or barrier of its own.  out(q, X, A).
template <class M, int R, int W>
__device__ __forceinline__ void fk_slide_regs(const typename M::T (&e)[R + W - 1], typename M::T (&a)[R]) {
  typedef typename M::T T;
  constexpr int N = R + W - 1;
  T suf[N], pre[N];
#pragma unroll
  for (int i = N - 1; i >= 0; --i) suf[i] = (i % W == W - 1 || i == N - 1) ? e[i] : M::comb(e[i], suf[i + 1]);
#pragma unroll
  for (int i = 0; i < N; ++i) pre[i] = (i % W == 0) ? e[i] : M::comb(pre[i - 1], e[i]);
#pragma unroll
  for (int k = 0; k < R; ++k) a[k] = (k % W == 0) ? suf[k] : M::comb(suf[k], pre[k + W - 1]);
}

template <class MC, class MA, int NT, int R, int IA, int IB, class ElemC, class ElemA, class Out>
__device__ __forceinline__ void fk_until(int q0, int q1, const ElemC &elemc, const ElemA &elema, const Out &out,
                                         void *scratch) {
  typedef typename MC::T T;
  typedef typename MA::T TA;
  constexpr int K = IB - IA + 1;
  constexpr int W = IA + 1;
  const int tid = threadIdx.x;
  if (q1 <= q0) return;
  if constexpr (K < 2 * R) {
    for (int q = q0 + tid; q < q1; q += NT) {
      TA a = elema(q);
#pragma unroll
      for (int i = 1; i <= IA; ++i) a = MA::comb(a, elema(q + i));
      T acc = elemc(q + IA);
#pragma unroll
      for (int i = IA + 1; i <= IB; ++i) acc = MC::comb(acc, elemc(q + i));
      out(q, acc, a);
    }
  } else {
    constexpr int NF = K / R - 1;
    constexpr int RHO = K - (NF + 1) * R;
    constexpr int L2 = 8;
    constexpr bool TWO = NF >= 3 * L2;
    T *ra = reinterpret_cast<T *>(scratch);
    T *a2 = ra + NT + NF + 8;
    for (int p0 = q0; p0 < q1; p0 += NT * R) {
      const int u = p0 + tid * R;
      const int nv = min(NT, (q1 - p0 + R - 1) / R);
      const int nr = nv + NF;
      T hv[R];
      if (tid < nr) {
        hv[R - 1] = elemc(u + IA + R - 1);
#pragma unroll
        for (int k = R - 2; k >= 0; --k) hv[k] = MC::comb(elemc(u + IA + k), hv[k + 1]);
        ra[tid] = hv[0];
      }
      for (int e = NT + tid; e < nr; e += NT) {
        const int s = p0 + IA + e * R;
        T acc = elemc(s);
#pragma unroll
        for (int k = 1; k < R; ++k) acc = MC::comb(acc, elemc(s + k));
        ra[e] = acc;
      }
      __syncthreads();
      if constexpr (TWO) {
        for (int m = tid; (m + 1) * L2 <= nr; m += NT) {
          T acc = ra[m * L2];
#pragma unroll
          for (int k = 1; k < L2; ++k) acc = MC::comb(acc, ra[m * L2 + k]);
          a2[m] = acc;
        }
        __syncthreads();
      }
      if (tid < nv) {
        TA av[R];
        {
          TA ev[R + IA];
#pragma unroll
          for (int i = 0; i < R + IA; ++i) ev[i] = elema(u + i);
          fk_slide_regs<MA, R, W>(ev, av);
        }
        T mid;
        if constexpr (TWO) {
          const int l = tid + 1, r = tid + NF;
          const int ml = (l + L2 - 1) / L2, mr = (r + 1) / L2 - 1;
          int j = l;
          if (j < ml * L2) {
            mid = ra[j++];
            for (; j < ml * L2; ++j) mid = MC::comb(mid, ra[j]);
            mid = MC::comb(mid, a2[ml]);
          } else {
            mid = a2[ml];
          }
          for (int m = ml + 1; m <= mr; ++m) mid = MC::comb(mid, a2[m]);
          for (j = (mr + 1) * L2; j <= r; ++j) mid = MC::comb(mid, ra[j]);
        } else {
          mid = ra[tid + 1];
#pragma unroll
          for (int i = 2; i <= NF; ++i) mid = MC::comb(mid, ra[tid + i]);
        }
        const int gs = u + IA + (NF + 1) * R;
        T ma = mid;
#pragma unroll
        for (int e = 0; e < RHO; ++e) ma = MC::comb(ma, elemc(gs + e));
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (u + k < q1) out(u + k, MC::comb(hv[k], ma), av[k]);
          if (k + 1 < R) ma = MC::comb(ma, elemc(gs + RHO + k));
        }
      }
      if (p0 + NT * R < q1) __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ elementwise passes
template <int NT, class F>
__device__ __forceinline__ void fk_each(int q0, int q1, const F &f) {
  for (int q = q0 + threadIdx.x; q < q1; q += NT) f(q);
}

// fill words [f0, f1) of a float buffer with v
template <int NT>
__device__ __forceinline__ void fk_fill(float *p, int f0, int f1, float v) {
  for (int i = f0 + threadIdx.x; i < f1; i += NT) p[i] = v;
}
template <int NT>
__device__ __forceinline__ void fk_fill16(fk_u16 *p, int f0, int f1, fk_u16 v) {
  for (int i = f0 + threadIdx.x; i < f1; i += NT) p[i] = v;
}

// ------------------------------------------------------------------ buffer moves
// One round of moving words [SRC, SRC + LEN) of p down to [0, LEN): the round copies words
// [C0 + SRC, C0 + SRC + n) to [C0, C0 + n), n = min(SRC, LEN - C0), so that a round's source
// and destination never overlap; the caller synchronises between rounds.  p is 16-byte
// aligned; SRC and C0 are multiples of 4 (16-byte copies).
template <int NT, int SRC, int C0, int LEN>
__device__ __forceinline__ void fk_move_round(float *p) {
  constexpr int n = (SRC < LEN - C0) ? SRC : LEN - C0;
  static_assert((SRC & 3) == 0 && (C0 & 3) == 0, "aligned moves");
  float *d = p + C0;
  const float *s = p + C0 + SRC;
  constexpr int nv = n >> 2;
  float4 *d4 = reinterpret_cast<float4 *>(d);
  const float4 *s4 = reinterpret_cast<const float4 *>(s);
  for (int i = threadIdx.x; i < nv; i += NT) d4[i] = s4[i];
  for (int i = 4 * nv + threadIdx.x; i < n; i += NT) d[i] = s[i];
}

template <int NT>
__device__ __forceinline__ void fk_zero(float *p, int w0, int w1) {
  int a = (w0 + 3) & ~3;
  if (a > w1) a = w1;
  for (int i = w0 + threadIdx.x; i < a; i += NT) p[i] = 0.f;
  const int nv = (w1 - a) >> 2;
  float4 *p4 = reinterpret_cast<float4 *>(p + a);
  for (int i = threadIdx.x; i < nv; i += NT) p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = a + 4 * nv + threadIdx.x; i < w1; i += NT) p[i] = 0.f;
}

// ------------------------------------------------------------------ fixed point
// Per trace, k is chosen from the largest root gradient M of the whole trace: M 2^k < 2^30,
// so a sum of up to 2^30 deposits stays below 2^61.  Each root gradient is scaled by 2^k (two
// exact power-of-two factors) and rounded to an integer before any addition.
struct FkFix { float f1, f2, i1, i2; };
__device__ __forceinline__ FkFix fk_fix_scale(float M) {
  const int k = M > 0.f ? 29 - ilogbf(M) : 0;
  const int k1 = k / 2, k2 = k - k1;
  FkFix s;
  s.f1 = ldexpf(1.f, k1);
  s.f2 = ldexpf(1.f, k2);
  s.i1 = ldexpf(1.f, -k1);
  s.i2 = ldexpf(1.f, -k2);
  return s;
}
__device__ __forceinline__ fk_i64 fk_to_fix(const FkFix &s, float v) { return __float2ll_rn((v * s.f1) * s.f2); }
__device__ __forceinline__ float fk_from_fix(const FkFix &s, fk_u64 a) {
  return (__ll2float_rn((fk_i64)a) * s.i1) * s.i2;
}
__device__ __forceinline__ void fk_red_add(fk_u64 *p, fk_i64 v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

// largest |g| over a trace's root gradients; the loads keep the row in L2 (evict-last): the
// walk reads it again step by step
template <int NT>
__device__ __forceinline__ float fk_trace_gmax(const float *g, int T) {
  fk_u64 pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  const int head = min((int)(((16 - (reinterpret_cast<unsigned long long>(g) & 15)) & 15) >> 2), T);
  float m = 0.f;
  for (int q = threadIdx.x; q < head; q += NT) m = fmaxf(m, fabsf(g[q]));
  const float4 *g4 = reinterpret_cast<const float4 *>(g + head);
  const int nv = (T - head) >> 2;
#pragma unroll 4
  for (int i = threadIdx.x; i < nv; i += NT) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(g4 + i), "l"(pol));
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int q = head + 4 * nv + threadIdx.x; q < T; q += NT) m = fmaxf(m, fabsf(g[q]));
  return m;
}

// Asynchronous L2 prefetch of the 16-byte aligned part of [p0, p1), kept inside [lo, hi) (the
// allocation); one thread issues it.
__device__ __forceinline__ void fk_prefetch_l2(const float *p0, const float *p1, const float *lo, const float *hi) {
  unsigned long long a = reinterpret_cast<unsigned long long>(p0), e = reinterpret_cast<unsigned long long>(p1);
  const unsigned long long l = (reinterpret_cast<unsigned long long>(lo) + 15) & ~15ull;
  const unsigned long long h = reinterpret_cast<unsigned long long>(hi) & ~15ull;
  a = (a + 15) & ~15ull;
  e &= ~15ull;
  if (a < l) a = l;
  if (e > h) e = h;
  if (e <= a) return;
  const unsigned n = (unsigned)min(e - a, 1ull << 20);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
}

__device__ __forceinline__ float fk_ldg_first(const float *p, fk_u64 pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
