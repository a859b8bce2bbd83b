// stl_interp.cuh -- streaming tile interpreter for STL robustness traces and their adjoints
// on sm_103a.
//
// One CTA owns one work item (trace b, segment [s0, s1)) at a time and walks it in steps of
// `tile` samples.  Every node of the formula keeps its robustness trace in a linear buffer
// (shared memory when it fits) covering the live range [t0 + lo, t1 + hi) of the step:
// sample p sits at index p - (t0 + lo).  Between steps the `hi - lo` samples that stay live
// are moved down by one tile.  Intermediate traces therefore never touch HBM: only the
// signal is read and only the root trace (forward) or the signal gradient (backward) is
// written.
//
// Temporal operators use a "thread-run" sliding-window decomposition: a thread owns R
// consecutive outputs; each output window is the combination of a suffix of the thread's
// first run, a fixed set of whole runs (shared through a small scratch array, combined
// directly or through blocks of 8 runs) and a prefix of a trailing run.  This is O(1) work
// per output for any window length and works for every associative combine used here:
//   max/min, with the earliest selected sample when gradients are needed (Eventually, Always)
//   composition of clamp functions f_j(v) = min(phi_j, max(psi_j, v))       (hard Until)
//   (max, scaled sum) pairs of logsumexp                  (smooth windows and their adjoint)
// The hard Until rests on  rho_t = min( min_{k<=a} phi_{t+k},
//                                       (f_{t+a} o ... o f_{t+b})(-inf) ),
// which follows from min distributing over max in the definition of Sec. IV-C.  R = 7 (15
// for long windows in the direct-read forward passes) is odd, so the strided runs of a warp
// fall in distinct shared-memory banks.
//
// Backward launches recompute the forward trace of every node step by step (values run
// ahead of the root by `hi`), and propagate adjoints in reverse order over the samples whose
// adjoint is complete (they lag behind by `lo`).  Sample T-1 of every node collects the
// gradient of all pad reads and is finished once at the end of the trace.
#pragma once
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include <type_traits>

#include "stl_internal.cuh"

namespace {

enum {
  OP_PGT = 0, OP_PLT = 1, OP_TRUE = 2, OP_NOT = 3, OP_AND = 4, OP_OR = 5, OP_EV = 6,
  OP_ALW = 7, OP_UNTIL = 8, OP_EVSM = 9, OP_ALWSM = 10, OP_NGT = 11, OP_NLT = 12, OP_UNTSM = 13
};

__device__ __forceinline__ bool is_until_op(int op) { return op == OP_UNTIL || op == OP_UNTSM; }

__device__ __forceinline__ bool is_pred_op(int op) { return op == OP_PGT || op == OP_PLT || op == OP_NGT || op == OP_NLT; }

constexpr unsigned FULL = 0xffffffffu;
constexpr int L2B = 8;   // runs per level-2 block in the window middle

// Float add into a node buffer or cell, which lives in shared memory unless its ring was
// spilled to the global workspace: a shared-space reduction when the address is shared (a
// generic atomic on a shared address is much slower), a global atomic otherwise.
__device__ __forceinline__ void buf_add(float *p, float v) {
  if (__isShared(p)) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
  } else {
    atomicAdd(p, v);
  }
}

// ------------------------------------------------------------------ combine monoids
struct MaxV {
  using T = float;
  static __device__ __forceinline__ T comb(T a, T b) { return b > a ? b : a; }
};
struct MinV {
  using T = float;
  static __device__ __forceinline__ T comb(T a, T b) { return b < a ? b : a; }
};
struct VI { float v; int i; };
struct MaxI {
  using T = VI;
  static __device__ __forceinline__ T comb(T a, T b) { return b.v > a.v ? b : a; }
};
struct MinI {
  using T = VI;
  static __device__ __forceinline__ T comb(T a, T b) { return b.v < a.v ? b : a; }
};

// clamp function v -> min(d, max(c, v)); comb(L, R) = L o R (L covers the earlier samples)
struct C2 { float c, d; };
struct ClampV {
  using T = C2;
  static __device__ __forceinline__ T comb(T L, T R) {
    T o;
    o.c = fminf(L.d, fmaxf(L.c, R.c));
    o.d = fminf(L.d, fmaxf(L.c, R.d));
    return o;
  }
};
// with the samples that supply c and d; ties: max keeps L's bound, min keeps d
struct CC { float c, d; int cs, ds; };
struct ClampI {
  using T = CC;
  static __device__ __forceinline__ T comb(T L, T R) {
    T o;
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

// logsumexp pair: value = m + log(s); s may be signed in the adjoint use
struct LS { float m, s; };
struct LseM {
  using T = LS;
  static __device__ __forceinline__ T comb(T a, T b) {
    if (b.m == -INFINITY) return a;
    if (a.m == -INFINITY) return b;
    T o;
    if (b.m > a.m) { o.m = b.m; o.s = fmaf(a.s, __expf(a.m - b.m), b.s); }
    else { o.m = a.m; o.s = fmaf(b.s, __expf(b.m - a.m), a.s); }
    return o;
  }
};

// the same pair with the scaled sum in double: the transposed (adjoint) windows sum upstream
// gradients of both signs over up to thousands of outputs, where a float sum loses digits to
// cancellation
struct LSd { float m; double s; };
struct LsdM {
  using T = LSd;
  static __device__ __forceinline__ T comb(T a, T b) {
    if (b.m == -INFINITY) return a;
    if (a.m == -INFINITY) return b;
    T o;
    if (b.m > a.m) { o.m = b.m; o.s = fma(a.s, (double)__expf(a.m - b.m), b.s); }
    else { o.m = a.m; o.s = fma(b.s, (double)__expf(b.m - a.m), a.s); }
    return o;
  }
};

// softmax-weighted reduction (Sec. III-C "soft" max / min): (m, s, n) = (largest exponent
// z = sgn tau v seen, sum e^{z - m}, sum v e^{z - m}); the value is n / s.  An entry with
// z = +inf dominates (kept with s = 1, n = its value), z = -inf carries no weight.
struct SW { float m, s, n; };
struct SwM {
  using T = SW;
  static __device__ __forceinline__ T comb(T a, T b) {
    if (b.m == -INFINITY || a.m == INFINITY) return a;
    if (a.m == -INFINITY || b.m == INFINITY) return b;
    T o;
    if (b.m > a.m) {
      const float f = __expf(a.m - b.m);
      o.m = b.m; o.s = fmaf(a.s, f, b.s); o.n = fmaf(a.n, f, b.n);
    } else {
      const float f = __expf(b.m - a.m);
      o.m = a.m; o.s = fmaf(b.s, f, a.s); o.n = fmaf(b.n, f, a.n);
    }
    return o;
  }
};
__device__ __forceinline__ SW sw_elem(float v, float st) {
  const float z = st * v;
  SW r;
  if (z == -INFINITY) { r.m = -INFINITY; r.s = 0.f; r.n = 0.f; }
  else { r.m = z; r.s = 1.f; r.n = v; }
  return r;
}
// value of a reduction with sign sgn (an empty one is -sgn inf); lse = log sum e^{z}
__device__ __forceinline__ float sw_value(const SW &r, float sgn) {
  if (r.m == INFINITY) return r.n;
  if (r.m == -INFINITY) return -sgn * INFINITY;
  return r.n / r.s;
}
__device__ __forceinline__ float sw_lse(const SW &r) {
  return (r.m == INFINITY || r.m == -INFINITY) ? r.m : r.m + __logf(r.s);
}
// softmax-weighted min (sg = -1) or max (sg = +1) of two values, and the weight of the first
__device__ __forceinline__ float sw2(float a, float b, float sg, float tau, float &wa) {
  if (a == b) { wa = 0.5f; return a; }
  if (sg * a == INFINITY || sg * b == -INFINITY) { wa = 1.f; return a; }
  if (sg * b == INFINITY || sg * a == -INFINITY) { wa = 0.f; return b; }
  wa = 1.f / (1.f + __expf(-sg * tau * (a - b)));
  return fmaf(wa, a - b, b);
}
// a running softmax-weighted reduction with its sums in double (sequential, per thread)
struct SWd {
  float m = -INFINITY;
  double s = 0.0, n = 0.0;
  float inf_v = 0.f;
  bool has_inf = false;
  __device__ __forceinline__ void add(float v, float st, float w = 1.f) {   // w: weight (> 0)
    const float z = st * v;
    if (z == -INFINITY) return;
    if (z == INFINITY) { if (!has_inf) inf_v = v; has_inf = true; return; }
    if (z > m) {
      const double f = (double)__expf(m - z);
      s = fma(s, f, (double)w);
      n = fma(n, f, (double)w * (double)v);
      m = z;
    } else {
      const double e = (double)w * (double)__expf(z - m);
      s += e;
      n = fma(e, (double)v, n);
    }
  }
  __device__ __forceinline__ float value(float sgn) const {
    if (has_inf) return inf_v;
    if (m == -INFINITY) return -sgn * INFINITY;
    return (float)(n / s);
  }
  __device__ __forceinline__ float lse() const {   // float log: s is a sum of terms in (0, 1]
    if (has_inf) return INFINITY;
    return m == -INFINITY ? -INFINITY : m + __logf((float)s);
  }
};

// d y / d v of a softmax-weighted reduction for an entry of weight w: w (1 + sgn tau (v - y))
__device__ __forceinline__ float sw_grad(float w, float v, float y, float st) {
  if (w == 0.f) return 0.f;
  if (isinf(v) || isinf(y)) return w;
  return w * fmaf(st, v - y, 1.f);
}

// two signed sums sharing one scale (the transposed softmax-weighted window).  The sums are
// kept in double: the adjoint combines them as s1 + tau x s2, which cancels by about tau |y|.
struct LS2 { float m; double s1, s2; };
struct Lse2M {
  using T = LS2;
  static __device__ __forceinline__ T comb(T a, T b) {
    if (b.m == -INFINITY) return a;
    if (a.m == -INFINITY) return b;
    T o;
    if (b.m > a.m) {
      const double f = (double)__expf(a.m - b.m);
      o.m = b.m; o.s1 = fma(a.s1, f, b.s1); o.s2 = fma(a.s2, f, b.s2);
    } else {
      const double f = (double)__expf(b.m - a.m);
      o.m = a.m; o.s1 = fma(b.s1, f, a.s1); o.s2 = fma(b.s2, f, a.s2);
    }
    return o;
  }
};

// The host sizes the window scratch for entries of 16 bytes (24 in softmax-weighted backward
// launches, the only users of LS2).
static_assert(sizeof(VI) <= 16 && sizeof(C2) <= 16 && sizeof(CC) <= 16 && sizeof(LS) <= 16 && sizeof(SW) <= 16 &&
                  sizeof(LSd) <= 16,
              "window aggregates must fit the 16-byte scratch entries");
static_assert(sizeof(LS2) <= 24, "softmax adjoint aggregates must fit the 24-byte scratch entries");

// ------------------------------------------------------------------ window framework
// middle combine of runagg[l .. r] (inclusive, in order), directly or via level-2 blocks
template <class M>
__device__ __forceinline__ typename M::T middle(const typename M::T *ra, const typename M::T *a2, int l, int r,
                                               bool two_level) {
  using T = typename M::T;
  if (!two_level) {
    T acc = ra[l];
    for (int j = l + 1; j <= r; ++j) acc = M::comb(acc, ra[j]);
    return acc;
  }
  const int ml = (l + L2B - 1) / L2B;   // first whole block
  const int mr = (r + 1) / L2B - 1;     // last whole block (ml <= mr since r - l + 1 >= 2*L2B)
  T acc;
  int j = l;
  if (j < ml * L2B) {
    acc = ra[j++];
    for (; j < ml * L2B; ++j) acc = M::comb(acc, ra[j]);
    acc = M::comb(acc, a2[ml]);
  } else {
    acc = a2[ml];
  }
  for (int m = ml + 1; m <= mr; ++m) acc = M::comb(acc, a2[m]);
  for (j = (mr + 1) * L2B; j <= r; ++j) acc = M::comb(acc, ra[j]);
  return acc;
}

// out(q, reduce_{i in [ia, ib]} elem(q + i)) for q in [q0, q1), combining in sample order.
// scratch holds the run aggregates (max(NT, nv + nf) entries) then the level-2 aggregates.
template <class M, int R, class Elem, class Out>
__device__ __forceinline__ void window_reduce(int q0, int q1, int ia, int ib, const Elem &elem,
                                              const Out &out, void *scratch) {
  using T = typename M::T;
  const int K = ib - ia + 1;
  const int tid = threadIdx.x, NT = blockDim.x;
  if (q1 <= q0) return;
  if (K < 2 * R) {
    for (int q = q0 + tid; q < q1; q += NT) {
      T acc = elem(q + ia);
      for (int i = ia + 1; i <= ib; ++i) acc = M::comb(acc, elem(q + i));
      out(q, acc);
    }
    return;
  }
  T *runagg = reinterpret_cast<T *>(scratch);
  const int nf = K / R - 1;           // whole runs strictly inside every window (>= 1)
  const int rho = K - (nf + 1) * R;   // lead of the trailing prefix
  const bool two = nf >= 3 * L2B;
  for (int p0 = q0; p0 < q1; p0 += NT * R) {
    const int u = p0 + tid * R;
    const int nv = min(NT, (q1 - p0 + R - 1) / R);   // threads that own outputs in this pass
    const int nruns = max(NT, nv + nf);
    T *agg2 = runagg + nruns;
    T hv[R];
    hv[R - 1] = elem(u + ia + R - 1);
#pragma unroll
    for (int k = R - 2; k >= 0; --k) hv[k] = M::comb(elem(u + ia + k), hv[k + 1]);
    runagg[tid] = hv[0];
    for (int e = NT + tid; e < nv + nf; e += NT) {
      const int s = p0 + ia + e * R;
      T acc = elem(s);
#pragma unroll
      for (int k = 1; k < R; ++k) acc = M::comb(acc, elem(s + k));
      runagg[e] = acc;
    }
    __syncthreads();
    if (two) {
      const int nb = (nv + nf) / L2B;
      for (int m = tid; m < nb; m += NT) {
        T acc = runagg[m * L2B];
#pragma unroll
        for (int k = 1; k < L2B; ++k) acc = M::comb(acc, runagg[m * L2B + k]);
        agg2[m] = acc;
      }
      __syncthreads();
    }
    if (tid < nv) {
      const T mid = middle<M>(runagg, agg2, tid + 1, tid + nf, two);
      const int gs = u + ia + (nf + 1) * R;
      T acc = mid;
      bool have = rho > 0;
      if (have) {
        acc = elem(gs);
        for (int e = 1; e < rho; ++e) acc = M::comb(acc, elem(gs + e));
      }
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (u + k < q1) {
          T r = M::comb(hv[k], mid);
          if (have) r = M::comb(r, acc);
          out(u + k, r);
        }
        if (k + 1 < R) {
          T e = elem(gs + rho + k);
          acc = have ? M::comb(acc, e) : e;
          have = true;
        }
      }
    }
    if (p0 + NT * R < q1) __syncthreads();   // the caller synchronises after the last pass
  }
}

constexpr int RUN = 7;   // thread-run length (odd)

// Short hard windows (6 <= K < 2 RUN) use runs of 3: about two child reads per output instead
// of the K of the direct loop.
template <class M> struct ShortRuns {
  static constexpr bool value = std::is_same<M, MaxV>::value || std::is_same<M, MinV>::value ||
                                std::is_same<M, MaxI>::value || std::is_same<M, MinI>::value;
};

template <class M, class Elem, class Out>
__device__ __forceinline__ void window_any(int K, int q0, int q1, int ia, int ib, const Elem &elem,
                                           const Out &out, void *scratch) {
  if constexpr (ShortRuns<M>::value) {
    if (K >= 6 && K < 2 * RUN) {
      window_reduce<M, 3>(q0, q1, ia, ib, elem, out, scratch);
      return;
    }
  }
  window_reduce<M, RUN>(q0, q1, ia, ib, elem, out, scratch);
}

// ------------------------------------------------------------------ interpreter state
struct Cta {
  const KProgram *P;
  NodeRt *rt;
  void *scratch;
  const float *sig;
  long long b;         // trace index (bounds row)
  long long row0;      // first sample row of the trace in the (packed) signal
  int T;
  int t0, t1;          // current root step [t0, t1)
  int root;
  float *out_row;      // forward: out + b*T
  bool fx;             // adjoint buffers hold 64-bit fixed point (hard and logsumexp backward)
  float fx1, fx2;      // fixed-point scale 2^k = fx1 * fx2 of this work item
  float ifx1, ifx2;    // and its inverse
};

// Hard-mode adjoints are summed in 64-bit fixed point, so that the result depends neither on
// the order in which warps deposit nor on the launch shape (integer addition is associative;
// float addition is not).  Per trace, k is chosen from the largest root gradient M of the
// whole trace: M * 2^k < 2^30, so a sum of up to 2^30 deposits (T <= 2^30) stays below 2^61,
// and the resolution 2^-k is below 2^-29 M.  Each root gradient is scaled by 2^k (exact: two
// powers of two, each representable) and rounded to an integer before any addition; a read
// converts the integer sum to float once and scales it back (exact).  The gradient is thus
// the float rounding of sum_q round(g_q 2^k) 2^-k, bit-identical for every tile, CTA size,
// segmentation and deposit order.
__device__ __forceinline__ void set_fix_scale(Cta &C, float M) {
  const int k = M > 0.f ? 29 - ilogbf(M) : 0;
  const int k1 = k / 2, k2 = k - k1;
  C.fx1 = ldexpf(1.f, k1);
  C.fx2 = ldexpf(1.f, k2);
  C.ifx1 = ldexpf(1.f, -k1);
  C.ifx2 = ldexpf(1.f, -k2);
}
__device__ __forceinline__ long long to_fix(const Cta &C, float v) { return __float2ll_rn((v * C.fx1) * C.fx2); }
__device__ __forceinline__ float from_fix(float ifx1, float ifx2, unsigned long long a) {
  return (__ll2float_rn((long long)a) * ifx1) * ifx2;
}
// largest |g| over a trace's root gradients (float4 loads, several in flight per thread),
// kept in L2 with an evict-last hint: the selection walk reads them again step by step
__device__ __forceinline__ float trace_gmax(const float *g, int T) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  const int NT = blockDim.x;
  const int head = min((int)(((16 - (reinterpret_cast<uintptr_t>(g) & 15)) & 15) >> 2), T);
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

__device__ __forceinline__ void fix_add(unsigned long long *p, long long v) {
  if (__isShared(p)) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
  } else {
    atomicAdd(p, (unsigned long long)v);
  }
}

__device__ __forceinline__ int frontier(const Cta &C, int n) {
  const int e = C.t1 + C.rt[n].hi;
  return e < C.T ? e : C.T;
}

// A parent's read access to child values.  Branch-free in the common case: the index is
// clamped into the computed range [start, fmax] (reads outside it feed no output), and sample
// T-1 and the pads past the end of the trace are selected from the per-node cells.
struct ChildView {
  const float *p;
  int start, T, fmax;
  float lastval, padv;
  bool padc;
  __device__ __forceinline__ float get(int j, int &src) const {
    const int jj = max(min(j, fmax), start);
    float v = p[jj - start];
    src = jj;
    if (j >= T - 1) {
      const bool pad = j >= T && padc;
      v = pad ? padv : lastval;
      src = pad ? -1 : T - 1;
    }
    return v;
  }
  __device__ __forceinline__ float get(int j) const {
    const int jj = max(min(j, fmax), start);
    float v = p[jj - start];
    if (j >= T - 1) v = (j >= T && padc) ? padv : lastval;
    return v;
  }
};

__device__ __forceinline__ ChildView child_view(const Cta &C, const KNode &p, int c) {
  const NodeRt &r = C.rt[c];
  ChildView cv;
  cv.p = r.val;
  cv.start = C.t0 + r.lo;
  const int f = frontier(C, c);
  cv.T = C.T;
  cv.fmax = f - 1;
  cv.lastval = r.lastval;
  cv.padv = p.pad_value;
  cv.padc = p.pad_const != 0;
  return cv;
}

// a node's own values / sources / adjoint (sample T-1 lives in per-node cells, because at
// the end of a trace it can lie below the live range of the last step)
struct OwnView {
  const float *v;
  const int *aux;
  const float *adj;
  int start, T;
  float lastval, padadj;
  int lastaux;
  bool fx;                    // adjoint in 64-bit fixed point, scale 1 / (i1 * i2)
  float i1, i2;
  unsigned long long padfx;
  __device__ __forceinline__ float val(int q) const { return q >= T - 1 ? lastval : v[q - start]; }
  __device__ __forceinline__ int src(int q) const { return q >= T - 1 ? lastaux : aux[q - start]; }
  __device__ __forceinline__ float g(int q) const {
    if (fx) {
      const unsigned long long a = q >= T - 1 ? padfx : reinterpret_cast<const unsigned long long *>(adj)[q - start];
      return from_fix(i1, i2, a);
    }
    return q >= T - 1 ? padadj : adj[q - start];
  }
};

__device__ __forceinline__ OwnView own_view(const Cta &C, int n) {
  const NodeRt &r = C.rt[n];
  OwnView o;
  o.v = r.val;
  o.aux = r.aux;
  o.adj = r.adj;
  o.start = C.t0 + r.lo;
  o.T = C.T;
  o.lastval = r.lastval;
  o.lastaux = r.lastaux;
  o.padadj = r.padadj;
  o.fx = C.fx;
  o.i1 = C.ifx1;
  o.i2 = C.ifx2;
  o.padfx = r.padfx;
  return o;
}

// writer of node n's values (and recorded sources in hard backward launches)
struct NodeOut {
  float *v;
  int *aux;
  float *out_row;
  NodeRt *rt;
  int start, T;
  __device__ __forceinline__ void put(int q, float val) const {
    v[q - start] = val;
    if (q == T - 1) rt->lastval = val;
    if (out_row) out_row[q] = val;
  }
  __device__ __forceinline__ void put(int q, float val, int src) const {
    v[q - start] = val;
    if (aux) aux[q - start] = src;
    if (q == T - 1) { rt->lastval = val; rt->lastaux = src; }
    if (out_row) out_row[q] = val;
  }
};

__device__ __forceinline__ NodeOut node_out(const Cta &C, int n) {
  NodeRt &r = C.rt[n];
  NodeOut o;
  o.v = r.val;
  o.aux = r.aux;
  o.out_row = (n == C.root) ? C.out_row : nullptr;
  o.rt = &r;
  o.start = C.t0 + r.lo;
  o.T = C.T;
  return o;
}

// a parent's write access to a child's adjoint (sample T-1 and pads go to the per-node cell)
// With fx, every contribution is rounded to the fixed-point grid before it is added (integer
// sums: exact and order-independent).
struct ChildAdj {
  float *a;
  float *padadj;
  unsigned long long *padfx;
  int start, T;
  bool fx;
  float f1, f2;               // fixed-point scale 2^k = f1 * f2
  __device__ __forceinline__ long long fix(float g) const { return __float2ll_rn((g * f1) * f2); }
  __device__ __forceinline__ void add_atomic(int j, float g) const {
    if (j < 0 || g == 0.f) return;
    if (fx) {
      const long long v = fix(g);
      if (j >= T - 1) fix_add(padfx, v);
      else fix_add(reinterpret_cast<unsigned long long *>(a) + (j - start), v);
      return;
    }
    if (j >= T - 1) buf_add(padadj, g);
    else buf_add(&a[j - start], g);
  }
  __device__ __forceinline__ void add_owned(int j, float g) const {
    if (j < 0) return;
    if (fx) {
      const long long v = fix(g);
      if (j >= T - 1) { if (v != 0) fix_add(padfx, v); }
      else reinterpret_cast<unsigned long long *>(a)[j - start] += (unsigned long long)v;
      return;
    }
    if (j >= T - 1) { if (g != 0.f) buf_add(padadj, g); }
    else a[j - start] += g;
  }
};

__device__ __forceinline__ ChildAdj child_adj(const Cta &C, int c) {
  NodeRt &r = C.rt[c];
  ChildAdj o;
  o.a = r.adj;
  o.padadj = &r.padadj;
  o.padfx = &r.padfx;
  o.start = C.t0 + r.lo;
  o.T = C.T;
  o.fx = C.fx;
  o.f1 = C.fx1;
  o.f2 = C.fx2;
  return o;
}

// ------------------------------------------------------------------ forward ops
// Predicates: a thread first issues the loads of all its samples of the step (BATCH samples
// at a time, independent loads in flight), then evaluates and stores them.
constexpr int BATCH = 8;

template <int DD>
__device__ __forceinline__ void pred_batch(const float *__restrict__ xs, const float *w, bool gt, float pc,
                                           const NodeOut &out, int F, int E) {
  const int NT = blockDim.x;
  float wr[DD];
#pragma unroll
  for (int d = 0; d < DD; ++d) wr[d] = w[d];
  for (int base = F + threadIdx.x; base < E; base += NT * BATCH) {
    float x[BATCH][DD];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
#pragma unroll
      for (int d = 0; d < DD; ++d) x[k][d] = q < E ? __ldg(xs + (size_t)q * DD + d) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
      if (q < E) {
        float s = __fmul_rn(wr[0], x[k][0]);
#pragma unroll
        for (int d = 1; d < DD; ++d) s = __fadd_rn(s, __fmul_rn(wr[d], x[k][d]));
        out.put(q, gt ? __fsub_rn(s, pc) : __fsub_rn(pc, s));
      }
    }
  }
}

// Norm predicates (region membership, Sec. VII-A): mu = ||diag(s)(x - g)||_2 with the same
// float32 order as the affine form (difference, scale, squares summed left to right, then a
// correctly rounded square root), value mu - r (outside) or r - mu (inside).
template <int DD>
__device__ __forceinline__ void norm_batch(const float *__restrict__ xs, const float *sg, bool gt, float r,
                                           const NodeOut &out, int F, int E) {
  const int NT = blockDim.x;
  float sr[DD], gr[DD];
#pragma unroll
  for (int d = 0; d < DD; ++d) { sr[d] = sg[d]; gr[d] = sg[DD + d]; }
  for (int base = F + threadIdx.x; base < E; base += NT * BATCH) {
    float x[BATCH][DD];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
#pragma unroll
      for (int d = 0; d < DD; ++d) x[k][d] = q < E ? __ldg(xs + (size_t)q * DD + d) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
      if (q < E) {
        float u = __fmul_rn(sr[0], __fsub_rn(x[k][0], gr[0]));
        float s = __fmul_rn(u, u);
#pragma unroll
        for (int d = 1; d < DD; ++d) {
          u = __fmul_rn(sr[d], __fsub_rn(x[k][d], gr[d]));
          s = __fadd_rn(s, __fmul_rn(u, u));
        }
        const float mu = __fsqrt_rn(s);
        out.put(q, gt ? __fsub_rn(mu, r) : __fsub_rn(r, mu));
      }
    }
  }
}

__device__ void eval_norm(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const int D = P.D;
  const float *sg = P.w + nd.w_off;   // scales [0, D), centre [D, 2D)
  const float *__restrict__ xs = C.sig + C.row0 * D;
  const NodeOut out = node_out(C, n);
  const bool gt = nd.op == OP_NGT;
  const float r = nd.pc;
  switch (D) {
    case 1: norm_batch<1>(xs, sg, gt, r, out, F, E); return;
    case 2: norm_batch<2>(xs, sg, gt, r, out, F, E); return;
    case 3: norm_batch<3>(xs, sg, gt, r, out, F, E); return;
    case 4: norm_batch<4>(xs, sg, gt, r, out, F, E); return;
    default: break;
  }
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    const float *x = xs + (size_t)q * D;
    float u = __fmul_rn(sg[0], __fsub_rn(__ldg(x), sg[D]));
    float s = __fmul_rn(u, u);
    for (int d = 1; d < D; ++d) {
      u = __fmul_rn(sg[d], __fsub_rn(__ldg(x + d), sg[D + d]));
      s = __fadd_rn(s, __fmul_rn(u, u));
    }
    const float mu = __fsqrt_rn(s);
    out.put(q, gt ? __fsub_rn(mu, r) : __fsub_rn(r, mu));
  }
}

__device__ void eval_pred(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const int D = P.D;
  const float *w = P.w + nd.w_off;
  const float *__restrict__ xs = C.sig + C.row0 * D;
  const NodeOut out = node_out(C, n);
  const bool gt = nd.op == OP_PGT;
  const float pc = nd.pc;
  switch (D) {
    case 1: pred_batch<1>(xs, w, gt, pc, out, F, E); return;
    case 2: pred_batch<2>(xs, w, gt, pc, out, F, E); return;
    case 3: pred_batch<3>(xs, w, gt, pc, out, F, E); return;
    case 4: pred_batch<4>(xs, w, gt, pc, out, F, E); return;
    default: break;
  }
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    const float *x = xs + (size_t)q * D;
    float s = __fmul_rn(w[0], __ldg(x));
    for (int d = 1; d < D; ++d) s = __fadd_rn(s, __fmul_rn(w[d], __ldg(x + d)));
    out.put(q, gt ? __fsub_rn(s, pc) : __fsub_rn(pc, s));
  }
}

// All predicates of the formula in one pass over the step (signals with D <= 4): a thread
// loads BATCH samples of the signal once and evaluates every predicate on them, each within
// its own range [F_k, E_k) of new samples; the arithmetic is that of eval_pred / eval_norm.
__device__ __forceinline__ void pred_range(const Cta &C, int n, int t0, int R0, int &F, int &E) {
  const NodeRt &r = C.rt[n];
  const int F0 = (t0 == R0) ? R0 + r.lo : t0 + r.hi;
  F = F0 < C.T ? F0 : C.T;
  E = frontier(C, n);
}

template <int DD>
__device__ void eval_preds_fused(const Cta &C, int t0, int R0) {
  const KProgram &P = *C.P;
  const int npred = P.npred, NT = blockDim.x;
  const float *__restrict__ xs = C.sig + C.row0 * DD;
  // union of the predicates' ranges; empty when every predicate is complete (late steps)
  int F = C.T, E = 0;
  for (int k = 0; k < npred; ++k) {
    int f, e;
    pred_range(C, P.pred[k], t0, R0, f, e);
    if (f < e) {
      F = min(F, f);
      E = max(E, e);
    }
  }
  if (F >= E) return;
  for (int base = F + threadIdx.x; base < E; base += NT * BATCH) {
    float x[BATCH][DD];
#pragma unroll
    for (int b = 0; b < BATCH; ++b) {
      const int q = base + b * NT;
#pragma unroll
      for (int d = 0; d < DD; ++d) x[b][d] = q < E ? __ldg(xs + (size_t)q * DD + d) : 0.f;
    }
    for (int k = 0; k < npred; ++k) {
      const int n = P.pred[k];
      const KNode &nd = P.nd[n];
      int f, e;
      pred_range(C, n, t0, R0, f, e);
      const NodeOut out = node_out(C, n);
      const float *w = P.w + nd.w_off;
      const float c = nd.pc;
      if (nd.op == OP_PGT || nd.op == OP_PLT) {
        const bool gt = nd.op == OP_PGT;
        float wr[DD];
#pragma unroll
        for (int d = 0; d < DD; ++d) wr[d] = w[d];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
          const int q = base + b * NT;
          if (q < f || q >= e) continue;
          float s = __fmul_rn(wr[0], x[b][0]);
#pragma unroll
          for (int d = 1; d < DD; ++d) s = __fadd_rn(s, __fmul_rn(wr[d], x[b][d]));
          out.put(q, gt ? __fsub_rn(s, c) : __fsub_rn(c, s));
        }
      } else {
        const bool gt = nd.op == OP_NGT;
        float sr[DD], gr[DD];
#pragma unroll
        for (int d = 0; d < DD; ++d) { sr[d] = w[d]; gr[d] = w[DD + d]; }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
          const int q = base + b * NT;
          if (q < f || q >= e) continue;
          float u = __fmul_rn(sr[0], __fsub_rn(x[b][0], gr[0]));
          float s = __fmul_rn(u, u);
#pragma unroll
          for (int d = 1; d < DD; ++d) {
            u = __fmul_rn(sr[d], __fsub_rn(x[b][d], gr[d]));
            s = __fadd_rn(s, __fmul_rn(u, u));
          }
          const float mu = __fsqrt_rn(s);
          out.put(q, gt ? __fsub_rn(mu, c) : __fsub_rn(c, mu));
        }
      }
    }
  }
}

__device__ void eval_preds(const Cta &C, int t0, int R0) {
  switch (C.P->D) {
    case 1: eval_preds_fused<1>(C, t0, R0); return;
    case 2: eval_preds_fused<2>(C, t0, R0); return;
    case 3: eval_preds_fused<3>(C, t0, R0); return;
    default: eval_preds_fused<4>(C, t0, R0); return;
  }
}

// Elementwise nodes: each thread first loads BATCH samples of its children (independent loads
// in flight), then combines and stores them.
template <bool SMOOTH>
__device__ void eval_elementwise(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const NodeOut out = node_out(C, n);
  const int op = nd.op;
  const int NT = blockDim.x;
  if (op == OP_TRUE) {
    for (int q = F + threadIdx.x; q < E; q += NT) out.put(q, INFINITY);
    return;
  }
  const ChildView x = child_view(C, nd, nd.c0);
  if (op == OP_NOT) {
    for (int base = F + threadIdx.x; base < E; base += NT * BATCH) {
      float a[BATCH];
#pragma unroll
      for (int k = 0; k < BATCH; ++k) {
        const int q = base + k * NT;
        a[k] = q < E ? x.get(q) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < BATCH; ++k) {
        const int q = base + k * NT;
        if (q < E) out.put(q, -a[k]);
      }
    }
    return;
  }
  const ChildView y = child_view(C, nd, nd.c1);
  const float tau = P.tau, itau = P.inv_tau;
  const float sg = op == OP_AND ? 1.f : -1.f;
  for (int base = F + threadIdx.x; base < E; base += NT * BATCH) {
    float a[BATCH], b[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
      a[k] = q < E ? x.get(q) : 0.f;
      b[k] = q < E ? y.get(q) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
      if (q >= E) continue;
      float v;
      if constexpr (!SMOOTH) {
        v = op == OP_AND ? (a[k] <= b[k] ? a[k] : b[k]) : (a[k] >= b[k] ? a[k] : b[k]);
      } else if (P.mode == 2) {
        float wa;
        v = sw2(a[k], b[k], -sg, tau, wa);
      } else {
        // two-term logsumexp min / max: min(x,y) - log1p(e^{-tau|x-y|}) / tau
        const float xs = sg * a[k], ys = sg * b[k];
        const float m = xs < ys ? xs : ys;
        float corr = (xs == ys) ? 0.69314718f * itau : log1pf(expf(-tau * fabsf(xs - ys))) * itau;
        if (isinf(xs) || isinf(ys)) corr = 0.f;
        v = sg * (m - corr);
      }
      out.put(q, v);
    }
  }
}

// hard window of node n over its child with offsets [ia, ib] (max or min)
template <bool BWD>
__device__ void eval_hard_window(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KNode &nd = C.P->nd[n];
  const ChildView cv = child_view(C, nd, nd.c0);
  const NodeOut o = node_out(C, n);
  const bool mx = nd.op == OP_EV || nd.op == OP_EVSM;
  const int K = ib - ia + 1;
  if constexpr (BWD) {
    auto elem = [&](int j) { VI r; r.v = cv.get(j, r.i); return r; };
    auto out = [&](int q, VI r) { o.put(q, r.v, r.i); };
    if (mx) window_any<MaxI>(K, F, E, ia, ib, elem, out, C.scratch);
    else window_any<MinI>(K, F, E, ia, ib, elem, out, C.scratch);
  } else {
    auto elem = [&](int j) { return cv.get(j); };
    auto out = [&](int q, float r) { o.put(q, r); };
    if (mx) window_any<MaxV>(K, F, E, ia, ib, elem, out, C.scratch);
    else window_any<MinV>(K, F, E, ia, ib, elem, out, C.scratch);
  }
}

// smooth window: (sgn/tau) log sum_i e^{sgn tau x_{q+i}}
__device__ void eval_smooth_window(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const ChildView cv = child_view(C, nd, nd.c0);
  const NodeOut o = node_out(C, n);
  const float sgn = nd.op == OP_EV ? 1.f : -1.f;
  const float st = sgn * P.tau, sit = sgn * P.inv_tau;
  if (P.mode == 2) {
    // softmax-weighted; the log-normaliser goes to the aux ring (backward launches)
    auto elem = [&](int j) { return sw_elem(cv.get(j), st); };
    auto out = [&](int q, SW r) { o.put(q, sw_value(r, sgn), __float_as_int(sw_lse(r))); };
    window_any<SwM>(ib - ia + 1, F, E, ia, ib, elem, out, C.scratch);
    return;
  }
  auto elem = [&](int j) { LS r; r.m = st * cv.get(j); r.s = 1.f; return r; };
  auto out = [&](int q, LS r) { o.put(q, (r.m + __logf(r.s)) * sit); };
  window_any<LseM>(ib - ia + 1, F, E, ia, ib, elem, out, C.scratch);
}

// hard Until: pass 1 stores A_q = min_{k in [0,a]} phi_{q+k} (with its sample), pass 2
// composes the clamps over [a, b] and keeps min(A_q, V_{q+a}) with A winning ties.
template <bool BWD>
__device__ void eval_hard_until(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KNode &nd = C.P->nd[n];
  const ChildView cp = child_view(C, nd, nd.c0);
  const ChildView cq = child_view(C, nd, nd.c1);
  const NodeOut o = node_out(C, n);
  if constexpr (BWD) {
    {
      auto elem = [&](int j) { VI r; int s; r.v = cp.get(j, s); r.i = s < 0 ? -1 : 2 * s; return r; };
      auto out = [&](int q, VI r) { o.put(q, r.v, r.i); };
      window_any<MinI>(ia + 1, F, E, 0, ia, elem, out, C.scratch);
    }
    __syncthreads();
    auto elem = [&](int j) {
      CC r;
      int sp, sq;
      const float p = cp.get(j, sp);
      const float q = cq.get(j, sq);
      const int ep = sp < 0 ? -1 : 2 * sp, eq = sq < 0 ? -1 : 2 * sq + 1;
      const bool pl = p <= q;
      r.c = pl ? p : q;
      r.cs = pl ? ep : eq;
      r.d = p;
      r.ds = ep;
      return r;
    };
    auto out = [&](int q, CC r) {
      const float A = o.v[q - o.start];
      if (!(A <= r.c)) o.put(q, r.c, r.cs);
    };
    window_reduce<ClampI, RUN>(F, E, ia, ib, elem, out, C.scratch);
  } else {
    {
      auto elem = [&](int j) { return cp.get(j); };
      auto out = [&](int q, float r) { o.put(q, r); };
      window_any<MinV>(ia + 1, F, E, 0, ia, elem, out, C.scratch);
    }
    __syncthreads();
    auto elem = [&](int j) {
      C2 r;
      const float p = cp.get(j), q = cq.get(j);
      r.c = fminf(p, q);
      r.d = p;
      return r;
    };
    auto out = [&](int q, C2 r) {
      const float A = o.v[q - o.start];
      if (!(A <= r.c)) o.put(q, r.c);
    };
    window_reduce<ClampV, RUN>(F, E, ia, ib, elem, out, C.scratch);
  }
}

// ------------------------------------------------------------------ lean hard forward passes
// Hard forward steps of the 512-thread kernels with at least STL_LEAN_MIN_SAMPLES new samples
// in a node evaluate windows, Until and the elementwise operators with direct reads of their
// children's buffers: no clamping and no end-of-trace test per read.  This is exact because
//  (1) a child computes every sample below its frontier min(t1 + hi, T), and a live output
//      of the parent reads only samples below that frontier or at or after T;
//  (2) before a temporal parent runs in a step where the child's frontier has reached T,
//      the child's samples from T on are filled with the parent's pad (the value at T-1, or
//      the constant), which is what a read past the end returns (padded unroll, Sec. IV-B);
//  (3) window passes may read up to R - 1 samples past a child's live range (the buffers are
//      allocated with that slack); such reads feed only outputs that are discarded.
// Long windows use runs of 15 samples per thread (fewer run aggregates per output).

__device__ __forceinline__ bool is_temporal_op(int op) {
  return op == OP_EV || op == OP_ALW || op == OP_EVSM || op == OP_ALWSM || op == OP_UNTIL || op == OP_UNTSM;
}

// Fill the pad samples of node n's children whose frontier has reached T; returns whether
// anything was written (the same on every thread), so that the caller can synchronise.
__device__ bool pad_fill(const Cta &C, int n) {
  const KNode &nd = C.P->nd[n];
  const int T = C.T;
  bool any = false;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int c = s == 0 ? nd.c0 : nd.c1;
    if (c < 0 || frontier(C, c) < T) continue;
    const NodeRt &r = C.rt[c];
    const int start = C.t0 + r.lo;
    // live outputs read at most ib samples past T-1, window runs at most 14 more
    const int f0 = max(T - start, 0), f1 = min(r.cap + STL_BUF_BACK, T - start + C.rt[n].ib + 16);
    const float v = nd.pad_const ? nd.pad_value : r.lastval;
    for (int i = f0 + threadIdx.x; i < f1; i += blockDim.x) r.val[i] = v;
    any = any || f0 < f1;
  }
  return any;
}

// Windowed reduction over direct child reads (the decomposition of window_reduce); threads
// whose runs no output uses read nothing, so that every read stays within the slack.
template <class M, int R, class Elem, class Out>
__device__ __forceinline__ void hwin(int q0, int q1, int ia, int ib, const Elem &elem, const Out &out,
                                     void *scratch) {
  using T = typename M::T;
  const int K = ib - ia + 1;
  const int tid = threadIdx.x, NT = blockDim.x;
  if (q1 <= q0) return;
  if (K < 2 * R) {
    for (int q = q0 + tid; q < q1; q += NT) {
      T acc = elem(q + ia);
      for (int i = ia + 1; i <= ib; ++i) acc = M::comb(acc, elem(q + i));
      out(q, acc);
    }
    return;
  }
  T *runagg = reinterpret_cast<T *>(scratch);
  const int nf = K / R - 1;           // whole runs strictly inside every window (>= 1)
  const int rho = K - (nf + 1) * R;   // lead of the trailing prefix
  const bool two = nf >= 3 * L2B;
  for (int p0 = q0; p0 < q1; p0 += NT * R) {
    const int u = p0 + tid * R;
    const int nv = min(NT, (q1 - p0 + R - 1) / R);   // threads that own outputs in this pass
    const int nr = nv + nf;                          // run aggregates the outputs use
    const int nruns = max(NT, nr);
    T *agg2 = runagg + nruns;
    T hv[R];
    if (tid < nr) {
      hv[R - 1] = elem(u + ia + R - 1);
#pragma unroll
      for (int k = R - 2; k >= 0; --k) hv[k] = M::comb(elem(u + ia + k), hv[k + 1]);
      runagg[tid] = hv[0];
    }
    for (int e = NT + tid; e < nr; e += NT) {
      const int s = p0 + ia + e * R;
      T acc = elem(s);
#pragma unroll
      for (int k = 1; k < R; ++k) acc = M::comb(acc, elem(s + k));
      runagg[e] = acc;
    }
    __syncthreads();
    if (two) {
      const int nb = nr / L2B;
      for (int m = tid; m < nb; m += NT) {
        T acc = runagg[m * L2B];
#pragma unroll
        for (int k = 1; k < L2B; ++k) acc = M::comb(acc, runagg[m * L2B + k]);
        agg2[m] = acc;
      }
      __syncthreads();
    }
    if (tid < nv) {
      const T mid = middle<M>(runagg, agg2, tid + 1, tid + nf, two);
      const int gs = u + ia + (nf + 1) * R;
      T acc = mid;
      bool have = rho > 0;
      if (have) {
        acc = elem(gs);
        for (int e = 1; e < rho; ++e) acc = M::comb(acc, elem(gs + e));
      }
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (u + k < q1) {
          T r = M::comb(hv[k], mid);
          if (have) r = M::comb(r, acc);
          out(u + k, r);
        }
        if (k + 1 < R) {
          T e = elem(gs + rho + k);
          acc = have ? M::comb(acc, e) : e;
          have = true;
        }
      }
    }
    if (p0 + NT * R < q1) __syncthreads();   // the caller synchronises after the last pass
  }
}

// runs of 15 for long windows, 7 and 3 for shorter ones, a direct loop below 6
template <class M, class Elem, class Out>
__device__ __forceinline__ void hwin_any(int q0, int q1, int ia, int ib, const Elem &elem, const Out &out,
                                         void *scratch) {
  const int K = ib - ia + 1;
  if (K >= 30) hwin<M, 15>(q0, q1, ia, ib, elem, out, scratch);
  else if (K >= 14) hwin<M, 7>(q0, q1, ia, ib, elem, out, scratch);
  else hwin<M, 3>(q0, q1, ia, ib, elem, out, scratch);
}

// What a lean pass needs, passed by value: the passes are separate (not inlined) functions,
// so that each gets its own register allocation (measured faster than inlining them).
struct Lean {
  NodeRt *rt;          // per-node runtime table
  void *scratch;       // window scratch
  float *out_row;      // root output row
  int n, c0, c1, op;
  int t0, T, root;
};
__device__ __forceinline__ Lean lean_args(const Cta &C, int n) {
  const KNode &nd = C.P->nd[n];
  Lean L;
  L.rt = C.rt;
  L.scratch = C.scratch;
  L.out_row = C.out_row;
  L.n = n;
  L.c0 = nd.c0;
  L.c1 = nd.c1;
  L.op = nd.op;
  L.t0 = C.t0;
  L.T = C.T;
  L.root = C.root;
  return L;
}

struct RawRead {       // child sample j, read directly (pad-filled past T-1)
  const float *p;
  int start;
  __device__ __forceinline__ float operator()(int j) const { return p[j - start]; }
};
__device__ __forceinline__ RawRead raw_read(const Lean &L, int c) {
  RawRead r;
  r.p = L.rt[c].val;
  r.start = L.t0 + L.rt[c].lo;
  return r;
}

// writer of a node's hard outputs into its own buffer (a temporal root is copied out to
// the output row by the step loop)
struct HardOut {
  float *v;
  NodeRt *rt;
  int start, T;
  __device__ __forceinline__ void put(int q, float val) const {
    v[q - start] = val;
    if (q == T - 1) rt->lastval = val;
  }
};
__device__ __forceinline__ HardOut hard_out(const Lean &L) {
  NodeRt &r = L.rt[L.n];
  HardOut o;
  o.v = r.val;
  o.rt = &r;
  o.start = L.t0 + r.lo;
  o.T = L.T;
  return o;
}

__device__ __noinline__ void lean_hard_window(const Lean L, int F, int E, int ia, int ib) {
  const RawRead x = raw_read(L, L.c0);
  const HardOut o = hard_out(L);
  auto out = [&](int q, float r) { o.put(q, r); };
  if (L.op == OP_EV || L.op == OP_EVSM) hwin_any<MaxV>(F, E, ia, ib, x, out, L.scratch);
  else hwin_any<MinV>(F, E, ia, ib, x, out, L.scratch);
}

// hard Until: pass 1 stores A_q = min_{k in [0,a]} phi_{q+k}, pass 2 composes the clamps over
// [a, b] and keeps min(A_q, V_{q+a})
__device__ __noinline__ void lean_hard_until(const Lean L, int F, int E, int ia, int ib) {
  const RawRead xp = raw_read(L, L.c0);
  const RawRead xq = raw_read(L, L.c1);
  const HardOut o = hard_out(L);
  {
    auto out = [&](int q, float r) { o.put(q, r); };
    hwin_any<MinV>(F, E, 0, ia, xp, out, L.scratch);
  }
  __syncthreads();
  auto elem = [&](int j) {
    C2 r;
    const float p = xp(j), q = xq(j);
    r.c = fminf(p, q);
    r.d = p;
    return r;
  };
  auto out = [&](int q, C2 r) {
    const float A = o.v[q - o.start];
    if (!(A <= r.c)) o.put(q, r.c);
  };
  hwin_any<ClampV>(F, E, ia, ib, elem, out, L.scratch);
}

// hard not / and / or over direct reads (a node reads its children at its own samples, all
// below T); the root writes the output row as it goes (consecutive threads, consecutive
// samples)
__device__ __noinline__ void lean_hard_elementwise(const Lean L, int F, int E) {
  const int op = L.op;
  const int NT = blockDim.x;
  NodeRt &r = L.rt[L.n];
  float *ov = r.val;
  const int ost = L.t0 + r.lo;
  float *orow = (L.n == L.root) ? L.out_row : nullptr;
  const int T = L.T;
  const RawRead x = raw_read(L, L.c0);
  const RawRead y = raw_read(L, op == OP_NOT ? L.c0 : L.c1);
  float last = 0.f;
  bool has_last = false;
  for (int base = F + threadIdx.x; base < E; base += NT * BATCH) {
    float a[BATCH], b[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
      a[k] = q < E ? x(q) : 0.f;
      b[k] = q < E ? y(q) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = base + k * NT;
      if (q >= E) continue;
      const float v = op == OP_NOT ? -a[k] : op == OP_AND ? (a[k] <= b[k] ? a[k] : b[k])
                                                         : (a[k] >= b[k] ? a[k] : b[k]);
      ov[q - ost] = v;
      if (orow) orow[q] = v;
      if (q == T - 1) { last = v; has_last = true; }
    }
  }
  if (has_last) r.lastval = last;
}

// Smooth Until (nested logsumexp of Sec. IV-C with the smooth min/max of Sec. III-C; the
// nesting flattens, Sec. IV-D):  U = (1/tau) log sum_{i in [a,b]} 1/(S_i + Q_i) with
// S_i = sum_{k<=i} e^{-tau phi_k}, Q_i = e^{-tau psi_i}.  Computed in the log domain with running
// maxima so that nothing overflows; one output per thread, O(b) taps.
struct LseAcc {   // running log(sum e^{z}) as (max, scaled sum)
  float m = -INFINITY, s = 0.f;
  __device__ __forceinline__ void add(float z) {
    if (z == -INFINITY) return;
    if (z > m) { s = fmaf(s, __expf(m - z), 1.f); m = z; }
    else s += __expf(z - m);
  }
  __device__ __forceinline__ float log() const { return m == -INFINITY ? -INFINITY : m + __logf(s); }
};

// L = log(S + Q) with S = e^{acc}, Q = e^{zq}: -tau * smin(P, psi)
__device__ __forceinline__ float log_s_plus_q(const LseAcc &acc, float zq) {
  if (acc.m == -INFINITY) return zq;
  if (zq == -INFINITY) return acc.log();
  if (zq > acc.m) return zq + __logf(fmaf(acc.s, __expf(acc.m - zq), 1.f));
  return acc.m + __logf(acc.s + __expf(zq - acc.m));
}

// w (masked-interval Until): weight m_i of offset i is w[i - ia]; nullptr for weights 1.
__device__ void eval_smooth_until(const Cta &C, int n, int F, int E, int ia, int ib, const float *w) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const ChildView cp = child_view(C, nd, nd.c0);
  const ChildView cq = child_view(C, nd, nd.c1);
  const NodeOut o = node_out(C, n);
  const float tau = P.tau, itau = P.inv_tau;
  // outputs whose taps all lie below T-1 inside both children's computed ranges read the
  // buffers directly (no per-tap clamp or end-of-trace select)
  const int qdirect = min(min(cp.fmax, cq.fmax), C.T - 2) - ib;
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    LseAcc S, Z;   // S: sum_k e^{-tau phi_k};  Z: sum_i m_i e^{tau z_i}
    if (q <= qdirect && q >= cp.start && q >= cq.start) {
      const float *pp = cp.p + (q - cp.start), *pq = cq.p + (q - cq.start);
      for (int i = 0; i < ia; ++i) S.add(-tau * pp[i]);
      for (int i = ia; i <= ib; ++i) {
        S.add(-tau * pp[i]);
        Z.add(-log_s_plus_q(S, -tau * pq[i]) + (w ? __logf(w[i - ia]) : 0.f));
      }
    } else {
      for (int i = 0; i <= ib; ++i) {
        S.add(-tau * cp.get(q + i));
        if (i >= ia) Z.add(-log_s_plus_q(S, -tau * cq.get(q + i)) + (w ? __logf(w[i - ia]) : 0.f));
      }
    }
    const float lz = Z.log();
    o.put(q, lz == -INFINITY ? -INFINITY : lz * itau);
  }
}

// Softmax-weighted Until (each of its three min/max levels is one softmax-weighted reduction
// over its own multiset, never a nesting of two-term operators): P_i = softmin_{k<=i} phi_{q+k}, z_i = softmin(P_i, psi_{q+i}),
// U = softmax_{i in [a,b]} z_i, each one softmax-weighted reduction; one output per thread.
__device__ void eval_soft_until(const Cta &C, int n, int F, int E, int ia, int ib, const float *w) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const ChildView cp = child_view(C, nd, nd.c0);
  const ChildView cq = child_view(C, nd, nd.c1);
  const NodeOut o = node_out(C, n);
  const float tau = P.tau;
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    SW pa{-INFINITY, 0.f, 0.f}, ua{-INFINITY, 0.f, 0.f};
    for (int i = 0; i <= ib; ++i) {
      pa = SwM::comb(pa, sw_elem(cp.get(q + i), -tau));
      if (i >= ia) {
        float wp;
        const float z = sw2(sw_value(pa, -1.f), cq.get(q + i), -1.f, tau, wp);
        SW e = sw_elem(z, tau);
        if (w) { e.s *= w[i - ia]; e.n *= w[i - ia]; }
        ua = SwM::comb(ua, e);
      }
    }
    o.put(q, sw_value(ua, 1.f));
  }
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

__device__ __forceinline__ float smask(float i, float a, float b, float c, float eps) {
  float m = sigmoidf_(c * (i - a)) - sigmoidf_(c * (i - b)) - eps;
  return m > 0.f ? m : 0.f;
}

// smooth-mask window in smooth mode: (sgn/tau) log sum_i m_i e^{sgn tau x_{q+i}}, with the
// weights m_i of this trace read from the node's table
__device__ void eval_smooth_mask(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const NodeRt &me = C.rt[n];
  const ChildView cv = child_view(C, nd, nd.c0);
  const NodeOut o = node_out(C, n);
  const int ia = me.ia, len = me.ib - me.ia + 1;
  const float *w = me.tab;
  const float sgn = nd.op == OP_EVSM ? 1.f : -1.f;
  const float st = sgn * P.tau;
  if (P.mode == 2) {
    // softmax-weighted with the mask as weight: sum m_i v_i e^{st v_i} / sum m_i e^{st v_i}
    // (sums in double: the weighted mean of up to a few hundred taps of both signs)
    for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
      float M = -INFINITY;
      double S = 0.0, N = 0.0;
      float inf_v = 0.f;
      bool has_inf = false;
      for (int i = 0; i < len; ++i) {
        const float m = w[i];
        if (m <= 0.f) continue;
        const float x = cv.get(q + ia + i), z = st * x;
        if (z == -INFINITY) continue;
        if (z == INFINITY) { if (!has_inf) inf_v = x; has_inf = true; continue; }
        if (z > M) {
          const double f = (double)__expf(M - z);
          S = S * f + m;
          N = N * f + (double)m * x;
          M = z;
        } else {
          const double e = (double)m * (double)__expf(z - M);
          S += e;
          N = fma(e, (double)x, N);
        }
      }
      float y, lse;
      if (has_inf) { y = inf_v; lse = INFINITY; }
      else if (M == -INFINITY) { y = -sgn * INFINITY; lse = -INFINITY; }
      else { y = (float)(N / S); lse = M + (float)log(S); }
      o.put(q, y, __float_as_int(lse));
    }
    return;
  }
  const int ja = me.ja, jb = me.jb, ib = me.ib;
  if (jb - ja + 1 >= 2 * RUN) {
    // O(1) per sample: the plateau [ja, jb] (every weight exactly w0 = fl(1 - eps)) is a sliding
    // logsumexp window scaled by w0; the two edge bands [ia, ja) and (jb, ib] are added tap by tap
    const float w0 = w[ja - ia];
    auto elem = [&](int j) { LS r; r.m = st * cv.get(j); r.s = 1.f; return r; };
    auto out = [&](int q, LS r) {
      float M = r.m, S = r.m == -INFINITY ? 0.f : r.s * w0;
      auto add = [&](int i) {
        const float m = w[i - ia];
        const float z = st * cv.get(q + i);
        if (z == -INFINITY || m <= 0.f) return;
        if (z > M) { S = fmaf(S, __expf(M - z), m); M = z; }
        else S = fmaf(m, __expf(z - M), S);
      };
      for (int i = ia; i < ja; ++i) add(i);
      for (int i = jb + 1; i <= ib; ++i) add(i);
      o.put(q, M == -INFINITY ? sgn * -INFINITY : sgn * (M + __logf(S)) * P.inv_tau);
    };
    window_any<LseM>(jb - ja + 1, F, E, ja, jb, elem, out, C.scratch);
    return;
  }
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    float M = -INFINITY, S = 0.f;
    for (int i = 0; i < len; ++i) {
      const float m = w[i];
      const float z = st * cv.get(q + ia + i);
      if (z > M) { S = fmaf(S, __expf(M - z), m); M = z; }
      else S = fmaf(m, __expf(z - M), S);
    }
    o.put(q, M == -INFINITY ? sgn * -INFINITY : sgn * (M + __logf(S)) * P.inv_tau);
  }
}

// lean: evaluate a hard forward node with the direct-read passes (the caller has filled the
// children's pads); otherwise with the clamped reads
template <bool BWD, bool SMOOTH, bool LEAN>
__device__ void eval_node(const Cta &C, int n, int F, int E, bool lean) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const NodeRt &r = C.rt[n];
  switch (nd.op) {
    case OP_PGT:
    case OP_PLT: eval_pred(C, n, F, E); break;
    case OP_NGT:
    case OP_NLT: eval_norm(C, n, F, E); break;
    case OP_TRUE: eval_elementwise<SMOOTH>(C, n, F, E); break;
    case OP_NOT:
    case OP_AND:
    case OP_OR:
      if (SMOOTH || BWD || !LEAN || !lean) eval_elementwise<SMOOTH>(C, n, F, E);
      else lean_hard_elementwise(lean_args(C, n), F, E);
      break;
    case OP_EV:
    case OP_ALW:
      if constexpr (SMOOTH) eval_smooth_window(C, n, F, E, r.ia, r.ib);
      else if (BWD || !LEAN || !lean) eval_hard_window<BWD>(C, n, F, E, r.ia, r.ib);
      else lean_hard_window(lean_args(C, n), F, E, r.ia, r.ib);
      break;
    case OP_EVSM:
    case OP_ALWSM:
      if constexpr (SMOOTH) eval_smooth_mask(C, n, F, E);
      else if (r.ia > r.ib) {
        // no offset has a positive mask (b - a too small for the sharpness): the max (min)
        // over an empty set, -inf (+inf), selecting no sample
        const NodeOut o = node_out(C, n);
        const float v = nd.op == OP_EVSM ? -INFINITY : INFINITY;
        for (int q = F + threadIdx.x; q < E; q += blockDim.x) o.put(q, v, -1);
      }
      else if (BWD || !LEAN || !lean) eval_hard_window<BWD>(C, n, F, E, r.ia, r.ib);
      else lean_hard_window(lean_args(C, n), F, E, r.ia, r.ib);
      break;
    case OP_UNTIL:
      if constexpr (SMOOTH) {
        if (P.mode == 2) eval_soft_until(C, n, F, E, r.ia, r.ib, nullptr);
        else eval_smooth_until(C, n, F, E, r.ia, r.ib, nullptr);
      }
      else if (BWD || !LEAN || !lean) eval_hard_until<BWD>(C, n, F, E, r.ia, r.ib);
      else lean_hard_until(lean_args(C, n), F, E, r.ia, r.ib);
      break;
    case OP_UNTSM:
      // Until over the masked interval: the support [ia, ib] of the mask; in the smooth modes
      // its offsets carry the mask weights (an empty support gives -inf)
      if (r.ia > r.ib) {
        const NodeOut o = node_out(C, n);
        for (int q = F + threadIdx.x; q < E; q += blockDim.x) o.put(q, -INFINITY, -1);
      } else if constexpr (SMOOTH) {
        if (P.mode == 2) eval_soft_until(C, n, F, E, r.ia, r.ib, r.tab);
        else eval_smooth_until(C, n, F, E, r.ia, r.ib, r.tab);
      } else if (BWD || !LEAN || !lean) {
        eval_hard_until<BWD>(C, n, F, E, r.ia, r.ib);
      } else {
        lean_hard_until(lean_args(C, n), F, E, r.ia, r.ib);
      }
      break;
  }
}

// ------------------------------------------------------------------ adjoint helpers
// warp-aggregated scatter: lanes hold (key, g); runs of equal keys in consecutive lanes are
// summed first, then one atomic per run.  key = sample (or 2*sample + child for Until), -1 none.
__device__ __forceinline__ void scatter_run(const ChildAdj &a0, const ChildAdj &a1, int key, float g,
                                            bool even_odd) {
  const int lane = threadIdx.x & 31;
  const int up = __shfl_up_sync(FULL, key, 1);
  const bool head = lane == 0 || up != key;
  const unsigned heads = __ballot_sync(FULL, head);
  const int rid = __popc(heads & (0xffffffffu >> (31 - lane)));
  float s = g;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float sv = __shfl_down_sync(FULL, s, off);
    const int rv = __shfl_down_sync(FULL, rid, off);
    if (lane + off < 32 && rv == rid) s += sv;
  }
  if (head && key >= 0) {
    if (even_odd) ((key & 1) ? a1 : a0).add_atomic(key >> 1, s);
    else a0.add_atomic(key, s);
  }
}

__device__ __forceinline__ void accumulate_shared(float *dst, float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
  if ((threadIdx.x & 31) == 0 && v != 0.f) buf_add(dst, v);
}

// the same with the warp sum in double (per-thread partial sums of both signs)
__device__ __forceinline__ void accumulate_shared_d(float *dst, double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
  if ((threadIdx.x & 31) == 0 && v != 0.0) buf_add(dst, (float)v);
}

// ------------------------------------------------------------------ adjoint ops
// Adjoint of node n over its complete samples [A0, A1): adds into the children.
// [own0, own1) are the samples whose bound gradients this work item owns.
template <bool SMOOTH>
__device__ void adjoint_node(const Cta &C, int n, int A0, int A1, int own0, int own1) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const float tau = P.tau;
  const int NT = blockDim.x;
  const int op = nd.op;
  if (is_pred_op(op) || op == OP_TRUE) return;
  const OwnView me = own_view(C, n);
  const ChildAdj a0 = child_adj(C, nd.c0);
  if (op == OP_NOT) {
    for (int q = A0 + threadIdx.x; q < A1; q += NT) a0.add_owned(q, -me.g(q));
    return;
  }
  if (op == OP_AND || op == OP_OR) {
    const ChildAdj a1 = child_adj(C, nd.c1);
    const ChildView x = child_view(C, nd, nd.c0), y = child_view(C, nd, nd.c1);
    const float sg = op == OP_AND ? 1.f : -1.f;
    for (int q = A0 + threadIdx.x; q < A1; q += NT) {
      const float g = me.g(q);
      const float a = x.get(q), b = y.get(q);
      if constexpr (!SMOOTH) {
        const bool left = op == OP_AND ? a <= b : a >= b;
        (left ? a0 : a1).add_owned(q, g);
      } else if (P.mode == 2) {
        float wa;
        const float y = sw2(a, b, -sg, tau, wa);
        a0.add_owned(q, g * sw_grad(wa, a, y, -sg * tau));
        a1.add_owned(q, g * sw_grad(1.f - wa, b, y, -sg * tau));
      } else {
        float wx, wy;
        if (isinf(a) && isinf(b)) { wx = 1.f; wy = 0.f; }
        else {
          wx = 1.f / (1.f + expf(-sg * tau * (b - a)));
          wy = 1.f / (1.f + expf(-sg * tau * (a - b)));
        }
        a0.add_owned(q, g * wx);
        a1.add_owned(q, g * wy);
      }
    }
    return;
  }
  const bool is_until = is_until_op(op);
  if constexpr (!SMOOTH) {
    // hard: every complete sample sends its adjoint to the recorded source
    const ChildAdj a1 = is_until ? child_adj(C, nd.c1) : a0;
    for (int qb = A0; qb < A1; qb += NT) {
      const int q = qb + threadIdx.x;
      int key = -1;
      float g = 0.f;
      if (q < A1) {
        g = me.g(q);
        key = me.src(q);
      }
      scatter_run(a0, a1, key, g, is_until);
    }
    return;
  } else {
    const ChildView cv = child_view(C, nd, nd.c0);
    if (op == OP_EVSM || op == OP_ALWSM) {
      // smooth-mask window.  Signal part as a gather (no atomics):
      //   x̄_j += sum_{i in support, q = j - i in [A0, A1)} g_q m_i e^{sgn tau (x_j - y_q)}
      // (every term <= |g_q|), bound part per parent sample over the two edge bands:
      //   ā += g_q (sgn/tau) sum_i dm_i/da e^{sgn tau (x_{q+i} - y_q)}, likewise b̄.
      NodeRt &rt = C.rt[n];
      const float sgn = op == OP_EVSM ? 1.f : -1.f;
      const float st = sgn * tau;
      const int ia = rt.ia, ib = rt.ib, len = ib - ia + 1;
      const float *w = rt.tab, *wa = rt.tab + len, *wb = rt.tab + 2 * len;
      if (P.mode == 2) {
        // softmax-weighted: p_{q,i} = m_i e^{st x_{q+i} - lse_q}; signal part
        //   x̄_j += sum_i g_q p_{q,i} (1 + st (x_j - y_q)),  q = j - i,
        // bound part d y_q / d a = sum_i (dm_i/da) e^{st x_{q+i} - lse_q} (x_{q+i} - y_q), likewise b
        for (int j = A0 + ia + threadIdx.x; j < A1 + ib; j += NT) {
          int src;
          const float x = cv.get(j, src);
          if (src < 0 || isinf(x)) continue;
          const int ilo = max(ia, j - (A1 - 1)), ihi = min(ib, j - A0);
          float acc = 0.f;
          const float sx = st * x;
          for (int i = ilo; i <= ihi; ++i) {
            const int q = j - i;
            const float g = me.g(q), lse = __int_as_float(me.src(q)), y = me.val(q);
            if (g == 0.f || isinf(lse) || isinf(y)) continue;
            acc = fmaf(g * w[i - ia] * __expf(sx - lse), fmaf(st, x - y, 1.f), acc);
          }
          a0.add_owned(src, acc);
        }
        double ga = 0.0, gbv = 0.0;   // sums of both signs over the owned samples
        for (int q = A0 + threadIdx.x; q < A1; q += NT) {
          if (q < own0 || q >= own1) continue;
          const float g = me.g(q), lse = __int_as_float(me.src(q)), y = me.val(q);
          if (g == 0.f || isinf(lse) || isinf(y)) continue;
          double sa = 0.0, sb = 0.0;
          for (int i = ia; i <= rt.band_a; ++i) {
            const float x = cv.get(q + i);
            if (!isinf(x)) sa = fma((double)(wa[i - ia] * __expf(st * x - lse)), (double)x - (double)y, sa);
          }
          for (int i = rt.band_b; i <= ib; ++i) {
            const float x = cv.get(q + i);
            if (!isinf(x)) sb = fma((double)(wb[i - ia] * __expf(st * x - lse)), (double)x - (double)y, sb);
          }
          ga = fma((double)g, sa, ga);
          gbv = fma((double)g, sb, gbv);
        }
        accumulate_shared_d(&rt.ga, ga);
        accumulate_shared_d(&rt.gb, gbv);
        return;
      }
      const int ja = rt.ja, jb = rt.jb;
      if (jb - ja + 1 >= 2 * RUN) {
        // plateau offsets: the transposed logsumexp window over the parent samples scaled by
        // w0, x̄_j += w0 e^{st x_j} sum_{q in [j-jb, j-ja]} g_q e^{-st y_q}; edge offsets tap by tap
        const float w0 = w[ja - ia];
        auto elem = [&](int q) {
          LSd r;
          if (q < A0 || q >= A1) { r.m = -INFINITY; r.s = 0.0; return r; }
          r.m = -st * me.val(q);
          r.s = me.g(q);
          return r;
        };
        auto out = [&](int j, LSd r) {
          int src;
          const float x = cv.get(j, src);
          if (src < 0) return;
          const float sx = st * x;
          float acc = (r.m == -INFINITY || r.s == 0.0) ? 0.f : w0 * (float)(r.s * (double)__expf(sx + r.m));
          auto edge = [&](int i) {
            const int q = j - i;
            if (q < A0 || q >= A1) return;
            const float g = me.g(q);
            acc = fmaf(g * w[i - ia], __expf(sx - st * me.val(q)), acc);
          };
          for (int i = ia; i < ja; ++i) edge(i);
          for (int i = jb + 1; i <= ib; ++i) edge(i);
          a0.add_owned(src, acc);
        };
        window_any<LsdM>(jb - ja + 1, A0 + ia, A1 + ib, -jb, -ja, elem, out, C.scratch);
      } else {
        for (int j = A0 + ia + threadIdx.x; j < A1 + ib; j += NT) {
          int src;
          const float x = cv.get(j, src);
          if (src < 0) continue;
          const int ilo = max(ia, j - (A1 - 1)), ihi = min(ib, j - A0);
          float acc = 0.f;
          const float sx = st * x;
          for (int i = ilo; i <= ihi; ++i) {
            const int q = j - i;
            const float g = me.g(q);
            acc = fmaf(g * w[i - ia], __expf(sx - st * me.val(q)), acc);
          }
          a0.add_owned(src, acc);
        }
      }
      float ga = 0.f, gbv = 0.f;
      for (int q = A0 + threadIdx.x; q < A1; q += NT) {
        if (q < own0 || q >= own1) continue;
        const float g = me.g(q);
        if (g == 0.f) continue;
        const float sy = st * me.val(q);
        float sa = 0.f, sb = 0.f;
        for (int i = ia; i <= rt.band_a; ++i) sa = fmaf(wa[i - ia], __expf(st * cv.get(q + i) - sy), sa);
        for (int i = rt.band_b; i <= ib; ++i) sb = fmaf(wb[i - ia], __expf(st * cv.get(q + i) - sy), sb);
        ga = fmaf(g * sgn * P.inv_tau, sa, ga);
        gbv = fmaf(g * sgn * P.inv_tau, sb, gbv);
      }
      accumulate_shared(&rt.ga, ga);
      accumulate_shared(&rt.gb, gbv);
      return;
    }
    // smooth Eventually / Always: transposed window over the parent samples,
    // x̄_j += e^{sgn tau x_j} sum_{q in [j-b, j-a] ∩ [A0,A1)} g_q e^{-sgn tau y_q}
    const float st = (op == OP_EV ? 1.f : -1.f) * tau;
    const NodeRt &rt = C.rt[n];
    const int ia = rt.ia, ib = rt.ib;
    if (P.mode == 2) {
      // softmax-weighted: with lse_q the log-normaliser of output q (aux ring),
      // x̄_j += e^{st x_j} sum_q e^{-lse_q} (g_q (1 - st y_q) + st x_j g_q)
      auto elem2 = [&](int q) {
        LS2 r{-INFINITY, 0.0, 0.0};
        if (q < A0 || q >= A1) return r;
        const float lse = __int_as_float(me.src(q)), y = me.val(q), g = me.g(q);
        if (g == 0.f || isinf(lse) || isinf(y)) return r;
        r.m = -lse;
        r.s1 = (double)g * (1.0 - (double)st * (double)y);
        r.s2 = g;
        return r;
      };
      // reads past the end all land on sample T-1: their terms are summed per thread in double
      // and added once per warp
      double pad_acc = 0.0;
      auto out2 = [&](int j, LS2 r) {
        if (r.m == -INFINITY) return;
        int src;
        const float x = cv.get(j, src);
        if (src < 0 || isinf(x)) return;
        const double v = (double)__expf(st * x + r.m) * fma((double)st * (double)x, r.s2, r.s1);
        if (j >= C.T - 1) pad_acc += v;
        else a0.add_owned(src, (float)v);
      };
      window_any<Lse2M>(ib - ia + 1, A0 + ia, A1 + ib, -ib, -ia, elem2, out2, C.scratch);
      accumulate_shared_d(a0.padadj, pad_acc);
      return;
    }
    auto elem = [&](int q) {
      LSd r;
      if (q < A0 || q >= A1) { r.m = -INFINITY; r.s = 0.0; return r; }
      r.m = -st * me.val(q);
      r.s = me.g(q);
      return r;
    };
    auto out = [&](int j, LSd r) {
      if (r.m == -INFINITY || r.s == 0.0) return;
      int src;
      const float x = cv.get(j, src);
      if (src < 0) return;
      a0.add_owned(src, (float)(r.s * (double)__expf(st * x + r.m)));
    };
    window_any<LsdM>(ib - ia + 1, A0 + ia, A1 + ib, -ib, -ia, elem, out, C.scratch);
  }
}

// Smooth Until adjoint.  With S_k = sum_{j<=k} e^{-tau phi_{q+j}}, Q_i = e^{-tau psi_{q+i}},
// L_i = log(S_i + Q_i) = -tau z_i and tau U = log W, W = sum_{i in [a,b]} e^{-L_i}:
//   dU/dpsi_{q+i} = e^{-2 L_i - tau U} Q_i
//   dU/dphi_{q+k} = e^{-tau phi_{q+k}} R_k,   R_k = sum_{i >= max(k, a)} e^{-2 L_i - tau U}
// (differentiate log W through S_i = ... + e^{-tau phi_k} for every i >= k).  R_k is a suffix sum
// of positive terms, accumulated from k = b down to 0 with the running maximum m_k of the
// exponents of S_k as scale, R'_k = e^{m_k} R_k = e^{m_k - m_{k+1}} R'_{k+1} + [k>=a] e^{-2 L_k - tau U + m_k},
// and dU/dphi_{q+k} = e^{-tau phi_{q+k} - m_k} R'_k: every exponent is <= 0, and the factor
// e^{m_k - m_{k+1}} is exactly 1 except where the maximum moves (products of rounded ratios of
// S would lose a few ulps per tap over windows of thousands of taps).  The recursion needs m_k
// and L_k from k = b down to 0, which a running sum cannot give without cancellation.  So a first
// pass over the taps keeps only the accumulator of S at every UCK-th tap (two floats per
// checkpoint in the per-thread workspace arrays), and a second pass walks the chunks from the
// last to the first: it restarts S from the chunk's checkpoint, recomputes m_k and L_k for the
// chunk's UCK taps into registers (depositing the psi adjoint and the bound gradients on the
// way), then runs the recursion over the chunk backwards.  Masked-interval Until: the terms of
// offset i carry the weight m_i (the node's table), and the bound gradients add
// g m'_i e^{tau (z_i - U)} / tau over the owned samples [own0, own1).
constexpr int UCK = 8;   // taps per checkpoint of the smooth Until adjoint

// Reads of an Until's children and deposits into their adjoints for one output q, through the
// clamped views (any output) or, for outputs whose taps q..q+b all lie below T-1, directly:
// plain loads of the children's buffers and fixed-point additions at the tap's offset, with
// no per-tap clamp, end-of-trace select or address-space test.
struct UntilIOView {
  const ChildView &cp, &cq;
  const ChildAdj &ap, &aq;
  int q;
  __device__ __forceinline__ float phi(int k, int &src) const { return cp.get(q + k, src); }
  __device__ __forceinline__ float psi(int k, int &src) const { return cq.get(q + k, src); }
  __device__ __forceinline__ void dep_phi(int src, float v) const { ap.add_atomic(src, v); }
  __device__ __forceinline__ void dep_psi(int src, float v) const { aq.add_atomic(src, v); }
};
struct UntilIODirect {
  const float *pp, *pq;              // the children's values at sample q
  unsigned long long *dp, *dq;       // their fixed-point adjoints at sample q
  unsigned dps, dqs;                 // the same as shared addresses (when sh)
  bool sh;                           // both adjoint buffers in shared memory
  float f1, f2;                      // fixed-point scale
  __device__ __forceinline__ float phi(int k, int &src) const { src = k; return pp[k]; }
  __device__ __forceinline__ float psi(int k, int &src) const { src = k; return pq[k]; }
  __device__ __forceinline__ void dep(unsigned long long *base, unsigned sbase, int k, float v) const {
    const long long f = __float2ll_rn((v * f1) * f2);
    if (f == 0) return;
    if (sh) asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(sbase + 8u * (unsigned)k), "l"(f) : "memory");
    else atomicAdd(base + k, (unsigned long long)f);
  }
  __device__ __forceinline__ void dep_phi(int k, float v) const { dep(dp, dps, k, v); }
  __device__ __forceinline__ void dep_psi(int k, float v) const { dep(dq, dqs, k, v); }
};

// the adjoint of one output q (see the derivation above); g its upstream gradient, tU = tau U_q
template <class IO>
__device__ __forceinline__ void until_adjoint_one(const IO &io, float g, float tU, int ia, int ib, float tau,
                                                  float itau, const float *w, const float *wa, const float *wb,
                                                  bool own, float *Cm, float *Cs, long long pstride, double &ga,
                                                  double &gbv) {
  {
    LseAcc S;
    for (int k = 0; k <= ib; ++k) {
      if ((k & (UCK - 1)) == 0) {
        Cm[(k / UCK) * pstride] = S.m;
        Cs[(k / UCK) * pstride] = S.s;
      }
      int src;
      S.add(-tau * io.phi(k, src));
    }
  }
  float Rn = 0.f, mnext = -INFINITY;   // R'_{k+1} and m_{k+1}
  for (int c0 = (ib / UCK) * UCK; c0 >= 0; c0 -= UCK) {
    LseAcc S;
    S.m = Cm[(c0 / UCK) * pstride];
    S.s = Cs[(c0 / UCK) * pstride];
    float Mc[UCK], Lc[UCK], Zc[UCK];
    int Sc[UCK];
#pragma unroll
    for (int j = 0; j < UCK; ++j) {
      const int k = c0 + j;
      Mc[j] = -INFINITY;
      Lc[j] = -INFINITY;
      Zc[j] = -INFINITY;
      Sc[j] = -1;
      if (k <= ib) {
        Zc[j] = -tau * io.phi(k, Sc[j]);
        S.add(Zc[j]);
        Mc[j] = S.m;
        if (k >= ia) {
          int sq;
          const float zq = -tau * io.psi(k, sq);
          const float L = log_s_plus_q(S, zq);
          Lc[j] = L;
          const float m = w ? w[k - ia] : 1.f;
          if (zq != -INFINITY && L != -INFINITY) io.dep_psi(sq, g * m * __expf(-L - tU + zq - L));
          if (own && L != -INFINITY) {
            const double e = (double)__expf(-L - tU) * (double)itau * (double)g;
            ga = fma(e, (double)wa[k - ia], ga);
            gbv = fma(e, (double)wb[k - ia], gbv);
          }
        }
      }
    }
#pragma unroll
    for (int j = UCK - 1; j >= 0; --j) {
      const int k = c0 + j;
      if (k > ib) continue;
      const float mk = Mc[j];
      float R = 0.f;
      if (mk != -INFINITY) {
        if (k < ib) R = (mk == mnext ? 1.f : __expf(mk - mnext)) * Rn;
        if (k >= ia && Lc[j] != -INFINITY) R += (w ? w[k - ia] : 1.f) * __expf(-2.f * Lc[j] - tU + mk);
        if (!isinf(Zc[j])) io.dep_phi(Sc[j], g * __expf(Zc[j] - mk) * R);
      }
      Rn = R;
      mnext = mk;
    }
  }
}

__device__ void adjoint_smooth_until(const Cta &C, int n, int A0, int A1, int own0, int own1, float *Pk,
                                     long long pstride) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  NodeRt &rt = C.rt[n];
  const OwnView me = own_view(C, n);
  const ChildView cp = child_view(C, nd, nd.c0), cq = child_view(C, nd, nd.c1);
  const ChildAdj ap = child_adj(C, nd.c0), aq = child_adj(C, nd.c1);
  const float tau = P.tau, itau = P.inv_tau;
  const int ia = rt.ia, ib = rt.ib;
  const bool masked = nd.op == OP_UNTSM;
  const int len = ib - ia + 1;
  const float *w = masked ? rt.tab : nullptr, *wa = masked ? rt.tab + len : nullptr, *wb = masked ? rt.tab + 2 * len : nullptr;
  float *Cm = Pk, *Cs = Pk + (long long)P.ut_len * pstride;   // checkpoints: max and scaled sum of S
  // outputs whose taps all lie below T-1 and inside both children's computed ranges take the
  // direct path (fixed-point adjoints only)
  const int qdirect = min(min(cp.fmax, cq.fmax), C.T - 2) - ib;   // last such output
  const bool can_direct = ap.fx && aq.fx;
  const bool sh = __isShared(ap.a) && __isShared(aq.a);
  double ga = 0.0, gbv = 0.0;
  for (int q = A0 + threadIdx.x; q < A1; q += blockDim.x) {
    const float g = me.g(q);
    if (g == 0.f) continue;
    const float tU = tau * me.val(q);
    const bool own = masked && q >= own0 && q < own1;
    if (can_direct && q <= qdirect && q >= cp.start && q >= cq.start) {
      UntilIODirect io;
      io.pp = cp.p + (q - cp.start);
      io.pq = cq.p + (q - cq.start);
      io.dp = reinterpret_cast<unsigned long long *>(ap.a) + (q - ap.start);
      io.dq = reinterpret_cast<unsigned long long *>(aq.a) + (q - aq.start);
      io.sh = sh;
      io.dps = sh ? (unsigned)__cvta_generic_to_shared(io.dp) : 0u;
      io.dqs = sh ? (unsigned)__cvta_generic_to_shared(io.dq) : 0u;
      io.f1 = ap.f1;
      io.f2 = ap.f2;
      until_adjoint_one(io, g, tU, ia, ib, tau, itau, w, wa, wb, own, Cm, Cs, pstride, ga, gbv);
    } else {
      const UntilIOView io{cp, cq, ap, aq, q};
      until_adjoint_one(io, g, tU, ia, ib, tau, itau, w, wa, wb, own, Cm, Cs, pstride, ga, gbv);
    }
  }
  if (masked) {
    accumulate_shared_d(&rt.ga, ga);
    accumulate_shared_d(&rt.gb, gbv);
  }
}

// Softmax-weighted Until adjoint (three softmax-weighted levels, as in the forward).  Per output q: a forward pass over the taps stores
// P_i, L_i = log sum_{k<=i} e^{-tau phi_k} and z_i (3 per-thread workspace arrays) and yields U
// and its log-normaliser; then
//   dU/dz_i = e^{tau z_i - lseU} (1 + tau (z_i - U)),
//   z_i = softmin(P_i, psi_i): dz/dP = w_P (1 - tau (P_i - z_i)), dz/dpsi = w_psi (1 - tau (psi_i - z_i)),
//   dP_i/dphi_k = e^{-tau phi_k - L_i} (1 + tau P_i - tau phi_k)   (k <= i),
// and a backward pass over k sums c_i = g dU/dz_i dz_i/dP_i as
//   phi_bar_k = e^{-tau phi_k - L_k} (R1_k - tau phi_k R2_k),
//   R1_k = sum_{i>=k} c_i e^{L_k - L_i} (1 + tau P_i),  R2_k = sum_{i>=k} c_i e^{L_k - L_i},
// whose recursions multiply by e^{L_k - L_{k+1}} <= 1 (nothing overflows).
// Masked-interval Until: U = sum m_i z_i e^{tau z_i} / sum m_i e^{tau z_i}, so dU/dz_i carries
// m_i and dU/dm_i = e^{tau z_i - lseU} (z_i - U) gives the bound gradients (owned samples).
__device__ void adjoint_soft_until(const Cta &C, int n, int A0, int A1, int own0, int own1, float *Pk,
                                   long long pstride) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  NodeRt &rt = C.rt[n];
  const OwnView me = own_view(C, n);
  const ChildView cp = child_view(C, nd, nd.c0), cq = child_view(C, nd, nd.c1);
  const ChildAdj ap = child_adj(C, nd.c0), aq = child_adj(C, nd.c1);
  const float tau = P.tau;
  const int ia = rt.ia, ib = rt.ib;
  const bool masked = nd.op == OP_UNTSM;
  const int len = ib - ia + 1;
  const float *w = masked ? rt.tab : nullptr, *wa = masked ? rt.tab + len : nullptr, *wb = masked ? rt.tab + 2 * len : nullptr;
  double ga = 0.0, gbv = 0.0;
  float *Zk = Pk + (long long)P.ut_len * pstride;
  float *Lk = Pk + 2LL * P.ut_len * pstride;
  const int T1 = C.T - 1;
  double pad_p = 0.0, pad_q = 0.0;   // reads at or past sample T-1, summed per thread in double
  for (int q = A0 + threadIdx.x; q < A1; q += blockDim.x) {
    const float g = me.g(q);
    if (g == 0.f) continue;
    SWd pa, ua;   // double sums: the adjoint below differentiates these reductions
    for (int i = 0; i <= ib; ++i) {
      pa.add(cp.get(q + i), -tau);
      const float Pv = pa.value(-1.f);
      Pk[i * pstride] = Pv;
      Lk[i * pstride] = pa.lse();
      if (i >= ia) {
        float wp;
        const float z = sw2(Pv, cq.get(q + i), -1.f, tau, wp);
        Zk[i * pstride] = z;
        ua.add(z, tau, w ? w[i - ia] : 1.f);
      }
    }
    const float U = ua.value(1.f), lU = ua.lse();
    if (isinf(U) || isinf(lU)) continue;
    double R1 = 0.0, R2 = 0.0;   // combined as R1 - tau phi R2, which cancels by about tau |phi|
    float Lnext = 0.f;
    for (int k = ib; k >= 0; --k) {
      const float Pv = Pk[k * pstride], L = Lk[k * pstride];
      if (k < ib) {
        const double f = (isinf(L) || isinf(Lnext)) ? 0.0 : (double)__expf(L - Lnext);
        R1 *= f;
        R2 *= f;
      }
      if (k >= ia) {
        const float z = Zk[k * pstride];
        if (!isinf(z) && masked && q >= own0 && q < own1) {
          const double dm = (double)g * (double)__expf(tau * z - lU) * ((double)z - (double)U);
          ga = fma(dm, (double)wa[k - ia], ga);
          gbv = fma(dm, (double)wb[k - ia], gbv);
        }
        if (!isinf(z)) {
          const float dUz = g * (w ? w[k - ia] : 1.f) * __expf(tau * z - lU) * fmaf(tau, z - U, 1.f);
          int sq;
          const float psi = cq.get(q + k, sq);
          float wP;
          sw2(Pv, psi, -1.f, tau, wP);
          if (!isinf(psi)) {
            const float v = dUz * sw_grad(1.f - wP, psi, z, -tau);
            if (sq == T1) pad_q += v;
            else aq.add_atomic(sq, v);
          }
          if (!isinf(Pv)) {
            const double c = (double)dUz * (double)sw_grad(wP, Pv, z, -tau);
            R1 = fma(c, 1.0 + (double)tau * (double)Pv, R1);
            R2 += c;
          }
        }
      }
      int sp;
      const float phi = cp.get(q + k, sp);
      if (!isinf(phi) && !isinf(L)) {
        const double v = (double)__expf(-tau * phi - L) * fma(-(double)tau * (double)phi, R2, R1);
        if (sp == T1) pad_p += v;
        else ap.add_atomic(sp, (float)v);
      }
      Lnext = L;
    }
  }
  accumulate_shared_d(ap.padadj, pad_p);
  accumulate_shared_d(aq.padadj, pad_q);
  if (masked) {
    accumulate_shared_d(&rt.ga, ga);
    accumulate_shared_d(&rt.gb, gbv);
  }
}

// ------------------------------------------------------------------ per-trace geometry
__device__ double smask_d(double i, double a, double b, double c, double eps) {
  double m = 1.0 / (1.0 + exp(-c * (i - a))) - 1.0 / (1.0 + exp(-c * (i - b))) - eps;
  return m > 0.0 ? m : 0.0;
}

__device__ void setup_geometry(Cta &C, const float *bounds, float *ws_cta, char *smem, int *status) {
  const KProgram &P = *C.P;
  if (threadIdx.x == 0) {
    for (int n = P.n - 1; n >= 0; --n) {
      const KNode &nd = P.nd[n];
      NodeRt &r = C.rt[n];
      float a = nd.a, b = nd.b;
      if (nd.slot >= 0 && bounds) {
        const float *bp = bounds + ((size_t)C.b * P.n_slots + nd.slot) * 2;
        a = bp[0];
        b = bp[1];
        if (!(a >= 0.f) || !(b >= a) || b > nd.b || a > nd.a) {
          if (status) atomicExch(status, 1);
          a = fminf(fmaxf(a, 0.f), nd.a);
          b = fminf(fmaxf(b, a), nd.b);
        }
      }
      r.fa = a;
      r.fb = b;
      if (nd.op == OP_EVSM || nd.op == OP_ALWSM || nd.op == OP_UNTSM) {
        // support {i >= 0 : sigma(c(i-a)) - sigma(c(i-b)) > eps} is an interval inside
        // [a - L - 1, b + L + 2], L = log((1-eps)/eps) / c; warp 0 finds its ends below
        const double c = P.mask_c, eps = P.mask_eps;
        const double L = log((1.0 - eps) / eps) / c;
        const int lo = (int)floor((double)a - L) - 1;
        r.ia = lo < 0 ? 0 : lo;
        r.ib = (int)ceil((double)b + L) + 2;
      } else if (nd.op == OP_EV || nd.op == OP_ALW || nd.op == OP_UNTIL) {
        r.ia = (int)a;
        r.ib = isinf(b) ? (int)(C.T - 1) : (int)b;
        if (r.ib < r.ia) r.ib = r.ia;
      } else {
        r.ia = r.ib = 0;
      }
      r.lo = nd.lo;
      r.hi = nd.hi;
      r.cap = nd.cap;
      float *base = nd.space == 0 ? reinterpret_cast<float *>(smem) : ws_cta;
      r.val = base + nd.val_off;
      r.adj = nd.adj_off >= 0 ? base + nd.adj_off : nullptr;
      r.aux = nd.aux_off >= 0 ? reinterpret_cast<int *>(base + nd.aux_off) : nullptr;
      r.lastval = 0.f;
      r.lastaux = -1;
      r.padadj = 0.f;
      r.padfx = 0ull;
      r.ga = r.gb = 0.f;
      r.base = 0;
      r.op = nd.op;
      r.c0 = nd.c0;
      r.c1 = nd.c1;
      r.pred_k = -1;
      r.tab = nd.tab_off >= 0 ? reinterpret_cast<float *>(smem) + nd.tab_off : nullptr;
    }
    for (int k = 0; k < P.npred; ++k) C.rt[P.pred[k]].pred_k = k;
  }
  __syncthreads();
  // smooth-mask supports: the lanes of warp 0 test 32 candidate offsets at a time from each end
  // (the double-precision mask costs two exponentials per offset), then fix the tables' range
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int n = 0; n < P.n; ++n) {
      const KNode &nd = P.nd[n];
      if (!(nd.op == OP_EVSM || nd.op == OP_ALWSM || nd.op == OP_UNTSM)) continue;
      NodeRt &r = C.rt[n];
      const double c = P.mask_c, eps = P.mask_eps;
      const double fa = r.fa, fb = r.fb;
      const int lo0 = r.ia, hi0 = r.ib;
      int lo = hi0 + 1;   // first positive offset (none: past the end)
      for (int base = lo0; base <= hi0; base += 32) {
        const int i = base + lane;
        const unsigned m = __ballot_sync(FULL, i <= hi0 && smask_d(i, fa, fb, c, eps) > 0.0);
        if (m) { lo = base + __ffs(m) - 1; break; }
      }
      int hi = hi0;       // last positive offset at or after lo
      for (int top = hi0; top >= lo; top -= 32) {
        const int i = top - lane;
        const unsigned m = __ballot_sync(FULL, i >= lo && smask_d(i, fa, fb, c, eps) > 0.0);
        if (m) { hi = top - (__ffs(m) - 1); break; }
      }
      if (lane == 0) {
        r.ia = lo;
        r.ib = hi;
        if (r.tab) {
          if (r.ib - r.ia + 1 > nd.tab_len) {   // cannot happen for bounds within the caps
            if (status) atomicExch(status, 1);
            r.ib = r.ia + nd.tab_len - 1;
          }
          // beyond 22/c from an edge, sigma(c d)(1 - sigma(c d)) < e^-22: the bound gradient
          // terms there are below float resolution of the sums they join
          const float band = 22.f / P.mask_c;
          r.band_a = min(r.ib, (int)ceilf(r.fa + band));
          r.band_b = max(r.ia, (int)floorf(r.fb - band));
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // smooth-mask tables m_i, dm_i/da, dm_i/db over the support (Eq. smooth mask)
  for (int n = 0; n < P.n; ++n) {
    const NodeRt &r = C.rt[n];
    if (!r.tab) continue;
    const int len = r.ib - r.ia + 1;
    const float c = P.mask_c, eps = P.mask_eps;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const float fi = (float)(r.ia + i);
      const float sa = 1.f / (1.f + expf(-c * (fi - r.fa)));
      const float sb = 1.f / (1.f + expf(-c * (fi - r.fb)));
      const float m = sa - sb - eps;
      r.tab[i] = m > 0.f ? m : 0.f;
      r.tab[len + i] = m > 0.f ? -c * sa * (1.f - sa) : 0.f;
      r.tab[2 * len + i] = m > 0.f ? c * sb * (1.f - sb) : 0.f;
    }
  }
  __syncthreads();
  // plateau of each mask: the offsets whose float weight is exactly 1 - eps (the sigmoid at a has
  // rounded to 1 and the one at b is below half an ulp of 1); they form one interval
  if (threadIdx.x == 0) {
    for (int n = 0; n < P.n; ++n) {
      NodeRt &r = C.rt[n];
      r.ja = 1;
      r.jb = 0;
      if (!r.tab) continue;
      const float w0 = 1.f - P.mask_eps;
      const int len = r.ib - r.ia + 1;
      // scanned in from both ends (a few entries each: the edge bands), not across the plateau,
      // while the other threads wait at the barrier below
      int lo = 0;
      while (lo < len && r.tab[lo] != w0) ++lo;
      int hi = len - 1;
      while (hi > lo && r.tab[hi] != w0) --hi;
      if (lo < len) {
        r.ja = r.ia + lo;
        r.jb = r.ia + hi;
      }
    }
  }
  __syncthreads();
}

// zero words [w0, w1) of a buffer (16-byte aligned base; vector stores for the bulk)
__device__ __forceinline__ void zero_words(float *p, int w0, int w1) {
  int a = (w0 + 3) & ~3;
  if (a > w1) a = w1;
  for (int i = w0 + threadIdx.x; i < a; i += blockDim.x) p[i] = 0.f;
  const int nv = (w1 - a) >> 2;
  float4 *p4 = reinterpret_cast<float4 *>(p + a);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = a + 4 * nv + threadIdx.x; i < w1; i += blockDim.x) p[i] = 0.f;
}

// move words [src, src+len) of p to [0, len); the two ranges are disjoint (len <= src)
__device__ __forceinline__ void move_down(float *p, int src, int len) {
  if ((src & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    const int nv = len >> 2;
    float4 *d4 = reinterpret_cast<float4 *>(p);
    const float4 *s4 = reinterpret_cast<const float4 *>(p + src);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) d4[i] = s4[i];
    for (int i = 4 * nv + threadIdx.x; i < len; i += blockDim.x) p[i] = p[src + i];
  } else {
    for (int i = threadIdx.x; i < len; i += blockDim.x) p[i] = p[src + i];
  }
}

// end of a step: keep the live samples [t1 + lo, t1 + hi) at the front of every buffer
template <bool BWD>   // AW: adjoint words per sample (2: fixed point)
__device__ void shift_buffers(const Cta &C, int tile, int AW) {
  const KProgram &P = *C.P;
  int max_span = 0;
  for (int n = 0; n < P.n; ++n) max_span = max(max_span, C.rt[n].hi - C.rt[n].lo);
  // rounds of at most `tile` words keep every source chunk disjoint from its destination
  for (int c0 = 0; c0 < max_span; c0 += tile) {
    for (int n = 0; n < P.n; ++n) {
      const NodeRt &r = C.rt[n];
      const int span = r.hi - r.lo;
      if (c0 >= span) continue;
      const int len = min(tile, span - c0);
      move_down(r.val + c0, tile, len);
      if (BWD) {
        if (r.adj) {
          if (AW == 1) move_down(r.adj + c0, tile, len);
          else move_down(r.adj + AW * c0, AW * tile, AW * len);
        }
        if (r.aux) move_down(reinterpret_cast<float *>(r.aux) + c0, tile, len);
      }
    }
    __syncthreads();
  }
  if (BWD) {
    // the next step's new samples start with a zero adjoint
    for (int n = 0; n < P.n; ++n) {
      const NodeRt &r = C.rt[n];
      if (r.adj) zero_words(r.adj, AW * (r.hi - r.lo), AW * r.cap);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ hard-mode selection walk
// In hard semantics the gradient of a root sample flows to exactly one predicate sample (or
// nowhere): follow the recorded selections down the tree and deposit the root gradient
// there (64-bit fixed point: the sums do not depend on the order of the deposits).  One pass
// over the root samples of the step, with no barrier between levels; internal nodes keep no
// adjoint at all.
__device__ void hard_walk(const Cta &C, const float *__restrict__ gout_row, int t0, int t1) {
  const NodeRt *rt = C.rt;
  const int T = C.T;
  const int lane = threadIdx.x & 31;
  const int NT = blockDim.x;
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  for (int qb0 = t0; qb0 < t1; qb0 += NT * BATCH) {
    float gb[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int q = qb0 + k * NT + threadIdx.x;
      gb[k] = 0.f;
      if (q < t1)   // last use of the root gradient (it was kept in L2 for this read)
        asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(gb[k]) : "l"(gout_row + q), "l"(pol));
    }
#pragma unroll 1
    for (int k = 0; k < BATCH; ++k) {
      const int qb = qb0 + k * NT;
      if (qb >= t1) break;
      const int q = qb + threadIdx.x;
      int pk = -1, j = -1;
      float g = 0.f;
      if (q < t1) {
        g = gb[k];
        int n = C.root;
        j = q;
        for (;;) {
          const NodeRt &r = rt[n];
          const int op = r.op;
          if (is_pred_op(op)) { pk = r.pred_k; break; }
          if (op == OP_TRUE) break;
          if (op == OP_NOT) { g = -g; n = r.c0; continue; }
          if (op == OP_AND || op == OP_OR) {
            const NodeRt &a = rt[r.c0], &b = rt[r.c1];
            const float x = j >= T - 1 ? a.lastval : a.val[j - (C.t0 + a.lo)];
            const float y = j >= T - 1 ? b.lastval : b.val[j - (C.t0 + b.lo)];
            const bool left = op == OP_AND ? x <= y : x >= y;
            n = left ? r.c0 : r.c1;
            continue;
          }
          const int key = j >= T - 1 ? r.lastaux : r.aux[j - (C.t0 + r.lo)];
          if (key < 0) break;
          if (is_until_op(op)) { n = (key & 1) ? r.c1 : r.c0; j = key >> 1; }
          else { n = r.c0; j = key; }
        }
      }
      // runs of consecutive lanes ending on the same predicate sample add once (integer sums:
      // exact, so the result does not depend on how samples fall into warps)
      long long v = pk >= 0 ? to_fix(C, g) : 0;
      const int pj = __shfl_up_sync(FULL, j, 1), pp = __shfl_up_sync(FULL, pk, 1);
      const bool head = lane == 0 || pj != j || pp != pk;
      const unsigned heads = __ballot_sync(FULL, head);
      if (heads != FULL) {   // some lanes share a target: segmented sum over the runs
        const int rid = __popc(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const long long sv = __shfl_down_sync(FULL, v, off);
          const int rv = __shfl_down_sync(FULL, rid, off);
          if (lane + off < 32 && rv == rid) v += sv;
        }
      }
      if (head && pk >= 0 && v != 0) {
        const NodeRt &r = rt[C.P->pred[pk]];
        if (j >= T - 1) fix_add(const_cast<unsigned long long *>(&r.padfx), v);
        else fix_add(reinterpret_cast<unsigned long long *>(r.adj) + (j - (C.t0 + r.lo)), v);
      }
    }
  }
}

// ------------------------------------------------------------------ signal gradient
// grad_sig[j, d] = sum_k pw[k][d] * pbar_k[j] over the affine predicates, plus, for each
// norm predicate k, pbar_k[j] * (+-) s_d u_d / mu with u = diag(s)(x_j - g), mu = ||u|| (zero
// at mu = 0, a subgradient of the norm there), for the complete samples [j0, j1); every
// predicate buffer starts at sample pst.  A thread handles SB samples per iteration, D
// unrolled when small (measured faster than one thread per element with coalesced stores).
__device__ __forceinline__ float norm_mu_d(const float *sg, const float *x, int D, int d, float *ud) {
  float q = 0.f;
  for (int e = 0; e < D; ++e) {
    const float u = sg[e] * (x[e] - sg[D + e]);
    if (e == d) *ud = u;
    q = fmaf(u, u, q);
  }
  return q;
}

// the norm term of dimension d of predicate k at one sample
__device__ __forceinline__ float norm_grad_dim(const KProgram &P, int k, const float *x, int D, int d, float a) {
  const KNode &nd = P.nd[P.pred[k]];
  const float *sg = P.w + nd.w_off;
  float ud = 0.f;
  const float q = norm_mu_d(sg, x, D, d, &ud);
  return q > 0.f ? (nd.op == OP_NGT ? a : -a) * rsqrtf(q) * sg[d] * ud : 0.f;
}

// predicate adjoint k at sample j: a float (smooth) or a fixed-point sum (hard)
template <bool FX>
__device__ __forceinline__ float padj_at(float *const *padj, int k, int idx, float i1, float i2) {
  if constexpr (FX) return from_fix(i1, i2, reinterpret_cast<const unsigned long long *>(padj[k])[idx]);
  else return padj[k][idx];
}

template <int DD, bool FX>
__device__ __forceinline__ void signal_gradient_d(const KProgram &P, float *const *padj, const float *xs, float *gs,
                                                  int pst, int j0, int j1, float i1, float i2) {
  constexpr int SB = 4;   // samples per thread per iteration (independent loads in flight)
  const int NT = blockDim.x;
  for (int base = j0 + threadIdx.x; base < j1; base += NT * SB) {
    float acc[SB][DD];
#pragma unroll
    for (int s = 0; s < SB; ++s)
#pragma unroll
      for (int d = 0; d < DD; ++d) acc[s][d] = 0.f;
    for (int k = 0; k < P.npred; ++k) {
      float w[DD], a[SB];
#pragma unroll
      for (int d = 0; d < DD; ++d) w[d] = P.pw[k * STL_MAX_D + d];
#pragma unroll
      for (int s = 0; s < SB; ++s) {
        const int j = base + s * NT;
        a[s] = j < j1 ? padj_at<FX>(padj, k, j - pst, i1, i2) : 0.f;
      }
#pragma unroll
      for (int s = 0; s < SB; ++s)
#pragma unroll
        for (int d = 0; d < DD; ++d) acc[s][d] = fmaf(w[d], a[s], acc[s][d]);
    }
    for (unsigned m = P.norm_mask; m; m &= m - 1) {
      const int k = __ffs(m) - 1;
#pragma unroll
      for (int s = 0; s < SB; ++s) {
        const int j = base + s * NT;
        if (j >= j1) continue;
        const float a = padj_at<FX>(padj, k, j - pst, i1, i2);
        if (a == 0.f) continue;
#pragma unroll
        for (int d = 0; d < DD; ++d) acc[s][d] += norm_grad_dim(P, k, xs + (size_t)j * DD, DD, d, a);
      }
    }
#pragma unroll
    for (int s = 0; s < SB; ++s) {
      const int j = base + s * NT;
      if (j >= j1) continue;
      float *o = gs + (size_t)j * DD;
#pragma unroll
      for (int d = 0; d < DD; ++d) o[d] = acc[s][d];
    }
  }
}

template <bool FX>
__device__ void signal_gradient(const Cta &C, float *gs, int pst, int j0, int j1) {
  const KProgram &P = *C.P;
  float **padj = reinterpret_cast<float **>(C.scratch);   // free between node evaluations
  if (threadIdx.x < P.npred) padj[threadIdx.x] = C.rt[P.pred[threadIdx.x]].adj;
  __syncthreads();
  const int D = P.D;
  const float *xs = C.sig + C.row0 * D;
  const float i1 = C.ifx1, i2 = C.ifx2;
  switch (D) {
    case 1: signal_gradient_d<1, FX>(P, padj, xs, gs, pst, j0, j1, i1, i2); break;
    case 2: signal_gradient_d<2, FX>(P, padj, xs, gs, pst, j0, j1, i1, i2); break;
    case 3: signal_gradient_d<3, FX>(P, padj, xs, gs, pst, j0, j1, i1, i2); break;
    case 4: signal_gradient_d<4, FX>(P, padj, xs, gs, pst, j0, j1, i1, i2); break;
    default: {
      for (int idx = threadIdx.x; idx < (j1 - j0) * D; idx += blockDim.x) {
        const int j = j0 + idx / D, d = idx - (idx / D) * D;
        float acc = 0.f;
        for (int k = 0; k < P.npred; ++k) acc = fmaf(P.pw[k * STL_MAX_D + d], padj_at<FX>(padj, k, j - pst, i1, i2), acc);
        for (unsigned m = P.norm_mask; m; m &= m - 1) {
          const int k = __ffs(m) - 1;
          const float a = padj_at<FX>(padj, k, j - pst, i1, i2);
          if (a != 0.f) acc += norm_grad_dim(P, k, xs + (size_t)j * D, D, d, a);
        }
        gs[(size_t)j * D + d] = acc;
      }
    }
  }
}

// ------------------------------------------------------------------ main kernel
// Dense launches walk (trace, segment) items with a static stride and use the program passed
// by value.  Ragged launches (A.table != nullptr) take whole traces from an atomic work
// counter, in the caller's order, and read each trace's program from the device table.
// Dense and ragged launches are separate instantiations: in the dense one every program read
// resolves to the by-value parameter (constant bank), in the ragged one to the device table.
// A tighter register cap (three 256-thread CTAs per SM, 85 registers) made the forward
// re-load program fields inside its sample loops (measured 25-30% slower).
// Every size is held to 128 registers per thread (two 256-thread or eight 64-thread CTAs
// per SM); without the hint the 256-thread variants drift just past 128 and lose half their
// resident CTAs.  The smooth forward (one output per thread in its O(b) Until loops) runs
// three 256-thread CTAs per SM: measured 23 % faster on the nested formula at T = 10000.
template <int NT, bool BWD, bool SMOOTH, bool RAGGED>
__global__ void __launch_bounds__(NT, (NT == 64 ? 8 : NT == 256 ? ((SMOOTH && !BWD) ? 3 : 2) : 1))
    stl_main(const __grid_constant__ KProgram Pdense, LaunchArgs A) {
  extern __shared__ float4 smem4[];
  char *smem = reinterpret_cast<char *>(smem4);
  __shared__ long long s_item;
  __shared__ unsigned s_gmax;
  constexpr bool ragged = RAGGED;
  constexpr bool kLean = !BWD && !SMOOTH && NT == 512;
  Cta C;
  C.sig = A.sig;
  const int gwords = ragged ? A.gwords : Pdense.gwords;
  const int ut_len = ragged ? A.ut_len : Pdense.ut_len;
  const long long ut_off = ragged ? A.ut_off : Pdense.ut_off;
  float *ws_cta = A.ws ? A.ws + (size_t)blockIdx.x * (size_t)gwords : nullptr;
  float *ut = (A.ws && ut_len > 0) ? A.ws + ut_off + blockIdx.x * (long long)NT + threadIdx.x : nullptr;
  const long long ut_stride = (long long)gridDim.x * NT;
  const long long n_items = ragged ? A.n_traces : Pdense.n_items;
  if constexpr (!ragged) {
    C.P = &Pdense;
    C.T = (int)Pdense.T;
    C.rt = reinterpret_cast<NodeRt *>(smem + (size_t)Pdense.rt_off * 4);
    C.scratch = smem + (size_t)Pdense.scratch_off * 4;
    C.root = Pdense.n - 1;
  }

  for (long long it = 0;; ++it) {
    long long item;
    if constexpr (ragged) {
      if (threadIdx.x == 0) s_item = atomicAdd(A.counter, 1ULL);
      __syncthreads();
      item = s_item;
      __syncthreads();
    } else {
      item = blockIdx.x + it * (long long)gridDim.x;
    }
    if (item >= n_items) break;
    int s0, s1;
    if constexpr (ragged) {
      // per-trace data is checked here: a bad entry sets the status word and skips the trace
      const long long b = A.order ? (long long)A.order[item] : item;
      if (b < 0 || b >= A.n_traces) { if (threadIdx.x == 0 && A.status) atomicExch(A.status, 1); continue; }
      const int k = A.fid[b];
      const long long r0 = A.offsets[b], len = A.offsets[b + 1] - r0;
      if (k < 0 || k >= A.n_formulas || r0 < 0 || len > A.T_max) {
        if (threadIdx.x == 0 && A.status) atomicExch(A.status, 1);
        continue;
      }
      if (len <= 0) continue;
      // the plan of the smallest length bucket (T_max >> bk) that holds this trace
      int bk = 0;
      while (bk + 1 < A.n_buckets && (A.T_max >> (bk + 1)) >= len) ++bk;
      C.P = A.table + (size_t)k * A.n_buckets + bk;
      C.b = b;
      C.row0 = r0;
      C.T = (int)len;
      s0 = 0;
      s1 = C.T;
    } else {
      C.b = item / Pdense.segs_per_trace;
      C.row0 = C.b * (long long)C.T;
      const int sidx = (int)(item % Pdense.segs_per_trace);
      s0 = sidx * Pdense.seg;
      s1 = (s0 + Pdense.seg < C.T) ? s0 + Pdense.seg : C.T;
    }
    const KProgram &P = ragged ? *C.P : Pdense;
    const int T = C.T;
    if constexpr (ragged) {
      C.rt = reinterpret_cast<NodeRt *>(smem + (size_t)P.rt_off * 4);
      C.scratch = smem + (size_t)P.scratch_off * 4;
      C.root = P.n - 1;
    }
    C.out_row = BWD ? nullptr : A.out + C.row0;
    setup_geometry(C, A.bounds, ws_cta, smem, A.status);
    // hard and logsumexp backward launches keep their adjoints in 64-bit fixed point (two words
    // per sample): every weight of those adjoints is in [0, 1] (selections, softmax weights of
    // logsumexp reductions), so no adjoint exceeds the sum of |grad_out| over a trace and the
    // scale below cannot overflow; softmax-weighted launches keep float adjoints
    C.fx = BWD && (!SMOOTH || P.mode == 1);
    const int AW = C.fx ? 2 : 1;   // adjoint words per sample
    if (BWD) {
      for (int n = 0; n < P.n; ++n)
        if (C.rt[n].adj) zero_words(C.rt[n].adj, 0, AW * C.rt[n].cap);
      __syncthreads();
    }
    const int R0 = BWD ? (s0 - P.hmax > 0 ? s0 - P.hmax : 0) : s0;
    C.fx1 = C.fx2 = C.ifx1 = C.ifx2 = 1.f;
    if (C.fx) {
      // fixed-point scale from the largest root gradient of the whole trace (not only of this
      // item's samples: every segmentation of a trace then rounds the same way)
      if (threadIdx.x == 0) s_gmax = 0u;
      __syncthreads();
      float m = trace_gmax(A.gout + C.row0, T);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, off));
      if ((threadIdx.x & 31) == 0) atomicMax(&s_gmax, __float_as_uint(m));   // m >= 0: bits order as values
      __syncthreads();
      set_fix_scale(C, __uint_as_float(s_gmax));
    }
    for (int t0 = R0; t0 < s1; t0 += P.tile) {
      const int t1 = (t0 + P.tile < s1) ? t0 + P.tile : s1;
      C.t0 = t0;
      C.t1 = t1;
      // forward: values of every node on its new samples
      // (with D <= 4 every predicate is evaluated by one fused pass at the first predicate's
      // place; predicates are leaves, so each still precedes its parent)
      const bool fuse = P.D <= 4 && P.npred > 0;
      for (int n = 0; n < P.n; ++n) {
        if (fuse && is_pred_op(P.nd[n].op)) {
          if (n != P.pred[0]) continue;
          eval_preds(C, t0, R0);
          __syncthreads();
          continue;
        }
        const NodeRt &r = C.rt[n];
        const int F0 = (t0 == R0) ? R0 + r.lo : t0 + r.hi;
        const int F = F0 < T ? F0 : T;
        const int E = frontier(C, n);
        // hard forward nodes with many new samples take the direct-read passes (separate
        // functions: their call costs more than it saves on short steps, e.g. short traces)
        // (512-thread kernels only: the others serve short traces, and carrying the direct-read
        // passes made their code slower even where the passes were not taken)
        const bool lean = kLean && P.lean && E - F >= STL_LEAN_MIN_SAMPLES;
        const bool temporal = lean && is_temporal_op(P.nd[n].op);
        if (F < E) {
          // the children's samples past the end hold the pad before a lean temporal node
          // reads them
          if (temporal && pad_fill(C, n)) __syncthreads();
          eval_node<BWD, SMOOTH, kLean>(C, n, F, E, lean);
        }
        __syncthreads();
        if (temporal && n == C.root) {
          // a temporal root keeps its outputs in its buffer: copy them out coalesced
          const float *rv = r.val;
          const int st = t0 + r.lo;
          for (int q = F + threadIdx.x; q < E; q += NT) C.out_row[q] = rv[q - st];
        }
      }
      if (BWD && A.out) {
        // robustness and gradient in one launch: the backward has just recomputed the root's
        // values; copy out those of the samples this work item owns (not its warm-up)
        const NodeRt &rr = C.rt[C.root];
        const float *rv = rr.val;
        const int st = t0 + rr.lo;
        float *orow = A.out + C.row0;
        for (int q = (t0 > s0 ? t0 : s0) + threadIdx.x; q < t1; q += NT) orow[q] = rv[q - st];
      }
      if constexpr (BWD && !SMOOTH) {
        hard_walk(C, A.gout + C.row0, t0, t1);
        __syncthreads();
      }
      if constexpr (BWD && SMOOTH) {
        // root adjoint for [t0, t1), then nodes in reverse order
        {
          NodeRt &r = C.rt[C.root];
          float *ra = r.adj;
          const int st = t0 + r.lo;
          const float *g = A.gout + C.row0;
          for (int q = t0 + threadIdx.x; q < t1; q += NT) {
            const float v = __ldg(g + q);
            if (C.fx) {
              const unsigned long long f = (unsigned long long)to_fix(C, v);
              if (q == T - 1) r.padfx += f;
              else reinterpret_cast<unsigned long long *>(ra)[q - st] = f;
            } else {
              if (q == T - 1) r.padadj += v;
              else ra[q - st] = v;
            }
          }
        }
        __syncthreads();
        for (int n = P.n - 1; n >= 0; --n) {
          const NodeRt &r = C.rt[n];
          const int A0 = t0 + r.lo;
          int A1 = t1 + r.lo;
          A1 = A1 < T - 1 ? A1 : T - 1;
          if (A0 < A1) {
            if (is_until_op(P.nd[n].op)) {
              if (P.mode == 2) adjoint_soft_until(C, n, A0, A1, s0 + r.lo, s1 + r.lo, ut, ut_stride);
              else adjoint_smooth_until(C, n, A0, A1, s0 + r.lo, s1 + r.lo, ut, ut_stride);
            }
            else
              adjoint_node<SMOOTH>(C, n, A0, A1, s0 + r.lo, s1 + r.lo);
          }
          __syncthreads();
        }
      }
      if constexpr (BWD) {
        // signal gradient for the samples whose predicate adjoints are complete
        int j0 = t0 + P.lp, j1 = t1 + P.lp;
        j0 = j0 > s0 ? j0 : s0;
        j1 = j1 < s1 ? j1 : s1;
        j1 = j1 < T - 1 ? j1 : T - 1;
        const int D = P.D;
        if (t0 == R0) {
          // samples before the first predicate offset are read by no predicate: zero gradient
          const int z1 = j0 < T - 1 ? j0 : T - 1;
          for (int idx = threadIdx.x; idx < (z1 - s0) * D; idx += NT)
            A.gsig[(C.row0 + s0) * D + idx] = 0.f;
        }
        if (C.fx) signal_gradient<true>(C, A.gsig + C.row0 * D, t0 + P.lp, j0, j1);
        else signal_gradient<false>(C, A.gsig + C.row0 * D, t0 + P.lp, j0, j1);
        __syncthreads();
      }
      if (t1 < s1) shift_buffers<BWD>(C, P.tile, AW);
    }
    if constexpr (BWD) {
      if (s1 == T) {
        // finish sample T-1 of every node, parents first (all reads go to the T-1 cells);
        // the hard walk already delivered sample T-1 of every root sample
        for (int n = P.n - 1; SMOOTH && n >= 0; --n) {
          if (is_until_op(P.nd[n].op)) {
            if (P.mode == 2) adjoint_soft_until(C, n, T - 1, T, T - 1, T, ut, ut_stride);
            else adjoint_smooth_until(C, n, T - 1, T, T - 1, T, ut, ut_stride);
          }
          else
            adjoint_node<SMOOTH>(C, n, T - 1, T, T - 1, T);
          __syncthreads();
        }
        const int D = P.D;
        const float *xl = C.sig + (C.row0 + (T - 1)) * D;
        for (int d = threadIdx.x; d < D; d += NT) {
          auto pad_of = [&](int k) {
            const NodeRt &pr = C.rt[P.pred[k]];
            return C.fx ? from_fix(C.ifx1, C.ifx2, pr.padfx) : pr.padadj;
          };
          float acc = 0.f;
          for (int k = 0; k < P.npred; ++k) acc = fmaf(P.pw[k * STL_MAX_D + d], pad_of(k), acc);
          for (unsigned m = P.norm_mask; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const float a = pad_of(k);
            if (a != 0.f) acc += norm_grad_dim(P, k, xl, D, d, a);
          }
          A.gsig[(C.row0 + (T - 1)) * D + d] = acc;
        }
      }
      __syncthreads();
      if (A.gbounds && threadIdx.x == 0) {
        for (int n = 0; n < P.n; ++n) {
          const KNode &nd = P.nd[n];
          if ((nd.op == OP_EVSM || nd.op == OP_ALWSM || nd.op == OP_UNTSM) && nd.slot >= 0) {
            float *gb = A.gbounds + ((size_t)C.b * P.n_slots + nd.slot) * 2;
            atomicAdd(gb, C.rt[n].ga);
            atomicAdd(gb + 1, C.rt[n].gb);
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

// instantiation helpers used by the per-variant translation units
#define STL_DEFINE_VARIANT(NT, BWD, SM, RG, NAME)                                                 \
  int stl_launch_##NAME(const KProgram &P, const LaunchArgs &A, bool set_smem_attr) {            \
    const size_t smem = (size_t)P.smem_words * 4;                                                 \
    if (set_smem_attr) {                                                                          \
      cudaError_t e = cudaFuncSetAttribute(stl_main<NT, BWD, SM, RG>,                             \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return (int)e;                                                        \
    }                                                                                             \
    stl_main<NT, BWD, SM, RG><<<A.grid, NT, smem, (cudaStream_t)A.stream>>>(P, A);                \
    return (int)cudaGetLastError();                                                               \
  }                                                                                               \
  int stl_occupancy_##NAME(int smem_bytes, int *blocks) {                                         \
    cudaError_t e = cudaFuncSetAttribute(stl_main<NT, BWD, SM, RG>,                               \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes); \
    if (e != cudaSuccess) return (int)e;                                                          \
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, stl_main<NT, BWD, SM, RG>, NT, \
                                                              smem_bytes);                        \
  }
