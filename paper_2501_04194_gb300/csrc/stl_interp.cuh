// stl_interp.cuh -- streaming tile interpreter for STL robustness traces and their adjoints
// on sm_103a.
//
// One CTA owns one work item (trace b, segment [s0, s1)) at a time and walks it in steps of
// `tile` samples.  Every node of the formula keeps its robustness trace in a ring buffer
// (shared memory when it fits) covering the live range [t0 + lo, t1 + hi) of the step, so
// that intermediate traces never touch HBM: only the signal is read and only the root trace
// (forward) or the signal gradient (backward) is written.
//
// Temporal operators use a "thread-run" sliding-window decomposition: a thread owns R
// consecutive outputs; each output window is the combination of a suffix of the thread's
// first run, a fixed set of whole runs (shared through a small scratch array) and a prefix
// of a trailing run.  This is O(1) work per output for any window length and works for every
// associative combine used here:
//   max/min with the earliest selected sample                (hard Eventually / Always)
//   composition of clamp functions f_j(v) = min(phi_j, max(psi_j, v))  (hard Until)
//   (max, scaled sum) pairs of logsumexp                     (smooth windows and adjoints)
// The hard Until rests on  rho_t = min( min_{k<=a} phi_{t+k},
//                                       (f_{t+a} o ... o f_{t+b})(-inf) ),
// which follows from min distributing over max in the definition of Sec. IV-C.
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

#include "stl_internal.cuh"

namespace {

enum {
  OP_PGT = 0, OP_PLT = 1, OP_TRUE = 2, OP_NOT = 3, OP_AND = 4, OP_OR = 5, OP_EV = 6,
  OP_ALW = 7, OP_UNTIL = 8, OP_EVSM = 9, OP_ALWSM = 10
};

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ ring access
// Positions of the live range map to pos mod cap.  The clamp keeps any position outside the
// live range inside the ring, so a logic error cannot address memory beyond it.
__device__ __forceinline__ int ring_slot(const NodeRt &r, int pos) {
  int s = pos - r.base;
  s = (s >= r.cap) ? s - r.cap : s;
  s = s < 0 ? 0 : (s >= r.cap ? r.cap - 1 : s);
  return s + (s >> 5);   // one pad word per 32: stride-R thread runs avoid bank conflicts
}

// ------------------------------------------------------------------ combine monoids
struct VI { float v; int i; };
struct MaxM {
  using T = VI;
  static __device__ __forceinline__ T comb(T a, T b) { return b.v > a.v ? b : a; }
};
struct MinM {
  using T = VI;
  static __device__ __forceinline__ T comb(T a, T b) { return b.v < a.v ? b : a; }
};

// clamp function v -> min(d, max(c, v)), with the samples that supply c and d.  comb(L, R) is
// L o R (L covers the earlier samples).  Ties: max keeps L's bound, min keeps d.
struct CC { float c, d; int cs, ds; };
struct ClampM {
  using T = CC;
  static __device__ __forceinline__ T comb(T L, T R) {
    T o;
    float m = R.c > L.c ? R.c : L.c;
    int ms = R.c > L.c ? R.cs : L.cs;
    bool dl = L.d <= m;
    o.c = dl ? L.d : m;
    o.cs = dl ? L.ds : ms;
    float m2 = R.d > L.c ? R.d : L.c;
    int ms2 = R.d > L.c ? R.ds : L.cs;
    bool dl2 = L.d <= m2;
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
    if (b.m > a.m) { o.m = b.m; o.s = fmaf(a.s, expf(a.m - b.m), b.s); }
    else { o.m = a.m; o.s = fmaf(b.s, expf(b.m - a.m), a.s); }
    return o;
  }
};

// ------------------------------------------------------------------ window framework
// out(q, reduce_{i in [ia, ib]} elem(q + i)) for q in [q0, q1), combining in sample order.
template <class M, int R, class Elem, class Out>
__device__ __forceinline__ void window_reduce(int q0, int q1, int ia, int ib, const Elem &elem,
                                              const Out &out, typename M::T *runagg) {
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
  const int nf = K / R - 1;           // whole runs strictly inside every window (>= 1)
  const int rho = K - (nf + 1) * R;   // lead of the trailing prefix
  for (int p0 = q0; p0 < q1; p0 += NT * R) {
    const int u = p0 + tid * R;
    T hv[R];
    hv[R - 1] = elem(u + ia + R - 1);
#pragma unroll
    for (int k = R - 2; k >= 0; --k) hv[k] = M::comb(elem(u + ia + k), hv[k + 1]);
    runagg[tid] = hv[0];
    for (int e = tid; e < nf; e += NT) {
      const int s = p0 + ia + (NT + e) * R;
      T acc = elem(s);
#pragma unroll
      for (int k = 1; k < R; ++k) acc = M::comb(acc, elem(s + k));
      runagg[NT + e] = acc;
    }
    __syncthreads();
    T mid = runagg[tid + 1];
    for (int j = 2; j <= nf; ++j) mid = M::comb(mid, runagg[tid + j]);
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
    __syncthreads();
  }
}

template <class M, class Elem, class Out>
__device__ __forceinline__ void window_reduce_r(int R, int q0, int q1, int ia, int ib, const Elem &elem,
                                                const Out &out, void *scratch) {
  if (R == 16) window_reduce<M, 16>(q0, q1, ia, ib, elem, out, (typename M::T *)scratch);
  else window_reduce<M, 8>(q0, q1, ia, ib, elem, out, (typename M::T *)scratch);
}

// ------------------------------------------------------------------ interpreter state
struct Cta {
  const KProgram *P;
  NodeRt *rt;
  void *scratch;
  const float *sig;
  long long b;
  int T;
  int t1;              // end of the current root step
  int root;
  float *out_row;      // forward: out + b*T
};

__device__ __forceinline__ int frontier(const Cta &C, int n) {
  int e = C.t1 + C.rt[n].hi;
  return e < C.T ? e : C.T;
}

// value of child c read by parent node p at sample j (pads past T-1); src = gradient target
__device__ __forceinline__ float child_val(const Cta &C, const KNode &p, int c, int j, int &src) {
  const NodeRt &r = C.rt[c];
  if (j >= C.T) {
    if (p.pad_const) { src = -1; return p.pad_value; }
    src = C.T - 1;
    return r.lastval;
  }
  int f = frontier(C, c) - 1;
  j = j < f ? j : f;
  src = j;
  if (j == C.T - 1) return r.lastval;
  return r.val[ring_slot(r, j)];
}

// node m's own value / recorded source at sample q (sample T-1 lives in per-node cells,
// because at the end of a trace it can lie below the live range of the last step)
__device__ __forceinline__ float val_at(const Cta &C, int m, int q) {
  const NodeRt &r = C.rt[m];
  return q >= C.T - 1 ? r.lastval : r.val[ring_slot(r, q)];
}
__device__ __forceinline__ int aux_at(const Cta &C, int m, int q) {
  const NodeRt &r = C.rt[m];
  return q >= C.T - 1 ? r.lastaux : r.aux[ring_slot(r, q)];
}

// store node n's value at sample q (and clear its adjoint slot for the backward)
__device__ __forceinline__ void put(const Cta &C, int n, int q, float v) {
  NodeRt &r = C.rt[n];
  const int s = ring_slot(r, q);
  r.val[s] = v;
  if (r.adj) r.adj[s] = 0.f;
  if (q == C.T - 1) r.lastval = v;
  if (n == C.root && C.out_row) C.out_row[q] = v;
}

__device__ __forceinline__ void put_aux(const Cta &C, int n, int q, int src) {
  NodeRt &r = C.rt[n];
  if (r.aux) r.aux[ring_slot(r, q)] = src;
  if (q == C.T - 1) r.lastaux = src;
}

// ------------------------------------------------------------------ forward ops
__device__ void eval_pred(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const int D = P.D;
  const float *w = P.w + nd.w_off;
  const float *xs = C.sig + (size_t)C.b * (size_t)C.T * D;
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    const float *x = xs + (size_t)q * D;
    float s = __fmul_rn(w[0], x[0]);
    for (int d = 1; d < D; ++d) s = __fadd_rn(s, __fmul_rn(w[d], x[d]));
    put(C, n, q, nd.op == OP_PGT ? __fsub_rn(s, nd.pc) : __fsub_rn(nd.pc, s));
  }
}

__device__ void eval_elementwise(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const bool smooth = P.mode == 1;
  const float tau = P.tau, itau = P.inv_tau;
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    float v;
    if (nd.op == OP_TRUE) {
      v = INFINITY;
    } else if (nd.op == OP_NOT) {
      const NodeRt &a = C.rt[nd.c0];
      v = -a.val[ring_slot(a, q)];
    } else {
      const NodeRt &a = C.rt[nd.c0], &bq = C.rt[nd.c1];
      const float x = a.val[ring_slot(a, q)], y = bq.val[ring_slot(bq, q)];
      if (!smooth) {
        v = nd.op == OP_AND ? (x <= y ? x : y) : (x >= y ? x : y);
      } else {
        // two-term logsumexp min / max: min(x,y) - log1p(e^{-tau|x-y|}) / tau
        const float sg = nd.op == OP_AND ? 1.f : -1.f;
        const float xs = sg * x, ys = sg * y;
        const float m = xs < ys ? xs : ys;
        float dlt = fabsf(xs - ys);
        float corr = (xs == ys) ? 0.69314718f * itau : log1pf(expf(-tau * dlt)) * itau;
        if (isinf(xs) || isinf(ys)) corr = 0.f;
        v = sg * (m - corr);
      }
    }
    put(C, n, q, v);
  }
}

// hard window of node n over its child with offsets [ia, ib] (max for sgn>0, min otherwise)
__device__ void eval_hard_window(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KNode &nd = C.P->nd[n];
  const int c = nd.c0;
  auto elem = [&](int j) { VI r; r.v = child_val(C, nd, c, j, r.i); return r; };
  auto out = [&](int q, VI r) { put(C, n, q, r.v); put_aux(C, n, q, r.i); };
  const bool mx = nd.op == OP_EV || nd.op == OP_EVSM;
  if (mx) window_reduce_r<MaxM>(C.P->win_r, F, E, ia, ib, elem, out, C.scratch);
  else window_reduce_r<MinM>(C.P->win_r, F, E, ia, ib, elem, out, C.scratch);
}

// smooth window: (sgn/tau) log sum_i e^{sgn tau x_{q+i}}
__device__ void eval_smooth_window(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const int c = nd.c0;
  const float st = (nd.op == OP_EV ? 1.f : -1.f) * P.tau;
  const float sgn = nd.op == OP_EV ? 1.f : -1.f;
  auto elem = [&](int j) { int s; LS r; r.m = st * child_val(C, nd, c, j, s); r.s = 1.f; return r; };
  auto out = [&](int q, LS r) { put(C, n, q, sgn * (r.m + logf(r.s)) * P.inv_tau); };
  window_reduce_r<LseM>(P.win_r, F, E, ia, ib, elem, out, C.scratch);
}

// hard Until: pass 1 stores A_q = min_{k in [0,a]} phi_{q+k} (with its sample), pass 2
// composes the clamps over [a, b] and keeps min(A_q, V_{q+a}) with A winning ties.
__device__ void eval_hard_until(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KNode &nd = C.P->nd[n];
  const int cp = nd.c0, cq = nd.c1;
  {
    auto elem = [&](int j) { VI r; int s; r.v = child_val(C, nd, cp, j, s); r.i = s < 0 ? -1 : 2 * s; return r; };
    auto out = [&](int q, VI r) { put(C, n, q, r.v); put_aux(C, n, q, r.i); };
    window_reduce_r<MinM>(C.P->win_r, F, E, 0, ia, elem, out, C.scratch);
  }
  __syncthreads();
  auto elem = [&](int j) {
    CC r;
    int sp, sq;
    const float p = child_val(C, nd, cp, j, sp);
    const float q = child_val(C, nd, cq, j, sq);
    const int ep = sp < 0 ? -1 : 2 * sp, eq = sq < 0 ? -1 : 2 * sq + 1;
    const bool pl = p <= q;
    r.c = pl ? p : q;
    r.cs = pl ? ep : eq;
    r.d = p;
    r.ds = ep;
    return r;
  };
  auto out = [&](int q, CC r) {
    NodeRt &me = C.rt[n];
    const int s = ring_slot(me, q);
    const float A = me.val[s];
    if (!(A <= r.c)) {
      me.val[s] = r.c;
      if (me.aux) me.aux[s] = r.cs;
      if (q == C.T - 1) { me.lastval = r.c; me.lastaux = r.cs; }
      if (n == C.root && C.out_row) C.out_row[q] = r.c;
    }
  };
  window_reduce_r<ClampM>(C.P->win_r, F, E, ia, ib, elem, out, C.scratch);
}

// smooth Until (nested logsumexp, Sec. IV-C with Sec. III-C), one output per thread
__device__ void eval_smooth_until(const Cta &C, int n, int F, int E, int ia, int ib) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const float tau = P.tau, itau = P.inv_tau;
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    float M1 = -INFINITY, S1 = 0.f;   // sum_k e^{-tau phi}: (max exponent, scaled sum)
    float M2 = -INFINITY, S2 = 0.f;   // sum_i e^{tau z_i}
    for (int i = 0; i <= ib; ++i) {
      int s;
      const float zp = -tau * child_val(C, nd, nd.c0, q + i, s);
      if (zp != -INFINITY) {
        if (zp > M1) { S1 = fmaf(S1, expf(M1 - zp), 1.f); M1 = zp; }
        else S1 += expf(zp - M1);
      }
      if (i >= ia) {
        const float Pv = M1 == -INFINITY ? INFINITY : -(M1 + logf(S1)) * itau;
        const float qv = child_val(C, nd, nd.c1, q + i, s);
        float z;
        if (isinf(Pv) || isinf(qv)) z = Pv < qv ? Pv : qv;
        else z = fminf(Pv, qv) - log1pf(expf(-tau * fabsf(Pv - qv))) * itau;
        const float e = tau * z;
        if (e != -INFINITY) {
          if (e > M2) { S2 = fmaf(S2, expf(M2 - e), 1.f); M2 = e; }
          else S2 += expf(e - M2);
        }
      }
    }
    put(C, n, q, M2 == -INFINITY ? -INFINITY : (M2 + logf(S2)) * itau);
  }
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

__device__ __forceinline__ float smask(float i, float a, float b, float c, float eps) {
  float m = sigmoidf_(c * (i - a)) - sigmoidf_(c * (i - b)) - eps;
  return m > 0.f ? m : 0.f;
}

// smooth-mask window in smooth mode: (sgn/tau) log sum_i m_i e^{sgn tau x_{q+i}}
__device__ void eval_smooth_mask(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const NodeRt &me = C.rt[n];
  const float sgn = nd.op == OP_EVSM ? 1.f : -1.f;
  const float st = sgn * P.tau;
  for (int q = F + threadIdx.x; q < E; q += blockDim.x) {
    float M = -INFINITY, S = 0.f;
    for (int i = me.ia; i <= me.ib; ++i) {
      const float m = smask((float)i, me.fa, me.fb, P.mask_c, P.mask_eps);
      if (m <= 0.f) continue;
      int s;
      const float z = st * child_val(C, nd, nd.c0, q + i, s);
      if (z > M) { S = fmaf(S, expf(M - z), m); M = z; }
      else S = fmaf(m, expf(z - M), S);
    }
    put(C, n, q, M == -INFINITY ? sgn * -INFINITY : sgn * (M + logf(S)) * P.inv_tau);
  }
}

__device__ void eval_node(const Cta &C, int n, int F, int E) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  const NodeRt &r = C.rt[n];
  const bool smooth = P.mode == 1;
  switch (nd.op) {
    case OP_PGT:
    case OP_PLT: eval_pred(C, n, F, E); break;
    case OP_TRUE:
    case OP_NOT:
    case OP_AND:
    case OP_OR: eval_elementwise(C, n, F, E); break;
    case OP_EV:
    case OP_ALW:
      if (smooth) eval_smooth_window(C, n, F, E, r.ia, r.ib);
      else eval_hard_window(C, n, F, E, r.ia, r.ib);
      break;
    case OP_EVSM:
    case OP_ALWSM:
      if (smooth) eval_smooth_mask(C, n, F, E);
      else if (r.ia <= r.ib) eval_hard_window(C, n, F, E, r.ia, r.ib);
      break;
    case OP_UNTIL:
      if (smooth) eval_smooth_until(C, n, F, E, r.ia, r.ib);
      else eval_hard_until(C, n, F, E, r.ia, r.ib);
      break;
  }
}

// ------------------------------------------------------------------ adjoint helpers
__device__ __forceinline__ float adj_at(const Cta &C, int n, int q) {
  const NodeRt &r = C.rt[n];
  return q >= C.T - 1 ? r.padadj : r.adj[ring_slot(r, q)];
}

// add g to child c's adjoint at sample j (j already mapped to a real sample, or -1)
__device__ __forceinline__ void add_adj_atomic(const Cta &C, int c, int j, float g) {
  if (j < 0 || g == 0.f) return;
  NodeRt &r = C.rt[c];
  if (j >= C.T - 1) atomicAdd(&r.padadj, g);
  else atomicAdd(&r.adj[ring_slot(r, j)], g);
}
__device__ __forceinline__ void add_adj_owned(const Cta &C, int c, int j, float g) {
  if (j < 0) return;
  NodeRt &r = C.rt[c];
  if (j >= C.T - 1) { if (g != 0.f) atomicAdd(&r.padadj, g); }
  else r.adj[ring_slot(r, j)] += g;
}

// warp-aggregated scatter: lanes hold (key, g); runs of equal keys in consecutive lanes are
// summed first, then one atomic per run.  key encodes child*(2^30) + sample, or -1.
__device__ __forceinline__ void scatter_run(const Cta &C, int c_even, int c_odd, int key, float g, bool even_odd) {
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
    if (even_odd) add_adj_atomic(C, (key & 1) ? c_odd : c_even, key >> 1, s);
    else add_adj_atomic(C, c_even, key, s);
  }
}

__device__ __forceinline__ void accumulate_shared(float *dst, float v) {
  // warp reduction then one shared atomic
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
  if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(dst, v);
}

// ------------------------------------------------------------------ adjoint ops
// Adjoint of node n over its complete samples [A0, A1): adds into the children.
__device__ void adjoint_node(const Cta &C, int n, int A0, int A1, int own0, int own1) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  NodeRt &me = C.rt[n];
  const bool smooth = P.mode == 1;
  const float tau = P.tau;
  const int NT = blockDim.x;
  switch (nd.op) {
    case OP_PGT:
    case OP_PLT:
    case OP_TRUE:
      return;
    case OP_NOT:
      for (int q = A0 + threadIdx.x; q < A1; q += NT) add_adj_owned(C, nd.c0, q, -adj_at(C, n, q));
      return;
    case OP_AND:
    case OP_OR: {
      for (int q = A0 + threadIdx.x; q < A1; q += NT) {
        const float g = adj_at(C, n, q);
        const float x = val_at(C, nd.c0, q), y = val_at(C, nd.c1, q);
        if (!smooth) {
          const bool left = nd.op == OP_AND ? x <= y : x >= y;
          add_adj_owned(C, left ? nd.c0 : nd.c1, q, g);
        } else {
          const float sg = nd.op == OP_AND ? 1.f : -1.f;
          float wx, wy;
          if (isinf(x) && isinf(y)) { wx = 1.f; wy = 0.f; }
          else {
            wx = 1.f / (1.f + expf(-sg * tau * (y - x)));
            wy = 1.f / (1.f + expf(-sg * tau * (x - y)));
          }
          add_adj_owned(C, nd.c0, q, g * wx);
          add_adj_owned(C, nd.c1, q, g * wy);
        }
      }
      return;
    }
    case OP_EV:
    case OP_ALW:
    case OP_EVSM:
    case OP_ALWSM:
    case OP_UNTIL:
      break;
  }
  const bool is_until = nd.op == OP_UNTIL;
  const bool is_sm = nd.op == OP_EVSM || nd.op == OP_ALWSM;
  if (!smooth) {
    // hard: every complete sample sends its adjoint to the recorded source
    for (int qb = A0; qb < A1; qb += NT) {
      const int q = qb + threadIdx.x;
      int key = -1;
      float g = 0.f;
      if (q < A1) {
        g = adj_at(C, n, q);
        key = aux_at(C, n, q);
      }
      scatter_run(C, nd.c0, nd.c1, key, g, is_until);
    }
    return;
  }
  if (is_sm) {
    // smooth-mask window: direct scatter over the support, plus bound gradients
    const float sgn = nd.op == OP_EVSM ? 1.f : -1.f;
    const float c = P.mask_c, eps = P.mask_eps;
    float ga = 0.f, gbv = 0.f;
    for (int qb = A0; qb < A1; qb += NT) {
      const int q = qb + threadIdx.x;
      if (q < A1) {
        const float g = adj_at(C, n, q);
        const float y = val_at(C, n, q);
        const bool own = q >= own0 && q < own1;
        if (g != 0.f) {
          for (int i = me.ia; i <= me.ib; ++i) {
            const float fi = (float)i;
            const float sa = sigmoidf_(c * (fi - me.fa)), sb = sigmoidf_(c * (fi - me.fb));
            const float m = sa - sb - eps;
            if (m <= 0.f) continue;
            int src;
            const float x = child_val(C, nd, nd.c0, q + i, src);
            const float e = expf(sgn * tau * (x - y));
            add_adj_atomic(C, nd.c0, src, g * m * e);
            if (own) {
              ga += g * sgn * P.inv_tau * (-c * sa * (1.f - sa)) * e;
              gbv += g * sgn * P.inv_tau * (c * sb * (1.f - sb)) * e;
            }
          }
        }
      }
    }
    accumulate_shared(&me.ga, ga);
    accumulate_shared(&me.gb, gbv);
    return;
  }
  // smooth Eventually / Always: transposed window over the parent samples,
  // x̄_j += e^{sgn tau x_j} sum_{q in [j-b, j-a] ∩ [A0,A1)} g_q e^{-sgn tau y_q}
  {
    const float st = (nd.op == OP_EV ? 1.f : -1.f) * tau;
    const int ia = me.ia, ib = me.ib;
    auto elem = [&](int q) {
      LS r;
      if (q < A0 || q >= A1) { r.m = -INFINITY; r.s = 0.f; return r; }
      const float g = adj_at(C, n, q);
      r.m = -st * val_at(C, n, q);
      r.s = g;
      return r;
    };
    auto out = [&](int j, LS r) {
      if (r.m == -INFINITY || r.s == 0.f) return;
      int src;
      const float x = child_val(C, nd, nd.c0, j, src);
      if (src < 0) return;
      add_adj_owned(C, nd.c0, src, r.s * expf(st * x + r.m));
    };
    window_reduce_r<LseM>(P.win_r, A0 + ia, A1 + ib, -ib, -ia, elem, out, C.scratch);
  }
}

// smooth Until adjoint (kept separate: it needs a per-thread array of length b+1)
__device__ void adjoint_smooth_until(const Cta &C, int n, int A0, int A1, float *Pk, long long pstride) {
  const KProgram &P = *C.P;
  const KNode &nd = P.nd[n];
  NodeRt &me = C.rt[n];
  const float tau = P.tau, itau = P.inv_tau;
  const int ia = me.ia, ib = me.ib;
  for (int q = A0 + threadIdx.x; q < A1; q += blockDim.x) {
    const float g = adj_at(C, n, q);
    if (g == 0.f) continue;
    const float U = val_at(C, n, q);
    float M1 = -INFINITY, S1 = 0.f;
    // forward pass: P_k for k = 0..ib; psi adjoint on the fly
    for (int k = 0; k <= ib; ++k) {
      int s;
      const float zp = -tau * child_val(C, nd, nd.c0, q + k, s);
      if (zp != -INFINITY) {
        if (zp > M1) { S1 = fmaf(S1, expf(M1 - zp), 1.f); M1 = zp; }
        else S1 += expf(zp - M1);
      }
      const float Pv = M1 == -INFINITY ? INFINITY : -(M1 + logf(S1)) * itau;
      Pk[k * pstride] = Pv;
      if (k >= ia) {
        int sq;
        const float qv = child_val(C, nd, nd.c1, q + k, sq);
        float z;
        if (isinf(Pv) || isinf(qv)) z = Pv < qv ? Pv : qv;
        else z = fminf(Pv, qv) - log1pf(expf(-tau * fabsf(Pv - qv))) * itau;
        const float alpha = expf(tau * (z - U));
        const float gq = isinf(qv) ? 0.f : 1.f / (1.f + expf(-tau * (Pv - qv)));
        add_adj_atomic(C, nd.c1, sq, g * alpha * gq);
      }
    }
    // backward pass over k: D_k recursion
    float Dn = 0.f, Pnext = 0.f;
    for (int k = ib; k >= 0; --k) {
      const float Pv = Pk[k * pstride];
      float D = (k < ib && !isinf(Pv)) ? expf(tau * (Pnext - Pv)) * Dn : 0.f;
      if (k >= ia) {
        int sq;
        const float qv = child_val(C, nd, nd.c1, q + k, sq);
        float z;
        if (isinf(Pv) || isinf(qv)) z = Pv < qv ? Pv : qv;
        else z = fminf(Pv, qv) - log1pf(expf(-tau * fabsf(Pv - qv))) * itau;
        const float alpha = expf(tau * (z - U));
        const float beta = isinf(Pv) ? 0.f : 1.f / (1.f + expf(-tau * (qv - Pv)));
        D += alpha * beta;
      }
      int sp;
      const float pv = child_val(C, nd, nd.c0, q + k, sp);
      if (!isinf(pv) && !isinf(Pv)) add_adj_atomic(C, nd.c0, sp, g * expf(tau * (Pv - pv)) * D);
      Dn = D;
      Pnext = Pv;
    }
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
      if (nd.op == OP_EVSM || nd.op == OP_ALWSM) {
        // support {i >= 0 : sigma(c(i-a)) - sigma(c(i-b)) > eps} is an interval
        const double c = P.mask_c, eps = P.mask_eps;
        const double L = log((1.0 - eps) / eps) / c;
        int lo = (int)floor((double)a - L) - 1;
        int hi = (int)ceil((double)b + L) + 2;
        lo = lo < 0 ? 0 : lo;
        while (lo <= hi && smask_d(lo, a, b, c, eps) <= 0.0) ++lo;
        while (hi >= lo && smask_d(hi, a, b, c, eps) <= 0.0) --hi;
        r.ia = lo;
        r.ib = hi;
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
      r.ga = r.gb = 0.f;
      r.base = 0;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ main kernel
template <int NT>
__global__ void __launch_bounds__(NT) stl_main(const __grid_constant__ KProgram P, LaunchArgs A) {
  extern __shared__ float4 smem4[];
  char *smem = reinterpret_cast<char *>(smem4);
  Cta C;
  C.P = &P;
  C.rt = reinterpret_cast<NodeRt *>(smem + (size_t)P.rt_off * 4);
  C.scratch = smem + (size_t)P.scratch_off * 4;
  C.sig = A.sig;
  C.T = (int)P.T;
  C.root = P.n - 1;
  float *ws_cta = A.ws ? A.ws + (size_t)blockIdx.x * (size_t)P.gwords : nullptr;
  float *ut = (A.ws && P.ut_len > 0) ? A.ws + P.ut_off + blockIdx.x * (long long)NT + threadIdx.x : nullptr;
  const long long ut_stride = (long long)gridDim.x * NT;
  const int T = C.T;

  for (long long item = blockIdx.x; item < P.n_items; item += gridDim.x) {
    C.b = item / P.segs_per_trace;
    const int sidx = (int)(item % P.segs_per_trace);
    const int s0 = sidx * P.seg;
    const int s1 = (s0 + P.seg < T) ? s0 + P.seg : T;
    C.out_row = P.bwd ? nullptr : A.out + (size_t)C.b * T;
    setup_geometry(C, A.bounds, ws_cta, smem, A.status);
    const int R0 = P.bwd ? (s0 - P.hmax > 0 ? s0 - P.hmax : 0) : s0;
    for (int t0 = R0; t0 < s1; t0 += P.tile) {
      const int t1 = (t0 + P.tile < s1) ? t0 + P.tile : s1;
      C.t1 = t1;
      if (threadIdx.x < P.n) {
        NodeRt &r = C.rt[threadIdx.x];
        const int L = t0 + r.lo;
        r.base = (L / r.cap) * r.cap;
      }
      __syncthreads();
      // forward: values of every node on its new samples
      for (int n = 0; n < P.n; ++n) {
        const NodeRt &r = C.rt[n];
        const int F0 = (t0 == R0) ? R0 + r.lo : t0 + r.hi;
        const int F = F0 < T ? F0 : T;
        const int E = frontier(C, n);
        if (F < E) eval_node(C, n, F, E);
        __syncthreads();
      }
      if (!P.bwd) continue;
      // backward: root adjoint for [t0, t1), then nodes in reverse order
      {
        NodeRt &r = C.rt[C.root];
        const float *g = A.gout + (size_t)C.b * T;
        for (int q = t0 + threadIdx.x; q < t1; q += NT) {
          if (q == T - 1) r.padadj += g[q];
          else r.adj[ring_slot(r, q)] = g[q];
        }
      }
      __syncthreads();
      for (int n = P.n - 1; n >= 0; --n) {
        const NodeRt &r = C.rt[n];
        const int A0 = t0 + r.lo;
        int A1 = t1 + r.lo;
        A1 = A1 < T - 1 ? A1 : T - 1;
        if (A0 < A1) {
          if (P.mode == 1 && P.nd[n].op == OP_UNTIL)
            adjoint_smooth_until(C, n, A0, A1, ut, ut_stride);
          else
            adjoint_node(C, n, A0, A1, s0 + r.lo, s1 + r.lo);
        }
        __syncthreads();
      }
      // signal gradient for the samples whose predicate adjoints are complete
      {
        int j0 = t0 + P.lp, j1 = t1 + P.lp;
        j0 = j0 > s0 ? j0 : s0;
        j1 = j1 < s1 ? j1 : s1;
        j1 = j1 < T - 1 ? j1 : T - 1;
        const int D = P.D;
        if (t0 == R0) {
          // samples before the first predicate offset are read by no predicate: zero gradient
          const int z1 = j0 < T - 1 ? j0 : T - 1;
          for (int idx = threadIdx.x; idx < (z1 - s0) * D; idx += NT)
            A.gsig[((size_t)C.b * T + s0) * D + idx] = 0.f;
        }
        for (int idx = threadIdx.x; idx < (j1 - j0) * D; idx += NT) {
          const int j = j0 + idx / D, d = idx - (idx / D) * D;
          float acc = 0.f;
          for (int n = 0; n < P.n; ++n) {
            const KNode &nd = P.nd[n];
            if (nd.op != OP_PGT && nd.op != OP_PLT) continue;
            const NodeRt &r = C.rt[n];
            const float w = P.w[nd.w_off + d];
            const float g = r.adj[ring_slot(r, j)];
            acc = fmaf(nd.op == OP_PGT ? w : -w, g, acc);
          }
          A.gsig[((size_t)C.b * T + j) * D + d] = acc;
        }
      }
      __syncthreads();
    }
    if (P.bwd) {
      if (s1 == T) {
        // finish sample T-1 of every node, parents first
        for (int n = P.n - 1; n >= 0; --n) {
          if (P.mode == 1 && P.nd[n].op == OP_UNTIL)
            adjoint_smooth_until(C, n, T - 1, T, ut, ut_stride);
          else
            adjoint_node(C, n, T - 1, T, T - 1, T);
          __syncthreads();
        }
        const int D = P.D;
        for (int d = threadIdx.x; d < D; d += NT) {
          float acc = 0.f;
          for (int n = 0; n < P.n; ++n) {
            const KNode &nd = P.nd[n];
            if (nd.op != OP_PGT && nd.op != OP_PLT) continue;
            const float w = P.w[nd.w_off + d];
            acc = fmaf(nd.op == OP_PGT ? w : -w, C.rt[n].padadj, acc);
          }
          A.gsig[((size_t)C.b * T + (T - 1)) * D + d] = acc;
        }
      }
      __syncthreads();
      if (A.gbounds && threadIdx.x == 0) {
        for (int n = 0; n < P.n; ++n) {
          const KNode &nd = P.nd[n];
          if ((nd.op == OP_EVSM || nd.op == OP_ALWSM) && nd.slot >= 0) {
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
