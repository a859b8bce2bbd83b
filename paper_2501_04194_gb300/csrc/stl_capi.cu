// stl_capi.cu -- host side of libstl: formula validation, per-call ring layout, launch shape
// selection and the extern "C" entry points declared in include/stl.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/stl.h"
#include "stl_internal.cuh"
#include "stl_fk.h"

namespace {

thread_local std::string g_err;

stl_status fail(stl_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

stl_status cuda_fail(int e, const char *what) {
  return fail(STL_ERR_CUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
}

bool is_until(int op) { return op == STL_OP_UNTIL || op == STL_OP_UNTIL_SM; }
bool is_temporal(int op) {
  return op == STL_OP_EVENTUALLY || op == STL_OP_ALWAYS || is_until(op) ||
         op == STL_OP_EVENTUALLY_SM || op == STL_OP_ALWAYS_SM;
}
bool is_sm(int op) { return op == STL_OP_EVENTUALLY_SM || op == STL_OP_ALWAYS_SM || op == STL_OP_UNTIL_SM; }
bool is_window(int op) {
  return op == STL_OP_EVENTUALLY || op == STL_OP_ALWAYS || op == STL_OP_EVENTUALLY_SM || op == STL_OP_ALWAYS_SM;
}
bool soft_mode(int mode) { return mode == STL_SMOOTH || mode == STL_SOFTMAX; }
// per-thread arrays of the smooth Until backward, in units of (taps x threads)
int until_arrays(int mode) { return mode == STL_SOFTMAX ? 3 : 2; }
bool is_norm(int op) { return op == STL_OP_NORM_GT || op == STL_OP_NORM_LT; }
bool is_pred(int op) { return op == STL_OP_PRED_GT || op == STL_OP_PRED_LT || is_norm(op); }
int arity(int op) {
  switch (op) {
    case STL_OP_PRED_GT: case STL_OP_PRED_LT: case STL_OP_NORM_GT: case STL_OP_NORM_LT:
    case STL_OP_TRUE: return 0;
    case STL_OP_NOT: case STL_OP_EVENTUALLY: case STL_OP_ALWAYS:
    case STL_OP_EVENTUALLY_SM: case STL_OP_ALWAYS_SM: return 1;
    case STL_OP_AND: case STL_OP_OR: case STL_OP_UNTIL: case STL_OP_UNTIL_SM: return 2;
    default: return -1;
  }
}

int round_up(long long v, int m) { return (int)(((v + m - 1) / m) * m); }

}  // namespace

struct stl_program {
  std::vector<stl_node> nodes;
  std::vector<float> w;
  int D = 0, n_slots = 0;
  bool has_sm = false, has_until = false;
  stl_launch launch_dir[2]{};   // [forward, backward]: explicit or tuned launch shapes
  stl_launch launch{};          // the shape used by the planner for the current direction
  // the pipelined host calls: their helper streams and the events that join them
  cudaStream_t pst[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
};

// A group of formulas evaluated together in one ragged launch.  The device table holds one
// program per formula for the prepared (T_max, semantics, direction).
struct SetState {
  bool ready = false;
  long long T_max = 0;
  stl_params p{};
  KProgram *dtable = nullptr;   // device copy (allocated at prepare time): [formula][bucket]
  size_t table_len = 0;         // programs the device table holds
  int n_buckets = 1;
  int threads = 256, grid = 1, smem_words = 0, gwords = 0, ut_len = 0;
  long long ut_off = 0;
  size_t ws_bytes = 0;
  stl_launch shape{};           // threads / tile of the launch (zero: the planner's choice)
};

struct stl_program_set {
  std::vector<stl_program *> formulas;
  int D = 0, n_slots = 0;
  SetState st[2];   // [forward, backward]
};

namespace {

struct Plan {
  KProgram P;
  int threads = 256;
  int grid = 1;
  size_t ws_bytes = 0;
};

// largest window span (b) a node can reach for this call
int window_hi(const stl_node &nd, long long T, const stl_params &p) {
  if (is_sm(nd.op)) {
    const double L = std::log((1.0 - p.mask_eps) / p.mask_eps) / p.mask_c;
    return (int)std::ceil((double)nd.b + L) + 2;
  }
  if (std::isinf(nd.b)) return (int)(T - 1);
  return (int)nd.b;
}
int window_lo(const stl_node &nd) {
  if (nd.bound_slot >= 0 || is_sm(nd.op)) return 0;
  return (int)nd.a;
}

// Compute node geometry, ring layout and launch shape for one call.
stl_status make_plan(const stl_program *hp, long long B, long long T, const stl_params &p, bool bwd, Plan &pl,
                     int force_threads = 0, int force_tile = 0) {
  stl_program hv = *hp;               // shallow copy carrying this direction's launch shape
  hv.launch = hp->launch_dir[bwd ? 1 : 0];
  const stl_program *h = &hv;
  KProgram &P = pl.P;
  std::memset(&P, 0, sizeof P);
  const int n = (int)h->nodes.size();
  P.n = n;
  P.D = h->D;
  P.n_slots = h->n_slots;
  P.mode = p.mode;
  P.tau = soft_mode(p.mode) ? p.tau : 1.f;
  P.inv_tau = 1.f / P.tau;
  P.mask_c = p.mask_c;
  P.mask_eps = p.mask_eps;
  P.bwd = bwd ? 1 : 0;
  P.T = T;
  P.B = B;
  std::copy(h->w.begin(), h->w.end(), P.w);

  // offsets: values run ahead by hi, adjoints complete behind by lo (root: 0, 0)
  std::vector<int> lo(n, 0), hi(n, 0);
  int maxK = 1;
  for (int i = n - 1; i >= 0; --i) {
    const stl_node &nd = h->nodes[i];
    const int a0 = window_lo(nd), b1 = window_hi(nd, T, p);
    if (is_temporal(nd.op)) maxK = std::max(maxK, b1 - a0 + 1);
    if (nd.child0 >= 0) {
      const int c = nd.child0;
      if (is_temporal(nd.op)) {
        lo[c] = lo[i] + (is_until(nd.op) ? 0 : a0);
        hi[c] = hi[i] + b1;
      } else { lo[c] = lo[i]; hi[c] = hi[i]; }
    }
    if (nd.child1 >= 0) {
      const int c = nd.child1;
      if (is_until(nd.op)) { lo[c] = lo[i] + a0; hi[c] = hi[i] + b1; }
      else { lo[c] = lo[i]; hi[c] = hi[i]; }
    }
  }
  // A node never stores samples at or past T (those reads go to the per-node cells), so its
  // live span hi - lo need not exceed T: long nested windows on short traces (ragged length
  // buckets) keep buffers of at most tile + T samples.  Hard forward plans that may take the
  // direct-read passes keep the full span (they fill pads past T into the buffers).
  const bool may_lean = !bwd && p.mode == STL_HARD;
  if (!may_lean)
    for (int i = 0; i < n; ++i) hi[i] = (int)std::min<long long>(hi[i], (long long)lo[i] + T);
  int lp = 1 << 30;
  for (int i = 0; i < n; ++i) if (is_pred(h->nodes[i].op)) lp = std::min(lp, lo[i]);
  if (lp == (1 << 30)) lp = 0;
  for (int i = 0; i < n; ++i) if (is_pred(h->nodes[i].op)) lo[i] = lp;
  int hmax = 0;
  for (int i = 0; i < n; ++i) hmax = std::max(hmax, hi[i]);
  P.hmax = hmax;
  P.lp = lp;

  int sms = 0, max_smem = 0;
  int e = stl_num_sms(&sms);
  if (e) return cuda_fail(e, "cudaDeviceGetAttribute(multiprocessors)");
  e = stl_max_smem_optin(&max_smem);
  if (e) return cuda_fail(e, "cudaDeviceGetAttribute(max shared memory)");
  max_smem -= 1024;   // the kernel's own static shared variables

  // A window pass covers threads x R outputs; by default the tile equals one pass and is the
  // largest that keeps every ring in shared memory.
  const int win_r = 7;    // thread-run length of the windows (odd: conflict-free strides)
  P.win_r = win_r;
  // measured defaults: forward launches prefer several 256-thread CTAs per SM, backward
  // launches (larger per-sample state) one or two 512-thread CTAs; short traces (one step of
  // at most two 64-thread passes) run many 64-thread CTAs per SM
  int threads = force_threads ? force_threads
                : h->launch.threads ? h->launch.threads
                : T <= 2 * 64 * win_r ? 64
                : (bwd ? 512 : 256);
  int tile = force_tile ? force_tile : h->launch.tile ? h->launch.tile : threads * win_r;
  tile = std::min(tile, round_up(T, 32));
  tile = std::max(32, round_up(tile, 32));

  // hard forward plans whose node steps can reach STL_LEAN_MIN_SAMPLES samples allocate every
  // buffer with STL_BUF_BACK words after its live range: their direct-read window passes read
  // a few samples past the range without clamping (those reads feed no output)
  int maxspan = 0;
  for (int i = 0; i < n; ++i) maxspan = std::max(maxspan, hi[i] - lo[i]);
  const bool lean_mode = !bwd && p.mode == STL_HARD;   // the 512-thread forward kernels take them
  auto slack_for = [&](int tl) {
    return (lean_mode && threads == 512 && (long long)tl + maxspan >= STL_LEAN_MIN_SAMPLES) ? STL_BUF_BACK : 0;
  };
  int slack = 0;
  auto padded = [&](int cap) { return cap + slack; };
  // window scratch: run aggregates (threads + K/7) and their blocks of 8, 16 bytes each (24
  // for the double-precision sums of the softmax-weighted adjoint); the signal gradient reuses
  // it for the predicate adjoint pointers
  const int entry_words = (bwd && p.mode == STL_SOFTMAX) ? 6 : 4;
  auto scratch_for = [&](int nt) {
    const int runs = nt + maxK / 7 + 4;
    return std::max((runs + runs / 8 + 8) * entry_words, 2 * STL_MAX_PRED);
  };
  auto layout = [&](int tl, std::vector<int> &space_out, int &smem_words, int &gwords) {
    slack = slack_for(tl);
    // scratch for window run aggregates: (threads + maxK/R + 2) entries of up to 16 bytes
    const int scratch_words = scratch_for(threads);
    const int rt_words = (int)((n * sizeof(NodeRt) + 15) / 16 * 4);
    std::vector<int> words(n);
    for (int i = 0; i < n; ++i) {
      const stl_node &nd = h->nodes[i];
      const int cap = round_up((long long)tl + hi[i] - lo[i], 4);
      int nrings = 1;
      if (bwd) {
        // hard backward: only predicates keep an adjoint (selection walk; 64-bit fixed-point
        // sums, two words per sample), temporal nodes keep their selected samples; logsumexp
        // backward: every node keeps a fixed-point adjoint; softmax-weighted: a float one
        if (p.mode == STL_SOFTMAX) nrings += 1;
        else if (p.mode == STL_SMOOTH || is_pred(nd.op)) nrings += 2;
        if (p.mode == STL_HARD && is_temporal(nd.op)) nrings += 1;
        // softmax windows keep each output's log-normaliser for their adjoint
        if (p.mode == STL_SOFTMAX && is_window(nd.op)) nrings += 1;
      }
      words[i] = nrings * padded(cap);
    }
    int tab_words = 0;
    for (int i = 0; i < n; ++i)
      if (is_sm(h->nodes[i].op) && soft_mode(p.mode))
        tab_words += round_up(3LL * (window_hi(h->nodes[i], T, p) + 2), 4);
    space_out.assign(n, 0);
    smem_words = scratch_words + rt_words + tab_words;
    for (int i = 0; i < n; ++i) smem_words += words[i];
    gwords = 0;
    // spill the largest rings to the global workspace until the arena fits
    while ((long long)smem_words * 4 > max_smem) {
      int best = -1;
      for (int i = 0; i < n; ++i)
        if (space_out[i] == 0 && (best < 0 || words[i] > words[best])) best = i;
      if (best < 0) break;
      space_out[best] = 1;
      smem_words -= words[best];
      gwords += words[best];
    }
    return (long long)smem_words * 4 <= max_smem;
  };
  std::vector<int> space;
  int smem_words = 0, gwords = 0;
  // shrink the tile while rings would have to leave shared memory -- but only if a smaller
  // tile avoids the spill: when even 256-sample steps spill (long nested windows), a large
  // tile amortises the per-step cost and the spilled rings stay L2-resident
  const bool fixed_tile = h->launch.tile || force_tile;
  bool spill_unavoidable = false;
  if (!fixed_tile) {
    std::vector<int> sp;
    int sw = 0, gw = 0;
    const int t_min = std::min(tile, 256);
    spill_unavoidable = layout(t_min, sp, sw, gw) && gw > 0;
  }
  for (;;) {
    bool ok = layout(tile, space, smem_words, gwords);
    if (!ok) return fail(STL_ERR_UNSUPPORTED, "formula scratch does not fit in shared memory");
    if (gwords == 0 || tile <= 256 || fixed_tile || spill_unavoidable) break;
    tile = std::max(256, round_up(tile / 2, 32));
    if (!force_threads && !h->launch.threads && tile < 512 * win_r) threads = 256;
  }
  P.tile = tile;
  slack = slack_for(tile);
  P.lean = slack > 0;

  // assign offsets
  int off_s = 0, off_g = 0;
  for (int i = 0; i < n; ++i) {
    const stl_node &nd = h->nodes[i];
    KNode &k = P.nd[i];
    k.op = nd.op;
    k.c0 = nd.child0;
    k.c1 = nd.child1;
    k.slot = nd.bound_slot;
    k.parent = -1;
    k.a = nd.a;
    k.b = nd.b;
    k.pad_const = nd.pad_mode == STL_PAD_CONST;
    k.pad_value = nd.pad_value;
    k.w_off = nd.pred_offset;
    k.pc = nd.pred_c;
    k.lo = lo[i];
    k.hi = hi[i];
    k.cap = round_up((long long)tile + hi[i] - lo[i], 4);
    k.space = space[i];
    int &off = space[i] ? off_g : off_s;
    const int pw = padded(k.cap);
    k.val_off = off; off += pw;
    k.adj_off = -1;
    k.aux_off = -1;
    if (bwd) {
      if (p.mode == STL_SOFTMAX) { k.adj_off = off; off += pw; }
      else if (p.mode == STL_SMOOTH || is_pred(nd.op)) { k.adj_off = off; off += 2 * pw; }   // 64-bit fixed point
      if ((p.mode == STL_HARD && is_temporal(nd.op)) || (p.mode == STL_SOFTMAX && is_window(nd.op))) {
        k.aux_off = off;
        off += pw;
      }
    }
    k.tab_off = -1;
    k.tab_len = 0;
  }
  // smooth-mask weight tables live in shared memory after the buffers
  for (int i = 0; i < n; ++i) {
    if (!(is_sm(h->nodes[i].op) && soft_mode(p.mode))) continue;
    KNode &k = P.nd[i];
    k.tab_len = window_hi(h->nodes[i], T, p) + 2;
    k.tab_off = off_s;
    off_s += round_up(3LL * k.tab_len, 4);
  }
  for (int i = 0; i < n; ++i) {
    if (P.nd[i].c0 >= 0) P.nd[P.nd[i].c0].parent = i;
    if (P.nd[i].c1 >= 0) P.nd[P.nd[i].c1].parent = i;
  }
  P.npred = 0;
  P.norm_mask = 0;
  for (int i = 0; i < n; ++i) {
    const stl_node &nd = h->nodes[i];
    if (!is_pred(nd.op)) continue;
    const int k = P.npred++;
    P.pred[k] = i;
    if (is_norm(nd.op)) P.norm_mask |= 1u << k;
    for (int d = 0; d < h->D; ++d)
      P.pw[k * STL_MAX_D + d] = is_norm(nd.op) ? 0.f
                                : nd.op == STL_OP_PRED_GT ? h->w[nd.pred_offset + d] : -h->w[nd.pred_offset + d];
  }
  const int scratch_words = scratch_for(threads);
  P.scratch_off = round_up(off_s, 4);
  P.scratch_words = scratch_words;
  P.rt_off = P.scratch_off + scratch_words;
  P.smem_words = P.rt_off + (int)((n * sizeof(NodeRt) + 15) / 16 * 4);
  P.gwords = round_up(off_g, 64);

  // launch shape
  int bps = 0;
  e = stl_blocks_per_sm(threads, bwd ? 1 : 0, soft_mode(p.mode) ? 1 : 0, 0, P.smem_words * 4, &bps);
  if (e) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (bps < 1) return fail(STL_ERR_UNSUPPORTED, "kernel does not fit on an SM (%d B shared)", P.smem_words * 4);
  const long long slots = (long long)sms * bps;
  int segs = 1;
  if (h->launch.segment > 0) {
    segs = (int)((T + h->launch.segment - 1) / h->launch.segment);
  } else if (B < 2 * slots) {
    // split traces so that there are about two items per resident CTA, while keeping
    // segments long compared with the backward warm-up
    const long long want = (2 * slots + B - 1) / B;
    const long long max_by_len = std::max(1LL, T / std::max(4LL * (hmax + tile), (long long)tile));
    segs = (int)std::max(1LL, std::min(want, max_by_len));
  }
  P.seg = (int)((T + segs - 1) / segs);
  P.segs_per_trace = (int)((T + P.seg - 1) / P.seg);
  P.n_items = B * P.segs_per_trace;
  pl.grid = (int)std::max(1LL, std::min(P.n_items, slots));
  pl.threads = threads;

  // smooth-until per-thread arrays
  size_t ws_words = (size_t)P.gwords * pl.grid;
  P.ut_len = 0;
  P.ut_off = (long long)ws_words;
  if (bwd && soft_mode(p.mode)) {
    int ut = 0;
    for (int i = 0; i < n; ++i)
      if (is_until(h->nodes[i].op)) ut = std::max(ut, window_hi(h->nodes[i], T, p) + 1);
    // per thread: logsumexp, two words per checkpoint (every 8th tap); softmax-weighted, P_k,
    // z_k and log S_k per tap (its double-precision prefix reduction is too costly to recompute)
    if (p.mode == STL_SMOOTH) ut = ut / 8 + 2;
    P.ut_len = ut;
    ws_words += (size_t)until_arrays(p.mode) * ut * pl.grid * threads;
  }
  pl.ws_bytes = ws_words * 4;
  return STL_OK;
}

stl_status check_params(const stl_program *h, const stl_params *p) {
  if (!p) return fail(STL_ERR_INVALID_ARG, "params is NULL");
  if (p->mode != STL_HARD && p->mode != STL_SMOOTH && p->mode != STL_SOFTMAX)
    return fail(STL_ERR_INVALID_ARG, "mode must be STL_HARD, STL_SMOOTH or STL_SOFTMAX");
  if (soft_mode(p->mode) && !(p->tau > 0.f && std::isfinite(p->tau)))
    return fail(STL_ERR_INVALID_ARG, "tau must be finite and > 0 in the smooth modes");
  if (h->has_sm) {
    if (!(p->mask_c > 0.f && std::isfinite(p->mask_c))) return fail(STL_ERR_INVALID_ARG, "mask_c must be finite and > 0");
    if (!(p->mask_eps > 0.f && p->mask_eps < 1.f)) return fail(STL_ERR_INVALID_ARG, "mask_eps must be in (0, 1)");
  }
  return STL_OK;
}

stl_status check_call(const stl_program *h, const float *sig, long long B, long long T, const float *bounds,
                      const stl_params *p) {
  if (!h) return fail(STL_ERR_INVALID_ARG, "handle is NULL");
  if (B < 0) return fail(STL_ERR_INVALID_ARG, "B must be >= 0");
  if (T < 1 || T > (1LL << 30)) return fail(STL_ERR_INVALID_ARG, "T must be in [1, 2^30]");
  if (B > 0 && !sig) return fail(STL_ERR_INVALID_ARG, "signal pointer is NULL");
  if (h->n_slots > 0 && B > 0 && !bounds) return fail(STL_ERR_INVALID_ARG, "formula uses per-trace bounds but bounds is NULL");
  return check_params(h, p);
}

}  // namespace

extern "C" {

const char *stl_version(void) { return "libstl 0.1 (sm_103a)"; }

const char *stl_status_string(int32_t s) {
  switch (s) {
    case STL_OK: return "ok";
    case STL_ERR_INVALID_ARG: return "invalid argument";
    case STL_ERR_UNSUPPORTED: return "unsupported";
    case STL_ERR_CUDA: return "CUDA error";
    case STL_ERR_WORKSPACE: return "workspace too small";
    case STL_ERR_TIMEOUT: return "device wait timed out";
    case STL_ERR_DEVICE_CHECK: return "device-side data check failed";
    default: return "unknown status";
  }
}

const char *stl_last_error(void) { return g_err.c_str(); }

stl_status stl_compile(const stl_node *nodes, int32_t n_nodes, const float *pred_weights, int32_t n_w,
                       int32_t D, int32_t n_slots, stl_handle *out) {
  if (!out) return fail(STL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!nodes || n_nodes < 1 || n_nodes > STL_MAX_NODES)
    return fail(STL_ERR_INVALID_ARG, "n_nodes must be in [1, %d]", STL_MAX_NODES);
  if (D < 1 || D > STL_MAX_D) return fail(STL_ERR_INVALID_ARG, "D must be in [1, %d]", STL_MAX_D);
  if (n_w < 0 || n_w > STL_MAX_WEIGHTS || (n_w > 0 && !pred_weights))
    return fail(STL_ERR_INVALID_ARG, "pred_weights: need 0 <= n_w <= %d and a pointer", STL_MAX_WEIGHTS);
  if (n_slots < 0 || n_slots > 64) return fail(STL_ERR_INVALID_ARG, "n_slots must be in [0, 64]");
  for (int i = 0; i < n_w; ++i)
    if (!std::isfinite(pred_weights[i])) return fail(STL_ERR_INVALID_ARG, "predicate weight %d is not finite", i);
  std::vector<int> parents(n_nodes, 0);
  bool has_sm = false, has_until = false;
  for (int i = 0; i < n_nodes; ++i) {
    const stl_node &nd = nodes[i];
    const int ar = arity(nd.op);
    if (ar < 0) return fail(STL_ERR_INVALID_ARG, "node %d: unknown op %d", i, nd.op);
    const int kids[2] = {nd.child0, nd.child1};
    for (int k = 0; k < 2; ++k) {
      if (k < ar) {
        if (kids[k] < 0 || kids[k] >= i)
          return fail(STL_ERR_INVALID_ARG, "node %d: child %d must be an earlier node", i, k);
        parents[kids[k]]++;
      } else if (kids[k] != -1) {
        return fail(STL_ERR_INVALID_ARG, "node %d: unused child %d must be -1", i, k);
      }
    }
    if (is_pred(nd.op)) {
      if (nd.pred_offset < 0 || nd.pred_offset + (is_norm(nd.op) ? 2 * D : D) > n_w)
        return fail(STL_ERR_INVALID_ARG, "node %d: predicate weights out of range", i);
      if (!std::isfinite(nd.pred_c)) return fail(STL_ERR_INVALID_ARG, "node %d: predicate constant not finite", i);
    }
    if (is_temporal(nd.op)) {
      if (nd.bound_slot < -1 || nd.bound_slot >= n_slots)
        return fail(STL_ERR_INVALID_ARG, "node %d: bound_slot out of range", i);
      if (!(nd.a >= 0.f) || !(nd.b >= nd.a) || std::isnan(nd.b))
        return fail(STL_ERR_INVALID_ARG, "node %d: need 0 <= a <= b", i);
      if (is_sm(nd.op)) {
        if (std::isinf(nd.b)) return fail(STL_ERR_INVALID_ARG, "node %d: smooth-mask bounds must be finite", i);
        has_sm = true;
      } else {
        if (nd.a != std::floor(nd.a) || (!std::isinf(nd.b) && nd.b != std::floor(nd.b)))
          return fail(STL_ERR_INVALID_ARG, "node %d: interval bounds must be integers", i);
      }
      if (!std::isinf(nd.b) && nd.b > (float)(1 << 24)) return fail(STL_ERR_INVALID_ARG, "node %d: b too large", i);
      if (nd.pad_mode != STL_PAD_LAST && nd.pad_mode != STL_PAD_CONST)
        return fail(STL_ERR_INVALID_ARG, "node %d: pad_mode must be STL_PAD_LAST or STL_PAD_CONST", i);
      if (nd.pad_mode == STL_PAD_CONST && !std::isfinite(nd.pad_value))
        return fail(STL_ERR_INVALID_ARG, "node %d: pad_value not finite", i);
      if (is_until(nd.op)) has_until = true;
    }
  }
  int npred = 0;
  for (int i = 0; i < n_nodes; ++i) npred += is_pred(nodes[i].op);
  if (npred > STL_MAX_PRED) return fail(STL_ERR_INVALID_ARG, "at most %d predicates per formula", STL_MAX_PRED);
  for (int i = 0; i < n_nodes - 1; ++i)
    if (parents[i] != 1) return fail(STL_ERR_INVALID_ARG, "node %d must have exactly one parent (tree, root last)", i);
  if (parents[n_nodes - 1] != 0) return fail(STL_ERR_INVALID_ARG, "the root (last node) cannot have a parent");
  stl_program *h = new (std::nothrow) stl_program;
  if (!h) return fail(STL_ERR_INVALID_ARG, "out of host memory");
  h->nodes.assign(nodes, nodes + n_nodes);
  h->w.assign(pred_weights, pred_weights + n_w);
  h->D = D;
  h->n_slots = n_slots;
  h->has_sm = has_sm;
  h->has_until = has_until;
  *out = h;
  return STL_OK;
}

void stl_destroy(stl_handle h) {
  if (!h) return;
  for (cudaEvent_t e : h->pev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t q : h->pst)
    if (q) cudaStreamDestroy(q);
  delete h;
}

namespace {
FkFormula fk_formula(const stl_program *h) { return FkFormula{&h->nodes, &h->w, h->D, h->n_slots}; }

// which kernel serves this call: the handle's choice for the direction, or (automatic) the
// formula-compiled kernel where it applies to a call of at least 2^20 samples
stl_status resolve_kernel(const stl_program *h, long long B, long long T, const stl_params &p, bool bwd, int *kind) {
  const int want = h->launch_dir[bwd ? 1 : 0].kernel;
  std::string why;
  if (want == STL_KERNEL_INTERPRETER) { *kind = want; return STL_OK; }
  const bool ok = stl_fk_eligible(fk_formula(h), p, T, &why) && stl_fk_available(&why);
  if (want == STL_KERNEL_COMPILED) {
    if (!ok) return fail(STL_ERR_UNSUPPORTED, "compiled kernel not applicable: %s", why.c_str());
    *kind = want;
    return STL_OK;
  }
  // automatic: the compiled kernel unless a launch shape for the interpreter was set, or its
  // buffers would not fit in shared memory even at the smallest tile
  const stl_launch &l = h->launch_dir[bwd ? 1 : 0];
  const bool shape_set = l.tile || l.threads || l.segment;
  bool use = ok && !shape_set && B * T >= (1LL << 20);
  if (use) {
    std::string err;
    use = stl_fk_plan_shape(fk_formula(h), bwd, 0, 0, nullptr, nullptr, nullptr, &err) == STL_OK;
  }
  *kind = use ? STL_KERNEL_COMPILED : STL_KERNEL_INTERPRETER;
  return STL_OK;
}

stl_status fk_launch(const stl_program *h, bool bwd, long long B, long long T, const float *sig, const float *gout,
                     float *out, float *gsig, void *ws, size_t ws_bytes, void *stream) {
  FkCall c;
  c.bwd = bwd;
  c.B = B;
  c.T = T;
  c.sig = sig;
  c.gout = gout;
  c.out = out;
  c.gsig = gsig;
  const stl_launch &l = h->launch_dir[bwd ? 1 : 0];
  c.threads = l.threads;
  c.tile = l.tile;
  c.segment = l.segment;
  c.ws = ws;
  c.ws_bytes = ws_bytes;
  c.stream = stream;
  std::string err;
  stl_status s = stl_fk_run(fk_formula(h), c, &err);
  if (s) return fail(s, "%s", err.c_str());
  return STL_OK;
}
}  // namespace

stl_status stl_set_launch(stl_handle h, const stl_launch *launch) {
  if (!h || !launch) return fail(STL_ERR_INVALID_ARG, "NULL argument");
  if (launch->threads && launch->threads != 64 && launch->threads != 256 && launch->threads != 512 &&
      !(launch->kernel == STL_KERNEL_COMPILED && (launch->threads == 768 || launch->threads == 1024)))
    return fail(STL_ERR_INVALID_ARG, "threads must be 0, 64, 256 or 512 (compiled kernels: 256, 512, 768, 1024)");
  if (launch->tile < 0 || (launch->tile && launch->tile % 32) || launch->segment < 0)
    return fail(STL_ERR_INVALID_ARG, "tile must be a non-negative multiple of 32; segment >= 0");
  if (launch->kernel < STL_KERNEL_AUTO || launch->kernel > STL_KERNEL_COMPILED)
    return fail(STL_ERR_INVALID_ARG, "kernel must be STL_KERNEL_AUTO, _INTERPRETER or _COMPILED");
  if (launch->kernel == STL_KERNEL_COMPILED && launch->threads == 64)
    return fail(STL_ERR_INVALID_ARG, "compiled kernels run 256 or 512 threads");
  h->launch_dir[0] = h->launch_dir[1] = *launch;
  return STL_OK;
}

stl_status stl_get_launch(stl_handle h, int64_t B, int64_t T, const stl_params *p, int32_t backward,
                          stl_launch *out) {
  if (!out) return fail(STL_ERR_INVALID_ARG, "out is NULL");
  stl_status s = check_call(h, (const float *)1, B, T, (const float *)1, p);
  if (s) return s;
  int kind = 0;
  s = resolve_kernel(h, B, T, *p, backward != 0, &kind);
  if (s) return s;
  if (kind == STL_KERNEL_COMPILED) {
    const stl_launch &l = h->launch_dir[backward ? 1 : 0];
    int tile = 0;
    std::string err;
    s = stl_fk_plan_shape(fk_formula(h), backward != 0, l.threads, l.tile, &tile, nullptr, nullptr, &err);
    if (s) return fail(s, "%s", err.c_str());
    out->tile = tile;
    out->threads = l.threads ? l.threads : 512;
    out->segment = l.segment;
    out->kernel = STL_KERNEL_COMPILED;
    return STL_OK;
  }
  Plan pl;
  s = make_plan(h, B, T, *p, backward != 0, pl);
  if (s) return s;
  out->tile = pl.P.tile;
  out->threads = pl.threads;
  out->segment = pl.P.seg;
  out->kernel = STL_KERNEL_INTERPRETER;
  return STL_OK;
}

stl_status stl_compile_kernel(stl_handle h, int32_t backward, int64_t T, const stl_launch *launch, int32_t *tile_out,
                              int32_t *smem_bytes) {
  if (!h) return fail(STL_ERR_INVALID_ARG, "handle is NULL");
  if (T < 1 || T > (1LL << 30)) return fail(STL_ERR_INVALID_ARG, "T must be in [1, 2^30]");
  stl_params hp{};
  hp.mode = STL_HARD;
  std::string why;
  if (!stl_fk_eligible(fk_formula(h), hp, T, &why)) return fail(STL_ERR_UNSUPPORTED, "%s", why.c_str());
  const int nt = launch ? launch->threads : 0, tile = launch ? launch->tile : 0;
  if (tile < 0 || tile % 32) return fail(STL_ERR_INVALID_ARG, "tile must be a non-negative multiple of 32");
  int to = 0, sm = 0;
  std::string err;
  stl_status s = stl_fk_compile_only(fk_formula(h), backward != 0, T, nt, tile, &to, &sm, nullptr, &err);
  if (s) return fail(s, "%s", err.c_str());
  if (tile_out) *tile_out = to;
  if (smem_bytes) *smem_bytes = sm;
  return STL_OK;
}

stl_status stl_workspace_size(stl_handle h, int64_t B, int64_t T, const stl_params *p, int32_t backward,
                              size_t *bytes) {
  if (!bytes) return fail(STL_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 0;
  stl_status s = check_call(h, (const float *)1, B, T, (const float *)1, p);
  if (s) return s;
  if (B == 0) return STL_OK;
  int kind = 0;
  s = resolve_kernel(h, B, T, *p, backward != 0, &kind);
  if (s) return s;
  if (kind == STL_KERNEL_COMPILED) {
    const stl_launch &l = h->launch_dir[backward ? 1 : 0];
    std::string err;
    s = stl_fk_plan_shape(fk_formula(h), backward != 0, l.threads, l.tile, nullptr, nullptr, bytes, &err);
    if (s) return fail(s, "%s", err.c_str());
    return STL_OK;
  }
  Plan pl;
  s = make_plan(h, B, T, *p, backward != 0, pl);
  if (s) return s;
  *bytes = pl.ws_bytes;
  return STL_OK;
}

stl_status stl_robustness(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds,
                          const stl_params *p, float *out, void *workspace, size_t workspace_bytes,
                          void *stream) {
  stl_status s = check_call(h, sig, B, T, bounds, p);
  if (s) return s;
  if (B > 0 && !out) return fail(STL_ERR_INVALID_ARG, "out is NULL");
  if (B == 0) return STL_OK;
  int kind = 0;
  s = resolve_kernel(h, B, T, *p, false, &kind);
  if (s) return s;
  if (kind == STL_KERNEL_COMPILED)
    return fk_launch(h, false, B, T, sig, nullptr, out, nullptr, workspace, workspace_bytes, stream);
  Plan pl;
  s = make_plan(h, B, T, *p, false, pl);
  if (s) return s;
  if (pl.ws_bytes > 0 && (!workspace || workspace_bytes < pl.ws_bytes))
    return fail(STL_ERR_WORKSPACE, "workspace of %zu bytes needed", pl.ws_bytes);
  LaunchArgs A{};
  int e0 = stl_status_ptr(&A.status);
  if (e0) return cuda_fail(e0, "cudaGetSymbolAddress(status)");
  A.sig = sig;
  A.bounds = h->n_slots ? bounds : nullptr;
  A.out = out;
  A.ws = (float *)workspace;
  A.grid = pl.grid;
  A.threads = pl.threads;
  A.stream = stream;
  int e = stl_launch_main(pl.P, A);
  if (e) return cuda_fail(e, "robustness kernel launch");
  return STL_OK;
}

namespace {
// backward launch; with out non-NULL the same launch also writes rho (every node's trace is
// recomputed by the backward anyway, so rho costs only its stores)
stl_status backward_launch(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds,
                           const stl_params *p, const float *grad_out, float *out, float *grad_sig,
                           float *grad_bounds, void *workspace, size_t workspace_bytes, void *stream) {
  stl_status s = check_call(h, sig, B, T, bounds, p);
  if (s) return s;
  if (B > 0 && (!grad_out || !grad_sig)) return fail(STL_ERR_INVALID_ARG, "grad_out / grad_sig is NULL");
  if (B == 0) return STL_OK;
  int kind = 0;
  s = resolve_kernel(h, B, T, *p, true, &kind);
  if (s) return s;
  if (kind == STL_KERNEL_COMPILED)
    return fk_launch(h, true, B, T, sig, grad_out, out, grad_sig, workspace, workspace_bytes, stream);
  Plan pl;
  s = make_plan(h, B, T, *p, true, pl);
  if (s) return s;
  if (pl.ws_bytes > 0 && (!workspace || workspace_bytes < pl.ws_bytes))
    return fail(STL_ERR_WORKSPACE, "workspace of %zu bytes needed", pl.ws_bytes);
  if (grad_bounds && h->n_slots > 0) {
    cudaError_t e = cudaMemsetAsync(grad_bounds, 0, (size_t)B * h->n_slots * 2 * sizeof(float), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail((int)e, "cudaMemsetAsync(grad_bounds)");
  }
  LaunchArgs A{};
  int e0 = stl_status_ptr(&A.status);
  if (e0) return cuda_fail(e0, "cudaGetSymbolAddress(status)");
  A.sig = sig;
  A.bounds = h->n_slots ? bounds : nullptr;
  A.gout = grad_out;
  A.out = out;
  A.gsig = grad_sig;
  A.gbounds = h->n_slots ? grad_bounds : nullptr;
  A.ws = (float *)workspace;
  A.grid = pl.grid;
  A.threads = pl.threads;
  A.stream = stream;
  int e = stl_launch_main(pl.P, A);
  if (e) return cuda_fail(e, "robustness backward kernel launch");
  return STL_OK;
}
}  // namespace

stl_status stl_robustness_backward(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds,
                                   const stl_params *p, const float *grad_out, float *grad_sig,
                                   float *grad_bounds, void *workspace, size_t workspace_bytes, void *stream) {
  return backward_launch(h, sig, B, T, bounds, p, grad_out, nullptr, grad_sig, grad_bounds, workspace,
                         workspace_bytes, stream);
}

stl_status stl_robustness_and_backward(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds,
                                       const stl_params *p, const float *grad_out, float *out, float *grad_sig,
                                       float *grad_bounds, void *workspace, size_t workspace_bytes,
                                       void *stream) {
  if (B > 0 && !out) return fail(STL_ERR_INVALID_ARG, "out is NULL");
  return backward_launch(h, sig, B, T, bounds, p, grad_out, out, grad_sig, grad_bounds, workspace,
                         workspace_bytes, stream);
}

// ------------------------------------------------------------------ host-buffer pipeline
namespace {
struct Staging {   // one slot of the double-buffered device staging area
  size_t sig, bnd, g, out, gsig, gb, ws, bytes;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int kPipeSlots = 3;   // chunk k: copies in, kernels, copies out on slot k mod 3

stl_status staging_layout(const stl_program *h, long long chunk, long long T, const stl_params &p, bool bwd,
                          Staging &L) {
  const size_t c = (size_t)chunk, t = (size_t)T, D = (size_t)h->D, S = (size_t)h->n_slots;
  // workspace of whichever kernel serves a chunk (interpreter or formula-compiled)
  size_t ws = 0, wb = 0;
  stl_status e = stl_workspace_size(const_cast<stl_program *>(h), chunk, T, &p, 0, &ws);
  if (e) return e;
  if (bwd) {
    e = stl_workspace_size(const_cast<stl_program *>(h), chunk, T, &p, 1, &wb);
    if (e) return e;
    ws = std::max(ws, wb);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += align256(bytes); return o; };
  L.sig = take(c * t * D * 4);
  L.bnd = take(c * S * 2 * 4);
  L.g = take(bwd ? c * t * 4 : 0);
  L.out = take(c * t * 4);
  L.gsig = take(bwd ? c * t * D * 4 : 0);
  L.gb = take(bwd ? c * S * 2 * 4 : 0);
  L.ws = take(ws);
  L.bytes = off;
  return STL_OK;
}
}  // namespace

stl_status stl_pipeline_staging_size(stl_handle h, int64_t chunk, int64_t T, const stl_params *p, int32_t backward,
                                     size_t *bytes) {
  if (!h || !p || !bytes) return fail(STL_ERR_INVALID_ARG, "NULL argument");
  if (chunk < 1 || T < 1 || T > (1LL << 30)) return fail(STL_ERR_INVALID_ARG, "need chunk >= 1 and T in [1, 2^30]");
  stl_status s = check_params(h, p);
  if (s) return s;
  Staging L;
  s = staging_layout(h, chunk, T, *p, backward != 0, L);
  if (s) return s;
  *bytes = kPipeSlots * L.bytes;
  return STL_OK;
}

stl_status stl_robustness_host_pipelined(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds,
                                         const stl_params *p, const float *grad_out, float *out, float *grad_sig,
                                         float *grad_bounds, int64_t chunk, void *staging, size_t staging_bytes,
                                         void *stream) {
  stl_status s = check_call(h, sig, B, T, bounds, p);
  if (s) return s;
  const bool bwd = grad_out != nullptr;
  if (bwd && !grad_sig) return fail(STL_ERR_INVALID_ARG, "grad_sig is NULL");
  if (!bwd && !out) return fail(STL_ERR_INVALID_ARG, "nothing to compute: out and grad_out are NULL");
  if (chunk < 1) return fail(STL_ERR_INVALID_ARG, "chunk must be >= 1");
  if (B == 0) return STL_OK;
  chunk = std::min<int64_t>(chunk, B);
  Staging L;
  s = staging_layout(h, chunk, T, *p, bwd, L);
  if (s) return s;
  if (!staging || staging_bytes < kPipeSlots * L.bytes)
    return fail(STL_ERR_WORKSPACE, "staging of %zu bytes needed (stl_pipeline_staging_size)", kPipeSlots * L.bytes);
  for (int i = 0; i < kPipeSlots; ++i)
    if (!h->pst[i] && cudaStreamCreateWithFlags(&h->pst[i], cudaStreamNonBlocking) != cudaSuccess) {
      h->pst[i] = nullptr;
      return fail(STL_ERR_CUDA, "cudaStreamCreate");
    }
  for (int i = 0; i < kPipeSlots + 1; ++i)
    if (!h->pev[i] && cudaEventCreateWithFlags(&h->pev[i], cudaEventDisableTiming) != cudaSuccess) {
      h->pev[i] = nullptr;
      return fail(STL_ERR_CUDA, "cudaEventCreate");
    }
  cudaStream_t caller = (cudaStream_t)stream;
  // the helper streams start after everything already queued on the caller's stream
  if (cudaEventRecord(h->pev[kPipeSlots], caller) != cudaSuccess) return fail(STL_ERR_CUDA, "cudaEventRecord");
  for (int i = 0; i < kPipeSlots; ++i)
    if (cudaStreamWaitEvent(h->pst[i], h->pev[kPipeSlots], 0) != cudaSuccess) return fail(STL_ERR_CUDA, "stream join");
  const size_t D = (size_t)h->D, S = (size_t)h->n_slots, t = (size_t)T;
  const auto H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
  for (int64_t c0 = 0, k = 0; c0 < B; c0 += chunk, ++k) {
    const int64_t n = std::min<int64_t>(chunk, B - c0);
    const int slot = (int)(k % kPipeSlots);
    cudaStream_t q = h->pst[slot];
    char *base = (char *)staging + slot * L.bytes;
    float *dsig = (float *)(base + L.sig), *dbnd = (float *)(base + L.bnd), *dg = (float *)(base + L.g);
    float *dout = (float *)(base + L.out), *dgs = (float *)(base + L.gsig), *dgb = (float *)(base + L.gb);
    void *dws = base + L.ws;
    const size_t ws_bytes = L.bytes - L.ws;
    cudaError_t ce = cudaMemcpyAsync(dsig, sig + (size_t)c0 * t * D, (size_t)n * t * D * 4, H2D, q);
    if (ce == cudaSuccess && S && bounds)
      ce = cudaMemcpyAsync(dbnd, bounds + (size_t)c0 * S * 2, (size_t)n * S * 2 * 4, H2D, q);
    if (ce == cudaSuccess && bwd) ce = cudaMemcpyAsync(dg, grad_out + (size_t)c0 * t, (size_t)n * t * 4, H2D, q);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "cudaMemcpyAsync (host to device)");
    if (out) {
      s = stl_robustness(h, dsig, n, T, S ? dbnd : nullptr, p, dout, dws, ws_bytes, q);
      if (s) return s;
    }
    if (bwd) {
      s = stl_robustness_backward(h, dsig, n, T, S ? dbnd : nullptr, p, dg, dgs, (S && grad_bounds) ? dgb : nullptr,
                                  dws, ws_bytes, q);
      if (s) return s;
    }
    if (out) {
      ce = cudaMemcpyAsync(out + (size_t)c0 * t, dout, (size_t)n * t * 4, D2H, q);
      if (ce != cudaSuccess) return cuda_fail((int)ce, "cudaMemcpyAsync (device to host)");
    }
    if (bwd) {
      ce = cudaMemcpyAsync(grad_sig + (size_t)c0 * t * D, dgs, (size_t)n * t * D * 4, D2H, q);
      if (ce == cudaSuccess && S && grad_bounds)
        ce = cudaMemcpyAsync(grad_bounds + (size_t)c0 * S * 2, dgb, (size_t)n * S * 2 * 4, D2H, q);
      if (ce != cudaSuccess) return cuda_fail((int)ce, "cudaMemcpyAsync (device to host)");
    }
  }
  // the caller's stream completes after all three pipelines
  for (int i = 0; i < kPipeSlots; ++i)
    if (cudaEventRecord(h->pev[i], h->pst[i]) != cudaSuccess || cudaStreamWaitEvent(caller, h->pev[i], 0) != cudaSuccess)
      return fail(STL_ERR_CUDA, "stream join");
  return STL_OK;
}

stl_status stl_get_device_status(void *stream, int32_t *status) {
  if (!status) return fail(STL_ERR_INVALID_ARG, "status is NULL");
  int st = 0;
  int e = stl_read_clear_status(stream, &st);
  if (e) return cuda_fail(e, "reading the device status");
  *status = st == 2 ? STL_ERR_TIMEOUT : st ? STL_ERR_DEVICE_CHECK : STL_OK;
  return STL_OK;
}

}  // extern "C"

// Internal: plan a backward launch whose workspace must fit in `capacity_bytes`; the grid is
// reduced (items are then walked by fewer resident CTAs) until it fits.  Used by the
// allocation-free entry point in stl_noalloc.cu.
stl_status stl_internal_plan_backward_capped(stl_handle h, const float *sig, int64_t B, int64_t T,
                                             const float *bounds, const stl_params *p, size_t capacity_bytes,
                                             KProgram *prog, int *grid, int *threads, size_t *ws_bytes) {
  stl_status s = check_call(h, sig, B, T, bounds, p);
  if (s) return s;
  if (B == 0) {   // nothing to launch: no plan, as in stl_robustness_backward
    *grid = 0;
    *threads = 0;
    *ws_bytes = 0;
    return STL_OK;
  }
  Plan pl;
  s = make_plan(h, B, T, *p, true, pl);
  if (s) return s;
  size_t per_cta_words = (size_t)pl.P.gwords + (size_t)until_arrays(p->mode) * pl.P.ut_len * pl.threads;
  if (per_cta_words * 4 > capacity_bytes && pl.threads > 64) {
    // the smooth Until's per-thread arrays scale with the CTA size: try the smallest CTAs
    Plan small;
    s = make_plan(h, B, T, *p, true, small, 64);
    if (s) return s;
    const size_t w64 = (size_t)small.P.gwords + (size_t)until_arrays(p->mode) * small.P.ut_len * small.threads;
    if (w64 < per_cta_words) {
      pl = small;
      per_cta_words = w64;
    }
  }
  if (per_cta_words * 4 > capacity_bytes)
    return fail(STL_ERR_WORKSPACE, "one CTA needs %zu bytes of scratch, the static scratch holds %zu",
                per_cta_words * 4, capacity_bytes);
  int g = pl.grid;
  const size_t fit = capacity_bytes / (per_cta_words * 4 > 0 ? per_cta_words * 4 : 1);
  if (per_cta_words > 0 && (size_t)g > fit) g = (int)fit;
  pl.P.ut_off = (long long)pl.P.gwords * g;
  *prog = pl.P;
  *grid = g;
  *threads = pl.threads;
  *ws_bytes = per_cta_words * 4 * (size_t)g;
  return STL_OK;
}

stl_status stl_internal_fail(stl_status st, const char *msg) { return fail(st, "%s", msg); }

// ------------------------------------------------------------------ formula sets (ragged)
extern "C" {

stl_status stl_set_create(const stl_handle *formulas, int32_t n_formulas, stl_set_handle *out) {
  if (!out) return fail(STL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!formulas || n_formulas < 1 || n_formulas > 65536)
    return fail(STL_ERR_INVALID_ARG, "n_formulas must be in [1, 65536]");
  stl_program_set *s = new (std::nothrow) stl_program_set;
  if (!s) return fail(STL_ERR_INVALID_ARG, "out of host memory");
  for (int i = 0; i < n_formulas; ++i) {
    if (!formulas[i]) { delete s; return fail(STL_ERR_INVALID_ARG, "formula %d is NULL", i); }
    if (i && formulas[i]->D != formulas[0]->D) {
      delete s;
      return fail(STL_ERR_INVALID_ARG, "formula %d has D=%d, formula 0 has D=%d", i, formulas[i]->D,
                  formulas[0]->D);
    }
    s->formulas.push_back(formulas[i]);
    s->n_slots = std::max(s->n_slots, formulas[i]->n_slots);
  }
  s->D = formulas[0]->D;
  *out = s;
  return STL_OK;
}

void stl_set_destroy(stl_set_handle s) {
  if (!s) return;
  for (auto &st : s->st)
    if (st.dtable) cudaFree(st.dtable);
  delete s;
}

stl_status stl_set_prepare(stl_set_handle s, int64_t n_traces, int64_t T_max, const stl_params *p,
                           int32_t backward, size_t *workspace_bytes) {
  if (!s || !p || !workspace_bytes) return fail(STL_ERR_INVALID_ARG, "NULL argument");
  if (n_traces < 1 || T_max < 1 || T_max > (1LL << 30)) return fail(STL_ERR_INVALID_ARG, "need n_traces >= 1 and T_max in [1, 2^30]");
  SetState &st = s->st[backward ? 1 : 0];
  const int nf = (int)s->formulas.size();
  // length buckets: every formula is planned for traces of at most T_max, T_max/2, T_max/4, ...
  // (down to 1024 samples, at most STL_MAX_BUCKETS plans); a trace runs the plan of the
  // smallest bucket that holds it, whose buffers and tile fit its length
  int nb = 1;
  while (nb < STL_MAX_BUCKETS && (T_max >> nb) >= 1024 && (long long)nf * (nb + 1) <= 8192) ++nb;
  std::vector<KProgram> progs((size_t)nf * nb);
  const int threads = st.shape.threads ? st.shape.threads : T_max <= 2 * 64 * 7 ? 64 : backward ? 512 : 256;
  int smem = 0, gwords = 0, ut_len = 0;
  for (int k = 0; k < nf; ++k) {
    stl_status e = check_params(s->formulas[k], p);
    if (e) return e;
    for (int bk = 0; bk < nb; ++bk) {
      const long long Tb = T_max >> bk;
      Plan pl;
      e = make_plan(s->formulas[k], n_traces, Tb, *p, backward != 0, pl, threads,
                    st.shape.tile ? (int)std::min<long long>(st.shape.tile, ((Tb + 31) / 32) * 32) : 0);
      if (e) return e;
      pl.P.n_slots = s->n_slots;          // one bounds array for the whole set
      pl.P.seg = (int)Tb;
      pl.P.segs_per_trace = 1;
      progs[(size_t)k * nb + bk] = pl.P;
      smem = std::max(smem, pl.P.smem_words);
      gwords = std::max(gwords, pl.P.gwords);
      ut_len = std::max(ut_len, pl.P.ut_len);
    }
  }
  int sms = 0, bps = 0;
  int e = stl_num_sms(&sms);
  if (e) return cuda_fail(e, "cudaDeviceGetAttribute(multiprocessors)");
  e = stl_blocks_per_sm(threads, backward ? 1 : 0, soft_mode(p->mode) ? 1 : 0, 1, smem * 4, &bps);
  if (e) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (bps < 1) return fail(STL_ERR_UNSUPPORTED, "kernel does not fit on an SM (%d B shared)", smem * 4);
  const long long grid = std::max(1LL, std::min((long long)sms * bps, (long long)n_traces));
  for (auto &P : progs) {
    P.smem_words = smem;   // every program sees the launch's shared arena
  }
  if (st.dtable && st.table_len < progs.size()) {
    cudaFree(st.dtable);
    st.dtable = nullptr;
  }
  if (!st.dtable) {
    cudaError_t ce = cudaMalloc((void **)&st.dtable, sizeof(KProgram) * progs.size());
    if (ce != cudaSuccess) { st.dtable = nullptr; return cuda_fail((int)ce, "cudaMalloc(program table)"); }
    st.table_len = progs.size();
  }
  cudaError_t ce = cudaMemcpy(st.dtable, progs.data(), sizeof(KProgram) * progs.size(), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return cuda_fail((int)ce, "cudaMemcpy(program table)");
  st.threads = threads;
  st.n_buckets = nb;
  st.grid = (int)grid;
  st.smem_words = smem;
  st.gwords = gwords;
  st.ut_len = ut_len;
  // workspace: [work counter: 256 B][global node buffers grid x gwords][smooth-until arrays]
  st.ut_off = (long long)gwords * grid;
  st.ws_bytes = 256 + ((size_t)gwords * grid + (size_t)until_arrays(p->mode) * ut_len * grid * threads) * 4;
  st.T_max = T_max;
  st.p = *p;
  st.ready = true;
  *workspace_bytes = st.ws_bytes;
  return STL_OK;
}

static stl_status ragged_common(stl_set_handle s, const float *sig, const int64_t *offsets, const int32_t *fid,
                                int64_t n_traces, const float *bounds, int32_t n_slots, const stl_params *p,
                                bool bwd, void *workspace, size_t workspace_bytes, SetState **out) {
  if (!s || !p) return fail(STL_ERR_INVALID_ARG, "NULL argument");
  SetState &st = s->st[bwd ? 1 : 0];
  if (!st.ready) return fail(STL_ERR_INVALID_ARG, "call stl_set_prepare for this direction first");
  if (std::memcmp(&st.p, p, sizeof *p) != 0) return fail(STL_ERR_INVALID_ARG, "params differ from stl_set_prepare");
  if (n_traces < 0) return fail(STL_ERR_INVALID_ARG, "n_traces must be >= 0");
  if (n_traces > 0 && (!sig || !offsets || !fid)) return fail(STL_ERR_INVALID_ARG, "signal / offsets / formula_id is NULL");
  if (n_slots != s->n_slots) return fail(STL_ERR_INVALID_ARG, "bounds must have %d slots", s->n_slots);
  if (s->n_slots > 0 && n_traces > 0 && !bounds) return fail(STL_ERR_INVALID_ARG, "bounds is NULL");
  if (!workspace || workspace_bytes < st.ws_bytes)
    return fail(STL_ERR_WORKSPACE, "workspace of %zu bytes needed", st.ws_bytes);
  *out = &st;
  return STL_OK;
}

static stl_status ragged_launch(stl_set_handle s, SetState &st, const float *sig, const int64_t *offsets,
                                const int32_t *fid, const int32_t *order, int64_t n_traces, const float *bounds,
                                const float *gout, float *out, float *gsig, float *gbounds, void *workspace,
                                void *stream) {
  if (n_traces == 0) return STL_OK;
  cudaError_t ce = cudaMemsetAsync(workspace, 0, 256, (cudaStream_t)stream);
  if (ce != cudaSuccess) return cuda_fail((int)ce, "cudaMemsetAsync(work counter)");
  LaunchArgs A{};
  int e0 = stl_status_ptr(&A.status);
  if (e0) return cuda_fail(e0, "cudaGetSymbolAddress(status)");
  A.sig = sig;
  A.bounds = s->n_slots ? bounds : nullptr;
  A.gout = gout;
  A.out = out;
  A.gsig = gsig;
  A.gbounds = s->n_slots ? gbounds : nullptr;
  A.ws = (float *)((char *)workspace + 256);
  A.table = st.dtable;
  A.offsets = (const long long *)offsets;
  A.fid = fid;
  A.order = order;
  A.counter = (unsigned long long *)workspace;
  A.n_traces = n_traces;
  A.n_formulas = (int)s->formulas.size();
  A.T_max = st.T_max;
  A.n_buckets = st.n_buckets;
  A.gwords = st.gwords;
  A.ut_len = st.ut_len;
  A.ut_off = st.ut_off;
  A.grid = (int)std::min<long long>(st.grid, n_traces);
  A.threads = st.threads;
  A.stream = stream;
  KProgram dummy;
  std::memset(&dummy, 0, sizeof dummy);
  dummy.smem_words = st.smem_words;
  dummy.bwd = gsig ? 1 : 0;
  dummy.mode = st.p.mode;
  int e = stl_launch_main(dummy, A);
  if (e) return cuda_fail(e, "ragged kernel launch");
  return STL_OK;
}

stl_status stl_robustness_ragged(stl_set_handle s, const float *sig, const int64_t *offsets, const int32_t *formula_id,
                                 const int32_t *order, int64_t n_traces, const float *bounds, int32_t n_slots,
                                 const stl_params *p, float *out, void *workspace, size_t workspace_bytes,
                                 void *stream) {
  SetState *st = nullptr;
  stl_status r = ragged_common(s, sig, offsets, formula_id, n_traces, bounds, n_slots, p, false, workspace,
                               workspace_bytes, &st);
  if (r) return r;
  if (n_traces > 0 && !out) return fail(STL_ERR_INVALID_ARG, "out is NULL");
  return ragged_launch(s, *st, sig, offsets, formula_id, order, n_traces, bounds, nullptr, out, nullptr, nullptr,
                       workspace, stream);
}

stl_status stl_robustness_ragged_backward(stl_set_handle s, const float *sig, const int64_t *offsets,
                                          const int32_t *formula_id, const int32_t *order, int64_t n_traces,
                                          const float *bounds, int32_t n_slots, const stl_params *p,
                                          const float *grad_out, float *grad_sig, float *grad_bounds,
                                          void *workspace, size_t workspace_bytes, void *stream) {
  SetState *st = nullptr;
  stl_status r = ragged_common(s, sig, offsets, formula_id, n_traces, bounds, n_slots, p, true, workspace,
                               workspace_bytes, &st);
  if (r) return r;
  if (n_traces > 0 && (!grad_out || !grad_sig)) return fail(STL_ERR_INVALID_ARG, "grad_out / grad_sig is NULL");
  if (grad_bounds && s->n_slots > 0 && n_traces > 0) {
    cudaError_t ce = cudaMemsetAsync(grad_bounds, 0, (size_t)n_traces * s->n_slots * 2 * sizeof(float),
                                     (cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "cudaMemsetAsync(grad_bounds)");
  }
  return ragged_launch(s, *st, sig, offsets, formula_id, order, n_traces, bounds, grad_out, nullptr, grad_sig,
                       grad_bounds, workspace, stream);
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
namespace {

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ULL) {
  const unsigned char *b = (const unsigned char *)data;
  for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ULL; }
  return h;
}

int log2_bucket(long long v) {
  int k = 0;
  while (v > 1) { v >>= 1; ++k; }
  return k;
}

std::string tune_key(const stl_program *h, long long B, long long T, const stl_params &p, bool bwd) {
  uint64_t x = fnv1a(h->nodes.data(), h->nodes.size() * sizeof(stl_node));
  x = fnv1a(h->w.data(), h->w.size() * sizeof(float), x);
  char buf[128];
  snprintf(buf, sizeof buf, "%016llx-D%d-S%d-m%d-%s-B%d-T%d", (unsigned long long)x, h->D, h->n_slots, p.mode,
           bwd ? "bwd" : "fwd", log2_bucket(B), log2_bucket(T));
  return buf;
}

bool cache_lookup(const char *path, const std::string &key, stl_launch *out) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    stl_launch l{};
    double ms;
    // line: key tile threads segment ms [kernel]
    if (is >> k >> l.tile >> l.threads >> l.segment >> ms && k == key) {
      int kind = 0;
      if (is >> kind) l.kernel = kind;
      *out = l;
      found = true;
    }
  }
  return found;
}

void cache_store(const char *path, const std::string &key, const stl_launch &l, double ms) {
  std::ofstream f(path, std::ios::app);
  if (f) f << key << " " << l.tile << " " << l.threads << " " << l.segment << " " << ms << " " << l.kernel << "\n";
}

}  // namespace

extern "C" {

stl_status stl_autotune(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds, const stl_params *p,
                        int32_t backward, const float *grad_out, float *out, float *grad_bounds, void *workspace,
                        size_t workspace_bytes, void *stream, stl_launch *best, float *best_ms) {
  stl_status s = check_call(h, sig, B, T, bounds, p);
  if (s) return s;
  if (!best) return fail(STL_ERR_INVALID_ARG, "best is NULL");
  if (B == 0) return fail(STL_ERR_INVALID_ARG, "nothing to tune for B = 0");
  const bool bwd = backward != 0;
  if (!out || (bwd && !grad_out)) return fail(STL_ERR_INVALID_ARG, "output buffers are NULL");
  const char *cache = std::getenv("STL_TUNE_CACHE");
  const std::string key = tune_key(h, B, T, *p, bwd);
  stl_launch hit{};
  if (cache && *cache && cache_lookup(cache, key, &hit)) {
    h->launch_dir[bwd ? 1 : 0] = hit;
    *best = hit;
    if (best_ms) *best_ms = -1.f;
    return STL_OK;
  }
  const stl_launch saved = h->launch_dir[bwd ? 1 : 0];
  std::vector<stl_launch> cands;
  for (int nt : {64, 256, 512})
    for (int mult : {4, 7, 14}) {
      if (nt == 64 && T > 8192) continue;   // 64-thread CTAs are for short traces
      stl_launch l{};
      l.threads = nt;
      l.tile = std::max(256, (nt * mult / 32) * 32);
      l.kernel = STL_KERNEL_INTERPRETER;
      cands.push_back(l);
    }
  // formula-compiled kernels (CTA size x tile), where they apply
  {
    std::string why;
    if (stl_fk_eligible(fk_formula(h), *p, T, &why) && stl_fk_available(&why))
      for (int nt : {512, 256})
        for (int mult : bwd ? std::vector<int>{11, 9, 7} : std::vector<int>{15, 11, 7}) {
          stl_launch l{};
          l.threads = nt;
          l.tile = nt * mult;
          l.kernel = STL_KERNEL_COMPILED;
          cands.push_back(l);
        }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(STL_ERR_CUDA, "cudaEventCreate failed");
  float best_t = 1e30f;
  stl_launch best_l = saved;
  bool any = false;
  for (const stl_launch &c : cands) {
    h->launch_dir[bwd ? 1 : 0] = c;
    size_t need = 0;
    if (stl_workspace_size(h, B, T, p, backward, &need) != STL_OK || need > workspace_bytes) continue;
    auto run = [&]() {
      return bwd ? stl_robustness_backward(h, sig, B, T, bounds, p, grad_out, out, grad_bounds, workspace,
                                           workspace_bytes, stream)
                 : stl_robustness(h, sig, B, T, bounds, p, out, workspace, workspace_bytes, stream);
    };
    if (run() != STL_OK) continue;
    cudaEventRecord(e0, (cudaStream_t)stream);
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = run() == STL_OK;
    cudaEventRecord(e1, (cudaStream_t)stream);
    if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.f;
    any = true;
    if (ms < best_t) { best_t = ms; best_l = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!any) {
    h->launch_dir[bwd ? 1 : 0] = saved;
    return fail(STL_ERR_WORKSPACE, "no candidate launch shape fits the given workspace");
  }
  h->launch_dir[bwd ? 1 : 0] = best_l;
  *best = best_l;
  if (best_ms) *best_ms = best_t;
  if (cache && *cache) cache_store(cache, key, best_l, best_t);
  return STL_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ ragged-set autotuner
namespace {
std::string set_tune_key(const stl_program_set *s, long long n, long long T_max, const stl_params &p, bool bwd) {
  uint64_t x = 1469598103934665603ULL;
  for (const stl_program *h : s->formulas) {
    x = fnv1a(h->nodes.data(), h->nodes.size() * sizeof(stl_node), x);
    x = fnv1a(h->w.data(), h->w.size() * sizeof(float), x);
  }
  char buf[160];
  snprintf(buf, sizeof buf, "set%016llx-F%zu-D%d-S%d-m%d-%s-N%d-T%d", (unsigned long long)x, s->formulas.size(), s->D,
           s->n_slots, p.mode, bwd ? "bwd" : "fwd", log2_bucket(n), log2_bucket(T_max));
  return buf;
}
}  // namespace

extern "C" {

stl_status stl_set_set_launch(stl_set_handle s, int32_t backward, const stl_launch *launch) {
  if (!s || !launch) return fail(STL_ERR_INVALID_ARG, "NULL argument");
  if (launch->threads != 0 && launch->threads != 64 && launch->threads != 256 && launch->threads != 512)
    return fail(STL_ERR_INVALID_ARG, "threads must be 0, 64, 256 or 512");
  if (launch->tile < 0 || launch->tile % 32 != 0) return fail(STL_ERR_INVALID_ARG, "tile must be a multiple of 32");
  s->st[backward ? 1 : 0].shape = *launch;
  return STL_OK;
}

stl_status stl_set_autotune(stl_set_handle s, int64_t n_traces, int64_t T_max, const stl_params *p, int32_t backward,
                            const float *sig, const int64_t *offsets, const int32_t *formula_id, const int32_t *order,
                            const float *bounds, int32_t n_slots, const float *grad_out, float *out,
                            float *grad_bounds, void *stream, stl_launch *best, float *best_ms,
                            size_t *workspace_bytes) {
  if (!s || !p || !best || !workspace_bytes) return fail(STL_ERR_INVALID_ARG, "NULL argument");
  if (n_traces < 1) return fail(STL_ERR_INVALID_ARG, "nothing to tune for n_traces < 1");
  const bool bwd = backward != 0;
  if (!sig || !offsets || !formula_id || !out || (bwd && !grad_out))
    return fail(STL_ERR_INVALID_ARG, "input / output buffers are NULL");
  SetState &st = s->st[bwd ? 1 : 0];
  const char *cache = std::getenv("STL_TUNE_CACHE");
  const std::string key = set_tune_key(s, n_traces, T_max, *p, bwd);
  stl_launch hit{};
  if (cache && *cache && cache_lookup(cache, key, &hit)) {
    st.shape = hit;
    *best = hit;
    if (best_ms) *best_ms = -1.f;
    return stl_set_prepare(s, n_traces, T_max, p, backward, workspace_bytes);
  }
  const stl_launch saved = st.shape;
  std::vector<stl_launch> cands;
  for (int nt : {64, 256, 512})
    for (int mult : {4, 7, 14}) {
      if (nt == 64 && T_max > 8192) continue;   // 64-thread CTAs are for short traces
      stl_launch l{};
      l.threads = nt;
      l.tile = std::max(256, (nt * mult / 32) * 32);
      l.kernel = STL_KERNEL_INTERPRETER;
      cands.push_back(l);
    }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(STL_ERR_CUDA, "cudaEventCreate failed");
  float best_t = 1e30f;
  stl_launch best_l = saved;
  bool any = false;
  for (const stl_launch &c : cands) {
    st.shape = c;
    size_t need = 0;
    if (stl_set_prepare(s, n_traces, T_max, p, backward, &need) != STL_OK) continue;
    void *ws = nullptr;
    if (cudaMalloc(&ws, need) != cudaSuccess) { cudaGetLastError(); continue; }
    auto run = [&]() {
      return bwd ? stl_robustness_ragged_backward(s, sig, offsets, formula_id, order, n_traces, bounds, n_slots, p,
                                                  grad_out, out, grad_bounds, ws, need, stream)
                 : stl_robustness_ragged(s, sig, offsets, formula_id, order, n_traces, bounds, n_slots, p, out, ws,
                                         need, stream);
    };
    bool ok = run() == STL_OK;
    if (ok) {
      cudaEventRecord(e0, (cudaStream_t)stream);
      for (int r = 0; r < 2 && ok; ++r) ok = run() == STL_OK;
      cudaEventRecord(e1, (cudaStream_t)stream);
      ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
    }
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(ws);
    if (!ok) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 2.f;
    any = true;
    if (ms < best_t) { best_t = ms; best_l = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st.shape = any ? best_l : saved;
  stl_status r = stl_set_prepare(s, n_traces, T_max, p, backward, workspace_bytes);
  if (r) return r;
  if (!any) return fail(STL_ERR_UNSUPPORTED, "no candidate launch shape ran");
  *best = best_l;
  if (best_ms) *best_ms = best_t;
  if (cache && *cache) cache_store(cache, key, best_l, best_t);
  return STL_OK;
}

}  // extern "C"
