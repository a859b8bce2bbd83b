// stl_fk.cu -- formula-compiled kernels: code generation, run-time compilation (NVRTC) and
// launch for hard-semantics calls whose intervals are static.
//
// The interpreter (stl_interp.cuh) reads the compiled program at run time, so every window
// length, buffer offset and loop bound is a register value and every child read goes through
// an index clamp; measured on the nested Until/Always/Eventually formula, about 400
// instructions per sample and direction, nearly all integer bookkeeping.  Here the program becomes source code: one
// __global__ function per (formula, direction, CTA size, tile) whose node passes are
// instantiations of the templates in stl_fk_dev.cuh with compile-time constants, a walk of
// the selections unrolled over the tree, and literal predicate weights.  NVRTC compiles it for
// sm_103a on first use and the cubin is kept for the life of the process.
//
// Semantics and bit patterns are those of the interpreter: the same float32 predicate
// arithmetic (no contraction), the same window and Until combines and tie rules, and the same
// 64-bit fixed-point gradient deposits, so both paths give bit-identical robustness and
// gradients.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "stl_fk.h"

int stl_status_ptr(int **ptr);   // the library's sticky device status word (stl_kernels.cu)

namespace {

// Untils whose phi prefix [0, a] has at most this many samples take it from registers in the
// same pass as the clamp composition
constexpr int FK_UNTIL_FUSE_W = 16;

// the device building blocks, embedded at build time from stl_fk_dev.cuh
const char *const k_dev_src =
#include "stl_fk_src.inc"
    ;

std::string fmt(const char *f, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

// exact float literal (C++17 hexadecimal floating literal; finite values only)
std::string flit(float v) {
  if (!std::isfinite(v)) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    return fmt("__int_as_float(0x%08xu)", u);
  }
  return fmt("(%af)", (double)v);
}

int round_up(long long v, int m) { return (int)(((v + m - 1) / m) * m); }
bool is_temporal(int op) { return op == STL_OP_EVENTUALLY || op == STL_OP_ALWAYS || op == STL_OP_UNTIL; }
bool is_elem2(int op) { return op == STL_OP_AND || op == STL_OP_OR; }
bool is_pred(int op) { return op == STL_OP_PRED_GT || op == STL_OP_PRED_LT; }

// ------------------------------------------------------------------ NVRTC (loaded on demand)
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram *nvrtcProgram_t;
struct Nvrtc {
  bool ok = false;
  std::string why;
  nvrtcResult_t (*create)(nvrtcProgram_t *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
  nvrtcResult_t (*compile)(nvrtcProgram_t, int, const char *const *) = nullptr;
  nvrtcResult_t (*log_size)(nvrtcProgram_t, size_t *) = nullptr;
  nvrtcResult_t (*log)(nvrtcProgram_t, char *) = nullptr;
  nvrtcResult_t (*cubin_size)(nvrtcProgram_t, size_t *) = nullptr;
  nvrtcResult_t (*cubin)(nvrtcProgram_t, char *) = nullptr;
  nvrtcResult_t (*destroy)(nvrtcProgram_t *) = nullptr;
  const char *(*err)(nvrtcResult_t) = nullptr;
};

Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    void *h = nullptr;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char *nm : names)
      if (!h) h = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
    if (!h) {
      const char *home = std::getenv("CUDA_HOME");
      std::string p = std::string(home && *home ? home : "/usr/local/cuda") + "/lib64/libnvrtc.so";
      h = dlopen((p + ".13").c_str(), RTLD_NOW | RTLD_LOCAL);
      if (!h) h = dlopen(p.c_str(), RTLD_NOW | RTLD_LOCAL);
    }
    if (!h) { n.why = "libnvrtc could not be loaded"; return; }
    auto sym = [&](const char *s) { return dlsym(h, s); };
    n.create = (decltype(n.create))sym("nvrtcCreateProgram");
    n.compile = (decltype(n.compile))sym("nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))sym("nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))sym("nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))sym("nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))sym("nvrtcGetCUBIN");
    n.destroy = (decltype(n.destroy))sym("nvrtcDestroyProgram");
    n.err = (decltype(n.err))sym("nvrtcGetErrorString");
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy && n.err;
    if (!n.ok) n.why = "libnvrtc lacks a needed entry point";
  });
  return n;
}

// ------------------------------------------------------------------ plan
struct GNode {
  int op = 0, c0 = -1, c1 = -1, parent = -1;
  int a = 0, b = 0;
  bool padc = false;
  float padv = 0.f;
  int lo = 0, hi = 0;
  int k = -1;              // predicate index
  bool tanc = false;       // has a temporal ancestor
  bool tparent = false;    // parent is temporal (its buffer holds the parent's pads past T-1)
  bool walkpad = false;    // backward walks may reach it at a pad position (>= T)
  bool has_val = false, has_aux = false;
  int cap = 0;             // buffer length in samples (slack included)
  int off_v = -1, off_a = -1;
  int R = 3, R1 = 3;       // run lengths: window / Until pass 2, Until pass 1
  int level = 0;           // 0 for leaves, 1 + the largest level of the children
  int off_s = -1;          // this node's window scratch (run aggregates)
};

struct GPlan {
  bool bwd = false;
  int D = 0, NT = 512, TILE = 0, SLACK = 16;
  int n = 0, root = 0, npred = 0;
  int LP = 0, HP = 0, HMAX = 0, LOMAX = 0;
  int capA = 0;            // predicate adjoint ring length (samples)
  int off_j = -1;          // adjoint rings (u64), predicate k at off_j + 8 * k * capA
  bool gring = false;      // backward: adjoint rings in the workspace (L2) instead of shared memory
  bool check = false;      // bounds-checked build (STL_FK_CHECK=1)
  int RING = 0;            // their length: a power of two >= TILE + HP - LP, indexed by (j - LP) mod RING
  int off_cells = 0, off_scr = 0, smem = 0;
  std::vector<GNode> g;
  std::vector<int> preds;  // node index of predicate k
  std::vector<float> pw;   // signal-gradient weights [k][d]: +w (>) or -w (<)
};

int odd_floor(int v) { return (v % 2) ? v : v - 1; }

// run length of a window of K samples: R consecutive outputs per thread, odd (conflict-free
// strided shared-memory access), at most rcap, K >= 2R (else the direct loop runs)
int pick_r(int K, int rcap) {
  if (K < 6) return 3;
  return std::max(3, std::min(rcap, odd_floor(K / 2)));
}

int elem_bytes(int op, bool bwd, bool until_pass2) {
  if (op == STL_OP_UNTIL && until_pass2) return bwd ? 16 : 8;
  return bwd ? 8 : 4;
}

// geometry for one tile; returns false if the formula is outside the compiled path
bool build_plan(const FkFormula &f, bool bwd, int NT, int TILE, GPlan &P, std::string *why, bool gring = false) {
  const std::vector<stl_node> &nd = *f.nodes;
  const int n = (int)nd.size();
  P = GPlan{};
  P.bwd = bwd;
  {
    const char *e = std::getenv("STL_FK_CHECK");
    P.check = e && *e && std::strcmp(e, "0") != 0;
  }
  P.D = f.D;
  P.NT = NT;
  P.TILE = TILE;
  P.n = n;
  P.root = n - 1;
  P.g.assign(n, GNode{});
  for (int i = 0; i < n; ++i) {
    GNode &x = P.g[i];
    x.op = nd[i].op;
    x.c0 = nd[i].child0;
    x.c1 = nd[i].child1;
    if (is_temporal(x.op)) {
      x.a = (int)nd[i].a;
      x.b = (int)nd[i].b;
      x.padc = nd[i].pad_mode == STL_PAD_CONST;
      x.padv = nd[i].pad_value;
    }
  }
  for (int i = 0; i < n; ++i) {
    if (P.g[i].c0 >= 0) P.g[P.g[i].c0].parent = i;
    if (P.g[i].c1 >= 0) P.g[P.g[i].c1].parent = i;
  }
  // live offsets: values run ahead by hi (sum of b along the path), the nearest sample a
  // node's parent reads is lo (sum of a; the Until's phi prefix starts at 0)
  for (int i = n - 1; i >= 0; --i) {
    GNode &x = P.g[i];
    const bool tmp = is_temporal(x.op);
    for (int s = 0; s < 2; ++s) {
      const int c = s == 0 ? x.c0 : x.c1;
      if (c < 0) continue;
      GNode &y = P.g[c];
      if (tmp) {
        y.lo = x.lo + ((x.op == STL_OP_UNTIL && s == 0) ? 0 : x.a);
        y.hi = x.hi + x.b;
      } else {
        y.lo = x.lo;
        y.hi = x.hi;
      }
      y.tanc = x.tanc || tmp;
      y.tparent = tmp;
      y.walkpad = x.walkpad || (tmp && !x.padc);
    }
  }
  P.LP = 1 << 30;
  P.HP = 0;
  for (int i = 0; i < n; ++i)
    if (is_pred(P.g[i].op)) {
      P.g[i].k = P.npred++;
      P.preds.push_back(i);
      P.LP = std::min(P.LP, P.g[i].lo);
      P.HP = std::max(P.HP, P.g[i].hi);
    }
  if (P.npred == 0) P.LP = 0;
  for (int i = 0; i < n; ++i)
    if (is_pred(P.g[i].op)) { P.g[i].lo = P.LP; P.g[i].hi = P.HP; }
  for (int i = 0; i < n; ++i) {
    P.HMAX = std::max(P.HMAX, P.g[i].hi);
    P.LOMAX = std::max(P.LOMAX, P.g[i].lo);
  }
  // selected offsets are stored in 16 bits (2 * offset + child for the Until)
  for (int i = 0; i < n; ++i)
    if (is_temporal(P.g[i].op) && P.g[i].b > 16000) {
      if (why) *why = "an interval end beyond 16000 samples";
      return false;
    }
  // run lengths
  const int rcap = std::max(3, std::min(15, odd_floor((TILE + NT - 1) / NT + 1)));
  int maxR = 3;
  for (int i = 0; i < n; ++i) {
    GNode &x = P.g[i];
    if (x.op == STL_OP_EVENTUALLY || x.op == STL_OP_ALWAYS) x.R = pick_r(x.b - x.a + 1, rcap);
    if (x.op == STL_OP_UNTIL) {
      x.R1 = pick_r(x.a + 1, rcap);
      x.R = pick_r(x.b - x.a + 1, rcap);
    }
    maxR = std::max(maxR, std::max(x.R, x.R1));
  }
  P.SLACK = round_up(maxR + 2, 4);
  // buffers
  int off = 0;
  auto take = [&](long long bytes) {
    const int o = off;
    off += round_up(bytes, 16);
    return o;
  };
  for (int i = 0; i < n; ++i) {
    GNode &x = P.g[i];
    const bool elem_root = i == P.root && (x.op == STL_OP_NOT || is_elem2(x.op) || x.op == STL_OP_TRUE);
    x.has_val = !elem_root;
    x.has_aux = bwd && (is_temporal(x.op) || (is_elem2(x.op) && x.tanc));
    x.cap = round_up((long long)TILE + x.hi - x.lo, 4) + P.SLACK;
    if (x.has_val) x.off_v = take(4LL * x.cap);
    if (x.has_aux) x.off_a = take(2LL * x.cap);
  }
  if (bwd && P.npred > 0 && gring) {
    P.gring = true;
    P.RING = 1;
    while (P.RING < TILE + P.HP - P.LP) P.RING <<= 1;
  } else if (bwd && P.npred > 0) {
    P.capA = round_up((long long)TILE + P.HP - P.LP, 4);
    P.off_j = take(8LL * P.capA * P.npred);
  }
  // cells: value and aux at T-1 per node, adjoint of sample T-1 per predicate
  P.off_cells = take(4LL * n + 4LL * n + 8LL * std::max(1, P.npred));
  // every window node has scratch of its own (run aggregates, then level-2 blocks: sliding for
  // max / min, aligned for the clamps), so that nodes of one level run without a barrier
  // between them
  for (int i = 0; i < n; ++i) {
    GNode &x = P.g[i];
    int scr = 0;
    auto need = [&](int K, int R, int eb, bool idem) {
      if (K < 2 * R) return;
      const int NF = K / R - 1;
      const bool two = NF >= 24;
      const int ent = NT + NF + 8 + (two ? (idem ? NT + NF : (NT + NF) / 8 + 8) : 0);
      scr = std::max(scr, ent * eb);
    };
    if (x.op == STL_OP_EVENTUALLY || x.op == STL_OP_ALWAYS) need(x.b - x.a + 1, x.R, elem_bytes(x.op, bwd, false), true);
    if (x.op == STL_OP_UNTIL) {
      if (x.a + 1 > FK_UNTIL_FUSE_W) need(x.a + 1, x.R1, elem_bytes(x.op, bwd, false), true);
      need(x.b - x.a + 1, x.R, elem_bytes(x.op, bwd, true), false);
    }
    if (scr > 0) x.off_s = take(scr);
  }
  P.off_scr = take(64);
  for (int i = 0; i < n; ++i) {
    GNode &x = P.g[i];
    const int l0 = x.c0 >= 0 ? P.g[x.c0].level : -1, l1 = x.c1 >= 0 ? P.g[x.c1].level : -1;
    x.level = (x.c0 < 0 && x.c1 < 0) ? 0 : 1 + std::max(l0, l1);
  }
  P.smem = off;
  P.pw.assign((size_t)P.npred * P.D, 0.f);
  for (int k = 0; k < P.npred; ++k) {
    const stl_node &q = nd[P.preds[k]];
    for (int d = 0; d < P.D; ++d) {
      const float w = (*f.w)[q.pred_offset + d];
      P.pw[(size_t)k * P.D + d] = q.op == STL_OP_PRED_GT ? w : -w;
    }
  }
  return true;
}

// ------------------------------------------------------------------ code generation
struct Gen {
  const GPlan &P;
  const FkFormula &f;
  std::string s;
  explicit Gen(const GPlan &p, const FkFormula &ff) : P(p), f(ff) {}
  void l(const std::string &x) { s += x; s += '\n'; }

  std::string base(int i) const { return fmt("(t0 + %d)", P.g[i].lo); }
  // new samples of node i in this step: [F, E)
  void range(int i) {
    const GNode &x = P.g[i];
    l(fmt("    const int base = t0 + %d;", x.lo));
    l(fmt("    const int F = min(first ? base : t0 + %d, T), E = min(t1 + %d, T);", x.hi, x.hi));
  }

  void pred_pass() {
    if (P.npred == 0) return;
    const int D = P.D;
    l("  {  // predicates (Sec. III-B): float32, left-to-right sums, no contraction");
    l(fmt("    const int base = t0 + %d;", P.LP));
    l(fmt("    const int F = min(first ? base : t0 + %d, T), E = min(t1 + %d, T);", P.HP, P.HP));
    // PB samples per thread per iteration: their loads are in flight together
    const int PB = D <= 4 ? 8 : 4;
    l(fmt("    for (int j0 = F + tid; j0 < E; j0 += NT * %d) {", PB));
    l(fmt("      float x[%d][%d];", PB, D));
    l("#pragma unroll");
    l(fmt("      for (int u = 0; u < %d; ++u) {", PB));
    l("        const int j = j0 + u * NT;");
    l("#pragma unroll");
    l(fmt("        for (int d = 0; d < %d; ++d) x[u][d] = j < E ? __ldg(xs + (long long)j * %d + d) : 0.f;", D, D));
    l("      }");
    l("#pragma unroll");
    l(fmt("      for (int u = 0; u < %d; ++u) {", PB));
    l("        const int j = j0 + u * NT;");
    l("        if (j >= E) continue;");
    l("        float s;");
    for (int k = 0; k < P.npred; ++k) {
      const int i = P.preds[k];
      const stl_node &q = (*f.nodes)[i];
      for (int d = 0; d < D; ++d) {
        const std::string w = flit((*f.w)[q.pred_offset + d]);
        if (d == 0) l(fmt("        s = __fmul_rn(%s, x[u][0]);", w.c_str()));
        else l(fmt("        s = __fadd_rn(s, __fmul_rn(%s, x[u][%d]));", w.c_str(), d));
      }
      const std::string c = flit(q.pred_c);
      if (q.op == STL_OP_PRED_GT) l(fmt("        fv%d[j - base] = __fsub_rn(s, %s);", i, c.c_str()));
      else l(fmt("        fv%d[j - base] = __fsub_rn(%s, s);", i, c.c_str()));
    }
    l("      }");
    l("    }");
    l("  }");
    l("  __syncthreads();");
    // pads of predicates read by temporal parents
    bool any = false;
    for (int i : P.preds) any = any || P.g[i].tparent;
    if (any) {
      l(fmt("  if (t1 + %d >= T) {", P.HP));
      l(fmt("    const int base = t0 + %d;", P.LP));
      l("    const bool inb = T - 1 >= base;");
      for (int i : P.preds)
        if (P.g[i].tparent) pad_fill_body(i);
      l("    __syncthreads();");
      l("  }");
    }
  }

  // pad values of node i's buffer past T-1 (its parent's pad: the value at T-1 or a constant)
  void pad_fill_body(int i) {
    const GNode &x = P.g[i];
    const GNode &par = P.g[x.parent];
    if (par.padc) {
      l(fmt("    fk_fill<NT>(FK_PTR(fv%d), max(T - base, 0), %d, %s);", i, x.cap, flit(par.padv).c_str()));
    } else {
      l("    {");
      l(fmt("      const float pv = inb ? fv%d[T - 1 - base] : fk_vcell[%d];", i, i));
      l(fmt("      if (inb && tid == 0) fk_vcell[%d] = pv;", i));
      l(fmt("      fk_fill<NT>(FK_PTR(fv%d), max(T - base, 0), %d, pv);", i, x.cap));
      l("    }");
    }
  }

  // node i's pass; `barrier`: synchronise after it (the next pass reads it); without, the
  // next pass belongs to the same level and reads neither this node nor its scratch
  void node_pass(int i, bool barrier) {
    const GNode &x = P.g[i];
    const bool bwd = P.bwd;
    if (is_pred(x.op)) return;
    if (i == P.root && !x.has_val) return;   // elementwise root: written by the output / walk
    l(fmt("  {  // node %d (level %d)", i, x.level));
    if (x.off_s >= 0) l(fmt("    void *const fk_scr = fk_sm + %d;", x.off_s));
    range(i);
    auto cb = [&](int c) { return fmt("t0 + %d", P.g[c].lo); };
    switch (x.op) {
      case STL_OP_TRUE:
        l(fmt("    for (int q = F + tid; q < E; q += NT) fv%d[q - base] = fk_inf();", i));
        break;
      case STL_OP_NOT:
        l(fmt("    const int b0 = %s;", cb(x.c0).c_str()));
        l(fmt("    for (int q = F + tid; q < E; q += NT) fv%d[q - base] = -fv%d[q - b0];", i, x.c0));
        break;
      case STL_OP_AND:
      case STL_OP_OR: {
        const char *cmp = x.op == STL_OP_AND ? "<=" : ">=";
        l(fmt("    const int b0 = %s, b1 = %s;", cb(x.c0).c_str(), cb(x.c1).c_str()));
        l("    for (int q = F + tid; q < E; q += NT) {");
        l(fmt("      const float a = fv%d[q - b0], c = fv%d[q - b1];", x.c0, x.c1));
        l(fmt("      const bool left = a %s c;", cmp));
        l(fmt("      fv%d[q - base] = left ? a : c;", i));
        if (x.has_aux) l(fmt("      fa%d[q - base] = left ? 0 : 1;", i));
        l("    }");
        break;
      }
      case STL_OP_EVENTUALLY:
      case STL_OP_ALWAYS: {
        const bool mx = x.op == STL_OP_EVENTUALLY;
        l(fmt("    const int cb = %s;", cb(x.c0).c_str()));
        l(fmt("    const auto o = fv%d;", i));
        l(fmt("    const auto xc = fv%d;", x.c0));
        if (!bwd) {
          l(fmt("    fk_window<%s, NT, %d, %d, %d>(F, E, [&](int j) { return xc[j - cb]; },", mx ? "FkMax" : "FkMin", x.R,
                x.a, x.b));
          l("        [&](int q, float v) { o[q - base] = v; }, fk_scr);");
        } else {
          l(fmt("    const auto oa = fa%d;", i));
          l(fmt("    fk_window<%s, NT, %d, %d, %d>(F, E, [&](int j) { FkVP r; r.v = xc[j - cb]; r.p = j; return r; },",
                mx ? "FkMaxP" : "FkMinP", x.R, x.a, x.b));
          l("        [&](int q, FkVP r) { o[q - base] = r.v; oa[q - base] = (fk_u16)(r.p - q); }, fk_scr);");
        }
        break;
      }
      case STL_OP_UNTIL: {
        l(fmt("    const int cp = %s, cq = %s;", cb(x.c0).c_str(), cb(x.c1).c_str()));
        l(fmt("    const auto o = fv%d;", i));
        l(fmt("    const auto xp = fv%d;", x.c0));
        l(fmt("    const auto xq = fv%d;", x.c1));
        if (x.a + 1 <= FK_UNTIL_FUSE_W) {
          // one pass: the phi prefix minimum over [q, q+a] comes from the thread's registers
          if (!bwd) {
            l(fmt("    fk_until<FkClamp, FkMin, NT, %d, %d, %d>(F, E, [&](int j) {", x.R, x.a, x.b));
            l("          const float p = xp[j - cp], s = xq[j - cq]; FkC2 r; r.c = fminf(p, s); r.d = p; return r; },");
            l("        [&](int j) { return xp[j - cp]; },");
            l("        [&](int q, FkC2 r, float a) { o[q - base] = (a <= r.c) ? a : r.c; }, fk_scr);");
          } else {
            l(fmt("    const auto oa = fa%d;", i));
            l(fmt("    fk_until<FkClampP, FkMinP, NT, %d, %d, %d>(F, E, [&](int j) {", x.R, x.a, x.b));
            l("          const float p = xp[j - cp], s = xq[j - cq]; const bool pl = p <= s; FkCC r;");
            l("          r.c = pl ? p : s; r.cs = pl ? 2 * j : 2 * j + 1; r.d = p; r.ds = 2 * j; return r; },");
            l("        [&](int j) { FkVP r; r.v = xp[j - cp]; r.p = j; return r; },");
            l("        [&](int q, FkCC r, FkVP a) {");
            l("          if (a.v <= r.c) { o[q - base] = a.v; oa[q - base] = (fk_u16)(2 * (a.p - q)); }");
            l("          else { o[q - base] = r.c; oa[q - base] = (fk_u16)(r.cs - 2 * q); } }, fk_scr);");
          }
          break;
        }
        if (!bwd) {
          l(fmt("    fk_window<FkMin, NT, %d, 0, %d>(F, E, [&](int j) { return xp[j - cp]; },", x.R1, x.a));
          l("        [&](int q, float v) { o[q - base] = v; }, fk_scr);");
          l("    __syncthreads();");
          l(fmt("    fk_window<FkClamp, NT, %d, %d, %d>(F, E, [&](int j) {", x.R, x.a, x.b));
          l("          const float p = xp[j - cp], s = xq[j - cq]; FkC2 r; r.c = fminf(p, s); r.d = p; return r; },");
          l("        [&](int q, FkC2 r) { const float a = o[q - base]; if (!(a <= r.c)) o[q - base] = r.c; }, fk_scr);");
        } else {
          l(fmt("    const auto oa = fa%d;", i));
          l(fmt("    fk_window<FkMinP, NT, %d, 0, %d>(F, E, [&](int j) { FkVP r; r.v = xp[j - cp]; r.p = j; return r; },",
                x.R1, x.a));
          l("        [&](int q, FkVP r) { o[q - base] = r.v; oa[q - base] = (fk_u16)(2 * (r.p - q)); }, fk_scr);");
          l("    __syncthreads();");
          l(fmt("    fk_window<FkClampP, NT, %d, %d, %d>(F, E, [&](int j) {", x.R, x.a, x.b));
          l("          const float p = xp[j - cp], s = xq[j - cq]; const bool pl = p <= s; FkCC r;");
          l("          r.c = pl ? p : s; r.cs = pl ? 2 * j : 2 * j + 1; r.d = p; r.ds = 2 * j; return r; },");
          l("        [&](int q, FkCC r) { const float a = o[q - base];");
          l("          if (!(a <= r.c)) { o[q - base] = r.c; oa[q - base] = (fk_u16)(r.cs - 2 * q); } }, fk_scr);");
        }
        break;
      }
      default:
        break;
    }
    l("  }");
    if (barrier) l("  __syncthreads();");
    if (x.tparent) {
      l(fmt("  if (t1 + %d >= T) {", x.hi));
      if (!barrier) l("    __syncthreads();");
      l(fmt("    const int base = t0 + %d;", x.lo));
      l("    const bool inb = T - 1 >= base;");
      pad_fill_body(i);
      l("    __syncthreads();");
      l("  }");
    }
  }

  // the root's value at sample q (q in [t0, t1))
  std::string root_value() const {
    const GNode &x = P.g[P.root];
    if (x.has_val) return fmt("fv%d[q - t0]", P.root);
    auto v = [&](int c) { return fmt("fv%d[q - (t0 + %d)]", c, P.g[c].lo); };
    if (x.op == STL_OP_TRUE) return "fk_inf()";
    if (x.op == STL_OP_NOT) return "(-" + v(x.c0) + ")";
    const char *cmp = x.op == STL_OP_AND ? "<=" : ">=";
    return fmt("([&]() { const float a = %s, c = %s; return a %s c ? a : c; }())", v(x.c0).c_str(), v(x.c1).c_str(),
               cmp);
  }

  // buffer moves at the end of a step: the live part of every buffer goes to its front
  void shift() {
    struct Mv { std::string p; int src, len; };
    std::vector<Mv> mv;
    for (int i = 0; i < P.n; ++i) {
      const GNode &x = P.g[i];
      const int span = x.hi - x.lo;
      if (span <= 0) continue;
      if (x.has_val) mv.push_back({fmt("FK_PTR(fv%d)", i), P.TILE, span});
      if (x.has_aux) mv.push_back({fmt("reinterpret_cast<float *>(FK_PTR(fa%d))", i), P.TILE / 2, (span + 1) / 2});
    }
    if (P.bwd && !P.gring && P.npred > 0 && P.HP - P.LP > 0)
      for (int k = 0; k < P.npred; ++k)
        mv.push_back({fmt("reinterpret_cast<float *>(FK_PTR(fj) + %d)", k * P.capA), 2 * P.TILE, 2 * (P.HP - P.LP)});
    int rounds = 0;
    for (auto &m : mv) rounds = std::max(rounds, (m.len + m.src - 1) / m.src);
    for (int r = 0; r < rounds; ++r) {
      for (auto &m : mv) {
        const int c0 = r * m.src;
        if (c0 >= m.len) continue;
        // round up so that the 16-byte copies stay aligned (the extra words are dead)
        const int len = round_up(m.len, 4);
        l(fmt("    fk_move_round<NT, %d, %d, %d>(%s);", m.src, c0, len, m.p.c_str()));
      }
      l("    __syncthreads();");
    }
    if (P.bwd && !P.gring && P.npred > 0) {
      // new samples of the predicate adjoint rings start at zero
      const int keep = 2 * (P.HP - P.LP);
      for (int k = 0; k < P.npred; ++k)
        l(fmt("    fk_zero<NT>(reinterpret_cast<float *>(FK_PTR(fj) + %d), %d, %d);", k * P.capA, keep, 2 * P.capA));
      l("    __syncthreads();");
    }
  }

  // selection walk from the root: sets leaf (predicate index or -1), pos and g
  void walk(int i, int ind) {
    const GNode &x = P.g[i];
    const std::string sp(ind, ' ');
    auto bs = [&](int c) { return fmt("(t0 + %d)", P.g[c].lo); };
    switch (x.op) {
      case STL_OP_PRED_GT:
      case STL_OP_PRED_LT:
        s += sp + fmt("leaf = %d;\n", x.k);
        return;
      case STL_OP_TRUE:
        return;
      case STL_OP_NOT:
        s += sp + "g = -g;\n";
        walk(x.c0, ind);
        return;
      case STL_OP_AND:
      case STL_OP_OR:
        if (x.has_aux) {
          s += sp + fmt("if (fa%d[pos - %s] == 0) {\n", i, bs(i).c_str());
        } else {
          const char *cmp = x.op == STL_OP_AND ? "<=" : ">=";
          s += sp + fmt("if (fv%d[pos - %s] %s fv%d[pos - %s]) {\n", x.c0, bs(x.c0).c_str(), cmp, x.c1, bs(x.c1).c_str());
        }
        walk(x.c0, ind + 2);
        s += sp + "} else {\n";
        walk(x.c1, ind + 2);
        s += sp + "}\n";
        return;
      case STL_OP_EVENTUALLY:
      case STL_OP_ALWAYS:
      case STL_OP_UNTIL: {
        const bool until = x.op == STL_OP_UNTIL;
        s += sp + "{\n";
        s += sp + fmt("  const int cd = fa%d[pos - %s];\n", i, bs(i).c_str());
        const std::string off = until ? "(cd >> 1)" : "cd";
        // with a constant pad, a read past T-1 carries no gradient; a pad position >= T of this
        // node stands for its sample T-1
        if (x.padc) s += sp + fmt("  if (min(pos, T - 1) + %s < T) {\n", off.c_str());
        else s += sp + "  {\n";
        s += sp + fmt("    pos += %s;\n", off.c_str());
        if (until) {
          s += sp + "    if (cd & 1) {\n";
          walk(x.c1, ind + 6);
          s += sp + "    } else {\n";
          walk(x.c0, ind + 6);
          s += sp + "    }\n";
        } else {
          walk(x.c0, ind + 4);
        }
        s += sp + "  }\n";
        s += sp + "}\n";
        return;
      }
      default:
        return;
    }
  }

  void aux_pad_fills() {
    bool any = false;
    for (int i = 0; i < P.n; ++i) any = any || (P.g[i].walkpad && P.g[i].has_aux);
    if (!any) return;
    l(fmt("  if (t1 + %d >= T) {   // selections past T-1 stand for those of sample T-1", P.HMAX + P.SLACK));
    for (int i = 0; i < P.n; ++i) {
      const GNode &x = P.g[i];
      if (!(x.walkpad && x.has_aux)) continue;
      l(fmt("    if (t1 + %d >= T) {", x.hi));
      l(fmt("      const int base = t0 + %d;", x.lo));
      l("      const bool inb = T - 1 >= base;");
      l(fmt("      const fk_u16 av = inb ? fa%d[T - 1 - base] : (fk_u16)fk_acell[%d];", i, i));
      l(fmt("      if (inb && tid == 0) fk_acell[%d] = av;", i));
      l(fmt("      fk_fill16<NT>(FK_PTR(fa%d), max(T - base, 0), %d, av);", i, x.cap));
      l("    }");
    }
    l("    __syncthreads();");
    l("  }");
  }

  std::string source(const std::string &name) {
    const int D = P.D, NT = P.NT, TILE = P.TILE;
    s.clear();
    l(fmt("// generated: formula of %d nodes, %s, %d threads, tile %d", P.n, P.bwd ? "backward" : "forward", NT, TILE));
    l(fmt("#define FK_CHECK %d", P.check ? 1 : 0));
    l(k_dev_src);
    l(fmt("#define NT %d", NT));
    l(fmt("extern \"C\" __global__ void __launch_bounds__(%d, 1) %s(", NT, name.c_str()));
    l("    const float *__restrict__ sig, const float *__restrict__ gout, float *__restrict__ out,");
    l("    float *__restrict__ gsig, fk_u64 *__restrict__ ws, int *__restrict__ fk_status, int T, int seg, int segs,");
    l("    long long n_items) {");
    l("  extern __shared__ float4 fk_sm4[];");
    l("  char *const fk_sm = reinterpret_cast<char *>(fk_sm4);");
    for (int i = 0; i < P.n; ++i) {
      const GNode &x = P.g[i];
      if (x.has_val)
        l(fmt("  FK_BUF(float) fv%d = FK_MAKE(float, fk_sm + %d, %d, %d);", i, x.off_v, x.cap, i));
      if (x.has_aux)
        l(fmt("  FK_BUF(fk_u16) fa%d = FK_MAKE(fk_u16, fk_sm + %d, %d, %d);", i, x.off_a, x.cap, 100 + i));
    }
    if (P.bwd && P.npred > 0 && !P.gring)
      l(fmt("  FK_BUF(fk_u64) fj = FK_MAKE(fk_u64, fk_sm + %d, %d, 200);", P.off_j, P.capA * P.npred));
    if (P.bwd && P.npred > 0 && P.gring)   // this CTA's adjoint rings
      l(fmt("  FK_BUF(fk_u64) fj = FK_MAKE(fk_u64, ws + (long long)blockIdx.x * %d, %d, 201);", P.npred * P.RING,
            P.npred * P.RING));
    l(fmt("  float *const fk_vcell = reinterpret_cast<float *>(fk_sm + %d);", P.off_cells));
    l(fmt("  int *const fk_acell = reinterpret_cast<int *>(fk_sm + %d);", P.off_cells + 4 * P.n));
    l(fmt("  fk_u64 *const fk_jcell = reinterpret_cast<fk_u64 *>(fk_sm + %d);", P.off_cells + 8 * P.n));
    l(fmt("  void *const fk_scr = fk_sm + %d;", P.off_scr));
    l("  const int tid = threadIdx.x;");
    l("  (void)fk_vcell; (void)fk_acell; (void)fk_jcell; (void)gout; (void)gsig; (void)out; (void)ws; (void)fk_status;");
    if (P.bwd) {
      l("  __shared__ unsigned s_gmax;");
      l("  fk_u64 pol_first;");
      l("  asm volatile(\"createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\" : \"=l\"(pol_first));");
    }
    l("  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {");
    l("    const long long b = item / segs;");
    l("    const int s0 = (int)(item - b * segs) * seg;");
    l("    const int s1 = min(s0 + seg, T);");
    l(fmt("    const float *__restrict__ xs = sig + b * (long long)T * %d;", D));
    if (!P.bwd) {
      l("    float *__restrict__ orow = out + b * (long long)T;");
      l("    const int R0 = s0;");
    } else {
      l("    const float *__restrict__ grow = gout + b * (long long)T;");
      l(fmt("    float *__restrict__ gs = gsig + b * (long long)T * %d;", D));
      l("    float *__restrict__ orow = out ? out + b * (long long)T : nullptr;");
      l(fmt("    const int R0 = max(0, s0 - %d);", P.HMAX));
      // fixed-point scale from the largest root gradient of the whole trace
      l("    if (tid == 0) s_gmax = 0u;");
      if (P.npred > 0) {
        if (P.gring) {
          // the first step's slots; later steps clear their new slots as they become live
          l(fmt("    for (int j = R0 + %d + tid; j < min(R0 + %d, s1) + %d; j += NT) {", P.LP, P.TILE, P.HP));
          l(fmt("      const int js = (j - %d) & %d;", P.LP, P.RING - 1));
          for (int k = 0; k < P.npred; ++k) l(fmt("      __stcg(&fj[%d + js], 0ull);", k * P.RING));
          l("    }");
        }
        else l(fmt("    fk_zero<NT>(reinterpret_cast<float *>(FK_PTR(fj)), 0, %d);", 2 * P.capA * P.npred));
        l(fmt("    if (tid < %d) fk_jcell[tid] = 0ull;", P.npred));
      }
      l("    __syncthreads();");
      l("    {");
      l("      float m = fk_trace_gmax<NT>(grow, T);");
      l("#pragma unroll");
      l("      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FK_FULL, m, o));");
      l("      if ((tid & 31) == 0) atomicMax(&s_gmax, __float_as_uint(m));");
      l("    }");
      l("    __syncthreads();");
      l("    const FkFix fx = fk_fix_scale(__uint_as_float(s_gmax));");
    }
    l(fmt("    for (int t0 = R0; t0 < s1; t0 += %d) {", TILE));
    l(fmt("      const int t1 = min(t0 + %d, s1);", TILE));
    l("      const bool first = t0 == R0;");
    if (P.bwd && P.gring && P.npred > 0) {
      // ring slots of the samples that become live in this step held samples RING earlier,
      // all emitted by now: clear them before this step's deposits (barriers follow)
      l("      if (!first) {");
      l(fmt("        for (int j = t0 + %d + tid; j < t1 + %d; j += NT) {", P.HP, P.HP));
      l(fmt("          const int js = (j - %d) & %d;", P.LP, P.RING - 1));
      for (int k = 0; k < P.npred; ++k) l(fmt("          __stcg(&fj[%d + js], 0ull);", k * P.RING));
      l("        }");
      l("      }");
    }
    if (P.npred > 0) {
      // the signal rows the next step's predicate pass reads, fetched into L2 in the background
      l("      if (tid == 0 && t1 < s1) {");
      l(fmt("        const long long r0 = min((long long)t1 + %d, (long long)T), r1 = min((long long)t1 + %d, (long long)T);",
            P.HP, P.TILE + P.HP));
      l(fmt("        fk_prefetch_l2(xs + r0 * %d, xs + r1 * %d, sig, sig + (long long)T * %d * (b + 1));", D, D, D));
      l("      }");
    }
    s += "      // ---- node passes\n";
    pred_pass();
    {
      // level by level (a node reads only lower levels); a barrier only where the level changes
      std::vector<int> order;
      for (int i = 0; i < P.n; ++i)
        if (!is_pred(P.g[i].op) && !(i == P.root && !P.g[i].has_val)) order.push_back(i);
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P.g[a].level < P.g[b].level; });
      for (size_t k = 0; k < order.size(); ++k) {
        const bool last = k + 1 == order.size();
        node_pass(order[k], last || P.g[order[k + 1]].level != P.g[order[k]].level);
      }
    }
    if (!P.bwd) {
      l("      for (int q = t0 + tid; q < t1; q += NT) orow[q] = " + root_value() + ";");
    } else {
      aux_pad_fills();
      // walk: a thread takes consecutive root samples, so that runs of equal targets add once
      const int RW = (TILE + NT - 1) / NT;
      if (P.npred > 0) l("      {  // selection walk and fixed-point deposits");
      else l("      if (false) {  // no predicate: no gradient reaches the signal");
      l(fmt("        const int qa = t0 + tid * %d, qb = min(qa + %d, t1);", RW, RW));
      l("        int ck = -1, cp = 0;");
      l("        fk_i64 acc = 0;");
      l("        auto flush = [&]() {");
      l("          if (ck < 0 || acc == 0) return;");
      l(fmt("          if (cp >= T - 1) fk_red_add(fk_jcell + ck, acc);"));
      if (P.npred == 0)
        ;
      else if (P.gring)
        l(fmt("          else atomicAdd(&fj[ck * %d + ((cp - %d) & %d)], (fk_u64)acc);", P.RING, P.LP, P.RING - 1));
      else
        l(fmt("          else fk_red_add(&fj[ck * %d + (cp - (t0 + %d))], acc);", P.capA, P.LP));
      l("        };");
      // the root gradients of the thread's samples, loaded together (the trace was kept in L2
      // by the scale pre-pass; this is its last use)
      l(fmt("        float gq[%d];", RW));
      l("#pragma unroll");
      l(fmt("        for (int r = 0; r < %d; ++r) gq[r] = qa + r < qb ? fk_ldg_first(grow + qa + r, pol_first) : 0.f;", RW));
      // first every sample's walk (independent: their loads overlap), then the runs of equal
      // targets and their deposits
      l(fmt("        int wl[%d], wp[%d];", RW, RW));
      l("#pragma unroll");
      l(fmt("        for (int r = 0; r < %d; ++r) {", RW));
      l("          const int q = qa + r;");
      l("          float g = gq[r];");
      l("          int pos = q, leaf = -1;");
      l("          if (q < qb) {");
      walk(P.root, 12);
      l("          }");
      l("          wl[r] = leaf;");
      l("          wp[r] = pos;");
      l("          gq[r] = g;");
      l("        }");
      l("#pragma unroll");
      l(fmt("        for (int r = 0; r < %d; ++r) {", RW));
      l("          if (wl[r] < 0) continue;");
      l("          const fk_i64 v = fk_to_fix(fx, gq[r]);");
      l("          if (wl[r] == ck && wp[r] == cp) acc += v;");
      l("          else { flush(); ck = wl[r]; cp = wp[r]; acc = v; }");
      l("        }");
      l("        flush();");
      l("      }");
      l("      if (orow) for (int q = max(t0, s0) + tid; q < t1; q += NT) orow[q] = " + root_value() + ";");
      l("      __syncthreads();");
      // signal gradient of the samples whose predicate adjoints are complete
      l("      {");
      l(fmt("        const int j0 = max(t0 + %d, s0), j1 = min(min(t1 + %d, s1), T - 1);", P.LP, P.LP));
      l(fmt("        if (first && s0 < j0) for (int i = s0 * %d + tid; i < min(j0, T - 1) * %d; i += NT) gs[i] = 0.f;", D,
            D));
      if (P.npred > 0) {
        // EB samples per thread per iteration: their adjoint loads are issued together
        const int EB = P.gring ? 4 : 2;
        l(fmt("        for (int jb = j0 + tid; jb < j1; jb += NT * %d) {", EB));
        l(fmt("          fk_u64 av[%d][%d];", EB, P.npred));
        l("#pragma unroll");
        l(fmt("          for (int e = 0; e < %d; ++e) {", EB));
        l("            const int j = jb + e * NT;");
        if (P.gring) {
          // L2 reads: the deposits of other threads are atomics performed at L2
          l(fmt("            const int js = (j - %d) & %d;", P.LP, P.RING - 1));
          for (int k = 0; k < P.npred; ++k)
            l(fmt("            av[e][%d] = j < j1 ? __ldcg(&fj[%d + js]) : 0ull;", k, k * P.RING));
        } else {
          l(fmt("            const int ja = j - (t0 + %d);", P.LP));
          for (int k = 0; k < P.npred; ++k) l(fmt("            av[e][%d] = j < j1 ? fj[%d + ja] : 0ull;", k, k * P.capA));
        }
        l("          }");
        l("#pragma unroll");
        l(fmt("          for (int e = 0; e < %d; ++e) {", EB));
        l("            const int j = jb + e * NT;");
        l("            if (j >= j1) break;");
        for (int k = 0; k < P.npred; ++k) l(fmt("            const float a%d = fk_from_fix(fx, av[e][%d]);", k, k));
        for (int d = 0; d < D; ++d) {
          l("            {");
          l("              float acc = 0.f;");
          // a zero weight adds a zero to a finite sum (acc starts at +0): skipping it leaves the
          // result's bits unchanged
          for (int k = 0; k < P.npred; ++k)
            if (P.pw[(size_t)k * D + d] != 0.f)
              l(fmt("              acc = fmaf(%s, a%d, acc);", flit(P.pw[(size_t)k * D + d]).c_str(), k));
          l(fmt("              gs[(long long)j * %d + %d] = acc;", D, d));
          l("            }");
        }
        l("          }");
        l("        }");
      } else {
        l(fmt("        for (int i = j0 * %d + tid; i < j1 * %d; i += NT) gs[i] = 0.f;", D, D));
      }
      l("      }");
      l("      __syncthreads();");
    }
    l("      if (t1 < s1) {");
    shift();
    l("      }");
    l("    }");
    if (P.bwd) {
      // sample T-1 collects every read at or past the end of the trace
      l("    if (s1 == T) {");
      l(fmt("      for (int d = tid; d < %d; d += NT) {", D));
      l("        float acc = 0.f;");
      if (P.npred > 0) {
        l(fmt("        const float *const w = fk_pw;"));
        l(fmt("        for (int k = 0; k < %d; ++k) acc = fmaf(w[k * %d + d], fk_from_fix(fx, fk_jcell[k]), acc);", P.npred, D));
      }
      l(fmt("        gs[(long long)(T - 1) * %d + d] = acc;", D));
      l("      }");
      l("    }");
    }
    l("    __syncthreads();");
    l("  }");
    l("}");
    // the predicate gradient weights for the final sample, as a device table
    std::string tbl = fmt("__device__ const float fk_pw[%d] = {", std::max(1, (int)P.pw.size()));
    for (size_t i = 0; i < P.pw.size(); ++i) tbl += (i ? ", " : "") + flit(P.pw[i]);
    if (P.pw.empty()) tbl += "0.f";
    tbl += "};\n";
    // insert the table before the kernel
    const std::string marker = "#define NT ";
    const size_t at = s.find(marker);
    s.insert(at, tbl);
    return s;
  }
};

// ------------------------------------------------------------------ compile cache
struct Compiled {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  int smem = 0;
  int bps = 0;             // resident CTAs per SM (from the occupancy API, per device below)
};

std::mutex g_mu;
std::map<std::string, std::shared_ptr<Compiled>> g_cache;   // key: generated source

stl_status compile_src(const std::string &src, const std::string &name, std::vector<char> *cubin, std::string *err) {
  Nvrtc &N = nvrtc();
  if (!N.ok) {
    *err = "formula-compiled kernels need NVRTC: " + N.why;
    return STL_ERR_UNSUPPORTED;
  }
  nvrtcProgram_t prog = nullptr;
  int r = N.create(&prog, src.c_str(), (name + ".cu").c_str(), 0, nullptr, nullptr);
  if (r != 0) {
    *err = std::string("nvrtcCreateProgram: ") + N.err(r);
    return STL_ERR_CUDA;
  }
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false"};
  r = N.compile(prog, 3, opts);
  if (r != 0) {
    size_t n = 0;
    N.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) N.log(prog, &log[0]);
    N.destroy(&prog);
    *err = "NVRTC failed on a generated kernel: " + log.substr(0, 4000);
    return STL_ERR_CUDA;
  }
  size_t n = 0;
  N.cubin_size(prog, &n);
  cubin->resize(n);
  N.cubin(prog, cubin->data());
  N.destroy(&prog);
  return STL_OK;
}

struct Shape {
  int NT, TILE;
};

// largest tile (multiple of 32, at most `want`) whose buffers fit the shared memory limit
bool fit_tile(const FkFormula &f, bool bwd, int NT, int want, int max_smem, GPlan &P, std::string *why,
              bool gring) {
  for (int tile = want; tile >= 512; tile -= (tile > 2048 ? 512 : 256)) {
    if (!build_plan(f, bwd, NT, tile, P, why, gring)) return false;
    if (P.smem <= max_smem) return true;
  }
  if (why) *why = "the formula's buffers do not fit in shared memory at a 512-sample tile";
  return false;
}

// one window pass per step (tile = threads x run length); backward runs of 9 measured best
// (the nested Until/Always/Eventually formula at B=1024 T=50000: runs of 7 / 9 / 11 at 512
// threads, 1.59 / 1.53 / 1.67 ms)
int default_tile(bool bwd, int NT) { return bwd ? NT * 9 : NT * 15; }

// The plan of one call shape.  Backward launches keep their 64-bit predicate adjoint rings in
// shared memory when the requested tile fits with them, else in the caller's workspace (L2:
// global 64-bit reductions, L2-only reads), which leaves shared memory to the node buffers: for
// the nested Until/Always/Eventually formula this allows a tile of 4608 instead of 3072 (backward
// at B=1024, T=50000: 2.18 -> 1.53 ms).
bool choose_plan(const FkFormula &f, bool bwd, int NT, int tile_req, int max_smem, GPlan &P, std::string *why) {
  const int want = tile_req > 0 ? tile_req : default_tile(bwd, NT);
  const bool shared_ok = fit_tile(f, bwd, NT, want, max_smem, P, why, false);
  if (!bwd || P.npred == 0 || (shared_ok && P.TILE >= want)) return shared_ok;
  GPlan G;
  std::string w2;
  if (fit_tile(f, bwd, NT, want, max_smem, G, &w2, true) && (!shared_ok || G.TILE > P.TILE)) {
    P = G;
    return true;
  }
  return shared_ok;
}

// CTAs that can be resident at once (an upper bound on the grid) for this plan
int grid_cap(const GPlan &P, int sms) {
  const int by_smem = std::max(1, (228 * 1024) / (P.smem + 1024));
  return sms * std::max(1, std::min(2048 / P.NT, by_smem));
}
size_t ws_bytes_for(const GPlan &P, int sms) {
  return P.gring ? (size_t)grid_cap(P, sms) * P.npred * P.RING * 8 : 0;
}

stl_status get_kernel(const FkFormula &f, bool bwd, int NT, int tile_req, int max_smem, GPlan &P,
                      std::shared_ptr<Compiled> &out, std::string *err, std::string *src_out, bool load) {
  std::string why;
  if (!choose_plan(f, bwd, NT, tile_req, max_smem, P, &why)) {
    *err = why;
    return STL_ERR_UNSUPPORTED;
  }
  Gen G(P, f);
  const std::string name = bwd ? "stl_fk_bwd" : "stl_fk_fwd";
  const std::string src = G.source(name);
  if (src_out) *src_out = src;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(src);
    if (it != g_cache.end() && (!load || it->second->kern)) { out = it->second; return STL_OK; }
  }
  // STL_FK_DUMP=<directory>: keep a copy of every generated source (for inspection)
  if (const char *dump = std::getenv("STL_FK_DUMP")) {
    if (*dump) {
      unsigned long long hsh = 1469598103934665603ULL;
      for (unsigned char ch : src) hsh = (hsh ^ ch) * 1099511628211ULL;
      const std::string path = fmt("%s/%s_%016llx.cu", dump, name.c_str(), hsh);
      if (FILE *fp = std::fopen(path.c_str(), "w")) {
        std::fwrite(src.data(), 1, src.size(), fp);
        std::fclose(fp);
      }
    }
  }
  std::vector<char> cubin;
  stl_status s = compile_src(src, name, &cubin, err);
  if (s) return s;
  auto c = std::make_shared<Compiled>();
  c->smem = P.smem;
  if (load) {
    cudaError_t e = cudaLibraryLoadData(&c->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) { *err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e); return STL_ERR_CUDA; }
    e = cudaLibraryGetKernel(&c->kern, c->lib, name.c_str());
    if (e != cudaSuccess) { *err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e); return STL_ERR_CUDA; }
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[src] = c;
  out = c;
  return STL_OK;
}

}  // namespace

bool stl_fk_available(std::string *why) {
  Nvrtc &N = nvrtc();
  if (!N.ok && why) *why = N.why;
  return N.ok;
}

bool stl_fk_eligible(const FkFormula &f, const stl_params &p, long long T, std::string *why) {
  auto no = [&](const char *m) { if (why) *why = m; return false; };
  if (p.mode != STL_HARD) return no("compiled kernels serve hard semantics");
  const std::vector<stl_node> &nd = *f.nodes;
  for (const stl_node &x : nd) {
    switch (x.op) {
      case STL_OP_PRED_GT: case STL_OP_PRED_LT: case STL_OP_TRUE: case STL_OP_NOT: case STL_OP_AND: case STL_OP_OR:
        break;
      case STL_OP_EVENTUALLY: case STL_OP_ALWAYS: case STL_OP_UNTIL:
        if (x.bound_slot >= 0) return no("per-trace interval bounds");
        if (std::isinf(x.b)) return no("an unbounded interval");
        if (x.b > 16000.f) return no("an interval end beyond 16000 samples");
        break;
      default:
        return no("an operator outside the compiled set (norm predicates, sigmoid-masked windows)");
    }
  }
  if (T > (1LL << 30)) return no("T beyond 2^30");
  // every node's first sample must lie in the trace (so that its value at T-1 is computed)
  GPlan P;
  std::string w;
  if (!build_plan(f, false, 512, 512, P, &w)) { if (why) *why = w; return false; }
  if (T < (long long)P.LOMAX + 1) return no("the trace is shorter than a node's first read");
  return true;
}

namespace {
int g_sms = 0, g_smem_optin = 0;
stl_status device_limits(std::string *err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) { *err = std::string("device query: ") + cudaGetErrorString(e); return STL_ERR_CUDA; }
  return STL_OK;
}
}  // namespace

stl_status stl_fk_plan_shape(const FkFormula &f, bool bwd, int threads, int tile, int *tile_out, int *smem_out,
                             size_t *ws_out, std::string *err) {
  const int NT = threads ? threads : 512;
  if (NT != 256 && NT != 512 && NT != 768 && NT != 1024) { *err = "threads must be 256, 512, 768 or 1024"; return STL_ERR_INVALID_ARG; }
  int max_smem = 232448;
  if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0) != cudaSuccess) {
    cudaGetLastError();
    max_smem = 232448;
  }
  GPlan P;
  std::string why;
  if (!choose_plan(f, bwd, NT, tile, max_smem - 1024, P, &why)) {
    *err = why;
    return STL_ERR_UNSUPPORTED;
  }
  if (tile_out) *tile_out = P.TILE;
  if (smem_out) *smem_out = P.smem;
  if (ws_out) {
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    *ws_out = ws_bytes_for(P, sms);
  }
  return STL_OK;
}

stl_status stl_fk_compile_only(const FkFormula &f, bool bwd, long long T, int threads, int tile, int *tile_out,
                               int *smem_out, std::string *src, std::string *err) {
  (void)T;
  const int NT = threads ? threads : 512;
  if (NT != 256 && NT != 512 && NT != 768 && NT != 1024) { *err = "threads must be 256, 512, 768 or 1024"; return STL_ERR_INVALID_ARG; }
  GPlan P;
  std::shared_ptr<Compiled> c;
  stl_status s = get_kernel(f, bwd, NT, tile, 232448 - 1024, P, c, err, src, false);
  if (s) return s;
  if (tile_out) *tile_out = P.TILE;
  if (smem_out) *smem_out = P.smem;
  return STL_OK;
}

stl_status stl_fk_run(const FkFormula &f, const FkCall &c, std::string *err) {
  std::string why;
  stl_params hp{};
  hp.mode = STL_HARD;
  if (!stl_fk_eligible(f, hp, c.T, &why)) { *err = "compiled kernel not applicable: " + why; return STL_ERR_UNSUPPORTED; }
  if (c.B == 0) return STL_OK;
  stl_status s = device_limits(err);
  if (s) return s;
  const int NT = c.threads ? c.threads : 512;
  if (NT != 256 && NT != 512 && NT != 768 && NT != 1024) {
    *err = "threads must be 256, 512, 768 or 1024 for the compiled kernels";
    return STL_ERR_INVALID_ARG;
  }
  GPlan P;
  std::shared_ptr<Compiled> k;
  s = get_kernel(f, c.bwd, NT, c.tile, g_smem_optin - 1024, P, k, err, nullptr, true);
  if (s) return s;
  const void *fn = (const void *)k->kern;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem);
  if (e != cudaSuccess) { *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e); return STL_ERR_CUDA; }
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, NT, P.smem);
  if (e != cudaSuccess || bps < 1) {
    *err = std::string("compiled kernel does not fit on an SM: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "");
    return STL_ERR_UNSUPPORTED;
  }
  // segments: about two work items per resident CTA when there are few traces, each long
  // compared with the backward warm-up, and the last one holding every node's first read
  const long long T = c.T, B = c.B;
  const long long slots = (long long)g_sms * bps;
  long long segs = 1;
  if (c.segment > 0) {
    segs = (T + c.segment - 1) / c.segment;
  } else if (B < 2 * slots) {
    const long long want = (2 * slots + B - 1) / B;
    const long long by_len = std::max(1LL, T / std::max(4LL * (P.HMAX + P.TILE), (long long)P.TILE));
    segs = std::max(1LL, std::min(want, by_len));
  }
  long long seg = (T + segs - 1) / segs;
  for (;;) {
    segs = (T + seg - 1) / seg;
    const long long last = T - (segs - 1) * seg;
    if (segs == 1 || last >= P.LOMAX + 1) break;
    seg = (T + segs - 2) / (segs - 1);   // one segment fewer
  }
  const long long n_items = B * segs;
  const int grid = (int)std::max(1LL, std::min(n_items, std::min(slots, (long long)grid_cap(P, g_sms))));
  if (P.gring) {
    const size_t need = (size_t)grid * P.npred * P.RING * 8;
    if (!c.ws || c.ws_bytes < need) {
      *err = fmt("workspace of %zu bytes needed (adjoint rings)", need);
      return STL_ERR_WORKSPACE;
    }
  }
  void *ws = c.ws;
  int *status = nullptr;
  if (stl_status_ptr(&status) != 0) { cudaGetLastError(); status = nullptr; }
  int Ti = (int)T, segi = (int)seg, segsi = (int)segs;
  long long items = n_items;
  const float *sig = c.sig, *gout = c.gout;
  float *out = c.out, *gsig = c.gsig;
  void *args[] = {(void *)&sig, (void *)&gout, (void *)&out, (void *)&gsig, (void *)&ws, (void *)&status, (void *)&Ti,
                  (void *)&segi, (void *)&segsi, (void *)&items};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, (size_t)P.smem, (cudaStream_t)c.stream);
  if (e != cudaSuccess) { *err = std::string("compiled kernel launch: ") + cudaGetErrorString(e); return STL_ERR_CUDA; }
  return STL_OK;
}
