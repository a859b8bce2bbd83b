/*
 * stl_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU evaluator of STL robustness traces and of their analytic
 * (sub)gradients, written directly from the definitions of STLCG++ (arXiv 2501.04194):
 *
 *   - the quantitative semantics, Sec. III-B, Eq. "quantitative";
 *   - the robustness trace, Sec. III-D, Definition 1 (one value per sub-trajectory);
 *   - the logsumexp smooth max / min, Sec. III-C;
 *   - the end padding of the unrolled signal, Sec. IV-B Step 1;
 *   - the Until trace, Sec. IV-C (max over i of min(min over tau<=i of phi, psi));
 *   - the sigmoid interval mask, Sec. VI, Eq. "smooth mask".
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of bench.py may load
 * this file.  It shares no code, header or constant with the CUDA library: it has its
 * own node encoding (below) and its own Python marshalling (oracle/__init__.py).
 *
 * Every temporal operator is an O(T * window) loop over the literal definition; Until
 * takes the literal triple loop (max over i, running min over tau).  There is no
 * blocking, no sliding-window trick and no reordering beyond those definitions.
 *
 * Readings where the paper is silent (numbered here; the comments below refer to them):
 *   R1  a trace has T samples, indices 0..T-1;
 *   R2  a read at j >= T returns the pad: the last sample (PAD_LAST, gradient to T-1)
 *       or a constant (PAD_CONST, no gradient); smooth windows count pad reads with
 *       multiplicity, exactly as the padded unroll of Sec. IV-B does;
 *   R3  b = +inf means the whole signal: b := T-1;
 *   R4  True has robustness +inf;
 *   R5  hard ties: window max/min take the earliest time index; And/Or take the left
 *       operand; Until takes the earliest maximising i, then in min(P, psi) the running
 *       minimum P wins ties, then the earliest argmin inside P;
 *   R6  the smooth mask enters the logsumexp as a weight: (1/tau) log sum_i m_i e^{tau x};
 *       in hard mode it selects the offsets with m_i > 0 and has no (a, b) gradient;
 *   R7  predicates are evaluated as float32 arithmetic without fused multiply-add:
 *       every operation is done in double and rounded to float (exact for +,-,x under
 *       double rounding since 53 >= 2*24+2); ``exact`` skips the rounding.
 *       Signals and bounds arrive as double (float32 inputs widen exactly), so that
 *       finite-difference checks can perturb them in double precision;
 *   R15 a norm predicate (Sec. VII-A "inside" a region) is mu(x) = ||diag(s)(x - g)||_2 with
 *       per-dimension scales s (0 drops a dimension) and centre g; "<" gives r - mu(x)
 *       (inside the ball of radius r), ">" gives mu(x) - r (outside it);
 *   R17 softmax-weighted mode (the "soft" approximation of Sec. III-C): every min/max over a
 *       multiset becomes sum v e^{sgn tau v} / sum e^{sgn tau v} over that same multiset
 *       (windows with pads counted with multiplicity; the two operands of and/or; the three
 *       levels of the Until construction of Sec. IV-C, each reduced once, so no nesting
 *       of the window itself, Sec. IV-D); the smooth mask enters as a weight m_i on both sums;
 *   R20 an Until over a sigmoid-masked interval weights the offsets i of its outer max by m_i
 *       (hard: the offsets with m_i > 0), the prefix over phi starting at i = 0 as before.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum {
  O_PRED_GT = 0, O_PRED_LT = 1, O_TRUE = 2, O_NOT = 3, O_AND = 4, O_OR = 5,
  O_EV = 6, O_ALW = 7, O_UNTIL = 8, O_EV_SM = 9, O_ALW_SM = 10, O_NORM_GT = 11, O_NORM_LT = 12,
  O_UNTIL_SM = 13
};
enum { O_PAD_LAST = 0, O_PAD_CONST = 1 };
enum { O_MAX_D = 64 };   /* largest signal dimension the oracle accepts */
enum { O_HARD = 0, O_SMOOTH = 1, O_SOFTMAX = 2 };

typedef struct {
  int32_t op, c0, c1, slot;
  double a, b;
  int32_t pad_mode, w_off;
  double pad_value, c;
} onode;

typedef struct {
  const onode *nodes;
  int n_nodes, root, D, n_slots, mode, exact, backward;
  const double *w;
  const double *sig;
  const int64_t *offsets; /* [B+1] start of each trace in sig (rows of D floats) */
  const double *bounds;   /* [B, n_slots, 2] or NULL */
  int64_t B;
  double tau, mask_c, mask_eps;
  double *out;            /* packed like sig rows: one value per sample */
  const double *gout;
  double *gsig, *gbounds;
  int64_t next;
  pthread_mutex_t lock;
  int status;
} octx;

/* ------------------------------------------------------------------ helpers */
static double f32(double v) { return (double)(float)v; }

/* read x at j with the node's padding (R2); *src = index that receives the gradient */
static double rd(const double *x, int64_t T, int64_t j, const onode *nd, int64_t *src) {
  if (j < T) { *src = j; return x[j]; }
  if (nd->pad_mode == O_PAD_CONST) { *src = -1; return nd->pad_value; }
  *src = T - 1;
  return x[T - 1];
}

static void bounds_of(const octx *cx, const onode *nd, int64_t b, double *a_out, double *b_out) {
  if (nd->slot >= 0 && cx->bounds) {
    const double *p = cx->bounds + ((size_t)b * cx->n_slots + nd->slot) * 2;
    *a_out = p[0]; *b_out = p[1];
  } else { *a_out = nd->a; *b_out = nd->b; }
}

/* integer window [ia, ib] for the hard/LSE temporal operators (R3) */
static void int_window(const octx *cx, const onode *nd, int64_t b, int64_t T, int64_t *ia, int64_t *ib) {
  double a, bb;
  bounds_of(cx, nd, b, &a, &bb);
  *ia = (int64_t)a;
  *ib = isinf(bb) ? T - 1 : (int64_t)bb;
  if (*ib < *ia) *ib = *ia;
}

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }

/* smooth interval mask, Eq. "smooth mask", with a, b already in steps (R6) */
static double smask(double i, double a, double b, double c, double eps) {
  double m = sigm(c * (i - a)) - sigm(c * (i - b)) - eps;
  return m > 0.0 ? m : 0.0;
}
static double smask_da(double i, double a, double b, double c, double eps) {
  if (smask(i, a, b, c, eps) <= 0.0) return 0.0;
  double s = sigm(c * (i - a));
  return -c * s * (1.0 - s);
}
static double smask_db(double i, double a, double b, double c, double eps) {
  if (smask(i, a, b, c, eps) <= 0.0) return 0.0;
  double s = sigm(c * (i - b));
  return c * s * (1.0 - s);
}
/* last offset with a possibly positive mask: beyond b + log((1-eps)/eps)/c the
   difference of sigmoids is below eps */
static int64_t smask_last(double b, double c, double eps) {
  return (int64_t)ceil(b + log((1.0 - eps) / eps) / c) + 2;
}

/* logsumexp of n values v[] scaled by sgn*tau: returns (1/tau) log sum w_i e^{tau*sgn*v_i},
   weights w may be NULL (all ones) */
static double lse(const double *v, const double *w, int64_t n, double tau, double sgn) {
  double m = -INFINITY;
  for (int64_t i = 0; i < n; i++) {
    if (w && w[i] <= 0.0) continue;
    double z = sgn * tau * v[i];
    if (z > m) m = z;
  }
  if (m == -INFINITY) return -INFINITY;
  if (m == INFINITY) return INFINITY;
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) {
    if (w && w[i] <= 0.0) continue;
    s += (w ? w[i] : 1.0) * exp(sgn * tau * v[i] - m);
  }
  return (m + log(s)) / tau;
}

/* softmax-weighted max (sgn = +1) or min (sgn = -1) of n values (Sec. III-C, the "soft"
   approximation; R17): y = sum w_i v_i e^{sgn tau v_i} / sum w_i e^{sgn tau v_i}, weights w may be
   NULL (all ones), entries with w_i <= 0 are absent.  Infinite entries: sgn*v = -inf carries no
   weight; if some sgn*v = +inf, y is that infinity; with no finite weight left y = -sgn*inf.
   p (may be NULL) receives the normalised weights p_i = w_i e^{sgn tau v_i} / sum (0 for
   absent or infinite entries). */
static double swm(const double *v, const double *w, int64_t n, double tau, double sgn, double *p) {
  double m = -INFINITY;
  for (int64_t i = 0; i < n; i++) {
    if (p) p[i] = 0.0;
    if (w && w[i] <= 0.0) continue;
    double z = sgn * v[i];
    if (z == INFINITY) return v[i];
    if (z == -INFINITY) continue;
    if (sgn * tau * v[i] > m) m = sgn * tau * v[i];
  }
  if (m == -INFINITY) return -sgn * INFINITY;
  double s = 0.0, num = 0.0;
  for (int64_t i = 0; i < n; i++) {
    if (w && w[i] <= 0.0) continue;
    if (isinf(v[i])) continue;
    double e = (w ? w[i] : 1.0) * exp(sgn * tau * v[i] - m);
    s += e;
    num += e * v[i];
    if (p) p[i] = e;
  }
  if (p)
    for (int64_t i = 0; i < n; i++) p[i] /= s;
  return num / s;
}

/* d y / d v_i of swm: p_i (1 + sgn tau (v_i - y)) (0 for absent or infinite entries) */
static double swm_d(double p, double v, double y, double tau, double sgn) {
  if (p == 0.0 || isinf(v) || isinf(y)) return 0.0;
  return p * (1.0 + sgn * tau * (v - y));
}

/* two-term smooth min / max (Sec. III-C): min(x,y) - log1p(e^{-tau|x-y|})/tau */
static double smin2(double x, double y, double tau) {
  if (x == y) return x - log(2.0) / tau;
  if (isinf(x) || isinf(y)) return x < y ? x : y;
  double m = x < y ? x : y;
  return m - log1p(exp(-tau * fabs(x - y))) / tau;
}
static double smax2(double x, double y, double tau) { return -smin2(-x, -y, tau); }

/* ------------------------------------------------------------------ per trace */
typedef struct {
  double **val, **adj;
  double *tmp, *tmp2, *tmp3;
  int64_t *itmp;
  int64_t cap;
} work;

static int work_init(work *wk, int n, int64_t T, int64_t wcap) {
  if (n <= 0 || T <= 0 || wcap <= 0) return -1;
  wk->val = calloc((size_t)(unsigned)n, sizeof(double *));
  wk->adj = calloc((size_t)(unsigned)n, sizeof(double *));
  if (!wk->val || !wk->adj) return -1;
  for (int i = 0; i < n; i++) {
    wk->val[i] = calloc((size_t)T, sizeof(double));
    wk->adj[i] = calloc((size_t)T, sizeof(double));
    if (!wk->val[i] || !wk->adj[i]) return -1;
  }
  wk->cap = wcap;
  wk->tmp = calloc((size_t)wcap, sizeof(double));
  wk->tmp2 = calloc((size_t)wcap, sizeof(double));
  wk->tmp3 = calloc((size_t)wcap * 3, sizeof(double));   /* up to three weight vectors (Until) */
  wk->itmp = calloc((size_t)wcap, sizeof(int64_t));
  return (wk->tmp && wk->tmp2 && wk->tmp3 && wk->itmp) ? 0 : -1;
}

static void work_free(work *wk, int n) {
  for (int i = 0; i < n && wk->val && wk->adj; i++) { free(wk->val[i]); free(wk->adj[i]); }
  free(wk->val); free(wk->adj); free(wk->tmp); free(wk->tmp2); free(wk->tmp3); free(wk->itmp);
}

/* mu(x) for a norm predicate: the Euclidean distance of the scaled offset from a centre,
 * mu(x) = sqrt(sum_d u_d^2), u_d = s_d (x_d - g_d), with s = w[0..D) and g = w[D..2D).  This
 * is the "inside region" predicate of the trajectory-planning example, Sec. VII-A (R15).
 * Rounded mode: every operation in float32 order, sum left to right, then a correctly
 * rounded square root (exact under double rounding, as for the other operations). */
static double norm_mu(const octx *cx, const onode *nd, const double *row, double *u) {
  const double *sc = cx->w + nd->w_off, *g = sc + cx->D;
  double q = 0.0;
  for (int d = 0; d < cx->D; d++) {
    if (cx->exact) {
      u[d] = sc[d] * (row[d] - g[d]);
      q += u[d] * u[d];
    } else {
      u[d] = f32(sc[d] * f32(row[d] - g[d]));
      q = d == 0 ? f32(u[d] * u[d]) : f32(q + f32(u[d] * u[d]));
    }
  }
  return cx->exact ? sqrt(q) : f32(sqrt(q));
}

/* predicate mu(x_t) - c or c - mu(x_t), Eq. "quantitative" (R7); mu affine or a norm */
static double pred_eval(const octx *cx, const onode *nd, const double *row) {
  const double *w = cx->w + nd->w_off;
  double s;
  const int gt = nd->op == O_PRED_GT || nd->op == O_NORM_GT;
  if (nd->op == O_NORM_GT || nd->op == O_NORM_LT) {
    double u[O_MAX_D];
    s = norm_mu(cx, nd, row, u);
  } else if (cx->exact) {
    s = 0.0;
    for (int d = 0; d < cx->D; d++) s += w[d] * row[d];
  } else {
    s = f32(w[0] * row[0]);
    for (int d = 1; d < cx->D; d++) s = f32(s + f32(w[d] * row[d]));
  }
  if (cx->exact) return gt ? s - nd->c : nd->c - s;
  return gt ? f32(s - nd->c) : f32(nd->c - s);
}

/* offsets i of a smooth-mask window for trace b: [0, last] (R6) */
static int64_t sm_range(const octx *cx, const onode *nd, int64_t b, double *a, double *bb) {
  bounds_of(cx, nd, b, a, bb);
  return smask_last(*bb, cx->mask_c, cx->mask_eps);
}

static void forward_node(const octx *cx, work *wk, int k, int64_t b, const double *xs, int64_t T) {
  const onode *nd = &cx->nodes[k];
  double *y = wk->val[k];
  const double tau = cx->tau;
  const int smooth = cx->mode == O_SMOOTH;
  const int soft = cx->mode == O_SOFTMAX;
  switch (nd->op) {
    case O_PRED_GT:
    case O_PRED_LT:
    case O_NORM_GT:
    case O_NORM_LT:
      for (int64_t t = 0; t < T; t++) y[t] = pred_eval(cx, nd, xs + t * cx->D);
      break;
    case O_TRUE:
      for (int64_t t = 0; t < T; t++) y[t] = INFINITY;
      break;
    case O_NOT: {
      const double *x = wk->val[nd->c0];
      for (int64_t t = 0; t < T; t++) y[t] = -x[t];
    } break;
    case O_AND:
    case O_OR: {
      const double *x = wk->val[nd->c0], *z = wk->val[nd->c1];
      for (int64_t t = 0; t < T; t++) {
        if (soft) {
          const double v2[2] = {x[t], z[t]};
          y[t] = swm(v2, NULL, 2, tau, nd->op == O_AND ? -1.0 : 1.0, NULL);
        } else if (smooth) y[t] = nd->op == O_AND ? smin2(x[t], z[t], tau) : smax2(x[t], z[t], tau);
        else if (nd->op == O_AND) y[t] = x[t] <= z[t] ? x[t] : z[t];
        else y[t] = x[t] >= z[t] ? x[t] : z[t];
      }
    } break;
    case O_EV:
    case O_ALW: {
      /* Eventually: max_{i in [a,b]} x_{t+i}; Always: min (Eq. quantitative, Sec. IV-B) */
      const double *x = wk->val[nd->c0];
      int64_t ia, ib, src;
      int_window(cx, nd, b, T, &ia, &ib);
      const double sgn = nd->op == O_EV ? 1.0 : -1.0;
      for (int64_t t = 0; t < T; t++) {
        int64_t n = 0;
        for (int64_t i = ia; i <= ib; i++) wk->tmp[n++] = rd(x, T, t + i, nd, &src);
        if (soft) {
          y[t] = swm(wk->tmp, NULL, n, tau, sgn, NULL);
        } else if (smooth) {
          y[t] = sgn * lse(wk->tmp, NULL, n, tau, sgn);
        } else {
          double best = wk->tmp[0];
          for (int64_t i = 1; i < n; i++)
            if (sgn * wk->tmp[i] > sgn * best) best = wk->tmp[i];
          y[t] = best;
        }
      }
    } break;
    case O_UNTIL: {
      /* max_{i in [a,b]} min( min_{k in [0,i]} phi_{t+k}, psi_{t+i} )  (Sec. IV-C) */
      const double *ph = wk->val[nd->c0], *ps = wk->val[nd->c1];
      int64_t ia, ib, src;
      int_window(cx, nd, b, T, &ia, &ib);
      for (int64_t t = 0; t < T; t++) {
        if (soft) {
          /* S1: softmin over phi_{t..t+i}; S2: softmin of the pair (S1, psi_{t+i}); S3: softmax
             over i in [a, b] (each level one softmax-weighted reduction, as in Sec. IV-C) */
          int64_t n = 0;
          for (int64_t i = 0; i <= ib; i++) wk->tmp2[i] = rd(ph, T, t + i, nd, &src);
          for (int64_t i = ia; i <= ib; i++) {
            const double v2[2] = {swm(wk->tmp2, NULL, i + 1, tau, -1.0, NULL), rd(ps, T, t + i, nd, &src)};
            wk->tmp[n++] = swm(v2, NULL, 2, tau, -1.0, NULL);
          }
          y[t] = swm(wk->tmp, NULL, n, tau, 1.0, NULL);
          continue;
        }
        if (!smooth) {
          double P = INFINITY, best = -INFINITY;
          for (int64_t i = 0; i <= ib; i++) {
            double v = rd(ph, T, t + i, nd, &src);
            if (v < P) P = v;
            if (i >= ia) {
              double q = rd(ps, T, t + i, nd, &src);
              double z = P <= q ? P : q;
              if (i == ia || z > best) best = z;
            }
          }
          y[t] = best;
        } else {
          /* nested smooth operators: P_i = smin over phi_{t..t+i}; z_i = smin(P_i, psi_{t+i});
             U = smax over i of z_i */
          int64_t n = 0;
          for (int64_t i = 0; i <= ib; i++) wk->tmp2[i] = rd(ph, T, t + i, nd, &src);
          for (int64_t i = ia; i <= ib; i++) {
            double P = -lse(wk->tmp2, NULL, i + 1, tau, -1.0);
            double q = rd(ps, T, t + i, nd, &src);
            wk->tmp[n++] = smin2(P, q, tau);
          }
          y[t] = lse(wk->tmp, NULL, n, tau, 1.0);
        }
      }
    } break;
    case O_EV_SM:
    case O_ALW_SM: {
      const double *x = wk->val[nd->c0];
      double a, bb;
      int64_t last = sm_range(cx, nd, b, &a, &bb), src;
      const double sgn = nd->op == O_EV_SM ? 1.0 : -1.0;
      for (int64_t t = 0; t < T; t++) {
        int64_t n = 0;
        for (int64_t i = 0; i <= last; i++) {
          double m = smask((double)i, a, bb, cx->mask_c, cx->mask_eps);
          if (m <= 0.0) continue;
          wk->tmp[n] = rd(x, T, t + i, nd, &src);
          wk->tmp3[n] = m;
          n++;
        }
        if (n == 0) { y[t] = sgn * -INFINITY; continue; }
        if (soft) {
          y[t] = swm(wk->tmp, wk->tmp3, n, tau, sgn, NULL);
        } else if (smooth) {
          y[t] = sgn * lse(wk->tmp, wk->tmp3, n, tau, sgn);
        } else {
          double best = wk->tmp[0];
          for (int64_t i = 1; i < n; i++)
            if (sgn * wk->tmp[i] > sgn * best) best = wk->tmp[i];
          y[t] = best;
        }
      }
    } break;
    case O_UNTIL_SM: {
      /* Until over the sigmoid-masked interval (R20): the offsets i >= 0 of the outer max carry
         the weights m_i of Eq. "smooth mask"; the prefix over phi still starts at i = 0 */
      const double *ph = wk->val[nd->c0], *ps = wk->val[nd->c1];
      double a, bb;
      int64_t last = sm_range(cx, nd, b, &a, &bb), src;
      for (int64_t t = 0; t < T; t++) {
        int64_t n = 0;
        double P = INFINITY, best = -INFINITY;
        int have = 0;
        for (int64_t i = 0; i <= last; i++) wk->tmp2[i] = rd(ph, T, t + i, nd, &src);
        for (int64_t i = 0; i <= last; i++) {
          if (wk->tmp2[i] < P) P = wk->tmp2[i];
          const double m = smask((double)i, a, bb, cx->mask_c, cx->mask_eps);
          if (m <= 0.0) continue;
          const double q = rd(ps, T, t + i, nd, &src);
          double z;
          if (soft) {
            const double v2[2] = {swm(wk->tmp2, NULL, i + 1, tau, -1.0, NULL), q};
            z = swm(v2, NULL, 2, tau, -1.0, NULL);
          } else if (smooth) {
            z = smin2(-lse(wk->tmp2, NULL, i + 1, tau, -1.0), q, tau);
          } else {
            z = P <= q ? P : q;
            if (!have || z > best) best = z;
            have = 1;
          }
          wk->tmp[n] = z;
          wk->tmp3[n] = m;
          n++;
        }
        if (n == 0) y[t] = -INFINITY;
        else if (soft) y[t] = swm(wk->tmp, wk->tmp3, n, tau, 1.0, NULL);
        else if (smooth) y[t] = lse(wk->tmp, wk->tmp3, n, tau, 1.0);
        else y[t] = best;
      }
    } break;
  }
}

/* reverse-mode adjoint of node k: adds into the adjoints of its children */
static void backward_node(const octx *cx, work *wk, int k, int64_t b, int64_t T, double *gb) {
  const onode *nd = &cx->nodes[k];
  const double *g = wk->adj[k];
  const double *y = wk->val[k];
  const double tau = cx->tau;
  const int smooth = cx->mode == O_SMOOTH;
  const int soft = cx->mode == O_SOFTMAX;
  switch (nd->op) {
    case O_PRED_GT:
    case O_PRED_LT:
    case O_NORM_GT:
    case O_NORM_LT:
    case O_TRUE:
      break;
    case O_NOT: {
      double *xa = wk->adj[nd->c0];
      for (int64_t t = 0; t < T; t++) xa[t] -= g[t];
    } break;
    case O_AND:
    case O_OR: {
      const double *x = wk->val[nd->c0], *z = wk->val[nd->c1];
      double *xa = wk->adj[nd->c0], *za = wk->adj[nd->c1];
      for (int64_t t = 0; t < T; t++) {
        if (g[t] == 0.0) continue;
        if (soft) {
          const double sg = nd->op == O_AND ? -1.0 : 1.0;
          const double v2[2] = {x[t], z[t]};
          double p2[2];
          swm(v2, NULL, 2, tau, sg, p2);
          xa[t] += g[t] * swm_d(p2[0], x[t], y[t], tau, sg);
          za[t] += g[t] * swm_d(p2[1], z[t], y[t], tau, sg);
          continue;
        }
        if (smooth) {
          /* d smin(x,z)/dx = sigmoid(tau (z - x)); d smax(x,z)/dx = sigmoid(tau (x - z)) */
          double s = nd->op == O_AND ? 1.0 : -1.0;
          if (isinf(x[t]) && isinf(z[t])) { xa[t] += g[t]; continue; }
          xa[t] += g[t] * sigm(s * tau * (z[t] - x[t]));
          za[t] += g[t] * sigm(s * tau * (x[t] - z[t]));
        } else {
          int left = nd->op == O_AND ? x[t] <= z[t] : x[t] >= z[t];
          if (left) xa[t] += g[t]; else za[t] += g[t];
        }
      }
    } break;
    case O_EV:
    case O_ALW: {
      const double *x = wk->val[nd->c0];
      double *xa = wk->adj[nd->c0];
      int64_t ia, ib;
      int_window(cx, nd, b, T, &ia, &ib);
      const double sgn = nd->op == O_EV ? 1.0 : -1.0;
      for (int64_t t = 0; t < T; t++) {
        if (g[t] == 0.0) continue;
        if (soft) {
          int64_t n = 0;
          for (int64_t i = ia; i <= ib; i++) {
            wk->tmp[n] = rd(x, T, t + i, nd, &wk->itmp[n]);
            n++;
          }
          swm(wk->tmp, NULL, n, tau, sgn, wk->tmp3);
          for (int64_t i = 0; i < n; i++)
            if (wk->itmp[i] >= 0) xa[wk->itmp[i]] += g[t] * swm_d(wk->tmp3[i], wk->tmp[i], y[t], tau, sgn);
          continue;
        }
        if (smooth) {
          /* d/dx_{t+i} of (sgn/tau) log sum e^{sgn tau x} = e^{sgn tau (x - y)} */
          for (int64_t i = ia; i <= ib; i++) {
            int64_t src;
            double v = rd(x, T, t + i, nd, &src);
            if (src >= 0) xa[src] += g[t] * exp(sgn * tau * (v - y[t]));
          }
        } else {
          int64_t bsrc, src;
          double best = rd(x, T, t + ia, nd, &bsrc);
          for (int64_t i = ia + 1; i <= ib; i++) {
            double v = rd(x, T, t + i, nd, &src);
            if (sgn * v > sgn * best) { best = v; bsrc = src; }
          }
          if (bsrc >= 0) xa[bsrc] += g[t];
        }
      }
    } break;
    case O_UNTIL: {
      const double *ph = wk->val[nd->c0], *ps = wk->val[nd->c1];
      double *pha = wk->adj[nd->c0], *psa = wk->adj[nd->c1];
      int64_t ia, ib;
      int_window(cx, nd, b, T, &ia, &ib);
      for (int64_t t = 0; t < T; t++) {
        if (g[t] == 0.0) continue;
        if (soft) {
          /* chain rule through the three levels: dU/dz_i, dz_i/dP_i and dz_i/dpsi_{t+i},
             dP_i/dphi_{t+k} (k <= i), each the derivative of one softmax-weighted reduction */
          int64_t n = 0, src;
          for (int64_t i = 0; i <= ib; i++) wk->tmp2[i] = rd(ph, T, t + i, nd, &src);
          for (int64_t i = ia; i <= ib; i++) {
            const double v2[2] = {swm(wk->tmp2, NULL, i + 1, tau, -1.0, NULL), rd(ps, T, t + i, nd, &src)};
            wk->tmp[n++] = swm(v2, NULL, 2, tau, -1.0, NULL);
          }
          swm(wk->tmp, NULL, n, tau, 1.0, wk->tmp3);   /* outer weights over i */
          for (int64_t i = ia; i <= ib; i++) {
            const double zi = wk->tmp[i - ia];
            const double dUz = g[t] * swm_d(wk->tmp3[i - ia], zi, y[t], tau, 1.0);
            if (dUz == 0.0) continue;
            double pk[2];
            int64_t qs;
            const double P = swm(wk->tmp2, NULL, i + 1, tau, -1.0, NULL);
            const double v2[2] = {P, rd(ps, T, t + i, nd, &qs)};
            swm(v2, NULL, 2, tau, -1.0, pk);
            if (qs >= 0) psa[qs] += dUz * swm_d(pk[1], v2[1], zi, tau, -1.0);
            const double dzP = dUz * swm_d(pk[0], P, zi, tau, -1.0);
            if (dzP == 0.0) continue;
            /* inner weights over k <= i (tmp3 is busy; reuse the node scratch of n entries after it) */
            double *pin = wk->tmp3 + n;
            swm(wk->tmp2, NULL, i + 1, tau, -1.0, pin);
            for (int64_t kk = 0; kk <= i; kk++) {
              int64_t ks;
              rd(ph, T, t + kk, nd, &ks);
              if (ks >= 0) pha[ks] += dzP * swm_d(pin[kk], wk->tmp2[kk], P, tau, -1.0);
            }
          }
          continue;
        }
        if (!smooth) {
          /* R5: earliest maximising i; P wins ties in min(P, psi); earliest argmin in P */
          double P = INFINITY, best = -INFINITY;
          int64_t Psrc = -1, src, bsrc = -1;
          int bphi = 0;
          for (int64_t i = 0; i <= ib; i++) {
            double v = rd(ph, T, t + i, nd, &src);
            if (v < P) { P = v; Psrc = src; }
            if (i >= ia) {
              int64_t qs;
              double q = rd(ps, T, t + i, nd, &qs);
              double z;
              int zphi;
              int64_t zs;
              if (P <= q) { z = P; zphi = 1; zs = Psrc; } else { z = q; zphi = 0; zs = qs; }
              if (i == ia || z > best) { best = z; bphi = zphi; bsrc = zs; }
            }
          }
          if (bsrc >= 0) { if (bphi) pha[bsrc] += g[t]; else psa[bsrc] += g[t]; }
        } else {
          /* U = (1/tau) log sum_i e^{tau z_i}; z_i = smin(P_i, psi_{t+i});
             P_i = smin_{k<=i} phi_{t+k}.  dU/dz_i = alpha_i = e^{tau (z_i - U)};
             dz_i/dP_i = beta_i = sigmoid(tau (psi - P_i)); dz_i/dpsi = sigmoid(tau (P_i - psi));
             dP_i/dphi_{t+k} = e^{tau (P_i - phi_{t+k})} for k <= i. */
          int64_t src;
          for (int64_t i = 0; i <= ib; i++) wk->tmp2[i] = rd(ph, T, t + i, nd, &src);
          for (int64_t i = ia; i <= ib; i++) {
            double P = -lse(wk->tmp2, NULL, i + 1, tau, -1.0);
            int64_t qs;
            double q = rd(ps, T, t + i, nd, &qs);
            double z = smin2(P, q, tau);
            double alpha = exp(tau * (z - y[t]));
            if (alpha == 0.0) continue;
            double beta = isinf(P) ? 0.0 : sigm(tau * (q - P));
            double gq = isinf(q) ? 0.0 : sigm(tau * (P - q));
            if (qs >= 0 && gq > 0.0) psa[qs] += g[t] * alpha * gq;
            if (beta == 0.0) continue;
            for (int64_t kk = 0; kk <= i; kk++) {
              int64_t ks;
              double v = rd(ph, T, t + kk, nd, &ks);
              if (ks >= 0 && !isinf(v)) pha[ks] += g[t] * alpha * beta * exp(tau * (P - v));
            }
          }
        }
      }
    } break;
    case O_EV_SM:
    case O_ALW_SM: {
      const double *x = wk->val[nd->c0];
      double *xa = wk->adj[nd->c0];
      double a, bb;
      int64_t last = sm_range(cx, nd, b, &a, &bb);
      const double sgn = nd->op == O_EV_SM ? 1.0 : -1.0;
      double ga = 0.0, gbv = 0.0;
      for (int64_t t = 0; t < T; t++) {
        if (g[t] == 0.0) continue;
        if (soft) {
          /* y = sum m_i v_i e_i / sum m_i e_i: dy/dv_i = p_i (1 + sgn tau (v_i - y)),
             dy/dm_i = p_i (v_i - y) / m_i, chained to a and b through the mask */
          int64_t n = 0;
          for (int64_t i = 0; i <= last; i++) {
            wk->tmp[i] = rd(x, T, t + i, nd, &wk->itmp[i]);
            wk->tmp2[i] = smask((double)i, a, bb, cx->mask_c, cx->mask_eps);
            n = i + 1;
          }
          swm(wk->tmp, wk->tmp2, n, tau, sgn, wk->tmp3);
          for (int64_t i = 0; i < n; i++) {
            if (wk->tmp2[i] <= 0.0 || wk->tmp3[i] == 0.0) continue;
            if (wk->itmp[i] >= 0) xa[wk->itmp[i]] += g[t] * swm_d(wk->tmp3[i], wk->tmp[i], y[t], tau, sgn);
            if (isinf(y[t]) || isinf(wk->tmp[i])) continue;
            const double dm = g[t] * wk->tmp3[i] * (wk->tmp[i] - y[t]) / wk->tmp2[i];
            ga += dm * smask_da((double)i, a, bb, cx->mask_c, cx->mask_eps);
            gbv += dm * smask_db((double)i, a, bb, cx->mask_c, cx->mask_eps);
          }
          continue;
        }
        if (smooth) {
          for (int64_t i = 0; i <= last; i++) {
            double m = smask((double)i, a, bb, cx->mask_c, cx->mask_eps);
            if (m <= 0.0) continue;
            int64_t src;
            double v = rd(x, T, t + i, nd, &src);
            double e = exp(sgn * tau * (v - y[t]));
            if (src >= 0) xa[src] += g[t] * m * e;
            ga += g[t] * sgn / tau * smask_da((double)i, a, bb, cx->mask_c, cx->mask_eps) * e;
            gbv += g[t] * sgn / tau * smask_db((double)i, a, bb, cx->mask_c, cx->mask_eps) * e;
          }
        } else {
          int64_t bsrc = -1, src;
          double best = 0.0;
          int have = 0;
          for (int64_t i = 0; i <= last; i++) {
            if (smask((double)i, a, bb, cx->mask_c, cx->mask_eps) <= 0.0) continue;
            double v = rd(x, T, t + i, nd, &src);
            if (!have || sgn * v > sgn * best) { best = v; bsrc = src; have = 1; }
          }
          if (bsrc >= 0) xa[bsrc] += g[t];
        }
      }
      if (gb && nd->slot >= 0) {
        gb[nd->slot * 2 + 0] += ga;
        gb[nd->slot * 2 + 1] += gbv;
      }
    } break;
    case O_UNTIL_SM: {
      const double *ph = wk->val[nd->c0], *ps = wk->val[nd->c1];
      double *pha = wk->adj[nd->c0], *psa = wk->adj[nd->c1];
      double a, bb;
      int64_t last = sm_range(cx, nd, b, &a, &bb);
      double ga = 0.0, gbv = 0.0;
      const double c = cx->mask_c, eps = cx->mask_eps;
      for (int64_t t = 0; t < T; t++) {
        if (g[t] == 0.0) continue;
        int64_t src;
        for (int64_t i = 0; i <= last; i++) wk->tmp2[i] = rd(ph, T, t + i, nd, &src);
        if (!smooth && !soft) {
          /* R5 with the masked offsets: earliest maximising i, P wins ties, earliest argmin */
          double P = INFINITY, best = -INFINITY;
          int64_t Psrc = -1, bsrc = -1;
          int bphi = 0, have = 0;
          for (int64_t i = 0; i <= last; i++) {
            int64_t ks;
            const double v = rd(ph, T, t + i, nd, &ks);
            if (v < P) { P = v; Psrc = ks; }
            if (smask((double)i, a, bb, c, eps) <= 0.0) continue;
            int64_t qs;
            const double q = rd(ps, T, t + i, nd, &qs);
            double z;
            int zphi;
            int64_t zs;
            if (P <= q) { z = P; zphi = 1; zs = Psrc; } else { z = q; zphi = 0; zs = qs; }
            if (!have || z > best) { best = z; bphi = zphi; bsrc = zs; }
            have = 1;
          }
          if (bsrc >= 0) { if (bphi) pha[bsrc] += g[t]; else psa[bsrc] += g[t]; }
          continue;
        }
        /* z_i, their outer weights p_i, then the chain of Until (smooth: as O_UNTIL) */
        int64_t n = 0;
        for (int64_t i = 0; i <= last; i++) {
          const double m = smask((double)i, a, bb, c, eps);
          if (m <= 0.0) continue;
          const double q = rd(ps, T, t + i, nd, &src);
          double z;
          if (soft) {
            const double v2[2] = {swm(wk->tmp2, NULL, i + 1, tau, -1.0, NULL), q};
            z = swm(v2, NULL, 2, tau, -1.0, NULL);
          } else {
            z = smin2(-lse(wk->tmp2, NULL, i + 1, tau, -1.0), q, tau);
          }
          wk->tmp[n] = z;
          wk->tmp3[n] = m;
          wk->itmp[n] = i;
          n++;
        }
        if (n == 0) continue;
        double *pw = wk->tmp3 + (last + 1);   /* outer weights */
        if (soft) swm(wk->tmp, wk->tmp3, n, tau, 1.0, pw);
        for (int64_t r = 0; r < n; r++) {
          const int64_t i = wk->itmp[r];
          const double z = wk->tmp[r], m = wk->tmp3[r];
          double dUz, dUm;
          if (soft) {
            dUz = swm_d(pw[r], z, y[t], tau, 1.0);
            dUm = (pw[r] == 0.0 || isinf(z) || isinf(y[t])) ? 0.0 : pw[r] * (z - y[t]) / m;
          } else {
            const double e = exp(tau * (z - y[t]));
            dUz = m * e;
            dUm = e / tau;
          }
          ga += g[t] * dUm * smask_da((double)i, a, bb, c, eps);
          gbv += g[t] * dUm * smask_db((double)i, a, bb, c, eps);
          if (dUz == 0.0) continue;
          int64_t qs;
          const double q = rd(ps, T, t + i, nd, &qs);
          double Pv, dzP, dzq;
          if (soft) {
            Pv = swm(wk->tmp2, NULL, i + 1, tau, -1.0, NULL);
            double p2[2];
            const double v2[2] = {Pv, q};
            swm(v2, NULL, 2, tau, -1.0, p2);
            dzP = swm_d(p2[0], Pv, z, tau, -1.0);
            dzq = swm_d(p2[1], q, z, tau, -1.0);
          } else {
            Pv = -lse(wk->tmp2, NULL, i + 1, tau, -1.0);
            dzP = isinf(Pv) ? 0.0 : sigm(tau * (q - Pv));
            dzq = isinf(q) ? 0.0 : sigm(tau * (Pv - q));
          }
          if (qs >= 0) psa[qs] += g[t] * dUz * dzq;
          if (dzP == 0.0) continue;
          double *pin = pw + n;   /* inner weights over k <= i */
          if (soft) swm(wk->tmp2, NULL, i + 1, tau, -1.0, pin);
          for (int64_t kk = 0; kk <= i; kk++) {
            int64_t ks;
            const double v = rd(ph, T, t + kk, nd, &ks);
            if (ks < 0 || isinf(v)) continue;
            const double dP = soft ? swm_d(pin[kk], v, Pv, tau, -1.0) : exp(tau * (Pv - v));
            pha[ks] += g[t] * dUz * dzP * dP;
          }
        }
      }
      if (gb && nd->slot >= 0) {
        gb[nd->slot * 2 + 0] += ga;
        gb[nd->slot * 2 + 1] += gbv;
      }
    } break;
  }
}

/* largest scratch length a node can need for trace length T */
static int64_t node_scratch(const octx *cx, int64_t b, int64_t T) {
  int64_t need = 1;
  for (int k = 0; k < cx->n_nodes; k++) {
    const onode *nd = &cx->nodes[k];
    int64_t n = 0;
    if (nd->op == O_EV || nd->op == O_ALW || nd->op == O_UNTIL) {
      int64_t ia, ib;
      int_window(cx, nd, b, T, &ia, &ib);
      n = ib + 1;
    } else if (nd->op == O_EV_SM || nd->op == O_ALW_SM || nd->op == O_UNTIL_SM) {
      double a, bb;
      n = sm_range(cx, nd, b, &a, &bb) + 1;
    }
    if (n > need) need = n;
  }
  return need;
}

static int run_trace(octx *cx, int64_t b) {
  const int64_t r0 = cx->offsets[b], T = cx->offsets[b + 1] - r0;
  if (T <= 0) return 0;
  work wk;
  memset(&wk, 0, sizeof wk);
  if (work_init(&wk, cx->n_nodes, T, node_scratch(cx, b, T) + 1) != 0) { work_free(&wk, cx->n_nodes); return -1; }
  const double *xs = cx->sig + r0 * cx->D;
  /* nodes are stored children-before-parents (post-order) */
  for (int k = 0; k < cx->n_nodes; k++) forward_node(cx, &wk, k, b, xs, T);
  if (!cx->backward) {
    memcpy(cx->out + r0, wk.val[cx->root], (size_t)T * sizeof(double));
  } else {
    memcpy(wk.adj[cx->root], cx->gout + r0, (size_t)T * sizeof(double));
    double *gb = cx->gbounds ? cx->gbounds + (size_t)b * cx->n_slots * 2 : NULL;
    for (int k = cx->n_nodes - 1; k >= 0; k--) backward_node(cx, &wk, k, b, T, gb);
    double *gs = cx->gsig + r0 * cx->D;
    memset(gs, 0, (size_t)T * cx->D * sizeof(double));
    /* d pred / d x_{t,d} = +w_d (GT) or -w_d (LT) for an affine mu;
     * for a norm mu: +-s_d u_d / mu, and 0 at mu = 0 (a subgradient of the norm there) */
    for (int k = 0; k < cx->n_nodes; k++) {
      const onode *nd = &cx->nodes[k];
      const int norm = nd->op == O_NORM_GT || nd->op == O_NORM_LT;
      if (nd->op != O_PRED_GT && nd->op != O_PRED_LT && !norm) continue;
      const double sg = (nd->op == O_PRED_GT || nd->op == O_NORM_GT) ? 1.0 : -1.0;
      for (int64_t t = 0; t < T; t++) {
        if (norm) {
          double u[O_MAX_D];
          const double mu = norm_mu(cx, nd, xs + t * cx->D, u);
          if (mu == 0.0) continue;
          for (int d = 0; d < cx->D; d++)
            gs[t * cx->D + d] += sg * cx->w[nd->w_off + d] * u[d] / mu * wk.adj[k][t];
        } else {
          for (int d = 0; d < cx->D; d++) gs[t * cx->D + d] += sg * cx->w[nd->w_off + d] * wk.adj[k][t];
        }
      }
    }
  }
  work_free(&wk, cx->n_nodes);
  return 0;
}

static void *worker(void *arg) {
  octx *cx = (octx *)arg;
  for (;;) {
    pthread_mutex_lock(&cx->lock);
    int64_t b = cx->next++;
    pthread_mutex_unlock(&cx->lock);
    if (b >= cx->B) break;
    if (run_trace(cx, b) != 0) cx->status = -1;
  }
  return NULL;
}

static int run_all(octx *cx, int n_threads) {
  if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > cx->B) n_threads = (int)(cx->B > 0 ? cx->B : 1);
  pthread_mutex_init(&cx->lock, NULL);
  cx->next = 0;
  cx->status = 0;
  pthread_t *th = calloc((size_t)n_threads, sizeof(pthread_t));
  for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, worker, cx);
  for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
  free(th);
  pthread_mutex_destroy(&cx->lock);
  return cx->status;
}

/* ------------------------------------------------------------------ exported */
int oracle_num_threads(void) { return (int)sysconf(_SC_NPROCESSORS_ONLN); }

/* Robustness trace of the root for B ragged traces (offsets[b]..offsets[b+1]).
   nodes are children-before-parents; out has one double per sample. */
int oracle_forward(const onode *nodes, int n_nodes, int root, const double *w, int D,
                   const double *sig, const int64_t *offsets, int64_t B,
                   const double *bounds, int n_slots, int mode, double tau, double mask_c,
                   double mask_eps, int exact, double *out, int n_threads) {
  if (D < 1 || D > O_MAX_D) return -2;
  octx cx;
  memset(&cx, 0, sizeof cx);
  cx.nodes = nodes; cx.n_nodes = n_nodes; cx.root = root; cx.w = w; cx.D = D;
  cx.sig = sig; cx.offsets = offsets; cx.B = B; cx.bounds = bounds; cx.n_slots = n_slots;
  cx.mode = mode; cx.tau = tau; cx.mask_c = mask_c; cx.mask_eps = mask_eps; cx.exact = exact;
  cx.out = out;
  return run_all(&cx, n_threads);
}

/* Gradient of sum_t grad_out[t] * rho_t with respect to the signal and the per-trace
   bounds (grad_bounds may be NULL; it is accumulated, so the caller zeroes it). */
int oracle_backward(const onode *nodes, int n_nodes, int root, const double *w, int D,
                    const double *sig, const int64_t *offsets, int64_t B,
                    const double *bounds, int n_slots, int mode, double tau, double mask_c,
                    double mask_eps, int exact, const double *grad_out, double *grad_sig,
                    double *grad_bounds, int n_threads) {
  if (D < 1 || D > O_MAX_D) return -2;
  octx cx;
  memset(&cx, 0, sizeof cx);
  cx.nodes = nodes; cx.n_nodes = n_nodes; cx.root = root; cx.w = w; cx.D = D;
  cx.sig = sig; cx.offsets = offsets; cx.B = B; cx.bounds = bounds; cx.n_slots = n_slots;
  cx.mode = mode; cx.tau = tau; cx.mask_c = mask_c; cx.mask_eps = mask_eps; cx.exact = exact;
  cx.backward = 1; cx.gout = grad_out; cx.gsig = grad_sig; cx.gbounds = grad_bounds;
  return run_all(&cx, n_threads);
}
