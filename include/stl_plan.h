/*
 * stl_plan.h -- C ABI of the trajectory-optimisation helpers of libstl: the batched
 * gradient-through-robustness planner and the small BF16 MLP that predicts its warm start.
 *
 * The planning problem follows the paper's trajectory-planning use (Sec. VII-A): controls u are
 * optimised by gradient steps on the smooth robustness of a reach/avoid specification of the
 * resulting trajectory, and a problem counts as solved once the hard robustness at t = 0 is
 * >= 0.  The dynamics are the 2-D single integrator with saturated controls,
 * x_{t+1} = x_t + dt tanh(u_t) from x_0 = 0; a trace holds x_1 .. x_T.  The robustness itself
 * comes from the ragged calls of stl.h (one formula per problem).
 *
 * All array arguments are DEVICE pointers owned by the caller; every call is asynchronous on
 * the given stream (void* = cudaStream_t), allocates nothing and returns a negative stl_status
 * (message in stl_last_error()) when an argument check fails on the host.  bf16 arrays are
 * passed as uint16_t (the bit pattern of IEEE bfloat16).  No counterpart in the paper's code:
 * these are the building blocks of the learned warm start.
 */
#ifndef STL_PLAN_H
#define STL_PLAN_H

#include <stdint.h>

#include "stl.h"

#ifdef __cplusplus
extern "C" {
#endif

/* x[b, t, :] = x_{t+1} = sum_{s <= t} dt * tanh(u[b, s, :]), for u, x float32 [B, T, 2].
 * One warp per problem; T in [1, 65536]. */
STL_API stl_status stl_rollout(const float *u, int64_t B, int32_t T, float dt, float *x, void *stream);

/* One Adam step on the controls of every active problem, through the rollout adjoint:
 *   ubar_t = dt (1 - tanh^2 u_t) sum_{s >= t} xbar_s          (xbar = dLoss/dx, [B, T, 2])
 *   m = b1 m + (1-b1) ubar;  v = b2 v + (1-b2) ubar^2;
 *   u -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 * then x is recomputed from the new u (as stl_rollout).  Problems with active[b] == 0 are left
 * untouched (u, m, v and x).  step >= 1.  u, m, v, x: float32 [B, T, 2]; active: int32 [B]. */
STL_API stl_status stl_plan_adam_step(float *u, float *m, float *v, const float *xbar, const int32_t *active,
                                      int64_t B, int32_t T, float dt, float lr, float beta1, float beta2,
                                      float eps, int32_t step, float *x, void *stream);

/* Bookkeeping after a hard-robustness launch on the current trajectories (rho_hard [B, T]):
 * every active problem with rho_hard[b, 0] >= 0 gets solved_iter[b] = iter and active[b] = 0.
 * Then grad_out[b, 0] = -1 for the problems still active and 0 for the others (the rest of
 * grad_out [B, T] is not touched): a backward with this grad_out gives xbar = -d rho_0 / dx,
 * so the next stl_plan_adam_step ascends the robustness at t = 0.  The number of problems still
 * active after the call is added to *n_active (device int32, may be NULL). */
STL_API stl_status stl_plan_check(const float *rho_hard, int32_t *active, int32_t *solved_iter, int32_t iter,
                                  float *grad_out, int64_t B, int32_t T, int32_t *n_active, void *stream);

/* ---- Trajectory optimisation with a learnable time interval (Sec. VII-A) ----
 * Problems b = 0..B-1, each with controls u [T, 2] of the single integrator
 * x_{t+1} = x_t + dt u_t from x_0 = start (trace x_1..x_T) and an interval (a, b) =
 * (sigmoid(alpha), sigmoid(beta)) of a sigmoid-masked operator whose per-trace bounds (aT, bT)
 * live in bounds[b, slot, :] (n_slots columns), minimise
 *   J = g1 max(-rho_0, 0) + g2 exp(2 (I_nom - b + a)) + g3 (1/T) sum_t max(|u_t| - u_max, 0)
 *       + g4 (1/T) sum_t |u_t|^2
 * with per-problem coefficients gam[b, 0..3] = (g1, g2, g3, g4).
 *
 * stl_trajopt_seed: grad_out[b, 0] = -g1 where rho[b, 0] < 0, else 0 (the rest of grad_out
 * [B, T] is not touched).
 * stl_trajopt_step: one Adam step on u (with xbar = dJ/dx [B, T, 2] from the robustness
 * backward: ubar_t = dt sum_{s >= t} xbar_s + the two control terms) and on theta [B, 2] =
 * (alpha, beta) (with the per-trace bound gradients gbounds [B, n_slots, 2] of the robustness
 * backward and the interval term), then the new trajectory x and bounds[b, slot, :].
 * mu, vu: Adam moments of u [B, T, 2]; mth, vth: of theta [B, 2].  step >= 1 (Adam with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8).  The update keeps a <= b - 1e-3. */
STL_API stl_status stl_trajopt_seed(const float *rho, const float *gam, int64_t B, int32_t T, float *grad_out,
                                    void *stream);
STL_API stl_status stl_trajopt_step(float *u, float *mu, float *vu, float *theta, float *mth, float *vth,
                                    const float *xbar, const float *gbounds, const float *gam, int64_t B, int32_t T,
                                    int32_t n_slots, int32_t slot, float dt, float start_x, float start_y,
                                    float u_max, float i_nom, float lr_u, float lr_theta, int32_t step, float *x,
                                    float *bounds, void *stream);

/* ---- BF16 matrix products and the pieces of an MLP training step ----
 * C[M, N] = op(A) op(B) (+ bias[N]) (then max(., 0) when relu), BF16 products accumulated in
 * FP32 on the 5th-generation tensor cores (tcgen05.mma kind::f16, the accumulator in tensor
 * memory, 128 x 128 tiles, one CTA each).  op(A) is A [M, K] (lda >= K) or, with trans_a, A^T for
 * A [K, M] (lda >= M); op(B) is B [K, N] (ldb >= N) or, with trans_b, B^T for B [N, K]
 * (ldb >= K); all row-major.  c_f32 and/or c_bf16 [M, N] (ldc >= N) receive the result; either
 * may be NULL, not both.  bias may be NULL.  M, N, K in [1, 2^20]. */
STL_API stl_status stl_gemm_bf16(const uint16_t *a, int32_t lda, int32_t trans_a, const uint16_t *b, int32_t ldb,
                                 int32_t trans_b, int32_t M, int32_t N, int32_t K, const float *bias, int32_t relu,
                                 float *c_f32, uint16_t *c_bf16, int32_t ldc, void *stream);

/* Mean-squared-error gradient: dz = scale (z - y) as bf16 (z, y float32 [n]); the sum of
 * (z - y)^2 over the n entries is added to *loss (device float, may be NULL). */
STL_API stl_status stl_mse_grad(const float *z, const float *y, int64_t n, float scale, uint16_t *dz,
                                float *loss, void *stream);

/* Backward of max(., 0): dz = (act > 0) ? da : 0 as bf16, for da float32 [n] and the
 * post-activation act bf16 [n]. */
STL_API stl_status stl_relu_backward(const float *da, const uint16_t *act, int64_t n, uint16_t *dz, void *stream);

/* Column sums of a bf16 matrix dz [M, N] (row-major): db[n] = sum_m dz[m, n] (float32, overwritten). */
STL_API stl_status stl_colsum_bf16(const uint16_t *dz, int32_t M, int32_t N, float *db, void *stream);

/* Adam on float32 parameters p [n] with gradient g and moments m, v (same update as
 * stl_plan_adam_step, no rollout); p_bf16 (may be NULL) receives the updated parameters
 * rounded to bf16. */
STL_API stl_status stl_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                            float beta2, float eps, int32_t step, uint16_t *p_bf16, void *stream);

/* Round float32 [n] to bf16 (round to nearest even). */
STL_API stl_status stl_to_bf16(const float *x, int64_t n, uint16_t *y, void *stream);

/* Row gather: dst[i, :] = src[idx[i], :] for float32 rows of `cols` entries, i < n_rows, from a
 * source of n_src rows; an index outside [0, n_src) yields a zero row. */
STL_API stl_status stl_gather_rows(const float *src, int64_t n_src, const int64_t *idx, int64_t n_rows, int32_t cols,
                                   float *dst, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* STL_PLAN_H */
