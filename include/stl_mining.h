/*
 * stl_mining.h -- C ABI of the time-interval mining helpers of libstl (Sec. VI and the
 * specification-mining example of Sec. VII-C): gradient descent on the interval [aT, bT] of a
 * smooth-masked formula over a dataset of N traces of T samples, with
 *
 *   loss(a, b) = (1/N) sum_n max(-rho_n(0), 0) + gamma (a - b),   a = sigmoid(alpha), b = sigmoid(beta),
 *
 * where rho_n(0) is the robustness at t = 0 of trace n under the per-trace bounds
 * (aT, bT) (all traces share them).  One descent step is: stl_robustness (rho), then
 * stl_mining_seed (grad_out and the loss), then stl_robustness_backward (per-trace bound
 * gradients), then stl_mining_update (new alpha, beta and bounds).  All array arguments are
 * DEVICE pointers owned by the caller; calls are asynchronous on the stream, allocate nothing,
 * and return a negative stl_status on a failed host-side argument check.  No counterpart in
 * the paper's code.
 */
#ifndef STL_MINING_H
#define STL_MINING_H

#include <stdint.h>

#include "stl.h"

#ifdef __cplusplus
extern "C" {
#endif

/* grad_out[n, 0] = -1/N where rho[n, 0] < 0, else 0 (the rest of grad_out [N, T] is not
 * touched); (1/N) sum_n max(-rho[n, 0], 0) is added to *loss (device float, may be NULL). */
STL_API stl_status stl_mining_seed(const float *rho, int64_t N, int32_t T, float *grad_out, float *loss,
                                   void *stream);

/* One gradient step on theta = (alpha, beta) (device float [2]) with step size lr:
 *   dL/dalpha = (T sum_n gbounds[n, slot, 0] + gamma) a (1 - a),
 *   dL/dbeta  = (T sum_n gbounds[n, slot, 1] - gamma) b (1 - b),
 * then bounds[n, slot, :] = (T sigmoid(alpha), T sigmoid(beta)) for every n.  gbounds and
 * bounds are float32 [N, n_slots, 2]; one CTA reduces over the N traces in a fixed order. */
STL_API stl_status stl_mining_update(float *theta, const float *gbounds, int64_t N, int32_t n_slots, int32_t slot,
                                     int32_t T, float lr, float gamma, float *bounds, void *stream);

/* Per-trace interval descent (the parameter-mining descent with one learnable interval per
 * trace, Sec. VI): every trace n takes one gradient step on its own bounds (a_n, b_n), in steps,
 * for the loss  max(-rho_n(0), 0) - gamma (b_n - a_n):
 *   a_n -= lr (scale gbounds[n, slot, 0] + gamma),  b_n -= lr (scale gbounds[n, slot, 1] - gamma),
 * then 0 <= a_n <= a_cap, a_n + min_width <= b_n <= b_cap.  scale undoes the 1/N of
 * stl_mining_seed (scale = N).  bounds, gbounds: float32 [N, n_slots, 2]. */
STL_API stl_status stl_mining_update_traces(float *bounds, const float *gbounds, int64_t N, int32_t n_slots,
                                            int32_t slot, float lr, float gamma, float scale, float a_cap,
                                            float b_cap, float min_width, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* STL_MINING_H */
