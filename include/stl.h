/*
 * stl.h -- C ABI of libstl: batched, differentiable Signal Temporal Logic robustness on one
 * GB300 (sm_103a), after STLCG++ (Kapoor, Mizuta, Kang, Leung; arXiv 2501.04194).
 *
 * What is computed.  For every trace b and every sample t the library returns the
 * robustness trace rho(x_t, phi) of a formula phi (Sec. III-D, Definition 1), i.e. the
 * quantitative semantics of Sec. III-B (Eq. "quantitative") applied to the sub-trajectory
 * that starts at t, together with its gradient with respect to the signal and to per-trace
 * interval bounds.  Operators:
 *   predicates     mu(x_t) - c  or  c - mu(x_t), mu(x) = sum_d w_d x_d      (Eq. quantitative)
 *   True           +inf                                                       (Eq. STL grammar)
 *   not / and / or -rho, min, max; smooth mode: logsumexp min / max         (Sec. III-B, III-C)
 *   eventually / always over [a,b]: max / min of the child over t+a..t+b    (Sec. IV-B)
 *   until over [a,b]: max_i min(min_{k<=i} phi_{t+k}, psi_{t+i})            (Sec. IV-C)
 *   eventually_sm / always_sm: the window weighted by the sigmoid mask
 *     m_i = max(sigma(c(i-a)) - sigma(c(i-b)) - eps, 0), entering the logsumexp as a weight,
 *     with gradients to a and b                                             (Sec. VI, Eq. smooth mask)
 * Reads past the end of a trace return the pad (Sec. IV-B Step 1): the last sample
 * (STL_PAD_LAST, its gradient goes to sample T-1) or a constant (STL_PAD_CONST).  Smooth
 * windows count pad reads with multiplicity, as the padded unroll does.  Hard-mode ties:
 * windows select the earliest sample, and/or the left operand, until the earliest maximising
 * offset, then the running minimum over the psi value, then the earliest minimiser.
 *
 * Layout.  Dense signals are float32 [B, T, D], row-major (sample-major inside a trace).
 * Robustness traces and their gradients are float32 [B, T].  Per-trace bounds are float32
 * [B, n_slots, 2] holding (a, b) in time steps.  All array arguments are DEVICE pointers.
 *
 * Ownership and execution.  The caller owns every pointer; the library never allocates or
 * frees device memory on the call path (only stl_set_prepare, which uploads the program
 * table of a formula set, allocates).  Calls are asynchronous on the given cudaStream_t
 * (passed as void*; NULL = the legacy default stream) and fully overwrite their outputs.
 * Argument errors are detected on the host before anything is launched and returned as a
 * negative stl_status; the message is available from stl_last_error() (thread-local).
 * Errors found on the device (per-trace bounds outside the compiled caps) are recorded in a
 * sticky per-device status word read by stl_get_device_status().  Inputs must be finite.
 */
#ifndef STL_H
#define STL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STL_API __attribute__((visibility("default")))
#else
#define STL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  STL_OK = 0,
  STL_ERR_INVALID_ARG = -1,  /* a host-side argument check failed */
  STL_ERR_UNSUPPORTED = -2,  /* valid but outside what the library supports (see message) */
  STL_ERR_CUDA = -3,         /* a CUDA runtime call failed (see message) */
  STL_ERR_WORKSPACE = -4,    /* workspace missing or smaller than stl_workspace_size() */
  STL_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  STL_ERR_DEVICE_CHECK = -6  /* the device found invalid per-trace data (bounds) */
} stl_status;

/* STL_SMOOTH: logsumexp min / max; STL_SOFTMAX: softmax-weighted min / max
 * sum_i v_i e^{+-tau v_i} / sum_i e^{+-tau v_i} over each operator's multiset (Sec. III-C). */
typedef enum { STL_HARD = 0, STL_SMOOTH = 1, STL_SOFTMAX = 2 } stl_mode;

typedef enum {
  STL_OP_PRED_GT = 0,       /* mu(x) - c */
  STL_OP_PRED_LT = 1,       /* c - mu(x) */
  STL_OP_TRUE = 2,          /* +inf */
  STL_OP_NOT = 3,
  STL_OP_AND = 4,
  STL_OP_OR = 5,
  STL_OP_EVENTUALLY = 6,    /* integer window [a, b] */
  STL_OP_ALWAYS = 7,
  STL_OP_UNTIL = 8,         /* child0 U_[a,b] child1 */
  STL_OP_EVENTUALLY_SM = 9, /* sigmoid-masked window, real a < b */
  STL_OP_ALWAYS_SM = 10,
  STL_OP_NORM_GT = 11,      /* ||diag(s)(x - g)||_2 - r: outside a ball (Sec. VII-A regions) */
  STL_OP_NORM_LT = 12,      /* r - ||diag(s)(x - g)||_2: inside it */
  STL_OP_UNTIL_SM = 13      /* child0 U child1 with the sigmoid-masked interval weighting the
                               offsets of the outer max (real a < b; hard: offsets with m > 0) */
} stl_op;

typedef enum { STL_PAD_LAST = 0, STL_PAD_CONST = 1 } stl_pad;

/* One node of a formula.  Nodes are listed children-before-parents; the root is the last
 * node and every other node has exactly one parent (a tree); at most 64 nodes. */
typedef struct {
  int32_t op;          /* stl_op */
  int32_t child0;      /* index of the (first) child, -1 if none */
  int32_t child1;      /* second child of and/or/until, -1 otherwise */
  int32_t bound_slot;  /* -1: the interval is (a, b) below; k >= 0: per-trace bounds[:, k, :],
                          and (a, b) below are the largest values they may take (caps) */
  float a, b;          /* interval in time steps; b = +INFINITY means the whole trace (b = T-1);
                          integers for EVENTUALLY/ALWAYS/UNTIL */
  int32_t pad_mode;    /* stl_pad, for temporal nodes */
  float pad_value;     /* STL_PAD_CONST value */
  int32_t pred_offset; /* predicates: weights are pred_weights[pred_offset .. pred_offset+D);
                          norm predicates: scales s then centre g, 2D entries from here */
  float pred_c;        /* predicates: the constant c (the radius r of a norm predicate) */
} stl_node;

/* Per-call semantics. */
typedef struct {
  int32_t mode;     /* stl_mode */
  float tau;        /* temperature of the smooth modes, > 0 (Sec. III-C) */
  float mask_c;     /* smooth-mask sharpness c, > 0 (Eq. smooth mask) */
  float mask_eps;   /* smooth-mask tolerance epsilon, in (0, 1) */
} stl_params;

/* Which kernel serves a call.
 *   STL_KERNEL_INTERPRETER  the streaming interpreter: one precompiled kernel family that
 *                           reads the compiled formula at run time; serves every call.
 *   STL_KERNEL_COMPILED     a kernel generated for this formula and direction, with every
 *                           node, interval, buffer offset and predicate weight a compile-time
 *                           constant, compiled at run time (NVRTC, sm_103a) on first use and
 *                           kept for the life of the process (first call: about a second).
 *                           Serves hard semantics (STL_HARD) with static integer intervals
 *                           (no bound slot, b finite, b <= 16000), affine predicates, True,
 *                           not / and / or / eventually / always / until, and T at least one
 *                           more than the largest sum of interval starts along a path.  Values
 *                           and gradients are bit-identical to the interpreter's.  Needs no
 *                           workspace and sets no device status.
 *   STL_KERNEL_AUTO         the compiled kernel where it applies, B*T >= 2^20 samples and
 *                           tile, threads and segment are all 0; else the interpreter.
 * Environment (read when a compiled kernel is generated): STL_FK_CHECK=1 generates it with
 * every shared-memory index compared with its buffer's length (an index outside is not
 * performed and sets the device status word to STL_ERR_DEVICE_CHECK; slower, for testing);
 * STL_FK_DUMP=<directory> writes each generated source there.  A compiled backward whose 64-bit
 * adjoint rings would not fit in shared memory beside the node buffers keeps them in the
 * workspace (stl_workspace_size reports the bytes); the compiled forward needs none. */
typedef enum { STL_KERNEL_AUTO = 0, STL_KERNEL_INTERPRETER = 1, STL_KERNEL_COMPILED = 2 } stl_kernel;

/* Launch shape.  Zero fields mean "choose automatically" (the autotuner's cached choice if
 * one was registered with stl_set_launch, else a heuristic). */
typedef struct {
  int32_t tile;      /* samples advanced per streaming step (multiple of 32) */
  int32_t threads;   /* CTA size: 64, 256 or 512 (compiled kernels: 256 or 512) */
  int32_t segment;   /* samples per work item (a trace is split into segments) */
  int32_t kernel;    /* stl_kernel */
} stl_launch;

typedef struct stl_program *stl_handle;
typedef struct stl_program_set *stl_set_handle;

/* Validate and compile a formula (host only; no device allocation).
 *   nodes[n_nodes]      the tree, children first, root last
 *   pred_weights[n_w]   predicate weights (float32), D per predicate
 *   D                   signal dimension (1..16)
 *   n_slots             columns of the per-trace bounds array (0 if unused)
 * Returns STL_ERR_INVALID_ARG for a malformed tree (see stl_last_error()). */
STL_API stl_status stl_compile(const stl_node *nodes, int32_t n_nodes, const float *pred_weights,
                       int32_t n_w, int32_t D, int32_t n_slots, stl_handle *out);

STL_API void stl_destroy(stl_handle h);

/* Override (or, with all-zero fields, reset) the launch shape used for this handle. */
STL_API stl_status stl_set_launch(stl_handle h, const stl_launch *launch);

/* Autotuner: time candidate launch shapes (CTA size x tile) for this handle, call shape and
 * direction on the caller's buffers (backward = 0: out is [B, T]; 1: grad_out [B, T] and
 * out = grad_sig [B, T, D]), keep the fastest in the handle for that direction and return it
 * (best_ms: mean time of the winner, -1 when taken from the cache).  Candidates whose
 * workspace exceeds workspace_bytes are skipped.  If the environment variable
 * STL_TUNE_CACHE names a file, results are looked up there first (key: formula hash, D,
 * slots, semantics, direction, log2 buckets of B and T) and appended after tuning.
 * Synchronous (events + synchronisation): call it before any stream capture.  The outputs
 * hold the result of the last timed launch. */
STL_API stl_status stl_autotune(stl_handle h, const float *sig, int64_t B, int64_t T, const float *bounds,
                                const stl_params *p, int32_t backward, const float *grad_out, float *out,
                                float *grad_bounds, void *workspace, size_t workspace_bytes, void *stream,
                                stl_launch *best, float *best_ms);

/* Launch shape the library would use for this call shape (after heuristics/overrides);
 * out->kernel is STL_KERNEL_INTERPRETER or STL_KERNEL_COMPILED. */
STL_API stl_status stl_get_launch(stl_handle h, int64_t B, int64_t T, const stl_params *p,
                          int32_t backward, stl_launch *out);

/* Generate and compile (NVRTC, sm_103a) the formula-compiled kernel of this handle for one
 * direction and launch shape, without launching it; needs no GPU.  launch: threads (0, 256
 * or 512) and tile (0: the default, else the largest tile up to this one whose buffers fit
 * in shared memory); tile_out / smem_bytes (either may be NULL) receive the tile and dynamic
 * shared memory the kernel uses.  Returns STL_ERR_UNSUPPORTED when the formula is outside
 * what the compiled kernels serve (reason in stl_last_error()) or NVRTC is missing. */
STL_API stl_status stl_compile_kernel(stl_handle h, int32_t backward, int64_t T, const stl_launch *launch,
                                      int32_t *tile_out, int32_t *smem_bytes);

/* Bytes of device workspace that stl_robustness (backward = 0) or stl_robustness_backward
 * (backward = 1) needs for B traces of length T; 0 when everything fits on chip. */
STL_API stl_status stl_workspace_size(stl_handle h, int64_t B, int64_t T, const stl_params *p,
                              int32_t backward, size_t *bytes);

/* Robustness traces.
 *   sig      [B, T, D] float32 device
 *   bounds   [B, n_slots, 2] float32 device, or NULL when the formula uses no slot
 *   out      [B, T] float32 device, overwritten
 *   workspace / workspace_bytes: device scratch of at least stl_workspace_size() bytes
 *   stream   cudaStream_t */
STL_API stl_status stl_robustness(stl_handle h, const float *sig, int64_t B, int64_t T,
                          const float *bounds, const stl_params *p, float *out,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Gradient of sum_{b,t} grad_out[b,t] * rho[b,t] (reverse mode; the forward pass is
 * recomputed on chip, no intermediate traces are stored).
 *   grad_out     [B, T] float32 device
 *   grad_sig     [B, T, D] float32 device, overwritten
 *   grad_bounds  [B, n_slots, 2] float32 device or NULL, overwritten (nonzero only for the
 *                sigmoid-masked operators in smooth mode)
 * Determinism.  STL_HARD and STL_SMOOTH accumulate adjoints in 64-bit fixed point: every
 * contribution is rounded to a multiple of 2^-k (2^-k below 2^-29 of the trace's largest
 * |grad_out|) before any addition, so the sums do not depend on the order of the additions.
 * STL_HARD: grad_sig is bit-identical across calls, launch shapes (stl_set_launch, autotuning),
 * segmentations, stl_robustness_and_backward, the host pipeline and the ragged path.
 * STL_SMOOTH: grad_sig is bit-identical across calls with the same launch shape (other shapes
 * evaluate the window sums in another order).  STL_SOFTMAX, and grad_bounds in the smooth
 * modes: float sums whose order follows warp scheduling, so two calls may differ in the last
 * bits (within float32 summation error). */
STL_API stl_status stl_robustness_backward(stl_handle h, const float *sig, int64_t B, int64_t T,
                                   const float *bounds, const stl_params *p,
                                   const float *grad_out, float *grad_sig, float *grad_bounds,
                                   void *workspace, size_t workspace_bytes, void *stream);

/* Robustness traces and their gradient in ONE launch: rho as stl_robustness (Sec. III-D,
 * the robustness trace) and the gradient of sum grad_out * rho as stl_robustness_backward.
 * The backward pass recomputes every node's trace on chip anyway, so rho costs only its
 * stores.  For callers that know the upstream gradient before the forward values (a loss
 * linear in rho, or a fixed weighting of the trace); a loss that depends on rho itself needs
 * the two separate calls.
 *   out          [B, T] float32 device, overwritten (NULL is rejected)
 *   other arguments, workspace (stl_workspace_size with backward = 1) and errors as
 *   stl_robustness_backward.  Hard-mode rho equals stl_robustness's bit for bit; smooth-mode
 *   rho may differ from it in the last bits when the two launches use different tiles (the
 *   window sums are then combined in a different order). */
STL_API stl_status stl_robustness_and_backward(stl_handle h, const float *sig, int64_t B, int64_t T,
                                               const float *bounds, const stl_params *p,
                                               const float *grad_out, float *out, float *grad_sig,
                                               float *grad_bounds, void *workspace,
                                               size_t workspace_bytes, void *stream);

/* Bytes of the static device scratch behind stl_robustness_backward_noalloc (32 MiB). */
#define STL_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/* Allocation-free backward (the paper has no counterpart; this serves callers that cannot
 * allocate device memory at all while they run -- a host application that forbids device
 * allocation after start-up, a real-time loop with frozen memory, or a plugin whose framework
 * owns every device byte).  Same arguments and results as stl_robustness_backward, without
 * the workspace: the scratch comes from a file-scope static __device__ array of
 * STL_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until exit.
 *   - Every call looks up that array's device address (cudaGetSymbolAddress, with the call's
 *     device current), so the address stays right after a device reset; the first call on a
 *     device may load the library's device code, so make it before any stream capture.
 *   - If the scratch cannot hold what all resident CTAs would need, fewer CTAs are launched
 *     (they walk all work items); if one CTA of the planned size needs more, the call is
 *     planned again with 64-thread CTAs (the smooth Until's per-thread arrays shrink with the
 *     CTA); if even that needs more, it returns STL_ERR_WORKSPACE with a message stating both
 *     sizes.  B = 0 is checked and returns STL_OK without planning.
 *   - Every call shares the one array and leaves its last contents there; the kernels write
 *     each scratch word before reading it.  Calls whose kernels overlap on the GPU (different
 *     streams, no ordering) race on the array and give undefined results: serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
STL_API stl_status stl_robustness_backward_noalloc(stl_handle h, const float *sig, int64_t B, int64_t T,
                                                   const float *bounds, const stl_params *p,
                                                   const float *grad_out, float *grad_sig,
                                                   float *grad_bounds, void *stream);

/* ---- Host buffers: copies overlapped with compute ----
 * Forward and/or backward of B traces whose signal, bounds, grad_out and outputs live in HOST
 * memory (page-locked for the copies to overlap), processed in chunks of `chunk` traces on
 * three helper streams owned by the handle: while one chunk is computed, the next chunks'
 * inputs are copied in and earlier chunks' outputs copied out.  staging: a DEVICE buffer of
 * stl_pipeline_staging_size() bytes (three slots of signal, bounds, grad_out, outputs and
 * workspace for one chunk).  out (may be NULL) receives rho [B, T]; with grad_out non-NULL the
 * backward runs and grad_sig (required) / grad_bounds (may be NULL) receive the gradients.  The
 * call orders itself after the work already queued on `stream`, and `stream` waits for all of
 * it: the results are in host memory once `stream` reaches the call's end.  The helper streams
 * and events are created on the first call (the only resources the library creates on a call
 * path).  Same semantics and errors as stl_robustness / stl_robustness_backward; calls on one
 * handle must not overlap. */
STL_API stl_status stl_pipeline_staging_size(stl_handle h, int64_t chunk, int64_t T, const stl_params *p,
                                             int32_t backward, size_t *bytes);
STL_API stl_status stl_robustness_host_pipelined(stl_handle h, const float *sig, int64_t B, int64_t T,
                                                 const float *bounds, const stl_params *p, const float *grad_out,
                                                 float *out, float *grad_sig, float *grad_bounds, int64_t chunk,
                                                 void *staging, size_t staging_bytes, void *stream);

/* ---- Ragged batches: many traces of different lengths and formulas in one launch ----
 * Traces are packed one after another: trace i has offsets[i+1] - offsets[i] samples starting
 * at row offsets[i] of sig [sum T, D]; outputs are packed the same way.  formula_id[i] selects
 * the formula of trace i in the set; order (optional, may be NULL) lists the traces in the
 * order CTAs take them from a shared work counter (longest first balances the tail).
 * Interval semantics per trace as in stl_robustness (Sec. IV-E: intervals are data). */

/* Group compiled formulas (same D; 1 <= n_formulas <= 65536) for ragged launches.  The set
 * refers to the handles, which must outlive it.  stl_set_prepare copies every formula's programs
 * into one device table (about 10 KB per program), allocated on the first prepare. */
STL_API stl_status stl_set_create(const stl_handle *formulas, int32_t n_formulas, stl_set_handle *out);
STL_API void stl_set_destroy(stl_set_handle s);

/* Prepare the set for up to n_traces traces of at most T_max samples with semantics p, for
 * the forward (backward = 0) or backward (1) launch: plans every formula for length buckets
 * T_max, T_max/2, T_max/4, ... (down to 1024 samples, at most 6 and at most 8192 programs in
 * all) and uploads the program table to the device (the only allocation of the ragged path,
 * freed by stl_set_destroy).  Each trace runs the plan of the smallest bucket that holds it.
 * Returns the workspace size the matching ragged calls need.  Host-side, synchronous; call it
 * before any stream capture. */
STL_API stl_status stl_set_prepare(stl_set_handle s, int64_t n_traces, int64_t T_max, const stl_params *p,
                                   int32_t backward, size_t *workspace_bytes);

/* Robustness of a ragged batch in ONE launch (capturable in a CUDA graph: no allocation, no
 * synchronisation).  p must equal the prepared params.  Device arrays:
 *   sig [sum T, D], offsets int64 [n_traces+1], formula_id int32 [n_traces],
 *   order int32 [n_traces] or NULL, bounds [n_traces, n_slots, 2] or NULL, out [sum T].
 * Traces with a formula_id outside the set, an order entry out of range or more than T_max
 * samples are skipped and set the device status word (stl_get_device_status). */
STL_API stl_status stl_robustness_ragged(stl_set_handle s, const float *sig, const int64_t *offsets,
                                         const int32_t *formula_id, const int32_t *order, int64_t n_traces,
                                         const float *bounds, int32_t n_slots, const stl_params *p, float *out,
                                         void *workspace, size_t workspace_bytes, void *stream);

/* Gradient of sum(grad_out * rho) for a ragged batch (grad_out [sum T], grad_sig [sum T, D],
 * grad_bounds [n_traces, n_slots, 2] or NULL), one launch, same rules as above. */
STL_API stl_status stl_robustness_ragged_backward(stl_set_handle s, const float *sig, const int64_t *offsets,
                                                  const int32_t *formula_id, const int32_t *order,
                                                  int64_t n_traces, const float *bounds, int32_t n_slots,
                                                  const stl_params *p, const float *grad_out, float *grad_sig,
                                                  float *grad_bounds, void *workspace, size_t workspace_bytes,
                                                  void *stream);

/* Launch shape of a formula set for one direction (threads 64 / 256 / 512 and tile, a multiple
 * of 32; zero fields: the planner's choice), used from the next stl_set_prepare on. */
STL_API stl_status stl_set_set_launch(stl_set_handle s, int32_t backward, const stl_launch *launch);

/* Autotuner of a formula set (the paper's static-graph batching, Sec. IV-E, over uneven
 * traces): times candidate launch shapes -- CTA size 64 / 256 / 512 (64 only for T_max <= 8192)
 * x tile 4, 7 or 14 samples per thread; the tile is the chunk of samples each streaming step
 * advances, i.e. how long windows are cut into shared-memory chunks -- on the caller's ragged
 * batch for one direction (backward = 0: out is rho [sum T]; 1: grad_out [sum T] and out =
 * grad_sig [sum T, D]), keeps the fastest in the set and leaves the set prepared with it
 * (as stl_set_prepare, whose workspace size it returns in *workspace_bytes).  Each candidate
 * runs in a temporary workspace that the call allocates and frees: a setup call, synchronous,
 * to be made before any stream capture.  STL_TUNE_CACHE (see stl_autotune) caches the result
 * under a key of the set's formulas, D, slots, semantics, direction and the log2 buckets of
 * n_traces and T_max.  best_ms: mean time of the winner (-1 when taken from the cache). */
STL_API stl_status stl_set_autotune(stl_set_handle s, int64_t n_traces, int64_t T_max, const stl_params *p,
                                    int32_t backward, const float *sig, const int64_t *offsets,
                                    const int32_t *formula_id, const int32_t *order, const float *bounds,
                                    int32_t n_slots, const float *grad_out, float *out, float *grad_bounds,
                                    void *stream, stl_launch *best, float *best_ms, size_t *workspace_bytes);

/* Sticky device-side status of the current device: STL_OK, STL_ERR_DEVICE_CHECK (invalid
 * per-trace data) or STL_ERR_TIMEOUT (a bounded device-side wait gave up, e.g. in the tensor-core
 * GEMM of stl_plan.h); synchronises `stream`, then reads and clears the word. */
STL_API stl_status stl_get_device_status(void *stream, int32_t *status);

STL_API const char *stl_status_string(int32_t status);
STL_API const char *stl_last_error(void);

/* Library version string. */
STL_API const char *stl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STL_H */
