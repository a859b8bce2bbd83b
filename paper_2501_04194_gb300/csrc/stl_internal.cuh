// Internal program description of libstl, shared by the host-side compiler (stl_capi.cu)
// and the device interpreter (stl_kernels.cu).  A compiled formula is passed BY VALUE as a
// __grid_constant__ kernel parameter, so a launch needs no device allocation for it.
#pragma once
#include <cstddef>
#include <cstdint>

#define STL_MAX_NODES 64
#define STL_MAX_WEIGHTS 256
#define STL_MAX_D 16
#define STL_MAX_PRED 32
#define STL_LEAN_MIN_SAMPLES 4096   // hard forward node steps this long take the direct-read passes
#define STL_BUF_BACK 16    // words after every node buffer of such plans (unclamped over-reads)
#define STL_MAX_BUCKETS 6  // ragged sets: length buckets (plans) per formula

// Node layout after compilation (per launch: the ring geometry depends on tile and bounds).
struct KNode {
  int op, c0, c1, slot, parent;
  float a, b;          // static interval, or the caps of a per-trace slot (b may be +inf)
  int pad_const;       // 0: reads past T-1 repeat the last sample; 1: constant pad_value
  float pad_value;
  int w_off;           // predicate weights offset into KProgram::w
  float pc;            // predicate constant
  int lo, hi;          // live offsets relative to the root step [t0, t1): [t0+lo, t1+hi)
  int cap;             // buffer length in samples (>= tile + hi - lo, multiple of 4)
  int val_off;         // word offsets of the buffers (shared arena or per-CTA global slice)
  int adj_off;         // -1 if the node keeps no adjoint buffer (hard backward: 2 words per
                       // sample, a 64-bit fixed-point accumulator; smooth: 1 float)
  int aux_off;         // -1 if the node keeps no selected-source buffer
  int space;           // 0: shared memory, 1: global workspace
  int tab_off;         // smooth-mask weight tables (3 x tab_len words in shared memory), -1 if none
  int tab_len;
};

struct KProgram {
  int n;               // nodes, children first, root = n-1
  int D;
  int n_slots;
  int mode;            // 0 hard, 1 smooth
  float tau, inv_tau, mask_c, mask_eps;
  int bwd;             // 1: backward launch
  int tile;            // samples per streaming step
  int seg;             // samples per work item
  int segs_per_trace;
  long long n_items;
  long long T;         // samples per trace
  long long B;
  int hmax;            // max hi over nodes (backward warm-up)
  int lp;              // common adjoint offset of the predicates
  int smem_words;      // dynamic shared memory words: buffers + scratch + node table
  int scratch_off;     // word offset of the window scratch in shared memory
  int scratch_words;
  int rt_off;          // word offset of the per-node runtime table
  int gwords;          // global buffer words per CTA
  long long ut_off;    // word offset of the smooth-until per-thread arrays in the workspace
  int ut_len;          // their length (max taps)
  int win_r;           // samples per thread-run of the largest windows (15)
  int lean;            // 1: buffers carry STL_BUF_BACK words of slack, direct-read passes allowed
  int npred;           // predicate nodes
  unsigned norm_mask;  // bit k: predicate k is a norm predicate (its pw row is zero)
  int pred[STL_MAX_PRED];
  float pw[STL_MAX_PRED * STL_MAX_D];   // +w (mu - c) or -w (c - mu) per affine predicate
  float w[STL_MAX_WEIGHTS];
  KNode nd[STL_MAX_NODES];
};

// Per-node runtime state, one per node in shared memory.
struct NodeRt {
  float *val;
  float *adj;
  int *aux;
  int ia, ib;          // integer window (or smooth-mask support) for this trace
  float fa, fb;        // smooth-mask real bounds for this trace
  int lo, hi, cap;
  int base;            // unused
  float lastval;       // value at sample T-1 (pad reads)
  int lastaux;         // recorded source at sample T-1
  float padadj;        // adjoint accumulated for sample T-1
  unsigned long long padfx;   // hard backward: the same as a 64-bit fixed-point sum
  float ga, gb;        // smooth-mask bound-gradient accumulators
  float *tab;          // smooth-mask tables: m_i, dm_i/da, dm_i/db for i in [ia, ib]
  int band_a, band_b;  // bound gradients use offsets [ia, band_a] and [band_b, ib]
  int ja, jb;          // smooth mask: the plateau offsets whose weight is exactly fl(1 - eps)
                       // (ja > jb: none); the rest of [ia, ib] are the two edge bands
  int op, c0, c1;      // copies of the node's operator and children (selection walk)
  int pred_k;          // index in the predicate list, or -1
};

// Host-side launch entry points (stl_kernels.cu).
struct LaunchArgs {
  const float *sig;
  const float *bounds;
  const float *gout;
  float *out;
  float *gsig;
  float *gbounds;
  float *ws;
  int *status;         // device status word (sticky error flag)
  // ragged launches (table != nullptr): per-trace programs and packed traces
  const KProgram *table;        // device table of programs, one per formula
  const long long *offsets;     // [n_traces + 1] first sample row of each trace
  const int *fid;               // [n_traces] formula of each trace
  const int *order;             // [n_traces] processing order, or nullptr
  unsigned long long *counter;  // work counter (zeroed before the launch)
  long long n_traces;
  int n_formulas;
  long long T_max;              // longest trace the table was prepared for
  int n_buckets;                // programs per formula: planned for T_max >> 0, 1, ...
  int gwords;                   // global buffer words per CTA (max over formulas)
  int ut_len;
  long long ut_off;
  int grid;
  int threads;
  void *stream;
};
int stl_launch_main(const KProgram &P, const LaunchArgs &A);   // returns a cudaError_t
int stl_max_smem_optin(int *bytes);
int stl_blocks_per_sm(int threads, int bwd, int smooth, int ragged, int smem_bytes, int *blocks);
int stl_num_sms(int *sms);
int stl_read_clear_status(void *stream, int *status);
int stl_status_ptr(int **ptr);
