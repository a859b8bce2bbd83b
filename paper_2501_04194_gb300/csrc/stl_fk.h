// stl_fk.h -- host interface of the formula-compiled kernels (stl_fk.cu), used by stl_capi.cu.
#pragma once
#include <string>
#include <vector>

#include "../../include/stl.h"

// The formula, as stl_compile stored it.
struct FkFormula {
  const std::vector<stl_node> *nodes;
  const std::vector<float> *w;
  int D;
  int n_slots;
};

// A call the compiled kernels can serve: hard semantics, static integer intervals with no
// per-trace bounds slot and a finite b, affine predicates, every node's nearest sample
// (sum of a along its path) inside the shortest segment, and selected offsets that fit 16 bits.
bool stl_fk_eligible(const FkFormula &f, const stl_params &p, long long T, std::string *why);

// Whether NVRTC could be loaded (the compiled kernels are generated at run time).
bool stl_fk_available(std::string *why);

struct FkCall {
  bool bwd = false;
  long long B = 0, T = 0;
  const float *sig = nullptr;
  const float *gout = nullptr;   // backward: upstream gradient [B, T]
  float *out = nullptr;          // robustness [B, T] (forward; optional in backward launches)
  float *gsig = nullptr;         // backward: signal gradient [B, T, D]
  int threads = 0, tile = 0, segment = 0;   // 0: automatic
  void *ws = nullptr;            // workspace (backward with adjoint rings in L2)
  size_t ws_bytes = 0;
  void *stream = nullptr;
};

// Plan the call, generate and compile its kernel (cached per shape) and launch it.  On
// failure returns a status and sets *err.
stl_status stl_fk_run(const FkFormula &f, const FkCall &c, std::string *err);

// The tile, shared memory and workspace bytes the compiled kernel of this shape would use (no
// code generation).
stl_status stl_fk_plan_shape(const FkFormula &f, bool bwd, int threads, int tile, int *tile_out, int *smem_out,
                             size_t *ws_out, std::string *err);

// Plan and compile without launching (no GPU needed): the launch shape the call would use and,
// if src is non-NULL, the generated source.
stl_status stl_fk_compile_only(const FkFormula &f, bool bwd, long long T, int threads, int tile, int *tile_out,
                               int *smem_out, std::string *src, std::string *err);
