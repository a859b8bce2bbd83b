// One instantiation of the interpreter: 64 threads, backward, smooth semantics, ragged (device program table)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(64, true, true, true, 64_bs_r)
