// One instantiation of the interpreter: 64 threads, backward, hard semantics, ragged (device program table)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(64, true, false, true, 64_bh_r)
