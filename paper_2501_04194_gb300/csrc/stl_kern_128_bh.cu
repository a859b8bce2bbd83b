// One instantiation of the interpreter: 128 threads, backward, hard semantics
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(128, true, false, 128_bh)
