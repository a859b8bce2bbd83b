// One instantiation of the interpreter: 128 threads, forward, hard semantics
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(128, false, false, 128_fh)
