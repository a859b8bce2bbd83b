// One instantiation of the interpreter: 128 threads, forward, smooth semantics
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(128, false, true, 128_fs)
