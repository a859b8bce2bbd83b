// One instantiation of the interpreter: 64 threads, backward, smooth semantics, dense (program by value)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(64, true, true, false, 64_bs)
