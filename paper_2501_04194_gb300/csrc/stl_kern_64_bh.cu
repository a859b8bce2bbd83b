// One instantiation of the interpreter: 64 threads, backward, hard semantics, dense (program by value)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(64, true, false, false, 64_bh)
