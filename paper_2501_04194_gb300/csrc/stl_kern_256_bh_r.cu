// One instantiation of the interpreter: 256 threads, backward, hard semantics, ragged (device program table)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(256, true, false, true, 256_bh_r)
