// One instantiation of the interpreter: 512 threads, backward, smooth semantics, ragged (device program table)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(512, true, true, true, 512_bs_r)
