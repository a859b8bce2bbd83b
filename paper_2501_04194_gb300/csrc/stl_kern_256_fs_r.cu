// One instantiation of the interpreter: 256 threads, forward, smooth semantics, ragged (device program table)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(256, false, true, true, 256_fs_r)
