// One instantiation of the interpreter: 512 threads, forward, smooth semantics, ragged (device program table)
// (one translation unit per variant so that the variants compile in parallel).
#include "stl_interp.cuh"

STL_DEFINE_VARIANT(512, false, true, true, 512_fs_r)
