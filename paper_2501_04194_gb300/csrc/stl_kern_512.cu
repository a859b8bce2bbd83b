// One CTA-size instantiation of the interpreter (separate translation unit so that the
// three sizes compile in parallel).
#include "stl_interp.cuh"

int stl_launch_nt512(const KProgram &P, const LaunchArgs &A) {
  const size_t smem = (size_t)P.smem_words * 4;
  cudaError_t e = cudaFuncSetAttribute(stl_main<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  stl_main<512><<<A.grid, 512, smem, (cudaStream_t)A.stream>>>(P, A);
  return (int)cudaGetLastError();
}

int stl_occupancy_nt512(int smem_bytes, int *blocks) {
  cudaError_t e = cudaFuncSetAttribute(stl_main<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, stl_main<512>, 512, smem_bytes);
}
