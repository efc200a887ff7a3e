// Launch wrapper for one instantiation of the column pass.
#pragma once
#include "colpass.cuh"

namespace spai {

template <typename VS, typename VC, bool PI = false>
cudaError_t launch_colpass(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  static size_t attr_smem = 0;
  if (!attr_set || smem > attr_smem) {
    cudaError_t e = cudaFuncSetAttribute(colpass_kernel<VS, VC, PI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
    attr_smem = smem;
  }
  colpass_kernel<VS, VC, PI><<<grid, block, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace spai
