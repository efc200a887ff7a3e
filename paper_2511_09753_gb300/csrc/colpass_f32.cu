// Column pass instantiation: FP32 values (mixed path).
#include "colpass_launch.cuh"

namespace spai {
cudaError_t launch_colpass_f32(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  return launch_colpass<float, float, false, kMR, kLOMR, kCGA, kCGB, kRES, kSCORE>(p, grid, block,
                                                                              smem, st);
}
}  // namespace spai
