// Column pass instantiations: FP64 values, and the FP64 residual norm of an
// FP32-valued M.
#include "colpass_launch.cuh"

namespace spai {
cudaError_t launch_colpass_f64(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  return launch_colpass<double, double, false, kMR, kLOMR, kCGA, kCGB, kRES, kSCORE>(
      p, grid, block, smem, st);
}
cudaError_t launch_colpass_res_f32(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st) {
  return launch_colpass<float, double, false, kRES>(p, grid, block, smem, st);
}
}  // namespace spai
