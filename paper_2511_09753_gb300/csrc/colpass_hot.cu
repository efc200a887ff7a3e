// Column pass instantiations for steady-state passes (steady_pass): FP32
// (mixed path) and FP64 values.
#include "colpass_launch.cuh"

namespace spai {
cudaError_t launch_colpass_hot_f32(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st) {
  return launch_colpass_steady<float, float, kMR, kLOMR, kCGA, kCGB>(p, grid, block, smem, st);
}
cudaError_t launch_colpass_hot_f64(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st) {
  return launch_colpass_steady<double, double, kMR, kLOMR, kCGA, kCGB>(p, grid, block, smem, st);
}
}  // namespace spai
