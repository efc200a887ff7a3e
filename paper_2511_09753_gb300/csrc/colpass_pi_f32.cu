// Column pass instantiation: Pi-preconditioned forms (Algorithms 5, 7, 8 with
// Pi = diag(A)^{-1}), FP32 values (mixed path).
#include "colpass_launch.cuh"

namespace spai {
cudaError_t launch_colpass_pi_f32(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st) {
  return launch_colpass<float, float, true, kMR, kLOMR, kCGA, kCGB>(p, grid, block, smem, st);
}
}  // namespace spai
