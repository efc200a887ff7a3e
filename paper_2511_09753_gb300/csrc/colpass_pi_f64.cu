// Column pass instantiation: Pi-preconditioned forms (Algorithms 5, 7, 8 with
// Pi = diag(A)^{-1}), FP64 values.
#include "colpass_launch.cuh"

namespace spai {
cudaError_t launch_colpass_pi_f64(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st) {
  return launch_colpass<double, double, true, kMR, kLOMR, kCGA, kCGB>(p, grid, block, smem, st);
}
}  // namespace spai
