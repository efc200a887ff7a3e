// Column pass instantiation: FP32 values (mixed path).
#include "colpass_launch.cuh"

namespace spai {
cudaError_t launch_colpass_f32(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  return launch_colpass<float, float, false, kMR, kLOMR, kCGA, kCGB, kRES, kSCORE>(p, grid, block,
                                                                              smem, st);
}
}  // namespace spai

#ifdef SPAI_PHASE_CLOCKS
// Profiling build only (libspai_phase.so): copies the per-phase cycle sums of
// the FP32 column-pass kernels, 8 pass kinds x 16 counters (see kPh* in
// colpass.cuh), to the host buffer out, then clears them when reset != 0.
extern "C" int spai_phase_clocks(unsigned long long* out, int reset) {
  if (!out) return -1;
  if (cudaMemcpyFromSymbol(out, spai::g_phase_clk, sizeof(spai::g_phase_clk)) != cudaSuccess)
    return -4;
  if (reset) {
    static const unsigned long long zero[8 * 16] = {};
    if (cudaMemcpyToSymbol(spai::g_phase_clk, zero, sizeof(zero)) != cudaSuccess) return -4;
  }
  return 0;
}
#endif
