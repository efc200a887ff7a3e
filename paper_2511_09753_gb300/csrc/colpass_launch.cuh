// Launch wrappers for the column pass: one kernel per (value types, Pi form,
// pass kind); the kinds a wrapper was instantiated with are its template
// arguments, and any other kind is refused with cudaErrorInvalidValue.
#pragma once
#include "colpass.cuh"

namespace spai {

template <typename VS, typename VC, bool PI, int KIND, bool HOT = false>
cudaError_t launch_colpass_kind(const PassParams& p, int grid, int block, size_t smem,
                                cudaStream_t st) {
  static bool attr_set = false;
  static size_t attr_smem = 0;
  if (!attr_set || smem > attr_smem) {
    cudaError_t e = cudaFuncSetAttribute(colpass_kernel<VS, VC, PI, KIND, HOT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
    attr_smem = smem;
  }
  colpass_kernel<VS, VC, PI, KIND, HOT><<<grid, block, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename VS, typename VC, bool PI, int... KINDS>
cudaError_t launch_colpass(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
  ((p.kind == KINDS ? (void)(e = launch_colpass_kind<VS, VC, PI, KINDS>(p, grid, block, smem, st))
                    : (void)0),
   ...);
  return e;
}

// The steady-state kernels (steady_pass(p) must hold).
template <typename VS, typename VC, int... KINDS>
cudaError_t launch_colpass_steady(const PassParams& p, int grid, int block, size_t smem,
                                  cudaStream_t st) {
  if (!steady_pass(p)) return cudaErrorInvalidValue;
  cudaError_t e = cudaErrorInvalidValue;
  ((p.kind == KINDS
        ? (void)(e = launch_colpass_kind<VS, VC, false, KINDS, true>(p, grid, block, smem, st))
        : (void)0),
   ...);
  return e;
}

}  // namespace spai
