// The best approximate inverse on a prescribed pattern (Exp. 09 of the
// paper): declarations shared by fixed_pattern.cu and the host API.
#pragma once
#include <cuda_runtime.h>

namespace spai {

struct FpArgs {
  long long n;
  int W;                     // ELL width of A
  const int* ell_col;        // A in ELL, rows column-sorted, padding -1 at the end
  const double* ell_val;     // FP64 values
  const long long* pptr;     // pattern J_j = prow[pptr[j] .. pptr[j+1]), rows ascending
  const int* prow;
  const long long* off;      // M slab offsets
  int* Mrow;
  void* Mval;
  int* Mlen;
  int Lmax;                  // largest |J_j|
  int warp_bytes;            // shared memory per warp
  int* err;                  // bit 1: a Gram matrix was not numerically SPD
};

cudaError_t launch_fixed_pattern(const FpArgs& a, int vs, int nw, cudaStream_t st);

}  // namespace spai
