// Block PCG: up to 32 independent PCG recurrences per matrix of a handle,
// sharing every SpMM (the Sec. 7 assessment applied to many right-hand
// sides at once).  Internal to libspai.so.
#pragma once
#include <cuda_runtime.h>

namespace spai {

constexpr int kBpRows = 256;  // rows per CTA; segments are whole CTAs
constexpr int kBpLd = 32;     // row stride of the block vectors (one lane per right-hand side)

struct BpcgArgs {
  int n;                 // rows (a multiple of kBpRows is not required)
  int R;                 // right-hand sides, 1..32
  int W;                 // ELL width of A
  const int* ell_col;    // [n][W], padding column -1
  const double* ell_val; // [n][W] FP64
  const double* diag;
  int precond;           // 0 none, 1 Jacobi, 2/3 CSR rows of M or of (M + M^T)/2
  const long long* mrp;
  const int* mci;
  const double* mv;
  double rtol;
  int maxit;
  const double* b;                 // [n][kBpLd]
  double *x, *r, *z, *p, *q;       // [n][kBpLd]
  const int* seg_of_cta;           // [ncta]
  const int* seg_cta0;             // [nseg]
  const int* seg_ncta;             // [nseg]
  // per (segment, rhs) state, index seg * kBpLd + rhs
  double *rho, *alpha, *beta, *bn, *tres;
  int *k, *done, *status;
  int* seg_live;                   // [nseg] recurrences of the segment still running
  int* live;                       // [1] recurrences still running
  double* bsum;                    // [ncta][kBpLd] CTA partials
  unsigned* cnt;                   // [nseg] arrival counters
  // mixed (FP32-values) products: A's ELL values and M's (or S's) row values
  // in FP32, FP32 copies of p and r ([n][kBpLd]) as their operands
  int mixed;
  const float* ell_val32;
  const float* mv32;
  float *p32, *r32;
};

cudaError_t launch_bp_setup(const BpcgArgs& a, int nseg, cudaStream_t st);
cudaError_t launch_bp_gather(const double* user, double* dst, int n, int R, const int* seg_of_cta,
                             const int* seg_row0, const int* seg_n, const long long* seg_boff,
                             cudaStream_t st);
cudaError_t launch_bp_scatter(const double* src, double* user, int n, int R, const int* seg_of_cta,
                              const int* seg_row0, const int* seg_n, const long long* seg_boff,
                              cudaStream_t st);
cudaError_t launch_bp_init(const BpcgArgs& a, cudaStream_t st);   // 3 launches
cudaError_t launch_bp_iter(const BpcgArgs& a, cudaStream_t st);   // 4 launches
cudaError_t launch_bp_tres(const BpcgArgs& a, cudaStream_t st);   // 1 launch

}  // namespace spai
