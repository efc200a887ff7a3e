// Declarations of the set-up, transpose and PCG kernels (vec_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace spai {

struct RedWS {  // last-arriver reduction workspace
  double* bsum;
  double* gsum;
  unsigned* cnt1;
  unsigned* cnt2;
  int nb, ngroups;
};

struct SellM {  // sliced ELL: slice s holds entries [sptr[s], sptr[s+1])
  const long long* sptr;
  const int* col;
  const double* val;
};

struct PcgScalars {
  double rho, alpha, beta, bn, rtol, tres;
  int k, maxit, done, status;
};

struct PcgArgs {
  int n;
  SellM A;           // A in sliced ELL
  const double* diag;
  int precond;       // 0 none, 1 Jacobi, 2/3 CSR rows of M or of (M + M^T)/2
  const long long* mrp;
  const int* mci;
  const double* mv;
  // the same rows of S = (M + M^T)/2 in sliced ELL (FP64 products with
  // precond 3 only; sell.sptr null: the CSR rows above are used); rows
  // longer than the sliced ELL's limit are listed in longrows[0..nlong) and
  // get a warp each
  SellM sell;
  const int* longrows;
  int nlong;
  // with long rows: slot i of `sell` holds row sperm[i] (rows by length,
  // longest first), so the rows of a 32-row slice have like lengths
  const int* sperm;
  const double* b;
  double *x, *r, *z, *p, *q;
  PcgScalars* s;
  RedWS ws;
  // the CTA partials of (r, r), apart from ws.bsum: their total is taken
  // with (r, z)'s, after the preconditioner product
  double* rrsum;
  // mixed (FP32-values) products: A's sliced-ELL values and M's (or S's)
  // row values in FP32, and FP32 copies of p and r as their operands
  int mixed;
  const float* aval32;
  const float* mv32;
  float *p32, *r32;
};

cudaError_t launch_seg_reset(DevScalars* sc, int nseg, int fresh, cudaStream_t st);
cudaError_t launch_build_ell(int n, int W, const int* rp, const int* ci, const double* v, int* ecol,
                             double* e64, float* e32, cudaStream_t st);
cudaError_t launch_build_dia(int n, int D, int Dp, const int* rp, const int* ci, const double* v,
                             const int* doff, const int* seg_of_col, const int* seg_doff,
                             const int* seg_D, double* d64, float* d32, cudaStream_t st);
cudaError_t launch_init_slab(int prec, int n, const long long* off, const double* diag, int* Mrow,
                             void* Mval, int* Mlen, int* Plen, int* Zlen, cudaStream_t st);
cudaError_t launch_exclusive_scan(const int* in, long long* out, int n, long long* tmp,
                                  cudaStream_t st);
cudaError_t launch_export_csc(int prec, int n, const long long* off, const int* Mrow,
                              const void* Mval, const long long* colptr, int* rowind, double* vals,
                              cudaStream_t st);
cudaError_t launch_ll_to_i32(const long long* a, int* b, int n, cudaStream_t st);
cudaError_t launch_transpose(int n, const long long* colptr, const int* rowind, const double* vals,
                             long long nnz, int* cnt, long long* rowptr, long long* scan_tmp,
                             int* ci, double* cv, int* tmpi, double* tmpv, cudaStream_t st);
cudaError_t launch_sym(int n, const long long* rp, const int* rci, const double* rv,
                       const long long* cp, const int* cri, const double* cvv, int pass, int* cnt,
                       const long long* srp, int* sci, double* sv, cudaStream_t st);
cudaError_t launch_apply(int n, const long long* rp, const int* ci, const double* v, const double* x,
                         double* y, int nrhs, long long ld, cudaStream_t st);
cudaError_t launch_sell_build_i32(int n, const int* rp, const int* ci, const double* v, int* w32,
                                  long long* sptr, long long* scan_tmp, int** scol, double** sval,
                                  long long* cap, long long* total, cudaStream_t st);
cudaError_t launch_sell_build_i64(int n, const long long* rp, const int* ci, const double* v,
                                  int* w32, long long* sptr, long long* scan_tmp, int** scol,
                                  double** sval, long long* cap, long long* total, cudaStream_t st,
                                  const int* perm);
// perm = the rows of the CSR rows rp ordered by length, longest first, in
// each window of 1,024 rows (rows past the sliced-ELL limit count as empty)
cudaError_t launch_len_order(int n, const long long* rp, int* perm, cudaStream_t st);
// out = the long rows in[0..nl) by length, longest first
cudaError_t launch_sort_long(const int* in, int nl, const long long* rp, int* out, cudaStream_t st);
cudaError_t launch_to_f32(const double* in, float* out, long long count, cudaStream_t st);
// rows of a CSR pattern longer than the sliced ELL's limit, compacted into out
// (count in *nout, device)
cudaError_t launch_long_rows(int n, const long long* rp, int* out, int* nout, cudaStream_t st);

// Lanczos on the rows of a symmetric matrix S (definiteness diagnostics)
struct LzArgs {
  int n;
  const long long* rp;  // CSR rows of S, column-sorted
  const int* ci;
  const double* v;
  double *vp, *vc, *w;  // v_{j-1}, v_j (v0 on entry), work
  double *alpha, *beta; // [steps]
  int* state;           // [0] steps done, [1] stopped
  double* nrm0;
  RedWS ws;
};
cudaError_t launch_lz_start(const LzArgs& a, cudaStream_t st);
cudaError_t launch_lz_step(const LzArgs& a, int j, cudaStream_t st);
// a second stream and two events for running S's long rows beside the
// others (st2 null: one stream)
struct PcgFork {
  cudaStream_t st2;
  cudaEvent_t fork, join;
};
cudaError_t launch_pcg_init(const PcgArgs& a, const PcgFork& f, cudaStream_t st);
cudaError_t launch_pcg_iter(const PcgArgs& a, const PcgFork& f, cudaStream_t st);
cudaError_t launch_true_res(const PcgArgs& a, cudaStream_t st);

cudaError_t launch_colpass_f32(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_colpass_f64(const PassParams& p, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_colpass_res_f32(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st);
cudaError_t launch_colpass_pi_f32(const PassParams& p, int grid, int block, size_t smem,
                                  cudaStream_t st);
cudaError_t launch_colpass_pi_f64(const PassParams& p, int grid, int block, size_t smem,
                                  cudaStream_t st);
// steady-state passes only (steady_pass(p))
cudaError_t launch_colpass_hot_f32(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st);
cudaError_t launch_colpass_hot_f64(const PassParams& p, int grid, int block, size_t smem,
                                   cudaStream_t st);

}  // namespace spai
