// Global dropping operators on a handle's column slabs (Sec. 6.1 Eq. 6.2,
// Appendix A): exact global selection by a two-stage radix select on
// 64-bit keys, then in-place compaction.  Internal to libspai.so.
#pragma once
#include <cuda_runtime.h>

namespace spai {

struct SelArgs {
  long long n;            // columns
  const long long* off;   // slab offsets
  int* len;               // slab lengths
  int* rows;
  void* vals;             // slab values (FP32 or FP64, vs bytes)
  int vs;
  const double* score;    // mode 1: score per slab entry (+inf: not eligible)
  int mode;               // 0: smaller key = larger |v|; 1: smaller key = smaller score
  // selection state: stage 0 ranks value keys, stage 1 position keys among
  // the entries whose value key equals ustar
  int stage;
  unsigned long long ustar;
  unsigned long long prefix, mask;  // digits fixed so far
  int shift;                        // the 16-bit digit counted now
  unsigned* hist;                   // 65536 bins
  unsigned long long pstar;         // compaction: last selected position among ties
  int keep_selected;                // compaction: 1 keeps the selected set, 0 drops it
};

cudaError_t launch_sel_hist(const SelArgs& a, cudaStream_t st);
cudaError_t launch_sel_compact(const SelArgs& a, cudaStream_t st);
cudaError_t launch_anrm(int n, int W, const int* ell_col, const void* ell_val, int vs, double* out,
                        cudaStream_t st);
// symmetric part (CSR rows, FP64) written back as the columns of M, each
// value rounded to the value type; off-diagonal |s| < u and zeros dropped;
// *ovf set if a column exceeds its capacity
cudaError_t launch_sym_to_slab(int n, const long long* srp, const int* sci, const double* sv,
                               const long long* off, const int* cap, int* rows, void* vals,
                               int* len, int vs, double u, int* ovf, cudaStream_t st);

}  // namespace spai
