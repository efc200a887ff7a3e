// The best approximate inverse on a prescribed pattern (the paper's Exp. 09,
// Figs. 1-2: the classic Frobenius-norm SPAI on supp(A^k)).  Column j of M
// minimises ||e_j - A m_j||_2 over supp(m_j) = J = supp(A^k e_j); with A
// symmetric its normal equations are
//     (A^2)[J, J] m = A[J, j],   (A^2)_ab = sum_t a_{J_a t} a_{J_b t},
// solved here by one warp per column: the Gram matrix from merged rows of A
// (an fma chain over ascending t), an FP64 Cholesky factorisation in shared
// memory and two triangular solves.  The pattern is built on the host.
#include <stdint.h>

#include "common.cuh"
#include "fixed_pattern.cuh"

namespace spai {

namespace {

// sum_t a_{r1 t} a_{r2 t} over the common columns of two ELL rows of A
// (columns ascending, padding -1 at the end of a row)
__device__ double row_dot(const FpArgs& a, int r1, int r2) {
  const int* c1 = a.ell_col + (long long)r1 * a.W;
  const int* c2 = a.ell_col + (long long)r2 * a.W;
  const double* v1 = a.ell_val + (long long)r1 * a.W;
  const double* v2 = a.ell_val + (long long)r2 * a.W;
  int p = 0, q = 0;
  double acc = 0.0;
  while (p < a.W && q < a.W) {
    const int x = c1[p], y = c2[q];
    if (x < 0 || y < 0) break;
    if (x < y) {
      p++;
    } else if (y < x) {
      q++;
    } else {
      acc = __fma_rn(v1[p], v2[q], acc);
      p++;
      q++;
    }
  }
  return acc;
}

__device__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

template <typename VS>
__global__ void k_fixed_pattern(FpArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long j = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= a.n) return;
  char* ws = smem + (size_t)warp * a.warp_bytes;
  double* G = (double*)ws;                              // [L][L], row-major
  double* y = G + (size_t)a.Lmax * a.Lmax;              // rhs, then solutions
  int* J = (int*)(y + a.Lmax);
  const long long p0 = a.pptr[j];
  const int L = (int)(a.pptr[j + 1] - p0);
  for (int t = lane; t < L; t += 32) J[t] = a.prow[p0 + t];
  __syncwarp();
  // Gram matrix (lower triangle computed, mirrored) and right-hand side
  for (int r = 0; r < L; r++)
    for (int c = lane; c <= r; c += 32) {
      const double g = row_dot(a, J[r], J[c]);
      G[r * L + c] = g;
      G[c * L + r] = g;
    }
  for (int r = lane; r < L; r += 32) {
    const int* cc = a.ell_col + (long long)J[r] * a.W;
    const double* vv = a.ell_val + (long long)J[r] * a.W;
    double v = 0.0;
    for (int e = 0; e < a.W && cc[e] >= 0; e++)
      if (cc[e] == (int)j) v = vv[e];
    y[r] = v;
  }
  __syncwarp();
  // Cholesky G = C C^T, C lower, in place
  bool bad = false;
  for (int p = 0; p < L; p++) {
    const double d = G[p * L + p];
    if (!(d > 0.0)) bad = true;
    const double s = d > 0.0 ? __dsqrt_rn(d) : 1.0;
    __syncwarp();
    if (lane == 0) G[p * L + p] = s;
    for (int r = p + 1 + lane; r < L; r += 32) G[r * L + p] = __ddiv_rn(G[r * L + p], s);
    __syncwarp();
    for (int r = p + 1; r < L; r++) {
      const double grp = G[r * L + p];
      for (int c = p + 1 + lane; c <= r; c += 32) G[r * L + c] = __fma_rn(-grp, G[c * L + p], G[r * L + c]);
    }
    __syncwarp();
  }
  // C z = y, then C^T m = z (in y)
  for (int r = 0; r < L; r++) {
    double part = 0.0;
    for (int c = lane; c < r; c += 32) part = __fma_rn(G[r * L + c], y[c], part);
    const double s = warp_sum(part);
    if (lane == 0) y[r] = __ddiv_rn(y[r] - s, G[r * L + r]);
    __syncwarp();
  }
  for (int r = L - 1; r >= 0; r--) {
    double part = 0.0;
    for (int c = r + 1 + lane; c < L; c += 32) part = __fma_rn(G[c * L + r], y[c], part);
    const double s = warp_sum(part);
    if (lane == 0) y[r] = __ddiv_rn(y[r] - s, G[r * L + r]);
    __syncwarp();
  }
  if (bad) {
    if (lane == 0) atomicOr(a.err, 1);
  }
  // store the column, exact zeros removed
  const long long off = a.off[j];
  VS* Mv = (VS*)a.Mval;
  int out = 0;
  for (int base = 0; base < L; base += 32) {
    const int t = base + lane;
    VS v = VS(0);
    if (t < L) v = (VS)y[t];
    const bool keep = t < L && v != VS(0);
    const unsigned b = __ballot_sync(kFull, keep);
    if (keep) {
      const int pos = out + __popc(b & ((1u << lane) - 1u));
      a.Mrow[off + pos] = J[t];
      Mv[off + pos] = v;
    }
    out += __popc(b);
  }
  if (lane == 0) a.Mlen[j] = out;
}

}  // namespace

cudaError_t launch_fixed_pattern(const FpArgs& a, int vs, int nw, cudaStream_t st) {
  const size_t smem = (size_t)nw * a.warp_bytes;
  const int grid = (int)((a.n + nw - 1) / nw);
  cudaError_t e;
  if (vs == 4) {
    e = cudaFuncSetAttribute(k_fixed_pattern<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_fixed_pattern<float><<<grid, 32 * nw, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_fixed_pattern<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_fixed_pattern<double><<<grid, 32 * nw, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace spai
