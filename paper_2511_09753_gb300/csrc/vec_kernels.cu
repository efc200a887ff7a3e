// Set-up, export, transpose and vector-PCG kernels of libspai.so.
//
// PCG (the assessment of Sec. 7): x_0 = 0, FP64 vectors and scalars;
// SpMV rows are fma chains over ascending column; vector inner products are
// balanced pairwise trees over the index range (same tree as the Frobenius
// sums of the column pass); the preconditioner is none, Jacobi, M or the
// symmetric part (M + M^T)/2.
#include <stdint.h>

#include "common.cuh"
#include "vec_kernels.cuh"
#include "warp_ops.cuh"

namespace spai {

// rows of S longer than this are multiplied by a whole warp (sliced-ELL
// threads take the others)
constexpr int kLongRow = 64;

// ------------------------------------------------------------- reduction

// Each thread contributes one term (its element); the CTA (256 threads)
// reduces by a contiguous tree, then the last-arriving CTA of each group of
// kGroup CTAs, then the last group, calls finish(total) in its thread 0.
//
// The CTA's tree runs in one warp: the terms are staged in shared memory and
// lane l adds its 8 consecutive terms pairwise before the warp's
// tree (GB300's FP64 pipe takes about 20 SM cycles per warp instruction,
// active lanes or not, so 13 such instructions replace 45).  The trailing
// + 0 stands for the zero-padded top of a tree over 32 warps of 32 (it
// turns -0 into +0 and changes nothing else).
template <typename F>
__device__ void reduce_finish(double term, const RedWS& w, F finish) {
  __shared__ double red[1024];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  red[threadIdx.x] = term;  // blockDim.x == 256 for every caller
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    double t[8];
#pragma unroll
    for (int q = 0; q < 8; q++) t[q] = red[lane * 8 + q];
#pragma unroll
    for (int len = 8; len > 1; len >>= 1)
#pragma unroll
      for (int q = 0; 2 * q + 1 < len; q++) t[q] = __dadd_rn(t[2 * q], t[2 * q + 1]);
    s = __dadd_rn(warp_tree32(t[0]), 0.0);
  }
  const int g = blockIdx.x / kGroup;
  if (threadIdx.x == 0) {
    w.bsum[blockIdx.x] = s;
    __threadfence();
    int gsize = min(kGroup, w.nb - g * kGroup);
    unsigned old = atomicAdd(&w.cnt1[g], 1u);
    s_last = old == (unsigned)(gsize - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (warp == 0) {
    int gsize = min(kGroup, w.nb - g * kGroup);
    const double* v = w.bsum + (long long)g * kGroup;
    double a = (2 * lane < gsize) ? __ldcg(v + 2 * lane) : 0.0;
    double b = (2 * lane + 1 < gsize) ? __ldcg(v + 2 * lane + 1) : 0.0;
    s = warp_tree32(__dadd_rn(a, b));
  }
  if (threadIdx.x == 0) {
    w.gsum[g] = s;
    w.cnt1[g] = 0;
    __threadfence();
    unsigned old = atomicAdd(w.cnt2, 1u);
    s_last = old == (unsigned)(w.ngroups - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (warp == 0) {
    int P2 = 32;
    while (P2 < w.ngroups) P2 <<= 1;
    int c = P2 / 32;
    for (int t = 0; t < c; t++) {
      int i = lane * c + t;
      red[i] = i < w.ngroups ? __ldcg(w.gsum + i) : 0.0;
    }
    __syncwarp();
    s = warp_pairwise(red, P2, lane);
  }
  if (threadIdx.x == 0) {
    *w.cnt2 = 0;
    finish(s);
    __threadfence();
  }
}

__device__ __forceinline__ bool finite_d(double x) { return !isnan(x) && !isinf(x); }

// y_i = fma chain over row i of a CSR matrix (ascending column)
template <typename RP, typename V>
__device__ __forceinline__ double row_chain(const RP* rp, const int* ci, const V* v, const double* x,
                                            int i) {
  double acc = 0.0;
  const RP e1 = rp[i + 1];
  for (RP e = rp[i]; e < e1; e++) acc = __fma_rn((double)v[e], x[ci[e]], acc);
  return acc;
}

// Sliced ELL (32 rows per slice, column-major inside a slice, padded with
// zero values): thread i reads entry t of its row at base + 32 t + lane, so
// a warp's loads are coalesced; entries keep ascending column order, so the
// fma chain of every row is the same as in CSR.
__device__ __forceinline__ double sell_chain(const SellM& m, const double* x, int i) {
  const int s = i >> 5, lane = i & 31;
  const long long b = m.sptr[s];
  const int w = (int)((m.sptr[s + 1] - b) >> 5);
  double acc = 0.0;
  for (int t = 0; t < w; t++) {
    long long e = b + 32LL * t + lane;
    acc = __fma_rn(m.val[e], x[m.col[e]], acc);
  }
  return acc;
}

// FP32-values variants for the mixed PCG: FP32 values and operand, an FP32
// fma chain in the same entry order, the row result widened to FP64
__device__ __forceinline__ double sell_chain_f32(const SellM& m, const float* v32, const float* x,
                                                 int i) {
  const int s = i >> 5, lane = i & 31;
  const long long b = m.sptr[s];
  const int w = (int)((m.sptr[s + 1] - b) >> 5);
  float acc = 0.0f;
  for (int t = 0; t < w; t++) {
    long long e = b + 32LL * t + lane;
    acc = __fmaf_rn(v32[e], x[m.col[e]], acc);
  }
  return (double)acc;
}

// Row i of a CSR matrix (row pointers rp) from its sliced-ELL copy: the loads
// are coalesced as in sell_chain, and the chain stops at the row's own length,
// so it is the CSR chain of row_chain entry for entry.
__device__ __forceinline__ double sell_row_chain(const SellM& m, const long long* rp,
                                                 const double* x, int i) {
  const int s = i >> 5, lane = i & 31;
  const long long b = m.sptr[s];
  const int len = (int)(rp[i + 1] - rp[i]);
  double acc = 0.0;
  for (int t = 0; t < len; t++) {
    long long e = b + 32LL * t + lane;
    acc = __fma_rn(m.val[e], x[m.col[e]], acc);
  }
  return acc;
}

// The chain of a row of length len stored in slot i of a sliced ELL
__device__ __forceinline__ double sell_slot_chain(const SellM& m, int len, const double* x, int i) {
  const int s = i >> 5, lane = i & 31;
  const long long b = m.sptr[s];
  double acc = 0.0;
  for (int t = 0; t < len; t++) {
    long long e = b + 32LL * t + lane;
    acc = __fma_rn(m.val[e], x[m.col[e]], acc);
  }
  return acc;
}

template <typename RP>
__device__ __forceinline__ double row_chain_f32(const RP* rp, const int* ci, const float* v,
                                                const float* x, int i) {
  float acc = 0.0f;
  const RP e1 = rp[i + 1];
  for (RP e = rp[i]; e < e1; e++) acc = __fmaf_rn(v[e], x[ci[e]], acc);
  return (double)acc;
}

__global__ void k_to_f32(const double* in, float* out, long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = __double2float_rn(in[i]);
}

cudaError_t launch_to_f32(const double* in, float* out, long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_to_f32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

// Rows longer than maxw are left out of the sliced ELL (stored as empty rows):
// their products are formed from the CSR arrays by a thread each.  perm
// (optional): slot i of the sliced ELL holds row perm[i] instead of row i.
template <typename RP>
__global__ void k_sell_width(int n, const RP* rp, int* w32, int maxw, const int* perm) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int ns = (n + 31) / 32;
  if (s >= ns) return;
  int w = 0;
  for (int i = 32 * s; i < min(n, 32 * s + 32); i++) {
    const int row = perm ? perm[i] : i;
    const int len = (int)(rp[row + 1] - rp[row]);
    if (len <= maxw) w = max(w, len);
  }
  w32[s] = 32 * w;
}

template <typename RP>
__global__ void k_sell_fill(int n, const RP* rp, const int* ci, const double* v,
                            const long long* sptr, int* scol, double* sval, int maxw,
                            const int* perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int ns = (n + 31) / 32;
  if (i >= 32 * ns) return;
  const int s = i >> 5, lane = i & 31;
  const long long b = sptr[s];
  const int w = (int)((sptr[s + 1] - b) >> 5);
  const int row = i < n ? (perm ? perm[i] : i) : 0;
  long long e0 = i < n ? (long long)rp[row] : 0, e1 = i < n ? (long long)rp[row + 1] : 0;
  if (e1 - e0 > maxw) e1 = e0;
  for (int t = 0; t < w; t++) {
    long long e = e0 + t;
    long long d = b + 32LL * t + lane;
    if (e < e1) {
      scol[d] = ci[e];
      sval[d] = v[e];
    } else {
      scol[d] = 0;
      sval[d] = 0.0;
    }
  }
}

template <typename RP>
static cudaError_t sell_build_t(int n, const RP* rp, const int* ci, const double* v, int* w32,
                                long long* sptr, long long* scan_tmp, int** scol, double** sval,
                                long long* cap, long long* total, cudaStream_t st, int maxw,
                                const int* perm) {
  int ns = (n + 31) / 32;
  k_sell_width<RP><<<(ns + 255) / 256, 256, 0, st>>>(n, rp, w32, maxw, perm);
  cudaError_t e = launch_exclusive_scan(w32, sptr, ns, scan_tmp, st);
  if (e != cudaSuccess) return e;
  long long tot = 0;
  e = cudaMemcpyAsync(&tot, sptr + ns, sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (tot > *cap || !*scol) {
    if (*scol) cudaFree(*scol);
    if (*sval) cudaFree(*sval);
    *scol = nullptr;
    *sval = nullptr;
    e = cudaMalloc((void**)scol, sizeof(int) * (size_t)(tot ? tot : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)sval, sizeof(double) * (size_t)(tot ? tot : 1));
    if (e != cudaSuccess) return e;
    *cap = tot;
  }
  k_sell_fill<RP><<<(32 * ns + 255) / 256, 256, 0, st>>>(n, rp, ci, v, sptr, *scol, *sval, maxw,
                                                         perm);
  *total = tot;
  return cudaGetLastError();
}

cudaError_t launch_sell_build_i32(int n, const int* rp, const int* ci, const double* v, int* w32,
                                  long long* sptr, long long* scan_tmp, int** scol, double** sval,
                                  long long* cap, long long* total, cudaStream_t st) {
  return sell_build_t<int>(n, rp, ci, v, w32, sptr, scan_tmp, scol, sval, cap, total, st,
                           0x7fffffff, nullptr);
}

cudaError_t launch_sell_build_i64(int n, const long long* rp, const int* ci, const double* v,
                                  int* w32, long long* sptr, long long* scan_tmp, int** scol,
                                  double** sval, long long* cap, long long* total, cudaStream_t st,
                                  const int* perm) {
  return sell_build_t<long long>(n, rp, ci, v, w32, sptr, scan_tmp, scol, sval, cap, total, st,
                                 kLongRow, perm);
}

// Rows of S ordered by length, longest first, inside each window of 1,024
// consecutive rows (32 slices of the sliced ELL), so that a slice's rows
// have like lengths while the operands a window gathers stay near each
// other; rows longer than kLongRow (multiplied apart) count as empty.  The
// order among rows of one length is arbitrary: each row's product is the
// same chain wherever it sits.
__global__ void __launch_bounds__(256) k_len_order(int n, const long long* rp, int* perm) {
  __shared__ int cnt[kLongRow + 1];
  const int w0 = blockIdx.x * 1024;
  for (int b = threadIdx.x; b <= kLongRow; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  int len[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int i = w0 + q * 256 + threadIdx.x;
    len[q] = -1;
    if (i < n) {
      const int l = (int)(rp[i + 1] - rp[i]);
      len[q] = l <= kLongRow ? l : 0;
      atomicAdd(&cnt[len[q]], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // counts -> first slot of each length, longest first
    int at = w0;
    for (int l = kLongRow; l >= 0; l--) {
      const int c = cnt[l];
      cnt[l] = at;
      at += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; q++)
    if (len[q] >= 0) perm[atomicAdd(&cnt[len[q]], 1)] = w0 + q * 256 + threadIdx.x;
}

cudaError_t launch_len_order(int n, const long long* rp, int* perm, cudaStream_t st) {
  k_len_order<<<(n + 1023) / 1024, 256, 0, st>>>(n, rp, perm);
  return cudaGetLastError();
}

// The long rows in[0..nl) by length, longest first (ties: the smaller row),
// by ranking in one CTA; more than kSortLongMax of them are copied as they
// are (their order changes no result, only how the warps share them out).
constexpr int kSortLongMax = 4096;
__global__ void k_sort_long(const int* in, int nl, const long long* rp, int* out) {
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    const int row = in[i];
    if (nl > kSortLongMax) {
      out[i] = row;
      continue;
    }
    const long long len = rp[row + 1] - rp[row];
    int rank = 0;
    for (int k = 0; k < nl; k++) {
      const int r2 = in[k];
      const long long l2 = rp[r2 + 1] - rp[r2];
      rank += (l2 > len) || (l2 == len && r2 < row);
    }
    out[rank] = row;
  }
}

cudaError_t launch_sort_long(const int* in, int nl, const long long* rp, int* out, cudaStream_t st) {
  k_sort_long<<<1, 1024, 0, st>>>(in, nl, rp, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ set-up

template <typename VS>
__global__ void k_init_slab(int n, const long long* off, const double* diag, int* Mrow, VS* Mval,
                            int* Mlen, int* Plen, int* Zlen) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double m0 = __ddiv_rn(1.0, diag[j]);
  VS v = (VS)m0;
  Mrow[off[j]] = j;
  Mval[off[j]] = v;
  Mlen[j] = v != VS(0) ? 1 : 0;
  Plen[j] = 0;
  Zlen[j] = 0;
}

cudaError_t launch_init_slab(int prec, int n, const long long* off, const double* diag, int* Mrow,
                             void* Mval, int* Mlen, int* Plen, int* Zlen, cudaStream_t st) {
  int g = (n + 255) / 256;
  if (prec == 1)
    k_init_slab<float><<<g, 256, 0, st>>>(n, off, diag, Mrow, (float*)Mval, Mlen, Plen, Zlen);
  else
    k_init_slab<double><<<g, 256, 0, st>>>(n, off, diag, Mrow, (double*)Mval, Mlen, Plen, Zlen);
  return cudaGetLastError();
}

// A's ELL layout from its CSR: row i's entries in CSR order, then padding
// column -1 with value 0; an FP32 copy of the values when v32 is given
__global__ void k_build_ell(int n, int W, const int* rp, const int* ci, const double* v,
                            int* ecol, double* e64, float* e32) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e0 = rp[i], len = rp[i + 1] - e0;
  for (int t = 0; t < W; t++) {
    const long long d = i * W + t;
    const int c = t < len ? ci[e0 + t] : -1;
    const double x = t < len ? v[e0 + t] : 0.0;
    ecol[d] = c;
    e64[d] = x;
    if (e32) e32[d] = __double2float_rn(x);
  }
}

// A's diagonal slots: value of row i at slot s is a_{i, i + off_s}, 0 where
// row i has no such entry.  The offsets of row i's matrix are doff (single
// matrix) or seg_doff[seg_of_col[i]] (batch), ascending, and every entry's
// offset is among them; columns ascend in a row, so slots do too.
struct DiaOffs {
  int off[32];
};
__global__ void k_build_dia(int n, int D0, int Dp, const int* rp, const int* ci, const double* v, DiaOffs doff,
                            const int* seg_of_col, const int* seg_doff, const int* seg_D,
                            double* d64, float* d32) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = seg_of_col ? seg_of_col[i] : -1;
  const int D = m >= 0 ? seg_D[m] : D0;
  for (int s = 0; s < Dp; s++) {
    d64[i * Dp + s] = 0.0;
    if (d32) d32[i * Dp + s] = 0.0f;
  }
  int s = 0;
  for (int e = rp[i]; e < rp[i + 1]; e++) {
    const int o = ci[e] - (int)i;
    while (s < D && (m >= 0 ? seg_doff[m * 32 + s] : doff.off[s]) < o) s++;
    if (s >= D) return;  // not reached: every offset was found on the host
    d64[i * Dp + s] = v[e];
    if (d32) d32[i * Dp + s] = __double2float_rn(v[e]);
  }
}

cudaError_t launch_build_ell(int n, int W, const int* rp, const int* ci, const double* v, int* ecol,
                             double* e64, float* e32, cudaStream_t st) {
  k_build_ell<<<(n + 255) / 256, 256, 0, st>>>(n, W, rp, ci, v, ecol, e64, e32);
  return cudaGetLastError();
}

cudaError_t launch_build_dia(int n, int D, int Dp, const int* rp, const int* ci, const double* v,
                             const int* doff, const int* seg_of_col, const int* seg_doff,
                             const int* seg_D, double* d64, float* d32, cudaStream_t st) {
  DiaOffs o;
  for (int s = 0; s < 32; s++) o.off[s] = doff ? doff[s] : 0;
  k_build_dia<<<(n + 255) / 256, 256, 0, st>>>(n, D, Dp, rp, ci, v, o, seg_of_col, seg_doff, seg_D,
                                               d64, d32);
  return cudaGetLastError();
}

// per-matrix scalars of a batched handle at the start of a call
__global__ void k_seg_reset(DevScalars* sc, int nseg, int fresh) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nseg) return;
  sc[m].stop = 0;
  sc[m].flags = 0;
  sc[m].done = 0;
  if (fresh) {
    sc[m].beta = 0.0;
    sc[m].rr = 0.0;
  }
}

cudaError_t launch_seg_reset(DevScalars* sc, int nseg, int fresh, cudaStream_t st) {
  k_seg_reset<<<(nseg + 127) / 128, 128, 0, st>>>(sc, nseg, fresh);
  return cudaGetLastError();
}

// ------------------------------------------------------------- scan

// exclusive scan of int32 counts into int32/int64 offsets, 1024 per block
__global__ void k_scan_block(const int* in, long long* out, long long* bsum, int n) {
  __shared__ long long s[1024];
  int i = blockIdx.x * 1024 + threadIdx.x;
  long long v = i < n ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}

__global__ void k_scan_add(long long* out, const long long* boff, int n) {
  int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_scan_small(const long long* in, long long* out, int n, long long* total) {
  // single block, sequential over chunks of 1024
  __shared__ long long s[1024];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    int i = base + threadIdx.x;
    long long v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      long long t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) out[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// out[0..n) = exclusive scan of in, out[n] = total.  tmp: >= 2*ceil(n/1024)+1
cudaError_t launch_exclusive_scan(const int* in, long long* out, int n, long long* tmp,
                                  cudaStream_t st) {
  int nb = (n + 1023) / 1024;
  if (nb == 0) nb = 1;
  k_scan_block<<<nb, 1024, 0, st>>>(in, out, tmp, n);
  k_scan_small<<<1, 1024, 0, st>>>(tmp, tmp + nb, nb, out + n);
  k_scan_add<<<nb, 1024, 0, st>>>(out, tmp + nb, n);
  return cudaGetLastError();
}

// ------------------------------------------------- export / transpose

// Slab columns are stored in no particular order; the CSC export sorts each
// column by row (rank by counting: rows within a column are distinct).
template <typename VS>
__global__ void k_export_csc(int n, const long long* off, const int* Mrow, const VS* Mval,
                             const long long* colptr, int* rowind, double* vals) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= n) return;
  long long src = off[j], dst = colptr[j];
  int len = (int)(colptr[j + 1] - dst);
  for (int e = lane; e < len; e += 32) {
    int r = Mrow[src + e];
    int rank = 0;
    for (int q = 0; q < len; q++) rank += Mrow[src + q] < r;
    rowind[dst + rank] = r;
    vals[dst + rank] = (double)Mval[src + e];
  }
}

__global__ void k_ll_to_i32(const long long* a, int* b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) b[i] = (int)a[i];
}

cudaError_t launch_export_csc(int prec, int n, const long long* off, const int* Mrow,
                              const void* Mval, const long long* colptr, int* rowind, double* vals,
                              cudaStream_t st) {
  int g = (int)(((long long)n * 32 + 255) / 256);
  if (prec == 1)
    k_export_csc<float><<<g, 256, 0, st>>>(n, off, Mrow, (const float*)Mval, colptr, rowind, vals);
  else
    k_export_csc<double><<<g, 256, 0, st>>>(n, off, Mrow, (const double*)Mval, colptr, rowind, vals);
  return cudaGetLastError();
}

cudaError_t launch_ll_to_i32(const long long* a, int* b, int n, cudaStream_t st) {
  k_ll_to_i32<<<(n + 1 + 255) / 256, 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

__global__ void k_count_rows(int n, const long long* colptr, const int* rowind, int* cnt) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= colptr[n]) return;
  atomicAdd(&cnt[rowind[e]], 1);
}

// scatter CSC entries into row buckets (unordered within a row)
__global__ void k_fill_rows(int n, const long long* colptr, const int* rowind, const double* vals,
                            const long long* rowptr, int* cursor, int* ci, double* cv) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= n) return;
  for (long long e = colptr[j] + lane; e < colptr[j + 1]; e += 32) {
    int r = rowind[e];
    int pos = atomicAdd(&cursor[r], 1);
    ci[rowptr[r] + pos] = j;
    cv[rowptr[r] + pos] = vals[e];
  }
}

// sort each row by column (keys unique): rank by counting, warp per row
__global__ void k_sort_rows(int n, const long long* rowptr, int* ci, double* cv, int* tmpi,
                            double* tmpv) {
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  long long b = rowptr[i], e = rowptr[i + 1];
  int L = (int)(e - b);
  for (int a = lane; a < L; a += 32) {
    int key = ci[b + a];
    int rank = 0;
    for (int t = 0; t < L; t++) rank += ci[b + t] < key;
    tmpi[b + rank] = key;
    tmpv[b + rank] = cv[b + a];
  }
  __syncwarp();
  for (int a = lane; a < L; a += 32) {
    ci[b + a] = tmpi[b + a];
    cv[b + a] = tmpv[b + a];
  }
}

// symmetric part S = (M + M^T)/2: row i of S merges CSR row i of M and CSC
// column i of M; s = 0.5 * (m_ij + m_ji); exact zeros dropped.
// pass 0 counts, pass 1 fills.
__global__ void k_sym_rows(int n, const long long* rp, const int* rci, const double* rv,
                           const long long* cp, const int* cri, const double* cvv, int pass,
                           int* cnt, const long long* srp, int* sci, double* sv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long a = rp[i], ae = rp[i + 1], b = cp[i], be = cp[i + 1];
  long long t = pass ? srp[i] : 0;
  int c = 0;
  while (a < ae || b < be) {
    int col;
    double u = 0.0, w = 0.0;
    if (b >= be || (a < ae && rci[a] < cri[b])) {
      col = rci[a];
      u = rv[a++];
    } else if (a >= ae || cri[b] < rci[a]) {
      col = cri[b];
      w = cvv[b++];
    } else {
      col = rci[a];
      u = rv[a++];
      w = cvv[b++];
    }
    double val = __dmul_rn(0.5, __dadd_rn(u, w));
    if (val != 0.0) {
      if (pass) {
        sci[t + c] = col;
        sv[t + c] = val;
      }
      c++;
    }
  }
  if (!pass) cnt[i] = c;
}

cudaError_t launch_transpose(int n, const long long* colptr, const int* rowind, const double* vals,
                             long long nnz, int* cnt, long long* rowptr, long long* scan_tmp,
                             int* ci, double* cv, int* tmpi, double* tmpv, cudaStream_t st) {
  cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, st);
  if (nnz > 0) k_count_rows<<<(int)((nnz + 255) / 256), 256, 0, st>>>(n, colptr, rowind, cnt);
  launch_exclusive_scan(cnt, rowptr, n, scan_tmp, st);
  cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, st);
  int g = (int)(((long long)n * 32 + 255) / 256);
  k_fill_rows<<<g, 256, 0, st>>>(n, colptr, rowind, vals, rowptr, cnt, ci, cv);
  k_sort_rows<<<g, 256, 0, st>>>(n, rowptr, ci, cv, tmpi, tmpv);
  return cudaGetLastError();
}

cudaError_t launch_sym(int n, const long long* rp, const int* rci, const double* rv,
                       const long long* cp, const int* cri, const double* cvv, int pass, int* cnt,
                       const long long* srp, int* sci, double* sv, cudaStream_t st) {
  k_sym_rows<<<(n + 255) / 256, 256, 0, st>>>(n, rp, rci, rv, cp, cri, cvv, pass, cnt, srp, sci, sv);
  return cudaGetLastError();
}

// -------------------------------------------------------- y = M x (apply)

__global__ void k_spmv_multi(int n, const long long* rp, const int* ci, const double* v,
                             const double* x, double* y, int nrhs, long long ld) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * nrhs) return;
  int k = (int)(t / n), i = (int)(t % n);
  const double* xk = x + (long long)k * ld;
  double acc = 0.0;
  for (long long e = rp[i]; e < rp[i + 1]; e++) acc = __fma_rn(v[e], xk[ci[e]], acc);
  y[(long long)k * ld + i] = acc;
}

cudaError_t launch_apply(int n, const long long* rp, const int* ci, const double* v, const double* x,
                         double* y, int nrhs, long long ld, cudaStream_t st) {
  long long tot = (long long)n * nrhs;
  k_spmv_multi<<<(int)((tot + 255) / 256), 256, 0, st>>>(n, rp, ci, v, x, y, nrhs, ld);
  return cudaGetLastError();
}

// --------------------------------------------------------------- residual
// FP64 ||b - A x|| helper terms: t_i = (b_i - (A x)_i)^2
__global__ void k_true_res(PcgArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    double y = sell_chain(a.A, a.x, i);
    double d = __dsub_rn(a.b[i], y);
    term = __dmul_rn(d, d);
  }
  PcgScalars* s = a.s;
  reduce_finish(term, a.ws, [s](double tot) { s->tres = tot; });
}

// ------------------------------------------------------------------- PCG
//
// An inner product of the iteration leaves one partial per CTA (the kernel
// that forms its terms stores them); k_pcg_fin, one CTA launched right after,
// adds the partials and takes the scalar step.  Between kernels of a graph
// this is shorter than the last-arriver chain of reduce_finish (fences and
// counter atomics in series), with the same tree.

// The CTA's contiguous tree of its 256 terms (in one warp, as reduce_finish
// forms it), stored to out[blockIdx.x] by thread 0.
__device__ __forceinline__ void cta_partial(double term, double* out) {
  __shared__ double red[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  red[threadIdx.x] = term;
  __syncthreads();
  if (warp == 0) {
    double t[8];
#pragma unroll
    for (int q = 0; q < 8; q++) t[q] = red[lane * 8 + q];
#pragma unroll
    for (int len = 8; len > 1; len >>= 1)
#pragma unroll
      for (int q = 0; 2 * q + 1 < len; q++) t[q] = __dadd_rn(t[2 * q], t[2 * q + 1]);
    const double s = __dadd_rn(warp_tree32(t[0]), 0.0);
    if (lane == 0) out[blockIdx.x] = s;
  }
}

// The total of the nb CTA partials v[0..nb): contiguous pairwise tree over
// nb zero-padded to a power of two P >= 256 (levels of the same tree as
// reduce_finish's groups and final level); one CTA of 256 threads.
__device__ double cta_total(const double* v, int nb) {
  __shared__ double red[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int P = 256;
  while (P < nb) P <<= 1;
  const int c = P >> 8, i0 = threadIdx.x * c;
  double s;
  if (c <= 8) {
    double t[8];
#pragma unroll
    for (int q = 0; q < 8; q++) t[q] = (q < c && i0 + q < nb) ? __ldcg(v + i0 + q) : 0.0;
    for (int len = c; len > 1; len >>= 1)
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (2 * q + 1 < len) t[q] = __dadd_rn(t[2 * q], t[2 * q + 1]);
    s = t[0];
  } else {  // binary-counter merging of the span (pairwise for a power of two)
    double st[32];
    int sz[32];
    int top = 0;
    for (int q = 0; q < c; q++) {
      double x = i0 + q < nb ? __ldcg(v + i0 + q) : 0.0;
      int w = 1;
      while (top > 0 && sz[top - 1] == w) {
        x = __dadd_rn(st[top - 1], x);
        w <<= 1;
        top--;
      }
      st[top] = x;
      sz[top] = w;
      top++;
    }
    s = st[0];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  double tot = 0.0;
  if (warp == 0) {
    double t[8];
#pragma unroll
    for (int q = 0; q < 8; q++) t[q] = red[lane * 8 + q];
#pragma unroll
    for (int len = 8; len > 1; len >>= 1)
#pragma unroll
      for (int q = 0; 2 * q + 1 < len; q++) t[q] = __dadd_rn(t[2 * q], t[2 * q + 1]);
    tot = warp_tree32(t[0]);
  }
  return tot;  // valid in warp 0
}


__device__ __forceinline__ double precond_apply(const PcgArgs& a, int i) {
  if (a.precond == 0) return a.r[i];
  if (a.precond == 1) return __ddiv_rn(a.r[i], a.diag[i]);
  if (a.mixed) return row_chain_f32(a.mrp, a.mci, a.mv32, a.r32, i);
  return row_chain(a.mrp, a.mci, a.mv, a.r, i);
}

// z_i = (S r)_i of a row of at most kLongRow entries from the sliced ELL (a
// longer row's z_i was written by k_pcg_prec_long before)
__device__ __forceinline__ double precond_sell(const PcgArgs& a, int i) {
  const int len = (int)(a.mrp[i + 1] - a.mrp[i]);
  if (len > kLongRow) return a.z[i];
  return sell_row_chain(a.sell, a.mrp, a.r, i);
}

// z_i of the rows longer than kLongRow, a warp each, one warp per CTA (the
// rows come longest first, so the longest chains start first and the warps
// spread over all SMs instead of sharing a few SMs' FP64 pipes): the lanes
// load 32 consecutive CSR entries and their operands at once; the chain
// itself -- the same fma chain over ascending column -- runs on the shuffled
// values
__global__ void __launch_bounds__(32) k_pcg_prec_long(PcgArgs a) {
  if (a.s->done) return;
  const int lane = threadIdx.x;
  const int row = a.longrows[blockIdx.x];
  const long long rb = a.mrp[row], re = a.mrp[row + 1];
  double acc = 0.0;
  for (long long base = rb; base < re; base += 32) {
    const long long e = base + lane;
    double vv = 0.0, xx = 0.0;
    if (e < re) {
      vv = a.mv[e];
      xx = a.r[a.mci[e]];
    }
    const int cnt = (int)min(32LL, re - base);
    for (int t = 0; t < cnt; t++)
      acc = __fma_rn(__shfl_sync(kFull, vv, t), __shfl_sync(kFull, xx, t), acc);
  }
  if (lane == 0) a.z[row] = acc;
}

__global__ void k_long_rows(int n, const long long* rp, int* out, int* nout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && rp[i + 1] - rp[i] > kLongRow) out[atomicAdd(nout, 1)] = i;
}

cudaError_t launch_long_rows(int n, const long long* rp, int* out, int* nout, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(nout, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_long_rows<<<(n + 255) / 256, 256, 0, st>>>(n, rp, out, nout);
  return cudaGetLastError();
}

// init: x = 0, r = b, terms b_i^2 -> bn
__global__ void k_pcg_init(PcgArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    double bi = a.b[i];
    a.x[i] = 0.0;
    a.r[i] = bi;
    if (a.mixed) a.r32[i] = __double2float_rn(bi);
    term = __dmul_rn(bi, bi);
  }
  PcgScalars* s = a.s;
  reduce_finish(term, a.ws, [s](double tot) {
    s->bn = __dsqrt_rn(tot);
    s->k = 0;
    s->status = 0;
    s->done = (tot == 0.0) ? 1 : 0;
  });
}

// rho = r.z of the iteration (breakdown if 0 or not finite) and beta
__device__ __forceinline__ void rho_finish(PcgScalars* s, int first, double rho1) {
  if (rho1 == 0.0 || !finite_d(rho1)) {
    s->done = 1;
    s->status = 2;
    return;
  }
  if (first) {
    s->rho = rho1;
    s->beta = 0.0;
  } else {
    s->beta = __ddiv_rn(rho1, s->rho);
    s->rho = rho1;
  }
}

// p.q: stop at maxit, breakdown if 0 or not finite, else alpha
__device__ __forceinline__ void pq_finish(PcgScalars* s, double pq) {
  if (s->k >= s->maxit) {
    s->done = 1;
    s->status = 1;
    return;
  }
  if (pq == 0.0 || !finite_d(pq)) {
    s->done = 1;
    s->status = 2;
    return;
  }
  s->alpha = __ddiv_rn(s->rho, pq);
}

// r.r: count the iteration, converged or not finite
__device__ __forceinline__ void rr_finish(PcgScalars* s, double rr) {
  s->k += 1;
  double rn = __dsqrt_rn(rr);
  if (!finite_d(rn)) {
    s->done = 1;
    s->status = 2;
  } else if (rn <= __dmul_rn(s->rtol, s->bn)) {
    s->done = 1;
    s->status = 0;
  }
}

// one CTA: the total of the partials the previous kernel stored, then its
// scalar step (which: 0 rho, 1 p.q; 3: the (r, r) total of the update first
// -- count the iteration, stop if converged -- then, if going on, rho)
__global__ void k_pcg_fin(PcgArgs a, int which, int first) {
  PcgScalars* s = a.s;
  if (s->done) return;
  if (which == 3) {
    const double rr = cta_total(a.rrsum, a.ws.nb);
    __syncthreads();  // cta_total's scratch is reused
    const double rz = cta_total(a.ws.bsum, a.ws.nb);
    if (threadIdx.x != 0) return;
    rr_finish(s, rr);
    if (!s->done) rho_finish(s, 0, rz);
    return;
  }
  const double tot = cta_total(a.ws.bsum, a.ws.nb);
  if (threadIdx.x != 0) return;
  if (which == 0) rho_finish(s, first, tot);
  else pq_finish(s, tot);
}

// z = Prec(r), terms r_i z_i -> partials of rho (first = 1: initial rho, p =
// z follows).
// zonly: z of the rows up to kLongRow entries only, no inner product (the
// long rows run beside it in k_pcg_prec_long, k_pcg_rz follows both)
__global__ void k_pcg_prec(PcgArgs a, int first, int zonly) {
  if (a.s->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (a.sell.sptr) {  // S in sliced ELL (FP64 products)
    if (i < a.n) {
      if (zonly) {  // slot i holds row sperm[i]
        const int row = a.sperm ? a.sperm[i] : i;
        const int len = (int)(a.mrp[row + 1] - a.mrp[row]);
        if (len <= kLongRow) a.z[row] = sell_slot_chain(a.sell, len, a.r, i);
        return;
      }
      const double z = precond_sell(a, i);
      a.z[i] = z;
      term = __dmul_rn(a.r[i], z);
    }
  } else if (i < a.n) {
    double z = precond_apply(a, i);
    a.z[i] = z;
    term = __dmul_rn(a.r[i], z);
  }
  if (zonly) return;
  cta_partial(term, a.ws.bsum);
}

// terms r_i z_i -> partials of rho, after k_pcg_prec (zonly) and
// k_pcg_prec_long
__global__ void k_pcg_rz(PcgArgs a, int first) {
  if (a.s->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double term = i < a.n ? __dmul_rn(a.r[i], a.z[i]) : 0.0;
  cta_partial(term, a.ws.bsum);
}

// p = z (first) or p = fma(beta, p, z)
__global__ void k_pcg_dir(PcgArgs a, int first) {
  if (a.s->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double p = first ? a.z[i] : __fma_rn(a.s->beta, a.p[i], a.z[i]);
  a.p[i] = p;
  if (a.mixed) a.p32[i] = __double2float_rn(p);
}

// q = A p, terms p_i q_i -> partials of p.q
__global__ void k_pcg_spmv(PcgArgs a) {
  if (a.s->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    double q = a.mixed ? sell_chain_f32(a.A, a.aval32, a.p32, i) : sell_chain(a.A, a.p, i);
    a.q[i] = q;
    term = __dmul_rn(a.p[i], q);
  }
  cta_partial(term, a.ws.bsum);
}

// x += alpha p, r -= alpha q, terms r_i^2 -> partials of r.r
__global__ void k_pcg_update(PcgArgs a) {
  if (a.s->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    double al = a.s->alpha;
    a.x[i] = __fma_rn(al, a.p[i], a.x[i]);
    double r = __fma_rn(-al, a.q[i], a.r[i]);
    a.r[i] = r;
    if (a.mixed) a.r32[i] = __double2float_rn(r);
    term = __dmul_rn(r, r);
  }
  cta_partial(term, a.rrsum);
}

// ---------------------------------------------------------------- Lanczos
// Three-term recurrence on S (no reorthogonalisation), FP64: S v rows are
// fma chains over ascending column, inner products and norms the pairwise
// tree of reduce_finish; the coefficients stay on the device.

// ||v0|| with v0 in vc
__global__ void k_lz_norm0(LzArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    double x = a.vc[i];
    term = __dmul_rn(x, x);
  }
  double* nrm = a.nrm0;
  int* stt = a.state;
  reduce_finish(term, a.ws, [nrm, stt](double tot) {
    *nrm = __dsqrt_rn(tot);
    stt[0] = 0;
    stt[1] = (tot == 0.0 || !finite_d(tot)) ? 1 : 0;
  });
}

// v_1 = v0 / ||v0||, v_0 = 0
__global__ void k_lz_scale0(LzArgs a) {
  if (a.state[1]) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  a.vc[i] = __ddiv_rn(a.vc[i], *a.nrm0);
  a.vp[i] = 0.0;
}

// w = S v_j, alpha_j = (w, v_j)
__global__ void k_lz_av(LzArgs a, int j) {
  if (a.state[1]) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    double wi = row_chain(a.rp, a.ci, a.v, a.vc, i);
    a.w[i] = wi;
    term = __dmul_rn(wi, a.vc[i]);
  }
  double* al = a.alpha;
  reduce_finish(term, a.ws, [al, j](double tot) { al[j] = tot; });
}

// w = fma(-beta_{j-1}, v_{j-1}, fma(-alpha_j, v_j, w)), beta_j = ||w||
__global__ void k_lz_orth(LzArgs a, int j) {
  if (a.state[1]) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.n) {
    const double al = a.alpha[j], bp = j ? a.beta[j - 1] : 0.0;
    double wi = __fma_rn(-bp, a.vp[i], __fma_rn(-al, a.vc[i], a.w[i]));
    a.w[i] = wi;
    term = __dmul_rn(wi, wi);
  }
  double* be = a.beta;
  int* stt = a.state;
  reduce_finish(term, a.ws, [be, stt, j](double tot) {
    double b = __dsqrt_rn(tot);
    be[j] = b;
    stt[0] = j + 1;
    if (b == 0.0 || !finite_d(b)) stt[1] = 1;
  });
}

// v_{j-1} = v_j, v_{j+1} = w / beta_j
__global__ void k_lz_next(LzArgs a, int j) {
  if (a.state[1]) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double b = a.beta[j];
  a.vp[i] = a.vc[i];
  a.vc[i] = __ddiv_rn(a.w[i], b);
}

cudaError_t launch_lz_start(const LzArgs& a, cudaStream_t st) {
  int g = (a.n + 255) / 256;
  k_lz_norm0<<<g, 256, 0, st>>>(a);
  k_lz_scale0<<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_lz_step(const LzArgs& a, int j, cudaStream_t st) {
  int g = (a.n + 255) / 256;
  k_lz_av<<<g, 256, 0, st>>>(a, j);
  k_lz_orth<<<g, 256, 0, st>>>(a, j);
  k_lz_next<<<g, 256, 0, st>>>(a, j);
  return cudaGetLastError();
}

// z = Prec(r) and rho: with rows longer than kLongRow (and a second stream),
// the long rows run on st2 beside the others on st, and k_pcg_rz joins them
static cudaError_t launch_pcg_prec(const PcgArgs& a, int first, int fin, const PcgFork& f,
                                   cudaStream_t st) {
  int g = (a.n + 255) / 256;
  if (!a.nlong) {
    k_pcg_prec<<<g, 256, 0, st>>>(a, first, 0);
    k_pcg_fin<<<1, 256, 0, st>>>(a, fin, first);
    return cudaGetLastError();
  }
  if (!f.st2) {
    k_pcg_prec_long<<<a.nlong, 32, 0, st>>>(a);
    k_pcg_prec<<<g, 256, 0, st>>>(a, first, 1);
    k_pcg_rz<<<g, 256, 0, st>>>(a, first);
    k_pcg_fin<<<1, 256, 0, st>>>(a, fin, first);
    return cudaGetLastError();
  }
  cudaError_t e = cudaEventRecord(f.fork, st);
  if (!e) e = cudaStreamWaitEvent(f.st2, f.fork, 0);
  if (e) return e;
  k_pcg_prec_long<<<a.nlong, 32, 0, f.st2>>>(a);
  e = cudaEventRecord(f.join, f.st2);
  if (e) return e;
  k_pcg_prec<<<g, 256, 0, st>>>(a, first, 1);
  e = cudaStreamWaitEvent(st, f.join, 0);
  if (e) return e;
  k_pcg_rz<<<g, 256, 0, st>>>(a, first);
  k_pcg_fin<<<1, 256, 0, st>>>(a, fin, first);
  return cudaGetLastError();
}

cudaError_t launch_pcg_init(const PcgArgs& a, const PcgFork& f, cudaStream_t st) {
  int g = (a.n + 255) / 256;
  k_pcg_init<<<g, 256, 0, st>>>(a);
  cudaError_t e = launch_pcg_prec(a, 1, 0, f, st);
  if (e) return e;
  k_pcg_dir<<<g, 256, 0, st>>>(a, 1);
  return cudaGetLastError();
}

cudaError_t launch_pcg_iter(const PcgArgs& a, const PcgFork& f, cudaStream_t st) {
  int g = (a.n + 255) / 256;
  k_pcg_spmv<<<g, 256, 0, st>>>(a);
  k_pcg_fin<<<1, 256, 0, st>>>(a, 1, 0);
  k_pcg_update<<<g, 256, 0, st>>>(a);
  // the preconditioner product runs before the update's (r, r) is totalled:
  // its fin counts the iteration and stops on convergence before it forms
  // rho, so a converged last iteration only forms a z that is not used
  cudaError_t e = launch_pcg_prec(a, 0, 3, f, st);
  if (e) return e;
  k_pcg_dir<<<g, 256, 0, st>>>(a, 0);
  return cudaGetLastError();
}

cudaError_t launch_true_res(const PcgArgs& a, cudaStream_t st) {
  k_true_res<<<(a.n + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace spai
