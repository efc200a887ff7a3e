// Global dropping operators (Sec. 6.1 Eq. 6.2 with a global density cap,
// Appendix A's heuristic for M).  A global selection of t entries by
// (key, position) is found exactly with two radix selects of four 16-bit
// digits each: first the t-th smallest 64-bit key u*, then, among the
// entries with key u*, the position (column << 32 | row) p* that completes
// the count; an entry is selected when u < u* or (u == u* and pos <= p*).
// The host drives the digits (one histogram kernel per digit); the
// compaction keeps each column's remaining entries in their slab order.
#include <stdint.h>

#include "common.cuh"
#include "dropping.cuh"

namespace spai {

namespace {

__device__ __forceinline__ unsigned long long value_key(const SelArgs& a, long long e, bool& ok) {
  ok = true;
  if (a.mode == 0) {  // larger |v| first
    unsigned long long bits;
    if (a.vs == 4) {
      bits = (unsigned long long)(__float_as_uint(((const float*)a.vals)[e]) & 0x7fffffffu);
    } else {
      bits = (unsigned long long)__double_as_longlong(((const double*)a.vals)[e]) & 0x7fffffffffffffffull;
    }
    return ~bits;
  }
  const double s = a.score[e];  // smaller score first; +inf is not eligible
  if (s == __longlong_as_double(0x7ff0000000000000ll)) {
    ok = false;
    return 0ull;
  }
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_sel_hist(SelArgs a) {
  const int lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= a.n) return;
  const long long off = a.off[j];
  const int L = a.len[j];
  for (int e = lane; e < L; e += 32) {
    bool ok;
    const unsigned long long u = value_key(a, off + e, ok);
    if (!ok) continue;
    unsigned long long key = u;
    if (a.stage == 1) {
      if (u != a.ustar) continue;
      key = ((unsigned long long)j << 32) | (unsigned)a.rows[off + e];
    }
    if ((key & a.mask) != a.prefix) continue;
    atomicAdd(&a.hist[(key >> a.shift) & 0xffffull], 1u);
  }
}

__global__ void k_sel_compact(SelArgs a) {
  const int lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= a.n) return;
  const long long off = a.off[j];
  const int L = a.len[j];
  int out = 0;
  for (int base = 0; base < L; base += 32) {
    const int e = base + lane;
    int r = 0;
    double vd = 0.0;
    float vf = 0.0f;
    bool keep = false;
    if (e < L) {
      r = a.rows[off + e];
      if (a.vs == 4) vf = ((const float*)a.vals)[off + e];
      else vd = ((const double*)a.vals)[off + e];
      bool ok;
      const unsigned long long u = value_key(a, off + e, ok);
      const unsigned long long pos = ((unsigned long long)j << 32) | (unsigned)r;
      const bool sel = ok && (u < a.ustar || (u == a.ustar && pos <= a.pstar));
      keep = a.keep_selected ? sel : !sel;
    }
    __syncwarp();
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int p = out + __popc(b & ((1u << lane) - 1u));
      a.rows[off + p] = r;
      if (a.vs == 4) ((float*)a.vals)[off + p] = vf;
      else ((double*)a.vals)[off + p] = vd;
    }
    out += __popc(b);
    __syncwarp();
  }
  if (lane == 0) a.len[j] = out;
}

// ||A e_k||^2 = sum_t a_kt^2 over row k (A symmetric), an FP64 fma chain
__global__ void k_anrm(int n, int W, const int* ell_col, const void* ell_val, int vs, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double acc = 0.0;
  for (int t = 0; t < W; t++) {
    if (ell_col[(long long)k * W + t] < 0) break;
    const double a = vs == 4 ? (double)((const float*)ell_val)[(long long)k * W + t]
                             : ((const double*)ell_val)[(long long)k * W + t];
    acc = __fma_rn(a, a, acc);
  }
  out[k] = acc;
}

__global__ void k_sym_to_slab(int n, const long long* srp, const int* sci, const double* sv,
                              const long long* off, const int* cap, int* rows, void* vals,
                              int* len, int vs, double u, int* ovf) {
  const int lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const long long b0 = srp[j], b1 = srp[j + 1];
  const long long o = off[j];
  const int c = cap[j];
  int out = 0;
  for (long long base = b0; base < b1; base += 32) {
    const long long e = base + lane;
    bool keep = false;
    int r = 0;
    double v = 0.0;
    if (e < b1) {
      r = sci[e];
      v = sv[e];
      if (vs == 4) v = (double)(float)v;
      keep = v != 0.0 && (r == (int)j || fabs(v) >= u);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int p = out + __popc(bal & ((1u << lane) - 1u));
      if (p < c) {
        rows[o + p] = r;
        if (vs == 4) ((float*)vals)[o + p] = (float)v;
        else ((double*)vals)[o + p] = v;
      }
    }
    out += __popc(bal);
  }
  if (lane == 0) {
    if (out > c) {
      atomicOr(ovf, 1);
      out = c;
    }
    len[j] = out;
  }
}

inline unsigned warp_grid(long long n) { return (unsigned)((n + 7) / 8); }

}  // namespace

cudaError_t launch_sel_hist(const SelArgs& a, cudaStream_t st) {
  k_sel_hist<<<warp_grid(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sel_compact(const SelArgs& a, cudaStream_t st) {
  k_sel_compact<<<warp_grid(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_anrm(int n, int W, const int* ell_col, const void* ell_val, int vs, double* out,
                        cudaStream_t st) {
  k_anrm<<<(n + 255) / 256, 256, 0, st>>>(n, W, ell_col, ell_val, vs, out);
  return cudaGetLastError();
}

cudaError_t launch_sym_to_slab(int n, const long long* srp, const int* sci, const double* sv,
                               const long long* off, const int* cap, int* rows, void* vals,
                               int* len, int vs, double u, int* ovf, cudaStream_t st) {
  k_sym_to_slab<<<warp_grid(n), 256, 0, st>>>(n, srp, sci, sv, off, cap, rows, vals, len, vs, u, ovf);
  return cudaGetLastError();
}

}  // namespace spai
