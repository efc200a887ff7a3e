// Differentiation of fixed-pattern MR and LOMR (no counterpart in the paper;
// the objective and its gradient form are Sec. 2 and Sec. 3 Eq. (gradient)):
//   MR (Algorithm 1 on S):  M_0 = diag(A)^{-1};  R_i = I - A M_i;
//     P_i = mask_S(R_i);  Q_i = A P_i;  alpha_i = (R_i, Q_i)_F / (Q_i, Q_i)_F;
//     M_{i+1} = M_i + alpha_i P_i;
//   LOMR (Algorithm 4 / Theorem 3 on S):  P_{-1} = 0;  Z_i = mask_S(R_i);
//     U = A Z_i;  V = A P_{i-1};  (delta_i, gamma_i) from the 2x2 normal
//     equations in (U,U), (V,V), (U,V), (U,R_i), (V,R_i), or the MR step
//     delta_i = (U,R_i)/(U,U), gamma_i = 0 when (V,V) = 0 or the system is
//     near singular;  S_i = delta_i Z_i + gamma_i P_{i-1};  M_{i+1} = M_i + S_i;
//     P_i = S_i;
//   L = ||I - A M_K||_F^2,  S = supp(A),
// and dL/dA over A's stored entries (independent values) by reverse mode.
//
// Every matrix lives on one of two fixed patterns: S (A, M_i, P_i and their
// adjoints, in A's CSR order) and T = supp(A S) + I (R_i, Q_i and their
// adjoints, CSR).  The three sparse products the method and its adjoint need
//   Y = A X            Y[r,j]  = sum_k a_rk x_kj      (T <- S, S)
//   mask_S(A^T dY)     dX[k,j] = sum_r a_rk dy_rj     (S <- S, T)
//   mask_S(dY X^T)     dA[r,k] = sum_j dy_rj x_kj     (S <- T, S)
// are lists of (index, index) pairs grouped by output entry, built once on
// the host in the order of the fma chain (ascending inner index) by merging
// sorted rows, so the GPU side is a gather-fma per output entry.  The
// backward pass recomputes R_i, P_i, Q_i from the stored M_i (one checkpoint
// per step, and of P_{i-1} for LOMR).  Values are FP64, or FP32 on the mixed
// path (FP32 products and
// stored values; inner products, step scalars and the axpy arithmetic in
// FP64, each stored value rounded once).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "spai.h"
#include "vec_kernels.cuh"

namespace {

struct ProdList {
  long long* ptr = nullptr;  // [nout + 1]
  int* ia = nullptr;         // first operand index
  int* ib = nullptr;         // second operand index
  long long nout = 0, len = 0;
};

}  // namespace

struct spai_fpmr_ctx {
  int n = 0, K = 0;
  int method = SPAI_MR;    // SPAI_MR or SPAI_LOMR
  long long nS = 0, nT = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int* d_diagS = nullptr;  // [n] position of (j,j) in S
  int* d_diagT = nullptr;  // [n] position of (j,j) in T
  int* d_s2t = nullptr;    // [nS] position of S's entry in T
  ProdList Y, X, D;        // the three products (see above)
  int vs = 8;               // bytes per stored value (8 FP64, 4 FP32)
  void *d_A = nullptr, *d_Mck = nullptr, *d_P = nullptr, *d_dM = nullptr, *d_dP = nullptr,
       *d_dA = nullptr;
  void *d_R = nullptr, *d_Q = nullptr, *d_dR = nullptr, *d_dQ = nullptr;
  // LOMR: checkpoints P_{i-1} ([K+1][nS], P_{-1} = 0 first), V = A P_{i-1}
  // and its adjoint on T, dS, dP_{i-1} and the incoming dP_i on S
  void *d_Pck = nullptr, *d_V = nullptr, *d_dV = nullptr, *d_dS = nullptr, *d_dPp = nullptr,
       *d_dPn = nullptr;
  std::vector<double> delta, gamma, prod;  // prod: uu, vv, uv, ur, vr per step
  std::vector<char> mrstep;
  double *d_part = nullptr, *d_res = nullptr, *d_stage = nullptr;
  std::vector<double> alpha, num, den;
  std::vector<double> diag;  // a_jj of the last forward values
  bool have_forward = false;
  long long launches = 0;
};

namespace {

#define FCK(x)                                                                \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      (void)cudaGetLastError();                                               \
      return e_ == cudaErrorMemoryAllocation ? SPAI_ERR_OOM : SPAI_ERR_CUDA;  \
    }                                                                         \
  } while (0)

template <typename T>
int falloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return SPAI_ERR_OOM;
  }
  return SPAI_OK;
}

template <typename T>
void ffree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

int valloc(void** p, size_t count, int vs) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(p, (size_t)vs * count) != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return SPAI_ERR_OOM;
  }
  return SPAI_OK;
}

constexpr int kDotChunk = 16;     // elements per thread in the dot partials
constexpr int kDotBlock = 256;

__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// out[s] (=|+=) scale * sum_t a[ia[t]] b[ib[t]] over t in [ptr[s], ptr[s+1]),
// an fma chain in list order in the value type; scale and accumulation in
// FP64, rounded once
template <typename T>
__global__ void k_seg_prod(long long nout, const long long* ptr, const int* ia, const int* ib,
                           const T* a, const T* b, T* out, double scale, int acc) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nout) return;
  T v = T(0);
  for (long long t = ptr[s]; t < ptr[s + 1]; t++) v = fma_t(a[ia[t]], b[ib[t]], v);
  double w = __dmul_rn(scale, (double)v);
  out[s] = (T)(acc ? __dadd_rn((double)out[s], w) : w);
}

template <typename T>
__global__ void k_add_diag(int n, const int* diag, T* x, double v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[diag[j]] = (T)__dadd_rn((double)x[diag[j]], v);
}

template <typename T>
__global__ void k_gather(long long m, const int* idx, const T* src, T* dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) dst[e] = src[idx[e]];
}

template <typename T>
__global__ void k_scatter_add(long long m, const int* idx, const T* src, T* dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) dst[idx[e]] = (T)__dadd_rn((double)dst[idx[e]], (double)src[e]);
}

// y = a x + b y in FP64 (b == 0: y = a x), rounded to the value type
template <typename T>
__global__ void k_axby(long long m, double a, const T* x, double b, T* y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m)
    y[e] = (T)(b == 0.0 ? __dmul_rn(a, (double)x[e])
                        : __fma_rn(a, (double)x[e], __dmul_rn(b, (double)y[e])));
}

// z = a x + b y in FP64, rounded to the value type
template <typename T>
__global__ void k_lin2(long long m, double a, const T* x, double b, const T* y, T* z) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) z[e] = (T)__fma_rn(a, (double)x[e], __dmul_rn(b, (double)y[e]));
}

// z = a x + b y + c w as fma(a, x, fma(b, y, c w)) in FP64, rounded to the value type
template <typename T>
__global__ void k_lin3(long long m, double a, const T* x, double b, const T* y, double c,
                       const T* w, T* z) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m)
    z[e] = (T)__fma_rn(a, (double)x[e], __fma_rn(b, (double)y[e], __dmul_rn(c, (double)w[e])));
}

template <typename T>
__global__ void k_copy(long long m, const T* x, T* y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) y[e] = x[e];
}

template <typename T>
__global__ void k_from_f64(long long m, const double* x, T* y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) y[e] = (T)x[e];
}

template <typename T>
__global__ void k_to_f64(long long m, const T* x, double* y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) y[e] = (double)x[e];
}

// M0 = diag(A)^{-1} on S: zero everywhere (k_m0), then the diagonal
template <typename T>
__global__ void k_m0(long long nS, T* M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nS) M[e] = T(0);
}
template <typename T>
__global__ void k_m0_diag(int n, const int* diag, const T* A, T* M) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) M[diag[j]] = (T)__ddiv_rn(1.0, (double)A[diag[j]]);
}

// dA[(j,j)] -= dM[(j,j)] / a_jj^2  (through M_0 = diag(A)^{-1})
template <typename T>
__global__ void k_m0_adjoint(int n, const int* diag, const T* A, const T* dM, T* dA) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double a = (double)A[diag[j]];
  dA[diag[j]] = (T)__dsub_rn((double)dA[diag[j]], __ddiv_rn((double)dM[diag[j]], __dmul_rn(a, a)));
}

__device__ __forceinline__ double warp_sum32(double v) {
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

// per block: kDotBlock * kDotChunk consecutive products x_e y_e (promoted to
// FP64) summed in a fixed order (sequential per thread, then a tree)
template <typename T>
__global__ void k_dot_part(long long m, const T* x, const T* y, double* part) {
  __shared__ double red[kDotBlock / 32];
  const long long base = (long long)blockIdx.x * kDotBlock * kDotChunk + threadIdx.x * kDotChunk;
  double s = 0.0;
  for (int t = 0; t < kDotChunk; t++) {
    const long long e = base + t;
    if (e < m) s = __fma_rn((double)x[e], (double)y[e], s);
  }
  s = warp_sum32(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kDotBlock / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum32(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_dot_final(long long nb, const double* part, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long b = threadIdx.x; b < nb; b += blockDim.x) s = __dadd_rn(s, part[b]);
  s = warp_sum32(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum32(v);
    if (threadIdx.x == 0) *out = v;
  }
}

inline unsigned nblk(long long m) { return (unsigned)((m + 255) / 256); }

// the kernels above for the handle's value type
template <typename T>
struct Ops {
  static int seg_prod(spai_fpmr_ctx* h, const ProdList& L, const void* a, const void* b, void* out,
                      double scale, int acc) {
    k_seg_prod<T><<<nblk(L.nout), 256, 0, h->stream>>>(L.nout, L.ptr, L.ia, L.ib, (const T*)a,
                                                        (const T*)b, (T*)out, scale, acc);
    h->launches++;
    FCK(cudaGetLastError());
    return SPAI_OK;
  }
  static int dot(spai_fpmr_ctx* h, long long m, const void* x, const void* y, int slot) {
    const long long nb = (m + (long long)kDotBlock * kDotChunk - 1) / ((long long)kDotBlock * kDotChunk);
    k_dot_part<T><<<(unsigned)std::max(nb, 1LL), kDotBlock, 0, h->stream>>>(m, (const T*)x, (const T*)y,
                                                                            h->d_part);
    k_dot_final<<<1, 1024, 0, h->stream>>>(std::max(nb, 1LL), h->d_part, h->d_res + slot);
    h->launches += 2;
    FCK(cudaGetLastError());
    return SPAI_OK;
  }
};

int seg_prod(spai_fpmr_ctx* h, const ProdList& L, const void* a, const void* b, void* out,
             double scale, int acc) {
  return h->vs == 4 ? Ops<float>::seg_prod(h, L, a, b, out, scale, acc)
                    : Ops<double>::seg_prod(h, L, a, b, out, scale, acc);
}

// (x, y) over m entries, into h->d_res[slot] (device)
int dot(spai_fpmr_ctx* h, long long m, const void* x, const void* y, int slot) {
  return h->vs == 4 ? Ops<float>::dot(h, m, x, y, slot) : Ops<double>::dot(h, m, x, y, slot);
}

inline void* at(void* base, int vs, long long idx) { return (char*)base + (size_t)vs * idx; }

// launch KERNEL<T_> with T_ the handle's value type (T_ may appear in the
// arguments)
#define FP_DISPATCH(h, KERNEL, GRID, ...)                                          \
  do {                                                                             \
    if ((h)->vs == 4) {                                                            \
      using T_ = float;                                                            \
      KERNEL<T_><<<(GRID), 256, 0, (h)->stream>>>(__VA_ARGS__);                    \
    } else {                                                                       \
      using T_ = double;                                                           \
      KERNEL<T_><<<(GRID), 256, 0, (h)->stream>>>(__VA_ARGS__);                    \
    }                                                                              \
    (h)->launches++;                                                               \
  } while (0)

int read_res(spai_fpmr_ctx* h, double* out, int count) {
  FCK(cudaMemcpyAsync(out, h->d_res, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
  FCK(cudaStreamSynchronize(h->stream));
  return SPAI_OK;
}

// R = I - A M (on T), P = mask_S(R), Q = A P
int step_products(spai_fpmr_ctx* h, const void* M, bool want_q) {
  int rc = seg_prod(h, h->Y, h->d_A, M, h->d_R, -1.0, 0);
  if (rc) return rc;
  if (h->vs == 4) {
    k_add_diag<float><<<nblk(h->n), 256, 0, h->stream>>>(h->n, h->d_diagT, (float*)h->d_R, 1.0);
    k_gather<float><<<nblk(h->nS), 256, 0, h->stream>>>(h->nS, h->d_s2t, (const float*)h->d_R,
                                                        (float*)h->d_P);
  } else {
    k_add_diag<double><<<nblk(h->n), 256, 0, h->stream>>>(h->n, h->d_diagT, (double*)h->d_R, 1.0);
    k_gather<double><<<nblk(h->nS), 256, 0, h->stream>>>(h->nS, h->d_s2t, (const double*)h->d_R,
                                                         (double*)h->d_P);
  }
  h->launches += 2;
  FCK(cudaGetLastError());
  if (want_q) return seg_prod(h, h->Y, h->d_A, h->d_P, h->d_Q, 1.0, 0);
  return SPAI_OK;
}

void free_list(ProdList& L) {
  ffree(L.ptr);
  ffree(L.ia);
  ffree(L.ib);
}

void free_fpmr(spai_fpmr_ctx* h) {
  ffree(h->d_diagS);
  ffree(h->d_diagT);
  ffree(h->d_s2t);
  free_list(h->Y);
  free_list(h->X);
  free_list(h->D);
  ffree(h->d_A);
  ffree(h->d_Mck);
  ffree(h->d_P);
  ffree(h->d_dM);
  ffree(h->d_dP);
  ffree(h->d_dA);
  ffree(h->d_R);
  ffree(h->d_Q);
  ffree(h->d_dR);
  ffree(h->d_dQ);
  ffree(h->d_Pck);
  ffree(h->d_V);
  ffree(h->d_dV);
  ffree(h->d_dS);
  ffree(h->d_dPp);
  ffree(h->d_dPn);
  ffree(h->d_part);
  ffree(h->d_res);
  ffree(h->d_stage);
}

int upload_list(ProdList& L, const std::vector<long long>& ptr, const std::vector<int>& ia,
                const std::vector<int>& ib, cudaStream_t st) {
  L.nout = (long long)ptr.size() - 1;
  L.len = (long long)ia.size();
  int rc = falloc(&L.ptr, ptr.size());
  if (!rc) rc = falloc(&L.ia, ia.size());
  if (!rc) rc = falloc(&L.ib, ib.size());
  if (rc) return rc;
  FCK(cudaMemcpyAsync(L.ptr, ptr.data(), sizeof(long long) * ptr.size(), cudaMemcpyHostToDevice, st));
  if (!ia.empty()) {
    FCK(cudaMemcpyAsync(L.ia, ia.data(), sizeof(int) * ia.size(), cudaMemcpyHostToDevice, st));
    FCK(cudaMemcpyAsync(L.ib, ib.data(), sizeof(int) * ib.size(), cudaMemcpyHostToDevice, st));
  }
  FCK(cudaStreamSynchronize(st));
  return SPAI_OK;
}

// position of column c in row r of a CSR pattern, -1 if absent
inline long long find_pos(const std::vector<long long>& ptr, const std::vector<int>& col, int r, int c) {
  const int* b = col.data() + ptr[r];
  const int* e = col.data() + ptr[r + 1];
  const int* f = std::lower_bound(b, e, c);
  return (f != e && *f == c) ? (long long)(f - col.data()) : -1;
}

// ------------------------------------------------ set-up on the device
// The patterns and product lists of spai_fpmr_create, built on the GPU when
// A's rows hold at most kSetupW entries: thread per row, two passes (count,
// then fill at the exclusive scan of the counts), so every list comes out
// in the order the host construction gives: output entries in CSR order,
// each with its pairs in ascending inner index.
constexpr int kSetupW = 64;

__device__ __forceinline__ int dfind(const int* col, long long b, long long e, int c) {
  while (b < e) {  // position of c in col[b, e) (sorted), or -1
    const long long m = (b + e) >> 1;
    const int x = col[m];
    if (x == c) return (int)m;
    if (x < c) b = m + 1;
    else e = m;
  }
  return -1;
}
__device__ __forceinline__ long long dfind64(const int* col, long long b, long long e, int c) {
  while (b < e) {
    const long long m = (b + e) >> 1;
    const int x = col[m];
    if (x == c) return m;
    if (x < c) b = m + 1;
    else e = m;
  }
  return -1;
}

// rows strictly ascending and in range: err[0] = 1 on any violation
__global__ void k_su_check(int n, const int* sp, const int* sc, int* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int b = sp[r], e = sp[r + 1];
  if (e < b) {
    atomicOr(err, 1);
    return;
  }
  for (int q = b; q < e; q++)
    if (sc[q] < 0 || sc[q] >= n || (q > b && sc[q] <= sc[q - 1])) atomicOr(err, 1);
}

// first row without a diagonal (err[1]) and first row with an entry whose
// mirror is missing (err[2]), as atomicMin over the row index
__global__ void k_su_diag_sym(int n, const int* sp, const int* sc, int* diagS, int* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int d = dfind(sc, sp[r], sp[r + 1], r);
  diagS[r] = d;
  if (d < 0) atomicMin(err + 1, r);
  for (int q = sp[r]; q < sp[r + 1]; q++) {
    const int c = sc[q];
    if (dfind(sc, sp[c], sp[c + 1], r) < 0) {
      atomicMin(err + 2, r);
      break;
    }
  }
}

// T(r) = {r} u union over k in S(r) of S(k), sorted: a merge of the rows k
// (at most kSetupW of them) by their heads.  fill = 0: count into tlen[r].
__global__ void k_su_trow(int n, const int* sp, const int* sc, int* tlen, const long long* tp,
                          int* tc, int fill) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int head[kSetupW];
  const int b = sp[r], L = sp[r + 1] - b;
  for (int t = 0; t < L; t++) head[t] = sp[sc[b + t]];
  long long out = fill ? tp[r] : 0;
  int cnt = 0, last = -1;
  bool diag_done = false;
  for (;;) {
    int best = 0x7fffffff;
    for (int t = 0; t < L; t++) {
      const int k = sc[b + t];
      if (head[t] < sp[k + 1]) best = min(best, sc[head[t]]);
    }
    if (!diag_done && r < best) best = r;  // the identity's entry
    if (best == 0x7fffffff) break;
    if (best == r) diag_done = true;
    for (int t = 0; t < L; t++) {
      const int k = sc[b + t];
      if (head[t] < sp[k + 1] && sc[head[t]] == best) head[t]++;
    }
    if (best != last) {
      if (fill) tc[out + cnt] = best;
      cnt++;
      last = best;
    }
  }
  if (!fill) tlen[r] = cnt;
}

// s2t (S entry -> its T position) and diagT
__global__ void k_su_s2t(int n, const int* sp, const int* sc, const long long* tp, const int* tc,
                         int* s2t, int* diagT) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int q = sp[r]; q < sp[r + 1]; q++) s2t[q] = (int)dfind64(tc, tp[r], tp[r + 1], sc[q]);
  diagT[r] = (int)dfind64(tc, tp[r], tp[r + 1], r);
}

// Y = A X: for (r,j) in T, k over S(r) merged with S(j); pairs (a_rk, x_kj)
__global__ void k_su_y(int n, const int* sp, const int* sc, const long long* tp, const int* tc,
                       int* cnt, const long long* ptr, int* ia, int* ib, int fill) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (long long f = tp[r]; f < tp[r + 1]; f++) {
    const int j = tc[f];
    int p = sp[r], q = sp[j], c = 0;
    long long o = fill ? ptr[f] : 0;
    while (p < sp[r + 1] && q < sp[j + 1]) {
      if (sc[p] < sc[q]) p++;
      else if (sc[q] < sc[p]) q++;
      else {
        if (fill) {
          const int k = sc[p];
          ia[o + c] = p;
          ib[o + c] = dfind(sc, sp[k], sp[k + 1], j);
        }
        c++;
        p++;
        q++;
      }
    }
    if (!fill) cnt[f] = c;
  }
}

// dX[k,j] = sum_r a_rk dy_rj: r over S(k) merged with T(j); pairs (a_rk, dy_rj)
__global__ void k_su_x(int n, const int* sp, const int* sc, const long long* tp, const int* tc,
                       int* cnt, const long long* ptr, int* ia, int* ib, int fill) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  for (int e = sp[k]; e < sp[k + 1]; e++) {
    const int j = sc[e];
    int p = sp[k];
    long long q = tp[j];
    int c = 0;
    long long o = fill ? ptr[e] : 0;
    while (p < sp[k + 1] && q < tp[j + 1]) {
      if (sc[p] < tc[q]) p++;
      else if (tc[q] < sc[p]) q++;
      else {
        if (fill) {
          const int r = sc[p];
          ia[o + c] = dfind(sc, sp[r], sp[r + 1], k);
          ib[o + c] = (int)dfind64(tc, tp[r], tp[r + 1], j);
        }
        c++;
        p++;
        q++;
      }
    }
    if (!fill) cnt[e] = c;
  }
}

// dA[r,k] = sum_j dy_rj x_kj: j over T(r) merged with S(k); pairs (dy_rj, x_kj)
__global__ void k_su_d(int n, const int* sp, const int* sc, const long long* tp, const int* tc,
                       int* cnt, const long long* ptr, int* ia, int* ib, int fill) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int e = sp[r]; e < sp[r + 1]; e++) {
    const int k = sc[e];
    long long p = tp[r];
    int q = sp[k], c = 0;
    long long o = fill ? ptr[e] : 0;
    while (p < tp[r + 1] && q < sp[k + 1]) {
      if (tc[p] < sc[q]) p++;
      else if (sc[q] < tc[p]) q++;
      else {
        if (fill) {
          ia[o + c] = (int)p;
          ib[o + c] = q;
        }
        c++;
        p++;
        q++;
      }
    }
    if (!fill) cnt[e] = c;
  }
}

// LOMR's step coefficients from uu, vv, uv, ur, vr (the same formulas and
// fallback as the column pass); returns true for an MR step (gamma = 0)
bool lomr_coef(const double* t, double* delta, double* gamma) {
  const double uu = t[0], vv = t[1], uv = t[2], ur = t[3], vr = t[4];
  const double t1 = uu * vv, t2 = uv * uv, cc = t1 - t2;
  if (vv == 0.0 || cc <= (64.0 * 2.220446049250313e-16) * t1) {
    *delta = ur / uu;
    *gamma = 0.0;
    return true;
  }
  const double d1 = vv * ur, d2 = uv * vr, g1 = uu * vr, g2 = uv * ur;
  *delta = (d1 - d2) / cc;
  *gamma = (g1 - g2) / cc;
  return false;
}

// LOMR buffers, allocated when the method is chosen
int alloc_lomr(spai_fpmr_ctx* h) {
  if (h->d_Pck) return SPAI_OK;
  const int vs = h->vs;
  int rc = valloc(&h->d_Pck, (size_t)(h->K + 1) * h->nS, vs);
  rc = rc ? rc : valloc(&h->d_V, h->nT, vs);
  rc = rc ? rc : valloc(&h->d_dV, h->nT, vs);
  rc = rc ? rc : valloc(&h->d_dS, h->nS, vs);
  rc = rc ? rc : valloc(&h->d_dPp, h->nS, vs);
  rc = rc ? rc : valloc(&h->d_dPn, h->nS, vs);
  if (rc) {
    ffree(h->d_Pck);
    ffree(h->d_V);
    ffree(h->d_dV);
    ffree(h->d_dS);
    ffree(h->d_dPp);
    ffree(h->d_dPn);
  }
  return rc;
}

// K LOMR steps from the M_0 already in the first checkpoint; loss in *loss
int forward_lomr(spai_fpmr_ctx* h, double* loss) {
  const long long nS = h->nS, nT = h->nT;
  const int vs = h->vs, K = h->K;
  FP_DISPATCH(h, k_m0, nblk(nS), nS, (T_*)h->d_Pck);  // P_{-1} = 0
  FCK(cudaGetLastError());
  h->delta.assign(K, 0.0);
  h->gamma.assign(K, 0.0);
  h->prod.assign(5 * (size_t)K, 0.0);
  h->mrstep.assign(K, 0);
  for (int i = 0; i < K; i++) {
    void* M = at(h->d_Mck, vs, (long long)i * nS);
    void* Mn = at(h->d_Mck, vs, (long long)(i + 1) * nS);
    void* Pp = at(h->d_Pck, vs, (long long)i * nS);
    void* Pn = at(h->d_Pck, vs, (long long)(i + 1) * nS);
    // R, Z = mask_S(R) (in d_P), U = A Z (in d_Q), V = A P_{i-1}
    int rc = step_products(h, M, true);
    if (!rc) rc = seg_prod(h, h->Y, h->d_A, Pp, h->d_V, 1.0, 0);
    if (!rc) rc = dot(h, nT, h->d_Q, h->d_Q, 0);
    if (!rc) rc = dot(h, nT, h->d_V, h->d_V, 1);
    if (!rc) rc = dot(h, nT, h->d_Q, h->d_V, 2);
    if (!rc) rc = dot(h, nT, h->d_Q, h->d_R, 3);
    if (!rc) rc = dot(h, nT, h->d_V, h->d_R, 4);
    double t[5];
    if (!rc) rc = read_res(h, t, 5);
    if (rc) return rc;
    if (!(t[0] > 0.0)) return SPAI_ERR_NONFINITE;
    double d, g;
    h->mrstep[i] = lomr_coef(t, &d, &g) ? 1 : 0;
    if (!std::isfinite(d) || !std::isfinite(g)) return SPAI_ERR_NONFINITE;
    h->delta[i] = d;
    h->gamma[i] = g;
    for (int q = 0; q < 5; q++) h->prod[5 * (size_t)i + q] = t[q];
    // S = delta Z + gamma P_{i-1} (= P_i);  M_{i+1} = M_i + S
    FP_DISPATCH(h, k_lin2, nblk(nS), nS, d, (const T_*)h->d_P, g, (const T_*)Pp, (T_*)Pn);
    FP_DISPATCH(h, k_copy, nblk(nS), nS, (const T_*)M, (T_*)Mn);
    FP_DISPATCH(h, k_axby, nblk(nS), nS, 1.0, (const T_*)Pn, 1.0, (T_*)Mn);
    FCK(cudaGetLastError());
  }
  int rc = step_products(h, at(h->d_Mck, vs, (long long)K * nS), false);
  if (!rc) rc = dot(h, nT, h->d_R, h->d_R, 0);
  if (!rc) rc = read_res(h, loss, 1);
  return rc;
}

// reverse mode through the K LOMR steps; dA (d_dA) and dM (d_dM) already
// hold the contributions of the final residual
int backward_lomr(spai_fpmr_ctx* h) {
  const long long nS = h->nS, nT = h->nT;
  const int vs = h->vs;
  FP_DISPATCH(h, k_m0, nblk(nS), nS, (T_*)h->d_dPn);  // nothing flows into P_{K-1}
  FCK(cudaGetLastError());
  for (int i = h->K - 1; i >= 0; i--) {
    const void* M = at(h->d_Mck, vs, (long long)i * nS);
    const void* Pp = at(h->d_Pck, vs, (long long)i * nS);
    const double d = h->delta[i], g = h->gamma[i];
    const double* t = &h->prod[5 * (size_t)i];
    const double uu = t[0], vv = t[1], uv = t[2], ur = t[3], vr = t[4];
    int rc = step_products(h, M, true);  // R, Z (d_P), U (d_Q)
    if (!rc) rc = seg_prod(h, h->Y, h->d_A, Pp, h->d_V, 1.0, 0);
    if (rc) return rc;
    // dS = dM_{i+1} + dP_i;  d(delta) = (dS, Z), d(gamma) = (dS, P_{i-1})
    FP_DISPATCH(h, k_lin2, nblk(nS), nS, 1.0, (const T_*)h->d_dM, 1.0, (const T_*)h->d_dPn,
                (T_*)h->d_dS);
    FCK(cudaGetLastError());
    rc = dot(h, nS, h->d_dS, h->d_P, 0);
    if (!rc) rc = dot(h, nS, h->d_dS, Pp, 1);
    double dg2[2];
    if (!rc) rc = read_res(h, dg2, 2);
    if (rc) return rc;
    const double dd = dg2[0], dgam = dg2[1];
    double duu, dvv, duv, dur, dvr;
    if (h->mrstep[i]) {
      duu = -dd * d / uu;
      dur = dd / uu;
      dvv = duv = dvr = 0.0;
    } else {
      const double c = uu * vv - uv * uv;
      duu = (dd * (-d * vv) + dgam * (vr - g * vv)) / c;
      dvv = (dd * (ur - d * uu) + dgam * (-g * uu)) / c;
      duv = (dd * (-vr + 2.0 * d * uv) + dgam * (-ur + 2.0 * g * uv)) / c;
      dur = (dd * vv - dgam * uv) / c;
      dvr = (-dd * uv + dgam * uu) / c;
    }
    // dZ = delta dS (in d_dP), dP_{i-1} = gamma dS;  dU, dV, dR on T
    FP_DISPATCH(h, k_axby, nblk(nS), nS, d, (const T_*)h->d_dS, 0.0, (T_*)h->d_dP);
    FP_DISPATCH(h, k_axby, nblk(nS), nS, g, (const T_*)h->d_dS, 0.0, (T_*)h->d_dPp);
    FP_DISPATCH(h, k_lin3, nblk(nT), nT, 2.0 * duu, (const T_*)h->d_Q, duv, (const T_*)h->d_V, dur,
                (const T_*)h->d_R, (T_*)h->d_dQ);
    FP_DISPATCH(h, k_lin3, nblk(nT), nT, 2.0 * dvv, (const T_*)h->d_V, duv, (const T_*)h->d_Q, dvr,
                (const T_*)h->d_R, (T_*)h->d_dV);
    FP_DISPATCH(h, k_lin2, nblk(nT), nT, dur, (const T_*)h->d_Q, dvr, (const T_*)h->d_V,
                (T_*)h->d_dR);
    FCK(cudaGetLastError());
    // U = A Z: dA += mask_S(dU Z^T), dZ += mask_S(A^T dU);  V = A P_{i-1} likewise
    rc = seg_prod(h, h->D, h->d_dQ, h->d_P, h->d_dA, 1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dQ, h->d_dP, 1.0, 1);
    if (!rc) rc = seg_prod(h, h->D, h->d_dV, Pp, h->d_dA, 1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dV, h->d_dPp, 1.0, 1);
    if (rc) return rc;
    // Z = mask_S(R): dR += dZ;  R = I - A M: dA -= mask_S(dR M^T), dM -= mask_S(A^T dR)
    FP_DISPATCH(h, k_scatter_add, nblk(nS), nS, h->d_s2t, (const T_*)h->d_dP, (T_*)h->d_dR);
    FCK(cudaGetLastError());
    rc = seg_prod(h, h->D, h->d_dR, M, h->d_dA, -1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dR, h->d_dM, -1.0, 1);
    if (rc) return rc;
    std::swap(h->d_dPn, h->d_dPp);  // dP_{i-1} flows into the step before
  }
  return SPAI_OK;
}

// The patterns and product lists built on the host (rows of any length).
int setup_host(spai_fpmr_ctx* h, const int32_t* rowptr, const int32_t* colind) {
  const int64_t n = h->n, nnz = h->nS;
  cudaStream_t st = h->stream;
  // S: A's pattern, rows strictly ascending, symmetric, full diagonal
  std::vector<long long> sp(n + 1);
  std::vector<int> sc(colind, colind + nnz);
  if (rowptr[0] != 0 || rowptr[n] != nnz) return SPAI_ERR_CSR;
  for (int64_t i = 0; i <= n; i++) sp[i] = rowptr[i];
  for (int64_t i = 0; i < n; i++) {
    if (sp[i + 1] < sp[i]) return SPAI_ERR_CSR;
    for (long long e = sp[i]; e < sp[i + 1]; e++) {
      if (sc[e] < 0 || sc[e] >= n || (e > sp[i] && sc[e] <= sc[e - 1])) return SPAI_ERR_CSR;
    }
  }
  std::vector<int> diagS(n), diagT(n);
  for (int64_t i = 0; i < n; i++) {
    long long d = find_pos(sp, sc, (int)i, (int)i);
    if (d < 0) return SPAI_ERR_NOT_SPD_DIAG;
    diagS[i] = (int)d;
    for (long long e = sp[i]; e < sp[i + 1]; e++)
      if (find_pos(sp, sc, sc[e], (int)i) < 0) return SPAI_ERR_NOT_SYMMETRIC;
  }
  // T = supp(A S) + I, rows sorted
  std::vector<long long> tp(n + 1, 0);
  std::vector<int> tc;
  {
    std::vector<int> mark(n, -1), row;
    for (int64_t r = 0; r < n; r++) {
      row.clear();
      mark[r] = (int)r;
      row.push_back((int)r);
      for (long long e = sp[r]; e < sp[r + 1]; e++) {
        const int k = sc[e];
        for (long long q = sp[k]; q < sp[k + 1]; q++) {
          const int j = sc[q];
          if (mark[j] != r) {
            mark[j] = (int)r;
            row.push_back(j);
          }
        }
      }
      std::sort(row.begin(), row.end());
      tc.insert(tc.end(), row.begin(), row.end());
      tp[r + 1] = (long long)tc.size();
    }
  }
  const long long nS = nnz, nT = (long long)tc.size();
  if (nT >= (1LL << 31)) return SPAI_ERR_UNSUPPORTED;
  h->nT = nT;
  std::vector<int> s2t(nS);
  for (int64_t r = 0; r < n; r++) {
    diagT[r] = (int)find_pos(tp, tc, (int)r, (int)r);
    for (long long e = sp[r]; e < sp[r + 1]; e++) s2t[e] = (int)find_pos(tp, tc, (int)r, sc[e]);
  }
  // Y = A X: for (r,j) in T, k over row r of S merged with row j of S
  // (column j of X by the pattern's symmetry; X's index is that of (k,j))
  std::vector<long long> yp(nT + 1, 0), xp(nS + 1, 0), dp(nS + 1, 0);
  std::vector<int> ya, yb, xa, xb, da, db;
  for (int64_t r = 0; r < n; r++)
    for (long long f = tp[r]; f < tp[r + 1]; f++) {
      const int j = tc[f];
      long long p = sp[r], q = sp[j];
      while (p < sp[r + 1] && q < sp[j + 1]) {
        if (sc[p] < sc[q]) p++;
        else if (sc[q] < sc[p]) q++;
        else {
          const int k = sc[p];
          ya.push_back((int)p);                             // a_rk
          yb.push_back((int)find_pos(sp, sc, k, j));        // x_kj
          p++;
          q++;
        }
      }
      yp[f + 1] = (long long)ya.size();
    }
  // dX[k,j] = sum_r a_rk dy_rj: r over row k of S merged with row j of T
  for (int64_t k = 0; k < n; k++)
    for (long long e = sp[k]; e < sp[k + 1]; e++) {
      const int j = sc[e];
      long long p = sp[k], q = tp[j];
      while (p < sp[k + 1] && q < tp[j + 1]) {
        if (sc[p] < tc[q]) p++;
        else if (tc[q] < sc[p]) q++;
        else {
          const int r = sc[p];
          xa.push_back((int)find_pos(sp, sc, r, (int)k));   // a_rk
          xb.push_back((int)find_pos(tp, tc, r, j));        // dy_rj
          p++;
          q++;
        }
      }
      xp[e + 1] = (long long)xa.size();
    }
  // dA[r,k] = sum_j dy_rj x_kj: j over row r of T merged with row k of S
  for (int64_t r = 0; r < n; r++)
    for (long long e = sp[r]; e < sp[r + 1]; e++) {
      const int k = sc[e];
      long long p = tp[r], q = sp[k];
      while (p < tp[r + 1] && q < sp[k + 1]) {
        if (tc[p] < sc[q]) p++;
        else if (sc[q] < tc[p]) q++;
        else {
          da.push_back((int)p);   // dy_rj
          db.push_back((int)q);   // x_kj
          p++;
          q++;
        }
      }
      dp[e + 1] = (long long)da.size();
    }
  int rc = SPAI_OK;
  rc = rc ? rc : falloc(&h->d_diagS, n);
  rc = rc ? rc : falloc(&h->d_diagT, n);
  rc = rc ? rc : falloc(&h->d_s2t, nS);
  rc = rc ? rc : upload_list(h->Y, yp, ya, yb, st);
  rc = rc ? rc : upload_list(h->X, xp, xa, xb, st);
  rc = rc ? rc : upload_list(h->D, dp, da, db, st);
  if (!rc) {
    bool ok = cudaMemcpyAsync(h->d_diagS, diagS.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) == 0;
    ok &= cudaMemcpyAsync(h->d_diagT, diagT.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) == 0;
    ok &= cudaMemcpyAsync(h->d_s2t, s2t.data(), sizeof(int) * nS, cudaMemcpyHostToDevice, st) == 0;
    ok &= cudaStreamSynchronize(st) == 0;
    if (!ok) rc = SPAI_ERR_CUDA;
  }
  return rc;
}

// The patterns and product lists built on the GPU (rows of at most kSetupW
// entries), in the same order as setup_host.
int setup_device(spai_fpmr_ctx* h, const int32_t* rowptr, const int32_t* colind) {
  const int n = h->n;
  const long long nS = h->nS;
  cudaStream_t st = h->stream;
  int *d_sp = nullptr, *d_sc = nullptr, *d_err = nullptr, *d_tlen = nullptr, *d_tc = nullptr,
      *d_cnt = nullptr;
  long long *d_tp = nullptr, *d_tmp = nullptr;
  auto done = [&](int rc) {
    ffree(d_sp);
    ffree(d_sc);
    ffree(d_err);
    ffree(d_tlen);
    ffree(d_tc);
    ffree(d_cnt);
    ffree(d_tp);
    ffree(d_tmp);
    return rc;
  };
  const unsigned gr = nblk(n);
  int rc = falloc(&d_sp, (size_t)n + 1);
  rc = rc ? rc : falloc(&d_sc, (size_t)nS);
  rc = rc ? rc : falloc(&d_err, 3);
  rc = rc ? rc : falloc(&h->d_diagS, (size_t)n);
  rc = rc ? rc : falloc(&h->d_diagT, (size_t)n);
  rc = rc ? rc : falloc(&h->d_s2t, (size_t)nS);
  rc = rc ? rc : falloc(&d_tlen, (size_t)n);
  rc = rc ? rc : falloc(&d_tp, (size_t)n + 1);
  if (rc) return done(rc);
  const int err0[3] = {0, 0x7fffffff, 0x7fffffff};
  int err[3];
  if (cudaMemcpyAsync(d_sp, rowptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_sc, colind, sizeof(int) * (size_t)nS, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_err, err0, sizeof(err0), cudaMemcpyHostToDevice, st))
    return done(SPAI_ERR_CUDA);
  // S: rows strictly ascending and in range; full diagonal; symmetric
  k_su_check<<<gr, 256, 0, st>>>(n, d_sp, d_sc, d_err);
  k_su_diag_sym<<<gr, 256, 0, st>>>(n, d_sp, d_sc, h->d_diagS, d_err);
  if (cudaMemcpyAsync(err, d_err, sizeof(err), cudaMemcpyDeviceToHost, st) ||
      cudaStreamSynchronize(st))
    return done(SPAI_ERR_CUDA);
  if (err[0]) return done(SPAI_ERR_CSR);
  if (err[1] != 0x7fffffff && err[1] <= err[2]) return done(SPAI_ERR_NOT_SPD_DIAG);
  if (err[2] != 0x7fffffff) return done(SPAI_ERR_NOT_SYMMETRIC);
  // an exclusive scan of counts c[0..m) into p[0..m], total read back
  long long tmp_cap = 0;
  auto scan = [&](const int* c, long long* p, long long m, long long* total) -> int {
    const long long need = 2 * ((m + 1023) / 1024) + 2;
    if (need > tmp_cap) {
      ffree(d_tmp);
      int r2 = falloc(&d_tmp, (size_t)need);
      if (r2) return r2;
      tmp_cap = need;
    }
    if (spai::launch_exclusive_scan(c, p, (int)m, d_tmp, st) != cudaSuccess) return SPAI_ERR_CUDA;
    if (cudaMemcpyAsync(total, p + m, sizeof(long long), cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
      return SPAI_ERR_CUDA;
    return SPAI_OK;
  };
  // T = supp(A S) + I
  k_su_trow<<<gr, 256, 0, st>>>(n, d_sp, d_sc, d_tlen, nullptr, nullptr, 0);
  long long nT = 0;
  rc = scan(d_tlen, d_tp, n, &nT);
  if (rc) return done(rc);
  if (nT >= (1LL << 31)) return done(SPAI_ERR_UNSUPPORTED);
  h->nT = nT;
  rc = falloc(&d_tc, (size_t)nT);
  if (rc) return done(rc);
  k_su_trow<<<gr, 256, 0, st>>>(n, d_sp, d_sc, nullptr, d_tp, d_tc, 1);
  k_su_s2t<<<gr, 256, 0, st>>>(n, d_sp, d_sc, d_tp, d_tc, h->d_s2t, h->d_diagT);
  // the three product lists: count, scan, fill
  rc = falloc(&d_cnt, (size_t)std::max(nT, nS));
  if (rc) return done(rc);
  for (int which = 0; which < 3; which++) {
    ProdList& L = which == 0 ? h->Y : which == 1 ? h->X : h->D;
    const long long nout = which == 0 ? nT : nS;
    auto run = [&](long long* ptr, int* ia, int* ib, int fill) {
      if (which == 0) k_su_y<<<gr, 256, 0, st>>>(n, d_sp, d_sc, d_tp, d_tc, d_cnt, ptr, ia, ib, fill);
      else if (which == 1) k_su_x<<<gr, 256, 0, st>>>(n, d_sp, d_sc, d_tp, d_tc, d_cnt, ptr, ia, ib, fill);
      else k_su_d<<<gr, 256, 0, st>>>(n, d_sp, d_sc, d_tp, d_tc, d_cnt, ptr, ia, ib, fill);
    };
    run(nullptr, nullptr, nullptr, 0);
    rc = falloc(&L.ptr, (size_t)nout + 1);
    if (rc) return done(rc);
    long long len = 0;
    rc = scan(d_cnt, L.ptr, nout, &len);
    if (rc) return done(rc);
    L.nout = nout;
    L.len = len;
    rc = falloc(&L.ia, (size_t)len);
    rc = rc ? rc : falloc(&L.ib, (size_t)len);
    if (rc) return done(rc);
    run(L.ptr, L.ia, L.ib, 1);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return done(SPAI_ERR_CUDA);
  return done(SPAI_OK);
}

// the value arrays of the forward and backward passes
int alloc_values(spai_fpmr_ctx* h) {
  const long long nS = h->nS, nT = h->nT;
  const int vs = h->vs, K = h->K;
  const long long nbmax =
      (nT + (long long)kDotBlock * kDotChunk - 1) / ((long long)kDotBlock * kDotChunk);
  int rc = SPAI_OK;
  rc = rc ? rc : valloc(&h->d_A, nS, vs);
  rc = rc ? rc : valloc(&h->d_Mck, (size_t)(K + 1) * nS, vs);
  rc = rc ? rc : valloc(&h->d_P, nS, vs);
  rc = rc ? rc : valloc(&h->d_dM, nS, vs);
  rc = rc ? rc : valloc(&h->d_dP, nS, vs);
  rc = rc ? rc : valloc(&h->d_dA, nS, vs);
  rc = rc ? rc : valloc(&h->d_R, nT, vs);
  rc = rc ? rc : valloc(&h->d_Q, nT, vs);
  rc = rc ? rc : valloc(&h->d_dR, nT, vs);
  rc = rc ? rc : valloc(&h->d_dQ, nT, vs);
  rc = rc ? rc : falloc(&h->d_stage, nS);
  rc = rc ? rc : falloc(&h->d_part, std::max(nbmax, 1LL));
  rc = rc ? rc : falloc(&h->d_res, 8);
  return rc;
}

}  // namespace

extern "C" {

int spai_fpmr_set_method(spai_fpmr_handle h, int method) {
  if (!h || (method != SPAI_MR && method != SPAI_LOMR)) return SPAI_ERR_ARG;
  if (method == SPAI_LOMR) {
    int rc = alloc_lomr(h);
    if (rc) return rc;
  }
  h->method = method;
  h->have_forward = false;
  return SPAI_OK;
}

int spai_fpmr_create(spai_fpmr_handle* out, int64_t n, int64_t nnz, const int32_t* rowptr,
                     const int32_t* colind, int K, int prec, void* stream) {
  if (!out) return SPAI_ERR_ARG;
  *out = nullptr;
  if (n < 1 || nnz < 1 || !rowptr || !colind || K < 0 || K > 1000) return SPAI_ERR_ARG;
  if (prec != SPAI_FP64 && prec != SPAI_MIXED) return SPAI_ERR_ARG;
  if (n >= (1LL << 31) || nnz >= (1LL << 31)) return SPAI_ERR_UNSUPPORTED;
  if (rowptr[0] != 0 || rowptr[n] != nnz) return SPAI_ERR_CSR;
  int W = 0;
  for (int64_t i = 0; i < n; i++) {
    if (rowptr[i + 1] < rowptr[i]) return SPAI_ERR_CSR;
    W = std::max(W, rowptr[i + 1] - rowptr[i]);
  }
  spai_fpmr_ctx* h = new (std::nothrow) spai_fpmr_ctx();
  if (!h) return SPAI_ERR_OOM;
  h->n = (int)n;
  h->K = K;
  h->vs = prec == SPAI_MIXED ? 4 : 8;
  h->nS = nnz;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      delete h;
      return SPAI_ERR_CUDA;
    }
    h->own_stream = true;
  }
  // SPAI_FPMR_HOST_SETUP=1 takes the host construction for any pattern (tests)
  const char* hs = getenv("SPAI_FPMR_HOST_SETUP");
  const bool host = W > kSetupW || (hs && atoi(hs) == 1);
  int rc = host ? setup_host(h, rowptr, colind) : setup_device(h, rowptr, colind);
  if (!rc) rc = alloc_values(h);
  if (rc) {
    (void)cudaGetLastError();
    free_fpmr(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return rc;
  }
  *out = h;
  return SPAI_OK;
}

int spai_fpmr_destroy(spai_fpmr_handle h) {
  if (!h) return SPAI_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  free_fpmr(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return SPAI_OK;
}

int spai_fpmr_forward(spai_fpmr_handle h, const double* vals, int on_device, double* loss) {
  if (!h || !vals || !loss) return SPAI_ERR_ARG;
  cudaStream_t st = h->stream;
  const long long nS = h->nS, nT = h->nT;
  const int vs = h->vs;
  FCK(cudaMemcpyAsync(h->d_stage, vals, sizeof(double) * nS,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  FP_DISPATCH(h, k_from_f64, nblk(nS), nS, h->d_stage, (T_*)h->d_A);
  FP_DISPATCH(h, k_m0, nblk(nS), nS, (T_*)h->d_Mck);
  FP_DISPATCH(h, k_m0_diag, nblk(h->n), h->n, h->d_diagS, (const T_*)h->d_A, (T_*)h->d_Mck);
  FCK(cudaGetLastError());
  if (h->method == SPAI_LOMR) {
    double l = 0.0;
    int rc = forward_lomr(h, &l);
    if (rc) return rc;
    *loss = l;
    h->have_forward = true;
    return std::isfinite(l) ? SPAI_OK : SPAI_ERR_NONFINITE;
  }
  h->alpha.assign(h->K, 0.0);
  h->num.assign(h->K, 0.0);
  h->den.assign(h->K, 0.0);
  for (int i = 0; i < h->K; i++) {
    void* M = at(h->d_Mck, vs, (long long)i * nS);
    void* Mn = at(h->d_Mck, vs, (long long)(i + 1) * nS);
    int rc = step_products(h, M, true);
    if (!rc) rc = dot(h, nT, h->d_R, h->d_Q, 0);
    if (!rc) rc = dot(h, nT, h->d_Q, h->d_Q, 1);
    double nd[2];
    if (!rc) rc = read_res(h, nd, 2);
    if (rc) return rc;
    if (!(nd[1] > 0.0) || !std::isfinite(nd[0])) return SPAI_ERR_NONFINITE;
    const double a = nd[0] / nd[1];
    h->num[i] = nd[0];
    h->den[i] = nd[1];
    h->alpha[i] = a;
    FP_DISPATCH(h, k_copy, nblk(nS), nS, (const T_*)M, (T_*)Mn);
    FP_DISPATCH(h, k_axby, nblk(nS), nS, a, (const T_*)h->d_P, 1.0, (T_*)Mn);
    FCK(cudaGetLastError());
  }
  int rc = step_products(h, at(h->d_Mck, vs, (long long)h->K * nS), false);
  if (!rc) rc = dot(h, nT, h->d_R, h->d_R, 0);
  double l;
  if (!rc) rc = read_res(h, &l, 1);
  if (rc) return rc;
  *loss = l;
  h->have_forward = true;
  return std::isfinite(l) ? SPAI_OK : SPAI_ERR_NONFINITE;
}

int spai_fpmr_backward(spai_fpmr_handle h, double dloss, double* dvals, int on_device) {
  if (!h || !dvals) return SPAI_ERR_ARG;
  if (!h->have_forward) return SPAI_ERR_STATE;
  cudaStream_t st = h->stream;
  const long long nS = h->nS, nT = h->nT;
  const int K = h->K, vs = h->vs;
  // dR_K = 2 dL R_K;  dA = -mask_S(dR M_K^T);  dM = -mask_S(A^T dR)
  void* MK = at(h->d_Mck, vs, (long long)K * nS);
  int rc = step_products(h, MK, false);
  if (rc) return rc;
  FP_DISPATCH(h, k_axby, nblk(nT), nT, 2.0 * dloss, (const T_*)h->d_R, 0.0, (T_*)h->d_dR);
  FCK(cudaGetLastError());
  rc = seg_prod(h, h->D, h->d_dR, MK, h->d_dA, -1.0, 0);
  if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dR, h->d_dM, -1.0, 0);
  if (rc) return rc;
  if (h->method == SPAI_LOMR) rc = backward_lomr(h);
  if (rc) return rc;
  for (int i = h->method == SPAI_LOMR ? -1 : K - 1; i >= 0; i--) {
    const void* M = at(h->d_Mck, vs, (long long)i * nS);
    const double a = h->alpha[i], den = h->den[i];
    rc = step_products(h, M, true);  // R_i, P_i, Q_i
    if (!rc) rc = dot(h, nS, h->d_dM, h->d_P, 0);
    double da;
    if (!rc) rc = read_res(h, &da, 1);
    if (rc) return rc;
    const double dnum = da / den, dden = -da * a / den;
    // dP = alpha dM;  dR = dnum Q;  dQ = dnum R + 2 dden Q
    FP_DISPATCH(h, k_axby, nblk(nS), nS, a, (const T_*)h->d_dM, 0.0, (T_*)h->d_dP);
    FP_DISPATCH(h, k_axby, nblk(nT), nT, dnum, (const T_*)h->d_Q, 0.0, (T_*)h->d_dR);
    FP_DISPATCH(h, k_lin2, nblk(nT), nT, dnum, (const T_*)h->d_R, 2.0 * dden, (const T_*)h->d_Q,
                (T_*)h->d_dQ);
    FCK(cudaGetLastError());
    // Q = A P:  dA += mask_S(dQ P^T);  dP += mask_S(A^T dQ)
    rc = seg_prod(h, h->D, h->d_dQ, h->d_P, h->d_dA, 1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dQ, h->d_dP, 1.0, 1);
    if (rc) return rc;
    // P = mask_S(R):  dR += dP on S's positions of T
    FP_DISPATCH(h, k_scatter_add, nblk(nS), nS, h->d_s2t, (const T_*)h->d_dP, (T_*)h->d_dR);
    FCK(cudaGetLastError());
    // R = I - A M:  dA -= mask_S(dR M^T);  dM -= mask_S(A^T dR)
    rc = seg_prod(h, h->D, h->d_dR, M, h->d_dA, -1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dR, h->d_dM, -1.0, 1);
    if (rc) return rc;
  }
  // M_0 = diag(A)^{-1}
  FP_DISPATCH(h, k_m0_adjoint, nblk(h->n), h->n, h->d_diagS, (const T_*)h->d_A, (const T_*)h->d_dM,
              (T_*)h->d_dA);
  FP_DISPATCH(h, k_to_f64, nblk(nS), nS, (const T_*)h->d_dA, h->d_stage);
  FCK(cudaGetLastError());
  FCK(cudaMemcpyAsync(dvals, h->d_stage, sizeof(double) * nS,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  FCK(cudaStreamSynchronize(st));
  return SPAI_OK;
}

int spai_fpmr_info(spai_fpmr_handle h, int64_t* nnz_t, int64_t* list_entries, int64_t* launches) {
  if (!h) return SPAI_ERR_ARG;
  if (nnz_t) *nnz_t = h->nT;
  if (list_entries) *list_entries = h->Y.len + h->X.len + h->D.len;
  if (launches) *launches = h->launches;
  return SPAI_OK;
}

}  // extern "C"
