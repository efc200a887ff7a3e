// Differentiation of fixed-pattern MR (no counterpart in the paper; its
// objective and gradient form are Sec. 2 and Sec. 3 Eq. (gradient)):
//   M_0 = diag(A)^{-1};  R_i = I - A M_i;  P_i = mask_S(R_i);  Q_i = A P_i;
//   alpha_i = (R_i, Q_i)_F / (Q_i, Q_i)_F;  M_{i+1} = M_i + alpha_i P_i;
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
// per step).  Values are FP64, or FP32 on the mixed path (FP32 products and
// stored values; inner products, step scalars and the axpy arithmetic in
// FP64, each stored value rounded once).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "spai.h"

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

}  // namespace

extern "C" {

int spai_fpmr_create(spai_fpmr_handle* out, int64_t n, int64_t nnz, const int32_t* rowptr,
                     const int32_t* colind, int K, int prec, void* stream) {
  if (!out) return SPAI_ERR_ARG;
  *out = nullptr;
  if (n < 1 || nnz < 1 || !rowptr || !colind || K < 0 || K > 1000) return SPAI_ERR_ARG;
  if (prec != SPAI_FP64 && prec != SPAI_MIXED) return SPAI_ERR_ARG;
  if (n >= (1LL << 31) || nnz >= (1LL << 31)) return SPAI_ERR_UNSUPPORTED;
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
  spai_fpmr_ctx* h = new (std::nothrow) spai_fpmr_ctx();
  if (!h) return SPAI_ERR_OOM;
  h->n = (int)n;
  h->K = K;
  h->vs = prec == SPAI_MIXED ? 4 : 8;
  h->nS = nS;
  h->nT = nT;
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
  cudaStream_t st = h->stream;
  const long long nbmax = (nT + (long long)kDotBlock * kDotChunk - 1) / ((long long)kDotBlock * kDotChunk);
  int rc = SPAI_OK;
  rc = rc ? rc : falloc(&h->d_diagS, n);
  rc = rc ? rc : falloc(&h->d_diagT, n);
  rc = rc ? rc : falloc(&h->d_s2t, nS);
  const int vs = h->vs;
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
  for (int i = K - 1; i >= 0; i--) {
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
