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
// per step).  FP64 throughout.
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
  double *d_A = nullptr, *d_Mck = nullptr, *d_P = nullptr, *d_dM = nullptr, *d_dP = nullptr,
         *d_dA = nullptr;
  double *d_R = nullptr, *d_Q = nullptr, *d_dR = nullptr, *d_dQ = nullptr;
  double *d_part = nullptr, *d_res = nullptr;
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

constexpr int kDotChunk = 16;     // elements per thread in the dot partials
constexpr int kDotBlock = 256;

// out[s] (=|+=) scale * sum_t a[ia[t]] b[ib[t]] over t in [ptr[s], ptr[s+1]),
// an fma chain in list order
__global__ void k_seg_prod(long long nout, const long long* ptr, const int* ia, const int* ib,
                           const double* a, const double* b, double* out, double scale, int acc) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nout) return;
  double v = 0.0;
  for (long long t = ptr[s]; t < ptr[s + 1]; t++) v = __fma_rn(a[ia[t]], b[ib[t]], v);
  v = __dmul_rn(scale, v);
  out[s] = acc ? __dadd_rn(out[s], v) : v;
}

__global__ void k_add_diag(int n, const int* diag, double* x, double v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[diag[j]] = __dadd_rn(x[diag[j]], v);
}

__global__ void k_gather(long long m, const int* idx, const double* src, double* dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) dst[e] = src[idx[e]];
}

__global__ void k_scatter_add(long long m, const int* idx, const double* src, double* dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) dst[idx[e]] = __dadd_rn(dst[idx[e]], src[e]);
}

// y = a x + b y  (b == 0: y = a x)
__global__ void k_axby(long long m, double a, const double* x, double b, double* y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) y[e] = b == 0.0 ? __dmul_rn(a, x[e]) : __fma_rn(a, x[e], __dmul_rn(b, y[e]));
}

// z = a x + b y
__global__ void k_lin2(long long m, double a, const double* x, double b, const double* y,
                       double* z) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) z[e] = __fma_rn(a, x[e], __dmul_rn(b, y[e]));
}

// M0 = diag(A)^{-1} on S: zero everywhere (k_m0), then the diagonal
__global__ void k_m0(long long nS, double* M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nS) M[e] = 0.0;
}
__global__ void k_m0_diag(int n, const int* diag, const double* A, double* M) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) M[diag[j]] = __ddiv_rn(1.0, A[diag[j]]);
}

// dA[(j,j)] -= dM[(j,j)] / a_jj^2  (through M_0 = diag(A)^{-1})
__global__ void k_m0_adjoint(int n, const int* diag, const double* A, const double* dM,
                             double* dA) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double a = A[diag[j]];
  dA[diag[j]] = __dsub_rn(dA[diag[j]], __ddiv_rn(dM[diag[j]], __dmul_rn(a, a)));
}

__device__ __forceinline__ double warp_sum32(double v) {
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

// per block: kDotBlock * kDotChunk consecutive products x_e y_e summed in a
// fixed order (sequential per thread, then a tree)
__global__ void k_dot_part(long long m, const double* x, const double* y, double* part) {
  __shared__ double red[kDotBlock / 32];
  const long long base = (long long)blockIdx.x * kDotBlock * kDotChunk + threadIdx.x * kDotChunk;
  double s = 0.0;
  for (int t = 0; t < kDotChunk; t++) {
    const long long e = base + t;
    if (e < m) s = __fma_rn(x[e], y[e], s);
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

int seg_prod(spai_fpmr_ctx* h, const ProdList& L, const double* a, const double* b, double* out,
             double scale, int acc) {
  k_seg_prod<<<nblk(L.nout), 256, 0, h->stream>>>(L.nout, L.ptr, L.ia, L.ib, a, b, out, scale, acc);
  h->launches++;
  FCK(cudaGetLastError());
  return SPAI_OK;
}

// (x, y) over m entries, into h->d_res[slot] (device)
int dot(spai_fpmr_ctx* h, long long m, const double* x, const double* y, int slot) {
  const long long nb = (m + (long long)kDotBlock * kDotChunk - 1) / ((long long)kDotBlock * kDotChunk);
  k_dot_part<<<(unsigned)std::max(nb, 1LL), kDotBlock, 0, h->stream>>>(m, x, y, h->d_part);
  k_dot_final<<<1, 1024, 0, h->stream>>>(std::max(nb, 1LL), h->d_part, h->d_res + slot);
  h->launches += 2;
  FCK(cudaGetLastError());
  return SPAI_OK;
}

int read_res(spai_fpmr_ctx* h, double* out, int count) {
  FCK(cudaMemcpyAsync(out, h->d_res, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
  FCK(cudaStreamSynchronize(h->stream));
  return SPAI_OK;
}

// R = I - A M (on T), P = mask_S(R), Q = A P
int step_products(spai_fpmr_ctx* h, const double* M, bool want_q) {
  int rc = seg_prod(h, h->Y, h->d_A, M, h->d_R, -1.0, 0);
  if (rc) return rc;
  k_add_diag<<<nblk(h->n), 256, 0, h->stream>>>(h->n, h->d_diagT, h->d_R, 1.0);
  k_gather<<<nblk(h->nS), 256, 0, h->stream>>>(h->nS, h->d_s2t, h->d_R, h->d_P);
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
                     const int32_t* colind, int K, void* stream) {
  if (!out) return SPAI_ERR_ARG;
  *out = nullptr;
  if (n < 1 || nnz < 1 || !rowptr || !colind || K < 0 || K > 1000) return SPAI_ERR_ARG;
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
  rc = rc ? rc : falloc(&h->d_A, nS);
  rc = rc ? rc : falloc(&h->d_Mck, (size_t)(K + 1) * nS);
  rc = rc ? rc : falloc(&h->d_P, nS);
  rc = rc ? rc : falloc(&h->d_dM, nS);
  rc = rc ? rc : falloc(&h->d_dP, nS);
  rc = rc ? rc : falloc(&h->d_dA, nS);
  rc = rc ? rc : falloc(&h->d_R, nT);
  rc = rc ? rc : falloc(&h->d_Q, nT);
  rc = rc ? rc : falloc(&h->d_dR, nT);
  rc = rc ? rc : falloc(&h->d_dQ, nT);
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
  FCK(cudaMemcpyAsync(h->d_A, vals, sizeof(double) * nS,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  k_m0<<<nblk(nS), 256, 0, st>>>(nS, h->d_Mck);
  k_m0_diag<<<nblk(h->n), 256, 0, st>>>(h->n, h->d_diagS, h->d_A, h->d_Mck);
  h->launches += 2;
  FCK(cudaGetLastError());
  h->alpha.assign(h->K, 0.0);
  h->num.assign(h->K, 0.0);
  h->den.assign(h->K, 0.0);
  for (int i = 0; i < h->K; i++) {
    double* M = h->d_Mck + (size_t)i * nS;
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
    FCK(cudaMemcpyAsync(M + nS, M, sizeof(double) * nS, cudaMemcpyDeviceToDevice, st));
    k_axby<<<nblk(nS), 256, 0, st>>>(nS, a, h->d_P, 1.0, M + nS);
    h->launches++;
    FCK(cudaGetLastError());
  }
  int rc = step_products(h, h->d_Mck + (size_t)h->K * nS, false);
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
  const int K = h->K;
  // dR_K = 2 dL R_K;  dA = -mask_S(dR M_K^T);  dM = -mask_S(A^T dR)
  int rc = step_products(h, h->d_Mck + (size_t)K * nS, false);
  if (rc) return rc;
  k_axby<<<nblk(nT), 256, 0, st>>>(nT, 2.0 * dloss, h->d_R, 0.0, h->d_dR);
  h->launches++;
  FCK(cudaGetLastError());
  rc = seg_prod(h, h->D, h->d_dR, h->d_Mck + (size_t)K * nS, h->d_dA, -1.0, 0);
  if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dR, h->d_dM, -1.0, 0);
  if (rc) return rc;
  for (int i = K - 1; i >= 0; i--) {
    const double* M = h->d_Mck + (size_t)i * nS;
    const double a = h->alpha[i], den = h->den[i];
    rc = step_products(h, M, true);  // R_i, P_i, Q_i
    if (!rc) rc = dot(h, nS, h->d_dM, h->d_P, 0);
    double da;
    if (!rc) rc = read_res(h, &da, 1);
    if (rc) return rc;
    const double dnum = da / den, dden = -da * a / den;
    // dP = alpha dM;  dR = dnum Q;  dQ = dnum R + 2 dden Q
    k_axby<<<nblk(nS), 256, 0, st>>>(nS, a, h->d_dM, 0.0, h->d_dP);
    k_axby<<<nblk(nT), 256, 0, st>>>(nT, dnum, h->d_Q, 0.0, h->d_dR);
    k_lin2<<<nblk(nT), 256, 0, st>>>(nT, dnum, h->d_R, 2.0 * dden, h->d_Q, h->d_dQ);
    h->launches += 3;
    FCK(cudaGetLastError());
    // Q = A P:  dA += mask_S(dQ P^T);  dP += mask_S(A^T dQ)
    rc = seg_prod(h, h->D, h->d_dQ, h->d_P, h->d_dA, 1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dQ, h->d_dP, 1.0, 1);
    if (rc) return rc;
    // P = mask_S(R):  dR += dP on S's positions of T
    k_scatter_add<<<nblk(nS), 256, 0, st>>>(nS, h->d_s2t, h->d_dP, h->d_dR);
    h->launches++;
    FCK(cudaGetLastError());
    // R = I - A M:  dA -= mask_S(dR M^T);  dM -= mask_S(A^T dR)
    rc = seg_prod(h, h->D, h->d_dR, M, h->d_dA, -1.0, 1);
    if (!rc) rc = seg_prod(h, h->X, h->d_A, h->d_dR, h->d_dM, -1.0, 1);
    if (rc) return rc;
  }
  // M_0 = diag(A)^{-1}
  k_m0_adjoint<<<nblk(h->n), 256, 0, st>>>(h->n, h->d_diagS, h->d_A, h->d_dM, h->d_dA);
  h->launches++;
  FCK(cudaGetLastError());
  FCK(cudaMemcpyAsync(dvals, h->d_dA, sizeof(double) * nS,
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
