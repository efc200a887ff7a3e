// Block PCG kernels of libspai.so.
//
// Each matrix of a handle (a segment of whole 256-row CTAs) carries R <= 32
// right-hand sides; recurrence (m, j) is the vector PCG of Sec. 7 on A_m
// with b_{m,j}: x_0 = 0, stop on the recurrence residual, FP64 throughout.
// The vectors are stored row-major with a row stride of 32 doubles, so a
// warp that owns a row holds right-hand side j in lane j: every SpMM entry
// is one broadcast (column, value) and one coalesced 256-byte row of the
// operand, and all R products share that load of A.
//
// Arithmetic is that of the single-vector PCG, per recurrence: SpMV rows are
// fma chains over ascending column; z = M r likewise over the rows of M (or
// of its symmetric part); inner products are balanced pairwise trees over the
// matrix's rows zero-padded to a power of two.  Here the tree is cut into
// 32-row warp subtrees, an 8-warp CTA tree, and a tree over the segment's
// CTAs finished by the last-arriving CTA, which also updates that segment's
// scalars.  A padded row or a row past n adds an exact zero, so every
// recurrence reproduces a plain one-vector run on its own matrix bitwise.
#include <stdint.h>

#include "bpcg.cuh"
#include "common.cuh"

namespace spai {

namespace {

__device__ __forceinline__ bool bp_finite(double x) { return !isnan(x) && !isinf(x); }

// Pairwise sum over the 32 rows of a warp, row t's term from f(t): groups
// of four rows ((f0 + f1) + (f2 + f3)), then a three-level binary counter
// over the eight groups held in named registers.
template <typename F>
__device__ __forceinline__ double rows32(F f) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, tot = 0.0;
#pragma unroll 1
  for (int g = 0; g < 8; g++) {
    const int t = 4 * g;
    const double f0 = f(t), f1 = f(t + 1), f2 = f(t + 2), f3 = f(t + 3);
    double v = __dadd_rn(__dadd_rn(f0, f1), __dadd_rn(f2, f3));
    if (g & 1) {
      v = __dadd_rn(s0, v);
      if (g & 2) {
        v = __dadd_rn(s1, v);
        if (g & 4)
          tot = __dadd_rn(s2, v);
        else
          s2 = v;
      } else {
        s1 = v;
      }
    } else {
      s0 = v;
    }
  }
  return tot;
}

// ((v0+v1)+(v2+v3))+((v4+v5)+(v6+v7)) of column lane of s[8][32]
__device__ __forceinline__ double tree8(const double (*s)[32], int lane) {
  double a = __dadd_rn(__dadd_rn(s[0][lane], s[1][lane]), __dadd_rn(s[2][lane], s[3][lane]));
  double b = __dadd_rn(__dadd_rn(s[4][lane], s[5][lane]), __dadd_rn(s[6][lane], s[7][lane]));
  return __dadd_rn(a, b);
}

// Pairwise sum of CTA partials start .. start+len-1 (len a power of two, at
// most 2048) of a segment; partials at index >= nc are zero.
__device__ __noinline__ double seq_pairwise(const double* bsum, int c0, int nc, int start,
                                            int len, int lane) {
  if (start >= nc) return 0.0;
  double stk[12];
  for (int t = 0; t < len; t++) {
    const int c = start + t;
    double v = c < nc ? __ldcg(bsum + (long long)(c0 + c) * kBpLd + lane) : 0.0;
    int l = 0;
    while ((t >> l) & 1) {
      v = __dadd_rn(stk[l], v);
      l++;
    }
    stk[l] = v;
  }
  int L = 0;
  while ((1 << L) < len) L++;
  return stk[L];
}

// CTA reduction of the warps' row sums, then, in the last-arriving CTA of
// the segment, the tree over the segment's CTAs; fin(state index, total) runs
// in lane j < R of warp 0 of that CTA.
template <typename Fin>
__device__ void bp_reduce(const BpcgArgs& a, int seg, double wsum, Fin fin) {
  __shared__ double sw[8][32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  sw[warp][lane] = wsum;
  __syncthreads();
  if (warp == 0) {
    a.bsum[(long long)blockIdx.x * kBpLd + lane] = tree8(sw, lane);
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned old = atomicAdd(&a.cnt[seg], 1u);
    s_last = old == (unsigned)(a.seg_ncta[seg] - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int c0 = a.seg_cta0[seg], nc = a.seg_ncta[seg];
  int P = 1;
  while (P < nc) P <<= 1;
  const int chunk = P >= 8 ? P / 8 : 1;
  const double v =
      warp * chunk < P ? seq_pairwise(a.bsum, c0, nc, warp * chunk, chunk, lane) : 0.0;
  sw[warp][lane] = v;
  __syncthreads();
  if (warp == 0) {
    const double s = tree8(sw, lane);
    if (lane == 0) a.cnt[seg] = 0;
    if (lane < a.R) fin(seg * kBpLd + lane, s);
    __threadfence();
  }
}

__device__ __forceinline__ void bp_retire(const BpcgArgs& a, int sl, int status) {
  a.done[sl] = 1;
  a.status[sl] = status;
  atomicSub(&a.seg_live[sl / kBpLd], 1);
  atomicSub(a.live, 1);
}

// (A v)_i for right-hand side lane: A's row from the ELL layout, entries
// broadcast with shuffles (all lanes take part; act selects the lanes whose
// product is formed)
__device__ __forceinline__ double a_row(const BpcgArgs& a, int i, const double* v, int lane,
                                        bool act) {
  double acc = 0.0;
  for (int t0 = 0; t0 < a.W; t0 += 32) {
    int c = -1;
    double av = 0.0;
    if (t0 + lane < a.W) {
      c = a.ell_col[(long long)i * a.W + t0 + lane];
      av = a.ell_val[(long long)i * a.W + t0 + lane];
    }
    const int m = min(32, a.W - t0);
    for (int t = 0; t < m; t++) {
      const int cc = __shfl_sync(kFull, c, t);
      const double vv = __shfl_sync(kFull, av, t);
      if (cc < 0) break;  // padding sits at the end of a row
      if (act) acc = __fma_rn(vv, v[(long long)cc * kBpLd + lane], acc);
    }
  }
  return acc;
}

// (M v)_i over the CSR rows of the preconditioner
__device__ __forceinline__ double m_row(const BpcgArgs& a, int i, const double* v, int lane,
                                        bool act) {
  const long long e0 = a.mrp[i], e1 = a.mrp[i + 1];
  double acc = 0.0;
  for (long long eb = e0; eb < e1; eb += 32) {
    int c = 0;
    double mv = 0.0;
    if (eb + lane < e1) {
      c = a.mci[eb + lane];
      mv = a.mv[eb + lane];
    }
    const int m = (int)min(32LL, e1 - eb);
    for (int t = 0; t < m; t++) {
      const int cc = __shfl_sync(kFull, c, t);
      const double vv = __shfl_sync(kFull, mv, t);
      if (act) acc = __fma_rn(vv, v[(long long)cc * kBpLd + lane], acc);
    }
  }
  return acc;
}

__global__ void k_bp_setup(BpcgArgs a, int nseg) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nseg * kBpLd) return;
  const int seg = t / kBpLd, lane = t % kBpLd;
  a.done[t] = lane < a.R ? 0 : 1;
  a.status[t] = 0;
  a.k[t] = 0;
  a.rho[t] = a.alpha[t] = a.beta[t] = a.bn[t] = a.tres[t] = 0.0;
  if (lane == 0) {
    a.cnt[seg] = 0;
    a.seg_live[seg] = a.R;
  }
  if (t == 0) *a.live = nseg * a.R;
}

// x = 0, r = b; terms b^2 -> ||b||
__global__ void __launch_bounds__(256) k_bp_init(BpcgArgs a) {
  const int seg = a.seg_of_cta[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool act = lane < a.R;
  const long long row0 = (long long)blockIdx.x * kBpRows + warp * 32;
  const double s = rows32([&](int t) {
    const long long i = row0 + t;
    if (i >= a.n || !act) return 0.0;
    const double bi = a.b[i * kBpLd + lane];
    a.x[i * kBpLd + lane] = 0.0;
    a.r[i * kBpLd + lane] = bi;
    return __dmul_rn(bi, bi);
  });
  bp_reduce(a, seg, s, [&](int sl, double tot) {
    a.bn[sl] = __dsqrt_rn(tot);
    a.k[sl] = 0;
    if (tot == 0.0) bp_retire(a, sl, 0);
  });
}

// z = Prec(r), terms r z -> rho (first: initial rho; else beta = rho1 / rho)
__global__ void __launch_bounds__(256) k_bp_prec(BpcgArgs a, int first) {
  const int seg = a.seg_of_cta[blockIdx.x];
  if (a.seg_live[seg] == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool act = lane < a.R && !a.done[seg * kBpLd + lane];
  const long long row0 = (long long)blockIdx.x * kBpRows + warp * 32;
  const double s = rows32([&](int t) {
    const long long i = row0 + t;
    if (i >= a.n) return 0.0;
    double z;
    if (a.precond == 0) {
      z = act ? a.r[i * kBpLd + lane] : 0.0;
    } else if (a.precond == 1) {
      z = act ? __ddiv_rn(a.r[i * kBpLd + lane], a.diag[i]) : 0.0;
    } else {
      z = m_row(a, (int)i, a.r, lane, act);
    }
    if (!act) return 0.0;
    a.z[i * kBpLd + lane] = z;
    return __dmul_rn(a.r[i * kBpLd + lane], z);
  });
  bp_reduce(a, seg, s, [&](int sl, double rho1) {
    if (a.done[sl]) return;
    if (rho1 == 0.0 || !bp_finite(rho1)) {
      bp_retire(a, sl, 2);
      return;
    }
    if (first) {
      a.rho[sl] = rho1;
      a.beta[sl] = 0.0;
    } else {
      a.beta[sl] = __ddiv_rn(rho1, a.rho[sl]);
      a.rho[sl] = rho1;
    }
  });
}

// p = z (first) or fma(beta, p, z)
__global__ void __launch_bounds__(256) k_bp_dir(BpcgArgs a, int first) {
  const int seg = a.seg_of_cta[blockIdx.x];
  if (a.seg_live[seg] == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sl = seg * kBpLd + lane;
  if (lane >= a.R || a.done[sl]) return;
  const double be = a.beta[sl];
  const long long row0 = (long long)blockIdx.x * kBpRows + warp * 32;
  for (int t = 0; t < 32; t++) {
    const long long i = row0 + t;
    if (i >= a.n) break;
    const long long e = i * kBpLd + lane;
    a.p[e] = first ? a.z[e] : __fma_rn(be, a.p[e], a.z[e]);
  }
}

// q = A p, terms p q -> alpha = rho / (p, A p); the iteration limit is
// checked here, before the update, as in the one-vector recurrence
__global__ void __launch_bounds__(256) k_bp_spmm(BpcgArgs a) {
  const int seg = a.seg_of_cta[blockIdx.x];
  if (a.seg_live[seg] == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool act = lane < a.R && !a.done[seg * kBpLd + lane];
  const long long row0 = (long long)blockIdx.x * kBpRows + warp * 32;
  const double s = rows32([&](int t) {
    const long long i = row0 + t;
    if (i >= a.n) return 0.0;
    const double q = a_row(a, (int)i, a.p, lane, act);
    if (!act) return 0.0;
    a.q[i * kBpLd + lane] = q;
    return __dmul_rn(a.p[i * kBpLd + lane], q);
  });
  bp_reduce(a, seg, s, [&](int sl, double pq) {
    if (a.done[sl]) return;
    if (a.k[sl] >= a.maxit) {
      bp_retire(a, sl, 1);
      return;
    }
    if (pq == 0.0 || !bp_finite(pq)) {
      bp_retire(a, sl, 2);
      return;
    }
    a.alpha[sl] = __ddiv_rn(a.rho[sl], pq);
  });
}

// x += alpha p, r -= alpha q, terms r^2 -> convergence test
__global__ void __launch_bounds__(256) k_bp_update(BpcgArgs a) {
  const int seg = a.seg_of_cta[blockIdx.x];
  if (a.seg_live[seg] == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sl0 = seg * kBpLd + lane;
  const bool act = lane < a.R && !a.done[sl0];
  const double al = act ? a.alpha[sl0] : 0.0;
  const long long row0 = (long long)blockIdx.x * kBpRows + warp * 32;
  const double s = rows32([&](int t) {
    const long long i = row0 + t;
    if (i >= a.n || !act) return 0.0;
    const long long e = i * kBpLd + lane;
    a.x[e] = __fma_rn(al, a.p[e], a.x[e]);
    const double r = __fma_rn(-al, a.q[e], a.r[e]);
    a.r[e] = r;
    return __dmul_rn(r, r);
  });
  bp_reduce(a, seg, s, [&](int sl, double rr) {
    if (a.done[sl]) return;
    a.k[sl] += 1;
    const double rn = __dsqrt_rn(rr);
    if (!bp_finite(rn))
      bp_retire(a, sl, 2);
    else if (rn <= __dmul_rn(a.rtol, a.bn[sl]))
      bp_retire(a, sl, 0);
  });
}

// terms (b - A x)^2 -> ||b - A x||^2 of every recurrence (no early exit)
__global__ void __launch_bounds__(256) k_bp_tres(BpcgArgs a) {
  const int seg = a.seg_of_cta[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool act = lane < a.R;
  const long long row0 = (long long)blockIdx.x * kBpRows + warp * 32;
  const double s = rows32([&](int t) {
    const long long i = row0 + t;
    if (i >= a.n) return 0.0;
    const double y = a_row(a, (int)i, a.x, lane, act);
    if (!act) return 0.0;
    const double d = __dsub_rn(a.b[i * kBpLd + lane], y);
    return __dmul_rn(d, d);
  });
  bp_reduce(a, seg, s, [&](int sl, double tot) { a.tres[sl] = tot; });
}

__global__ void k_bp_gather(const double* user, double* dst, int n, int R, const int* seg_of_cta,
                            const int* seg_row0, const int* seg_n, const long long* seg_boff) {
  const long long i = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const int lane = threadIdx.x;
  if (i >= n) return;
  const int seg = seg_of_cta[i / kBpRows];
  const long long loc = i - seg_row0[seg];
  const int nm = seg_n[seg];
  double v = 0.0;
  if (lane < R && loc < nm) v = user[seg_boff[seg] + (long long)lane * nm + loc];
  dst[i * kBpLd + lane] = v;
}

__global__ void k_bp_scatter(const double* src, double* user, int n, int R, const int* seg_of_cta,
                             const int* seg_row0, const int* seg_n, const long long* seg_boff) {
  const long long i = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const int lane = threadIdx.x;
  if (i >= n) return;
  const int seg = seg_of_cta[i / kBpRows];
  const long long loc = i - seg_row0[seg];
  const int nm = seg_n[seg];
  if (lane < R && loc < nm) user[seg_boff[seg] + (long long)lane * nm + loc] = src[i * kBpLd + lane];
}

inline int bp_grid(int n) { return (n + kBpRows - 1) / kBpRows; }

}  // namespace

cudaError_t launch_bp_setup(const BpcgArgs& a, int nseg, cudaStream_t st) {
  k_bp_setup<<<(nseg * kBpLd + 255) / 256, 256, 0, st>>>(a, nseg);
  return cudaGetLastError();
}

cudaError_t launch_bp_gather(const double* user, double* dst, int n, int R, const int* seg_of_cta,
                             const int* seg_row0, const int* seg_n, const long long* seg_boff,
                             cudaStream_t st) {
  k_bp_gather<<<(n + 7) / 8, dim3(32, 8), 0, st>>>(user, dst, n, R, seg_of_cta, seg_row0, seg_n,
                                                    seg_boff);
  return cudaGetLastError();
}

cudaError_t launch_bp_scatter(const double* src, double* user, int n, int R, const int* seg_of_cta,
                              const int* seg_row0, const int* seg_n, const long long* seg_boff,
                              cudaStream_t st) {
  k_bp_scatter<<<(n + 7) / 8, dim3(32, 8), 0, st>>>(src, user, n, R, seg_of_cta, seg_row0, seg_n,
                                                     seg_boff);
  return cudaGetLastError();
}

cudaError_t launch_bp_init(const BpcgArgs& a, cudaStream_t st) {
  const int g = bp_grid(a.n);
  k_bp_init<<<g, 256, 0, st>>>(a);
  k_bp_prec<<<g, 256, 0, st>>>(a, 1);
  k_bp_dir<<<g, 256, 0, st>>>(a, 1);
  return cudaGetLastError();
}

cudaError_t launch_bp_iter(const BpcgArgs& a, cudaStream_t st) {
  const int g = bp_grid(a.n);
  k_bp_spmm<<<g, 256, 0, st>>>(a);
  k_bp_update<<<g, 256, 0, st>>>(a);
  k_bp_prec<<<g, 256, 0, st>>>(a, 0);
  k_bp_dir<<<g, 256, 0, st>>>(a, 0);
  return cudaGetLastError();
}

cudaError_t launch_bp_tres(const BpcgArgs& a, cudaStream_t st) {
  k_bp_tres<<<bp_grid(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace spai
