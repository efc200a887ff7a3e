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

// Pairwise sum over the 32 rows of a warp.  g(t, o) computes rows t .. t+3
// together (so their loads are in flight at once) and leaves their terms in
// o[0..3]; each group gives ((o0 + o1) + (o2 + o3)), and a three-level binary
// counter in named registers combines the eight groups.
template <typename G>
__device__ __forceinline__ double rows32(G g) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, tot = 0.0;
#pragma unroll 1
  for (int k = 0; k < 8; k++) {
    double o[4];
    g(4 * k, o);
    double v = __dadd_rn(__dadd_rn(o[0], o[1]), __dadd_rn(o[2], o[3]));
    if (k & 1) {
      v = __dadd_rn(s0, v);
      if (k & 2) {
        v = __dadd_rn(s1, v);
        if (k & 4)
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

__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Rows of A with at most 8 entries are handled four at a time: lane 8r + e
// holds entry e of row i0 + r (column -1 where the row has fewer), loaded in
// one coalesced access; AGroup keeps the entries of the current group and
// prefetches those of the next while the current group's operands are read.
// VT is the value type of the products: double, or float on the mixed path.
template <typename VT>
struct AGroup {
  int cn;
  VT vn;
};

template <typename VT>
__device__ __forceinline__ void a_group_load(const BpcgArgs& a, const VT* vals, long long i0,
                                             int lane, int& c, VT& v) {
  const long long i = i0 + (lane >> 3);
  const int e = lane & 7;
  c = -1;
  v = VT(0);
  if (i < a.n && e < a.W) {
    c = __ldg(a.ell_col + i * a.W + e);
    v = __ldg(vals + i * a.W + e);
  }
}

// (A x)_i, i = i0 .. i0+3, for right-hand side lane into y[0..3] (an fma
// chain in VT over ascending column, widened to FP64).  Every operand of the
// four rows is fetched before the chains run (32 gathers in flight per
// warp); padding (column -1) ends a row.
template <typename VT>
__device__ __forceinline__ void a_rows4_small(const BpcgArgs& a, const VT* vals, AGroup<VT>& g,
                                              long long i0, bool more, const VT* x, int lane,
                                              bool act, double* y) {
  const int c = g.cn;
  const VT av = g.vn;
  if (more) a_group_load(a, vals, i0 + 4, lane, g.cn, g.vn);
  VT pv[32];
#pragma unroll
  for (int s = 0; s < 32; s++) {
    const int cc = __shfl_sync(kFull, c, s);
    pv[s] = (act && cc >= 0) ? __ldg(x + (long long)cc * kBpLd + lane) : VT(0);
  }
#pragma unroll
  for (int r = 0; r < 4; r++) {
    VT acc = VT(0);
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int cc = __shfl_sync(kFull, c, 8 * r + e);
      const VT vv = __shfl_sync(kFull, av, 8 * r + e);
      if (cc >= 0) acc = fma_rn(vv, pv[8 * r + e], acc);
    }
    y[r] = (double)acc;
  }
}

// General rows (more than 8 entries): entry by entry, 32 per load
template <typename VT>
__device__ __forceinline__ void a_rows4_wide(const BpcgArgs& a, const VT* vals, long long i0,
                                             const VT* x, int lane, bool act, double* y) {
  for (int r = 0; r < 4; r++) {
    const long long i = i0 + r;
    VT acc = VT(0);
    if (i < a.n) {
      for (int t0 = 0; t0 < a.W; t0 += 32) {
        int c = -1;
        VT av = VT(0);
        if (t0 + lane < a.W) {
          c = __ldg(a.ell_col + i * a.W + t0 + lane);
          av = __ldg(vals + i * a.W + t0 + lane);
        }
        const int m = min(32, a.W - t0);
        for (int t = 0; t < m; t++) {
          const int cc = __shfl_sync(kFull, c, t);
          const VT vv = __shfl_sync(kFull, av, t);
          if (cc < 0) break;
          if (act) acc = fma_rn(vv, __ldg(x + (long long)cc * kBpLd + lane), acc);
        }
      }
    }
    y[r] = (double)acc;
  }
}

template <typename VT>
__device__ __forceinline__ void a_rows4(const BpcgArgs& a, const VT* vals, AGroup<VT>& g,
                                        long long i0, bool more, const VT* x, int lane, bool act,
                                        double* y) {
  if (a.W <= 8)
    a_rows4_small(a, vals, g, i0, more, x, lane, act, y);
  else
    a_rows4_wide(a, vals, i0, x, lane, act, y);
}

// (M x)_i, i = i0 .. i0+3, over the CSR rows of the preconditioner: lanes
// 8r .. 8r+7 walk row r eight entries at a time (the next eight prefetched),
// and the 32 operands of a step are fetched before their fmas.  Entries stay
// in ascending column order within each row's chain.
template <typename VT>
__device__ __forceinline__ void m_rows4(const BpcgArgs& a, const VT* mvals, long long i0,
                                        const VT* x, int lane, bool act, double* y) {
  const int e = lane & 7;
  const long long i = i0 + (lane >> 3);
  long long b0 = 0, b1 = 0;
  if (i < a.n) {
    b0 = __ldg(a.mrp + i);
    b1 = __ldg(a.mrp + i + 1);
  }
  int nch = (int)((b1 - b0 + 7) >> 3);
  nch = max(nch, __shfl_xor_sync(kFull, nch, 8));
  nch = max(nch, __shfl_xor_sync(kFull, nch, 16));
  int c = -1;
  VT mv = VT(0);
  if (b0 + e < b1) {
    c = __ldg(a.mci + b0 + e);
    mv = __ldg(mvals + b0 + e);
  }
  VT acc[4] = {VT(0), VT(0), VT(0), VT(0)};
  for (int t = 0; t < nch; t++) {
    int cn = -1;
    VT mn = VT(0);
    const long long en = b0 + 8LL * (t + 1) + e;
    if (en < b1) {
      cn = __ldg(a.mci + en);
      mn = __ldg(mvals + en);
    }
    VT pv[32];
#pragma unroll
    for (int s = 0; s < 32; s++) {
      const int cc = __shfl_sync(kFull, c, s);
      pv[s] = (act && cc >= 0) ? __ldg(x + (long long)cc * kBpLd + lane) : VT(0);
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int e2 = 0; e2 < 8; e2++) {
        const int cc = __shfl_sync(kFull, c, 8 * r + e2);
        const VT mm = __shfl_sync(kFull, mv, 8 * r + e2);
        if (cc >= 0) acc[r] = fma_rn(mm, pv[8 * r + e2], acc[r]);
      }
    c = cn;
    mv = mn;
  }
#pragma unroll
  for (int r = 0; r < 4; r++) y[r] = (double)acc[r];
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
  const double s = rows32([&](int t, double* o) {
    double bv[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      bv[r] = (act && i < a.n) ? __ldg(a.b + i * kBpLd + lane) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      o[r] = 0.0;
      if (act && i < a.n) {
        a.x[i * kBpLd + lane] = 0.0;
        a.r[i * kBpLd + lane] = bv[r];
        if (a.mixed) a.r32[i * kBpLd + lane] = __double2float_rn(bv[r]);
        o[r] = __dmul_rn(bv[r], bv[r]);
      }
    }
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
  const double* __restrict__ rv = a.r;
  const double s = rows32([&](int t, double* o) {
    double rr[4], z[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      rr[r] = (act && i < a.n) ? __ldg(rv + i * kBpLd + lane) : 0.0;
    }
    if (a.precond == 0) {
#pragma unroll
      for (int r = 0; r < 4; r++) z[r] = rr[r];
    } else if (a.precond == 1) {
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const long long i = row0 + t + r;
        z[r] = (act && i < a.n) ? __ddiv_rn(rr[r], __ldg(a.diag + i)) : 0.0;
      }
    } else if (a.mixed) {
      m_rows4(a, a.mv32, row0 + t, (const float*)a.r32, lane, act, z);
    } else {
      m_rows4(a, a.mv, row0 + t, rv, lane, act, z);
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      o[r] = 0.0;
      if (act && i < a.n) {
        a.z[i * kBpLd + lane] = z[r];
        o[r] = __dmul_rn(rr[r], z[r]);
      }
    }
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
  const double* __restrict__ zv = a.z;
  double* __restrict__ pv = a.p;
  for (int t = 0; t < 32; t += 8) {
    double zz[8], pp[8];
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const long long i = row0 + t + r;
      zz[r] = i < a.n ? __ldg(zv + i * kBpLd + lane) : 0.0;
      pp[r] = (!first && i < a.n) ? pv[i * kBpLd + lane] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const long long i = row0 + t + r;
      if (i < a.n) {
        const double pn = first ? zz[r] : __fma_rn(be, pp[r], zz[r]);
        pv[i * kBpLd + lane] = pn;
        if (a.mixed) a.p32[i * kBpLd + lane] = __double2float_rn(pn);
      }
    }
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
  AGroup<double> g;
  AGroup<float> g32;
  if (a.W <= 8) {
    if (a.mixed)
      a_group_load(a, a.ell_val32, row0, lane, g32.cn, g32.vn);
    else
      a_group_load(a, a.ell_val, row0, lane, g.cn, g.vn);
  }
  const double s = rows32([&](int t, double* o) {
    double q[4];
    if (a.mixed)
      a_rows4(a, a.ell_val32, g32, row0 + t, t + 4 < 32, (const float*)a.p32, lane, act, q);
    else
      a_rows4(a, a.ell_val, g, row0 + t, t + 4 < 32, (const double*)a.p, lane, act, q);
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      o[r] = 0.0;
      if (act && i < a.n) {
        a.q[i * kBpLd + lane] = q[r];
        o[r] = __dmul_rn(__ldg(a.p + i * kBpLd + lane), q[r]);
      }
    }
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
  double* __restrict__ xv = a.x;
  double* __restrict__ rv = a.r;
  const double* __restrict__ pv = a.p;
  const double* __restrict__ qv = a.q;
  const double s = rows32([&](int t, double* o) {
    double xx[4], pp[4], qq[4], rr[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      const bool ok = act && i < a.n;
      const long long e = i * kBpLd + lane;
      xx[r] = ok ? xv[e] : 0.0;
      pp[r] = ok ? __ldg(pv + e) : 0.0;
      qq[r] = ok ? __ldg(qv + e) : 0.0;
      rr[r] = ok ? rv[e] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      o[r] = 0.0;
      if (act && i < a.n) {
        const long long e = i * kBpLd + lane;
        xv[e] = __fma_rn(al, pp[r], xx[r]);
        const double rn = __fma_rn(-al, qq[r], rr[r]);
        rv[e] = rn;
        if (a.mixed) a.r32[e] = __double2float_rn(rn);
        o[r] = __dmul_rn(rn, rn);
      }
    }
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
  AGroup<double> g;
  if (a.W <= 8) a_group_load(a, a.ell_val, row0, lane, g.cn, g.vn);
  const double s = rows32([&](int t, double* o) {
    double y[4];
    a_rows4(a, a.ell_val, g, row0 + t, t + 4 < 32, (const double*)a.x, lane, act, y);
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const long long i = row0 + t + r;
      o[r] = 0.0;
      if (act && i < a.n) {
        const double d = __dsub_rn(__ldg(a.b + i * kBpLd + lane), y[r]);
        o[r] = __dmul_rn(d, d);
      }
    }
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
