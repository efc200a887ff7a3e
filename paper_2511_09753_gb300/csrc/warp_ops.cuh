// Warp-level building blocks of the column pass.  One warp owns one column
// at a time; every list lives in that warp's shared-memory scratch as a
// row-sorted array of (row, value) with value != 0.  All functions are
// called by the 32 lanes of the warp together.
//
// Arithmetic order is fixed so that results do not depend on the launch
// shape:
//   (A X)[r]      fma chain over k ascending, acc = fma(a_rk, x_k, acc)
//   column dot    x*y in FP64 over the common rows, balanced pairwise tree over
//                 the row-ascending term list padded with zeros
//   combination   computed in FP64, rounded once to the value type
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace spai {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// |v| as an unsigned key that orders like the magnitude
__device__ __forceinline__ uint32_t absbits(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ __forceinline__ uint64_t absbits(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

template <typename V> struct KeyOf;
template <> struct KeyOf<float> { typedef uint32_t T; };
template <> struct KeyOf<double> { typedef uint64_t T; };

// Balanced pairwise sum across the 32 lanes (lane i holds term i): the xor
// butterfly combines adjacent blocks level by level, and IEEE addition is
// commutative, so every lane ends with the same contiguous-tree sum.
__device__ __forceinline__ double warp_tree32(double v) {
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, m));
  return v;
}

__device__ __forceinline__ int lower_bound(const int* a, int L, int x) {
  int lo = 0, hi = L;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Pairwise sum of t[0..L) padded to max(32, next power of two); t must have
// room for that many doubles.  Levels above 32 pair adjacent entries in place.
__device__ inline double warp_pairwise(double* t, int L, int lane) {
  int P2 = 32;
  while (P2 < L) P2 <<= 1;
  for (int i = L + lane; i < P2; i += 32) t[i] = 0.0;
  __syncwarp();
  for (int len = P2; len > 32; len >>= 1) {
    int half = len >> 1;
    for (int base = 0; base < half; base += 32) {
      int i = base + lane;
      double a = t[2 * i], b = t[2 * i + 1];
      __syncwarp();
      t[i] = __dadd_rn(a, b);
      __syncwarp();
    }
  }
  double v = t[lane];
  __syncwarp();
  return warp_tree32(v);
}

template <typename V>
__device__ double warp_norm2(const V* v, int L, double* t, int lane) {
  for (int i = lane; i < L; i += 32) {
    double x = (double)v[i];
    t[i] = __dmul_rn(x, x);
  }
  __syncwarp();
  return warp_pairwise(t, L, lane);
}

// Inner product over the common rows of two row-sorted lists.
template <typename V>
__device__ double warp_dot(const int* xr, const V* xv, int Lx, const int* yr, const V* yv, int Ly,
                           double* t, int lane) {
  int L = 0;
  for (int base = 0; base < Lx; base += 32) {
    int i = base + lane;
    bool hit = false;
    double term = 0.0;
    if (i < Lx) {
      int r = xr[i];
      int lb = lower_bound(yr, Ly, r);
      if (lb < Ly && yr[lb] == r) {
        hit = true;
        term = __dmul_rn((double)xv[i], (double)yv[lb]);
      }
    }
    unsigned b = __ballot_sync(kFull, hit);
    if (hit) t[L + __popc(b & lanemask_lt())] = term;
    L += __popc(b);
  }
  __syncwarp();
  return warp_pairwise(t, L, lane);
}

// In-place removal of exact zeros, order kept.
template <typename V>
__device__ int compact_nonzero(int* r, V* v, int L, int lane) {
  int outn = 0;
  for (int base = 0; base < L; base += 32) {
    int i = base + lane;
    int rr = 0;
    V vv = V(0);
    bool nz = false;
    if (i < L) {
      rr = r[i];
      vv = v[i];
      nz = vv != V(0);
    }
    unsigned b = __ballot_sync(kFull, nz);
    __syncwarp();
    if (nz) {
      int pos = outn + __popc(b & lanemask_lt());
      r[pos] = rr;
      v[pos] = vv;
    }
    outn += __popc(b);
    __syncwarp();
  }
  return outn;
}

// Combination functors: computed in FP64, rounded once to V.
template <typename V> struct CombAxpy {  // x + c*y
  double c;
  __device__ V operator()(V x, V y) const { return (V)__fma_rn(c, (double)y, (double)x); }
};
template <typename V> struct CombLin {   // d*x + g*y
  double d, g;
  __device__ V operator()(V x, V y) const {
    return (V)__fma_rn(d, (double)x, __dmul_rn(g, (double)y));
  }
};
template <typename V> struct CombAdd {   // x + y
  __device__ V operator()(V x, V y) const { return (V)__dadd_rn((double)x, (double)y); }
};

// out = pattern union of A and B with value f(a or 0, b or 0); zeros removed.
// dp needs Lb + 1 u16 entries.  Returns the output length.
template <typename V, typename F>
__device__ int warp_union(const int* ar, const V* av, int La, const int* br, const V* bv, int Lb,
                          int* outr, V* outv, uint16_t* dp, F f, int lane) {
  int run = 0;
  for (int base = 0; base < Lb; base += 32) {
    int i = base + lane;
    bool dup = false;
    if (i < Lb) {
      int r = br[i];
      int lb = lower_bound(ar, La, r);
      dup = lb < La && ar[lb] == r;
    }
    unsigned b = __ballot_sync(kFull, dup);
    if (i < Lb) dp[i] = (uint16_t)(run + __popc(b & lanemask_lt()));
    run += __popc(b);
  }
  if (lane == 0) dp[Lb] = (uint16_t)run;
  __syncwarp();
  int U = La + Lb - run;
  for (int i = lane; i < La; i += 32) {
    int r = ar[i];
    int lb = lower_bound(br, Lb, r);
    bool has = lb < Lb && br[lb] == r;
    int pos = i + lb - (int)dp[lb];
    outr[pos] = r;
    outv[pos] = f(av[i], has ? bv[lb] : V(0));
  }
  for (int i = lane; i < Lb; i += 32) {
    int r = br[i];
    int lb = lower_bound(ar, La, r);
    if (!(lb < La && ar[lb] == r)) {
      int pos = i - (int)dp[i] + lb;
      outr[pos] = r;
      outv[pos] = f(V(0), bv[i]);
    }
  }
  __syncwarp();
  return compact_nonzero(outr, outv, U, lane);
}

// Hard thresholding (Sec. 6.1, per column): copy the `cap` entries of the
// row-sorted list src with the largest |v| (ties: smaller row) to dst, in row
// order.  If L <= cap the list is copied unchanged.  When `drop` is 0 the
// list is not thresholded; a list longer than cap then raises *overflow and
// is truncated so that no buffer is overrun.
template <typename V>
__device__ int warp_select(const int* sr, const V* sv, int L, int cap, int* dr, V* dv,
                           uint32_t* hist, int drop, int* overflow, int lane) {
  typedef typename KeyOf<V>::T K;
  if (L <= cap || !drop) {
    if (L > cap) {
      *overflow = 1;
      L = cap;
    }
    for (int i = lane; i < L; i += 32) {
      dr[i] = sr[i];
      dv[i] = sv[i];
    }
    __syncwarp();
    return L;
  }
  K prefix = 0, pmask = 0;
  int need = cap;
  bool exact = false;
  for (int d = (int)sizeof(K) - 1; d >= 0; d--) {
    const int shift = 8 * d;
    for (int b = lane; b < 256; b += 32) hist[b] = 0;
    __syncwarp();
    for (int i = lane; i < L; i += 32) {
      K k = absbits(sv[i]);
      if ((k & pmask) == prefix) atomicAdd(&hist[(unsigned)(k >> shift) & 255u], 1u);
    }
    __syncwarp();
    unsigned c[8];
    int tot = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
      c[t] = hist[8 * lane + t];
      tot += (int)c[t];
    }
    int suf = tot;  // inclusive suffix over lanes >= lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int x = __shfl_down_sync(kFull, suf, o);
      if (lane + o < 32) suf += x;
    }
    int above = suf - tot;
    int found = -1, f_above = 0, f_cnt = 0;
#pragma unroll
    for (int t = 7; t >= 0; t--) {
      if (found < 0 && above < need && above + (int)c[t] >= need) {
        found = 8 * lane + t;
        f_above = above;
        f_cnt = (int)c[t];
      }
      above += (int)c[t];
    }
    unsigned fb = __ballot_sync(kFull, found >= 0);
    int src = __ffs(fb) - 1;
    found = __shfl_sync(kFull, found, src);
    f_above = __shfl_sync(kFull, f_above, src);
    f_cnt = __shfl_sync(kFull, f_cnt, src);
    need -= f_above;
    prefix |= (K)found << shift;
    pmask |= (K)255 << shift;
    __syncwarp();
    if (f_cnt == need) {
      exact = true;
      break;
    }
  }
  int outn = 0, ties = 0;
  for (int base = 0; base < L; base += 32) {
    int i = base + lane;
    bool keep = false, tie = false;
    int rr = 0;
    V vv = V(0);
    if (i < L) {
      rr = sr[i];
      vv = sv[i];
      K k = absbits(vv) & pmask;
      keep = k > prefix;
      tie = k == prefix;
    }
    if (exact) {
      keep = keep || tie;
    } else {
      unsigned tb = __ballot_sync(kFull, tie);
      int trank = ties + __popc(tb & lanemask_lt());
      keep = keep || (tie && trank < need);
      ties += __popc(tb);
    }
    unsigned kb = __ballot_sync(kFull, keep);
    if (keep) {
      int pos = outn + __popc(kb & lanemask_lt());
      dr[pos] = rr;
      dv[pos] = vv;
    }
    outn += __popc(kb);
  }
  __syncwarp();
  return outn;
}

// One stable LSD radix pass over 8 bits of the keys.
__device__ inline void radix_pass(const uint32_t* kin, const uint16_t* iin, uint32_t* kout,
                           uint16_t* iout, int N, int shift, uint32_t* hist, int lane) {
  for (int b = lane; b < 256; b += 32) hist[b] = 0;
  __syncwarp();
  for (int q = lane; q < N; q += 32) atomicAdd(&hist[(kin[q] >> shift) & 255u], 1u);
  __syncwarp();
  unsigned c[8];
  unsigned tot = 0;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    c[t] = hist[8 * lane + t];
    tot += c[t];
  }
  unsigned inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned x = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += x;
  }
  unsigned run = inc - tot;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    hist[8 * lane + t] = run;
    run += c[t];
  }
  __syncwarp();
  for (int base = 0; base < N; base += 32) {
    int q = base + lane;
    bool act = q < N;
    unsigned am = __ballot_sync(kFull, act);
    if (act) {
      uint32_t k = kin[q];
      unsigned d = (k >> shift) & 255u;
      unsigned peers = __match_any_sync(am, d);
      int rank = __popc(peers & lanemask_lt());
      unsigned pos = hist[d] + rank;
      kout[pos] = k;
      iout[pos] = iin[q];
      __syncwarp(am);
      if (rank == 0) hist[d] += __popc(peers);
    }
    __syncwarp();
  }
}

struct SpgemmScratch {
  uint32_t* key0;
  uint32_t* key1;
  uint16_t* idx0;
  uint16_t* idx1;
  uint16_t* hp;
  uint32_t* hist;
};

// out = A X (diag < 0) or e_diag - A X (diag >= 0) for one column X; exact
// zeros removed; output row-sorted.  Expansion-sort-compress: every product
// (k, r) of the column is expanded, stably sorted by r (so k stays ascending
// inside each r), and each r is accumulated by an fma chain.
template <typename VC>
__device__ int warp_spgemm(const PassParams& p, const SpgemmScratch& s, VC* aval, const int* xr,
                           const VC* xv, int L, int diag, int* outr, VC* outv, int lane) {
  const int W = p.W;
  const int P = L * W;
  const int Ptot = P + (diag >= 0 ? 1 : 0);
  if (Ptot == 0) return 0;
  const VC* ev = (const VC*)p.ell_val;
  unsigned rmin = 0xffffffffu, rmax = 0u;
  for (int q = lane; q < P; q += 32) {
    int i = (int)__umulhi((unsigned)q, p.magicW);
    int t = q - i * W;
    long long e = (long long)xr[i] * W + t;
    int col = __ldg(p.ell_col + e);
    VC a = __ldg(ev + e);
    s.key0[q] = (uint32_t)col;
    aval[q] = a;
    rmin = min(rmin, (unsigned)col);
    rmax = max(rmax, (unsigned)col);
  }
  if (diag >= 0) {
    if (lane == 0) s.key0[P] = (uint32_t)diag;
    rmin = min(rmin, (unsigned)diag);
    rmax = max(rmax, (unsigned)diag);
  }
  rmin = __reduce_min_sync(kFull, rmin);
  rmax = __reduce_max_sync(kFull, rmax);
  __syncwarp();
  for (int q = lane; q < Ptot; q += 32) {
    s.key0[q] -= rmin;
    s.idx0[q] = (uint16_t)q;
  }
  __syncwarp();
  unsigned range = rmax - rmin;
  int bits = range ? 32 - __clz(range) : 0;
  int passes = (bits + 7) >> 3;
  uint32_t* kin = s.key0;
  uint16_t* iin = s.idx0;
  uint32_t* kout = s.key1;
  uint16_t* iout = s.idx1;
  for (int ps = 0; ps < passes; ps++) {
    radix_pass(kin, iin, kout, iout, Ptot, 8 * ps, s.hist, lane);
    uint32_t* tk = kin; kin = kout; kout = tk;
    uint16_t* ti = iin; iin = iout; iout = ti;
  }
  int U = 0;
  for (int base = 0; base < Ptot; base += 32) {
    int q = base + lane;
    bool head = q < Ptot && (q == 0 || kin[q] != kin[q - 1]);
    unsigned b = __ballot_sync(kFull, head);
    if (head) s.hp[U + __popc(b & lanemask_lt())] = (uint16_t)q;
    U += __popc(b);
  }
  if (lane == 0) s.hp[U] = (uint16_t)Ptot;
  __syncwarp();
  int outn = 0;
  for (int base = 0; base < U; base += 32) {
    int u = base + lane;
    VC val = VC(0);
    int r = 0;
    bool nz = false;
    if (u < U) {
      int s0 = s.hp[u], s1 = s.hp[u + 1];
      VC acc = VC(0);
      for (int q = s0; q < s1; q++) {
        int pi = iin[q];
        if (pi < P) {
          int i = (int)__umulhi((unsigned)pi, p.magicW);
          acc = vfma(aval[pi], xv[i], acc);
        }
      }
      r = (int)(kin[s0] + rmin);
      if (diag >= 0) val = (r == diag) ? (VC(1) - acc) : -acc;
      else val = acc;
      nz = val != VC(0);
    }
    unsigned b = __ballot_sync(kFull, nz);
    if (nz) {
      int pos = outn + __popc(b & lanemask_lt());
      outr[pos] = r;
      outv[pos] = val;
    }
    outn += __popc(b);
  }
  __syncwarp();
  return outn;
}

}  // namespace spai
