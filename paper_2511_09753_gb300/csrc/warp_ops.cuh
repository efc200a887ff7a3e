// Warp-level building blocks of the column pass.  One warp owns one column
// at a time; every list lives in that warp's shared-memory scratch as an
// array of (row, value) with distinct rows and value != 0, in no particular
// order.  All functions are called by the 32 lanes of the warp together.
//
// The arithmetic does not depend on list order or launch shape:
//   (A X)[r]      fma chain over k ascending, acc = fma(a_rk, x_k, acc)
//   column dot    FP64 products over the common rows, summed exactly in a
//                 128-bit fixed point anchored at the largest term, rounded once
//   combination   computed in FP64, rounded once to the value type
//   hard threshold keeps the cap largest |v|, ties to the smaller row
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

// Pairwise sum of t[0..L) zero-padded to max(32, next power of two); levels
// above 32 pair adjacent entries in place (t needs only L entries).
__device__ inline double warp_pairwise(double* t, int L, int lane) {
  int P2 = 32;
  while (P2 < L) P2 <<= 1;
  int cur = L;
  for (int len = P2; len > 32; len >>= 1) {
    const int next = (cur + 1) >> 1;
    for (int base = 0; base < next; base += 32) {
      int i = base + lane;
      double a = (2 * i < cur) ? t[2 * i] : 0.0;
      double b = (2 * i + 1 < cur) ? t[2 * i + 1] : 0.0;
      __syncwarp();
      if (i < next) t[i] = __dadd_rn(a, b);
      __syncwarp();
    }
    cur = next;
  }
  double v = lane < cur ? t[lane] : 0.0;
  __syncwarp();
  return warp_tree32(v);
}

// ------------------------------------------------------ order-free dot sum
// A column inner product is the exact two's-complement sum of its FP64 terms
// in a 128-bit fixed point with unit 2^(E-110), E the largest exponent among
// the terms (each term truncated toward zero to the unit), rounded once to
// the nearest double (ties to even).  Integer addition is associative, so
// neither the term order nor the reduction order matters.  Terms come from
// functors f(i), i < L, each lane taking i = lane, lane + 32, ...; up to
// three sums are reduced together so their latencies overlap.

// A term held exactly as sign, biased FP64 exponent (0 for a zero, 1 for a
// subnormal) and 53-bit significand (hidden bit included): the fields of the
// FP64 number it equals.
struct Term {
  unsigned long long m;
  int e;
  int neg;
};

__device__ __forceinline__ Term term_of(double t) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(t);
  Term r;
  const int b = (int)((bits >> 52) & 0x7ff);
  r.m = bits & ((1ull << 52) - 1);
  r.neg = (int)(bits >> 63);
  if (b == 0) {
    r.e = r.m ? 1 : 0;
  } else {
    r.e = b;
    r.m |= 1ull << 52;
  }
  return r;
}

// The product of two FP32 numbers is exact in FP64 (48 significant bits), so
// its FP64 fields follow from the integer product of the significands: the
// same Term as term_of((double)a * (double)b), without FP64 instructions
// (GB300's FP64 pipe is narrow).  Inf or NaN operands give an exponent of
// 2047, so the sum comes out non-finite as in FP64.
__device__ __forceinline__ Term term_prod(float a, float b) {
  const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
  int ea = (int)((ua >> 23) & 0xff), eb = (int)((ub >> 23) & 0xff);
  uint32_t ma = ua & 0x7fffffu, mb = ub & 0x7fffffu;
  Term r;
  r.neg = (int)((ua ^ ub) >> 31);
  if (ea == 255 || eb == 255) {
    r.e = 2047;
    r.m = 1ull << 52;
    return r;
  }
  if (ea) ma |= 0x800000u; else ea = 1;
  if (eb) mb |= 0x800000u; else eb = 1;
  const unsigned long long mm = (unsigned long long)ma * mb;
  if (mm == 0ull) {
    r.e = 0;
    r.m = 0ull;
    return r;
  }
  const int top = 63 - __clzll((long long)mm);  // <= 47
  r.e = top + ea + eb - 300 + 1023;              // >= 1: no FP64 subnormal arises
  r.m = mm << (52 - top);
  return r;
}

__device__ __forceinline__ Term term_prod(double a, double b) { return term_of(__dmul_rn(a, b)); }

// 128-bit two's-complement accumulator held as (hi, lo) 64-bit limbs.
struct Fix128 {
  unsigned long long lo;
  long long hi;
};

// S += t at unit 2^(eb-1133), t truncated toward zero to that unit.  No
// branches: the shifts are clamped (m < 2^53, so a right shift by 53 or more
// leaves nothing), and a negative term is added as its two's complement.
__device__ __forceinline__ void term_add(Fix128& S, const Term& t, int eb) {
  const unsigned long long m = t.m;
  const int sh = (t.e ? t.e : 1) - eb + 58;  // <= 58: the term fits in 111 bits
  const int sl = max(sh, 0), sr = min(max(-sh, 0), 63);
  const unsigned long long lo = (m << sl) >> sr;
  const unsigned long long hi = (m >> 1) >> (63 - sl);  // m >> (64 - sl), 0 for sl = 0
  const unsigned __int128 nm = (unsigned __int128)0 - (unsigned __int128)(unsigned)t.neg;
  const unsigned __int128 v = ((((unsigned __int128)hi << 64) | lo) ^ nm) - nm;
  const unsigned __int128 acc =
      ((((unsigned __int128)(unsigned long long)S.hi) << 64) | S.lo) + v;
  S.lo = (unsigned long long)acc;
  S.hi = (long long)(unsigned long long)(acc >> 64);
}

// Warp sum of the 32 lanes' accumulators: each 128-bit two's-complement value
// is cut into six 24-bit limbs (the top one sign-extended to 24 bits, so the
// limbs represent it modulo 2^144); a limb's warp sum stays below 2^29 and
// comes from one redux.sync; the limb sums, shifted into place, add up to the
// total modulo 2^128, which is exact because the total fits in 128 bits.
__device__ __forceinline__ void fix_limb_sums(const Fix128& S, unsigned s[6]) {
  const unsigned long long lo = S.lo, hi = (unsigned long long)S.hi;
  const unsigned l0 = (unsigned)lo & 0xffffffu;
  const unsigned l1 = (unsigned)(lo >> 24) & 0xffffffu;
  const unsigned l2 = (unsigned)((lo >> 48) | (hi << 16)) & 0xffffffu;
  const unsigned l3 = (unsigned)(hi >> 8) & 0xffffffu;
  const unsigned l4 = (unsigned)(hi >> 32) & 0xffffffu;
  const unsigned l5 = (unsigned)(hi >> 56) | (S.hi < 0 ? 0xffff00u : 0u);
  s[0] = __reduce_add_sync(kFull, l0);
  s[1] = __reduce_add_sync(kFull, l1);
  s[2] = __reduce_add_sync(kFull, l2);
  s[3] = __reduce_add_sync(kFull, l3);
  s[4] = __reduce_add_sync(kFull, l4);
  s[5] = __reduce_add_sync(kFull, l5);
}

__device__ __forceinline__ Fix128 fix_from_limbs(const unsigned s[6]) {
  unsigned __int128 t = (unsigned __int128)s[0] + ((unsigned __int128)s[1] << 24) +
                        ((unsigned __int128)s[2] << 48) + ((unsigned __int128)s[3] << 72) +
                        ((unsigned __int128)s[4] << 96) + ((unsigned __int128)s[5] << 120);
  Fix128 S;
  S.lo = (unsigned long long)t;
  S.hi = (long long)(unsigned long long)(t >> 64);
  return S;
}

__device__ __forceinline__ void fix_allreduce(Fix128& S) {
  unsigned s[6];
  fix_limb_sums(S, s);
  S = fix_from_limbs(s);
}

// round S * 2^(eb-1133) to the nearest double (ties to even)
__device__ __forceinline__ double fix_to_double(Fix128 S, int eb) {
  if ((S.lo | (unsigned long long)S.hi) == 0ull || eb == 0) return 0.0;
  const bool neg = S.hi < 0;
  unsigned long long ulo = S.lo, uhi = (unsigned long long)S.hi;
  if (neg) {
    ulo = ~ulo + 1ull;
    uhi = ~uhi + (ulo == 0ull ? 1ull : 0ull);
  }
  const int bl = uhi ? 128 - __clzll((long long)uhi) : 64 - __clzll((long long)ulo);
  unsigned long long mant;
  int shift = 0;
  if (bl <= 53) {
    mant = ulo;
  } else {
    shift = bl - 53;  // 1 .. 74
    bool up;
    if (shift < 64) {
      mant = (ulo >> shift) | (uhi << (64 - shift));
      unsigned long long rem = ulo & ((1ull << shift) - 1ull);
      unsigned long long half = 1ull << (shift - 1);
      up = rem > half || (rem == half && (mant & 1ull));
    } else if (shift == 64) {
      mant = uhi;
      unsigned long long half = 1ull << 63;
      up = ulo > half || (ulo == half && (mant & 1ull));
    } else {
      const int s2 = shift - 64;  // 1 .. 10
      mant = uhi >> s2;
      unsigned long long rhi = uhi & ((1ull << s2) - 1ull);
      unsigned long long hhi = 1ull << (s2 - 1);
      up = rhi > hhi || (rhi == hhi && (ulo != 0ull || (mant & 1ull)));
    }
    if (up) mant++;
  }
  // mant * 2^k; mant <= 2^53 converts exactly.  While the product stays
  // normal and finite, scaling by 2^k only adds k to the exponent field.
  const int k = shift + eb - 1133;
  const double d = __ull2double_rn(mant);
  const double r = (k >= -1022 && k <= 969)
                       ? __longlong_as_double(__double_as_longlong(d) + (long long)k * (1ll << 52))
                       : ldexp(d, k);
  return neg ? -r : r;
}

struct NoTerms {
  __device__ Term operator()(int) const { return Term{0ull, 0, 0}; }
};

template <typename F>
__device__ __forceinline__ Term term_at(const F& f, int i, int L) {
  return i < L ? f(i) : Term{0ull, 0, 0};
}

// The first two terms of each lane stay in registers between the exponent
// pass and the accumulation pass; only the terms past 64 are evaluated twice.
template <int K, typename F0, typename F1 = NoTerms, typename F2 = NoTerms>
__device__ void fixsum(double* out, int lane, const F0& f0, int L0, const F1& f1 = F1(), int L1 = 0,
                       const F2& f2 = F2(), int L2 = 0) {
  const Term a0 = term_at(f0, lane, L0), b0 = term_at(f0, lane + 32, L0);
  Term a1 = {0ull, 0, 0}, b1 = {0ull, 0, 0}, a2 = {0ull, 0, 0}, b2 = {0ull, 0, 0};
  if (K > 1) {
    a1 = term_at(f1, lane, L1);
    b1 = term_at(f1, lane + 32, L1);
  }
  if (K > 2) {
    a2 = term_at(f2, lane, L2);
    b2 = term_at(f2, lane + 32, L2);
  }
  int e0 = max(a0.e, b0.e), e1 = max(a1.e, b1.e), e2 = max(a2.e, b2.e);
  for (int i = lane + 64; i < L0; i += 32) e0 = max(e0, f0(i).e);
  if (K > 1) for (int i = lane + 64; i < L1; i += 32) e1 = max(e1, f1(i).e);
  if (K > 2) for (int i = lane + 64; i < L2; i += 32) e2 = max(e2, f2(i).e);
  e0 = __reduce_max_sync(kFull, e0);
  if (K > 1) e1 = __reduce_max_sync(kFull, e1);
  if (K > 2) e2 = __reduce_max_sync(kFull, e2);
  // the cached terms (zero past a list's end) in one straight-line block, so
  // the sums' carry chains interleave
  Fix128 S0 = {0ull, 0ll}, S1 = {0ull, 0ll}, S2 = {0ull, 0ll};
  term_add(S0, a0, e0);
  if (K > 1) term_add(S1, a1, e1);
  if (K > 2) term_add(S2, a2, e2);
  term_add(S0, b0, e0);
  if (K > 1) term_add(S1, b1, e1);
  if (K > 2) term_add(S2, b2, e2);
  for (int i = lane + 64; i < L0; i += 32) term_add(S0, f0(i), e0);
  if (K > 1) for (int i = lane + 64; i < L1; i += 32) term_add(S1, f1(i), e1);
  if (K > 2) for (int i = lane + 64; i < L2; i += 32) term_add(S2, f2(i), e2);
  if (K == 1) {
    fix_allreduce(S0);
    out[0] = fix_to_double(S0, e0);
    return;
  }
  // lane q < K rounds sum q (the other lanes sum 0); the doubles are then
  // broadcast, so each rounding runs once per warp instead of K times
  unsigned a[6], b[6], c[6] = {0u, 0u, 0u, 0u, 0u, 0u};
  fix_limb_sums(S0, a);
  fix_limb_sums(S1, b);
  if (K > 2) fix_limb_sums(S2, c);
  unsigned s[6];
#pragma unroll
  for (int i = 0; i < 6; i++) s[i] = lane == 1 ? b[i] : (K > 2 && lane == 2) ? c[i] : a[i];
  const int e = lane == 1 ? e1 : (K > 2 && lane == 2) ? e2 : e0;
  const double d = fix_to_double(fix_from_limbs(s), e);
  out[0] = __shfl_sync(kFull, d, 0);
  out[1] = __shfl_sync(kFull, d, 1);
  if (K > 2) out[2] = __shfl_sync(kFull, d, 2);
}

// ------------------------------------------------------------- hash table
// Open addressing with linear probing in shared memory: keys (row, -1 =
// empty), values, and the list of occupied slots in insertion order.  The
// capacity is a power of two above the largest possible number of distinct
// rows, so probing always terminates.

struct HashT {
  int* key;
  void* val;
  uint16_t* occ;
  int H;
};

// the top log2(H) bits of the product (H a power of two, at least 32 in
// every layout)
__device__ __forceinline__ int hslot(int r, int H) {
  return (int)(((unsigned)r * 0x9E3779B1u) >> (__clz(H) + 1));
}

// insert r; a new slot gets value 0 and *isnew = true
template <typename V>
__device__ __forceinline__ int hash_insert(const HashT& h, int r, bool* isnew) {
  V* hv = (V*)h.val;
  int s = hslot(r, h.H);
  for (;;) {
    int k = atomicCAS(&h.key[s], -1, r);
    if (k == -1) {
      hv[s] = V(0);
      *isnew = true;
      return s;
    }
    if (k == r) return s;
    s = (s + 1) & (h.H - 1);
  }
}

// value of row r, or 0 if absent
template <typename V>
__device__ __forceinline__ V hash_find(const HashT& h, int r) {
  const V* hv = (const V*)h.val;
  int s = hslot(r, h.H);
  for (;;) {
    int k = h.key[s];
    if (k == r) return hv[s];
    if (k == -1) return V(0);
    s = (s + 1) & (h.H - 1);
  }
}

// finish the insertion of r whose first attempt, at its home slot, returned
// got (-1: claimed there): probe on as hash_insert does; returns the slot
__device__ __forceinline__ int hash_settle(const HashT& h, int r, int got, bool* isnew) {
  int q = hslot(r, h.H);
  while (got != -1 && got != r) {
    q = (q + 1) & (h.H - 1);
    got = atomicCAS(&h.key[q], -1, r);
  }
  *isnew = got == -1;
  return q;
}

// append the slots that lanes inserted as new to the occupied list
__device__ __forceinline__ void occ_append(const HashT& h, int& cnt, bool isnew, int slot) {
  unsigned b = __ballot_sync(kFull, isnew);
  if (isnew) h.occ[cnt + __popc(b & lanemask_lt())] = (uint16_t)slot;
  cnt += __popc(b);
}

__device__ __forceinline__ void hash_clear_all(const HashT& h, int lane) {
  int4* k4 = (int4*)h.key;
  const int4 e = make_int4(-1, -1, -1, -1);
  for (int i = lane; i < h.H / 4; i += 32) k4[i] = e;
  __syncwarp();
}

// empty the table again (only the occupied slots are touched)
__device__ __forceinline__ void hash_clear(const HashT& h, int cnt, int lane) {
  __syncwarp();
  for (int i = lane; i < cnt; i += 32) h.key[h.occ[i]] = -1;
  __syncwarp();
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

// Union table: keys, the A value and the B value of each row.
struct UnionT {
  int* key;
  void* va;
  void* vb;
  uint16_t* occ;
  int H;
};

// slot of row r, or -1 if absent
__device__ __forceinline__ int hash_slot_of(const HashT& h, int r) {
  int s = hslot(r, h.H);
  for (;;) {
    const int k = h.key[s];
    if (k == r) return s;
    if (k == -1) return -1;
    s = (s + 1) & (h.H - 1);
  }
}

// out = pattern union of A and B with value f(a or 0, b or 0); exact zeros
// removed.  Returns the output length.  Rows are distinct within each list,
// so only B goes into the table: A's rows look B up and go straight to the
// output (a matched B slot is flagged), then B's unflagged rows follow.
template <typename V, typename F>
__device__ int warp_union(const UnionT& u, const int* ar, const V* av, int La, const int* br,
                          const V* bv, int Lb, int* outr, V* outv, F f, int lane) {
  HashT h;
  h.key = u.key;
  h.val = u.vb;
  h.occ = u.occ;
  h.H = u.H;
  V* hit = (V*)u.va;  // V(1) once an A row matched the slot
  V* vb = (V*)u.vb;
  hash_clear_all(h, lane);  // the table's bytes are shared with other scratch
  int cnt = 0;
  for (int base = 0; base < Lb; base += 32) {
    int i = base + lane;
    bool isnew = false;
    int s = -1;
    if (i < Lb) {
      s = hash_insert<V>(h, br[i], &isnew);
      vb[s] = bv[i];
      hit[s] = V(0);
    }
    occ_append(h, cnt, isnew, s);
  }
  __syncwarp();
  int outn = 0;
  for (int base = 0; base < La; base += 32) {
    int i = base + lane;
    bool nz = false;
    int r = 0;
    V v = V(0);
    if (i < La) {
      r = ar[i];
      const int s = hash_slot_of(h, r);
      V y = V(0);
      if (s >= 0) {
        y = vb[s];
        hit[s] = V(1);
      }
      v = f(av[i], y);
      nz = v != V(0);
    }
    unsigned bm = __ballot_sync(kFull, nz);
    if (nz) {
      int pos = outn + __popc(bm & lanemask_lt());
      outr[pos] = r;
      outv[pos] = v;
    }
    outn += __popc(bm);
  }
  __syncwarp();
  for (int base = 0; base < cnt; base += 32) {
    int i = base + lane;
    bool nz = false;
    int r = 0;
    V v = V(0);
    if (i < cnt) {
      const int s = u.occ[i];
      if (hit[s] == V(0)) {
        r = u.key[s];
        v = f(V(0), vb[s]);
        nz = v != V(0);
      }
    }
    unsigned bm = __ballot_sync(kFull, nz);
    if (nz) {
      int pos = outn + __popc(bm & lanemask_lt());
      outr[pos] = r;
      outv[pos] = v;
    }
    outn += __popc(bm);
  }
  __syncwarp();
  return outn;
}

// LOMR's two combinations from one table: S = f(Z, P) (exact zeros removed)
// and T = g(S, M) (exact zeros removed), the same values as
// warp_union(Z, P, f) followed by warp_union(S list, M, g).  M and P enter
// the table (a row of both has one slot); Z's rows look it up, and a slot a
// Z row matched is marked by storing -2 - row as its key (lookups of other
// rows probe past it, and the table is cleared before its next use); then
// the unmarked slots give the rows of P or M that Z does not have.
template <typename V, typename FS, typename FT>
__device__ void warp_union3(const UnionT& u, const int* zr, const V* zv, int Lz, const int* pr,
                            const V* pv, int Lp, const int* mr, const V* mv, int Lm, int* sr, V* sv,
                            int* Ls, int* tr, V* tv, int* Lt, FS f, FT g, int lane) {
  HashT h;
  h.key = u.key;
  h.val = u.vb;
  h.occ = u.occ;
  h.H = u.H;
  V* hm = (V*)u.va;  // M's value of the slot, or 0
  V* hp = (V*)u.vb;  // P's value of the slot, or 0
  hash_clear_all(h, lane);
  int cnt = 0;
  for (int base = 0; base < Lm; base += 32) {
    int i = base + lane;
    bool isnew = false;
    int q = -1;
    if (i < Lm) {
      q = hash_insert<V>(h, mr[i], &isnew);
      hm[q] = mv[i];
      hp[q] = V(0);
    }
    occ_append(h, cnt, isnew, q);
  }
  __syncwarp();
  for (int base = 0; base < Lp; base += 32) {
    int i = base + lane;
    bool isnew = false;
    int q = -1;
    if (i < Lp) {
      q = hash_insert<V>(h, pr[i], &isnew);
      if (isnew) hm[q] = V(0);
      hp[q] = pv[i];
    }
    occ_append(h, cnt, isnew, q);
  }
  __syncwarp();
  int ns = 0, nt = 0;
  for (int base = 0; base < Lz; base += 32) {
    int i = base + lane;
    bool s_nz = false, t_nz = false;
    int r = 0;
    V s = V(0), t = V(0);
    if (i < Lz) {
      r = zr[i];
      const int q = hash_slot_of(h, r);
      V p = V(0), m = V(0);
      if (q >= 0) {
        p = hp[q];
        m = hm[q];
        h.key[q] = -2 - r;
      }
      s = f(zv[i], p);
      s_nz = s != V(0);
      t = s_nz ? g(s, m) : m;  // a zero s is no row of the S list
      t_nz = t != V(0);
    }
    unsigned bs = __ballot_sync(kFull, s_nz), bt = __ballot_sync(kFull, t_nz);
    if (s_nz) {
      const int at = ns + __popc(bs & lanemask_lt());
      sr[at] = r;
      sv[at] = s;
    }
    if (t_nz) {
      const int at = nt + __popc(bt & lanemask_lt());
      tr[at] = r;
      tv[at] = t;
    }
    ns += __popc(bs);
    nt += __popc(bt);
  }
  __syncwarp();
  for (int base = 0; base < cnt; base += 32) {
    int i = base + lane;
    bool s_nz = false, t_nz = false;
    int r = 0;
    V s = V(0), t = V(0);
    if (i < cnt) {
      const int q = u.occ[i];
      r = u.key[q];
      if (r >= 0) {  // not matched by a Z row
        const V p = hp[q], m = hm[q];
        s = p != V(0) ? f(V(0), p) : V(0);
        s_nz = s != V(0);
        t = s_nz ? g(s, m) : m;
        t_nz = t != V(0);
      }
    }
    unsigned bs = __ballot_sync(kFull, s_nz), bt = __ballot_sync(kFull, t_nz);
    if (s_nz) {
      const int at = ns + __popc(bs & lanemask_lt());
      sr[at] = r;
      sv[at] = s;
    }
    if (t_nz) {
      const int at = nt + __popc(bt & lanemask_lt());
      tr[at] = r;
      tv[at] = t;
    }
    ns += __popc(bs);
    nt += __popc(bt);
  }
  __syncwarp();
  *Ls = ns;
  *Lt = nt;
}

// ------------------------------------------------------ 256-bin histograms
// 16-bit counts packed two per word (128 words): lane l owns bins [8l, 8l+8)
// = words [4l, 4l+4), read and cleared with one 16-byte access.

__device__ __forceinline__ void hist_clear(uint32_t* hist, int lane) {
  ((uint4*)hist)[lane] = make_uint4(0u, 0u, 0u, 0u);
}

// one count per active lane in bin d: a shared-memory atomic per lane (lanes
// with the same digit are serialised by the hardware; measured faster than
// grouping them with __match_any_sync first)
__device__ __forceinline__ void hist_add(uint32_t* hist, bool act, unsigned d) {
  if (act) atomicAdd(&hist[d >> 1], 1u << ((d & 1u) * 16u));
}

// The selection key of an entry: |v| as bits, or the largest key for the row
// that is always kept (keep_row; -1 for none), so that it ranks first.
template <typename V>
__device__ __forceinline__ typename KeyOf<V>::T sel_key(V v, int r, int keep_row) {
  typedef typename KeyOf<V>::T K;
  return r == keep_row ? (K)(~(K)0 >> 1) : absbits(v);
}

// Hard thresholding (Sec. 6.1, per column): copy the `cap` entries of list
// src with the largest |v| to dst (ties: smaller row), keeping src order.
// Row keep_row (>= 0), when present, is kept and counts toward cap.  With
// L <= cap the list is copied.  When `drop` is 0 the list is not
// thresholded; a list longer than cap then raises *overflow and is truncated
// so that no buffer is overrun.  tie: scratch of L ints.
template <typename V>
__device__ int warp_select(const int* sr, const V* sv, int L, int cap, int* dr, V* dv,
                           uint32_t* hist, int* tie, int drop, int* overflow, int lane,
                           int keep_row) {
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
  // lists of at most 64 entries (the usual case) keep their two keys per
  // lane in registers for every digit pass
  const bool small = L <= 64;
  K k0 = 0, k1 = 0;
  if (small) {
    if (lane < L) k0 = sel_key(sv[lane], sr[lane], keep_row);
    if (lane + 32 < L) k1 = sel_key(sv[lane + 32], sr[lane + 32], keep_row);
  }
  // digits of 8 bits from the top of the key's 31 (63) significant bits, so
  // the first digit is the exponent field of an FP32 |v|; the last is shorter
  for (int hi = 8 * (int)sizeof(K) - 1; hi > 0; hi -= 8) {
    const int shift = hi > 8 ? hi - 8 : 0;
    const unsigned dmask = (1u << (hi - shift)) - 1u;
    hist_clear(hist, lane);
    __syncwarp();
    if (small) {
      hist_add(hist, lane < L && (k0 & pmask) == prefix, (unsigned)(k0 >> shift) & dmask);
      hist_add(hist, lane + 32 < L && (k1 & pmask) == prefix, (unsigned)(k1 >> shift) & dmask);
    } else {
      for (int base = 0; base < L; base += 32) {
        int i = base + lane;
        bool act = false;
        unsigned dig = 0;
        if (i < L) {
          K k = absbits(sv[i]);
          if (keep_row >= 0 && sr[i] == keep_row) k = ~(K)0 >> 1;
          act = (k & pmask) == prefix;
          dig = (unsigned)(k >> shift) & dmask;
        }
        hist_add(hist, act, dig);
      }
    }
    __syncwarp();
    // the lane's 8 bins in two packed sums (their halves cannot carry: the
    // counts of all bins add up to at most L < 2^16)
    const uint4 w = ((const uint4*)hist)[lane];
    const unsigned ws = w.x + w.y + w.z + w.w;
    const int tot = (int)((ws & 0xffffu) + (ws >> 16));
    int suf = tot;  // inclusive suffix over lanes >= lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int x = __shfl_down_sync(kFull, suf, o);
      if (lane + o < 32) suf += x;
    }
    const int above = suf - tot;
    // the one lane whose bins hold the need-th largest key (1 <= need <= the
    // entries left), then its bins from the top, one per lane 0..7
    const int lh = max(__ffs(__ballot_sync(kFull, above < need && suf >= need)) - 1, 0);
    const int ab = __shfl_sync(kFull, above, lh);
    int ct = 0;
    if (lane < 8) {
      const int bin = 8 * lh + 7 - lane;
      ct = (int)((hist[bin >> 1] >> ((bin & 1) * 16)) & 0xffffu);
    }
    int inc = ct;  // inclusive prefix over lanes 0..7
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      int x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    const int t =
        max(__ffs(__ballot_sync(kFull, lane < 8 && ab + inc >= need && ab + inc - ct < need)) - 1, 0);
    const int found = 8 * lh + 7 - t;
    const int f_cnt = __shfl_sync(kFull, ct, t);
    const int f_above = ab + __shfl_sync(kFull, inc - ct, t);
    need -= f_above;
    prefix |= (K)found << shift;
    pmask |= (K)dmask << shift;
    __syncwarp();
    if (f_cnt == need) {
      exact = true;
      break;
    }
  }
  // exact: every entry whose masked key equals the prefix is kept.
  // Otherwise the full key equals the threshold for more than `need`
  // entries: keep the `need` of them with the smallest rows.
  int ntie = 0;
  if (!exact) {
    for (int base = 0; base < L; base += 32) {
      int i = base + lane;
      bool t = i < L && sel_key(sv[i], sr[i], keep_row) == prefix;
      unsigned b = __ballot_sync(kFull, t);
      if (t) tie[ntie + __popc(b & lanemask_lt())] = sr[i];
      ntie += __popc(b);
    }
    __syncwarp();
  }
  int outn = 0;
  for (int base = 0; base < L; base += 32) {
    int i = base + lane;
    bool keep = false;
    int rr = 0;
    V vv = V(0);
    if (i < L) {
      rr = sr[i];
      vv = sv[i];
      K k = (small ? (base ? k1 : k0) : sel_key(vv, rr, keep_row)) & pmask;
      keep = k > prefix;
      if (k == prefix) {
        if (exact) {
          keep = true;
        } else {
          int rank = 0;
          for (int q = 0; q < ntie; q++) rank += tie[q] < rr;
          keep = rank < need;
        }
      }
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

// ---------------------------------------------------------------- SpGEMM
// Accumulate A X (one column X, rows xr, values xv, length L, any order) in
// the hash table: after the call the table holds, for every row r reached,
// the fma chain over k ascending; returns the number of occupied slots (the
// occupied list holds them).  If diag >= 0, row diag is inserted as well.
//
// DIA layout (A stored by diagonal slots, offsets ascending): the product of
// x_k with slot s lands on r = k + off_s.  Slots are processed in descending
// offset, which for any fixed r is ascending k = r - off_s, so every chain
// has the canonical order; inside one slot distinct k give distinct r, so no
// two lanes touch the same accumulator.
template <typename VC>
__device__ int spgemm_dia(const PassParams& p, const HashT& h, const int* xr, const VC* xv, int L,
                          int diag, int seg, int lane) {
  const VC* dv = (const VC*)p.dia_val;
  VC* hv = (VC*)h.val;
  const int D = seg >= 0 ? p.seg_D[seg] : p.D, Dp = p.Dp;
  int cnt = 0;
  for (int s = D - 1; s >= 0; s--) {
    const int o = seg >= 0 ? p.seg_doff[seg * 32 + s] : p.dia_off[s];
    for (int base = 0; base < L; base += 32) {
      int i = base + lane;
      bool isnew = false;
      int slot = -1;
      if (i < L) {
        int k = xr[i];
        VC a = __ldg(dv + (long long)k * Dp + s);
        if (a != VC(0)) {
          slot = hash_insert<VC>(h, k + o, &isnew);
          hv[slot] = vfma(a, xv[i], hv[slot]);
        }
      }
      occ_append(h, cnt, isnew, slot);
    }
    __syncwarp();
  }
  if (diag >= 0) {
    bool isnew = false;
    int slot = -1;
    if (lane == 0) slot = hash_insert<VC>(h, diag, &isnew);
    occ_append(h, cnt, isnew, slot);
    __syncwarp();
  }
  return cnt;
}

// Short inputs (L <= 32, D <= 8): lane i owns entry i and gathers its row's
// slot values at once.  The rows of all products are claimed in the table
// first (order-free: the first attempts at the home slots are issued
// together, collisions probe on as in hash_insert), then the products are
// added slot by slot in descending offset -- the same chains as above, each
// round now a read-modify-write of slots already known.
template <typename VC>
__device__ int spgemm_dia32(const PassParams& p, const HashT& h, const int* xr, const VC* xv, int L,
                            int diag, int seg, int lane) {
  const VC* dv = (const VC*)p.dia_val;
  VC* hv = (VC*)h.val;
  const int D = seg >= 0 ? p.seg_D[seg] : p.D;
  const bool act = lane < L;
  int k = 0;
  VC x = VC(0);
  if (act) {
    k = xr[lane];
    x = xv[lane];
  }
  VC a[8];
  int sl[8];
#pragma unroll
  for (int s = 0; s < 8; s++) a[s] = VC(0);
  if (act) {  // rows padded to a multiple of 4 slots (zeros): whole vectors
    const VC* row = dv + (long long)k * p.Dp;
    if constexpr (sizeof(VC) == 4) {
      const float4 v0 = __ldg((const float4*)row);
      a[0] = v0.x; a[1] = v0.y; a[2] = v0.z; a[3] = v0.w;
      if (D > 4) {
        const float4 v1 = __ldg((const float4*)row + 1);
        a[4] = v1.x; a[5] = v1.y; a[6] = v1.z; a[7] = v1.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (2 * q < D) {
          const double2 v = __ldg((const double2*)row + q);
          a[2 * q] = v.x;
          a[2 * q + 1] = v.y;
        }
      }
    }
  }
  // first attempts: sl = the key found at the home slot (-1: claimed), or
  // -2 when there is no product
#pragma unroll
  for (int s = 0; s < 8; s++) {
    sl[s] = -2;
    if (s < D && a[s] != VC(0)) {
      const int r = k + (seg >= 0 ? p.seg_doff[seg * 32 + s] : p.dia_off[s]);
      sl[s] = atomicCAS(&h.key[hslot(r, h.H)], -1, r);
    }
  }
  // the diagonal row (R's "1 -"), claimed with the products' rows
  const int gd = (diag >= 0 && lane == 0) ? atomicCAS(&h.key[hslot(diag, h.H)], -1, diag) : -2;
  int cnt = 0;
  if (diag >= 0) {
    bool isnew = false;
    int slot = -1;
    if (gd != -2) {
      slot = hash_settle(h, diag, gd, &isnew);
      if (isnew) hv[slot] = VC(0);
    }
    occ_append(h, cnt, isnew, slot);
  }
#pragma unroll
  for (int s = 7; s >= 0; s--) {
    if (s < D) {
      bool isnew = false;
      int slot = -1;
      if (sl[s] != -2) {
        const int r = k + (seg >= 0 ? p.seg_doff[seg * 32 + s] : p.dia_off[s]);
        int q = hslot(r, h.H);
        int got = sl[s];
        while (got != -1 && got != r) {
          q = (q + 1) & (h.H - 1);
          got = atomicCAS(&h.key[q], -1, r);
        }
        isnew = got == -1;
        slot = q;
        if (isnew) hv[q] = VC(0);
      }
      sl[s] = slot;
      occ_append(h, cnt, isnew, slot);
    }
  }
  __syncwarp();
#pragma unroll
  for (int s = 7; s >= 0; s--) {
    if (s < D) {
      if (sl[s] >= 0) hv[sl[s]] = vfma(a[s], x, hv[sl[s]]);
      __syncwarp();
    }
  }
  return cnt;
}

// General ELL layout (A rows padded with column -1).  X must be row-sorted:
// products are generated k-major and lanes of one chunk that hit the same r
// apply their fma in lane order, so each r sees the chain over ascending k.
template <typename VC>
__device__ int spgemm_ell(const PassParams& p, const HashT& h, const int* xr, const VC* xv, int L,
                          int diag, int lane) {
  const int W = p.W;
  const int P = L * W;
  const VC* ev = (const VC*)p.ell_val;
  VC* hv = (VC*)h.val;
  int cnt = 0;
  for (int base = 0; base < P; base += 32) {
    int q = base + lane;
    bool act = false, isnew = false;
    int slot = -1;
    VC a = VC(0), x = VC(0);
    if (q < P) {
      int i = (int)__umulhi((unsigned)q, p.magicW);
      int t = q - i * W;
      long long e = (long long)xr[i] * W + t;
      int col = __ldg(p.ell_col + e);
      if (col >= 0) {
        act = true;
        a = __ldg(ev + e);
        x = xv[i];
        slot = hash_insert<VC>(h, col, &isnew);
      }
    }
    occ_append(h, cnt, isnew, slot);
    __syncwarp();
    unsigned am = __ballot_sync(kFull, act);
    int rank = 0;
    if (act) {
      unsigned peers = __match_any_sync(am, slot);
      rank = __popc(peers & lanemask_lt());
    }
    int maxr = __reduce_max_sync(kFull, rank);
    for (int rho = 0; rho <= maxr; rho++) {
      if (act && rank == rho) hv[slot] = vfma(a, x, hv[slot]);
      __syncwarp();
    }
  }
  if (diag >= 0) {
    bool isnew = false;
    int slot = -1;
    if (lane == 0) slot = hash_insert<VC>(h, diag, &isnew);
    occ_append(h, cnt, isnew, slot);
    __syncwarp();
  }
  return cnt;
}

// sort a short list by row in place (rank by counting; rows distinct)
template <typename V>
__device__ void sort_rows_small(int* r, V* v, int L, int* tr, V* tv, int lane) {
  for (int i = lane; i < L; i += 32) {
    int x = r[i], rank = 0;
    for (int q = 0; q < L; q++) rank += r[q] < x;
    tr[rank] = x;
    tv[rank] = v[i];
  }
  __syncwarp();
  for (int i = lane; i < L; i += 32) {
    r[i] = tr[i];
    v[i] = tv[i];
  }
  __syncwarp();
}

// Move the table's rows to a list: value = acc (diag < 0) or the residual
// 1 - acc on the diagonal / -acc elsewhere (diag >= 0); the transformed
// value is also written back to the table so later lookups see R itself.
// Exact zeros are left out of the list.  CLEAR: the table is emptied on the
// way instead (each lane clears the slots it read; nothing is written back).
template <typename VC, bool CLEAR = false>
__device__ int table_to_list(const HashT& h, int cnt, int diag, int* outr, VC* outv, int lane) {
  VC* hv = (VC*)h.val;
  int outn = 0;
  for (int base = 0; base < cnt; base += 32) {
    int i = base + lane;
    bool nz = false;
    int r = 0;
    VC val = VC(0);
    if (i < cnt) {
      int s = h.occ[i];
      r = h.key[s];
      if (CLEAR) h.key[s] = -1;
      VC acc = hv[s];
      if (diag >= 0) {
        val = (r == diag) ? (VC(1) - acc) : -acc;
        if (!CLEAR) hv[s] = val;
      } else {
        val = acc;
      }
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

// ----------------------------------------------------- term functors

template <typename V> struct TermSq {        // x_i^2 of a list
  const V* v;
  __device__ Term operator()(int i) const { return term_prod(v[i], v[i]); }
};
template <typename V> struct TermSqTable {   // x^2 of the occupied slots of a table
  const V* v;
  const uint16_t* occ;
  __device__ Term operator()(int i) const {
    const V x = v[occ[i]];
    return term_prod(x, x);
  }
};

// Pi-weighted terms of Section 5's inner products: fl(fl(x y) pi_k), the
// product of the two values (exact for FP32 values) times the row weight,
// each rounded in FP64.
template <typename V>
__device__ __forceinline__ Term term_wprod(V x, V y, double w) {
  return term_of(__dmul_rn(__dmul_rn((double)x, (double)y), w));
}
template <typename V> struct TermWSq {       // pi_k x_k^2 of a list
  const int* r;
  const V* v;
  const double* pi;
  __device__ Term operator()(int i) const { return term_wprod(v[i], v[i], pi[r[i]]); }
};
template <typename V> struct TermWSqTable {  // pi_k x_k^2 of the occupied slots of a table
  const int* key;
  const V* v;
  const uint16_t* occ;
  const double* pi;
  __device__ Term operator()(int i) const {
    const int s = occ[i];
    return term_wprod(v[s], v[s], pi[key[s]]);
  }
};

// The same products with the second factor found in a hash table (0 when
// its row is absent), for inner products over rows of two different columns.
template <typename V> struct TermProdFind {        // x_i * b(r_i)
  const int* r;
  const V* x;
  HashT b;
  __device__ Term operator()(int i) const { return term_prod(x[i], hash_find<V>(b, r[i])); }
};
template <typename V> struct TermProdTableFind {   // a[s] * b(key[s]), s = occ[i]
  const int* key;
  const V* a;
  const uint16_t* occ;
  HashT b;
  __device__ Term operator()(int i) const {
    const int s = occ[i];
    return term_prod(a[s], hash_find<V>(b, key[s]));
  }
};
template <typename V> struct TermWProdFind {       // pi_k x_i b(k), k = r_i
  const int* r;
  const V* x;
  HashT b;
  const double* pi;
  __device__ Term operator()(int i) const {
    const int k = r[i];
    return term_wprod(x[i], hash_find<V>(b, k), pi[k]);
  }
};
template <typename V> struct TermWProdTableFind {  // pi_k a[s] b(k), s = occ[i], k = key[s]
  const int* key;
  const V* a;
  const uint16_t* occ;
  HashT b;
  const double* pi;
  __device__ Term operator()(int i) const {
    const int s = occ[i];
    const int k = key[s];
    return term_wprod(a[s], hash_find<V>(b, k), pi[k]);
  }
};

// (Pi R)_j of a list: z_k = pi_k r_k in FP64 rounded to the value type,
// exact zeros removed (Algorithms 5, 7, 8: Z := Pi R).  Returns the length.
template <typename V>
__device__ int list_scale_pi(const int* rr, const V* rv, int L, const double* pi, int* zr, V* zv,
                             int lane) {
  int out = 0;
  for (int base = 0; base < L; base += 32) {
    const int i = base + lane;
    int r = 0;
    V z = V(0);
    if (i < L) {
      r = rr[i];
      z = (V)__dmul_rn(pi[r], (double)rv[i]);
    }
    const bool keep = i < L && z != V(0);
    const unsigned b = __ballot_sync(kFull, keep);
    if (keep) {
      const int pos = out + __popc(b & lanemask_lt());
      zr[pos] = r;
      zv[pos] = z;
    }
    out += __popc(b);
  }
  __syncwarp();
  return out;
}

}  // namespace spai
