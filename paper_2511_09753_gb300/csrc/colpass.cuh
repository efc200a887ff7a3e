// The fused column pass: one launch performs, for every column j, the
// column-local part of one MR / LOMR / CG iteration (pattern-union update,
// hard thresholding, explicit residual, direction, direction product and the
// per-column Frobenius partials), then reduces the partials over all
// columns with a fixed pairwise tree and lets the last-arriving CTA compute
// the step coefficients for the next pass.  Columns only interact through
// those few FP64 sums (Sec. 2: the iterations are global only through the
// Frobenius inner products).
#pragma once
#include "common.cuh"
#include "warp_ops.cuh"

namespace spai {

// Contiguous pairwise tree over v[0..len) (len a power of two <= 1024 or
// any len with zero padding to 32 minimum), computed by warp 0.  Values are
// read from global memory with L1 bypass.
__device__ inline double block_tree_global(const double* v, int len, double* red, int lane, int warp) {
  // len <= 32*32; lane handles c contiguous entries, c = P2/32
  int P2 = 32;
  while (P2 < len) P2 <<= 1;
  int c = P2 / 32;
  double s = 0.0;
  if (warp == 0) {
    for (int t = 0; t < c; t++) {
      int i = lane * c + t;
      red[i] = i < len ? __ldcg(v + i) : 0.0;
    }
    __syncwarp();
    s = warp_pairwise(red, P2, lane);
  }
  return s;
}

// Phase boundaries of the column work.  In the library built with
// SPAI_PHASE_CLOCKS (a profiling build) they count cycles per phase:
// g_phase_clk[kind * 16 + phase] sums, over all warps, the clock64() cycles a
// warp spent in that phase; kPhCols counts the columns and kPhTail the cycles
// thread 0 of each CTA spent in the reduction tail.  In the product library
// some of them are CTA barriers of MR and LOMR passes (ColCtx::mark).
enum : int {
  kPhLoad = 0, kPhUnion, kPhSelect, kPhStore, kPhSpgemm, kPhList, kPhFixsum, kPhTail, kPhCols,
  kPhWarp, kPhCount
};
#ifdef SPAI_PHASE_CLOCKS
__device__ unsigned long long g_phase_clk[8 * 16];
#endif

template <typename VS, typename VC>
struct ColCtx {
  const PassParams& p;
  char* ws;
  int lane;
  int overflow;
  unsigned long long bytes;
  unsigned long long rbytes;  // of bytes: CG's R slab
  unsigned long long spg;
  unsigned long long nnzM;    // nnz of the M columns this warp produced (history)
  const DevScalars* sc;  // the coefficients of this column's matrix
  int seg;               // its segment in batched mode, else -1
#ifdef SPAI_PHASE_CLOCKS
  long long ph_t0;
  long long ph[kPhCount];
  __device__ ColCtx(const PassParams& pp, char* w, int l, const DevScalars* s, int sg)
      : p(pp), ws(w), lane(l), overflow(0), bytes(0), rbytes(0), spg(0), nnzM(0), sc(s), seg(sg),
        ph_t0(0) {
    for (int k = 0; k < kPhCount; k++) ph[k] = 0;
  }
  __device__ __forceinline__ void ph_start() { ph_t0 = clock64(); }
  __device__ __forceinline__ void mark(int k) {
    const long long t = clock64();
    ph[k] += t - ph_t0;
    ph_t0 = t;
  }
#else
  int nsync = 0;  // threads of this warp's barrier group with a column in this round
  int bar = 1;    // the group's named barrier
  __device__ ColCtx(const PassParams& pp, char* w, int l, const DevScalars* s, int sg)
      : p(pp), ws(w), lane(l), overflow(0), bytes(0), rbytes(0), spg(0), nnzM(0), sc(s), seg(sg) {}
  __device__ __forceinline__ void ph_start() {}
  // phase boundary: the round's warps pass the ends of the selections, the
  // products and the sums together, so they run the same code at about the
  // same time and the SM fetches it once for all of them (barriers at the
  // other boundaries too measured slower)
  __device__ __forceinline__ void mark(int k) {
    constexpr int kSyncAt = (1 << kPhSelect) | (1 << kPhSpgemm) | (1 << kPhFixsum);
    if (nsync > 32 && ((kSyncAt >> k) & 1))
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nsync) : "memory");
  }
#endif
  template <typename T> __device__ T* at(int off) const { return (T*)(ws + off); }
};

template <typename VS, typename VC>
__device__ int load_col(ColCtx<VS, VC>& c, const int* grow, const void* gval, long long off, int len,
                        int* sr, VC* sv) {
  const VS* gv = (const VS*)gval;
  for (int e = c.lane; e < len; e += 32) {
    sr[e] = grow[off + e];
    sv[e] = (VC)gv[off + e];
  }
  __syncwarp();
  c.bytes += (unsigned long long)len * (sizeof(int) + sizeof(VS)) + sizeof(int);
  return len;
}

// Load the M column and, when asked, the P and Z columns of the same slab
// offset: every global load of a lane is issued before its shared-memory
// stores, so the three latencies overlap.
template <typename VS, typename VC>
__device__ void load_cols(ColCtx<VS, VC>& c, long long off, int Lm, int* Mr, VC* Mv, int Lp, int* Pr,
                          VC* Pv, int Lz, int* Zr, VC* Zv) {
  const PassParams& p = c.p;
  const VS* mv = (const VS*)p.Mval;
  const VS* pv = (const VS*)p.Pval;
  const VS* zv = (const VS*)p.Zval;
  const int Lx = max(Lm, max(Lp, Lz));
  for (int e = c.lane; e < Lx; e += 32) {
    const bool am = e < Lm, ap = e < Lp, az = e < Lz;
    int rm = 0, rp = 0, rz = 0;
    VS xm = VS(0), xp = VS(0), xz = VS(0);
    if (am) {
      rm = p.Mrow[off + e];
      xm = mv[off + e];
    }
    if (ap) {
      rp = p.Prow[off + e];
      xp = pv[off + e];
    }
    if (az) {
      rz = p.Zrow[off + e];
      xz = zv[off + e];
    }
    if (am) {
      Mr[e] = rm;
      Mv[e] = (VC)xm;
    }
    if (ap) {
      Pr[e] = rp;
      Pv[e] = (VC)xp;
    }
    if (az) {
      Zr[e] = rz;
      Zv[e] = (VC)xz;
    }
  }
  __syncwarp();
}

// CG: the R list of column j kept between pass A and the next pass B
template <typename VS, typename VC>
__device__ void store_r(ColCtx<VS, VC>& c, int j, int LR, const int* Rr, const VC* Rv) {
  const PassParams& p = c.p;
  const long long o = (long long)j * (p.capmax * p.W + 1);
  VC* gv = (VC*)p.Rval;
  for (int e = c.lane; e < LR; e += 32) {
    p.Rrow[o + e] = Rr[e];
    gv[o + e] = Rv[e];
  }
  if (c.lane == 0) p.Rlen[j] = LR;
  const unsigned long long b = (unsigned long long)LR * (sizeof(int) + sizeof(VC)) + sizeof(int);
  c.bytes += b;
  c.rbytes += b;
}

template <typename VS, typename VC>
__device__ int load_r(ColCtx<VS, VC>& c, int j, int* Rr, VC* Rv) {
  const PassParams& p = c.p;
  const long long o = (long long)j * (p.capmax * p.W + 1);
  const VC* gv = (const VC*)p.Rval;
  const int LR = p.Rlen[j];
  for (int e = c.lane; e < LR; e += 32) {
    const int r = p.Rrow[o + e];
    const VC v = gv[o + e];
    Rr[e] = r;
    Rv[e] = v;
  }
  __syncwarp();
  const unsigned long long b = (unsigned long long)LR * (sizeof(int) + sizeof(VC)) + sizeof(int);
  c.bytes += b;
  c.rbytes += b;
  return LR;
}

template <typename VS, typename VC>
__device__ void store_col(ColCtx<VS, VC>& c, int* grow, void* gval, int* glen, int j, long long off,
                          int len, const int* sr, const VC* sv) {
  VS* gv = (VS*)gval;
  for (int e = c.lane; e < len; e += 32) {
    grow[off + e] = sr[e];
    gv[off + e] = (VS)sv[e];
  }
  if (c.lane == 0) glen[j] = len;
  c.bytes += (unsigned long long)len * (sizeof(int) + sizeof(VS)) + sizeof(int);
}

// HOT: the kernel of steady-state passes (steady_pass), whose inputs all have
// the short DIA form, so only that product is compiled in.
template <bool HOT, typename VC>
__device__ __forceinline__ int spgemm(const PassParams& p, const HashT& h, int* xr, VC* xv, int L,
                                      int diag, int* sr, VC* sv, int lane, int seg) {
  if constexpr (HOT) return spgemm_dia32(p, h, xr, xv, L, diag, seg, lane);
  if (p.dia) {
    if (L <= 32 && (seg >= 0 ? p.seg_D[seg] : p.D) <= 8)
      return spgemm_dia32(p, h, xr, xv, L, diag, seg, lane);
    return spgemm_dia(p, h, xr, xv, L, diag, seg, lane);
  }
  sort_rows_small(xr, xv, L, sr, sv, lane);
  return spgemm_ell(p, h, xr, xv, L, diag, lane);
}

// Column work of one pass.  part[0..nq) receives the column partials.
// PI: the Pi-preconditioned forms (Algorithms 5, 7, 8 with Pi = diag(A)^{-1}):
// directions from Z = Pi R, Pi-weighted coefficient inner products.
// HOT: a steady-state pass (steady_pass), whose flags are fixed at compile
// time, so the kernel holds only the code such a pass runs (a smaller kernel
// misses less in the instruction cache).
template <typename VS, typename VC, bool PI, int KIND, bool HOT>
__device__ void column_work(ColCtx<VS, VC>& c, int j, double* part) {
  const PassParams& p = c.p;
  const WarpLayout& L = p.lay;
  const int lane = c.lane;
  const long long off = p.off[j];
  const int cap = p.cap[j];
  const int keep = p.keep_diag ? j : -1;  // the row every drop of this column keeps
  const bool upd = HOT || p.do_update, dir = HOT || p.do_dir;
  const bool slab = !HOT && p.dir_from_slab, store = !HOT && p.dir_store;
  const bool fresh = !HOT && p.fresh, rin = HOT || p.r_in, rout = HOT || p.r_out;
  int* Mr = c.template at<int>(L.Mr);
  VC* Mv = c.template at<VC>(L.Mv);
  int* Pr = c.template at<int>(L.Pr);
  VC* Pv = c.template at<VC>(L.Pv);
  int* Tr = c.template at<int>(L.Tr);
  VC* Tv = c.template at<VC>(L.Tv);
  int* Rr = c.template at<int>(L.Rr);
  VC* Rv = c.template at<VC>(L.Rv);
  uint32_t* hist = c.template at<uint32_t>(L.hist);
  int* tie = c.template at<int>(L.tie);
  HashT ha;
  ha.key = c.template at<int>(L.hk);
  ha.val = c.template at<VC>(L.hv);
  ha.occ = c.template at<uint16_t>(L.ho);
  ha.H = L.H;
  UnionT un;
  un.key = c.template at<int>(L.uk);
  un.va = c.template at<VC>(L.ua);
  un.vb = c.template at<VC>(L.ub);
  un.occ = c.template at<uint16_t>(L.uo);
  un.H = L.HU;
  int* ovf = &c.overflow;

  // the columns this pass reads from the slabs, loaded together
  const bool needP = (KIND == kMR && upd) || KIND == kLOMR ||
                     (KIND == kCGA && upd) || KIND == kCGB;
  const bool needZ = KIND == kLOMR && upd;
  const bool needM = !(KIND == kCGB && rin);  // M only feeds R there
  int Lm = needM ? p.Mlen[j] : 0;
  int Lp = needP ? p.Plen[j] : 0;
  const int Lz0 = needZ ? p.Zlen[j] : 0;
  load_cols(c, off, Lm, Mr, Mv, Lp, Pr, Pv, Lz0, c.template at<int>(L.Zr), c.template at<VC>(L.Zv));
  c.mark(kPhLoad);
  c.bytes += (unsigned long long)(Lm + Lp + Lz0) * (sizeof(int) + sizeof(VS)) +
             ((int)needM + (int)needP + (int)needZ) * sizeof(int);

  if constexpr (KIND == kSCORE) {
    // Appendix A, Eq. 430: dropping m_kj alone changes ||R||_F^2 by
    // m^2 ||A e_k||^2 + 2 m (A R)_kj; (A R)_kj from row k of A and the R table
    int cnt = spgemm<HOT>(p, ha, Mr, Mv, Lm, j, Tr, Tv, lane, c.seg);
    table_to_list(ha, cnt, j, Rr, Rv, lane);  // the table now holds R
    c.spg++;
    const VC* av = (const VC*)p.ell_val;
    for (int e = lane; e < Lm; e += 32) {
      const int k = Mr[e];
      double s;
      if (k == j) {
        s = __longlong_as_double(0x7ff0000000000000ll);  // the diagonal is kept
      } else {
        const double m = (double)Mv[e];
        double ar = 0.0;
        for (int t = 0; t < p.W; t++) {
          const int col = p.ell_col[(long long)k * p.W + t];
          if (col < 0) break;
          ar = __fma_rn((double)av[(long long)k * p.W + t], (double)hash_find<VC>(ha, col), ar);
        }
        s = __fma_rn(__dmul_rn(2.0, m), ar, __dmul_rn(__dmul_rn(m, m), p.anrm[k]));
      }
      p.score[off + e] = s;
    }
    __syncwarp();
    hash_clear(ha, cnt, lane);
    part[0] = 0.0;
    return;
  }

  if constexpr (KIND == kRES) {
    int cnt = spgemm<HOT>(p, ha, Mr, Mv, Lm, j, Tr, Tv, lane, c.seg);
    int LR = table_to_list<VC, true>(ha, cnt, j, Rr, Rv, lane);
    c.spg++;
    fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
    return;
  }

  if constexpr (KIND == kMR) {
    if (upd) {
      CombAxpy<VC> f{c.sc->alpha};
      int Lt = warp_union(un, Mr, Mv, Lm, Pr, Pv, Lp, Tr, Tv, f, lane);
      c.mark(kPhUnion);
      Lm = warp_select(Tr, Tv, Lt, cap, Mr, Mv, hist, tie, p.drop, ovf, lane, keep);
      c.mark(kPhSelect);
      store_col(c, p.Mrow, p.Mval, p.Mlen, j, off, Lm, Mr, Mv);
      c.mark(kPhStore);
    }
    c.nnzM += Lm;  // M_iter
    int cnt = spgemm<HOT>(p, ha, Mr, Mv, Lm, j, Tr, Tv, lane, c.seg);
    c.mark(kPhSpgemm);
    int LR = table_to_list<VC, true>(ha, cnt, j, Rr, Rv, lane);
    c.mark(kPhList);
    c.spg++;
    if (!dir && !store) {
      fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
      return;
    }
    if (slab) {  // a direction chosen outside the pass (global dropping)
      Lp = load_col(c, p.Prow, p.Pval, off, p.Plen[j], Pr, Pv);
    } else {
      if (PI) {  // P = D(Pi R) (Algorithm 5)
        int* Zr = c.template at<int>(L.zr);
        VC* Zv = c.template at<VC>(L.zv);
        int Lz = list_scale_pi(Rr, Rv, LR, p.pi, Zr, Zv, lane);
        Lp = warp_select(Zr, Zv, Lz, cap, Pr, Pv, hist, tie, p.drop, ovf, lane, keep);
      } else {
        Lp = warp_select(Rr, Rv, LR, cap, Pr, Pv, hist, tie, p.drop, ovf, lane, keep);
      }
      c.mark(kPhSelect);
      store_col(c, p.Prow, p.Pval, p.Plen, j, off, Lp, Pr, Pv);
      c.mark(kPhStore);
    }
    if (!dir) {  // dir_store: the direction candidate is all this pass forms
      fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
      return;
    }
    int cq = spgemm<HOT>(p, ha, Pr, Pv, Lp, -1, Tr, Tv, lane, c.seg);  // table holds Q = A P
    c.mark(kPhSpgemm);
    c.spg++;
    if (PI)  // (R,R), (R,Pi Q), (Q,Pi Q)
      fixsum<3>(part, lane, TermSq<VC>{Rv}, LR, TermWProdFind<VC>{Rr, Rv, ha, p.pi}, LR,
                TermWSqTable<VC>{ha.key, (const VC*)ha.val, ha.occ, p.pi}, cq);
    else     // (R,R), (R,Q), (Q,Q)
      fixsum<3>(part, lane, TermSq<VC>{Rv}, LR, TermProdFind<VC>{Rr, Rv, ha}, LR,
                TermSqTable<VC>{(const VC*)ha.val, ha.occ}, cq);
    c.mark(kPhFixsum);
    hash_clear(ha, cq, lane);
    c.mark(kPhList);
    return;
  }

  if constexpr (KIND == kLOMR) {
    int* Zr = c.template at<int>(L.Zr);
    VC* Zv = c.template at<VC>(L.Zv);
    int* Sr = c.template at<int>(L.Sr);
    VC* Sv = c.template at<VC>(L.Sv);
    HashT hb;
    hb.key = c.template at<int>(L.gk);
    hb.val = c.template at<VC>(L.gv);
    hb.occ = c.template at<uint16_t>(L.go);
    hb.H = L.H;
    if (upd) {
      // S = delta Z + gamma P and T = M + S from one table (P_i = D(S),
      // M_{i+1} = D(T))
      CombLin<VC> fl{c.sc->delta, c.sc->gamma};
      CombAdd<VC> fa;
      int Ls, Lt;
      warp_union3(un, Zr, Zv, Lz0, Pr, Pv, Lp, Mr, Mv, Lm, Sr, Sv, &Ls, Tr, Tv, &Lt, fl, fa, lane);
      c.mark(kPhUnion);
      Lp = warp_select(Sr, Sv, Ls, cap, Pr, Pv, hist, tie, p.drop, ovf, lane, keep);
      c.mark(kPhSelect);
      store_col(c, p.Prow, p.Pval, p.Plen, j, off, Lp, Pr, Pv);
      c.mark(kPhStore);
      Lm = warp_select(Tr, Tv, Lt, cap, Mr, Mv, hist, tie, p.drop, ovf, lane, keep);
      c.mark(kPhSelect);
      store_col(c, p.Mrow, p.Mval, p.Mlen, j, off, Lm, Mr, Mv);
      c.mark(kPhStore);
    }
    c.nnzM += Lm;  // M_iter
    int cr = spgemm<HOT>(p, ha, Mr, Mv, Lm, j, Tr, Tv, lane, c.seg);
    c.mark(kPhSpgemm);
    int LR = table_to_list<VC, true>(ha, cr, j, Rr, Rv, lane);
    c.mark(kPhList);
    c.spg++;
    if (!dir && !store) {
      fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
      return;
    }
    int Lz;
    if (slab) {  // a Z chosen outside the pass (global dropping)
      Lz = load_col(c, p.Zrow, p.Zval, off, p.Zlen[j], Zr, Zv);
    } else {
      if (PI) {  // Z = D(Pi R) (Algorithm 8)
        int* Xr = c.template at<int>(L.zr);
        VC* Xv = c.template at<VC>(L.zv);
        int Lx = list_scale_pi(Rr, Rv, LR, p.pi, Xr, Xv, lane);
        Lz = warp_select(Xr, Xv, Lx, cap, Zr, Zv, hist, tie, p.drop, ovf, lane, keep);
      } else {
        Lz = warp_select(Rr, Rv, LR, cap, Zr, Zv, hist, tie, p.drop, ovf, lane, keep);
      }
      c.mark(kPhSelect);
      store_col(c, p.Zrow, p.Zval, p.Zlen, j, off, Lz, Zr, Zv);
      c.mark(kPhStore);
    }
    if (!dir) {  // dir_store: the Z candidate is all this pass forms
      fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
      return;
    }
    int cu = spgemm<HOT>(p, ha, Zr, Zv, Lz, -1, Tr, Tv, lane, c.seg);   // table A: U = A Z
    c.mark(kPhSpgemm);
    double t3[3];
    if (PI)  // (R,R), (U,Pi U), (U,Pi R)
      fixsum<3>(t3, lane, TermSq<VC>{Rv}, LR,
                TermWSqTable<VC>{ha.key, (const VC*)ha.val, ha.occ, p.pi}, cu,
                TermWProdFind<VC>{Rr, Rv, ha, p.pi}, LR);
    else     // (R,R), (U,U), (U,R)
      fixsum<3>(t3, lane, TermSq<VC>{Rv}, LR, TermSqTable<VC>{(const VC*)ha.val, ha.occ}, cu,
                TermProdFind<VC>{Rr, Rv, ha}, LR);
    part[0] = t3[0];
    part[1] = t3[1];
    part[4] = t3[2];
    c.mark(kPhFixsum);
    hash_clear_all(hb, lane);  // its bytes also held the union table and the select scratch
    c.mark(kPhList);
    int cv = spgemm<HOT>(p, hb, Pr, Pv, Lp, -1, Tr, Tv, lane, c.seg);   // table B: V = A P
    c.mark(kPhSpgemm);
    c.spg += 2;
    if (PI)  // (V,Pi V), (U,Pi V), (V,Pi R)
      fixsum<3>(t3, lane, TermWSqTable<VC>{hb.key, (const VC*)hb.val, hb.occ, p.pi}, cv,
                TermWProdTableFind<VC>{ha.key, (const VC*)ha.val, ha.occ, hb, p.pi}, cu,
                TermWProdFind<VC>{Rr, Rv, hb, p.pi}, LR);
    else     // (V,V), (U,V), (V,R)
      fixsum<3>(t3, lane, TermSqTable<VC>{(const VC*)hb.val, hb.occ}, cv,
                TermProdTableFind<VC>{ha.key, (const VC*)ha.val, ha.occ, hb}, cu,
                TermProdFind<VC>{Rr, Rv, hb}, LR);
    part[2] = t3[0];
    part[3] = t3[1];
    part[5] = t3[2];
    c.mark(kPhFixsum);
    hash_clear(ha, cu, lane);
    c.mark(kPhList);
    return;
  }

  if constexpr (KIND == kCGA) {
    if (upd) {  // without it: R and beta of an M changed outside (global dropping)
      CombAxpy<VC> f{c.sc->alpha};
      int Lt = warp_union(un, Mr, Mv, Lm, Pr, Pv, Lp, Tr, Tv, f, lane);
      c.mark(kPhUnion);
      Lm = warp_select(Tr, Tv, Lt, cap, Mr, Mv, hist, tie, p.drop, ovf, lane, keep);
      c.mark(kPhSelect);
      store_col(c, p.Mrow, p.Mval, p.Mlen, j, off, Lm, Mr, Mv);
      c.mark(kPhStore);
      c.nnzM += Lm;  // M_{iter+1}
    }
    if (!dir) {  // the update only: M is dropped outside before R is formed
      part[0] = 0.0;
      return;
    }
    int cr = spgemm<HOT>(p, ha, Mr, Mv, Lm, j, Tr, Tv, lane, c.seg);
    c.mark(kPhSpgemm);
    int LR = table_to_list<VC, true>(ha, cr, j, Rr, Rv, lane);
    c.mark(kPhList);
    c.spg++;
    if (rout) store_r(c, j, LR, Rr, Rv);
    c.mark(kPhStore);
    if (PI)  // (R,R), (R,Pi R)
      fixsum<2>(part, lane, TermSq<VC>{Rv}, LR, TermWSq<VC>{Rr, Rv, p.pi}, LR);
    else
      fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
    c.mark(kPhFixsum);
    return;
  }

  if constexpr (KIND == kCGB) {
    if (fresh) c.nnzM += Lm;  // M_0 of the call (loaded: no R slab on the first pass)
    int LR;
    if (rin) {  // R as the previous pass A computed it
      LR = load_r(c, j, Rr, Rv);
      c.mark(kPhLoad);
    } else {
      int cr = spgemm<HOT>(p, ha, Mr, Mv, Lm, j, Tr, Tv, lane, c.seg);
      LR = table_to_list<VC, true>(ha, cr, j, Rr, Rv, lane);
      c.spg++;
    }
    if (!slab) {  // else P, loaded above, was chosen outside (global dropping)
      CombAxpy<VC> f{c.sc->beta};
      int Lt;
      if (PI) {  // P = D(Pi R + beta P) (Algorithm 7)
        int* Zr = c.template at<int>(L.zr);
        VC* Zv = c.template at<VC>(L.zv);
        int Lz = list_scale_pi(Rr, Rv, LR, p.pi, Zr, Zv, lane);
        Lt = warp_union(un, Zr, Zv, Lz, Pr, Pv, Lp, Tr, Tv, f, lane);
      } else {
        Lt = warp_union(un, Rr, Rv, LR, Pr, Pv, Lp, Tr, Tv, f, lane);
      }
      c.mark(kPhUnion);
      Lp = warp_select(Tr, Tv, Lt, cap, Pr, Pv, hist, tie, p.drop, ovf, lane, keep);
      c.mark(kPhSelect);
      store_col(c, p.Prow, p.Pval, p.Plen, j, off, Lp, Pr, Pv);
      c.mark(kPhStore);
    }
    if (!dir) {  // the direction candidate only (global dropping follows)
      fixsum<1>(part, lane, TermSq<VC>{Rv}, LR);
      return;
    }
    if (L.hk == L.uk) hash_clear_all(ha, lane);  // the union and selection used its bytes
    int cq = spgemm<HOT>(p, ha, Pr, Pv, Lp, -1, Tr, Tv, lane, c.seg);  // table holds Q = A P
    c.mark(kPhSpgemm);
    c.spg++;
    // (R,R) and (R,Pi R) are needed only by the first pass B of a call: the
    // pass A before each later one has stored them (alpha's numerator)
    if (fresh) {
      if (PI)  // (R,R), (P,Q), (R,Pi R)
        fixsum<3>(part, lane, TermSq<VC>{Rv}, LR, TermProdFind<VC>{Pr, Pv, ha}, Lp,
                  TermWSq<VC>{Rr, Rv, p.pi}, LR);
      else     // (R,R), (P,Q)
        fixsum<2>(part, lane, TermSq<VC>{Rv}, LR, TermProdFind<VC>{Pr, Pv, ha}, Lp);
    } else {  // (P,Q)
      part[0] = 0.0;
      part[2] = 0.0;
      fixsum<1>(part + 1, lane, TermProdFind<VC>{Pr, Pv, ha}, Lp);
    }
    c.mark(kPhFixsum);
    hash_clear(ha, cq, lane);
    c.mark(kPhList);
  }
}

__device__ __forceinline__ bool isfin(double x) { return !isnan(x) && !isinf(x); }

// Step coefficients from the global sums t[0..nq) of one matrix; thread 0 of
// the last CTA of that matrix.  hist_res / hist_coef point at its histories.
__device__ inline void coefficients(const PassParams& p, DevScalars* sc, double* hist_res,
                                    double* hist_coef, const double* t) {
  const int it = p.iter;
  if (p.kind == kRES || p.kind == kSCORE) {
    sc->result = t[0];
    return;
  }
  if (p.kind == kMR || p.kind == kLOMR) {
    double rr = t[0];
    if (p.do_update) sc->done += 1;
    if (hist_res) hist_res[it] = __dsqrt_rn(rr);
    if (!p.do_dir) return;
    if (rr == 0.0) {
      sc->stop = 1;
      sc->flags |= kFlagConverged;
      return;
    }
    if (p.kind == kMR) {
      double rq = t[1], qq = t[2];
      if (qq == 0.0) {
        sc->stop = 1;
        sc->flags |= kFlagConverged;
        return;
      }
      double alpha = __ddiv_rn(rq, qq);
      if (!isfin(alpha)) {
        sc->stop = 1;
        sc->flags |= kFlagNonfinite;
        return;
      }
      sc->alpha = alpha;
      if (hist_coef) {
        hist_coef[2 * it] = alpha;
        hist_coef[2 * it + 1] = 0.0;
      }
    } else {
      double uu = t[1], vv = t[2], uv = t[3], ur = t[4], vr = t[5];
      if (uu == 0.0) {
        sc->stop = 1;
        sc->flags |= kFlagConverged;
        return;
      }
      double t1 = __dmul_rn(uu, vv), t2 = __dmul_rn(uv, uv);
      double cc = __dsub_rn(t1, t2);
      const double eps = 2.220446049250313e-16;
      double delta, gamma;
      if (vv == 0.0 || cc <= __dmul_rn(__dmul_rn(64.0, eps), t1)) {
        delta = __ddiv_rn(ur, uu);
        gamma = 0.0;
        if (vv != 0.0) sc->flags |= kFlagFallback;
      } else {
        double d1 = __dmul_rn(vv, ur), d2 = __dmul_rn(uv, vr);
        double g1 = __dmul_rn(uu, vr), g2 = __dmul_rn(uv, ur);
        delta = __ddiv_rn(__dsub_rn(d1, d2), cc);
        gamma = __ddiv_rn(__dsub_rn(g1, g2), cc);
      }
      if (!isfin(delta) || !isfin(gamma)) {
        sc->stop = 1;
        sc->flags |= kFlagNonfinite;
        return;
      }
      sc->delta = delta;
      sc->gamma = gamma;
      if (hist_coef) {
        hist_coef[2 * it] = delta;
        hist_coef[2 * it + 1] = gamma;
      }
    }
    return;
  }
  if (p.kind == kCGB) {
    if (!p.do_dir) return;  // a direction candidate: no step
    // alpha = (R, R) / (P, AP), or (R, Pi R) / (P, AP) with Pi; after the
    // first pass B of a call the numerator is the one the pass A before it
    // stored (the same sum over the same R), and this pass skips it
    double rr = p.fresh ? (p.pi ? t[2] : t[0]) : sc->rr, pq = t[1];
    if (p.fresh && hist_res) hist_res[0] = __dsqrt_rn(t[0]);
    if (rr == 0.0 || pq == 0.0) {
      sc->stop = 1;
      sc->flags |= kFlagConverged;
      return;
    }
    double alpha = __ddiv_rn(rr, pq);
    if (!isfin(alpha)) {
      sc->stop = 1;
      sc->flags |= kFlagNonfinite;
      return;
    }
    sc->alpha = alpha;
    sc->rr = rr;
    return;
  }
  // kCGA: beta = (R+, R+) / (R, R), or the Pi-weighted ratio with Pi
  if (!p.do_dir) return;  // the update only: no R yet
  {
    double rr1 = p.pi ? t[1] : t[0];
    double beta = __ddiv_rn(rr1, sc->rr);
    if (hist_res) hist_res[it + 1] = __dsqrt_rn(t[0]);
    if (hist_coef) {
      hist_coef[2 * it] = sc->alpha;
      hist_coef[2 * it + 1] = beta;
    }
    sc->done += 1;
    sc->rr = rr1;
    sc->beta = beta;
    if (rr1 == 0.0) {
      sc->stop = 1;
      sc->flags |= kFlagConverged;
    }
  }
}

// warps per phase-barrier group of the MR and LOMR passes
constexpr int kBarWarps = 8;

// One instantiation per pass kind keeps each kernel's code small: with all
// kinds behind a runtime switch the instruction cache missed often.
template <typename VS, typename VC, bool PI, int KIND, bool HOT = false>
__global__ void __launch_bounds__(sizeof(VC) == 4 ? 512 : 256, sizeof(VC) == 4 ? 2 : 3) colpass_kernel(const PassParams p) {
  extern __shared__ __align__(16) char smem[];
  const int seg = p.nseg ? p.seg_of_col[(long long)blockIdx.x * p.B] : -1;
  DevScalars* sc = seg >= 0 ? p.segsc + seg : p.sc;
  if (sc->stop) return;  // set by an earlier pass for this matrix
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nq = p.do_dir ? pass_nq(KIND, PI) : 1;
  double* part = (double*)(smem + p.part_off);  // [nq][B]
  double* red = (double*)(smem + p.red_off);    // reduction scratch (>= 1024 doubles)
  ColCtx<VS, VC> c(p, smem + warp * p.lay.bytes, lane, sc, seg);
  {
    HashT h0;
    h0.key = c.template at<int>(p.lay.hk);
    h0.H = p.lay.H;
    hash_clear_all(h0, lane);
    if (KIND == kLOMR) {
      h0.key = c.template at<int>(p.lay.gk);
      hash_clear_all(h0, lane);
    }
    if (KIND != kRES && KIND != kSCORE) {
      h0.key = c.template at<int>(p.lay.uk);
      h0.H = p.lay.HU;
      hash_clear_all(h0, lane);
    }
  }
  const int B = p.B;
  const long long j0 = (long long)blockIdx.x * B;
#ifdef SPAI_PHASE_CLOCKS
  const long long w_t0 = clock64();
#endif
  for (int base = 0; base < B; base += p.NW) {
    const int cc = base + warp;
    long long j = j0 + cc;
    // the round's warps with a column are the lowest nv (every warp of the
    // CTA computes the same nv)
    const long long nv = min((long long)p.NW, min((long long)(B - base), p.n - (j0 + base)));
#ifndef SPAI_PHASE_CLOCKS
    // MR and LOMR keep the round's warps together phase by phase: their
    // kernels are larger than the SM's instruction cache, and warps spread
    // over the code miss in it (measured: MR 67 -> 78 %, LOMR 54 -> 62 %
    // hits); CG's smaller passes lose more to the waits than they gain
    // (groups of kBarWarps warps, each on its own named barrier: fewer warps
    // wait for the slowest of a group)
    if (KIND == kMR || KIND == kLOMR) {
      const int g0 = warp / kBarWarps * kBarWarps;
      c.bar = 1 + warp / kBarWarps;
      c.nsync = 32 * (int)max(0LL, min((long long)kBarWarps, nv - g0));
    }
#endif
    double pr[6] = {0, 0, 0, 0, 0, 0};
    c.ph_start();
    if (warp < nv) {
      column_work<VS, VC, PI, KIND, HOT>(c, (int)j, pr);
#ifdef SPAI_PHASE_CLOCKS
      c.ph[kPhCols]++;
#endif
    }
    if (lane == 0 && cc < B)
      for (int q = 0; q < nq; q++) part[q * B + cc] = pr[q];
  }
#ifdef SPAI_PHASE_CLOCKS
  c.ph[kPhWarp] = clock64() - w_t0;
  if (lane == 0)
    for (int k = 0; k < kPhCount; k++)
      if (k != kPhTail) atomicAdd(&g_phase_clk[KIND * 16 + k], (unsigned long long)c.ph[k]);
  const long long t_tail = clock64();  // thread 0 adds the cycles from here to its return
#define SPAI_TAIL_DONE()                                                                 \
  do {                                                                                   \
    if (threadIdx.x == 0)                                                                \
      atomicAdd(&g_phase_clk[KIND * 16 + kPhTail], (unsigned long long)(clock64() - t_tail)); \
  } while (0)
#else
#define SPAI_TAIL_DONE() ((void)0)
#endif
  // per-CTA counters
  __shared__ unsigned long long s_bytes, s_spg, s_rbytes, s_nnz;
  __shared__ int s_ovf, s_last1, s_last2;
  if (threadIdx.x == 0) {
    s_bytes = 0;
    s_spg = 0;
    s_rbytes = 0;
    s_nnz = 0;
    s_ovf = 0;
  }
  __syncthreads();
  if (lane == 0) {
    atomicAdd(&s_bytes, c.bytes);
    atomicAdd(&s_spg, c.spg);
    if (KIND == kCGA || KIND == kCGB) atomicAdd(&s_rbytes, c.rbytes);
    if (KIND <= kCGB) atomicAdd(&s_nnz, c.nnzM);
    if (c.overflow) atomicOr(&s_ovf, 1);
  }
  // CTA tree over the B column partials of each quantity
  for (int q = 0; q < nq; q++) {
    const double* v = part + q * B;
    double s = 0.0;
    if (B <= 32) {
      if (warp == 0) s = warp_tree32(lane < B ? v[lane] : 0.0);
    } else {
      int nw = B / 32;  // <= 32
      if (warp < nw) {
        double w = warp_tree32(v[warp * 32 + lane]);
        if (lane == 0) red[warp] = w;
      }
      __syncthreads();
      if (warp == 0) s = warp_tree32(lane < nw ? red[lane] : 0.0);
      __syncthreads();
    }
    if (threadIdx.x == 0) p.bsum[(long long)q * p.nb + blockIdx.x] = s;
  }
  __syncthreads();
  // nnz(M_i) history: MR, LOMR passes hold M_iter, CG pass A M_{iter+1},
  // the first CG pass B of a call M_0
  if (KIND <= kCGB && threadIdx.x == 0 && p.hist_nnz && (KIND != kCGB || p.fresh) &&
      (KIND != kCGA || p.do_update)) {
    const int idx = KIND == kCGA ? p.iter + 1 : KIND == kCGB ? 0 : p.iter;
    atomicAdd(p.hist_nnz + (seg >= 0 ? (long long)seg * p.hist_stride : 0LL) + idx, s_nnz);
  }
  __shared__ double tot[6];
  if (seg >= 0) {
    // batched: the last CTA of this matrix reduces its CTAs' sums (aligned,
    // so this is the matrix's own pairwise tree) and sets its coefficients
    if (threadIdx.x == 0) {
      if (s_ovf) atomicOr(&sc->flags, kFlagCapacity);
      atomicAdd(&p.sc->bytes, s_bytes);
      atomicAdd(&p.sc->spgemm_cols, s_spg);
      if (KIND == kCGA || KIND == kCGB) atomicAdd(&p.sc->r_bytes, s_rbytes);
      __threadfence();
      unsigned old = atomicAdd(&p.seg_cnt[seg], 1u);
      s_last1 = (old == (unsigned)(p.seg_npad[seg] / p.B - 1));
    }
    __syncthreads();
    if (!s_last1) {
      SPAI_TAIL_DONE();
      return;
    }
    __threadfence();
    for (int q = 0; q < nq; q++) {
      double s = block_tree_global(p.bsum + (long long)q * p.nb + p.seg_col0[seg] / p.B,
                                   p.seg_npad[seg] / p.B, red, lane, warp);
      if (threadIdx.x == 0) tot[q] = s;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      p.seg_cnt[seg] = 0;
      coefficients(p, sc, p.hist_res ? p.hist_res + (long long)seg * p.hist_stride : nullptr,
                   p.hist_coef ? p.hist_coef + (long long)seg * 2 * (p.hist_stride - 1) : nullptr,
                   tot);
      __threadfence();
    }
    SPAI_TAIL_DONE();
    return;
  }
  // last-arriver tree: groups of kGroup blocks, then all groups
  const int g = blockIdx.x / kGroup;
  if (threadIdx.x == 0) {
    if (s_ovf) atomicOr(&p.sc->flags, kFlagCapacity);
    atomicAdd(&p.sc->bytes, s_bytes);
    atomicAdd(&p.sc->spgemm_cols, s_spg);
    if (KIND == kCGA || KIND == kCGB) atomicAdd(&p.sc->r_bytes, s_rbytes);
    __threadfence();
    int gsize = min(kGroup, p.nb - g * kGroup);
    unsigned old = atomicAdd(&p.cnt1[g], 1u);
    s_last1 = (old == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_last1) {
    SPAI_TAIL_DONE();
    return;
  }
  __threadfence();
  {
    int gsize = min(kGroup, p.nb - g * kGroup);
    for (int q = 0; q < nq; q++) {
      // contiguous tree over the group's 64 blocks (zero padded)
      double s = 0.0;
      if (warp == 0) {
        const double* v = p.bsum + (long long)q * p.nb + (long long)g * kGroup;
        double a = (2 * lane < gsize) ? __ldcg(v + 2 * lane) : 0.0;
        double b = (2 * lane + 1 < gsize) ? __ldcg(v + 2 * lane + 1) : 0.0;
        s = warp_tree32(__dadd_rn(a, b));
      }
      if (threadIdx.x == 0) p.gsum[(long long)q * p.ngroups + g] = s;
    }
  }
  if (threadIdx.x == 0) {
    p.cnt1[g] = 0;
    __threadfence();
    unsigned old = atomicAdd(p.cnt2, 1u);
    s_last2 = (old == (unsigned)(p.ngroups - 1));
  }
  __syncthreads();
  if (!s_last2) {
    SPAI_TAIL_DONE();
    return;
  }
  __threadfence();
  for (int q = 0; q < nq; q++) {
    double s = block_tree_global(p.gsum + (long long)q * p.ngroups, p.ngroups, red, lane, warp);
    if (threadIdx.x == 0) tot[q] = s;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *p.cnt2 = 0;
    coefficients(p, p.sc, p.hist_res, p.hist_coef, tot);
    __threadfence();
  }
  SPAI_TAIL_DONE();
}
#undef SPAI_TAIL_DONE

}  // namespace spai
