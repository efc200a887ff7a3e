// Per-warp shared-memory layout and launch shape of the column pass (host
// code; included by api.cu).  Results do not depend on either: the layout
// only places buffers, and the reduction tree is fixed by the column index.
#pragma once
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace spai {

struct PassCfg {
  WarpLayout lay;
  int NW, B, grid, nb, ngroups;
  size_t smem;
  int part_off, red_off;
  bool ok;
};

inline int align16(int x) { return (x + 15) & ~15; }

inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Per-warp scratch layout of a pass kind.
inline WarpLayout make_layout(int kind, int vc, int CAP, int W, bool dia, bool pi = false) {
  WarpLayout L;
  memset(&L, 0, sizeof(L));
  const int PMAX = CAP * W;
  const int LMAX = PMAX + 1;
  int TMAX = 2 * CAP;  // union output, also the general path's input-sort scratch
  if (kind == kLOMR) TMAX = 3 * CAP;
  if (kind == kCGB) TMAX = LMAX + CAP;
  const int H = std::max(32, next_pow2((4 * LMAX + 2) / 3 + 1));
  const int HU = std::max(32, next_pow2((4 * TMAX + 2) / 3 + 1));
  const int LIST = std::max(LMAX, TMAX);
  int o = 0;
  auto take = [&](int bytes) {
    int at = o;
    o = align16(o + bytes);
    return at;
  };
  const bool hasP = kind != kRES;
  const bool lomr = kind == kLOMR;
  L.H = H;
  L.HU = HU;
  // The R list comes first.  The update phase of MR, LOMR and CG pass A (the
  // union, LOMR's S list, and -- with A in diagonal slots -- the union's
  // output T) is over before R is formed, so those buffers share R's bytes;
  // T stays apart on the ELL path, which also uses it as the input-sort
  // scratch of products taken while R is live.
  L.Rr = take(4 * LMAX);
  L.Rv = take(vc * LMAX);
  const int rbase = L.Rr, rbytes = o - L.Rr;
  const bool upd = kind == kMR || kind == kLOMR || kind == kCGA;
  int ru = 0;  // bytes of R's region handed out so far
  auto in_r = [&](int bytes) {
    if (!upd || ru + align16(bytes) > rbytes) return -1;
    int at = rbase + ru;
    ru += align16(bytes);
    return at;
  };
  const bool cgb = kind == kCGB;
  if (cgb) {
    // CG pass B: table A, the union table, the tie rows and the histogram
    // share one region.  A holds R = I - A M (when R is not read from the
    // slab) until R is listed, then the union, then the selection use the
    // bytes, and the pass clears A's keys before Q = A P.
    const int a_bytes = align16(4 * H) + align16(vc * H) + align16(2 * H);
    const int u_bytes = align16(4 * HU) + 2 * align16(vc * HU) + align16(2 * HU);
    const int x = take(std::max(std::max(a_bytes, u_bytes), align16(4 * LIST) + 4 * 128));
    L.hk = x;
    L.hv = L.hk + align16(4 * H);
    L.ho = L.hv + align16(vc * H);
    L.uk = x;
    L.ua = L.uk + align16(4 * HU);
    L.ub = L.ua + align16(vc * HU);
    L.uo = L.ub + align16(vc * HU);
    L.tie = x;
    L.hist = x + align16(4 * LIST);
  } else {
    L.hk = take(4 * H);
    L.hv = take(vc * H);
    L.ho = take(2 * H);
  }
  L.gk = take(lomr ? 4 * H : 0);
  L.gv = take(lomr ? vc * H : 0);
  L.go = take(lomr ? 2 * H : 0);
  // the union table: in R's region when it fits, else with the tie scratch
  const int u_bytes = align16(4 * HU) + 2 * align16(vc * HU) + align16(2 * HU);
  const int uat = cgb ? -1 : in_r(u_bytes);
  bool u_placed = cgb;
  if (uat >= 0) {
    L.uk = uat;
    L.ua = L.uk + align16(4 * HU);
    L.ub = L.ua + align16(vc * HU);
    L.uo = L.ub + align16(vc * HU);
    u_placed = true;
  }
  // LOMR: the select scratch (tie rows, histogram), and the union table when
  // R's region had no room, live in table B's bytes, which they use only
  // while table B is empty (the pass clears it before its first product);
  // the tie rows share the union table's bytes (a drop runs after its union)
  bool in_b = false;
  if (lomr) {
    const int u = u_placed ? 0 : u_bytes;
    const int hist_at = align16(std::max(u, 4 * LIST));
    if (hist_at + 4 * 128 <= o - L.gk) {  // all of it fits in table B
      if (!u_placed) {
        L.uk = L.gk;
        L.ua = L.uk + align16(4 * HU);
        L.ub = L.ua + align16(vc * HU);
        L.uo = L.ub + align16(vc * HU);
        u_placed = true;
      }
      L.tie = L.gk;
      L.hist = L.gk + hist_at;
      in_b = true;
    }
  }
  // the union table (if not placed yet) and the tie scratch share one region
  if (!in_b && !cgb) {
    int base = o;
    int u = 0;
    if (!u_placed) {
      L.uk = base;
      L.ua = L.uk + align16(4 * HU);
      L.ub = L.ua + align16(vc * HU);
      L.uo = L.ub + align16(vc * HU);
      u = u_bytes;
    }
    int region = std::max(u, 4 * LIST);
    L.tie = base;
    o = align16(base + region);
  }
  L.Mr = take(4 * CAP);
  L.Mv = take(vc * CAP);
  L.Pr = take(hasP ? 4 * CAP : 0);
  L.Pv = take(hasP ? vc * CAP : 0);
  L.Zr = take(lomr ? 4 * CAP : 0);
  L.Zv = take(lomr ? vc * CAP : 0);
  if (lomr) {
    const int sr = in_r(4 * 2 * CAP), sv = sr >= 0 ? in_r(vc * 2 * CAP) : -1;
    L.Sr = sr >= 0 && sv >= 0 ? sr : take(4 * 2 * CAP);
    L.Sv = sr >= 0 && sv >= 0 ? sv : take(vc * 2 * CAP);
  }
  {
    const int tr = dia ? in_r(4 * TMAX) : -1, tv = tr >= 0 ? in_r(vc * TMAX) : -1;
    L.Tr = tr >= 0 && tv >= 0 ? tr : take(4 * TMAX);
    L.Tv = tr >= 0 && tv >= 0 ? tv : take(vc * TMAX);
  }
  if (!in_b && !cgb) L.hist = take(4 * 128);  // 256 packed 16-bit bins
  L.zr = take(pi ? 4 * LMAX : 0);
  L.zv = take(pi ? vc * LMAX : 0);
  L.bytes = o;
  return L;
}

// Launch shape of the column pass.  Results do not depend on it (the
// reduction tree is fixed by the column index), so it is a pure tuning knob:
// occ = CTAs per SM the shared memory should allow, cpw = columns per warp.
// SPAI_COLPASS_OCC / SPAI_COLPASS_CPW override the defaults.
inline int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  int x = atoi(v);
  return x > 0 ? x : dflt;
}

inline PassCfg make_cfg(int kind, int vc, int n, int CAP, int W, bool dia, int smem_max, int Bmin = 1,
                 int Bmax = 1024, bool pi = false, int occ_req = 0, int cpw_req = 0) {
  PassCfg c;
  memset(&c, 0, sizeof(c));
  c.lay = make_layout(kind, vc, CAP, W, dia, pi);
  const int nq = 6;
  const int extra_fixed = 8 * 1024;  // reduction scratch (1024 doubles)
  // defaults measured on GB300 (64^3 operator, cap 3, 50 iterations from
  // M_0): 8-warp CTAs for MR and CG (smaller CTAs that pack more warps leave
  // too little L1 for the gathers of A), 16-warp CTAs for LOMR (FP32 values:
  // its warps pass phase barriers together, and fewer, larger groups per SM
  // share more of the instruction cache), LOMR with one column per warp, MR
  // and the CG passes with eight
  const int occ = occ_req > 0 ? occ_req
                             : env_int("SPAI_COLPASS_OCC", kind == kLOMR ? (vc == 4 ? 2 : 3) : 4);
  const int cpw = cpw_req > 0 ? cpw_req : env_int("SPAI_COLPASS_CPW", kind == kLOMR ? 1 : 8);
  c.ok = false;
  // up to 16 warps with FP32 values (the kernels' launch bound), else 8
  for (int NW = vc == 4 ? 16 : 8; NW >= 1; NW >>= 1) {
    // B: columns per CTA, a power of two: cpw per warp, fewer when n is
    // small, more when needed to keep at most 65536 CTAs (two-level tree).
    int B = NW;
    long long target = (long long)n / (152LL * 8);
    while ((long long)B * 2 <= target && B * 2 <= cpw * NW) B *= 2;
    while (((long long)n + B - 1) / B > 65536LL && B < 1024) B *= 2;
    while (B < Bmin) B *= 2;
    if (B > Bmax) return c;  // batched: a CTA must not straddle two matrices
    // the CTA reduction buffer (1024 doubles) reuses the warps' scratch,
    // which is free once every column of the block is done
    size_t smem = std::max((size_t)NW * c.lay.bytes, (size_t)extra_fixed);
    int part_off = (int)smem;
    smem += (size_t)8 * nq * B;
    int red_off = 0;
    bool fits = smem <= (size_t)smem_max;
    bool good = smem <= (size_t)(smem_max / occ) || NW == 1;
    if (fits && (good || NW == 1)) {
      c.NW = NW;
      c.B = B;
      c.grid = (int)(((long long)n + B - 1) / B);
      c.nb = c.grid;
      c.ngroups = (c.nb + kGroup - 1) / kGroup;
      c.smem = smem;
      c.part_off = part_off;
      c.red_off = red_off;
      c.ok = c.ngroups <= 1024;
      return c;
    }
  }
  return c;
}

}  // namespace spai
