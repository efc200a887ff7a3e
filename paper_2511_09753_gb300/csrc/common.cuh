// Internal types shared by the column-pass kernels, the PCG kernels and the
// host API of libspai.so.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spai {

constexpr unsigned kFull = 0xffffffffu;

// Device-resident scalars of one handle.  Written only by the last-arriving
// CTA of a pass (or by the host between calls); read by the next pass.
struct DevScalars {
  double alpha, beta, delta, gamma;  // step coefficients for the next pass
  double rr;                         // CG: ||R_i||_F^2 of the current residual
  double result;                     // scalar result of a norm pass
  int stop;                          // nonzero: later passes of this call do nothing
  int flags;                         // kFlag* bits
  int done;                          // iterations completed in this call
  int pad;
  unsigned long long bytes;          // algorithmic bytes moved by column passes
  unsigned long long spgemm_cols;    // column SpGEMMs performed
  unsigned long long r_bytes;        // of bytes: CG's R slab (pass A writes it, pass B reads it)
};

enum : int {
  kFlagConverged = 1,
  kFlagFallback = 2,
  kFlagNonfinite = 4,
  kFlagCapacity = 8,
};

// Which column pass a launch performs.
enum PassKind : int {
  kMR = 0,     // [update M with alpha] then R, P = D(R), Q = A P; partials rr, rq, qq
  kLOMR = 1,   // [S, P = D(S), M = D(M+S)] then R, Z = D(R), U = A Z, V = A P; 6 partials
  kCGA = 2,    // [M = D(M + alpha P)]; R; partial rr
  kCGB = 3,    // R; P = D(R + beta P); Q = A P; partials rr, pq
  kRES = 4,    // R = I - A M in FP64; partial rr
  kSCORE = 5,  // R = I - A M, then the Appendix A drop score of every entry of M
};

// Byte offsets of one warp's scratch inside the CTA's dynamic shared memory.
struct WarpLayout {
  int Mr, Mv, Pr, Pv, Zr, Zv;   // capped lists (CAP)
  int Sr, Sv;                   // LOMR S list (2 CAP)
  int Tr, Tv;                   // union output before drop (TMAX)
  int Rr, Rv;                   // SpGEMM output list (LMAX)
  int hk, hv, ho;               // hash table A: keys, values, occupied slots (H)
  int gk, gv, go;               // hash table B (LOMR)
  int uk, ua, ub, uo;           // union table (HU); shares its bytes with tie
  int tie;                      // int scratch of the threshold tie-break
  int zr, zv;                   // Pi-preconditioned forms: the list Pi R (LMAX)
  int hist;                     // 256 packed 16-bit bins (128 words)
  int H, HU;                    // table capacities (powers of two)
  int bytes;                    // total per warp (multiple of 16)
};

struct PassParams {
  int n;
  int W;             // ELL width of A
  uint32_t magicW;   // ceil(2^32 / W): q / W == __umulhi(q, magicW) for q < 2^16
  int B;             // columns per CTA (power of two)
  int NW;            // warps per CTA
  int capmax, pmax, lmax, tmax;
  int kind;
  int do_update, do_dir, drop;
  int keep_diag;     // per-column drops keep the column's diagonal entry
  int dir_from_slab;     // take the direction (MR, CG: P; LOMR: Z) stored in its slab instead of forming it
  int dir_store;         // MR, LOMR with do_dir = 0: still form the direction (P; Z) from R and store it
  int iter;          // history slot of this pass
  int fresh;         // CG: first B pass of a call (writes history[0])
  const long long* off;  // slab offsets (per column)
  const int* cap;        // per-column cap
  int* Mrow; void* Mval; int* Mlen;
  int* Prow; void* Pval; int* Plen;
  int* Zrow; void* Zval; int* Zlen;
  // CG: R of pass A kept for the next pass B, VC values, [n][capmax*W+1]
  int* Rrow; void* Rval; int* Rlen;
  int r_out;             // pass A: store R there
  int r_in;              // pass B: read R there instead of recomputing it
  const int* ell_col;
  const void* ell_val;   // VC values of A in ELL layout (padding column -1)
  int dia;               // nonzero: A is also stored by diagonal slots
  int D, Dp;             // number of distinct offsets, padded slot stride
  int dia_off[32];       // the offsets, ascending
  const void* dia_val;   // VC values [n][Dp], 0 where row k has no entry k+off
  const double* pi;      // Pi = diag(A)^{-1} per row (Pi-preconditioned forms), else null
  double* score;         // kSCORE: drop score per slab entry of M (+inf on the diagonal)
  const double* anrm;    // kSCORE: ||A e_k||^2 per row k
  DevScalars* sc;
  double* hist_res;      // [iters+1]
  unsigned long long* hist_nnz;  // [iters+1] nnz(M_i) (counts added per CTA), or null
  double* hist_coef;     // [2*iters]
  double* bsum;          // [NQ][nb]
  double* gsum;          // [NQ][ngroups]
  unsigned* cnt1;        // [ngroups]
  unsigned* cnt2;        // [1]
  int nb, ngroups;
  // batched mode (nseg > 0): independent matrices laid block-diagonally, each
  // padded to whole CTAs; every CTA belongs to one matrix (segment)
  int nseg;
  const int* seg_of_col;   // [n] segment of each column
  const int* seg_col0;     // [nseg] first column of each segment
  const int* seg_npad;     // [nseg] padded size (a multiple of B)
  DevScalars* segsc;       // [nseg] per-segment scalars
  const int* seg_D;        // [nseg] diagonal slots of each segment
  const int* seg_doff;     // [nseg][32] their offsets, ascending
  unsigned* seg_cnt;       // [nseg] arrival counters
  int hist_stride;         // per-segment history stride (iters + 1)
  WarpLayout lay;
  int part_off;          // byte offset of the CTA partials [NQ][B]
  int red_off;           // byte offset of CTA reduction scratch
};

// A steady-state pass: an update-and-direction pass of MR, LOMR or CG in the
// middle of a run (CG's passes exchanging R through its slab), in the plain
// forms, on an operator whose column products all take the short DIA form
// (columns of at most 32 entries, at most 8 diagonal slots).  Such passes
// run a kernel compiled for exactly these flags.
__host__ __device__ inline bool steady_pass(const PassParams& p) {
  if (p.kind != kMR && p.kind != kLOMR && p.kind != kCGA && p.kind != kCGB) return false;
  if (p.pi || !p.dia || p.capmax > 32 || p.D > 8) return false;
  if (!p.do_dir || p.dir_from_slab || p.dir_store) return false;
  if (p.kind == kCGB) return !p.fresh && p.r_in;
  if (p.kind == kCGA) return p.do_update && p.r_out;
  return p.do_update != 0;
}

constexpr int kGroup = 64;  // blocks per group in the last-arriver reduction tree

// partials per column: MR (R,R) (R,Q) (Q,Q); LOMR (R,R) (U,U) (V,V) (U,V)
// (U,R) (V,R); CG pass B (R,R) (P,Q) [+ (R,Pi R)]; CG pass A (R,R) [+ (R,Pi R)]
__host__ __device__ inline int pass_nq(int kind, bool pi = false) {
  return kind == kMR ? 3 : kind == kLOMR ? 6 : kind == kCGB ? (pi ? 3 : 2) : kind == kCGA ? (pi ? 2 : 1) : 1;
}

}  // namespace spai
