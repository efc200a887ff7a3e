// Host side of libspai.so: the C ABI declared in include/spai.h.
//
// A handle owns A (CSR for PCG, ELL for the column passes), three capped
// column slabs (M and the search directions P, Z), the device scalars and
// the reduction workspace.  Every numeric step runs in the kernels of
// colpass_*.cu and vec_kernels.cu; the host only validates input, lays out
// memory and sequences launches on the handle's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <thread>
#include <vector>

#include "spai.h"
#include "common.cuh"
#include "vec_kernels.cuh"
#include "bpcg.cuh"
#include "fixed_pattern.cuh"
#include "dropping.cuh"
#include "colpass_shape.cuh"

using namespace spai;

namespace {

constexpr int kSegAlign = 256;  // batched segments start at multiples of this

struct BatchDesc {
  int nseg;
  const long long* col0;   // first global column of each matrix
  const long long* nreal;  // its size
  const long long* npad;   // its padded size (multiple of kSegAlign)
};

}  // namespace

struct spai_ctx {
  int n = 0;
  long long nnz = 0;
  int prec = SPAI_FP64;
  double cap_factor = 2.0;
  int W = 1;
  uint32_t magicW = 0;
  int capmax = 1;
  long long slab_total = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // A
  int *d_rowptr = nullptr, *d_colind = nullptr;
  double *d_vals = nullptr, *d_diag = nullptr;
  int* d_ell_col = nullptr;
  float* d_ell32 = nullptr;
  double* d_ell64 = nullptr;
  bool dia = false;  // A also stored by diagonal slots
  int D = 0, Dp = 0;
  int dia_off[32];
  float* d_dia32 = nullptr;
  double* d_dia64 = nullptr;
  // slabs
  long long* d_off = nullptr;
  int* d_cap = nullptr;
  int *d_Mrow = nullptr, *d_Prow = nullptr, *d_Zrow = nullptr;
  void *d_Mval = nullptr, *d_Pval = nullptr, *d_Zval = nullptr;
  int *d_Mlen = nullptr, *d_Plen = nullptr, *d_Zlen = nullptr;
  // CG: the residual of pass A kept for the next pass B ([n][capmax*W+1])
  int *d_Rrow = nullptr, *d_Rlen = nullptr;
  void* d_Rval = nullptr;
  // scalars and reduction workspace
  DevScalars* d_sc = nullptr;
  double *d_hres = nullptr, *d_hcoef = nullptr;
  unsigned long long* d_hnnz = nullptr;  // nnz(M_i) history
  int hist_cap = 0;
  double *d_bsum = nullptr, *d_gsum = nullptr;
  unsigned *d_cnt1 = nullptr, *d_cnt2 = nullptr;
  int red_nb = 0, red_ng = 0;
  PassCfg cfg[5];
  // Pi-preconditioned forms: pi_k = 1 / a_kk, and the pass shapes of their
  // (larger) per-warp layouts for MR, LOMR, CG-A, CG-B
  double* d_pi = nullptr;
  PassCfg cfg_pi[4];
  bool pi_ok = false;
  // global dropping: ||A e_k||^2 per row and a score per slab entry of M
  double *d_anrm = nullptr, *d_score = nullptr;
  unsigned* d_hist = nullptr;
  // inputs of make_cfg kept for the launch-shape autotuner
  int smem_max = 0, Bmin = 1, Bmax = 1024;
  // batched mode: nseg matrices laid block-diagonally, each padded with
  // identity rows/columns to a multiple of kSegAlign
  int nseg = 0;
  std::vector<long long> seg_col0, seg_n, seg_npad;
  int *d_seg_of_col = nullptr, *d_seg_col0 = nullptr, *d_seg_npad = nullptr;
  int *d_seg_D = nullptr, *d_seg_doff = nullptr;
  DevScalars* d_segsc = nullptr;
  unsigned* d_seg_cnt = nullptr;
  int last_iters = 0;
  // method state (host mirror)
  int method = -1;
  int it = 0;
  // row-wise copies of M for spai_apply / PCG
  bool mt_valid = false, sym_valid = false;
  long long* d_ccolptr = nullptr;  // CSC export of M
  int* d_crow = nullptr;
  double* d_cval = nullptr;
  long long* d_mrp = nullptr;
  int* d_mci = nullptr;
  double* d_mv = nullptr;
  long long* d_srp = nullptr;
  int* d_sci = nullptr;
  double* d_sv = nullptr;
  // S's rows in sliced ELL for the FP64 PCG products (built with S)
  long long* d_ssp = nullptr;
  int* d_sscol = nullptr;
  double* d_ssval = nullptr;
  long long ss_cap = 0;
  int* d_slong = nullptr;  // rows of S too long for the sliced ELL, and their count
  int* d_nlong = nullptr;
  int nlong = 0;
  // with long rows: S's rows by length, longest first in each window of
  // 1,024 rows (slot order of its sliced ELL), and the long rows by length
  int* d_sperm = nullptr;
  int* d_slongs = nullptr;
  int* d_cnt = nullptr;
  long long* d_scan = nullptr;
  int *d_tmpi = nullptr;
  double* d_tmpv = nullptr;
  long long mt_cap = 0, sym_cap = 0;
  bool ssell_valid = false;
  // sliced-ELL copies for PCG: A (built on first use), and M or S
  long long* d_asp = nullptr;
  int *d_acol = nullptr, *d_w32 = nullptr;
  double* d_aval = nullptr;
  long long a_cap = 0;
  // PCG vectors
  double *d_b = nullptr, *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr,
         *d_q = nullptr;
  PcgScalars* d_ps = nullptr;
  double *d_vbsum = nullptr, *d_vgsum = nullptr;
  double* d_vrrsum = nullptr;  // PCG: the CTA partials of (r, r)
  unsigned *d_vcnt1 = nullptr, *d_vcnt2 = nullptr;
  // PCG arithmetic (SPAI_FP64, or SPAI_MIXED: FP32-values products) and the
  // FP32 copies it uses: A's sliced-ELL values, M's and S's row values, the
  // operand vectors
  int pcg_prec = SPAI_FP64;
  float *d_aval32 = nullptr, *d_mv32 = nullptr, *d_sv32 = nullptr, *d_p32 = nullptr,
        *d_r32 = nullptr, *d_bp32 = nullptr, *d_br32 = nullptr;
  long long mt_nnz = 0, sym_nnz = 0, mv32_cap = 0, sv32_cap = 0;
  bool m32_valid = false, s32_valid = false;
  // block PCG: vectors [n][32], per (matrix, rhs) state, segment maps
  double *d_bb = nullptr, *d_bx = nullptr, *d_br = nullptr, *d_bz = nullptr, *d_bp = nullptr,
         *d_bq = nullptr, *d_bstage = nullptr;
  long long bstage_cap = 0;
  double* d_bstate = nullptr;  // rho, alpha, beta, bn, tres: 5 x [nseg][32]
  int* d_bistate = nullptr;    // k, done, status: 3 x [nseg][32]
  int *d_bseg_live = nullptr, *d_blive = nullptr;
  double* d_bbsum = nullptr;
  unsigned* d_bcnt = nullptr;
  int *d_bseg_of_cta = nullptr, *d_bseg_cta0 = nullptr, *d_bseg_ncta = nullptr,
      *d_bseg_row0 = nullptr, *d_bseg_n = nullptr;
  long long* d_bseg_boff = nullptr;
  cudaGraphExec_t bp_graph = nullptr;
  unsigned char bp_graph_key[sizeof(spai::BpcgArgs)];
  cudaGraphExec_t pcg_graph = nullptr;  // a chunk of vector-PCG iterations
  // S's long rows run beside the others on a second stream (made on first use)
  cudaStream_t pcg_st2 = nullptr;
  cudaEvent_t pcg_fork = nullptr, pcg_join = nullptr;
  bool pcg_graph_forked = false;  // pcg_graph was captured with the second stream
  unsigned char pcg_graph_key[sizeof(spai::PcgArgs)];
  // stats
  long long colpass_launches = 0, pcg_launches = 0, other_launches = 0;
  long long steady_launches = 0;
  unsigned long long a_bytes_total = 0;
  double colpass_ms = 0.0;
  bool timing = false;
  // SPAI_GENERAL_KERNELS=1 at a run's start: steady-state passes take the
  // general kernels too (tests compare the two)
  bool general_only = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
};

namespace {

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) {               \
      (void)cudaGetLastError();            \
      return e_ == cudaErrorMemoryAllocation ? SPAI_ERR_OOM : SPAI_ERR_CUDA; \
    }                                      \
  } while (0)

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return SPAI_ERR_OOM;
  }
  return SPAI_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

int ensure_hist(spai_ctx* h, int iters) {
  if (iters + 1 <= h->hist_cap) return SPAI_OK;
  dfree(h->d_hres);
  dfree(h->d_hcoef);
  dfree(h->d_hnnz);
  int cap = std::max(iters + 1, 64);
  int rc = dalloc(&h->d_hres, cap);
  if (rc) return rc;
  rc = dalloc(&h->d_hcoef, 2 * cap);
  if (rc) return rc;
  rc = dalloc(&h->d_hnnz, cap);
  if (rc) return rc;
  h->hist_cap = cap;
  return SPAI_OK;
}

cudaError_t timed_launch(spai_ctx* h, const PassParams& p, const PassCfg& c, bool res) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->timing) {
    while ((int)h->ev.size() < h->ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      h->ev.push_back(e);
    }
    if ((int)h->ev.size() >= h->ev_used + 2) {
      e0 = h->ev[h->ev_used];
      e1 = h->ev[h->ev_used + 1];
      h->ev_used += 2;
      cudaEventRecord(e0, h->stream);
    }
  }
  cudaError_t err;
  if (p.pi)
    err = h->prec == SPAI_MIXED ? launch_colpass_pi_f32(p, c.grid, 32 * c.NW, c.smem, h->stream)
                                : launch_colpass_pi_f64(p, c.grid, 32 * c.NW, c.smem, h->stream);
  else if (res && h->prec == SPAI_MIXED)
    err = launch_colpass_res_f32(p, c.grid, 32 * c.NW, c.smem, h->stream);
  else if (!res && !h->general_only && steady_pass(p)) {
    err = h->prec == SPAI_MIXED ? launch_colpass_hot_f32(p, c.grid, 32 * c.NW, c.smem, h->stream)
                                : launch_colpass_hot_f64(p, c.grid, 32 * c.NW, c.smem, h->stream);
    h->steady_launches++;
  }
  else if (res || h->prec == SPAI_FP64)
    err = launch_colpass_f64(p, c.grid, 32 * c.NW, c.smem, h->stream);
  else
    err = launch_colpass_f32(p, c.grid, 32 * c.NW, c.smem, h->stream);
  if (e1) cudaEventRecord(e1, h->stream);
  h->colpass_launches++;
  int vc = (res || h->prec == SPAI_FP64) ? 8 : 4;
  h->a_bytes_total += (unsigned long long)h->n * h->W * (4 + vc);
  return err;
}

void collect_timing(spai_ctx* h) {
  for (int k = 0; k + 1 < h->ev_used; k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]) == cudaSuccess) h->colpass_ms += ms;
  }
  h->ev_used = 0;
}

PassParams base_params(spai_ctx* h, int kind, bool res, bool pi = false) {
  PassParams p;
  memset(&p, 0, sizeof(p));
  const PassCfg& c = pi ? h->cfg_pi[kind] : h->cfg[kind];
  p.pi = pi ? h->d_pi : nullptr;
  p.n = h->n;
  p.W = h->W;
  p.magicW = h->magicW;
  p.B = c.B;
  p.NW = c.NW;
  p.capmax = h->capmax;
  p.kind = kind;
  p.off = h->d_off;
  p.cap = h->d_cap;
  p.Mrow = h->d_Mrow;
  p.Mval = h->d_Mval;
  p.Mlen = h->d_Mlen;
  p.Prow = h->d_Prow;
  p.Pval = h->d_Pval;
  p.Plen = h->d_Plen;
  p.Zrow = h->d_Zrow;
  p.Zval = h->d_Zval;
  p.Zlen = h->d_Zlen;
  p.Rrow = h->d_Rrow;
  p.Rval = h->d_Rval;
  p.Rlen = h->d_Rlen;
  p.ell_col = h->d_ell_col;
  p.ell_val = (res || h->prec == SPAI_FP64) ? (const void*)h->d_ell64 : (const void*)h->d_ell32;
  p.dia = h->dia ? 1 : 0;
  p.D = h->D;
  p.Dp = h->Dp;
  for (int s2 = 0; s2 < 32; s2++) p.dia_off[s2] = h->dia ? h->dia_off[s2 < h->D ? s2 : 0] : 0;
  p.dia_val = (res || h->prec == SPAI_FP64) ? (const void*)h->d_dia64 : (const void*)h->d_dia32;
  p.nseg = h->nseg;
  p.seg_of_col = h->d_seg_of_col;
  p.seg_col0 = h->d_seg_col0;
  p.seg_npad = h->d_seg_npad;
  p.segsc = h->d_segsc;
  p.seg_D = h->d_seg_D;
  p.seg_doff = h->d_seg_doff;
  p.seg_cnt = h->d_seg_cnt;
  p.hist_stride = h->last_iters + 1;
  p.sc = h->d_sc;
  p.hist_res = h->d_hres;
  p.hist_coef = h->d_hcoef;
  p.bsum = h->d_bsum;
  p.gsum = h->d_gsum;
  p.cnt1 = h->d_cnt1;
  p.cnt2 = h->d_cnt2;
  p.nb = c.nb;
  p.ngroups = c.ngroups;
  p.lay = c.lay;
  p.part_off = c.part_off;
  p.red_off = c.red_off;
  return p;
}

// reset the per-call device scalars (stop, flags, done)
int reset_call_scalars(spai_ctx* h) {
  CK(cudaMemsetAsync((char*)h->d_sc + offsetof(DevScalars, stop), 0, 4 * sizeof(int), h->stream));
  return SPAI_OK;
}

void free_all(spai_ctx* h) {
  dfree(h->d_rowptr);
  dfree(h->d_colind);
  dfree(h->d_vals);
  dfree(h->d_diag);
  dfree(h->d_pi);
  dfree(h->d_ell_col);
  dfree(h->d_ell32);
  dfree(h->d_ell64);
  dfree(h->d_dia32);
  dfree(h->d_dia64);
  dfree(h->d_off);
  dfree(h->d_cap);
  dfree(h->d_Mrow);
  dfree(h->d_Prow);
  dfree(h->d_Zrow);
  dfree(h->d_Mval);
  dfree(h->d_Pval);
  dfree(h->d_Zval);
  dfree(h->d_Mlen);
  dfree(h->d_Plen);
  dfree(h->d_Zlen);
  dfree(h->d_Rrow);
  dfree(h->d_Rval);
  dfree(h->d_Rlen);
  dfree(h->d_sc);
  dfree(h->d_seg_of_col);
  dfree(h->d_seg_col0);
  dfree(h->d_seg_npad);
  dfree(h->d_seg_D);
  dfree(h->d_seg_doff);
  dfree(h->d_segsc);
  dfree(h->d_seg_cnt);
  dfree(h->d_hres);
  dfree(h->d_hcoef);
  dfree(h->d_hnnz);
  dfree(h->d_bsum);
  dfree(h->d_gsum);
  dfree(h->d_cnt1);
  dfree(h->d_cnt2);
  dfree(h->d_ccolptr);
  dfree(h->d_crow);
  dfree(h->d_cval);
  dfree(h->d_mrp);
  dfree(h->d_mci);
  dfree(h->d_mv);
  dfree(h->d_srp);
  dfree(h->d_sci);
  dfree(h->d_sv);
  dfree(h->d_ssp);
  dfree(h->d_sscol);
  dfree(h->d_ssval);
  dfree(h->d_slong);
  dfree(h->d_nlong);
  dfree(h->d_sperm);
  dfree(h->d_slongs);
  dfree(h->d_cnt);
  dfree(h->d_scan);
  dfree(h->d_tmpi);
  dfree(h->d_tmpv);
  dfree(h->d_asp);
  dfree(h->d_acol);
  dfree(h->d_w32);
  dfree(h->d_aval);
  dfree(h->d_b);
  dfree(h->d_x);
  dfree(h->d_r);
  dfree(h->d_z);
  dfree(h->d_p);
  dfree(h->d_q);
  dfree(h->d_ps);
  dfree(h->d_vbsum);
  dfree(h->d_vrrsum);
  dfree(h->d_vgsum);
  dfree(h->d_vcnt1);
  dfree(h->d_vcnt2);
  dfree(h->d_bb);
  dfree(h->d_bx);
  dfree(h->d_br);
  dfree(h->d_bz);
  dfree(h->d_bp);
  dfree(h->d_bq);
  dfree(h->d_bstage);
  dfree(h->d_anrm);
  dfree(h->d_score);
  dfree(h->d_hist);
  dfree(h->d_aval32);
  dfree(h->d_mv32);
  dfree(h->d_sv32);
  dfree(h->d_p32);
  dfree(h->d_r32);
  dfree(h->d_bp32);
  dfree(h->d_br32);
  dfree(h->d_bstate);
  dfree(h->d_bistate);
  dfree(h->d_bseg_live);
  dfree(h->d_blive);
  dfree(h->d_bbsum);
  dfree(h->d_bcnt);
  dfree(h->d_bseg_of_cta);
  dfree(h->d_bseg_cta0);
  dfree(h->d_bseg_ncta);
  dfree(h->d_bseg_row0);
  dfree(h->d_bseg_n);
  dfree(h->d_bseg_boff);
  if (h->bp_graph) cudaGraphExecDestroy(h->bp_graph);
  h->bp_graph = nullptr;
  if (h->pcg_graph) cudaGraphExecDestroy(h->pcg_graph);
  h->pcg_graph = nullptr;
  if (h->pcg_fork) cudaEventDestroy(h->pcg_fork);
  if (h->pcg_join) cudaEventDestroy(h->pcg_join);
  if (h->pcg_st2) cudaStreamDestroy(h->pcg_st2);
  h->pcg_fork = h->pcg_join = nullptr;
  h->pcg_st2 = nullptr;
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
}

// CSC export of M into h->d_ccolptr / d_crow / d_cval; returns nnz via *nnz
int export_csc(spai_ctx* h, long long* nnz) {
  const int n = h->n;
  if (!h->d_ccolptr) {
    int rc = dalloc(&h->d_ccolptr, (size_t)n + 1);
    if (rc) return rc;
    rc = dalloc(&h->d_scan, 2 * (size_t)((n + 1023) / 1024) + 2);
    if (rc) return rc;
  }
  CK(launch_exclusive_scan(h->d_Mlen, h->d_ccolptr, n, h->d_scan, h->stream));
  long long tot = 0;
  CK(cudaMemcpyAsync(&tot, h->d_ccolptr + n, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (tot > h->mt_cap || !h->d_crow) {
    dfree(h->d_crow);
    dfree(h->d_cval);
    dfree(h->d_mci);
    dfree(h->d_mv);
    dfree(h->d_tmpi);
    dfree(h->d_tmpv);
    long long cap = std::max(tot, (long long)h->slab_total);
    int rc = dalloc(&h->d_crow, (size_t)cap);
    if (!rc) rc = dalloc(&h->d_cval, (size_t)cap);
    if (!rc) rc = dalloc(&h->d_mci, (size_t)cap);
    if (!rc) rc = dalloc(&h->d_mv, (size_t)cap);
    if (!rc) rc = dalloc(&h->d_tmpi, (size_t)cap);
    if (!rc) rc = dalloc(&h->d_tmpv, (size_t)cap);
    if (rc) return rc;
    h->mt_cap = cap;
  }
  CK(launch_export_csc(h->prec, n, h->d_off, h->d_Mrow, h->d_Mval, h->d_ccolptr, h->d_crow,
                       h->d_cval, h->stream));
  h->other_launches += 4;
  *nnz = tot;
  return SPAI_OK;
}

// row-wise copy of M (and optionally its symmetric part) for apply / PCG
int ensure_rows(spai_ctx* h, bool sym) {
  const int n = h->n;
  if (!h->mt_valid) {
    long long nnz = 0;
    int rc = export_csc(h, &nnz);
    if (rc) return rc;
    if (!h->d_mrp) {
      rc = dalloc(&h->d_mrp, (size_t)n + 1);
      if (!rc) rc = dalloc(&h->d_cnt, (size_t)n + 1);
      if (rc) return rc;
    }
    CK(launch_transpose(n, h->d_ccolptr, h->d_crow, h->d_cval, nnz, h->d_cnt, h->d_mrp, h->d_scan,
                        h->d_mci, h->d_mv, h->d_tmpi, h->d_tmpv, h->stream));
    h->mt_nnz = nnz;
    h->other_launches += 7;
    h->mt_valid = true;
    h->sym_valid = false;
  }
  if (sym && !h->sym_valid) {
    if (!h->d_srp) {
      int rc = dalloc(&h->d_srp, (size_t)n + 1);
      if (rc) return rc;
    }
    CK(launch_sym(n, h->d_mrp, h->d_mci, h->d_mv, h->d_ccolptr, h->d_crow, h->d_cval, 0, h->d_cnt,
                  nullptr, nullptr, nullptr, h->stream));
    CK(launch_exclusive_scan(h->d_cnt, h->d_srp, n, h->d_scan, h->stream));
    long long tot = 0;
    CK(cudaMemcpyAsync(&tot, h->d_srp + n, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (tot > h->sym_cap || !h->d_sci) {
      dfree(h->d_sci);
      dfree(h->d_sv);
      int rc = dalloc(&h->d_sci, (size_t)tot);
      if (!rc) rc = dalloc(&h->d_sv, (size_t)tot);
      if (rc) return rc;
      h->sym_cap = tot;
    }
    CK(launch_sym(n, h->d_mrp, h->d_mci, h->d_mv, h->d_ccolptr, h->d_crow, h->d_cval, 1, h->d_cnt,
                  h->d_srp, h->d_sci, h->d_sv, h->stream));
    h->sym_nnz = tot;
    h->other_launches += 5;
    h->sym_valid = true;
    h->ssell_valid = false;
  }
  return SPAI_OK;
}

// S's rows in sliced ELL (coalesced loads for the FP64 preconditioner
// product); needs ensure_rows(h, true) first
int ensure_sym_sell(spai_ctx* h) {
  if (h->ssell_valid) return SPAI_OK;
  const int n = h->n, ns = (n + 31) / 32;
  if (!h->d_ssp) {
    int rc = dalloc(&h->d_ssp, (size_t)ns + 1);
    if (rc) return rc;
  }
  if (!h->d_w32) {
    int rc = dalloc(&h->d_w32, (size_t)ns + 1);
    if (rc) return rc;
  }
  if (!h->d_slong) {
    int rc = dalloc(&h->d_slong, (size_t)n);
    if (!rc) rc = dalloc(&h->d_nlong, 1);
    if (rc) return rc;
  }
  CK(launch_long_rows(n, h->d_srp, h->d_slong, h->d_nlong, h->stream));
  CK(cudaMemcpyAsync(&h->nlong, h->d_nlong, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->other_launches += 1;
  // with long rows the preconditioner product forms z apart from (r, z), so
  // its slots can hold the rows in any order: longest first, so that the 32
  // rows of a slice have like lengths and the slice's width wastes little
  const int* perm = nullptr;
  if (h->nlong) {
    if (!h->d_sperm) {
      int rc = dalloc(&h->d_sperm, (size_t)n);
      if (!rc) rc = dalloc(&h->d_slongs, (size_t)n);
      if (rc) return rc;
    }
    CK(launch_len_order(n, h->d_srp, h->d_sperm, h->stream));
    CK(launch_sort_long(h->d_slong, h->nlong, h->d_srp, h->d_slongs, h->stream));
    h->other_launches += 2;
    perm = h->d_sperm;
  }
  long long tot = 0;
  CK(launch_sell_build_i64(n, h->d_srp, h->d_sci, h->d_sv, h->d_w32, h->d_ssp, h->d_scan,
                           &h->d_sscol, &h->d_ssval, &h->ss_cap, &tot, h->stream, perm));
  h->other_launches += 5;
  h->ssell_valid = true;
  return SPAI_OK;
}

void invalidate_rows(spai_ctx* h) {
  h->mt_valid = false;
  h->sym_valid = false;
  h->ssell_valid = false;
  h->m32_valid = false;
  h->s32_valid = false;
}

}  // namespace

namespace {

// The first failure of a check over rows [0, n), f(lo, hi) returning
// {row, code} of its range's first failure or {hi, SPAI_OK}: ranges in
// parallel (host_threads); of the ranges that failed, the one at the
// smallest row wins, so the result is that of one scan in row order.
struct RowFail {
  int64_t row;
  int code;
};

// Host threads for a pass over the rows of a matrix: up to 16 when it is
// large (nnz >= 2^20), at least 1,024 rows each.
unsigned host_threads(int64_t n, int64_t nnz) {
  unsigned T = nnz >= (1LL << 20) ? std::min(16u, std::thread::hardware_concurrency()) : 1u;
  if (T > (unsigned)(n / 1024)) T = (unsigned)std::max<int64_t>(1, n / 1024);
  return std::max(T, 1u);
}

// f(t, lo, hi) for the T row ranges [n t / T, n (t + 1) / T), range 0 on the
// calling thread; ranges without a thread (none could be started) run here.
template <typename F>
void for_ranges(int64_t n, unsigned T, const F& f) {
  std::vector<std::thread> th;
  try {
    for (unsigned t = 1; t < T; t++)
      th.emplace_back([&, t] { f(t, n * t / T, n * (t + 1) / T); });
  } catch (...) {
  }
  for (unsigned t = (unsigned)th.size() + 1; t < T; t++) f(t, n * t / T, n * (t + 1) / T);
  f(0u, (int64_t)0, n / T);
  for (auto& x : th) x.join();
}

template <typename F>
RowFail over_rows(int64_t n, int64_t nnz, const F& f) {
  const unsigned T = host_threads(n, nnz);
  if (T <= 1) return f(0, n);
  std::vector<RowFail> r(T, RowFail{n, SPAI_OK});
  for_ranges(n, T, [&](unsigned t, int64_t lo, int64_t hi) { r[t] = f(lo, hi); });
  for (unsigned t = 0; t < T; t++)
    if (r[t].code) return r[t];
  return RowFail{n, SPAI_OK};
}

}  // namespace

extern "C" {

const char* spai_status_string(int code) {
  switch (code) {
    case SPAI_OK: return "ok";
    case SPAI_CONVERGED_EARLY: return "converged early (residual or step denominator reached zero)";
    case SPAI_LOMR_FALLBACK: return "LOMR took at least one MR step (near-singular 2x2 system)";
    case SPAI_PCG_MAXIT: return "PCG reached maxit";
    case SPAI_PCG_BREAKDOWN: return "PCG breakdown ((p,Ap) or (r,z) zero or non-finite)";
    case SPAI_ERR_ARG: return "invalid argument";
    case SPAI_ERR_CSR: return "malformed CSR matrix";
    case SPAI_ERR_NOT_SPD_DIAG: return "missing or non-positive diagonal entry";
    case SPAI_ERR_NOT_SYMMETRIC: return "matrix is not exactly symmetric";
    case SPAI_ERR_NONFINITE: return "non-finite value";
    case SPAI_ERR_CUDA: return "CUDA runtime error";
    case SPAI_ERR_OOM: return "device out of memory";
    case SPAI_ERR_CAPACITY: return "a column outgrew its slab capacity";
    case SPAI_ERR_UNSUPPORTED: return "size outside the kernels' limits";
    case SPAI_ERR_STATE: return "saved state does not match this handle";
    default: return "unknown status";
  }
}

int spai_validate_csr(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                      const double* vals, int check_symmetry) {
  if (n < 1 || nnz < 1 || !rowptr || !colind || !vals) return SPAI_ERR_ARG;
  if (n >= (1LL << 31) || nnz >= (1LL << 31)) return SPAI_ERR_UNSUPPORTED;
  if (rowptr[0] != 0 || rowptr[n] != nnz) return SPAI_ERR_CSR;
  // rows up to the first with a bad pointer (decreasing, or past nnz) have
  // entries that can be read; the checks run over row ranges in parallel,
  // and the failure at the smallest row is the one reported, as a scan in
  // row order would find it
  int64_t rows_ok = n;
  for (int64_t i = 0; i < n; i++)
    if (rowptr[i + 1] < rowptr[i] || rowptr[i + 1] > nnz) {
      rows_ok = i;
      break;
    }
  const auto check = [&](int64_t lo, int64_t hi) -> RowFail {
    for (int64_t i = lo; i < hi; i++) {
      bool diag = false;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
        int32_t c = colind[e];
        if (c < 0 || c >= n) return {i, SPAI_ERR_CSR};
        if (e > rowptr[i] && colind[e - 1] >= c) return {i, SPAI_ERR_CSR};
        if (!isfinite(vals[e])) return {i, SPAI_ERR_NONFINITE};
        if (c == i) {
          if (!(vals[e] > 0.0)) return {i, SPAI_ERR_NOT_SPD_DIAG};
          diag = true;
        }
      }
      if (!diag) return {i, SPAI_ERR_NOT_SPD_DIAG};
    }
    return {hi, SPAI_OK};
  };
  RowFail f = over_rows(rows_ok, nnz, check);
  if (f.code) return f.code;
  if (rows_ok < n) return SPAI_ERR_CSR;
  if (check_symmetry) {
    // every off-diagonal entry (i, c) has its mirror (c, i), found by
    // bisection in the sorted row c, with the same value
    const auto mirror = [&](int64_t lo, int64_t hi) -> RowFail {
      for (int64_t i = lo; i < hi; i++)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
          const int32_t c = colind[e];
          if (c == i) continue;
          const int32_t* b = colind + rowptr[c];
          const int32_t* en = colind + rowptr[c + 1];
          const int32_t* q = std::lower_bound(b, en, (int32_t)i);
          if (q == en || *q != i || vals[q - colind] != vals[e]) return {i, SPAI_ERR_NOT_SYMMETRIC};
        }
      return {hi, SPAI_OK};
    };
    f = over_rows(n, nnz, mirror);
    if (f.code) return f.code;
  }
  return SPAI_OK;
}

}  // extern "C"

namespace {

// Build a handle from a validated host CSR.  bd != nullptr: the CSR is the
// block-diagonal, padded concatenation of bd->nseg matrices.
int create_impl(spai_handle* out, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                const double* va, const spai_opts* opts, void* stream, const BatchDesc* bd) {
  int rc = SPAI_OK;
  spai_ctx* h = new (std::nothrow) spai_ctx();
  if (!h) return SPAI_ERR_OOM;
  h->n = (int)n;
  h->nnz = nnz;
  h->prec = opts->prec;
  h->cap_factor = opts->cap_factor;
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
  // ELL layout of A; padding entries point at the row itself with value 0
  int W = 1;
  for (int64_t i = 0; i < n; i++) W = std::max(W, (int)(rp[i + 1] - rp[i]));
  std::vector<int> cap(n);
  std::vector<long long> off(n + 1);
  off[0] = 0;
  int capmax = 1;
  std::vector<int> seg_of_col;
  if (bd) {
    seg_of_col.assign(n, 0);
    for (int m = 0; m < bd->nseg; m++)
      for (long long q = 0; q < bd->npad[m]; q++) seg_of_col[bd->col0[m] + q] = m;
  }
  for (int64_t j = 0; j < n; j++) {
    double c = floor(opts->cap_factor * (double)(rp[j + 1] - rp[j]));
    const double lim = bd ? (double)bd->nreal[seg_of_col[j]] : (double)n;
    if (!(c >= 1.0)) c = 1.0;
    if (c > lim) c = lim;
    if (c < 1.0) c = 1.0;
    cap[j] = (int)c;
    capmax = std::max(capmax, cap[j]);
    off[j + 1] = off[j] + cap[j];
  }
  if (W > 64 || (long long)capmax * W + 2 > 65535) {
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return SPAI_ERR_UNSUPPORTED;
  }
  h->W = W;
  h->magicW = (uint32_t)((((uint64_t)1 << 32) + W - 1) / W);
  h->capmax = capmax;
  h->slab_total = off[n];
  // A's ELL and diagonal-slot copies are built on the device from its CSR
  // (launch_build_ell / launch_build_dia below); the host finds the diagonal
  // and the slot offsets
  std::vector<double> diag(n);
  const unsigned T = host_threads(n, nnz);
  for_ranges(n, T, [&](unsigned, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; i++)
      for (int64_t e = rp[i]; e < rp[i + 1]; e++)
        if (ci[e] == i) diag[i] = va[e];
  });
  // diagonal-slot layout when A has at most 32 distinct offsets col - row
  std::vector<int> seg_D, seg_doff;
  if (bd) {
    // per-matrix diagonal slots; every matrix must have at most 32
    bool ok = true;
    seg_D.assign(bd->nseg, 0);
    seg_doff.assign((size_t)bd->nseg * 32, 0);
    int Dmax = 0;
    for (int m = 0; m < bd->nseg && ok; m++) {
      std::vector<long long> offs;
      std::vector<int> hint;  // as for a single matrix below
      for (long long i = bd->col0[m]; i < bd->col0[m] + bd->npad[m] && ok; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
          const long long o = (long long)ci[e] - i;
          const size_t t = (size_t)(e - rp[i]);
          if (t < hint.size() && offs[hint[t]] == o) continue;
          auto f = std::find(offs.begin(), offs.end(), o);
          if (f == offs.end()) {
            offs.push_back(o);
            if (offs.size() > 32) {
              ok = false;
              break;
            }
            f = offs.end() - 1;
          }
          if (t >= hint.size()) hint.resize(t + 1, 0);
          hint[t] = (int)(f - offs.begin());
        }
      if (!ok) break;
      std::sort(offs.begin(), offs.end());
      seg_D[m] = (int)offs.size();
      for (size_t s2 = 0; s2 < offs.size(); s2++) seg_doff[(size_t)m * 32 + s2] = (int)offs[s2];
      Dmax = std::max(Dmax, seg_D[m]);
    }
    if (ok) {
      h->dia = true;
      h->D = Dmax;
      h->Dp = (Dmax + 3) & ~3;
      for (int s2 = 0; s2 < 32; s2++) h->dia_off[s2] = 0;
    } else {
      seg_D.clear();
      seg_doff.clear();
    }
  } else {
    // the distinct offsets col - row of each row range (more than 32 in a
    // range or in all: no diagonal slots), then their union
    std::vector<std::vector<long long>> part(T);
    for_ranges(n, T, [&](unsigned r, int64_t lo, int64_t hi) {
      std::vector<long long>& offs = part[r];
      std::vector<int> hint;  // index in offs of the t-th entry's offset in the previous row
      bool rok = true;
      for (int64_t i = lo; i < hi && rok; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
          const long long o = (long long)ci[e] - i;
          const size_t t = (size_t)(e - rp[i]);
          if (t < hint.size() && offs[hint[t]] == o) continue;
          auto f = std::find(offs.begin(), offs.end(), o);
          if (f == offs.end()) {
            offs.push_back(o);
            if (offs.size() > 32) {
              rok = false;
              break;
            }
            f = offs.end() - 1;
          }
          if (t >= hint.size()) hint.resize(t + 1, 0);
          hint[t] = (int)(f - offs.begin());
        }
    });
    std::vector<long long> offs;
    for (auto& pr : part) offs.insert(offs.end(), pr.begin(), pr.end());
    std::sort(offs.begin(), offs.end());
    offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
    const bool ok = offs.size() <= 32;
    if (ok) {
      std::sort(offs.begin(), offs.end());
      h->dia = true;
      h->D = (int)offs.size();
      h->Dp = (h->D + 3) & ~3;
      for (int s2 = 0; s2 < h->D; s2++) h->dia_off[s2] = (int)offs[s2];
    }
  }
  int dev = 0;
  cudaGetDevice(&dev);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem_max <= 0) smem_max = 227 * 1024;
  const int vc = h->prec == SPAI_MIXED ? 4 : 8;
  for (int k = 0; k < 5; k++) {
    int Bmin = 1, Bmax = 1024;
    if (bd) {
      long long npmax = 0;
      for (int m = 0; m < bd->nseg; m++) npmax = std::max(npmax, bd->npad[m]);
      while ((long long)Bmin * 1024 < npmax) Bmin *= 2;  // <= 1024 CTAs per matrix
      Bmax = kSegAlign;
    }
    h->cfg[k] = make_cfg(k, k == kRES ? 8 : vc, (int)n, capmax, W, h->dia, smem_max, Bmin, Bmax);
    if (!h->cfg[k].ok) {
      if (h->own_stream) cudaStreamDestroy(h->stream);
      delete h;
      return SPAI_ERR_UNSUPPORTED;
    }
    h->red_nb = std::max(h->red_nb, h->cfg[k].nb);
    h->red_ng = std::max(h->red_ng, h->cfg[k].ngroups);
  }
  h->smem_max = smem_max;
  {
    int Bmin = 1, Bmax = 1024;
    if (bd) {
      long long npmax = 0;
      for (int m = 0; m < bd->nseg; m++) npmax = std::max(npmax, bd->npad[m]);
      while ((long long)Bmin * 1024 < npmax) Bmin *= 2;
      Bmax = kSegAlign;
    }
    h->Bmin = Bmin;
    h->Bmax = Bmax;
  }
  h->pi_ok = true;
  for (int k = 0; k < 4; k++) {
    int Bmin = 1, Bmax = 1024;
    if (bd) {
      long long npmax = 0;
      for (int m = 0; m < bd->nseg; m++) npmax = std::max(npmax, bd->npad[m]);
      while ((long long)Bmin * 1024 < npmax) Bmin *= 2;
      Bmax = kSegAlign;
    }
    h->cfg_pi[k] = make_cfg(k, vc, (int)n, capmax, W, h->dia, smem_max, Bmin, Bmax, true);
    if (!h->cfg_pi[k].ok) {
      h->pi_ok = false;
      continue;
    }
    h->red_nb = std::max(h->red_nb, h->cfg_pi[k].nb);
    h->red_ng = std::max(h->red_ng, h->cfg_pi[k].ngroups);
  }
  const size_t vs = h->prec == SPAI_MIXED ? 4 : 8;
  rc = SPAI_OK;
  rc = rc ? rc : dalloc(&h->d_rowptr, n + 1);
  rc = rc ? rc : dalloc(&h->d_colind, nnz);
  rc = rc ? rc : dalloc(&h->d_vals, nnz);
  rc = rc ? rc : dalloc(&h->d_diag, n);
  rc = rc ? rc : dalloc(&h->d_pi, n);
  rc = rc ? rc : dalloc(&h->d_ell_col, (size_t)n * W);
  rc = rc ? rc : dalloc(&h->d_ell64, (size_t)n * W);
  if (h->prec == SPAI_MIXED) rc = rc ? rc : dalloc(&h->d_ell32, (size_t)n * W);
  if (h->dia) {
    rc = rc ? rc : dalloc(&h->d_dia64, (size_t)n * h->Dp);
    if (h->prec == SPAI_MIXED) rc = rc ? rc : dalloc(&h->d_dia32, (size_t)n * h->Dp);
  }
  rc = rc ? rc : dalloc(&h->d_off, n + 1);
  rc = rc ? rc : dalloc(&h->d_cap, n);
  rc = rc ? rc : dalloc(&h->d_Mrow, h->slab_total);
  rc = rc ? rc : dalloc(&h->d_Prow, h->slab_total);
  rc = rc ? rc : dalloc(&h->d_Zrow, h->slab_total);
  rc = rc ? rc : dalloc((char**)&h->d_Mval, h->slab_total * vs);
  rc = rc ? rc : dalloc((char**)&h->d_Pval, h->slab_total * vs);
  rc = rc ? rc : dalloc((char**)&h->d_Zval, h->slab_total * vs);
  rc = rc ? rc : dalloc(&h->d_Mlen, n);
  rc = rc ? rc : dalloc(&h->d_Plen, n);
  rc = rc ? rc : dalloc(&h->d_Zlen, n);
  rc = rc ? rc : dalloc(&h->d_sc, 1);
  rc = rc ? rc : dalloc(&h->d_bsum, (size_t)6 * h->red_nb);
  rc = rc ? rc : dalloc(&h->d_gsum, (size_t)6 * h->red_ng);
  rc = rc ? rc : dalloc(&h->d_cnt1, h->red_ng);
  rc = rc ? rc : dalloc(&h->d_cnt2, 1);
  rc = rc ? rc : ensure_hist(h, 64);
  if (bd) {
    h->nseg = bd->nseg;
    h->seg_col0.assign(bd->col0, bd->col0 + bd->nseg);
    h->seg_n.assign(bd->nreal, bd->nreal + bd->nseg);
    h->seg_npad.assign(bd->npad, bd->npad + bd->nseg);
    rc = rc ? rc : dalloc(&h->d_seg_of_col, n);
    rc = rc ? rc : dalloc(&h->d_seg_col0, bd->nseg);
    rc = rc ? rc : dalloc(&h->d_seg_npad, bd->nseg);
    rc = rc ? rc : dalloc(&h->d_seg_D, bd->nseg);
    rc = rc ? rc : dalloc(&h->d_seg_doff, (size_t)bd->nseg * 32);
    rc = rc ? rc : dalloc(&h->d_segsc, bd->nseg);
    rc = rc ? rc : dalloc(&h->d_seg_cnt, bd->nseg);
    rc = rc ? rc : ensure_hist(h, 64 * bd->nseg);
  }
  if (rc) {
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return rc;
  }
  cudaStream_t st = h->stream;
  bool ok = true;
  ok &= cudaMemcpyAsync(h->d_rowptr, rp, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st) == 0;
  ok &= cudaMemcpyAsync(h->d_colind, ci, sizeof(int) * nnz, cudaMemcpyHostToDevice, st) == 0;
  ok &= cudaMemcpyAsync(h->d_vals, va, sizeof(double) * nnz, cudaMemcpyHostToDevice, st) == 0;
  ok &= cudaMemcpyAsync(h->d_diag, diag.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) == 0;
  std::vector<double> piv(n);
  for (int64_t i = 0; i < n; i++) piv[i] = 1.0 / diag[i];
  ok &= cudaMemcpyAsync(h->d_pi, piv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) == 0;
  ok &= cudaMemcpyAsync(h->d_off, off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                        st) == 0;
  ok &= cudaMemcpyAsync(h->d_cap, cap.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) == 0;
  ok &= cudaMemsetAsync(h->d_sc, 0, sizeof(DevScalars), st) == 0;
  if (bd) {
    std::vector<int> c0(bd->nseg), np(bd->nseg);
    for (int m = 0; m < bd->nseg; m++) {
      c0[m] = (int)bd->col0[m];
      np[m] = (int)bd->npad[m];
    }
    if (seg_D.empty()) {
      seg_D.assign(bd->nseg, 0);
      seg_doff.assign((size_t)bd->nseg * 32, 0);
    }
    ok &= cudaMemcpyAsync(h->d_seg_of_col, seg_of_col.data(), sizeof(int) * n,
                          cudaMemcpyHostToDevice, st) == 0;
    ok &= cudaMemcpyAsync(h->d_seg_col0, c0.data(), sizeof(int) * bd->nseg, cudaMemcpyHostToDevice,
                          st) == 0;
    ok &= cudaMemcpyAsync(h->d_seg_npad, np.data(), sizeof(int) * bd->nseg, cudaMemcpyHostToDevice,
                          st) == 0;
    ok &= cudaMemcpyAsync(h->d_seg_D, seg_D.data(), sizeof(int) * bd->nseg, cudaMemcpyHostToDevice,
                          st) == 0;
    ok &= cudaMemcpyAsync(h->d_seg_doff, seg_doff.data(), sizeof(int) * seg_doff.size(),
                          cudaMemcpyHostToDevice, st) == 0;
    ok &= cudaMemsetAsync(h->d_segsc, 0, sizeof(DevScalars) * bd->nseg, st) == 0;
    ok &= cudaMemsetAsync(h->d_seg_cnt, 0, sizeof(unsigned) * bd->nseg, st) == 0;
    // keep the host copies alive until the copies have run
    ok &= cudaStreamSynchronize(st) == 0;
  }
  ok &= cudaMemsetAsync(h->d_cnt1, 0, sizeof(unsigned) * h->red_ng, st) == 0;
  ok &= cudaMemsetAsync(h->d_cnt2, 0, sizeof(unsigned), st) == 0;
  ok &= launch_build_ell((int)n, W, h->d_rowptr, h->d_colind, h->d_vals, h->d_ell_col, h->d_ell64,
                         h->prec == SPAI_MIXED ? h->d_ell32 : nullptr, st) == 0;
  if (h->dia)
    ok &= launch_build_dia((int)n, h->D, h->Dp, h->d_rowptr, h->d_colind, h->d_vals,
                           bd ? nullptr : h->dia_off, bd ? h->d_seg_of_col : nullptr,
                           bd ? h->d_seg_doff : nullptr, bd ? h->d_seg_D : nullptr, h->d_dia64,
                           h->prec == SPAI_MIXED ? h->d_dia32 : nullptr, st) == 0;
  h->other_launches += h->dia ? 2 : 1;
  ok &= launch_init_slab(h->prec, (int)n, h->d_off, h->d_diag, h->d_Mrow, h->d_Mval, h->d_Mlen,
                         h->d_Plen, h->d_Zlen, st) == 0;
  ok &= cudaStreamSynchronize(st) == 0;
  h->other_launches += 1;
  if (!ok) {
    (void)cudaGetLastError();
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return SPAI_ERR_CUDA;
  }
  *out = h;
  return SPAI_OK;
}

}  // namespace

extern "C" {

int spai_create(spai_handle* out, int64_t n, int64_t nnz, const int32_t* rowptr,
                const int32_t* colind, const double* vals, int on_device, const spai_opts* opts,
                void* stream) {
  if (!out) return SPAI_ERR_ARG;
  *out = nullptr;
  if (!opts || n < 1 || nnz < 1 || !rowptr || !colind || !vals) return SPAI_ERR_ARG;
  if (opts->prec != SPAI_FP64 && opts->prec != SPAI_MIXED) return SPAI_ERR_ARG;
  if (!(opts->cap_factor > 0.0)) return SPAI_ERR_ARG;
  if (n >= (1LL << 26) || nnz >= (1LL << 31)) return SPAI_ERR_UNSUPPORTED;
  std::vector<int32_t> hrp, hci;
  std::vector<double> hv;
  const int32_t* rp = rowptr;
  const int32_t* ci = colind;
  const double* va = vals;
  if (on_device) {
    hrp.resize(n + 1);
    hci.resize(nnz);
    hv.resize(nnz);
    if (cudaMemcpy(hrp.data(), rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(hci.data(), colind, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(hv.data(), vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost)) {
      (void)cudaGetLastError();
      return SPAI_ERR_CUDA;
    }
    rp = hrp.data();
    ci = hci.data();
    va = hv.data();
  }
  int rc = spai_validate_csr(n, nnz, rp, ci, va, 1);
  if (rc) return rc;
  return create_impl(out, n, nnz, rp, ci, va, opts, stream, nullptr);
}

int spai_create_batched(spai_handle* out, int nmat, const int64_t* n, const int64_t* nnz,
                        const int32_t* const* rowptr, const int32_t* const* colind,
                        const double* const* vals, const spai_opts* opts, void* stream) {
  if (!out) return SPAI_ERR_ARG;
  *out = nullptr;
  if (!opts || nmat < 1 || !n || !nnz || !rowptr || !colind || !vals) return SPAI_ERR_ARG;
  if (opts->prec != SPAI_FP64 && opts->prec != SPAI_MIXED) return SPAI_ERR_ARG;
  if (!(opts->cap_factor > 0.0)) return SPAI_ERR_ARG;
  std::vector<long long> col0(nmat), nreal(nmat), npad(nmat);
  long long N = 0, NNZ = 0;
  for (int m = 0; m < nmat; m++) {
    if (!rowptr[m] || !colind[m] || !vals[m]) return SPAI_ERR_ARG;
    int rc = spai_validate_csr(n[m], nnz[m], rowptr[m], colind[m], vals[m], 1);
    if (rc) return rc;
    nreal[m] = n[m];
    npad[m] = (n[m] + kSegAlign - 1) / kSegAlign * kSegAlign;
    if (npad[m] > 1024LL * kSegAlign) return SPAI_ERR_UNSUPPORTED;
    col0[m] = N;
    N += npad[m];
    NNZ += nnz[m] + (npad[m] - n[m]);
  }
  if (N >= (1LL << 26) || NNZ >= (1LL << 31)) return SPAI_ERR_UNSUPPORTED;
  // block-diagonal concatenation; padding rows are identity rows
  std::vector<int32_t> grp(N + 1), gci(NNZ);
  std::vector<double> gv(NNZ);
  long long e = 0, row = 0;
  grp[0] = 0;
  for (int m = 0; m < nmat; m++) {
    for (long long i = 0; i < n[m]; i++, row++) {
      for (int32_t q = rowptr[m][i]; q < rowptr[m][i + 1]; q++, e++) {
        gci[e] = (int32_t)(colind[m][q] + col0[m]);
        gv[e] = vals[m][q];
      }
      grp[row + 1] = (int32_t)e;
    }
    for (long long i = n[m]; i < npad[m]; i++, row++) {
      gci[e] = (int32_t)row;
      gv[e] = 1.0;
      e++;
      grp[row + 1] = (int32_t)e;
    }
  }
  BatchDesc bd{nmat, col0.data(), nreal.data(), npad.data()};
  return create_impl(out, N, NNZ, grp.data(), gci.data(), gv.data(), opts, stream, &bd);
}

int spai_destroy(spai_handle h) {
  if (!h) return SPAI_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return SPAI_OK;
}

int spai_set_stream(spai_handle h, void* stream) {
  if (!h) return SPAI_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  return SPAI_OK;
}

int spai_reset(spai_handle h) {
  if (!h) return SPAI_ERR_ARG;
  CK(launch_init_slab(h->prec, h->n, h->d_off, h->d_diag, h->d_Mrow, h->d_Mval, h->d_Mlen,
                      h->d_Plen, h->d_Zlen, h->stream));
  h->other_launches++;
  h->method = -1;
  h->it = 0;
  invalidate_rows(h);
  CK(cudaStreamSynchronize(h->stream));
  return SPAI_OK;
}

int spai_run(spai_handle h, int method, int iters, int drop_rule, spai_history* hist) {
  if (!h || iters < 0 || method < SPAI_MR || method > SPAI_CG_PI) return SPAI_ERR_ARG;
  const bool pim = method >= SPAI_MR_PI;  // Section 5's forms with Pi = diag(A)^{-1}
  if (pim && !h->pi_ok) return SPAI_ERR_UNSUPPORTED;
  const int base = pim ? method - SPAI_MR_PI : method;
  if (drop_rule != SPAI_DROP_NONE && drop_rule != SPAI_DROP_TOPK_COL &&
      drop_rule != SPAI_DROP_TOPK_COL_DIAG)
    return SPAI_ERR_ARG;
  const int nh = std::max(h->nseg, 1);
  int rc = ensure_hist(h, (iters + 1) * nh);
  if (rc) return rc;
  h->last_iters = iters;
  cudaStream_t st = h->stream;
  const bool fresh = h->method != method;
  if (fresh) {
    CK(cudaMemsetAsync(h->d_Plen, 0, sizeof(int) * h->n, st));
    CK(cudaMemsetAsync(h->d_Zlen, 0, sizeof(int) * h->n, st));
    CK(cudaMemsetAsync((char*)h->d_sc + offsetof(DevScalars, beta), 0, sizeof(double), st));
    CK(cudaMemsetAsync((char*)h->d_sc + offsetof(DevScalars, rr), 0, sizeof(double), st));
  }
  rc = reset_call_scalars(h);
  if (rc) return rc;
  if (h->nseg) CK(launch_seg_reset(h->d_segsc, h->nseg, fresh ? 1 : 0, st));
  CK(cudaMemsetAsync(h->d_hres, 0xff, sizeof(double) * (iters + 1) * nh, st));
  CK(cudaMemsetAsync(h->d_hcoef, 0xff, sizeof(double) * 2 * std::max(iters, 1) * nh, st));
  CK(cudaMemsetAsync(h->d_hnnz, 0, sizeof(unsigned long long) * (iters + 1) * nh, st));
  invalidate_rows(h);
  const int drop = drop_rule != SPAI_DROP_NONE ? 1 : 0;
  const int keep_diag = drop_rule == SPAI_DROP_TOPK_COL_DIAG ? 1 : 0;
  // CG: pass A keeps R_{i+1} for pass B of the next iteration, which then
  // reads it instead of repeating the product (the same values)
  // (the slab is an optimisation: without device memory for it, pass B
  // recomputes R as before)
  // SPAI_CG_NO_R_SLAB=1 takes the recomputing path on purpose (tests)
  bool keep_r = base == SPAI_CG && iters > 1 && !env_int("SPAI_CG_NO_R_SLAB", 0);
  h->general_only = env_int("SPAI_GENERAL_KERNELS", 0) != 0;
  if (keep_r && !h->d_Rrow) {
    const size_t cnt = (size_t)h->n * ((size_t)h->capmax * h->W + 1);
    const size_t vb = h->prec == SPAI_FP64 ? 8 : 4;
    rc = dalloc(&h->d_Rrow, cnt);
    if (!rc) rc = dalloc((char**)&h->d_Rval, cnt * vb);
    if (!rc) rc = dalloc(&h->d_Rlen, (size_t)h->n);
    if (rc) {
      dfree(h->d_Rrow);
      dfree(h->d_Rval);
      dfree(h->d_Rlen);
      keep_r = false;
      rc = SPAI_OK;
    }
  }
  auto pass = [&](int kind, int upd, int dir, int iter, int fresh_b, int r_in = 0,
                  int r_out = 0) -> cudaError_t {
    PassParams p = base_params(h, kind, false, pim);
    p.do_update = upd;
    p.do_dir = dir;
    p.drop = drop;
    p.keep_diag = keep_diag;
    p.hist_nnz = h->d_hnnz;
    p.iter = iter;
    p.fresh = fresh_b;
    p.r_in = r_in;
    p.r_out = r_out;
    return timed_launch(h, p, pim ? h->cfg_pi[kind] : h->cfg[kind], false);
  };
  if (base == SPAI_MR || base == SPAI_LOMR) {
    const int kind = base == SPAI_MR ? kMR : kLOMR;
    if (iters == 0) {
      CK(pass(kind, 0, 0, 0, 0));
    } else {
      CK(pass(kind, 0, 1, 0, 0));
      for (int i = 1; i < iters; i++) CK(pass(kind, 1, 1, i, 0));
      CK(pass(kind, 1, 0, iters, 0));
    }
  } else {
    if (iters == 0) {
      CK(pass(kCGB, 0, 1, 0, 1));
    } else {
      for (int i = 0; i < iters; i++) {
        CK(pass(kCGB, 0, 1, i, i == 0, keep_r && i > 0));
        CK(pass(kCGA, 1, 1, i, 0, 0, keep_r && i + 1 < iters));
      }
    }
  }
  DevScalars sc;
  CK(cudaMemcpyAsync(&sc, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
  if (hist && hist->resnorm)
    CK(cudaMemcpyAsync(hist->resnorm, h->d_hres, sizeof(double) * (iters + 1),
                       cudaMemcpyDeviceToHost, st));
  if (hist && hist->coef && iters > 0)
    CK(cudaMemcpyAsync(hist->coef, h->d_hcoef, sizeof(double) * 2 * iters, cudaMemcpyDeviceToHost,
                       st));
  std::vector<unsigned long long> hnnz;
  if (hist && hist->nnz && !h->nseg) {
    hnnz.resize(iters + 1);
    CK(cudaMemcpyAsync(hnnz.data(), h->d_hnnz, sizeof(unsigned long long) * (iters + 1),
                       cudaMemcpyDeviceToHost, st));
  }
  std::vector<DevScalars> ssc;
  if (h->nseg) {
    ssc.resize(h->nseg);
    CK(cudaMemcpyAsync(ssc.data(), h->d_segsc, sizeof(DevScalars) * h->nseg,
                       cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  if (h->timing) collect_timing(h);
  if (h->nseg) {
    // batched: combine the matrices' outcomes (fewest iterations done, all flags)
    int done = iters, flags = 0;
    for (const DevScalars& x : ssc) {
      done = std::min(done, x.done);
      flags |= x.flags;
    }
    sc.done = done;
    sc.flags |= flags;
  }
  if (hist) {
    hist->iters_done = sc.done;
    hist->flags = sc.flags & 3;
    // entries up to the last history entry written: iters_done (+1 for the
    // final residual when every iteration ran)
    if (hist->nnz && !h->nseg) {
      const int last = sc.done == iters ? iters : sc.done;
      for (int i = 0; i <= last && i <= iters; i++) hist->nnz[i] = (int64_t)hnnz[i];
    }
  }
  h->method = method;
  h->it += sc.done;
  if (sc.flags & kFlagCapacity) {
    h->method = -1;
    return SPAI_ERR_CAPACITY;
  }
  if (sc.flags & kFlagNonfinite) {
    h->method = -1;
    return SPAI_ERR_NONFINITE;
  }
  if (sc.flags & kFlagConverged) {
    h->method = -1;
    return SPAI_CONVERGED_EARLY;
  }
  if (sc.flags & kFlagFallback) return SPAI_LOMR_FALLBACK;
  return SPAI_OK;
}

int spai_autotune(spai_handle h, int method, int iters, double* best_ms) {
  if (!h || iters < 1 || method < SPAI_MR || method > SPAI_CG_PI) return SPAI_ERR_ARG;
  const bool pim = method >= SPAI_MR_PI;
  if (pim && !h->pi_ok) return SPAI_ERR_UNSUPPORTED;
  const int base = pim ? method - SPAI_MR_PI : method;
  int kinds[2] = {base == SPAI_MR ? kMR : base == SPAI_LOMR ? kLOMR : kCGA, kCGB};
  const int nk = base == SPAI_CG ? 2 : 1;
  PassCfg* cfgs = pim ? h->cfg_pi : h->cfg;
  const int vc = h->prec == SPAI_MIXED ? 4 : 8;
  PassCfg keep[2] = {cfgs[kinds[0]], cfgs[kinds[1]]};
  double best = 1e300;
  PassCfg bestc[2] = {keep[0], keep[1]};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    (void)cudaGetLastError();
    return SPAI_ERR_CUDA;
  }
  int rc = SPAI_OK;
  std::vector<long long> tried;  // (NW, B) of each kind, packed
  for (int occ = 1; occ <= 8 && !rc; occ++)
    for (int cpw = 1; cpw <= 8 && !rc; cpw *= 2) {
      PassCfg c[2];
      bool ok = true;
      long long key = 0;
      for (int q = 0; q < nk; q++) {
        c[q] = make_cfg(kinds[q], vc, h->n, h->capmax, h->W, h->dia, h->smem_max, h->Bmin, h->Bmax,
                        pim, occ, cpw);
        ok &= c[q].ok && c[q].nb <= h->red_nb && c[q].ngroups <= h->red_ng;
        key = key * 65536 + (long long)c[q].NW * 2048 + c[q].B;
      }
      if (!ok || std::find(tried.begin(), tried.end(), key) != tried.end()) continue;
      tried.push_back(key);
      for (int q = 0; q < nk; q++) cfgs[kinds[q]] = c[q];
      // untimed: `iters` iterations from M_0, so that the columns have
      // filled towards their caps before the timed iterations
      rc = spai_reset(h);
      if (!rc) {
        int r1 = spai_run(h, method, iters, SPAI_DROP_TOPK_COL, nullptr);
        if (r1 < 0) rc = r1;
      }
      if (rc) break;
      cudaEventRecord(e0, h->stream);
      int r2 = spai_run(h, method, iters, SPAI_DROP_TOPK_COL, nullptr);
      cudaEventRecord(e1, h->stream);
      if (r2 < 0) {
        rc = r2;
        break;
      }
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = SPAI_ERR_CUDA;
        break;
      }
      const double per = (double)ms / iters;
      if (per < best) {
        best = per;
        bestc[0] = c[0];
        bestc[1] = c[1];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int q = 0; q < nk; q++) cfgs[kinds[q]] = rc ? keep[q] : bestc[q];
  int r3 = spai_reset(h);
  if (rc) return rc;
  if (best_ms) *best_ms = best;
  return r3;
}

int spai_batch_info(spai_handle h, int* nmat, int64_t* n_each) {
  if (!h || !nmat) return SPAI_ERR_ARG;
  *nmat = h->nseg ? h->nseg : 1;
  if (n_each) {
    if (h->nseg)
      for (int m = 0; m < h->nseg; m++) n_each[m] = h->seg_n[m];
    else
      n_each[0] = h->n;
  }
  return SPAI_OK;
}

int spai_batch_history(spai_handle h, double* resnorm, int* iters_done, int* flags) {
  if (!h) return SPAI_ERR_ARG;
  const int nh = std::max(h->nseg, 1);
  const int stride = h->last_iters + 1;
  cudaStream_t st = h->stream;
  if (resnorm)
    CK(cudaMemcpyAsync(resnorm, h->d_hres, sizeof(double) * stride * nh, cudaMemcpyDeviceToHost,
                       st));
  std::vector<DevScalars> ssc(nh);
  CK(cudaMemcpyAsync(ssc.data(), h->nseg ? h->d_segsc : h->d_sc, sizeof(DevScalars) * nh,
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int m = 0; m < nh; m++) {
    if (iters_done) iters_done[m] = ssc[m].done;
    if (flags) flags[m] = ssc[m].flags & 3;
  }
  return SPAI_OK;
}

int spai_mr(spai_handle h, int iters, int drop_rule, spai_history* hist) {
  return spai_run(h, SPAI_MR, iters, drop_rule, hist);
}
int spai_lomr(spai_handle h, int iters, int drop_rule, spai_history* hist) {
  return spai_run(h, SPAI_LOMR, iters, drop_rule, hist);
}
int spai_cg(spai_handle h, int iters, int drop_rule, spai_history* hist) {
  return spai_run(h, SPAI_CG, iters, drop_rule, hist);
}

int spai_residual_norm(spai_handle h, double* out) {
  if (!h || !out) return SPAI_ERR_ARG;
  if (h->nseg) {
    std::vector<double> r(h->nseg);
    int rc = spai_batch_residual_norms(h, r.data());
    if (rc) return rc;
    double s2 = 0.0;
    for (double x : r) s2 += x * x;
    *out = sqrt(s2);
    return SPAI_OK;
  }
  int rc = reset_call_scalars(h);
  if (rc) return rc;
  PassParams p = base_params(h, kRES, true);
  p.do_dir = 0;
  p.hist_res = nullptr;
  p.hist_coef = nullptr;
  CK(timed_launch(h, p, h->cfg[kRES], true));
  DevScalars sc;
  CK(cudaMemcpyAsync(&sc, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) collect_timing(h);
  *out = sqrt(sc.result);
  return SPAI_OK;
}

int spai_batch_residual_norms(spai_handle h, double* out) {
  if (!h || !out) return SPAI_ERR_ARG;
  if (!h->nseg) return spai_residual_norm(h, out);
  int rc = reset_call_scalars(h);
  if (rc) return rc;
  CK(launch_seg_reset(h->d_segsc, h->nseg, 0, h->stream));
  PassParams p = base_params(h, kRES, true);
  p.do_dir = 0;
  p.hist_res = nullptr;
  p.hist_coef = nullptr;
  CK(timed_launch(h, p, h->cfg[kRES], true));
  std::vector<DevScalars> ssc(h->nseg);
  CK(cudaMemcpyAsync(ssc.data(), h->d_segsc, sizeof(DevScalars) * h->nseg, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) collect_timing(h);
  for (int m = 0; m < h->nseg; m++) out[m] = sqrt(ssc[m].result);
  return SPAI_OK;
}

int spai_batch_get_M(spai_handle h, int m, int64_t* nnz, int32_t* colptr, int32_t* rowind,
                     double* vals) {
  if (!h || !nnz) return SPAI_ERR_ARG;
  const int nh = h->nseg ? h->nseg : 1;
  if (m < 0 || m >= nh) return SPAI_ERR_ARG;
  if (!h->nseg) return spai_get_M(h, nnz, colptr, rowind, vals, 0);
  long long tot = 0;
  int rc = export_csc(h, &tot);
  if (rc) return rc;
  const long long c0 = h->seg_col0[m], nm = h->seg_n[m];
  std::vector<long long> cp(nm + 1);
  CK(cudaMemcpyAsync(cp.data(), h->d_ccolptr + c0, sizeof(long long) * (nm + 1),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *nnz = cp[nm] - cp[0];
  if (!colptr) return SPAI_OK;
  if (!rowind || !vals) return SPAI_ERR_ARG;
  CK(cudaMemcpyAsync(rowind, h->d_crow + cp[0], sizeof(int) * (size_t)*nnz, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(vals, h->d_cval + cp[0], sizeof(double) * (size_t)*nnz,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (long long q = 0; q <= nm; q++) colptr[q] = (int32_t)(cp[q] - cp[0]);
  for (long long e = 0; e < *nnz; e++) rowind[e] -= (int32_t)c0;
  return SPAI_OK;
}

int spai_get_nnz(spai_handle h, int64_t* out) {
  if (!h || !out) return SPAI_ERR_ARG;
  long long nnz = 0;
  int rc = export_csc(h, &nnz);
  if (rc) return rc;
  *out = nnz;
  return SPAI_OK;
}

int spai_get_M(spai_handle h, int64_t* nnz, int32_t* colptr, int32_t* rowind, double* vals,
               int on_device) {
  if (!h || !nnz) return SPAI_ERR_ARG;
  long long tot = 0;
  int rc = export_csc(h, &tot);
  if (rc) return rc;
  *nnz = tot;
  if (!colptr) return SPAI_OK;
  if (!rowind || !vals) return SPAI_ERR_ARG;
  const int n = h->n;
  cudaStream_t st = h->stream;
  if (on_device) {
    CK(launch_ll_to_i32(h->d_ccolptr, colptr, n, st));
    CK(cudaMemcpyAsync(rowind, h->d_crow, sizeof(int) * tot, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(vals, h->d_cval, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  } else {
    std::vector<long long> cp(n + 1);
    CK(cudaMemcpyAsync(cp.data(), h->d_ccolptr, sizeof(long long) * (n + 1),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(rowind, h->d_crow, sizeof(int) * tot, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(vals, h->d_cval, sizeof(double) * tot, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i <= n; i++) colptr[i] = (int32_t)cp[i];
  }
  CK(cudaStreamSynchronize(st));
  return SPAI_OK;
}

int spai_set_M(spai_handle h, const int32_t* colptr, const int32_t* rowind, const double* vals,
               int on_device) {
  if (!h || !colptr || !rowind || !vals) return SPAI_ERR_ARG;
  const int n = h->n;
  std::vector<int32_t> cp(n + 1);
  if (on_device) {
    CK(cudaMemcpy(cp.data(), colptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
  } else {
    memcpy(cp.data(), colptr, sizeof(int32_t) * (n + 1));
  }
  long long nnz = cp[n];
  if (cp[0] != 0 || nnz < 0) return SPAI_ERR_CSR;
  std::vector<int32_t> ri(nnz);
  std::vector<double> va(nnz);
  if (on_device) {
    CK(cudaMemcpy(ri.data(), rowind, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(va.data(), vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
  } else {
    memcpy(ri.data(), rowind, sizeof(int32_t) * nnz);
    memcpy(va.data(), vals, sizeof(double) * nnz);
  }
  std::vector<long long> off(n + 1);
  std::vector<int> cap(n);
  CK(cudaMemcpy(off.data(), h->d_off, sizeof(long long) * (n + 1), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(cap.data(), h->d_cap, sizeof(int) * n, cudaMemcpyDeviceToHost));
  std::vector<int> srow(h->slab_total, 0), slen(n, 0);
  std::vector<double> sval(h->slab_total, 0.0);
  for (int j = 0; j < n; j++) {
    if (cp[j + 1] < cp[j]) return SPAI_ERR_CSR;
    int L = 0;
    for (long long e = cp[j]; e < cp[j + 1]; e++) {
      if (ri[e] < 0 || ri[e] >= n) return SPAI_ERR_CSR;
      if (e > cp[j] && ri[e - 1] >= ri[e]) return SPAI_ERR_CSR;
      if (!isfinite(va[e])) return SPAI_ERR_NONFINITE;
      double v = h->prec == SPAI_MIXED ? (double)(float)va[e] : va[e];
      if (v == 0.0) continue;
      if (L >= cap[j]) return SPAI_ERR_CAPACITY;
      srow[off[j] + L] = ri[e];
      sval[off[j] + L] = v;
      L++;
    }
    slen[j] = L;
  }
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(h->d_Mrow, srow.data(), sizeof(int) * h->slab_total, cudaMemcpyHostToDevice, st));
  if (h->prec == SPAI_MIXED) {
    std::vector<float> f(h->slab_total);
    for (long long k = 0; k < h->slab_total; k++) f[k] = (float)sval[k];
    CK(cudaMemcpyAsync(h->d_Mval, f.data(), sizeof(float) * h->slab_total, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    CK(cudaMemcpyAsync(h->d_Mval, sval.data(), sizeof(double) * h->slab_total,
                       cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(h->d_Mlen, slen.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h->d_Plen, 0, sizeof(int) * n, st));
  CK(cudaMemsetAsync(h->d_Zlen, 0, sizeof(int) * n, st));
  CK(cudaStreamSynchronize(st));
  h->method = -1;
  h->it = 0;
  invalidate_rows(h);
  return SPAI_OK;
}

int spai_apply(spai_handle h, const double* x, double* y, int nrhs, int64_t ld) {
  if (!h || !x || !y || nrhs < 1 || ld < h->n) return SPAI_ERR_ARG;
  int rc = ensure_rows(h, false);
  if (rc) return rc;
  CK(launch_apply(h->n, h->d_mrp, h->d_mci, h->d_mv, x, y, nrhs, ld, h->stream));
  h->other_launches++;
  return SPAI_OK;
}

static int ensure_pcg(spai_ctx* h) {
  if (h->d_x) return SPAI_OK;
  const int n = h->n;
  int nb = (n + 255) / 256;
  int ng = (nb + kGroup - 1) / kGroup;
  if (ng > 1024) return SPAI_ERR_UNSUPPORTED;
  int rc = SPAI_OK;
  rc = rc ? rc : dalloc(&h->d_b, n);
  rc = rc ? rc : dalloc(&h->d_x, n);
  rc = rc ? rc : dalloc(&h->d_r, n);
  rc = rc ? rc : dalloc(&h->d_z, n);
  rc = rc ? rc : dalloc(&h->d_p, n);
  rc = rc ? rc : dalloc(&h->d_q, n);
  rc = rc ? rc : dalloc(&h->d_ps, 1);
  rc = rc ? rc : dalloc(&h->d_vbsum, nb);
  rc = rc ? rc : dalloc(&h->d_vrrsum, nb);
  rc = rc ? rc : dalloc(&h->d_vgsum, ng);
  rc = rc ? rc : dalloc(&h->d_vcnt1, ng);
  rc = rc ? rc : dalloc(&h->d_vcnt2, 1);
  const int ns = (n + 31) / 32;
  rc = rc ? rc : dalloc(&h->d_asp, (size_t)ns + 1);
  rc = rc ? rc : dalloc(&h->d_w32, (size_t)ns + 1);
  if (!h->d_scan) rc = rc ? rc : dalloc(&h->d_scan, 2 * (size_t)((n + 1023) / 1024) + 2);
  if (rc) return rc;
  long long tot = 0;
  CK(launch_sell_build_i32(n, h->d_rowptr, h->d_colind, h->d_vals, h->d_w32, h->d_asp, h->d_scan,
                           &h->d_acol, &h->d_aval, &h->a_cap, &tot, h->stream));
  h->other_launches += 5;
  CK(cudaMemsetAsync(h->d_vcnt1, 0, sizeof(unsigned) * ng, h->stream));
  CK(cudaMemsetAsync(h->d_vcnt2, 0, sizeof(unsigned), h->stream));
  return SPAI_OK;
}

// FP32 copies for the mixed PCG products (made on first use; M's and S's
// again after M changes).  block: the ELL values of A and [n][32] operand
// copies instead of the sliced-ELL values and n-vectors.
static int ensure_pcg32(spai_ctx* h, int precond, bool block) {
  cudaStream_t st = h->stream;
  int rc = SPAI_OK;
  if (!block) {
    if (!h->d_aval32) {
      rc = dalloc(&h->d_aval32, (size_t)h->a_cap);
      if (rc) return rc;
      CK(launch_to_f32(h->d_aval, h->d_aval32, h->a_cap, st));
      h->other_launches++;
    }
    if (!h->d_p32) {
      rc = dalloc(&h->d_p32, (size_t)h->n);
      if (!rc) rc = dalloc(&h->d_r32, (size_t)h->n);
      if (rc) return rc;
    }
  } else {
    if (!h->d_ell32) {
      rc = dalloc(&h->d_ell32, (size_t)h->n * h->W);
      if (rc) return rc;
      CK(launch_to_f32(h->d_ell64, h->d_ell32, (long long)h->n * h->W, st));
      h->other_launches++;
    }
    if (!h->d_bp32) {
      rc = dalloc(&h->d_bp32, (size_t)h->n * kBpLd);
      if (!rc) rc = dalloc(&h->d_br32, (size_t)h->n * kBpLd);
      if (rc) return rc;
    }
  }
  if (precond == SPAI_PREC_SPAI && !h->m32_valid) {
    if (h->mt_nnz > h->mv32_cap || !h->d_mv32) {
      dfree(h->d_mv32);
      h->mv32_cap = 0;
      rc = dalloc(&h->d_mv32, (size_t)std::max(h->mt_nnz, 1LL));
      if (rc) return rc;
      h->mv32_cap = std::max(h->mt_nnz, 1LL);
    }
    CK(launch_to_f32(h->d_mv, h->d_mv32, h->mt_nnz, st));
    h->other_launches++;
    h->m32_valid = true;
  }
  if (precond == SPAI_PREC_SPAI_SYM && !h->s32_valid) {
    if (h->sym_nnz > h->sv32_cap || !h->d_sv32) {
      dfree(h->d_sv32);
      h->sv32_cap = 0;
      rc = dalloc(&h->d_sv32, (size_t)std::max(h->sym_nnz, 1LL));
      if (rc) return rc;
      h->sv32_cap = std::max(h->sym_nnz, 1LL);
    }
    CK(launch_to_f32(h->d_sv, h->d_sv32, h->sym_nnz, st));
    h->other_launches++;
    h->s32_valid = true;
  }
  return SPAI_OK;
}

int spai_set_pcg_prec(spai_handle h, int prec) {
  if (!h || (prec != SPAI_FP64 && prec != SPAI_MIXED)) return SPAI_ERR_ARG;
  h->pcg_prec = prec;
  return SPAI_OK;
}

int pcg_solve(spai_handle h, const double* b, double* x, int nrhs, double rtol, int maxit,
              int precond, int on_device, int* iters, double* relres) {
  if (!h || !b || !x || !iters || nrhs != 1 || maxit < 0 || !(rtol >= 0.0)) return SPAI_ERR_ARG;
  if (precond < SPAI_PREC_NONE || precond > SPAI_PREC_SPAI_SYM) return SPAI_ERR_ARG;
  int rc = ensure_pcg(h);
  if (rc) return rc;
  if (precond == SPAI_PREC_SPAI || precond == SPAI_PREC_SPAI_SYM) {
    rc = ensure_rows(h, precond == SPAI_PREC_SPAI_SYM);
    if (rc) return rc;
  }
  const int n = h->n;
  cudaStream_t st = h->stream;
  if (on_device)
    CK(cudaMemcpyAsync(h->d_b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else
    CK(cudaMemcpyAsync(h->d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  PcgScalars ps;
  memset(&ps, 0, sizeof(ps));
  ps.rtol = rtol;
  ps.maxit = maxit;
  CK(cudaMemcpyAsync(h->d_ps, &ps, sizeof(ps), cudaMemcpyHostToDevice, st));
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.A.sptr = h->d_asp;
  a.A.col = h->d_acol;
  a.A.val = h->d_aval;
  a.diag = h->d_diag;
  a.precond = precond;
  if (precond == SPAI_PREC_SPAI) {
    a.mrp = h->d_mrp;
    a.mci = h->d_mci;
    a.mv = h->d_mv;
  } else if (precond == SPAI_PREC_SPAI_SYM) {
    a.mrp = h->d_srp;
    a.mci = h->d_sci;
    a.mv = h->d_sv;
    if (h->pcg_prec != SPAI_MIXED) {
      rc = ensure_sym_sell(h);
      if (rc) return rc;
      a.sell.sptr = h->d_ssp;
      a.sell.col = h->d_sscol;
      a.sell.val = h->d_ssval;
      a.longrows = h->nlong ? h->d_slongs : h->d_slong;
      a.nlong = h->nlong;
      a.sperm = h->nlong ? h->d_sperm : nullptr;
    }
  }
  a.b = h->d_b;
  a.x = h->d_x;
  a.r = h->d_r;
  a.z = h->d_z;
  a.p = h->d_p;
  a.q = h->d_q;
  a.s = h->d_ps;
  if (h->pcg_prec == SPAI_MIXED) {
    rc = ensure_pcg32(h, precond, false);
    if (rc) return rc;
    a.mixed = 1;
    a.aval32 = h->d_aval32;
    a.mv32 = precond == SPAI_PREC_SPAI ? h->d_mv32 : precond == SPAI_PREC_SPAI_SYM ? h->d_sv32 : nullptr;
    a.p32 = h->d_p32;
    a.r32 = h->d_r32;
  }
  a.ws.bsum = h->d_vbsum;
  a.rrsum = h->d_vrrsum;
  a.ws.gsum = h->d_vgsum;
  a.ws.cnt1 = h->d_vcnt1;
  a.ws.cnt2 = h->d_vcnt2;
  a.ws.nb = (n + 255) / 256;
  a.ws.ngroups = (a.ws.nb + kGroup - 1) / kGroup;
  PcgFork fk{nullptr, nullptr, nullptr};
  if (a.nlong) {
    if (!h->pcg_st2) {
      bool ok = cudaStreamCreateWithFlags(&h->pcg_st2, cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&h->pcg_fork, cudaEventDisableTiming) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&h->pcg_join, cudaEventDisableTiming) == cudaSuccess;
      if (!ok) {  // one stream then
        (void)cudaGetLastError();
        if (h->pcg_fork) cudaEventDestroy(h->pcg_fork);
        if (h->pcg_st2) cudaStreamDestroy(h->pcg_st2);
        h->pcg_fork = h->pcg_join = nullptr;
        h->pcg_st2 = nullptr;
      }
    }
    if (h->pcg_st2) fk = PcgFork{h->pcg_st2, h->pcg_fork, h->pcg_join};
  }
  // kernels of one preconditioner application with its inner product: 2, or
  // 3 (long rows, the others, the total), or 4 (long rows beside the others,
  // then the inner product and its total)
  const int prec_launches = !a.nlong ? 2 : fk.st2 ? 4 : 3;
  CK(launch_pcg_init(a, fk, st));
  h->pcg_launches += 2 + prec_launches;
  // the iterations run as replays of a captured graph of `chunk` iterations
  // (their kernels read every scalar from device memory, so the launches do
  // not change while the arguments do not); the host polls the done flag
  // between replays
  const int chunk = 16;
  if (!h->pcg_graph || memcmp(h->pcg_graph_key, &a, sizeof(a)) != 0 ||
      h->pcg_graph_forked != (fk.st2 != nullptr)) {
    if (h->pcg_graph) cudaGraphExecDestroy(h->pcg_graph);
    h->pcg_graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = cudaSuccess;
      for (int c = 0; c < chunk && e == cudaSuccess; c++) e = launch_pcg_iter(a, fk, st);
      cudaError_t e2 = cudaStreamEndCapture(st, &g);
      if (e == cudaSuccess && e2 == cudaSuccess && g)
        if (cudaGraphInstantiate(&h->pcg_graph, g, 0) != cudaSuccess) h->pcg_graph = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    (void)cudaGetLastError();
    if (h->pcg_graph) memcpy(h->pcg_graph_key, &a, sizeof(a));
    h->pcg_graph_forked = fk.st2 != nullptr;
  }
  for (;;) {
    if (h->pcg_graph) {
      CK(cudaGraphLaunch(h->pcg_graph, st));
    } else {
      for (int c = 0; c < chunk; c++) CK(launch_pcg_iter(a, fk, st));
    }
    h->pcg_launches += (4 + prec_launches) * chunk;
    CK(cudaMemcpyAsync(&ps, h->d_ps, sizeof(ps), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ps.done) break;
  }
  CK(launch_true_res(a, st));
  h->pcg_launches += 1;
  CK(cudaMemcpyAsync(&ps, h->d_ps, sizeof(ps), cudaMemcpyDeviceToHost, st));
  if (on_device)
    CK(cudaMemcpyAsync(x, h->d_x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else
    CK(cudaMemcpyAsync(x, h->d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *iters = ps.k;
  if (relres) *relres = ps.bn > 0 ? sqrt(ps.tres) / ps.bn : 0.0;
  if (ps.status == 1) return SPAI_PCG_MAXIT;
  if (ps.status == 2) return SPAI_PCG_BREAKDOWN;
  return SPAI_OK;
}

// ------------------------------------------------------- diagnostics

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..k) and off-diagonal b[0..k-1) (Sturm sequence of the LDL^T
// pivots; a zero pivot is replaced by a tiny negative one).
static int sturm_count(const double* a, const double* b, int k, double x) {
  int c = 0;
  double q = 1.0;
  for (int i = 0; i < k; i++) {
    q = (a[i] - x) - (i ? (b[i - 1] * b[i - 1]) / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) c++;
  }
  return c;
}

// Smallest and largest eigenvalue of that tridiagonal matrix by bisection
// inside its Gershgorin interval, to the last bit.
static void tri_extremes(const double* a, const double* b, int k, double* lmin, double* lmax) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; i++) {
    double r = (i ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int which = 0; which < 2; which++) {
    double l = lo, u = hi;
    const int need = which == 0 ? 1 : k;  // count(x) >= need means x is past the eigenvalue
    for (int it = 0; it < 2100; it++) {
      double m = 0.5 * (l + u);
      if (m <= l || m >= u) break;
      if (sturm_count(a, b, k, m) >= need) u = m;
      else l = m;
    }
    (which == 0 ? *lmin : *lmax) = 0.5 * (l + u);
  }
}

int spai_sym_lanczos(spai_handle h, int steps, const double* v0, double* alpha, double* beta,
                     int* steps_done, double* lmin, double* lmax) {
  if (!h || steps < 1 || !v0 || !steps_done) return SPAI_ERR_ARG;
  if (h->nseg) return SPAI_ERR_UNSUPPORTED;
  const int n = h->n;
  bool nonzero = false;
  for (int i = 0; i < n; i++) {
    if (!std::isfinite(v0[i])) return SPAI_ERR_ARG;
    nonzero |= v0[i] != 0.0;
  }
  if (!nonzero) return SPAI_ERR_ARG;
  int rc = ensure_pcg(h);
  if (rc) return rc;
  rc = ensure_rows(h, true);
  if (rc) return rc;
  double* d_ab = nullptr;
  int* d_st = nullptr;
  rc = dalloc(&d_ab, 2 * (size_t)steps + 1);
  if (!rc) rc = dalloc(&d_st, 2);
  if (rc) {
    dfree(d_ab);
    return rc;
  }
  cudaStream_t st = h->stream;
  LzArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.rp = h->d_srp;
  a.ci = h->d_sci;
  a.v = h->d_sv;
  a.vp = h->d_x;
  a.vc = h->d_r;
  a.w = h->d_z;
  a.alpha = d_ab;
  a.beta = d_ab + steps;
  a.nrm0 = d_ab + 2 * steps;
  a.state = d_st;
  a.ws.bsum = h->d_vbsum;
  a.ws.gsum = h->d_vgsum;
  a.ws.cnt1 = h->d_vcnt1;
  a.ws.cnt2 = h->d_vcnt2;
  a.ws.nb = (n + 255) / 256;
  a.ws.ngroups = (a.ws.nb + kGroup - 1) / kGroup;
  std::vector<double> ab(2 * (size_t)steps);
  int stt[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h->d_r, v0, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (!e) e = launch_lz_start(a, st);
  for (int j = 0; j < steps && !e; j++) e = launch_lz_step(a, j, st);
  h->other_launches += 2 + 3LL * steps;
  if (!e) e = cudaMemcpyAsync(ab.data(), d_ab, sizeof(double) * 2 * steps, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaMemcpyAsync(stt, d_st, sizeof(stt), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(d_ab);
  dfree(d_st);
  if (e) {
    (void)cudaGetLastError();
    return SPAI_ERR_CUDA;
  }
  const int k = stt[0];
  *steps_done = k;
  if (alpha) for (int j = 0; j < k; j++) alpha[j] = ab[j];
  if (beta) for (int j = 0; j < k; j++) beta[j] = ab[steps + j];
  if (k == 0) return SPAI_ERR_NONFINITE;
  double l0 = 0.0, l1 = 0.0;
  tri_extremes(ab.data(), ab.data() + steps, k, &l0, &l1);
  if (lmin) *lmin = l0;
  if (lmax) *lmax = l1;
  return SPAI_OK;
}

int spai_fixed_pattern(spai_handle h, int k) {
  if (!h || k < 0) return SPAI_ERR_ARG;
  const int n = h->n;
  cudaStream_t st = h->stream;
  // pattern supp(A^k e_j) by breadth-first search on A's (symmetric) graph
  std::vector<int> rp(n + 1), ci(h->nnz), cap(n);
  CK(cudaMemcpyAsync(rp.data(), h->d_rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ci.data(), h->d_colind, sizeof(int) * h->nnz, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(cap.data(), h->d_cap, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<long long> pptr(n + 1, 0);
  std::vector<int> prow;
  std::vector<int> mark(n, -1), front, next;
  int Lmax = 1;
  for (int j = 0; j < n; j++) {
    const size_t start = prow.size();
    prow.push_back(j);
    mark[j] = j;
    front.assign(1, j);
    for (int lev = 0; lev < k && !front.empty(); lev++) {
      next.clear();
      for (int u : front)
        for (int e = rp[u]; e < rp[u + 1]; e++) {
          const int c = ci[e];
          if (mark[c] != j) {
            mark[c] = j;
            next.push_back(c);
            prow.push_back(c);
          }
        }
      front.swap(next);
    }
    std::sort(prow.begin() + start, prow.end());
    const int L = (int)(prow.size() - start);
    if (L > cap[j]) return SPAI_ERR_CAPACITY;
    Lmax = std::max(Lmax, L);
    pptr[j + 1] = (long long)prow.size();
  }
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem_max <= 0) smem_max = 227 * 1024;
  const int wb = align16(8 * Lmax * Lmax + 8 * Lmax + 4 * Lmax);
  const int nw = std::min(8, smem_max / wb);
  if (nw < 1) return SPAI_ERR_UNSUPPORTED;
  long long* d_pptr = nullptr;
  int *d_prow = nullptr, *d_err = nullptr;
  int rc = dalloc(&d_pptr, (size_t)n + 1);
  if (!rc) rc = dalloc(&d_prow, prow.size());
  if (!rc) rc = dalloc(&d_err, 1);
  if (rc) {
    dfree(d_pptr);
    dfree(d_prow);
    return rc;
  }
  FpArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.W = h->W;
  a.ell_col = h->d_ell_col;
  a.ell_val = h->d_ell64;
  a.pptr = d_pptr;
  a.prow = d_prow;
  a.off = h->d_off;
  a.Mrow = h->d_Mrow;
  a.Mval = h->d_Mval;
  a.Mlen = h->d_Mlen;
  a.Lmax = Lmax;
  a.warp_bytes = wb;
  a.err = d_err;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(d_pptr, pptr.data(), sizeof(long long) * (n + 1),
                                  cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(d_prow, prow.data(), sizeof(int) * prow.size(), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (!e) e = launch_fixed_pattern(a, h->prec == SPAI_MIXED ? 4 : 8, nw, st);
  if (!e) e = cudaMemsetAsync(h->d_Plen, 0, sizeof(int) * n, st);
  if (!e) e = cudaMemsetAsync(h->d_Zlen, 0, sizeof(int) * n, st);
  if (!e) e = cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  h->other_launches += 1;
  dfree(d_pptr);
  dfree(d_prow);
  dfree(d_err);
  if (e) {
    (void)cudaGetLastError();
    return SPAI_ERR_CUDA;
  }
  h->method = -1;
  h->it = 0;
  invalidate_rows(h);
  return err ? SPAI_ERR_NONFINITE : SPAI_OK;
}

// ------------------------------------------------------ global dropping

// Histogram of one 16-bit digit of the selection keys (see dropping.cu)
static int sel_hist(spai_ctx* h, SelArgs& a, std::vector<unsigned>& hh) {
  CK(cudaMemsetAsync(h->d_hist, 0, sizeof(unsigned) * 65536, h->stream));
  CK(launch_sel_hist(a, h->stream));
  h->other_launches++;
  CK(cudaMemcpyAsync(hh.data(), h->d_hist, sizeof(unsigned) * 65536, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SPAI_OK;
}

// t-th smallest (1-based) key of the current stage; *less = keys below it
static int sel_select(spai_ctx* h, SelArgs& a, long long t, unsigned long long* key,
                      long long* less) {
  std::vector<unsigned> hh(65536);
  a.prefix = 0;
  a.mask = 0;
  long long rem = t, below = 0;
  for (int d = 0; d < 4; d++) {
    a.shift = 48 - 16 * d;
    int rc = sel_hist(h, a, hh);
    if (rc) return rc;
    long long acc = 0;
    int bucket = -1;
    for (int b = 0; b < 65536; b++) {
      if (acc + hh[b] >= rem) {
        bucket = b;
        break;
      }
      acc += hh[b];
    }
    if (bucket < 0) return SPAI_ERR_STATE;
    rem -= acc;
    below += acc;
    a.prefix |= (unsigned long long)bucket << a.shift;
    a.mask |= 0xffffull << a.shift;
  }
  *key = a.prefix;
  *less = below;
  return SPAI_OK;
}

// Select the t first entries by (key, position) and keep (keep_selected) or
// drop them, in place
static int select_and_compact(spai_ctx* h, SelArgs& a, long long t, int keep_selected) {
  if (!h->d_hist) {
    int rc = dalloc(&h->d_hist, 65536);
    if (rc) return rc;
  }
  unsigned long long ustar = 0, pstar = 0;
  long long less = 0, less2 = 0;
  a.stage = 0;
  int rc = sel_select(h, a, t, &ustar, &less);
  if (rc) return rc;
  a.stage = 1;
  a.ustar = ustar;
  rc = sel_select(h, a, t - less, &pstar, &less2);
  if (rc) return rc;
  a.pstar = pstar;
  a.keep_selected = keep_selected;
  CK(launch_sel_compact(a, h->stream));
  h->other_launches++;
  CK(cudaStreamSynchronize(h->stream));
  return SPAI_OK;
}

static long long count_entries(spai_ctx* h, const int* d_len) {
  std::vector<int> l(h->n);
  if (cudaMemcpyAsync(l.data(), d_len, sizeof(int) * h->n, cudaMemcpyDeviceToHost, h->stream) ||
      cudaStreamSynchronize(h->stream)) {
    (void)cudaGetLastError();
    return -1;
  }
  long long s = 0;
  for (int x : l) s += x;
  return s;
}

// which: 0 = M, 1 = P, 2 = Z (LOMR's residual direction, internal)
static int drop_global_impl(spai_ctx* h, int which, int64_t m) {
  int* len = which == 0 ? h->d_Mlen : which == 1 ? h->d_Plen : h->d_Zlen;
  const long long N = count_entries(h, len);
  if (N < 0) return SPAI_ERR_CUDA;
  if (N > m) {
    SelArgs a;
    memset(&a, 0, sizeof(a));
    a.n = h->n;
    a.off = h->d_off;
    a.len = len;
    a.rows = which == 0 ? h->d_Mrow : which == 1 ? h->d_Prow : h->d_Zrow;
    a.vals = which == 0 ? h->d_Mval : which == 1 ? h->d_Pval : h->d_Zval;
    a.vs = h->prec == SPAI_MIXED ? 4 : 8;
    a.mode = 0;
    a.hist = nullptr;
    if (!h->d_hist) {
      int rc = dalloc(&h->d_hist, 65536);
      if (rc) return rc;
    }
    a.hist = h->d_hist;
    if (m == 0) {
      CK(cudaMemsetAsync(len, 0, sizeof(int) * h->n, h->stream));
    } else {
      int rc = select_and_compact(h, a, m, 1);
      if (rc) return rc;
    }
  }
  invalidate_rows(h);
  return SPAI_OK;
}

int spai_drop_global(spai_handle h, int which, int64_t m) {
  if (!h || (which != 0 && which != 1) || m < 0) return SPAI_ERR_ARG;
  if (h->nseg) return SPAI_ERR_UNSUPPORTED;
  h->method = -1;
  return drop_global_impl(h, which, m);
}

static int drop_heuristic_impl(spai_ctx* h, int64_t m) {
  cudaStream_t st = h->stream;
  const int vs = h->prec == SPAI_MIXED ? 4 : 8;
  // 1-2: M := (M + M^T)/2 in FP64, rounded to the value type; off-diagonal
  // entries below the unit round-off dropped
  int rc = ensure_rows(h, true);
  if (rc) return rc;
  int* d_ovf = nullptr;
  rc = dalloc(&d_ovf, 1);
  if (rc) return rc;
  int ovf = 0;
  cudaError_t e = cudaMemsetAsync(d_ovf, 0, sizeof(int), st);
  if (!e) e = launch_sym_to_slab(h->n, h->d_srp, h->d_sci, h->d_sv, h->d_off, h->d_cap, h->d_Mrow,
                                 h->d_Mval, h->d_Mlen, vs, vs == 4 ? 0x1p-24 : 0x1p-53, d_ovf, st);
  if (!e) e = cudaMemcpyAsync(&ovf, d_ovf, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(d_ovf);
  h->other_launches++;
  h->method = -1;
  invalidate_rows(h);
  if (e) {
    (void)cudaGetLastError();
    return SPAI_ERR_CUDA;
  }
  if (ovf) return SPAI_ERR_CAPACITY;
  const long long N = count_entries(h, h->d_Mlen);
  if (N < 0) return SPAI_ERR_CUDA;
  if (N <= m) return SPAI_OK;
  // 3: scores m^2 ||A e_k||^2 + 2 m (A R)_kl of the off-diagonal entries
  if (!h->d_anrm) {
    rc = dalloc(&h->d_anrm, h->n);
    if (!rc) rc = dalloc(&h->d_score, (size_t)h->slab_total);
    if (rc) return rc;
    CK(launch_anrm(h->n, h->W, h->d_ell_col, vs == 4 ? (const void*)h->d_ell32 : (const void*)h->d_ell64,
                   vs, h->d_anrm, st));
    h->other_launches++;
  }
  rc = reset_call_scalars(h);
  if (rc) return rc;
  PassParams p = base_params(h, kRES, false);
  p.kind = kSCORE;
  p.do_dir = 0;
  p.hist_res = nullptr;
  p.hist_coef = nullptr;
  p.score = h->d_score;
  p.anrm = h->d_anrm;
  CK(timed_launch(h, p, h->cfg[kRES], false));
  SelArgs a;
  memset(&a, 0, sizeof(a));
  a.n = h->n;
  a.off = h->d_off;
  a.len = h->d_Mlen;
  a.rows = h->d_Mrow;
  a.vals = h->d_Mval;
  a.vs = vs;
  a.score = h->d_score;
  a.mode = 1;
  if (!h->d_hist) {
    rc = dalloc(&h->d_hist, 65536);
    if (rc) return rc;
  }
  a.hist = h->d_hist;
  // eligible (off-diagonal) entries: the first digit's histogram total
  std::vector<unsigned> hh(65536);
  a.stage = 0;
  a.prefix = 0;
  a.mask = 0;
  a.shift = 48;
  rc = sel_hist(h, a, hh);
  if (rc) return rc;
  long long E = 0;
  for (unsigned x : hh) E += x;
  const long long D = std::min(N - (long long)m, E);
  if (D > 0) {
    rc = select_and_compact(h, a, D, 0);
    if (rc) return rc;
  }
  invalidate_rows(h);
  return SPAI_OK;
}

int spai_drop_heuristic(spai_handle h, int64_t m) {
  if (!h || m < 0) return SPAI_ERR_ARG;
  if (h->nseg) return SPAI_ERR_UNSUPPORTED;
  h->method = -1;
  return drop_heuristic_impl(h, m);
}

int spai_run_global(spai_handle h, int method, int iters, int64_t m_dir, int64_t m_M,
                    spai_history* hist) {
  if (!h || iters < 0 || m_dir < 0 || m_M < 0) return SPAI_ERR_ARG;
  if (method < SPAI_MR || method > SPAI_CG_PI) return SPAI_ERR_ARG;
  if (h->nseg) return SPAI_ERR_UNSUPPORTED;
  const bool pim = method >= SPAI_MR_PI;
  if (pim && !h->pi_ok) return SPAI_ERR_UNSUPPORTED;
  const int base = pim ? method - SPAI_MR_PI : method;
  int rc = ensure_hist(h, iters + 1);
  if (rc) return rc;
  h->last_iters = iters;
  cudaStream_t st = h->stream;
  CK(cudaMemsetAsync(h->d_Plen, 0, sizeof(int) * h->n, st));
  CK(cudaMemsetAsync(h->d_Zlen, 0, sizeof(int) * h->n, st));
  CK(cudaMemsetAsync((char*)h->d_sc + offsetof(DevScalars, beta), 0, sizeof(double), st));
  CK(cudaMemsetAsync((char*)h->d_sc + offsetof(DevScalars, rr), 0, sizeof(double), st));
  rc = reset_call_scalars(h);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->d_hres, 0xff, sizeof(double) * (iters + 1), st));
  CK(cudaMemsetAsync(h->d_hcoef, 0xff, sizeof(double) * 2 * std::max(iters, 1), st));
  h->method = -1;
  invalidate_rows(h);
  // one column pass, no per-column dropping (drop = 0: columns are kept whole)
  auto pass = [&](int kind, int upd, int dir, int iter, int from_slab, int store, int fresh) -> int {
    PassParams p = base_params(h, kind, false, pim);
    p.do_update = upd;
    p.do_dir = dir;
    p.drop = 0;
    p.iter = iter;
    p.fresh = fresh;
    p.dir_from_slab = from_slab;
    p.dir_store = store;
    CK(timed_launch(h, p, pim ? h->cfg_pi[kind] : h->cfg[kind], false));
    invalidate_rows(h);
    return SPAI_OK;
  };
  DevScalars sc;
  memset(&sc, 0, sizeof(sc));
  auto read_sc = [&]() -> int {
    CK(cudaMemcpyAsync(&sc, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SPAI_OK;
  };
  auto halted = [&]() { return (sc.flags & (kFlagCapacity | kFlagNonfinite)) || sc.stop; };
  int i = 0;
  if (base == SPAI_MR) {
    for (; i < iters; i++) {
      // R_i and the direction candidate (Pi) R_i, kept whole
      if ((rc = pass(kMR, 0, 0, i, 0, 1, 0)) || (rc = read_sc())) return rc;
      if (halted()) break;
      // P_i: the m_dir largest entries over the whole matrix (Sec. 6.1)
      if ((rc = drop_global_impl(h, 1, m_dir))) return rc;
      // alpha_i from that P_i
      if ((rc = pass(kMR, 0, 1, i, 1, 0, 0)) || (rc = read_sc())) return rc;
      if (halted()) break;
      // M_i + alpha_i P_i, whole, then the Appendix A heuristic with cap m_M
      if ((rc = pass(kMR, 1, 0, i + 1, 0, 0, 0)) || (rc = read_sc())) return rc;
      if (sc.flags & kFlagCapacity) break;
      if ((rc = drop_heuristic_impl(h, m_M))) return rc;
    }
  } else if (base == SPAI_LOMR) {
    for (; i < iters; i++) {
      // R_i and the candidate Z_i = (Pi) R_i, whole
      if ((rc = pass(kLOMR, 0, 0, i, 0, 1, 0)) || (rc = read_sc())) return rc;
      if (halted()) break;
      if ((rc = drop_global_impl(h, 2, m_dir))) return rc;
      // delta_i, gamma_i from that Z_i and P_{i-1} (Theorem 3)
      if ((rc = pass(kLOMR, 0, 1, i, 1, 0, 0)) || (rc = read_sc())) return rc;
      if (halted()) break;
      // S_i = delta Z_i + gamma P_{i-1}; P_i = S_i and M_i + S_i, whole
      if ((rc = pass(kLOMR, 1, 0, i + 1, 0, 0, 0)) || (rc = read_sc())) return rc;
      if (sc.flags & kFlagCapacity) break;
      if ((rc = drop_global_impl(h, 1, m_dir))) return rc;
      if ((rc = drop_heuristic_impl(h, m_M))) return rc;
    }
  } else {
    while (i < iters) {
      // the candidate (Pi) R_i + beta_{i-1} P_{i-1} (P_{-1} = 0), whole
      if ((rc = pass(kCGB, 0, 0, i, 0, 0, 0)) || (rc = read_sc())) return rc;
      if (halted()) break;
      if ((rc = drop_global_impl(h, 1, m_dir))) return rc;
      // alpha_i from that P_i
      if ((rc = pass(kCGB, 0, 1, i, 1, 0, i == 0)) || (rc = read_sc())) return rc;
      if (halted()) break;
      // M_i + alpha_i P_i, whole, then the heuristic; R_{i+1} and beta_i after it
      if ((rc = pass(kCGA, 1, 0, i, 0, 0, 0)) || (rc = read_sc())) return rc;
      if (sc.flags & kFlagCapacity) break;
      if ((rc = drop_heuristic_impl(h, m_M))) return rc;
      if ((rc = pass(kCGA, 0, 1, i, 0, 0, 0)) || (rc = read_sc())) return rc;
      if (sc.flags & kFlagNonfinite) break;
      i++;
      if (sc.stop) break;
    }
  }
  // MR and LOMR end with the norm of the last M; CG's last pass A recorded
  // it, except when no iteration was asked for
  if ((base != SPAI_CG || iters == 0) && i == iters && !(sc.flags & kFlagCapacity)) {
    const int f0 = sc.flags;
    rc = reset_call_scalars(h);  // clear stop for the final norm
    if (rc) return rc;
    if ((rc = pass(base == SPAI_LOMR ? kLOMR : kMR, 0, 0, iters, 0, 0, 0)) || (rc = read_sc()))
      return rc;
    sc.flags |= f0;
  }
  if (hist && hist->resnorm)
    CK(cudaMemcpyAsync(hist->resnorm, h->d_hres, sizeof(double) * (iters + 1),
                       cudaMemcpyDeviceToHost, st));
  if (hist && hist->coef && iters > 0)
    CK(cudaMemcpyAsync(hist->coef, h->d_hcoef, sizeof(double) * 2 * iters, cudaMemcpyDeviceToHost,
                       st));
  CK(cudaStreamSynchronize(st));
  if (hist) {
    hist->iters_done = i;
    hist->flags = sc.flags & 3;
  }
  invalidate_rows(h);
  h->method = -1;
  if (sc.flags & kFlagCapacity) return SPAI_ERR_CAPACITY;
  if (sc.flags & kFlagNonfinite) return SPAI_ERR_NONFINITE;
  if (sc.flags & kFlagConverged) return SPAI_CONVERGED_EARLY;
  return SPAI_OK;
}

// ------------------------------------------------------------ block PCG

static void free_bpcg(spai_ctx* h) {
  dfree(h->d_bb);
  dfree(h->d_bx);
  dfree(h->d_br);
  dfree(h->d_bz);
  dfree(h->d_bp);
  dfree(h->d_bq);
  dfree(h->d_bstate);
  dfree(h->d_bistate);
  dfree(h->d_bseg_live);
  dfree(h->d_blive);
  dfree(h->d_bbsum);
  dfree(h->d_bcnt);
  dfree(h->d_bseg_of_cta);
  dfree(h->d_bseg_cta0);
  dfree(h->d_bseg_ncta);
  dfree(h->d_bseg_row0);
  dfree(h->d_bseg_n);
  dfree(h->d_bseg_boff);
}

// Block vectors [n][32], per-(matrix, rhs) state and the segment maps, on
// first use.  A single-matrix handle is one segment of ceil(n / 256) CTAs.
static int ensure_bpcg(spai_ctx* h) {
  if (h->d_bb) return SPAI_OK;
  const long long n = h->n;
  const int nseg = std::max(h->nseg, 1);
  const int ncta = (int)((n + kBpRows - 1) / kBpRows);
  std::vector<int> soc(ncta, 0), c0(nseg), nc(nseg), r0(nseg), nn(nseg);
  if (h->nseg) {
    for (int m = 0; m < nseg; m++) {
      c0[m] = (int)(h->seg_col0[m] / kBpRows);
      nc[m] = (int)(h->seg_npad[m] / kBpRows);
      r0[m] = (int)h->seg_col0[m];
      nn[m] = (int)h->seg_n[m];
      for (int c = 0; c < nc[m]; c++) soc[c0[m] + c] = m;
    }
  } else {
    c0[0] = 0;
    nc[0] = ncta;
    r0[0] = 0;
    nn[0] = (int)n;
  }
  // the last-arriving CTA sums at most 8 x 2048 CTA partials per segment
  for (int m = 0; m < nseg; m++)
    if (nc[m] > 16384) return SPAI_ERR_UNSUPPORTED;
  const size_t V = (size_t)n * kBpLd, S = (size_t)nseg * kBpLd;
  int rc = SPAI_OK;
  rc = rc ? rc : dalloc(&h->d_bb, V);
  rc = rc ? rc : dalloc(&h->d_bx, V);
  rc = rc ? rc : dalloc(&h->d_br, V);
  rc = rc ? rc : dalloc(&h->d_bz, V);
  rc = rc ? rc : dalloc(&h->d_bp, V);
  rc = rc ? rc : dalloc(&h->d_bq, V);
  rc = rc ? rc : dalloc(&h->d_bstate, 5 * S);
  rc = rc ? rc : dalloc(&h->d_bistate, 3 * S);
  rc = rc ? rc : dalloc(&h->d_bseg_live, nseg);
  rc = rc ? rc : dalloc(&h->d_blive, 1);
  rc = rc ? rc : dalloc(&h->d_bbsum, (size_t)ncta * kBpLd);
  rc = rc ? rc : dalloc(&h->d_bcnt, nseg);
  rc = rc ? rc : dalloc(&h->d_bseg_of_cta, ncta);
  rc = rc ? rc : dalloc(&h->d_bseg_cta0, nseg);
  rc = rc ? rc : dalloc(&h->d_bseg_ncta, nseg);
  rc = rc ? rc : dalloc(&h->d_bseg_row0, nseg);
  rc = rc ? rc : dalloc(&h->d_bseg_n, nseg);
  rc = rc ? rc : dalloc(&h->d_bseg_boff, nseg);
  if (rc) {
    free_bpcg(h);
    return rc;
  }
  cudaStream_t st = h->stream;
  bool ok = true;
  ok &= cudaMemcpyAsync(h->d_bseg_of_cta, soc.data(), sizeof(int) * ncta, cudaMemcpyHostToDevice,
                        st) == cudaSuccess;
  ok &= cudaMemcpyAsync(h->d_bseg_cta0, c0.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice,
                        st) == cudaSuccess;
  ok &= cudaMemcpyAsync(h->d_bseg_ncta, nc.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice,
                        st) == cudaSuccess;
  ok &= cudaMemcpyAsync(h->d_bseg_row0, r0.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice,
                        st) == cudaSuccess;
  ok &= cudaMemcpyAsync(h->d_bseg_n, nn.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice,
                        st) == cudaSuccess;
  ok &= cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    free_bpcg(h);
    return SPAI_ERR_CUDA;
  }
  return SPAI_OK;
}

int pcg_solve_block(spai_handle h, int nrhs, const double* b, double* x, double rtol, int maxit,
                    int precond, int on_device, int* iters, int* status, double* relres) {
  if (!h || !b || !x || !iters || !status || nrhs < 1 || nrhs > kBpLd || maxit < 0 ||
      !(rtol >= 0.0))
    return SPAI_ERR_ARG;
  if (precond < SPAI_PREC_NONE || precond > SPAI_PREC_SPAI_SYM) return SPAI_ERR_ARG;
  int rc = ensure_bpcg(h);
  if (rc) return rc;
  if (precond == SPAI_PREC_SPAI || precond == SPAI_PREC_SPAI_SYM) {
    rc = ensure_rows(h, precond == SPAI_PREC_SPAI_SYM);
    if (rc) return rc;
  }
  const int nseg = std::max(h->nseg, 1);
  std::vector<long long> boff(nseg);
  long long tot = 0;
  for (int m = 0; m < nseg; m++) {
    boff[m] = tot;
    tot += (long long)nrhs * (h->nseg ? h->seg_n[m] : h->n);
  }
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(h->d_bseg_boff, boff.data(), sizeof(long long) * nseg, cudaMemcpyHostToDevice,
                     st));
  const double* ub = b;
  double* ux = x;
  if (!on_device) {
    if (tot > h->bstage_cap) {
      dfree(h->d_bstage);
      h->bstage_cap = 0;
      rc = dalloc(&h->d_bstage, (size_t)tot);
      if (rc) return rc;
      h->bstage_cap = tot;
    }
    CK(cudaMemcpyAsync(h->d_bstage, b, sizeof(double) * tot, cudaMemcpyHostToDevice, st));
    ub = h->d_bstage;
    ux = h->d_bstage;  // reused for the result once b is gathered
  }
  const int n = h->n;
  CK(launch_bp_gather(ub, h->d_bb, n, nrhs, h->d_bseg_of_cta, h->d_bseg_row0, h->d_bseg_n,
                      h->d_bseg_boff, st));
  BpcgArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.R = nrhs;
  a.W = h->W;
  a.ell_col = h->d_ell_col;
  a.ell_val = h->d_ell64;
  a.diag = h->d_diag;
  a.precond = precond;
  if (precond == SPAI_PREC_SPAI) {
    a.mrp = h->d_mrp;
    a.mci = h->d_mci;
    a.mv = h->d_mv;
  } else if (precond == SPAI_PREC_SPAI_SYM) {
    a.mrp = h->d_srp;
    a.mci = h->d_sci;
    a.mv = h->d_sv;
  }
  a.rtol = rtol;
  a.maxit = maxit;
  a.b = h->d_bb;
  a.x = h->d_bx;
  a.r = h->d_br;
  a.z = h->d_bz;
  a.p = h->d_bp;
  a.q = h->d_bq;
  a.seg_of_cta = h->d_bseg_of_cta;
  a.seg_cta0 = h->d_bseg_cta0;
  a.seg_ncta = h->d_bseg_ncta;
  const size_t S = (size_t)nseg * kBpLd;
  a.rho = h->d_bstate;
  a.alpha = h->d_bstate + S;
  a.beta = h->d_bstate + 2 * S;
  a.bn = h->d_bstate + 3 * S;
  a.tres = h->d_bstate + 4 * S;
  a.k = h->d_bistate;
  a.done = h->d_bistate + S;
  a.status = h->d_bistate + 2 * S;
  a.seg_live = h->d_bseg_live;
  a.live = h->d_blive;
  a.bsum = h->d_bbsum;
  a.cnt = h->d_bcnt;
  if (h->pcg_prec == SPAI_MIXED) {
    rc = ensure_pcg32(h, precond, true);
    if (rc) return rc;
    a.mixed = 1;
    a.ell_val32 = h->d_ell32;
    a.mv32 = precond == SPAI_PREC_SPAI ? h->d_mv32 : precond == SPAI_PREC_SPAI_SYM ? h->d_sv32 : nullptr;
    a.p32 = h->d_bp32;
    a.r32 = h->d_br32;
  }
  CK(launch_bp_setup(a, nseg, st));
  CK(launch_bp_init(a, st));
  h->other_launches += 2;
  h->pcg_launches += 3;
  // the iterations run as replays of a captured graph of `chunk` iterations;
  // the host polls the number of running recurrences between replays
  const int chunk = 8;
  if (!h->bp_graph || memcmp(h->bp_graph_key, &a, sizeof(a)) != 0) {
    if (h->bp_graph) cudaGraphExecDestroy(h->bp_graph);
    h->bp_graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = cudaSuccess;
      for (int c = 0; c < chunk && e == cudaSuccess; c++) e = launch_bp_iter(a, st);
      cudaError_t e2 = cudaStreamEndCapture(st, &g);
      if (e == cudaSuccess && e2 == cudaSuccess && g)
        if (cudaGraphInstantiate(&h->bp_graph, g, 0) != cudaSuccess) h->bp_graph = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    (void)cudaGetLastError();
    if (h->bp_graph) memcpy(h->bp_graph_key, &a, sizeof(a));
  }
  const int reps = maxit / chunk + 2;
  int live = 0;
  for (int rep = 0; rep < reps; rep++) {
    if (h->bp_graph) {
      CK(cudaGraphLaunch(h->bp_graph, st));
    } else {
      for (int c = 0; c < chunk; c++) CK(launch_bp_iter(a, st));
    }
    h->pcg_launches += 4 * chunk;
    CK(cudaMemcpyAsync(&live, h->d_blive, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (live == 0) break;
  }
  CK(launch_bp_tres(a, st));
  h->pcg_launches += 1;
  CK(launch_bp_scatter(h->d_bx, ux, n, nrhs, h->d_bseg_of_cta, h->d_bseg_row0, h->d_bseg_n,
                       h->d_bseg_boff, st));
  h->other_launches += 2;
  if (!on_device)
    CK(cudaMemcpyAsync(x, h->d_bstage, sizeof(double) * tot, cudaMemcpyDeviceToHost, st));
  std::vector<double> dst(5 * S);
  std::vector<int> ist(3 * S);
  CK(cudaMemcpyAsync(dst.data(), h->d_bstate, sizeof(double) * 5 * S, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ist.data(), h->d_bistate, sizeof(int) * 3 * S, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (live != 0) return SPAI_ERR_STATE;  // cannot happen: every recurrence stops by maxit
  bool brk = false, lim = false;
  for (int m = 0; m < nseg; m++)
    for (int j = 0; j < nrhs; j++) {
      const size_t s = (size_t)m * kBpLd + j;
      const int o = m * nrhs + j;
      iters[o] = ist[s];
      const int code = ist[2 * S + s];
      status[o] = code == 0 ? SPAI_OK : code == 1 ? SPAI_PCG_MAXIT : SPAI_PCG_BREAKDOWN;
      brk |= code == 2;
      lim |= code == 1;
      if (relres) {
        const double bn = dst[3 * S + s];
        relres[o] = bn > 0 ? sqrt(dst[4 * S + s]) / bn : 0.0;
      }
    }
  return brk ? SPAI_PCG_BREAKDOWN : lim ? SPAI_PCG_MAXIT : SPAI_OK;
}

// ------------------------------------------------------------ checkpoint

namespace {
struct StateHeader {
  char magic[8];
  int64_t n, slab_total;
  int32_t prec, capmax, method, it, W, pad;
  double cap_factor;
};
}  // namespace

int spai_save_state(spai_handle h, void* buf, size_t* bytes) {
  if (!h || !bytes) return SPAI_ERR_ARG;
  const size_t vs = h->prec == SPAI_MIXED ? 4 : 8;
  const size_t n = h->n, S = h->slab_total;
  size_t need = sizeof(StateHeader) + sizeof(DevScalars) + 3 * n * 4 + 3 * S * 4 + 3 * S * vs;
  if (!buf) {
    *bytes = need;
    return SPAI_OK;
  }
  if (*bytes < need) return SPAI_ERR_ARG;
  char* o = (char*)buf;
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "SPAIST01", 8);
  hd.n = h->n;
  hd.slab_total = h->slab_total;
  hd.prec = h->prec;
  hd.capmax = h->capmax;
  hd.method = h->method;
  hd.it = h->it;
  hd.W = h->W;
  hd.cap_factor = h->cap_factor;
  memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(o, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
  o += sizeof(DevScalars);
  int* lens[3] = {h->d_Mlen, h->d_Plen, h->d_Zlen};
  int* rows[3] = {h->d_Mrow, h->d_Prow, h->d_Zrow};
  void* vals[3] = {h->d_Mval, h->d_Pval, h->d_Zval};
  for (int k = 0; k < 3; k++) {
    CK(cudaMemcpyAsync(o, lens[k], n * 4, cudaMemcpyDeviceToHost, st));
    o += n * 4;
    CK(cudaMemcpyAsync(o, rows[k], S * 4, cudaMemcpyDeviceToHost, st));
    o += S * 4;
    CK(cudaMemcpyAsync(o, vals[k], S * vs, cudaMemcpyDeviceToHost, st));
    o += S * vs;
  }
  CK(cudaStreamSynchronize(st));
  *bytes = need;
  return SPAI_OK;
}

int spai_load_state(spai_handle h, const void* buf, size_t bytes) {
  if (!h || !buf) return SPAI_ERR_ARG;
  const size_t vs = h->prec == SPAI_MIXED ? 4 : 8;
  const size_t n = h->n, S = h->slab_total;
  size_t need = sizeof(StateHeader) + sizeof(DevScalars) + 3 * n * 4 + 3 * S * 4 + 3 * S * vs;
  if (bytes < need) return SPAI_ERR_STATE;
  const char* o = (const char*)buf;
  StateHeader hd;
  memcpy(&hd, o, sizeof(hd));
  if (memcmp(hd.magic, "SPAIST01", 8) != 0 || hd.n != h->n || hd.slab_total != h->slab_total ||
      hd.prec != h->prec || hd.capmax != h->capmax || hd.W != h->W)
    return SPAI_ERR_STATE;
  {
    // every slab column must hold at most cap_j distinct rows in [0, n):
    // the kernels rely on it, so a damaged checkpoint is refused here
    std::vector<long long> offv(n + 1);
    std::vector<int> capv(n);
    CK(cudaMemcpy(offv.data(), h->d_off, sizeof(long long) * (n + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(capv.data(), h->d_cap, sizeof(int) * n, cudaMemcpyDeviceToHost));
    const char* q = o + sizeof(hd) + sizeof(DevScalars);
    std::vector<int> tmp;
    for (int k = 0; k < 3; k++) {
      const int* lens = (const int*)q;
      const int* rows = (const int*)(q + n * 4);
      for (size_t jj = 0; jj < n; jj++) {
        int len = lens[jj];
        if (len < 0 || len > capv[jj]) return SPAI_ERR_STATE;
        tmp.assign(rows + offv[jj], rows + offv[jj] + len);
        std::sort(tmp.begin(), tmp.end());
        for (int e = 0; e < len; e++)
          if (tmp[e] < 0 || tmp[e] >= (int)n || (e > 0 && tmp[e] == tmp[e - 1])) return SPAI_ERR_STATE;
      }
      q += n * 4 + S * 4 + S * vs;
    }
  }
  o += sizeof(hd);
  cudaStream_t st = h->stream;
  // keep this handle's counters, restore the iteration scalars
  DevScalars cur, sv;
  CK(cudaMemcpyAsync(&cur, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  memcpy(&sv, o, sizeof(sv));
  sv.bytes = cur.bytes;
  sv.spgemm_cols = cur.spgemm_cols;
  sv.r_bytes = cur.r_bytes;
  CK(cudaMemcpyAsync(h->d_sc, &sv, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  o += sizeof(DevScalars);
  int* lens[3] = {h->d_Mlen, h->d_Plen, h->d_Zlen};
  int* rows[3] = {h->d_Mrow, h->d_Prow, h->d_Zrow};
  void* vals[3] = {h->d_Mval, h->d_Pval, h->d_Zval};
  for (int k = 0; k < 3; k++) {
    CK(cudaMemcpyAsync(lens[k], o, n * 4, cudaMemcpyHostToDevice, st));
    o += n * 4;
    CK(cudaMemcpyAsync(rows[k], o, S * 4, cudaMemcpyHostToDevice, st));
    o += S * 4;
    CK(cudaMemcpyAsync(vals[k], o, S * vs, cudaMemcpyHostToDevice, st));
    o += S * vs;
  }
  CK(cudaStreamSynchronize(st));
  h->method = hd.method;
  h->it = hd.it;
  invalidate_rows(h);
  return SPAI_OK;
}

int spai_set_timing(spai_handle h, int enable) {
  if (!h) return SPAI_ERR_ARG;
  h->timing = enable != 0;
  return SPAI_OK;
}

int spai_get_stats(spai_handle h, spai_stats* out) {
  if (!h || !out) return SPAI_ERR_ARG;
  DevScalars sc;
  CK(cudaMemcpyAsync(&sc, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out->colpass_launches = h->colpass_launches;
  out->colpass_bytes = (int64_t)(sc.bytes + h->a_bytes_total);
  out->colpass_ms = h->colpass_ms;
  out->pcg_launches = h->pcg_launches;
  out->other_launches = h->other_launches;
  out->spgemm_columns = (int64_t)sc.spgemm_cols;
  out->colpass_r_bytes = (int64_t)sc.r_bytes;
  out->colpass_steady_launches = h->steady_launches;
  return SPAI_OK;
}

}  // extern "C"
