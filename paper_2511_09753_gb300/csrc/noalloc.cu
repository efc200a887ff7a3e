// spai_true_residual_noalloc: the residual norms ||b - A x||_2 and ||b||_2
// of a linear system, for callers that must not allocate device memory.
//
// Who needs this: code whose device memory is owned by another allocator
// (for example a framework's caching allocator that reserves the GPU's memory
// and does not let libraries call cudaMalloc behind its back), and
// latency-sensitive loops that cannot afford cudaMalloc / cudaFree, which can
// synchronise the whole device.  The handle-based calls of this library
// allocate their workspace when a handle is created; this entry point takes
// no handle and uses a fixed workspace that lives in the library image.
//
// The workspace is the file-scope array g_na_scratch below (about 1 MB).
// Every GPU that loads the library keeps it until the process exits.  In
// host code its name is only a host-side stand-in, so the address the kernel
// receives comes from cudaGetSymbolAddress, looked up once per device on the
// first call made with that device current.  Because of that set-up, make the
// first call on each device before starting any stream capture.
//
// Every call shares the one array and it keeps the previous call's contents:
// the call clears the counters that must start at zero before launching.
// Calls whose kernels overlap on the GPU (two streams, or two host threads)
// race on the array and give wrong results; order them on one stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "spai.h"
#include "warp_ops.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr long long kNaMaxN = 1LL << 24;                       // 16,777,216 rows
constexpr int kNaMaxBlocks = (int)(kNaMaxN / kNaThreads);      // 65,536
constexpr int kNaGroup = 64;
constexpr int kNaMaxGroups = kNaMaxBlocks / kNaGroup;          // 1,024

struct NaScratch {
  double bsum[2][kNaMaxBlocks];   // per-CTA sums of the two quantities
  double gsum[2][kNaMaxGroups];   // per-group sums
  unsigned cnt1[kNaMaxGroups];    // arrivals per group (must start at 0)
  unsigned cnt2;                  // arrivals of groups (must start at 0)
};

}  // namespace

static __device__ __align__(256) unsigned char g_na_scratch[sizeof(NaScratch)];

namespace {

// Row i of A: fma chain over ascending column (the library's SpMV order);
// per-thread terms (b_i - (A x)_i)^2 and b_i^2, reduced by the balanced
// pairwise tree over the row index that pcg_solve uses for its residual.
__global__ void __launch_bounds__(kNaThreads)
k_true_residual_noalloc(int n, const int32_t* rp, const int32_t* ci, const double* av,
                        const double* b, const double* x, double* out, NaScratch* ws) {
  __shared__ double red[2][32];
  __shared__ double top[1024];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = gridDim.x;
  const int ngroups = (nb + kNaGroup - 1) / kNaGroup;
  const int i = blockIdx.x * kNaThreads + threadIdx.x;
  double t[2] = {0.0, 0.0};
  if (i < n) {
    double acc = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; e++) acc = __fma_rn(av[e], x[ci[e]], acc);
    double bi = b[i];
    double d = __dsub_rn(bi, acc);
    t[0] = __dmul_rn(d, d);
    t[1] = __dmul_rn(bi, bi);
  }
  for (int q = 0; q < 2; q++) {
    double s = spai::warp_tree32(t[q]);
    if (lane == 0) red[q][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
    for (int q = 0; q < 2; q++) {
      double s = spai::warp_tree32(lane < kNaThreads / 32 ? red[q][lane] : 0.0);
      if (lane == 0) ws->bsum[q][blockIdx.x] = s;
    }
  }
  const int g = blockIdx.x / kNaGroup;
  if (threadIdx.x == 0) {
    __threadfence();
    int gsize = min(kNaGroup, nb - g * kNaGroup);
    unsigned old = atomicAdd(&ws->cnt1[g], 1u);
    s_last = old == (unsigned)(gsize - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (warp == 0) {
    int gsize = min(kNaGroup, nb - g * kNaGroup);
    for (int q = 0; q < 2; q++) {
      const double* v = ws->bsum[q] + (long long)g * kNaGroup;
      double a = (2 * lane < gsize) ? __ldcg(v + 2 * lane) : 0.0;
      double c = (2 * lane + 1 < gsize) ? __ldcg(v + 2 * lane + 1) : 0.0;
      double s = spai::warp_tree32(__dadd_rn(a, c));
      if (lane == 0) ws->gsum[q][g] = s;
    }
  }
  // the host clears cnt1 and cnt2 before every launch (they keep whatever an
  // earlier or aborted call left), so the kernel leaves them as they are
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned old = atomicAdd(&ws->cnt2, 1u);
    s_last = old == (unsigned)(ngroups - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (warp == 0) {
    int P2 = 32;
    while (P2 < ngroups) P2 <<= 1;
    int c = P2 / 32;
    for (int q = 0; q < 2; q++) {
      for (int k = 0; k < c; k++) {
        int idx = lane * c + k;
        top[idx] = idx < ngroups ? __ldcg(&ws->gsum[q][idx]) : 0.0;
      }
      __syncwarp();
      double s = spai::warp_pairwise(top, P2, lane);
      if (lane == 0) out[q] = __dsqrt_rn(s);
      __syncwarp();
    }
  }
}

std::mutex g_na_mutex;
void* g_na_ptr[256] = {nullptr};

}  // namespace

extern "C" int spai_true_residual_noalloc(int64_t n, const int32_t* rowptr, const int32_t* colind,
                                          const double* vals, const double* b, const double* x,
                                          double* out, void* stream) {
  if (n < 1) return SPAI_ERR_ARG;
  if (n > kNaMaxN) return SPAI_ERR_UNSUPPORTED;
  if (!rowptr || !colind || !vals || !b || !x || !out) return SPAI_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    (void)cudaGetLastError();
    return SPAI_ERR_CUDA;
  }
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return SPAI_ERR_CUDA;
      }
      g_na_ptr[dev] = p;
    }
    ptr = g_na_ptr[dev];
  }
  NaScratch* ws = (NaScratch*)ptr;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((n + kNaThreads - 1) / kNaThreads);
  const int ngroups = (nb + kNaGroup - 1) / kNaGroup;
  // the arrival counters must start at zero whatever a previous call left
  if (cudaMemsetAsync(ws->cnt1, 0, sizeof(unsigned) * (size_t)ngroups, st) != cudaSuccess ||
      cudaMemsetAsync(&ws->cnt2, 0, sizeof(unsigned), st) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAI_ERR_CUDA;
  }
  k_true_residual_noalloc<<<nb, kNaThreads, 0, st>>>((int)n, rowptr, colind, vals, b, x, out, ws);
  if (cudaGetLastError() != cudaSuccess) return SPAI_ERR_CUDA;
  return SPAI_OK;
}
