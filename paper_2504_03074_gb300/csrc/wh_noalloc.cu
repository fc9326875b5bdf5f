// wh_noalloc.cu -- the allocation-free entry point wh_multidot_noalloc.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by another
// allocator working to a fixed budget, and latency-critical loops in which cudaMalloc /
// cudaFree (which synchronise the device) are not acceptable.  For them this file offers
// the GMRES inner products <X_k, y> without a context and without any allocation: the
// per-block partial sums live in the file-scope array below, which every GPU that loads
// the library holds until the process exits.
//
// Rules of use:
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (host code cannot use the array's name as a device pointer);
//     make that first call before any stream capture on that device;
//   - every call on a device shares the one array and it keeps the last call's contents;
//     each call writes every partial sum it later reads, so nothing needs clearing, but
//     calls that overlap on the GPU (different streams, or host threads racing) race on
//     the array and give wrong results: serialise them.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/waveholtz.h"
#include "wh_internal.h"

namespace {

constexpr int kBlocks = WH_NOALLOC_BLOCKS;
constexpr int kMaxVectors = WH_NOALLOC_MAX_VECTORS;
constexpr int kMaxDevices = 64;

// partial sums: kMaxVectors x kBlocks doubles (256 KiB)
static __device__ __align__(256) double g_partial[kMaxVectors * kBlocks];

double *g_partial_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

}  // namespace

extern "C" wh_status wh_multidot_noalloc(const double *X, int64_t ldx, int32_t nv,
                                         const double *y, int64_t n, double *out,
                                         void *stream) {
  // sizes beyond the fixed scratch are refused before any device work
  if (nv < 1 || nv > kMaxVectors) return WH_ERR_ARG;
  if (n < 0 || (nv > 1 && ldx < n)) return WH_ERR_ARG;
  if (!out || (n > 0 && (!X || !y))) return WH_ERR_ARG;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WH_ERR_CUDA;
  double *partial = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partial_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_partial);
      if (e != cudaSuccess || !p) return WH_ERR_CUDA;
      g_partial_addr[dev] = (double *)p;
    }
    partial = g_partial_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int nb = (int)((n + wh::kRedThreads - 1) / wh::kRedThreads);
  nb = nb < 1 ? 1 : (nb > kBlocks ? kBlocks : nb);
  // the first pass writes partial[k * nb + b] for every k < nv and b < nb; the second
  // pass reads exactly those entries
  wh::launch_multidot(nb, s, X, ldx, nv, y, n, partial, out);
  e = cudaGetLastError();
  return e == cudaSuccess ? WH_OK : WH_ERR_CUDA;
}
