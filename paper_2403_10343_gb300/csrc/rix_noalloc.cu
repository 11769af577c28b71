// rix_energy_noalloc: the exchange-energy reduction without any device allocation.
//
// Some callers must not allocate device memory at the point where they need
// the energy: a framework whose caching allocator has already reserved the
// GPU's free memory (a fresh cudaMalloc would fail or fragment its pool), or
// a timing-critical SCF loop that forbids allocation and the implicit device
// synchronisation cudaMalloc/cudaFree can cause.  This entry point computes
// the same reduction as rix_energy, but its scratch (the per-CTA partial sums)
// lives in the fixed device array below instead of context-owned memory.
//
// Limits and sharing rules:
//  * the array holds RIX_NOALLOC_MAX_PARTIALS doubles (512 KB), one per 256
//    pairs, so the pair list may hold at most 256 * 65536 = 16,777,216 pairs;
//    larger contexts are rejected with RIX_EINVAL;
//  * every GPU that loads the library keeps this array until the process exits;
//  * all calls on a device share the one array, and it keeps the previous
//    call's partial sums; each call overwrites every slot it reads, so nothing
//    needs clearing, but calls whose work overlaps on the GPU (different
//    streams, or another context on the same device) race on it;
//  * the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture is started.
#include <mutex>

#include "rix_internal.h"

#define RIX_NOALLOC_MAX_PARTIALS 65536
#define RIX_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_partials[RIX_NOALLOC_MAX_PARTIALS];

rix_status rix_launch_energy_partials(rix_ctx *ctx, const double *D, const double *K, double *Ex,
                                      double *partials, cudaStream_t st);

namespace {
std::mutex g_mu;
double *g_addr[RIX_NOALLOC_MAX_DEVICES] = {nullptr};
}  // namespace

extern "C" rix_status rix_energy_noalloc(rix_ctx *ctx, const double *D, const double *K, double *Ex,
                                         void *stream) {
  if (!ctx || !D || !K || !Ex) return RIX_EINVAL;
  if (ctx->n_epart > RIX_NOALLOC_MAX_PARTIALS) {
    ctx->last_error = "rix_energy_noalloc: more than 16,777,216 pairs (fixed scratch of 65536 partial sums)";
    return RIX_EINVAL;
  }
  int dev = 0;
  RIX_CUDA_TRY(ctx, cudaGetDevice(&dev));
  if (dev < 0 || dev >= RIX_NOALLOC_MAX_DEVICES) {
    ctx->last_error = "rix_energy_noalloc: device ordinal beyond 63";
    return RIX_EUNSUPPORTED;
  }
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // host code cannot use g_noalloc_partials directly: its host-side name
      // is only a stand-in, so fetch the device address once per device
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->last_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return RIX_ECUDA;
      }
      g_addr[dev] = (double *)p;
    }
    scratch = g_addr[dev];
  }
  return rix_launch_energy_partials(ctx, D, K, Ex, scratch, (cudaStream_t)stream);
}
