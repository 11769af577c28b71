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
//  * the array's device address is looked up once per context, in rix_setup,
//    with the context's device current (host code cannot use the array's name:
//    on the host it is only a stand-in for the device symbol), so the entry
//    point itself makes no CUDA runtime call besides its two kernel launches.
#include "rix_internal.h"

#define RIX_NOALLOC_MAX_PARTIALS 65536

static __device__ __align__(256) double g_noalloc_partials[RIX_NOALLOC_MAX_PARTIALS];

rix_status rix_launch_energy_partials(rix_ctx *ctx, const double *D, const double *K, double *Ex,
                                      double *partials, cudaStream_t st);

rix_status rix_noalloc_attach(rix_ctx *ctx) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return RIX_ECUDA;
  }
  ctx->noalloc_scratch = (double *)p;
  return RIX_OK;
}

extern "C" rix_status rix_energy_noalloc(rix_ctx *ctx, const double *D, const double *K, double *Ex,
                                         void *stream) {
  if (!ctx || !D || !K || !Ex) return RIX_EINVAL;
  if (ctx->n_epart > RIX_NOALLOC_MAX_PARTIALS) {
    ctx->last_error = "rix_energy_noalloc: more than 16,777,216 pairs (fixed scratch of 65536 partial sums)";
    return RIX_EINVAL;
  }
  if (!ctx->noalloc_scratch) {
    ctx->last_error = "rix_energy_noalloc: scratch address not set up";
    return RIX_ESTATE;
  }
  rix_status s = rix_take_err(ctx);
  if (s != RIX_OK) return s;
  if (D != ctx->fwd_D) ctx->fwd_valid = false;  // the D screening flags follow this D
  return rix_launch_energy_partials(ctx, D, K, Ex, ctx->noalloc_scratch, (cudaStream_t)stream);
}
