// Force and stress chain of the exchange energy (the paper's Sec. "EXX force
// and stress contributions" and "Computation of Forces and Stress").
//
// The RI coefficients C(A,B,n) and the Coulomb matrix V(A,B,n) of a pair depend
// on the geometry through the pair vector r_p = x_B + n . a - x_A.  With the
// adjoint dE/dC and dE/dV of the stored entries (rix_backward) and the
// caller's derivatives dC/dr_p, dV/dr_p (one Cartesian component c at a time,
// the paper's split of the force/stress work into three parts to bound memory):
//
//   g_p      = sum_e dE/dC_pe dC_pe/d(r_p)_c + sum_e dE/dV_pe dV_pe/d(r_p)_c
//   F_X,c    = -dE/dx_X,c = sum_{p: A_p = X} (g_p - g_partner(p))
//              (r_p moves with x_B and against x_A; partner(p) = (B, A, -n) is
//              the pair whose B is X)
//   S_c,b    = (1/Omega) sum_p g_p (r_p)_b   = (1/Omega) dE/d eps_cb
//              (a homogeneous strain eps maps every r_p to (1 + eps) r_p)
//
// D is held fixed (its geometry dependence is the SCF's, not the exchange
// build's).  Every sum runs in a fixed order: one warp per pair, one thread per
// atom over its contiguous pairs, a fixed tree for the stress.
#include "rix_internal.h"

namespace {

__global__ void k_gpair(int64_t np, const int64_t *offC, const int64_t *offV, const double *__restrict__ dEdC,
                        const double *__restrict__ dCdr, const double *__restrict__ dEdV,
                        const double *__restrict__ dVdr, double *g) {
  const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= np) return;
  double s = 0.0;
  if (dEdC)
    for (int64_t e = offC[p] + lane; e < offC[p + 1]; e += 32) s = fma(dEdC[e], dCdr[e], s);
  if (dEdV)
    for (int64_t e = offV[p] + lane; e < offV[p + 1]; e += 32) s = fma(dEdV[e], dVdr[e], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) g[p] = s;
}

__global__ void k_force(int nat, const int64_t *row1, const int32_t *partner, const double *g, double *F) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nat) return;
  double f = 0.0;
  for (int64_t p = row1[x]; p < row1[x + 1]; p++) f += g[p] - g[partner[p]];
  F[x] = f;
}

// one CTA of 256 threads: S_b = scale * sum_p g_p r_p,b in a fixed order
__global__ void k_stress(int64_t np, const double *g, const double *rvec, double scale, double *S) {
  __shared__ double red[3][256];
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t p = threadIdx.x; p < np; p += 256)
    for (int b = 0; b < 3; b++) s[b] = fma(g[p], rvec[3 * p + b], s[b]);
  for (int b = 0; b < 3; b++) red[b][threadIdx.x] = s[b];
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if (threadIdx.x < w)
      for (int b = 0; b < 3; b++) red[b][threadIdx.x] += red[b][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) S[threadIdx.x] = scale * red[threadIdx.x][0];
}

}  // namespace

extern "C" rix_status rix_force_stress(rix_ctx *ctx, int32_t c, const double *dEdC, const double *dEdV,
                                       const double *dCdr_c, const double *dVdr_c, double *F, double *stress,
                                       void *stream) {
  if (!ctx || c < 0 || c > 2 || (!dEdC && !dEdV) || (dEdC && !dCdr_c) || (dEdV && !dVdr_c)) return RIX_EINVAL;
  if (!F && !stress) return RIX_EINVAL;
  if (stress && !ctx->periodic) {
    ctx->last_error = "rix_force_stress: a cluster has no stress";
    return RIX_EINVAL;
  }
  rix_status s = rix_take_err(ctx);
  if (s != RIX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((ctx->np * 32 + 255) / 256);
  k_gpair<<<grid, 256, 0, st>>>(ctx->np, ctx->d_offC, ctx->d_offV, dEdC, dCdr_c, dEdV, dVdr_c, ctx->d_gpair);
  if (F) k_force<<<(ctx->nat + 127) / 128, 128, 0, st>>>(ctx->nat, ctx->d_row1, ctx->d_partner1, ctx->d_gpair, F);
  if (stress) k_stress<<<1, 256, 0, st>>>(ctx->np, ctx->d_gpair, ctx->d_rvec, 1.0 / ctx->volume, stress);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string("force/stress: ") + cudaGetErrorString(e);
    return RIX_ECUDA;
  }
  return RIX_OK;
}
