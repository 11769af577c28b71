// K(R) -> K(k) Bloch sums and collinear spin (the paper's Eq. 3 and the spin
// index sigma of Eqs. 3-5).
//
//   K^sigma_IL(k) = sum_n exp(2 pi i kappa . n) K^sigma(A,E,n)[i][l]
//
// with k = sum_c kappa_c b_c (b the reciprocal lattice, b_c . a_d = 2 pi
// delta_cd) and R = sum_c n_c a_c, so k . R = 2 pi kappa . n.  The exchange
// build is linear in D, so the spin channels are two builds with the per-spin
// densities D^sigma (no factor 2 of the closed shell), and
//   E_x = -1/2 sum_sigma Tr(D^sigma K^sigma)   (n_spin = 2)
//   E_x = -1/4 Tr(D K)                          (n_spin = 1, D = D_up + D_dn).
#include <cmath>

#include "rix_internal.h"

rix_status rix_launch_energy_scaled(rix_ctx *ctx, const double *D, const double *K, double *Ex, double scale,
                                    int accumulate, cudaStream_t st);

namespace {

// One CTA per fold group (the K blocks of one atom pair (A, E), all images):
// Kk[I][L] = sum over the group's blocks of exp(2 pi i kappa . n) K[x][i][l].
__global__ void k_bloch(int64_t ng, const int64_t *fold, const int32_t *atomA3, const int32_t *atomB3,
                        const int32_t *nb, const int64_t *offK, const int64_t *bofs, const char4 *n3,
                        int64_t nbasis, double k0, double k1, double k2, const double *__restrict__ K,
                        double2 *Kk) {
  const int64_t gi = blockIdx.x;
  if (gi >= ng) return;
  const int64_t x0 = fold[gi], x1 = fold[gi + 1];
  const int a = atomA3[x0], e = atomB3[x0];
  const int nbA = nb[a], nbE = nb[e];
  __shared__ double2 ph[64];
  for (int64_t xb = x0; xb < x1; xb += 64) {
    const int nx = (int)min((int64_t)64, x1 - xb);
    __syncthreads();
    if (threadIdx.x < nx) {
      const char4 n = n3[xb + threadIdx.x];
      // 2 pi kappa . n = pi (2 kappa . n); sincospi keeps the phase exact for integer multiples
      const double t = 2.0 * (k0 * n.x + k1 * n.y + k2 * n.z);
      double sn, cs;
      sincospi(t, &sn, &cs);
      ph[threadIdx.x] = make_double2(cs, sn);
    }
    __syncthreads();
    for (int el = threadIdx.x; el < nbA * nbE; el += blockDim.x) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < nx; j++) {
        const double v = K[offK[xb + j] + el];
        re = fma(ph[j].x, v, re);
        im = fma(ph[j].y, v, im);
      }
      const int i = el / nbE, l = el - i * nbE;
      double2 *dst = Kk + (bofs[a] + i) * nbasis + bofs[e] + l;
      if (xb == x0) {
        *dst = make_double2(re, im);
      } else {
        const double2 o = *dst;
        *dst = make_double2(o.x + re, o.y + im);
      }
    }
  }
}

}  // namespace

extern "C" rix_status rix_bloch(rix_ctx *ctx, const double *K, int32_t n_k, const double *kfrac, double *Kk,
                                void *stream) {
  if (!ctx || !K || !Kk || n_k < 0 || (n_k > 0 && !kfrac)) return RIX_EINVAL;
  for (int q = 0; q < 3 * n_k; q++)
    if (!std::isfinite(kfrac[q])) return RIX_EINVAL;
  if (!ctx->periodic) {
    for (int q = 0; q < 3 * n_k; q++)
      if (kfrac[q] != 0.0) {
        ctx->last_error = "rix_bloch: a cluster has only the Gamma point";
        return RIX_EINVAL;
      }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t per_k = (size_t)ctx->nbasis * (size_t)ctx->nbasis;
  for (int q = 0; q < n_k; q++) {
    double2 *out = (double2 *)Kk + (size_t)q * per_k;
    RIX_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(double2) * per_k, st));
    if (ctx->n_fold == 0) continue;
    k_bloch<<<(unsigned)ctx->n_fold, 128, 0, st>>>(ctx->n_fold, ctx->d_fold, ctx->d_atomA3, ctx->d_atomB3, ctx->d_nb,
                                                   ctx->d_offK, ctx->d_bofs, ctx->d_n3, ctx->nbasis, kfrac[3 * q],
                                                   kfrac[3 * q + 1], kfrac[3 * q + 2], K, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ctx->last_error = std::string("k_bloch: ") + cudaGetErrorString(e);
      return RIX_ECUDA;
    }
  }
  return RIX_OK;
}

extern "C" rix_status rix_build_K_spin(rix_ctx *ctx, int32_t n_spin, const double *D, double *K, void *stream) {
  if (!ctx || !D || !K || n_spin < 1 || n_spin > 2) return RIX_EINVAL;
  const int64_t nd = ctx->offD[ctx->np], nk = ctx->offK[ctx->nk];
  for (int sgm = 0; sgm < n_spin; sgm++) {
    rix_status s = rix_build_K(ctx, D + sgm * nd, K + sgm * nk, stream);
    if (s != RIX_OK) return s;
  }
  return RIX_OK;
}

extern "C" rix_status rix_energy_spin(rix_ctx *ctx, int32_t n_spin, const double *D, const double *K, double *Ex,
                                      void *stream) {
  if (!ctx || !D || !K || !Ex || n_spin < 1 || n_spin > 2) return RIX_EINVAL;
  rix_status s = rix_take_err(ctx);
  if (s != RIX_OK) return s;
  const int64_t nd = ctx->offD[ctx->np], nk = ctx->offK[ctx->nk];
  const double scale = n_spin == 1 ? -0.25 : -0.5;
  ctx->fwd_valid = false;
  for (int sgm = 0; sgm < n_spin; sgm++) {
    s = rix_launch_energy_scaled(ctx, D + sgm * nd, K + sgm * nk, Ex, scale, sgm > 0, (cudaStream_t)stream);
    if (s != RIX_OK) return s;
  }
  return RIX_OK;
}
