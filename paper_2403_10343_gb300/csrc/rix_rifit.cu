// RI-LVL coefficient fit (the paper's Eq. 8 with the pair-restricted Coulomb
// metric of Eq. 10; the "Initialization" stage of the exchange build):
//
//   C^mu_ij = sum_{nu in P(IJ)} (ij|nu) L^{IJ}_{nu mu},   L^{IJ} = (V^{IJ})^{-1},
//
// for every atom pair (I, J, n), with P(IJ) = aux(I) u aux(J) (aux(I) alone for
// the on-site pair) and V^{IJ} the Coulomb matrix restricted to P(IJ): the
// on-site blocks V(I,I,0), V(J,J,0) on the diagonal and V(I,J,n) off it.  Each
// representative pair (I < J, or I == J with n > 0, or on-site) is one CTA:
// it assembles V^{IJ} + lambda 1 in a workspace, factors it by Cholesky
// (right-looking, in place, lower triangle) and solves L L^T x = (ij|.) for
// every (i, j) column; the partner pair (J, I, -n) receives the same numbers
// with (i, j) and the two aux sets swapped, so the fitted C is exactly pair
// symmetric.  lambda > 0 shifts the diagonal (a Tikhonov fit) for metrics that
// are numerically singular.
#include <algorithm>
#include <vector>

#include "rix_internal.h"

namespace {

constexpr int FIT_THREADS = 256;

// M = V^{IJ} + lambda 1 for pair p (n x n, row-major)
__device__ void assemble(double *M, int n, int naA, int naB, bool onsite, const double *Vaa, const double *Vbb,
                         const double *Vab, double lambda) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    double v;
    if (r < naA && c < naA) v = Vaa[r * naA + c];
    else if (onsite) v = 0.0;  // not reached: n == naA
    else if (r >= naA && c >= naA) v = Vbb[(r - naA) * naB + (c - naA)];
    else if (r < naA) v = Vab[r * naB + (c - naA)];
    else v = Vab[c * naB + (r - naA)];
    M[e] = r == c ? v + lambda : v;
  }
}

__global__ void k_rifit(int64_t nrep, const int32_t *rep, const int32_t *pA, const int32_t *pB,
                        const int32_t *partner, const uint8_t *onsite, const int32_t *onsite_pair, const int32_t *nb,
                        const int32_t *na, const double *__restrict__ V, const int64_t *offV,
                        const double *__restrict__ eri, const int64_t *offC, double lambda, double *work,
                        const int64_t *woff, double *C, int *err) {
  const int64_t r = blockIdx.x;
  if (r >= nrep) return;
  const int p = rep[r];
  const int a = pA[p], b = pB[p];
  const bool ons = onsite[p];
  const int naA = na[a], naB = na[b], nbA = nb[a], nbB = nb[b];
  const int n = naA + (ons ? 0 : naB);
  double *M = work + woff[r];
  assemble(M, n, naA, naB, ons, V + offV[onsite_pair[a]], V + offV[onsite_pair[b]], V + offV[p], lambda);
  __syncthreads();
  // Cholesky, right-looking: column k scaled by 1/sqrt(pivot), trailing lower triangle updated
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int k = 0; k < n; k++) {
    if (threadIdx.x == 0) {
      const double d = M[k * n + k];
      if (!(d > 0.0)) bad = 1;
      piv = d > 0.0 ? sqrt(d) : 1.0;
      M[k * n + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) M[i * n + k] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) M[i * n + j] -= M[i * n + k] * M[j * n + k];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  // one (i, j) column per thread: forward then backward substitution in place in C(p)
  const double *rhs = eri + offC[p];
  double *x = C + offC[p];
  const int cols = nbA * nbB;
  for (int col = threadIdx.x; col < cols; col += blockDim.x) {
    for (int i = 0; i < n; i++) {
      double s = rhs[(int64_t)i * cols + col];
      for (int j = 0; j < i; j++) s -= M[i * n + j] * x[(int64_t)j * cols + col];
      x[(int64_t)i * cols + col] = s / M[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = x[(int64_t)i * cols + col];
      for (int j = i + 1; j < n; j++) s -= M[j * n + i] * x[(int64_t)j * cols + col];
      x[(int64_t)i * cols + col] = s / M[i * n + i];
    }
  }
  if (ons) return;
  __syncthreads();
  // the partner (B, A, -n): C(q)[mu'][j][i] = C(p)[mu][i][j], mu' = mu with the aux sets swapped
  const int64_t q = partner[p];
  double *y = C + offC[q];
  for (int e = threadIdx.x; e < n * cols; e += blockDim.x) {
    const int mu = e / cols, ij = e - mu * cols, i = ij / nbB, j = ij - i * nbB;
    const int mq = mu < naA ? naB + mu : mu - naA;
    y[((int64_t)mq * nbB + j) * nbA + i] = x[e];
  }
}

}  // namespace

extern "C" rix_status rix_fit_C(rix_ctx *ctx, const double *V, const double *eri, double lambda, double *C,
                                void *stream) {
  if (!ctx || !V || !eri || !C || !(lambda >= 0.0)) return RIX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // representative pairs, their metric sizes, and the on-site pair of every atom
  std::vector<int32_t> rep, ons(ctx->nat, -1);
  for (int64_t p = 0; p < ctx->np; p++) {
    const int a = ctx->pA[p], b = ctx->pB[p];
    if (ctx->onsite[p]) ons[a] = (int32_t)p;
    bool is_rep = ctx->onsite[p] || a < b;
    if (a == b && !ctx->onsite[p]) {
      const int8_t *n = &ctx->pn[3 * p];
      is_rep = n[0] > 0 || (n[0] == 0 && (n[1] > 0 || (n[1] == 0 && n[2] > 0)));
    }
    if (is_rep) rep.push_back((int32_t)p);
  }
  for (int a = 0; a < ctx->nat; a++)
    if (ons[a] < 0) {
      ctx->last_error = "rix_fit_C: an atom without its on-site pair";
      return RIX_EINVAL;
    }
  // batches of representative pairs whose metrics fit a 1 GB workspace
  const int64_t budget = (int64_t)1 << 27;  // doubles
  int32_t *d_rep = nullptr, *d_ons = nullptr;
  int64_t *d_woff = nullptr;
  double *d_work = nullptr;
  int *d_err = nullptr;
  std::vector<int64_t> woff;
  size_t first = 0;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMallocAsync(p, bytes, st);
  };
  int64_t maxw = 0;
  {
    int64_t w = 0;
    for (size_t r = 0; r < rep.size(); r++) {
      const int p = rep[r];
      const int64_t n = ctx->na_at[ctx->pA[p]] + (ctx->onsite[p] ? 0 : ctx->na_at[ctx->pB[p]]);
      if (w + n * n > budget && w > 0) { maxw = std::max(maxw, w); w = 0; }
      w += n * n;
    }
    maxw = std::max(maxw, w);
  }
  alloc((void **)&d_rep, sizeof(int32_t) * std::max<size_t>(rep.size(), 1));
  alloc((void **)&d_ons, sizeof(int32_t) * ctx->nat);
  alloc((void **)&d_woff, sizeof(int64_t) * std::max<size_t>(rep.size(), 1));
  alloc((void **)&d_work, sizeof(double) * std::max<int64_t>(maxw, 1));
  alloc((void **)&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rep, rep.data(), sizeof(int32_t) * rep.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ons, ons.data(), sizeof(int32_t) * ctx->nat, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  woff.assign(rep.size(), 0);
  while (e == cudaSuccess && first < rep.size()) {
    size_t last = first;
    int64_t w = 0;
    while (last < rep.size()) {
      const int p = rep[last];
      const int64_t n = ctx->na_at[ctx->pA[p]] + (ctx->onsite[p] ? 0 : ctx->na_at[ctx->pB[p]]);
      if (w + n * n > budget && last > first) break;
      woff[last] = w;
      w += n * n;
      last++;
    }
    e = cudaMemcpyAsync(d_woff + first, woff.data() + first, sizeof(int64_t) * (last - first), cudaMemcpyHostToDevice,
                        st);
    if (e != cudaSuccess) break;
    // the copy of woff must land before the host vector is reused: pageable memory makes it synchronous
    k_rifit<<<(unsigned)(last - first), FIT_THREADS, 0, st>>>(
        (int64_t)(last - first), d_rep + first, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_onsite, d_ons,
        ctx->d_nb, ctx->d_na, V, ctx->d_offV, eri, ctx->d_offC, lambda, d_work, d_woff + first, C, d_err);
    e = cudaGetLastError();
    first = last;
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  for (void *p : {(void *)d_rep, (void *)d_ons, (void *)d_woff, (void *)d_work, (void *)d_err})
    if (p) cudaFreeAsync(p, st);
  if (e != cudaSuccess) {
    ctx->last_error = std::string("rix_fit_C: ") + cudaGetErrorString(e);
    return RIX_ECUDA;
  }
  if (herr) {
    ctx->last_error = "rix_fit_C: a pair's Coulomb metric is not positive definite (raise lambda)";
    return RIX_EINVAL;
  }
  return RIX_OK;
}
