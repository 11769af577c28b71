// rix_count_flops: the algorithmic FLOPs of one build after block screening.
//
// The FLOP counts of rix_stats are taken at setup from the product lists and
// include every product.  The build then skips the products whose C, V or D
// block is below the screening threshold tau (Sec. "Screening": a block is
// negligible when its largest element is below tau), and which blocks of D are
// negligible is known only once D is.  These kernels walk the same product
// lists as the FP64 stage kernels, apply the same tests to the same flags and
// add up 2 x multiply-adds of every product that is kept, so that a stage's
// throughput can be quoted on the work it actually does.  Every count is an
// integer below 2^53 and every partial sum is exact in FP64, so the atomic
// order does not matter.
#include "rix_internal.h"

namespace {

constexpr int CNT_THREADS = 256;

// out: [0] T, [1] U2, [2] terms 1+2, [3] Z, [4] terms 3+4, [5] symmetrise (set
// on the host), [6] the term-2 part of [2], [7] the term-1 part of [2] for the
// column atoms whose term 1 runs on the tensor cores, [8] the part of [3] for
// the middle atoms whose Z products run on the tensor cores, [9] the part of
// [0] for the row atoms whose T runs on the tensor cores.
__device__ __forceinline__ void add_out(double *out, int i, double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out + i, v);
}

// T(A,G') <- C(A,B') D(B',G'): 2 na_A nb_A nb_B nb_G per kept product.
__global__ void k_cnt_T(int64_t n2, const int64_t *ptrT, const int2 *LT, const int32_t *atomA2,
                        const int32_t *atomB2, const int32_t *pB, const int32_t *nb, const int32_t *na,
                        const uint8_t *keepC, const uint8_t *keepD, const uint8_t *ttc, rix::PScreen ps,
                        double *out) {
  double all = 0.0, tc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = atomA2[t], g = atomB2[t];
    const double f = 2.0 * na[a] * nb[a] * nb[g];
    double s = 0.0;
    for (int64_t e = ptrT[t]; e < ptrT[t + 1]; e++) {
      const int2 en = LT[e];
      if (keepC[en.x] && keepD[en.y] && !ps.drop2(en.x, en.y)) s += f * nb[pB[en.x]];
    }
    all += s;
    if (ttc && ttc[a]) tc += s;
  }
  add_out(out, 0, all);
  add_out(out, 9, tc);
}

// U2(A,G') = V(A,G') T(A,G'): 2 na_A na_G nb_A nb_G per pair with a kept V.
__global__ void k_cnt_U2(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *nb, const int32_t *na,
                         const uint8_t *keepV, double *out) {
  double s = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const int a = pA[p], g = pB[p];
    if (keepV[p]) s += 2.0 * na[a] * na[g] * nb[a] * nb[g];
  }
  add_out(out, 1, s);
}

// Terms 1 and 2 of X(A,E'), the tests of the FP64 kernel: term 1 needs C(G',E')
// and V(A,E'), term 2 needs C(G',E') and V(A,G').
__global__ void k_cnt_X12(int64_t n2, const int64_t *ptr, const rix::X12Entry *L, const int32_t *atomA2,
                          const int32_t *atomB2, const int32_t *map2to1, const int32_t *pA,
                          const int32_t *nb, const int32_t *na, const uint8_t *keepC, const uint8_t *keepV,
                          const uint8_t *t1tc, const uint8_t *rep1, double *out) {
  double all = 0.0, t2 = 0.0, t1tc_s = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n2; s += (int64_t)gridDim.x * blockDim.x) {
    const int a = atomA2[s], e = atomB2[s];
    const int pae = map2to1[s];
    const bool has1 = pae >= 0 && keepV[pae] && rep1[pae];  // one orientation per pair
    double s1 = 0.0;
    for (int64_t it = ptr[s]; it < ptr[s + 1]; it++) {
      const rix::X12Entry en = L[it];
      if (!keepC[en.p3]) continue;
      const int g = pA[en.p3];
      if (en.t1 && has1) s1 += 2.0 * na[e] * na[a] * nb[a] * nb[g] + 2.0 * na[e] * nb[a] * nb[g] * nb[e];
      if (en.u2 >= 0 && keepV[en.u2]) t2 += 2.0 * na[g] * nb[a] * nb[g] * nb[e];
    }
    all += s1;
    if (t1tc && t1tc[e]) t1tc_s += s1;
  }
  add_out(out, 2, all + t2);
  add_out(out, 6, t2);
  add_out(out, 7, t1tc_s);
}

// Z(B,E') <- D(B,G') V(B,G') C(G',E'): 2 na_B na_G nb_G nb_E + 2 na_B nb_B nb_G nb_E per kept product.
__global__ void k_cnt_Z(int64_t n2, const int64_t *ptrZ, const int2 *LZ, const int32_t *atomA2,
                        const int32_t *atomB2, const int32_t *pB, const int32_t *nb, const int32_t *na,
                        const uint8_t *keepC, const uint8_t *keepV, const uint8_t *keepD, const uint8_t *ztc,
                        rix::PScreen ps, double *out) {
  double all = 0.0, tc = 0.0;
  for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < n2; z += (int64_t)gridDim.x * blockDim.x) {
    const int b = atomA2[z], e = atomB2[z];
    for (int64_t x = ptrZ[z]; x < ptrZ[z + 1]; x++) {
      const int2 en = LZ[x];
      if (!keepD[en.x] || !keepV[en.x] || !keepC[en.y] || ps.drop3(en.x, en.x, en.y)) continue;
      const int g = pB[en.x];
      const double f = 2.0 * na[b] * na[g] * nb[g] * nb[e] + 2.0 * na[b] * nb[b] * nb[g] * nb[e];
      all += f;
      if (ztc && ztc[g]) tc += f;
    }
  }
  add_out(out, 3, all);
  add_out(out, 8, tc);
}

// X(A,E') <- C(A,B') Z(B,E'): 2 na_B nb_B nb_A nb_E per product with a kept C.
__global__ void k_cnt_X34(int64_t nk, const int64_t *ptr, const int2 *L, const int32_t *atomA3,
                          const int32_t *atomB3, const int32_t *pB, const int32_t *nb, const int32_t *na,
                          const uint8_t *keepC, const uint8_t *rep3, double *out) {
  double s = 0.0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nk; x += (int64_t)gridDim.x * blockDim.x) {
    if (!rep3[x]) continue;  // one orientation per K block
    const int a = atomA3[x], e = atomB3[x];
    for (int64_t it = ptr[x]; it < ptr[x + 1]; it++) {
      const int2 en = L[it];
      if (!keepC[en.x]) continue;
      const int b = pB[en.x];
      s += 2.0 * na[b] * nb[b] * nb[a] * nb[e];
    }
  }
  add_out(out, 4, s);
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + CNT_THREADS - 1) / CNT_THREADS;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

extern "C" rix_status rix_count_flops(rix_ctx *ctx, const double *D, double *flops, void *stream) {
  if (ctx) ctx->fwd_valid = false;  // the D screening flags follow this D
  if (!ctx || !D || !flops) return RIX_EINVAL;
  if (!ctx->have_cv) return RIX_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    ctx->last_error = "rix_count_flops reads its result back and cannot run inside a graph capture";
    return RIX_ESTATE;
  }
  rix_status s;
  if ((s = rix_launch_flags(ctx, D, ctx->d_offD, ctx->np, ctx->d_keepD, st, ctx->d_normD)) != RIX_OK) return s;
  double *d_out = nullptr;
  RIX_CUDA_TRY(ctx, cudaMallocAsync((void **)&d_out, 10 * sizeof(double), st));
  rix_status r = RIX_OK;
  do {
    if (cudaMemsetAsync(d_out, 0, 10 * sizeof(double), st) != cudaSuccess) { r = RIX_ECUDA; break; }
    const int64_t n2 = ctx->stats.n_pairs2, nk = ctx->stats.n_kblocks;
    k_cnt_T<<<grid_for(n2), CNT_THREADS, 0, st>>>(n2, ctx->d_ptrT, ctx->d_LT, ctx->d_atomA2, ctx->d_atomB2,
                                                  ctx->d_pB, ctx->d_nb, ctx->d_na, ctx->d_keepC, ctx->d_keepD,
                                                  ctx->d_ttc, rix_pscreen(ctx), d_out);
    k_cnt_U2<<<grid_for(ctx->np), CNT_THREADS, 0, st>>>(ctx->np, ctx->d_pA, ctx->d_pB, ctx->d_nb, ctx->d_na,
                                                        ctx->d_keepV, d_out);
    k_cnt_X12<<<grid_for(n2), CNT_THREADS, 0, st>>>(n2, ctx->d_ptrX12, ctx->d_LX12, ctx->d_atomA2,
                                                    ctx->d_atomB2, ctx->d_map2to1, ctx->d_pA, ctx->d_nb, ctx->d_na, ctx->d_keepC, ctx->d_keepV,
                                                    ctx->d_t1tc, ctx->d_rep1, d_out);
    k_cnt_Z<<<grid_for(n2), CNT_THREADS, 0, st>>>(n2, ctx->d_ptrZ, ctx->d_LZ, ctx->d_atomA2, ctx->d_atomB2,
                                                  ctx->d_pB, ctx->d_nb, ctx->d_na, ctx->d_keepC, ctx->d_keepV,
                                                  ctx->d_keepD, ctx->d_ztc, rix_pscreen(ctx), d_out);
    k_cnt_X34<<<grid_for(nk), CNT_THREADS, 0, st>>>(nk, ctx->d_ptrX34, ctx->d_LX34, ctx->d_atomA3,
                                                    ctx->d_atomB3, ctx->d_pB, ctx->d_nb, ctx->d_na, ctx->d_keepC,
                                                    ctx->d_rep3, d_out);
    if (cudaGetLastError() != cudaSuccess) { r = RIX_ECUDA; break; }
    if (cudaMemcpyAsync(flops, d_out, 10 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      r = RIX_ECUDA;
      break;
    }
  } while (0);
  cudaFreeAsync(d_out, st);
  if (r != RIX_OK) {
    ctx->last_error = std::string("rix_count_flops: ") + cudaGetErrorString(cudaGetLastError());
    return r;
  }
  flops[5] = ctx->stats.flops_stage[5];
  return RIX_OK;
}
