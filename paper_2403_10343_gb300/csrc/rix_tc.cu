// FP64-accurate GEMM on the BF16 tensor cores (tcgen05) by error-free slicing.
//
// C = A B with A [M x K], B [K x N] in FP64.  Every row of A (column of B) is
// scaled by a power of two 2^e so that |x| < 2^e, and its 64-bit fixed-point
// fraction |x| / 2^e is cut into S signed 7-bit digits (integers in
// [-127, 127], exact in BF16).  This is the error-free splitting of Ozaki,
// Ogita, Oishi and Rump (2012) with per-row/column exponents.  With
// a = sum_s a_s 2^-7s and b = sum_t b_t 2^-7t,
//
//   A B = 2^(eA + eB) sum_{s+t <= S+1} 2^{-7(s+t)} (A_s B_t)
//
// and every slice product A_s B_t is a sum of integers below 2^14 per term.
// All products with the same s+t share one FP32 accumulator in tensor memory;
// over a group of 128 K values and at most S slice pairs such a sum stays
// below 2^24, so the tensor cores accumulate it exactly.  After each group the
// accumulators are folded into a 64-bit fixed-point sum per output element
// (integer arithmetic), and the FP64 result is formed once at the end.  The
// error is the truncation of the operands after S digits (about 2^-7S of the
// row/column scale) plus the dropped terms s+t > S+1.
//
// Kernel layout: one CTA per 128 x 64 output tile; warp 0 issues the bulk
// copies (cp.async.bulk, mbarrier completion), one thread of warp 1 issues
// tcgen05.mma (A and B from shared memory, accumulators in tensor memory),
// warps 4-7 drain tensor memory (tcgen05.ld) into the fixed-point sums.  Every
// wait is bounded; on a timeout the kernel records an error and returns.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>

#include "rix_internal.h"

namespace rixtc {

constexpr int TM = 128;         // output rows per tile (one TMEM lane each)
constexpr int TN = 64;          // output columns per tile
constexpr int KC = 32;          // K per pipeline stage
constexpr int GROUP = 4;        // stages per exact accumulation group (128 K)
constexpr int MAXS = 8;         // slices supported
constexpr int NSTAGE = 2;
constexpr uint64_t WAIT_NS = 2000000000ull;  // a wait gives up after 2 s

// bytes of one packed tile (no-swizzle K-major core matrices, 8 rows x 16 B)
constexpr int A_TILE = TM * KC * 2;  // 8 KB
constexpr int B_TILE = TN * KC * 2;  // 4 KB

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase with the given parity; returns false after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = now_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (now_ns() - t0 > WAIT_NS) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, swizzle none
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ------------------------------------------------------------------ packing
// Byte offset of element (row r, k) inside a packed tile of `rows` rows x KC
// columns: core matrix (r/8, k/8) at ((r/8) * (KC/8) + k/8) * 128, then row
// r%8 at 16 B, element k%8 at 2 B.  LBO (K direction) = 128 B, SBO (row
// direction) = (KC/8) * 128 B.
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// exponent e with |x| < 2^e for the largest |x| of a row: max unbiased exponent + 1
__device__ __forceinline__ int exp_of(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  int ex = (int)((b >> 52) & 0x7FF);
  return ex == 0 ? -2000 : ex - 1023 + 1;  // zero and subnormals count as tiny
}

// digit s (1-based) of |x| / 2^e in base 2^7, with the sign of x
__device__ __forceinline__ void digits_of(double x, int e, int S, float *d) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  int ex = (int)((b >> 52) & 0x7FF);
  for (int s = 0; s < S; s++) d[s] = 0.f;
  if (ex == 0) return;
  uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  int sh = 12 + (ex - 1023) - e;  // fraction bits: frac = m << sh (sh <= 11)
  uint64_t frac;
  if (sh >= 0) frac = m << sh;
  else if (sh > -64) frac = m >> (-sh);
  else frac = 0;
  const float sg = (b >> 63) ? -1.f : 1.f;
  for (int s = 0; s < S; s++) d[s] = sg * (float)((frac >> (64 - 7 * (s + 1))) & 127u);
}

// Row exponents of a row-major matrix X [R x Kd] (ld = row stride); zero and padded rows get -2000.
__global__ void k_row_exp(const double *X, int64_t ld, int R, int Kd, int Rpad, int *e) {
  const int r = blockIdx.x * blockDim.y + threadIdx.y;
  if (r >= Rpad) return;
  int m = -2000;
  if (r < R)
    for (int k = threadIdx.x; k < Kd; k += 32) m = max(m, exp_of(fabs(X[(int64_t)r * ld + k])));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x == 0) e[r] = m;
}

// Column exponents of a row-major matrix X [Kd x C] (ld = row stride).
__global__ void k_col_exp(const double *X, int64_t ld, int Kd, int Cn, int Cpad, int *e) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cpad) return;
  int m = -2000;
  if (c < Cn)
    for (int k = 0; k < Kd; k++) m = max(m, exp_of(fabs(X[(int64_t)k * ld + c])));
  e[c] = m;
}

// Pack "rows" of an operand into slice tiles.  Element (r, k) is X[r*sr + k*sk].
// Output: planes[s][rt][kt] tiles of `rows_per_tile` x KC BF16 digits.
__global__ void k_pack(const double *X, int64_t sr, int64_t sk, int R, int Kd, int Rpad, int Kpad, const int *e,
                       int S, int rows_per_tile, __nv_bfloat16 *planes) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)Rpad * Kpad;
  if (idx >= total) return;
  const int r = (int)(idx / Kpad), k = (int)(idx % Kpad);
  const double x = (r < R && k < Kd) ? X[(int64_t)r * sr + (int64_t)k * sk] : 0.0;
  float d[MAXS];
  digits_of(x, e[r], S, d);
  const int rt = r / rows_per_tile, kt = k / KC;
  const int64_t tile_bytes = (int64_t)rows_per_tile * KC * 2;
  const int64_t ntile = (int64_t)(Rpad / rows_per_tile) * (Kpad / KC);
  const int64_t tbase = ((int64_t)rt * (Kpad / KC) + kt) * tile_bytes + tile_off(r % rows_per_tile, k % KC);
  char *base = (char *)planes;
  for (int s = 0; s < S; s++)
    *(__nv_bfloat16 *)(base + (int64_t)s * ntile * tile_bytes + tbase) = __float2bfloat16_rn(d[s]);
}

// ------------------------------------------------------------------ the GEMM
struct GemmArgs {
  const __nv_bfloat16 *A;  // planes [S][Mpad/128][Kpad/32] tiles
  const __nv_bfloat16 *B;  // planes [S][Npad/64][Kpad/32] tiles
  const int *eA, *eB;      // row / column exponents
  double *C;               // output, row-major with ldc
  int64_t ldc;
  int M, N, Mpad, Npad, Kpad, S;
  int accumulate;          // 1: C += result
  int drop;                // low bits dropped from the fixed-point sum (keeps it in 63 bits)
  int *err;                // set to 1 on a timed-out wait
};

// Bits the fixed-point sum needs: products below 2^14, at most Kpad of them per
// diagonal sum, the top diagonal shifted by 7(S-1), plus sign; keep <= 62.
__host__ __device__ inline int fixed_point_drop(int Kpad, int S) {
  int lk = 0;
  while ((1 << lk) < Kpad) lk++;
  const int bits = lk + 14 + 7 * (S - 1) + 2;  // sign plus the lower diagonals (< 2 %)
  return bits > 62 ? bits - 62 : 0;
}

__global__ void __launch_bounds__(256, 1) k_gemm_sliced(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // layout: [stage][A tiles S][B tiles S], then barriers, then TMEM address
  const int S = g.S;
  const int stage_bytes = S * (A_TILE + B_TILE);
  uint64_t *full = (uint64_t *)(smem + NSTAGE * stage_bytes);
  uint64_t *empty = full + NSTAGE;
  uint64_t *accfull = empty + NSTAGE;
  uint64_t *accempty = accfull + 1;
  uint32_t *tmem_slot = (uint32_t *)(accempty + 1);
  int *abort_flag = (int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, nt = blockIdx.y;
  const int nk = g.Kpad / KC;
  const int ngroups = (nk + GROUP - 1) / GROUP;
  const int64_t a_tiles = (int64_t)(g.Mpad / TM) * nk;  // tiles per A plane
  const int64_t b_tiles = (int64_t)(g.Npad / TN) * nk;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, 128);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {  // TMEM: S diagonals x TN columns, rounded to a power of two >= 32
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(S * TN)) ncols <<= 1;
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    for (int c = 0; c < nk; c++) {
      const int st = c % NSTAGE;
      if (c >= NSTAGE && !mbar_wait(&empty[st], ((c / NSTAGE) - 1) & 1)) {
        atomicExch(abort_flag, 1);
        break;
      }
      if (*(volatile int *)abort_flag) break;
      uint8_t *sa = smem + st * stage_bytes;
      uint8_t *sb = sa + S * A_TILE;
      mbar_expect_tx(&full[st], (uint32_t)stage_bytes);
      for (int s = 0; s < S; s++) {
        const char *ga = (const char *)g.A + ((int64_t)s * a_tiles + (int64_t)mt * nk + c) * A_TILE;
        bulk_g2s(sa + s * A_TILE, ga, A_TILE, &full[st]);
        const char *gb = (const char *)g.B + ((int64_t)s * b_tiles + (int64_t)nt * nk + c) * B_TILE;
        bulk_g2s(sb + s * B_TILE, gb, B_TILE, &full[st]);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = idesc_bf16(TM, TN);
    for (int c = 0; c < nk; c++) {
      const int st = c % NSTAGE;
      const int grp = c / GROUP;
      if (c % GROUP == 0 && grp > 0 && !mbar_wait(accempty, (grp - 1) & 1)) {
        atomicExch(abort_flag, 1);
        break;
      }
      if (!mbar_wait(&full[st], (c / NSTAGE) & 1)) {
        atomicExch(abort_flag, 1);
        break;
      }
      if (*(volatile int *)abort_flag) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + st * stage_bytes);
      const uint32_t sb = sa + S * A_TILE;
      for (int d = 2; d <= S + 1; d++) {
        const uint32_t tcol = tmem + (uint32_t)((d - 2) * TN);
        bool first = (c % GROUP == 0);
        for (int s = 1; s <= S; s++) {
          const int t = d - s;
          if (t < 1 || t > S) continue;
          for (int kk = 0; kk < KC / 16; kk++) {
            // K step kk covers core-matrix columns 2kk, 2kk+1 (LBO = 128 B apart)
            const uint64_t ad = sdesc(sa + (s - 1) * A_TILE + kk * 256, 128, (KC / 8) * 128);
            const uint64_t bd = sdesc(sb + (t - 1) * B_TILE + kk * 256, 128, (KC / 8) * 128);
            mma_bf16(tcol, ad, bd, idesc, first ? 0u : 1u);
            first = false;
          }
        }
      }
      mma_commit(&empty[st]);
      if (c % GROUP == GROUP - 1 || c == nk - 1) mma_commit(accfull);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ drain and fold
    const int q = warp - 4;              // TMEM lane quadrant
    const int row = q * 32 + lane;       // output row inside the tile
    int64_t acc[TN];
#pragma unroll
    for (int n = 0; n < TN; n++) acc[n] = 0;
    bool ok = true;
    for (int grp = 0; grp < ngroups; grp++) {
      if (!mbar_wait(accfull, grp & 1)) {
        atomicExch(abort_flag, 1);
        ok = false;
        break;
      }
      tc_fence_after();
      for (int d = 2; d <= S + 1; d++) {
        const int sh = 7 * (S + 1 - d) - g.drop;
#pragma unroll
        for (int n0 = 0; n0 < TN; n0 += 16) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((d - 2) * TN + n0), r);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int64_t v = (int64_t)__float2ll_rn(__uint_as_float(r[j]));
            acc[n0 + j] += sh >= 0 ? (v << sh) : (v >> (-sh));
          }
        }
      }
      tc_fence_before();
      mbar_arrive(accempty);
    }
    if (ok) {
      const int gr = mt * TM + row;
      if (gr < g.M) {
        const int er = g.eA[gr];
        for (int n = 0; n < TN; n++) {
          const int gc = nt * TN + n;
          if (gc >= g.N) break;
          const int sc = er + g.eB[gc] - 7 * (S + 1) + g.drop;
          double v = ldexp((double)acc[n], sc);
          double *dst = g.C + (int64_t)gr * g.ldc + gc;
          if (g.accumulate) *dst += v;
          else *dst = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*(volatile int *)abort_flag && threadIdx.x == 0) atomicExch(g.err, 1);
  if (warp == 2) {
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(S * TN)) ncols <<= 1;
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

}  // namespace rixtc

using namespace rixtc;

// C[M x N] (row-major, ldc) = A[M x K] (row-major, lda) * B[K x N] (row-major, ldb),
// all FP64 device pointers; scratch for the slices is allocated here.
extern "C" rix_status rix_gemm_sliced(const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                                      int64_t ldc, int32_t M, int32_t N, int32_t K, int32_t n_slices,
                                      void *stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || n_slices < 1 || n_slices > MAXS) return RIX_EINVAL;
  if (lda < K || ldb < N || ldc < N) return RIX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int S = n_slices;
  const int Mpad = (M + TM - 1) / TM * TM, Npad = (N + TN - 1) / TN * TN, Kpad = (K + KC - 1) / KC * KC;
  const size_t pa = (size_t)S * Mpad * Kpad * 2, pb = (size_t)S * Npad * Kpad * 2;
  void *buf = nullptr;
  const size_t bytes = pa + pb + (size_t)(Mpad + Npad) * 4 + 16;
  if (cudaMallocAsync(&buf, bytes, st) != cudaSuccess) return RIX_ENOMEM;
  __nv_bfloat16 *Ap = (__nv_bfloat16 *)buf;
  __nv_bfloat16 *Bp = (__nv_bfloat16 *)((char *)buf + pa);
  int *eA = (int *)((char *)buf + pa + pb);
  int *eB = eA + Mpad;
  int *err = eB + Npad;
  cudaMemsetAsync(err, 0, 4, st);
  k_row_exp<<<(Mpad + 7) / 8, dim3(32, 8), 0, st>>>(A, lda, M, K, Mpad, eA);
  k_col_exp<<<(Npad + 127) / 128, 128, 0, st>>>(B, ldb, K, N, Npad, eB);
  {
    const int64_t n = (int64_t)Mpad * Kpad;
    k_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, lda, 1, M, K, Mpad, Kpad, eA, S, TM, Ap);
  }
  {
    // B^T as rows: element (n, k) = B[k*ldb + n]
    const int64_t n = (int64_t)Npad * Kpad;
    k_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, 1, ldb, N, K, Npad, Kpad, eB, S, TN, Bp);
  }
  GemmArgs g{Ap, Bp, eA, eB, C, ldc, M, N, Mpad, Npad, Kpad, S, 0, fixed_point_drop(Kpad, S), err};
  const int smem = NSTAGE * S * (A_TILE + B_TILE) + 8 * (2 * NSTAGE + 2) + 16;
  cudaFuncSetAttribute(k_gemm_sliced, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_gemm_sliced<<<dim3(Mpad / TM, Npad / TN), 256, smem, st>>>(g);
  cudaError_t e = cudaGetLastError();
  int herr = 0;
  cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return RIX_ECUDA;
  if (herr) return RIX_ETIMEOUT;
  return RIX_OK;
}
