// FP64-accurate GEMM on the BF16 tensor cores (tcgen05) by error-free slicing.
//
// C = A B with A [M x K], B [K x N] in FP64.  Every row of A (column of B) is
// scaled by a power of two 2^e so that |x| < 2^e, and its 64-bit fixed-point
// fraction |x| / 2^e is written with S balanced base-2^7 digits: the leading
// one in [0, 128], the others in [-64, 63], the last rounded to nearest (all
// exact in BF16, the sign of x applied to every digit).  This is the
// error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) with
// per-row/column exponents and balanced digits.  With a = sum_s a_s 2^-7s and
// b = sum_t b_t 2^-7t,
//
//   A B = 2^(eA + eB) sum_{s+t <= S+1} 2^{-7(s+t)} (A_s B_t)
//
// and every slice product A_s B_t is a sum of integers: below 2^14 on the
// leading diagonal, 2^13 where one digit is a leading one and 2^12 otherwise.
// Slice s is stored pre-scaled by 2^-7(s-1) (exact in BF16), so a product
// carries its own power of two.  Six FP32 accumulators in tensor memory take
// the products with s+t = 2, 3, 4, 5, 6 and s+t >= 7: by those bounds the
// first five hold integers (times 2^-7(s+t-2)) below 2^24 over a group of 512
// K values, so the tensor cores accumulate them exactly; the sixth holds
// terms at least 2^-35 below the leading one, where the tensor cores' FP32
// accumulation costs about 2^-53 of the row x column x K scale.  After each
// group the accumulators are folded into a 64-bit fixed-point sum per output
// element, and the FP64 result is formed once at the end.  The error is the
// rounding of the operands to S digits (at most half a unit of 2^-7S of the
// row/column scale), the dropped terms s+t > S+1 and the rounding of the
// sixth accumulator.
//
// Kernel layout: persistent CTAs over 128 x 80 output tiles; warp 0 issues the
// bulk copies (cp.async.bulk, mbarrier completion), one thread of warp 1
// issues tcgen05.mma (A and B from shared memory, accumulators in tensor
// memory), warps 4-11 drain tensor memory (tcgen05.ld, two warps per 32-lane
// quadrant, 40 columns each) into the fixed-point sums.  Every wait is
// bounded; on a timeout the kernel records an error and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "rix_internal.h"

namespace rixtc {

constexpr int TM = 128;         // output rows per tile (one TMEM lane each)
constexpr int TN = 80;          // output columns per tile
constexpr int KC = 32;          // K per pipeline stage (two MMA K steps)
// Accumulation groups of GROUP K stages (512 K values).  Accumulator a < NACC-1
// holds diagonal a: pairs (0, a) and (a, 0) with a leading digit (<= 128)
// and a balanced one (<= 64), and a - 1 pairs of balanced digits (a = 0: the
// one pair of leading digits), so its sum stays an integer below 2^24.
constexpr int GROUP = 16;
constexpr int64_t diag_bound(int a) {  // largest |sum over one K value| of diagonal a
  return a == 0 ? 128 * 128 : 2 * 128 * 64 + (int64_t)(a - 1) * 64 * 64;
}
constexpr bool exact_group(int a) { return diag_bound(a) * GROUP * KC < ((int64_t)1 << 24); }
static_assert(exact_group(0) && exact_group(1) && exact_group(2) && exact_group(3) && exact_group(4),
              "accumulation groups must stay exact");
constexpr int NACC = 6;         // accumulators: s+t = 2 .. 6 and s+t >= 7 (480 TMEM columns)
constexpr int NTHR = 384;       // warps 0-3: copies, MMA, TMEM allocation; warps 4-11: drain
constexpr int MAXS = 8;         // slices supported
constexpr uint64_t WAIT_NS = 2000000000ull;  // a wait gives up after 2 s

// bytes of one packed tile (no-swizzle K-major core matrices, 8 rows x 16 B)
constexpr int A_TILE = TM * KC * 2;  // 8 KB
constexpr int B_TILE = TN * KC * 2;  // 5 KB

constexpr int NSTAGE = 3;            // pipeline stages when they fit in shared memory
constexpr int SMEM_LIMIT = 227 * 1024;
// Scatter epilogue staging: per drain warp 32 rows x EPI_CW values plus each row's
// output-block base and in-block row offset
constexpr int EPI_CW = 4;
constexpr int EPI_WARP_BYTES = 32 * EPI_CW * 8 + 32 * 8 + 32 * 4;
constexpr int EPI_BYTES = 8 * EPI_WARP_BYTES;

// stages that fit for S slices, and the dynamic shared memory they need
__host__ __device__ inline int n_stages(int S) {
  const int st = S * (A_TILE + B_TILE);
  const int fit = (SMEM_LIMIT - 256 - EPI_BYTES) / st;
  return fit >= NSTAGE ? NSTAGE : (fit >= 2 ? fit : 1);
}
__host__ __device__ inline int smem_bytes(int S) {
  return n_stages(S) * S * (A_TILE + B_TILE) + EPI_BYTES + 8 * (2 * NSTAGE + 4) + 16;
}

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

// bounded wait for the phase with the given parity; returns false after WAIT_NS.
// try_wait may suspend the thread for up to SUSPEND_NS until the phase completes,
// so waiting warps leave the issue slots to the copy and MMA threads.
constexpr uint32_t SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = WAIT_NS) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(SUSPEND_NS)
        : "memory");
    if (ok) return true;
    const uint64_t t = now_ns();
    if (!t0) t0 = t;
    else if (t - t0 > limit_ns) return false;
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

// The MMAs of one K stage: slice pairs (s, u) with s + u < S, each into
// accumulator min(s + u, NACC - 1), two K steps of 16.  ad0 / bd0 are the
// descriptors of slice 0 of the stage; the others follow at fixed offsets (the
// start-address field counts 16-byte units and stays below 2^14 in shared
// memory).  In this order the first MMA into every accumulator is the one with
// s = 0, kk = 0 and u <= NACC - 1; for the accumulators whose bit is set in
// open (a group of them starts at this stage) it overwrites the accumulator.
template <int S>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint64_t ad0, uint64_t bd0, uint32_t idesc,
                                            uint32_t open) {
#pragma unroll
  for (int s = 0; s < S; s++)
#pragma unroll
    for (int u = 0; u < S - s; u++) {
      const int a = s + u < NACC - 1 ? s + u : NACC - 1;
#pragma unroll
      for (int kk = 0; kk < KC / 16; kk++) {
        const uint64_t ad = ad0 + (uint64_t)((s * A_TILE + kk * 256) >> 4);
        const uint64_t bd = bd0 + (uint64_t)((u * B_TILE + kk * 256) >> 4);
        const bool first = s == 0 && kk == 0 && u <= NACC - 1;
        mma_bf16(tmem + (uint32_t)(a * TN), ad, bd, idesc, first ? 1u - ((open >> a) & 1u) : 1u);
      }
    }
}

__device__ __forceinline__ void issue_stage_s(int S, uint32_t tmem, uint64_t ad0, uint64_t bd0, uint32_t idesc,
                                              uint32_t open) {
  switch (S) {
    case 1: issue_stage<1>(tmem, ad0, bd0, idesc, open); break;
    case 2: issue_stage<2>(tmem, ad0, bd0, idesc, open); break;
    case 3: issue_stage<3>(tmem, ad0, bd0, idesc, open); break;
    case 4: issue_stage<4>(tmem, ad0, bd0, idesc, open); break;
    case 5: issue_stage<5>(tmem, ad0, bd0, idesc, open); break;
    case 6: issue_stage<6>(tmem, ad0, bd0, idesc, open); break;
    case 7: issue_stage<7>(tmem, ad0, bd0, idesc, open); break;
    default: issue_stage<8>(tmem, ad0, bd0, idesc, open); break;
  }
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// An FP32 accumulator value times 2^sh as a 64-bit integer, truncated toward
// zero, with integer operations only (the conversion instructions with a
// 64-bit side run at the FP64 rate).  The general fallback of drain_any for
// the last accumulator, which holds several diagonals and is not an integer in
// its own units; below the fixed-point unit it is truncated (< 1 unit per
// group).
__device__ __forceinline__ int64_t f32_fixed(uint32_t b, int sh) {
  const int e = (int)((b >> 23) & 0xFF);
  if (e == 0) return 0;  // zero; subnormals lie far below the fixed-point unit
  const int64_t m = (int64_t)((b & 0x7FFFFFu) | 0x800000u);
  const int s = e - 150 + sh;  // value = m 2^s
  const int64_t v = s >= 0 ? (m << (s < 39 ? s : 39)) : (s > -40 ? (m >> -s) : 0);
  return (b >> 31) ? -v : v;
}

// Drain of one exactly accumulated diagonal a into the fixed-point sums: the
// FP32 value is an integer I times 2^-7a with |I| < 2^24, so I = trunc(v 2^7a)
// is exact in a 32-bit conversion, and I 2^L (L = 7(S-1) - drop - 7a, the same
// for the whole tile) is added with one 32 x 32 -> 64-bit multiply-add: for
// 0 <= L <= 37 as (I 2^pre) 2^(L-pre) with pre = max(0, L - 30), both factors
// within 32 bits (|I 2^pre| < 2^31); other L by a 64-bit shift.
template <int N>
__device__ __forceinline__ void drain_exact(int64_t *acc, const uint32_t (&r)[N], int a, int L) {
  const float up = __int_as_float((127 + 7 * a) << 23);
  if (L >= 0 && L <= 37) {
    const int pre = L > 30 ? L - 30 : 0;
    const int32_t mul = 1 << (L - pre);
#pragma unroll
    for (int j = 0; j < N; j++) {
      const int32_t I = __float2int_rz(__uint_as_float(r[j]) * up);
      acc[j] += (int64_t)(I << pre) * (int64_t)mul;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; j++) {
      const int64_t I = __float2int_rz(__uint_as_float(r[j]) * up);
      acc[j] += L >= 0 ? (I << (L < 63 ? L : 63)) : (I >> (-L < 63 ? -L : 63));
    }
  }
}

// Drain of the last accumulator (s+t >= NACC-1, not an integer in any one
// unit): trunc(v 2^sh) in the fixed point.  For sh <= 35 one 32-bit conversion
// (|v 2^sh| < 2^31).  Otherwise x = v 2^35 (|x| < 2^25) is split exactly into
// 8 h (x + 1.5 2^26 rounds it to a multiple of 8; h is read from the bits) and
// a remainder |r| <= 4, which is scaled by 2^(sh-35) and converted; the sum of
// the two parts differs from trunc(v 2^sh) by < 1 unit.  This keeps the
// conversion unit, not the integer pipe, the busy one.
template <int N>
__device__ __forceinline__ void drain_any(int64_t *acc, const uint32_t (&r)[N], int sh) {
  if (sh <= 35) {
    const float p2 = __int_as_float((127 + sh) << 23);
#pragma unroll
    for (int j = 0; j < N; j++) acc[j] += __float2int_rz(__uint_as_float(r[j]) * p2);
  } else if (sh <= 63) {
    const float M = 100663296.f;  // 1.5 * 2^26
    const uint32_t Mb = __float_as_uint(M);
    const float p2 = __int_as_float((127 + sh - 35) << 23);
#pragma unroll
    for (int j = 0; j < N; j++) {
      const float x = __uint_as_float(r[j]) * 34359738368.f;  // 2^35
      const float t = x + M;
      const int32_t h8 = (int32_t)(__float_as_uint(t) - Mb);
      const float rem = x - (t - M);
      const int32_t lo = __float2int_rz(rem * p2);
      acc[j] += ((int64_t)h8 << (sh - 32)) + lo;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; j++) acc[j] += f32_fixed(r[j], sh);
  }
}

// x 2^sc as a double, built with integer operations (the FP64 pipe is the
// scarcest unit here): the leading 53 bits of |x|, truncated toward zero
// (relative error below 2^-52).  Exponents outside the normal range go
// through ldexp.
__device__ __forceinline__ double fixed_to_double(int64_t x, int sc) {
  if (x == 0) return 0.0;
  const uint64_t sgn = (uint64_t)x & (1ull << 63);
  const uint64_t ax = sgn ? (uint64_t)(-x) : (uint64_t)x;
  const int lz = __clzll((long long)ax);
  const int E = 1023 + 63 - lz + sc;
  if (E <= 0 || E >= 2047) return ldexp((double)x, sc);
  const uint64_t mant = ((ax << lz) >> 11) & ((1ull << 52) - 1);
  return __longlong_as_double((long long)(sgn | ((uint64_t)E << 52) | mant));
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

// |x| / 2^e as a 64-bit fixed-point fraction (0 for zero and subnormal x)
__device__ __forceinline__ uint64_t frac_of(uint64_t b, int e) {
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = 12 + (ex - 1023) - e;  // fraction bits: frac = m << sh (sh <= 11)
  return ex == 0 ? 0 : sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0);
}

// The S balanced base-2^7 digits of a fraction, leading digit first: the
// plain digits (fr >> (57 - 7t)) & 127 are rounded at digit S - 1 (the next
// bit) and folded from the last one up, a digit >= 64 becoming digit - 128
// with a carry into the one before; the leading digit takes the last carry
// and lies in [0, 128], the others in [-64, 63].
template <int S>
__device__ __forceinline__ void balanced_digits(uint64_t fr, int (&d)[S]) {
  int carry = (int)((fr >> (63 - 7 * S)) & 1u);
#pragma unroll
  for (int t = S - 1; t >= 1; t--) {
    const int c = (int)((fr >> (57 - 7 * t)) & 127u) + carry;
    carry = c >= 64;
    d[t] = c - (carry << 7);
  }
  d[0] = (int)(fr >> 57) + carry;
}

// digit s (0-based) of x: balanced digit of |x| / 2^e with the sign of x
template <int S>
__device__ __forceinline__ void digits_of(double x, int e, float (&d)[S]) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  int di[S];
  balanced_digits<S>(frac_of(b, e), di);
  const float sg = (b >> 63) ? -1.f : 1.f;
#pragma unroll
  for (int t = 0; t < S; t++) d[t] = sg * (float)di[t];
}

// 2^-7s as a float (exact): slice s (0-based) is stored pre-scaled by it
__device__ __forceinline__ float slice_scale(int s) { return __int_as_float((127 - 7 * s) << 23); }

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
template <int S>
__global__ void k_pack(const double *X, int64_t sr, int64_t sk, int R, int Kd, int Rpad, int Kpad, const int *e,
                       int rows_per_tile, __nv_bfloat16 *planes) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)Rpad * Kpad;
  if (idx >= total) return;
  const int r = (int)(idx / Kpad), k = (int)(idx % Kpad);
  const double x = (r < R && k < Kd) ? X[(int64_t)r * sr + (int64_t)k * sk] : 0.0;
  float d[S];
  digits_of<S>(x, e[r], d);
  const int rt = r / rows_per_tile, kt = k / KC;
  const int64_t tile_bytes = (int64_t)rows_per_tile * KC * 2;
  const int64_t ntile = (int64_t)(Rpad / rows_per_tile) * (Kpad / KC);
  const int64_t tbase = ((int64_t)rt * (Kpad / KC) + kt) * tile_bytes + tile_off(r % rows_per_tile, k % KC);
  char *base = (char *)planes;
#pragma unroll
  for (int t = 0; t < S; t++)
    *(__nv_bfloat16 *)(base + (int64_t)t * ntile * tile_bytes + tbase) = __float2bfloat16_rn(d[t] * slice_scale(t));
}

void launch_pack(const double *X, int64_t sr, int64_t sk, int R, int Kd, int Rpad, int Kpad, const int *e, int S,
                 int rows_per_tile, __nv_bfloat16 *planes, cudaStream_t st) {
  const int64_t n = (int64_t)Rpad * Kpad;
  const unsigned grid = (unsigned)((n + 255) / 256);
  switch (S) {
    case 1: k_pack<1><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    case 2: k_pack<2><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    case 3: k_pack<3><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    case 4: k_pack<4><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    case 5: k_pack<5><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    case 6: k_pack<6><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    case 7: k_pack<7><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
    default: k_pack<8><<<grid, 256, 0, st>>>(X, sr, sk, R, Kd, Rpad, Kpad, e, rows_per_tile, planes); break;
  }
}

// ------------------------------------------------------------------ the GEMM
// Middle atoms batched into one problem of the plans of terms 2, 3+4 and Z (at most).
constexpr int GMAX = 4;
// xmap entries of the terms-3+4 plan: output block index, with this bit set for the self
// block (A, A, 0), which takes half the weight of the other blocks
constexpr int32_t XHALF = 1 << 30;

// One problem of a batched launch: its packed operands, exponents and the
// scatter maps of its output (rows (row block q, i), columns (col block z, l)).
// In the plans of terms 2, 3+4 and Z a problem sums over ng middle atoms: its K
// axis is their contraction ranges back to back, member m at [kb[m], kb[m+1]).
struct Prob {
  int64_t aoff, boff;      // byte offsets of the A and B slice planes
  int64_t eaoff, eboff;    // offsets into the exponent arrays
  int64_t rowoff, coloff;  // offsets into rowinfo / colinfo
  int64_t xoff;            // offset into xmap ([nq][nz])
  int32_t Mpad, Npad, Kpad, M, N, nz, drop, pad_;
  int32_t ng;              // middle atoms of the problem (grouped plans)
  int32_t kb[GMAX + 1];    // their K ranges; kb[ng] = K
};

// Output row block of a term-1 problem: the K block X(A',E'), the pair (A',E')
// carrying V(A',E') (offset voff), nb of A', and whether the block takes term 1
// with weight 1/2 (the on-site pair; every other pair takes it with weight 1 in
// one orientation).
struct QInfo {
  int64_t voff;
  int32_t x, vpair, nbA, half;
};

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
  // batched scatter mode (tiles != nullptr): C, ldc, M, N, Mpad, Npad, Kpad, drop come from Prob
  const int4 *tiles;       // (problem, mt, nt, -)
  const Prob *probs;
  const int2 *rowinfo;     // (q, i) per packed row; q < 0 for padding
  const int4 *colinfo;     // (z, l, nbE, -) per packed column; z < 0 for padding
  const int32_t *xmap;     // output block index per (q, z)
  const int64_t *offK;
  double *X;               // X[offK[x] + i * nbE + l] += value (atomic)
  // mode 1 (term 1): rows (q, P nbA + i), columns (l, Q, nbE, naE) l-major;
  // X(A',E')[i][l] += oscale w sum_Q V(A',E')[P][Q] R[row][col], one atomic per l (w: QInfo)
  int mode;
  const QInfo *qinfo;      // per row block, indexed from Prob::xoff
  const double *V;
  const uint8_t *keepV;
  double oscale;           // scale of the added values (modes 0 and 1)
  int64_t xshift;          // mode 0: X + offK[x] - xshift is the output block
  int ntiles;              // output tiles of the launch (persistent CTAs loop over them)
  const uint8_t *row_live = nullptr;  // batched mode: per row tile (tiles[t].w), 0 = all its rows are zero
  // batched mode: a bit mask of the K stages to run, (Kpad / KC + 63) / 64 words per tile:
  // per (problem, column tile) at kmask + tiles[t].w (T plan: stages whose B tile is not all
  // zero), or per row tile at kmask + kmask_off[tiles[t].w] (grouped plans: stages of the
  // members that meet a kept block of the tile's rows); stages without a bit are skipped
  const unsigned long long *kmask = nullptr;
  const int64_t *kmask_off = nullptr;
  unsigned long long *chunks = nullptr;  // profiling: 128 x 80 x 16 MMAs issued (K stages x K steps x slice pairs)
  unsigned long long *X128 = nullptr;  // deterministic mode: X additions as 128-bit fixed point (2 words each)
  uint64_t wait_ns = WAIT_NS;  // limit of every bounded wait
  int stall = 0;           // 1: the MMA issuer waits on a barrier nothing completes (timeout test)
};

// X(output block x)[el] += v: an FP64 atomic, or the 128-bit fixed-point addition of a
// deterministic build
__device__ __forceinline__ void x_add(const GemmArgs &g, int x, int64_t el, double v) {
  const int64_t o = g.offK[x] + el;
  if (g.X128) rix::add_x128(g.X128 + 2 * o, rix::to_x128(v));
  else atomicAdd(g.X + o, v);
}

// Bits the fixed-point sum needs: products below 2^14, at most Kpad of them in
// the leading diagonal, scaled up by 7(S-1), plus sign and the lower
// diagonals (< 2 %); keep <= 62.
__host__ __device__ inline int fixed_point_drop(int Kpad, int S) {
  int lk = 0;
  while ((1 << lk) < Kpad) lk++;
  const int bits = lk + 14 + 7 * (S - 1) + 2;  // sign plus the lower diagonals (< 2 %)
  return bits > 62 ? bits - 62 : 0;
}

// Operands and sizes of output tile t (dense: t = nt * (Mpad / TM) + mt).
struct TileInfo {
  const Prob *pr;
  const __nv_bfloat16 *gA, *gB;
  const int *geA, *geB;
  int mt, nt, Mpad, Npad, Kpad, M, N, drop;
  bool live;  // false: the tile's A rows are all zero (screened), every role skips it
  const unsigned long long *km;  // live K stages (nullptr: all)
  int nlive;                      // number of live K stages
};

__device__ __forceinline__ bool stage_live(const TileInfo &ti, int c) {
  return !ti.km || ((ti.km[c >> 6] >> (c & 63)) & 1ull);
}

__device__ __forceinline__ TileInfo tile_info(const GemmArgs &g, int t) {
  TileInfo ti;
  if (g.tiles) {
    const int4 tt = g.tiles[t];
    const Prob *pr = g.probs + tt.x;
    ti.pr = pr;
    ti.mt = tt.y;
    ti.nt = tt.z;
    ti.gA = (const __nv_bfloat16 *)((const char *)g.A + pr->aoff);
    ti.gB = (const __nv_bfloat16 *)((const char *)g.B + pr->boff);
    ti.geA = g.eA + pr->eaoff;
    ti.geB = g.eB + pr->eboff;
    ti.Mpad = pr->Mpad; ti.Npad = pr->Npad; ti.Kpad = pr->Kpad; ti.M = pr->M; ti.N = pr->N; ti.drop = pr->drop;
    ti.live = !g.row_live || g.row_live[tt.w];
    ti.km = nullptr;
    ti.nlive = ti.Kpad / KC;
    if (g.kmask) {
      ti.km = g.kmask + (g.kmask_off ? g.kmask_off[tt.w] : (int64_t)tt.w);
      int n = 0;
      for (int w = 0; w < (ti.nlive + 63) / 64; w++) n += __popcll(ti.km[w]);
      ti.nlive = n;
      ti.live = ti.live && n > 0;
    }
  } else {
    const int mtiles = g.Mpad / TM;
    ti.pr = nullptr;
    ti.mt = t % mtiles;
    ti.nt = t / mtiles;
    ti.gA = g.A; ti.gB = g.B; ti.geA = g.eA; ti.geB = g.eB;
    ti.Mpad = g.Mpad; ti.Npad = g.Npad; ti.Kpad = g.Kpad; ti.M = g.M; ti.N = g.N; ti.drop = g.drop;
    ti.live = true;
    ti.km = nullptr;
    ti.nlive = ti.Kpad / KC;
  }
  return ti;
}

// Persistent: CTA b handles tiles b, b + gridDim.x, ...  The shared-memory stage
// ring and the accumulator barriers run on across tiles, so the copies and the
// MMAs of a tile overlap the previous tile's epilogue (the drain warps release
// tensor memory before they convert and scatter their sums).
__global__ void __launch_bounds__(NTHR, 1) k_gemm_sliced(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // layout: [stage][A tiles S][B tiles S], the scatter staging of the drain warps,
  // then barriers, then TMEM address
  const int S = g.S;
  const int stage_bytes = S * (A_TILE + B_TILE);
  const int nst = n_stages(S);
  uint8_t *epi = smem + nst * stage_bytes;
  uint64_t *full = (uint64_t *)(epi + EPI_BYTES);
  uint64_t *empty = full + NSTAGE;
  uint64_t *accfull = empty + NSTAGE;
  uint64_t *accempty = accfull + 1;
  uint64_t *mmadone = accempty + 1;  // the MMA issuer's last commit (no MMA in flight at exit)
  uint64_t *never = mmadone + 1;     // completed by nothing: the stall of the timeout test
  uint32_t *tmem_slot = (uint32_t *)(never + 1);
  int *abort_flag = (int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = g.ntiles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, NTHR - 128);
    mbar_init(mmadone, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int nacc = S < NACC ? S : NACC;
  if (warp == 2) {  // TMEM: nacc accumulators x TN columns, rounded to a power of two >= 32
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(nacc * TN)) ncols <<= 1;
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t issued_chunks = 0;  // producer thread: chunks whose copies it issued

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    uint32_t cg = 0;  // chunks issued by this CTA
    bool aborted = false;
    for (int t = blockIdx.x; t < ntiles && !aborted; t += gridDim.x) {
      const TileInfo ti = tile_info(g, t);
      if (!ti.live) continue;  // all-zero rows: no copies (the other roles skip it too)
      const int nk = ti.Kpad / KC;
      const int64_t a_tiles = (int64_t)(ti.Mpad / TM) * nk;  // tiles per A plane
      const int64_t b_tiles = (int64_t)(ti.Npad / TN) * nk;
      for (int c = 0; c < nk; c++) {
        if (!stage_live(ti, c)) continue;  // an all-zero B tile: neither copied nor multiplied
        const int st = cg % nst;
        if (cg >= (uint32_t)nst && !mbar_wait(&empty[st], ((cg / nst) - 1) & 1, g.wait_ns)) {
          atomicExch(abort_flag, 1);
          aborted = true;
          break;
        }
        if (*(volatile int *)abort_flag) {
          aborted = true;
          break;
        }
        uint8_t *sa = smem + st * stage_bytes;
        uint8_t *sb = sa + S * A_TILE;
        mbar_expect_tx(&full[st], (uint32_t)stage_bytes);
        for (int s = 0; s < S; s++) {
          const char *ga = (const char *)ti.gA + ((int64_t)s * a_tiles + (int64_t)ti.mt * nk + c) * A_TILE;
          bulk_g2s(sa + s * A_TILE, ga, A_TILE, &full[st]);
          const char *gb = (const char *)ti.gB + ((int64_t)s * b_tiles + (int64_t)ti.nt * nk + c) * B_TILE;
          bulk_g2s(sb + s * B_TILE, gb, B_TILE, &full[st]);
        }
        cg++;
      }
      if (*(volatile int *)abort_flag) aborted = true;
    }
    issued_chunks = cg;
    if (g.chunks && cg)
      atomicAdd(g.chunks, (unsigned long long)cg * (unsigned long long)(S * (S + 1) / 2) * (KC / 16));
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = idesc_bf16(TM, TN);
    uint32_t cg = 0, gg = 0;  // chunks consumed, accumulation groups completed
    bool issued = false;
    if (g.stall && !mbar_wait(never, 0, g.wait_ns)) atomicExch(abort_flag, 1);
    for (int t = blockIdx.x; t < ntiles && !*(volatile int *)abort_flag; t += gridDim.x) {
      const TileInfo ti = tile_info(g, t);
      if (!ti.live) continue;
      const int nk = ti.Kpad / KC;
      int lc = 0;  // live K stages issued for this tile
      for (int c = 0; c < nk; c++) {
        if (!stage_live(ti, c)) continue;
        const int st = cg % nst;
        if (lc % GROUP == 0 && gg > 0 && !mbar_wait(accempty, (gg - 1) & 1, g.wait_ns)) {
          atomicExch(abort_flag, 1);
          break;
        }
        if (!mbar_wait(&full[st], (cg / nst) & 1, g.wait_ns)) {
          atomicExch(abort_flag, 1);
          break;
        }
        if (*(volatile int *)abort_flag) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * stage_bytes);
        const uint32_t sb = sa + S * A_TILE;
        // K step kk covers core-matrix columns 2kk, 2kk+1 (LBO = 128 B apart)
        const uint32_t open = lc % GROUP == 0 ? 0xFFu : 0u;  // every accumulator starts a group
        issue_stage_s(S, tmem, sdesc(sa, 128, (KC / 8) * 128), sdesc(sb, 128, (KC / 8) * 128), idesc, open);
        issued = true;
        mma_commit(&empty[st]);
        if (lc % GROUP == GROUP - 1 || lc == ti.nlive - 1) {
          mma_commit(accfull);
          gg++;
        }
        lc++;
        cg++;
      }
      if (*(volatile int *)abort_flag) break;
    }
    if (issued) {
      // every MMA this thread issued has completed before tensor memory is freed
      mma_commit(mmadone);
      mbar_wait(mmadone, 0);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ drain, fold, epilogue
    constexpr int HN = TN / 2;           // columns per drain warp
    const int q = warp & 3;              // TMEM lane quadrant (a warp reaches lanes 32 (warp % 4) ..)
    const int h = (warp - 4) >> 2;       // column half
    const int row = q * 32 + lane;       // output row inside the tile
    uint32_t gg = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TileInfo ti = tile_info(g, t);
      if (!ti.live) continue;  // its output is zero: nothing to drain or add
      const int ngroups = (ti.nlive + GROUP - 1) / GROUP;  // accumulation groups of live K stages
      const int mt = ti.mt, nt = ti.nt, drop = ti.drop, Ncols = ti.N;
      const Prob *pr = ti.pr;
      const int *geA = ti.geA, *geB = ti.geB;
      // accumulator units -> fixed point: scale by 2^(7(S-1) - drop)
      const int fsh = 7 * (S - 1) - drop;
      const int nexact = S < NACC ? S : NACC - 1;  // accumulators holding one diagonal, exactly
      int64_t acc[HN];
#pragma unroll
      for (int n = 0; n < HN; n++) acc[n] = 0;
      for (int grp = 0; grp < ngroups; grp++, gg++) {
        // warp-uniform outcome: the tensor-memory loads and the scatter below are warp-collective
        if (!__all_sync(0xffffffffu, mbar_wait(accfull, gg & 1, g.wait_ns))) {
          atomicExch(abort_flag, 1);
          ok = false;
          break;
        }
        tc_fence_after();
        static_assert(HN == 40, "drain loads: 16 + 16 + 8 columns");
        for (int a = 0; a < nacc; a++) {
          // all loads of the accumulator in flight before one wait
          const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * TN + h * HN);
          uint32_t r0[16], r1[16], r2[8];
          tmem_ld16(ta, r0);
          tmem_ld16(ta + 16, r1);
          tmem_ld8(ta + 32, r2);
          tmem_wait_ld();
          if (a < nexact) {
            drain_exact(acc, r0, a, fsh - 7 * a);
            drain_exact(acc + 16, r1, a, fsh - 7 * a);
            drain_exact(acc + 32, r2, a, fsh - 7 * a);
          } else {
            drain_any(acc, r0, fsh);
            drain_any(acc + 16, r1, fsh);
            drain_any(acc + 32, r2, fsh);
          }
        }
        tc_fence_before();
        mbar_arrive(accempty);  // tensor memory free for the next group (or tile)
      }
      if (!ok) break;
      const int gr = mt * TM + row;
      if (pr && g.mode == 0) {
        // Batched scatter.  A lane holds one output row; the rows of a warp lie nbE (or nbG)
        // elements apart in the output, so row-wise additions touch one sector each.  The
        // warp therefore stages EPI_CW columns of its 32 rows in shared memory and adds them
        // with the lanes running along the columns: EPI_CW consecutive output elements per
        // row, a few sectors per warp-wide reduction.
        uint8_t *wb = epi + (warp - 4) * EPI_WARP_BYTES;
        double *sv = (double *)wb;
        int64_t *sxb = (int64_t *)(wb + 32 * EPI_CW * 8);
        int *sry = (int *)(wb + 32 * EPI_CW * 8 + 32 * 8);
        int64_t xbase = -1;
        int ry = 0, er = 0;
        if (gr < ti.M) {
          const int2 ri = g.rowinfo[pr->rowoff + gr];
          if (ri.x >= 0) {
            xbase = pr->xoff + (int64_t)ri.x * pr->nz;
            ry = ri.y;
            er = geA[gr];
          }
        }
        sxb[lane] = xbase;
        sry[lane] = ry;
        const int cbase = nt * TN + h * HN;
#pragma unroll
        for (int c0 = 0; c0 < HN; c0 += EPI_CW) {
#pragma unroll
          for (int j = 0; j < EPI_CW; j++) {
            const int gc = cbase + c0 + j;
            double v = 0.0;
            if (xbase >= 0 && gc < Ncols) v = fixed_to_double(acc[c0 + j], er + geB[gc] - 7 * (S + 1) + drop);
            sv[lane * EPI_CW + j] = v;
          }
          __syncwarp();
#pragma unroll
          for (int it = 0; it < EPI_CW; it++) {
            const int r = it * (32 / EPI_CW) + lane / EPI_CW, j = lane % EPI_CW;
            const int gc = cbase + c0 + j;
            const int64_t xb = sxb[r];
            if (xb >= 0 && gc < Ncols) {
              const int4 ci = g.colinfo[pr->coloff + gc];
              // xmap < 0: no middle atom of the problem joins this row and column block, or
              // the block is left to its transpose partner
              const int32_t xi = ci.x >= 0 ? g.xmap[xb + ci.x] : -1;
              if (xi >= 0) {
                const int64_t o = (g.offK[xi & ~XHALF] - g.xshift) + (int64_t)sry[r] * ci.z + ci.y;
                const double v = (xi & XHALF ? 0.5 * g.oscale : g.oscale) * sv[r * EPI_CW + j];
                if (g.X128) rix::add_x128(g.X128 + 2 * o, rix::to_x128(v));
                else atomicAdd(g.X + o, v);
              }
            }
          }
          __syncwarp();
        }
      } else if (gr < ti.M) {
        const int er = geA[gr];
        // fully unrolled with predicates so acc[] stays in registers
        if (!pr) {
#pragma unroll
          for (int n = 0; n < HN; n++) {
            const int gc = nt * TN + h * HN + n;
            if (gc < Ncols) {
              const int sc = er + geB[gc] - 7 * (S + 1) + drop;
              const double v = fixed_to_double(acc[n], sc);
              double *dst = g.C + (int64_t)gr * g.ldc + gc;
              if (g.accumulate) *dst += v;
              else *dst = v;
            }
          }
        } else if (g.mode == 1) {
          const int2 ri = g.rowinfo[pr->rowoff + gr];
          if (ri.x >= 0) {
            const QInfo qi = g.qinfo[pr->xoff + ri.x];
            if (g.keepV[qi.vpair]) {
              const double osc = qi.half ? 0.5 * g.oscale : g.oscale;
              const int P = ri.y / qi.nbA, i = ri.y - P * qi.nbA;
              int lcur = -1, nbE = 0;
              double part = 0.0;
#pragma unroll
              for (int n = 0; n < HN; n++) {
                const int gc = nt * TN + h * HN + n;
                if (gc < Ncols) {
                  const int4 ci = g.colinfo[pr->coloff + gc];  // (l, Q, nbE, naE)
                  if (ci.x >= 0) {
                    if (ci.x != lcur) {
                      if (lcur >= 0) x_add(g, qi.x, (int64_t)i * nbE + lcur, osc * part);
                      lcur = ci.x;
                      nbE = ci.z;
                      part = 0.0;
                    }
                    const int sc = er + geB[gc] - 7 * (S + 1) + drop;
                    part = fma(g.V[qi.voff + (int64_t)P * ci.w + ci.y], fixed_to_double(acc[n], sc), part);
                  }
                }
              }
              if (lcur >= 0) x_add(g, qi.x, (int64_t)i * nbE + lcur, osc * part);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*(volatile int *)abort_flag) {
    if (warp == 0 && lane == 0) {
      // after an abort the MMAs may not have consumed every chunk: no bulk copy may
      // still be writing shared memory when the CTA exits, so wait (bounded) for the
      // last chunk issued on every stage (earlier ones completed before their stage
      // was reused)
      const uint32_t cg = issued_chunks;
      const uint32_t first = cg > (uint32_t)nst ? cg - (uint32_t)nst : 0u;
      for (uint32_t c2 = first; c2 < cg; c2++) mbar_wait(&full[c2 % nst], (c2 / nst) & 1);
      *(volatile int *)g.err = 1;  // may be mapped host memory
    }
    __syncthreads();
  }
  if (warp == 2) {
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(nacc * TN)) ncols <<= 1;
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

// CTAs of a persistent launch: one per SM (the kernel's shared memory allows one)
inline int persistent_grid(int64_t ntiles) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  return (int)std::min<int64_t>(ntiles, nsm);
}

}  // namespace rixtc

using namespace rixtc;

// C[M x N] (row-major, ldc) = A[M x K] (row-major, lda) * B[K x N] (row-major, ldb),
// all FP64 device pointers; scratch for the slices is allocated here.  stall and
// wait_ns serve the timeout test only (rix_test_stalled_gemm).
static rix_status gemm_sliced_impl(const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                                   int64_t ldc, int32_t M, int32_t N, int32_t K, int32_t n_slices,
                                   cudaStream_t st, int stall, uint64_t wait_ns, int *ext_err) {
  const int S = n_slices;
  const int Mpad = (M + TM - 1) / TM * TM, Npad = (N + TN - 1) / TN * TN, Kpad = (K + KC - 1) / KC * KC;
  const size_t pa = (size_t)S * Mpad * Kpad * 2, pb = (size_t)S * Npad * Kpad * 2;
  void *buf = nullptr;
  const size_t bytes = pa + pb + (size_t)(Mpad + Npad) * 4 + 16;
  if (cudaMallocAsync(&buf, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return RIX_ENOMEM;
  }
  __nv_bfloat16 *Ap = (__nv_bfloat16 *)buf;
  __nv_bfloat16 *Bp = (__nv_bfloat16 *)((char *)buf + pa);
  int *eA = (int *)((char *)buf + pa + pb);
  int *eB = eA + Mpad;
  int *err = ext_err ? ext_err : eB + Npad;
  cudaError_t e = ext_err ? cudaSuccess : cudaMemsetAsync(err, 0, 4, st);
  if (e == cudaSuccess) {
    k_row_exp<<<(Mpad + 7) / 8, dim3(32, 8), 0, st>>>(A, lda, M, K, Mpad, eA);
    k_col_exp<<<(Npad + 127) / 128, 128, 0, st>>>(B, ldb, K, N, Npad, eB);
    launch_pack(A, lda, 1, M, K, Mpad, Kpad, eA, S, TM, Ap, st);
    launch_pack(B, 1, ldb, N, K, Npad, Kpad, eB, S, TN, Bp, st);  // B^T as rows: element (n, k) = B[k*ldb + n]
    GemmArgs g{Ap, Bp, eA, eB, C, ldc, M, N, Mpad, Npad, Kpad, S, 0, fixed_point_drop(Kpad, S), err,
               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    g.ntiles = (Mpad / TM) * (Npad / TN);
    g.stall = stall;
    g.wait_ns = wait_ns;
    const int smem = smem_bytes(S);
    // the same (largest) limit the build's launches set: a smaller one would make
    // their later launches with more slices fail
    e = cudaFuncSetAttribute(k_gemm_sliced, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    if (e == cudaSuccess) {
      k_gemm_sliced<<<persistent_grid(g.ntiles), NTHR, smem, st>>>(g);
      e = cudaGetLastError();
    }
  }
  int herr = 0;
  if (ext_err) {  // asynchronous: the status goes to the caller's status word
    const cudaError_t ef = cudaFreeAsync(buf, st);
    return (e == cudaSuccess && ef == cudaSuccess) ? RIX_OK : RIX_ECUDA;
  }
  // the kernel's status is read only after the stream has finished without a CUDA error
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
  const cudaError_t ef = cudaFreeAsync(buf, st);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) {
    return RIX_ECUDA;
  }
  return herr ? RIX_ETIMEOUT : RIX_OK;
}

extern "C" rix_status rix_gemm_sliced(const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                                      int64_t ldc, int32_t M, int32_t N, int32_t K, int32_t n_slices,
                                      void *stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || n_slices < 1 || n_slices > MAXS) return RIX_EINVAL;
  if (lda < K || ldb < N || ldc < N) return RIX_EINVAL;
  return gemm_sliced_impl(A, lda, B, ldb, C, ldc, M, N, K, n_slices, (cudaStream_t)stream, 0, WAIT_NS, nullptr);
}

extern "C" rix_status rix_test_stalled_gemm(rix_ctx *ctx, int64_t wait_ns, void *stream) {
  if (wait_ns <= 0 || wait_ns > (int64_t)WAIT_NS) return RIX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int M = 130, N = 90, K = 70;  // two row tiles, two column tiles, three K stages
  double *buf = nullptr;
  const size_t n = (size_t)M * K + (size_t)K * N + (size_t)M * N;
  if (cudaMallocAsync((void **)&buf, n * sizeof(double), st) != cudaSuccess) {
    cudaGetLastError();
    return RIX_ENOMEM;
  }
  cudaMemsetAsync(buf, 0, n * sizeof(double), st);
  rix_status s = gemm_sliced_impl(buf, K, buf + (size_t)M * K, N, buf + (size_t)M * K + (size_t)K * N, N, M, N, K,
                                  3, st, 1, (uint64_t)wait_ns, ctx ? ctx->d_err : nullptr);
  if (cudaFreeAsync(buf, st) != cudaSuccess) return RIX_ECUDA;
  if (ctx) return s;  // reported later by rix_check or the next entry point
  if (cudaStreamSynchronize(st) != cudaSuccess) return RIX_ECUDA;
  return s;
}

// ==========================================================================
// Batched sliced GEMMs of the build, one problem per middle atom (and, where
// the intermediate is resident per memory-plan block, per block of rows):
//
//   terms 3+4 (middle atom B):  X(A,E') += sum_{P on B, j} C(A,B')[P][i][j] Z(B,E')[P][j][l]
//     rows (A', i) over B's neighbours A' != B, K = (P, j), columns (E', l) over B's Z blocks;
//   term 2 (middle atom G):     X(A,E') += sum_{Q on G, k} U2(A,G')[Q][i][k] C(G',E')[Q on G][k][l]
//     rows (A', i) over G's neighbours (U2 of the pair (A', G)), K = (Q, k),
//     columns (E', l) over G's neighbours E' != G;
//   term 4 intermediate (middle atom G, rows of one block):
//     Z(B,E')[P][j][l] += 1/2 sum_{Q on G, k} V(B,G')[P][Q] D(B,G')[j][k] C(G',E')[Q on G][k][l]
//     rows (B, P, j), K = (Q, k), columns (E', l) as for term 2.  The row
//     operand is the Kronecker product of the V and D blocks, formed while
//     slicing; this costs about nb_B times the FLOPs of the FP64 grouping, so a
//     middle atom runs here only where its estimated tensor time is lower.
//
// Both operands are sliced per build into one reusable buffer, a group of
// consecutive problems at a time; results are added with FP64 atomics.
// ==========================================================================
namespace rixtc {

// One packed row (A operand) or column (B operand): element k < K of it is
//   X[off - shift + o * outer + in * inner_st] * (off2 < 0 ? 1 : X2[off2 + in]),
// o = k / inner_n, in = k % inner_n.  off < 0 marks padding; flag >= 0 zeroes
// the row unless keep[flag] (and keep2[flag] when given).
struct Src {
  int64_t off, off2;
  int32_t outer, inner_st, inner_n, flag;
};

// ---------------------------------------------------------------- slicing in two passes
// Pass 1 (one warp per packed row/column): the exponent of its largest |x|.
// Pass 2 (one warp per 8 packed rows): lane -> row (lane & 7) and 8 consecutive
// K values, so each warp writes whole core-matrix rows (16 B per slice, 256 B
// contiguous per warp and slice).  The accessor gives element k of packed row w.
template <class Acc>
__global__ void k_slice_exp(int64_t n0, int64_t n, Acc acc, int *e) {
  const int64_t w = n0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n0 + n) return;
  const typename Acc::Row R = acc.row(w);
  int m = -2000;
  // four elements per lane in flight (their gathers are independent)
  for (int k = lane; k < R.pr.Kpad; k += 128) {
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = k + 32 * j < R.pr.Kpad ? acc.at(R, k + 32 * j) : 0.0;
#pragma unroll
    for (int j = 0; j < 4; j++) m = max(m, exp_of(fabs(v[j])));
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) e[(acc.is_b ? R.pr.eboff : R.pr.eaoff) + R.r] = m;
}

// Digit t of two values as a packed BF16 pair (low half: x0), with integer
// and FMA-pipe operations only (the conversion unit is the scarce one): the
// balanced digit d (|d| <= 128) is made exact in FP32 by adding it to the bits
// of 1.5 2^23, scaled by 2^-7t in the same FMA (exact: at most 8 significant
// bits, 128 being a power of two), and its top 16 bits are its BF16 encoding;
// the signs of the values are applied to the pair at the end.
template <int S>
__device__ __forceinline__ void digit_pairs(double x0, double x1, int e, uint32_t (&w)[S]) {
  int d[2][S];
  uint32_t sg = 0;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const uint64_t b = (uint64_t)__double_as_longlong(h ? x1 : x0);
    balanced_digits<S>(frac_of(b, e), d[h]);
    sg |= (uint32_t)(b >> 63) << (15 + 16 * h);
  }
#pragma unroll
  for (int t = 0; t < S; t++) {
    const float sc = __int_as_float((127 - 7 * t) << 23);  // 2^-7t
    const float f0 = __fmaf_rn(__uint_as_float(0x4B400000u + (uint32_t)d[0][t]), sc, -12582912.f * sc);
    const float f1 = __fmaf_rn(__uint_as_float(0x4B400000u + (uint32_t)d[1][t]), sc, -12582912.f * sc);
    w[t] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632) ^ sg;
  }
}

// Element access of the digit pass, eight consecutive K values at a time, and whether
// the GEMM reads the K stage at all.  Accessors with cheaper forms overload these
// (found by argument-dependent lookup when the kernel is instantiated).
template <class Acc>
__device__ __forceinline__ void load8(const Acc &acc, const typename Acc::Row &R, int k0, double (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; j++) v[j] = acc.at(R, k0 + j);
}
template <class Acc>
__device__ __forceinline__ bool dig_live(const Acc &, const typename Acc::Row &, int) {
  return true;
}

template <class Acc, int S>
__global__ void k_slice_dig(int64_t n0, int64_t n, Acc acc, __nv_bfloat16 *planes, const int *e) {
  const int64_t g8 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g8 * 8 >= n) return;  // n is a multiple of 8 (problems pad to whole tiles)
  const int64_t w = n0 + g8 * 8 + (lane & 7);
  const typename Acc::Row R = acc.row(w);
  const int m = e[(acc.is_b ? R.pr.eboff : R.pr.eaoff) + R.r];
  const int trows = acc.is_b ? TN : TM, tbytes = acc.is_b ? B_TILE : A_TILE;
  const int rows_pad = acc.is_b ? R.pr.Npad : R.pr.Mpad;
  const int nkt = R.pr.Kpad / KC;
  char *base = (char *)planes + (acc.is_b ? R.pr.boff : R.pr.aoff);
  const int64_t plane = (int64_t)(rows_pad / trows) * nkt * tbytes;
  const int rt = R.r / trows, rr = R.r % trows;
  for (int k0 = (lane >> 3) * 8; k0 < R.pr.Kpad; k0 += 32) {
    if (!dig_live(acc, R, k0)) continue;  // a stage the GEMM skips: its tile is never read
    // the eight loads first (independent, so their latencies overlap), then the digits
    double v[8];
    load8(acc, R, k0, v);
    uint32_t pk[4][S];
#pragma unroll
    for (int j = 0; j < 4; j++) digit_pairs<S>(v[2 * j], v[2 * j + 1], m, pk[j]);
    const int64_t off = ((int64_t)rt * nkt + k0 / KC) * tbytes + tile_off(rr, k0 % KC);
#pragma unroll
    for (int t = 0; t < S; t++)
      *reinterpret_cast<uint4 *>(base + t * plane + off) = make_uint4(pk[0][t], pk[1][t], pk[2][t], pk[3][t]);
  }
}

// exponents and digit planes of rows [n0, n0 + n) (n a multiple of 8): the exponent pass,
// then the digit pass
template <class Acc>
void slice_rows(int64_t n0, int64_t n, const Acc &acc, int S, __nv_bfloat16 *planes, int *e, int kmax,
                cudaStream_t st);

// k_slice_dig over rows [n0, n0 + n) (n a multiple of 8) for S slices
template <class Acc>
void launch_slice_dig(int64_t n0, int64_t n, const Acc &acc, int S, __nv_bfloat16 *planes, const int *e,
                      cudaStream_t st) {
  const unsigned grid = (unsigned)((n / 8 * 32 + 255) / 256);
  switch (S) {
    case 1: k_slice_dig<Acc, 1><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    case 2: k_slice_dig<Acc, 2><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    case 3: k_slice_dig<Acc, 3><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    case 4: k_slice_dig<Acc, 4><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    case 5: k_slice_dig<Acc, 5><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    case 6: k_slice_dig<Acc, 6><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    case 7: k_slice_dig<Acc, 7><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
    default: k_slice_dig<Acc, 8><<<grid, 256, 0, st>>>(n0, n, acc, planes, e); break;
  }
}

template <class Acc>
void slice_rows(int64_t n0, int64_t n, const Acc &acc, int S, __nv_bfloat16 *planes, int *e, int,
                cudaStream_t st) {
  if (n <= 0) return;
  k_slice_exp<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(n0, n, acc, e);
  launch_slice_dig(n0, n, acc, S, planes, e, st);
}

// element access of the plans of terms 2, 3+4 and Z: packed row (or column) w
// has one Src record per middle atom of its problem (G records per row, off < 0
// where the atom does not meet the row), and K value k lies in the range of
// member m, kb[m] <= k < kb[m+1]
struct SrcAcc {
  const int64_t *prob_of;
  const Prob *probs;
  const Src *src;
  int G;
  const double *X;
  int64_t shift;
  const double *X2;
  const uint8_t *keep, *keep2;
  int is_b;
  struct Row {
    Prob pr;
    const Src *s;
    int r;
  };
  __device__ Row row(int64_t w) const {
    Row R;
    R.pr = probs[prob_of[w]];
    R.s = src + w * G;
    R.r = (int)(w - (is_b ? R.pr.coloff : R.pr.rowoff));
    return R;
  }
  __device__ double at(const Row &R, int k) const {
    if (k >= R.pr.pad_) return 0.0;
    // member of k (kb[j] = K for j >= ng; constant indices keep the record in registers)
    static_assert(GMAX == 4, "member search");
    const int m = (k >= R.pr.kb[1]) + (k >= R.pr.kb[2]) + (k >= R.pr.kb[3]);
    const int k0 = m == 0 ? 0 : m == 1 ? R.pr.kb[1] : m == 2 ? R.pr.kb[2] : R.pr.kb[3];
    const Src sr = R.s[m];
    if (sr.off < 0 || (sr.flag >= 0 && !(keep[sr.flag] && (!keep2 || keep2[sr.flag])))) return 0.0;
    const int kl = k - k0;
    const int o = kl / sr.inner_n, in = kl - o * sr.inner_n;
    const double v = X[sr.off - shift + (int64_t)o * sr.outer + (int64_t)in * sr.inner_st];
    return sr.off2 >= 0 ? v * X2[sr.off2 + in] : v;
  }
};

// Row exponents of the Z plan's Kronecker rows, one thread per packed row: row
// (B, P, j) holds V(B,G'_k)[P][Q] D(B,G'_k)[j][k'] over member k's range, so its
// largest magnitude is max_k (max_Q |V[P][Q]|) (max_k' |D[j][k']|), attained by
// the product of the two maximising entries: the same FP64 product, hence the same
// exponent, as the element-wise pass, from na + nb loads per member instead of
// na nb products.
__global__ void k_kron_exp(int64_t n0, int64_t n, SrcAcc acc, int *e) {
  const int64_t w = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= n0 + n) return;
  const SrcAcc::Row R = acc.row(w);
  int m = -2000;
  for (int k = 0; k < R.pr.ng; k++) {
    const Src sr = R.s[k];
    if (sr.off < 0 || (sr.flag >= 0 && !(acc.keep[sr.flag] && (!acc.keep2 || acc.keep2[sr.flag])))) continue;
    const int kn = (k == 0 ? R.pr.kb[1] : k == 1 ? R.pr.kb[2] - R.pr.kb[1] : k == 2 ? R.pr.kb[3] - R.pr.kb[2]
                                                                                   : R.pr.kb[4] - R.pr.kb[3]);
    const int nq = kn / sr.inner_n;
    double mv = 0.0, md = 0.0;
    for (int q = 0; q < nq; q++) mv = fmax(mv, fabs(acc.X[sr.off - acc.shift + (int64_t)q * sr.outer]));
    for (int i = 0; i < sr.inner_n; i++) md = fmax(md, fabs(acc.X2[sr.off2 + i]));
    m = max(m, exp_of(mv * md));
  }
  e[R.pr.eaoff + R.r] = m;
}

// Per row tile r of a grouped plan, for this build: bit c of its K-stage mask is set
// when a row of the tile has a kept block with a middle atom whose K range meets
// stage c (entries (pair, first stage | last stage << 16) in rtq), and live[r] tells
// whether any bit is.  A pair is kept when keep (and keep2) flag it; with product
// screening (Z plan) a pair (B, G') also counts as dead when |V| |D| times the
// largest C block of G' is below the threshold.
__global__ void k_rt_mask(int64_t n, const int2 *rt, const int2 *rtq, const int64_t *rtkw, const uint8_t *keep,
                          const uint8_t *keep2, const int32_t *pB, const float *maxCatom, rix::PScreen ps,
                          unsigned long long *kmask, uint8_t *live) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int2 e = rt[r];
  unsigned long long *m = kmask + rtkw[r];
  const int nw = (int)(rtkw[r + 1] - rtkw[r]);
  for (int w = 0; w < nw; w++) m[w] = 0ull;
  uint8_t v = 0;
  for (int i = 0; i < e.y; i++) {
    const int2 x = rtq[e.x + i];
    const int q = x.x;
    bool ok = keep[q] && (!keep2 || keep2[q]);
    if (ok && ps.tau > 0.f && ps.nD) ok = !(ps.nV[q] * ps.nD[q] * maxCatom[pB[q]] < ps.tau);
    if (!ok) continue;
    v = 1;
    const int lo = x.y & 0xFFFF, hi = x.y >> 16;  // stages lo..hi
    for (int w = lo >> 6; w <= hi >> 6; w++) {
      const int a = max(lo - 64 * w, 0), b = min(hi - 64 * w, 63);
      const unsigned long long bits = (b == 63 ? ~0ull : ((1ull << (b + 1)) - 1)) & ~((1ull << a) - 1);
      m[w] |= bits;
    }
  }
  live[r] = v;
}

__global__ void k_flag_set(int n, const int32_t *idx, uint8_t *flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) flags[idx[t]] = 1;
}

}  // namespace rixtc

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <vector>

// Host and device state of one batched plan.
struct rix_mx_plan {
  int kind = 0;                          // 0: terms 3+4, 1: term 2, 2: term-4 intermediate Z
  int S = 6;                             // slices of this plan
  int G = 1;                             // Src records per packed row / column (largest group)
  int kmax = 0;                          // longest K (padded) of its problems
  std::vector<int32_t> grp;              // problems [grp[g], grp[g+1])
  std::vector<int32_t> grp_blk;          // memory-plan block of each group (-1: any)
  std::vector<int64_t> tile_seg, row_seg, col_seg;
  int64_t buf_bytes = 0;                 // largest group
  double tflops = 0, fl64 = 0;           // issued tensor FLOPs, FP64 FLOPs of the same work
  Prob *d_probs = nullptr;
  int2 *d_rowinfo = nullptr;
  int4 *d_colinfo = nullptr, *d_tiles = nullptr;
  int64_t *d_rowprob = nullptr, *d_colprob = nullptr;
  rixtc::Src *d_rowsrc = nullptr, *d_colsrc = nullptr;
  int32_t *d_xmap = nullptr;
  int *d_eA = nullptr, *d_eB = nullptr;
  // row tiles: per build, the K stages that meet a kept block of their rows (a member
  // of the problem whose blocks with these rows are all screened or absent is skipped)
  int64_t n_rt = 0;
  int2 *d_rt = nullptr;
  int2 *d_rtq = nullptr;
  int64_t *d_rtkw = nullptr;
  unsigned long long *d_kmask = nullptr;
  uint8_t *d_rtlive = nullptr;
};

namespace {

// The output tiles of one problem, in the order the persistent CTAs take them:
// the panels of the larger operand outer, so that each of its row (or column)
// panels is read from memory once while the ~150 tiles in flight share it through
// L2, and the smaller operand's panels are the ones re-read.  w(mt, nt) fills the
// tile's fourth field.
template <class W>
void push_tiles(std::vector<int4> &tiles, int pidx, int mtn, int ntn, W w) {
  if (mtn >= ntn) {
    for (int mt = 0; mt < mtn; mt++)
      for (int nt = 0; nt < ntn; nt++) tiles.push_back(make_int4(pidx, mt, nt, w(mt, nt)));
  } else {
    for (int nt = 0; nt < ntn; nt++)
      for (int mt = 0; mt < mtn; mt++) tiles.push_back(make_int4(pidx, mt, nt, w(mt, nt)));
  }
}
// the same, keeping only the tiles for which live(mt, nt) holds
template <class W, class L>
void push_tiles_if(std::vector<int4> &tiles, int pidx, int mtn, int ntn, W w, L live) {
  if (mtn >= ntn) {
    for (int mt = 0; mt < mtn; mt++)
      for (int nt = 0; nt < ntn; nt++)
        if (live(mt, nt)) tiles.push_back(make_int4(pidx, mt, nt, w(mt, nt)));
  } else {
    for (int nt = 0; nt < ntn; nt++)
      for (int mt = 0; mt < mtn; mt++)
        if (live(mt, nt)) tiles.push_back(make_int4(pidx, mt, nt, w(mt, nt)));
  }
}


using rix::key_a;
using rix::key_b;
using rix::key_n;
using rix::pair_key;

struct PlanHost {
  std::vector<Prob> probs;
  std::vector<int32_t> pblk;
  std::vector<int2> rowinfo;
  std::vector<int4> colinfo, tiles;
  std::vector<int64_t> rowprob, colprob, pbytes;
  std::vector<rixtc::Src> rowsrc, colsrc;
  std::vector<int32_t> xmap;
  std::vector<uint8_t> use;                // kind 2: middle atoms that run here
  std::vector<int2> rt;                    // per row tile, (first, count) of its entries in rtq
  std::vector<int2> rtq;                   // (pair, first | last K stage << 16) of each row block and member
  std::vector<int64_t> rtkw;               // per row tile (and one past the last): first word of its mask
  int G = 1;                               // Src records per packed row / column
  int64_t eaoff = 0, eboff = 0;
  double tflops = 0, fl64 = 0;
};

}  // namespace

// Slices per plan: the regrouped forms (term 1 as T x C, Z with Kronecker rows)
// sum many more products of widely ranging size per output than the FP64
// grouping, and T feeds every term, so these take one slice more than the
// GEMMs of terms 2-4 (capped at 8).
int rix_plan_slices(const rix_ctx *ctx, int kind) {
  if (kind < 2) return ctx->mx_S;
  const int r = ctx->opt.n_slices_regrouped;
  return r > 0 ? std::min(r, (int)rixtc::MAXS) : std::min(ctx->mx_S + 1, (int)rixtc::MAXS);
}

namespace {

int plan_slices(const rix_ctx *ctx, int kind) { return rix_plan_slices(ctx, kind); }

// Rates measured on GB300 (the (H2O)64 and 768-atom ice builds) for the
// choice between an FP64 kernel and a tensor-core regrouping: the FP64 kernels
// of term 1 (k_X12, ~0.7 TFLOP/s), of Z (k_Z, ~1.2) and of T (k_T, ~1.0), and
// the sliced GEMM with its slicing kernels (~0.75 PFLOP/s issued).
constexpr double FP64_RATE_T1 = 0.7e12, FP64_RATE_Z = 1.2e12, FP64_RATE_T = 1.0e12, TC_RATE = 7.5e14;

// Middle atoms within this distance of a group's first atom join its problem (2.5 A).
constexpr double GROUP_R = 2.5 / 0.529177210903;

// Build the problems of one plan (see the section comment for the three kinds).
// count_only: no host arrays, just the map bytes, the largest problem's slices
// and the total slice bytes (the memory plan is not known yet: one block).
rix_status plan_host(rix_ctx *ctx, int kind, const std::vector<int64_t> &ptrZ, PlanHost &h, bool count_only,
                     int64_t *maps_out, int64_t *maxp_out, int64_t *total_out) {
  using namespace rixtc;
  const int nat = ctx->nat, S = plan_slices(ctx, kind);
  auto &row1 = ctx->row1, &row2 = ctx->row2, &row3 = ctx->row3;
  auto find_sorted = [&](const std::vector<int64_t> &keys, int64_t lo, int64_t hi, int64_t key) {
    auto it = std::lower_bound(keys.begin() + lo, keys.begin() + hi, key);
    return (it == keys.begin() + hi || *it != key) ? (int64_t)-1 : (int64_t)(it - keys.begin());
  };
  const int npairs = S * (S + 1) / 2;
  int64_t total = 0, maxp = 0, maps = 0;
  // kind 2: which middle atoms G' run on the tensor cores (estimated times)
  h.use.assign(nat, kind == 2 ? 0 : 1);
  if (kind == 2) {
    for (int g = 0; g < nat; g++) {
      double sB1 = 0, sB2 = 0, sE = 0, M = 0;
      for (int64_t q = row1[g]; q < row1[g + 1]; q++) {
        const int b = ctx->pB[q];
        sB1 += ctx->na_at[b];
        sB2 += (double)ctx->na_at[b] * ctx->nb_at[b];
        if (!ctx->onsite[q]) sE += ctx->nb_at[b];
      }
      M = sB2;
      const double naG = ctx->na_at[g], nbG = ctx->nb_at[g];
      const double f64 = 2.0 * sB1 * naG * nbG * sE + 2.0 * sB2 * nbG * sE;
      const double Mp = std::ceil(M / TM) * TM, Np = std::ceil(sE / TN) * TN,
                   Kp = std::ceil(naG * nbG / KC) * KC;
      const double tc = 2.0 * Mp * Np * Kp * npairs;
      // (a deterministic build keeps Z on the output-stationary FP64 kernel: Z adds the
      // contributions of many middle atoms, which the tensor-core plan does with atomics)
      if (sE > 0 && tc / TC_RATE < f64 / FP64_RATE_Z && !ctx->opt.deterministic) {
        h.use[g] = 1;
        h.fl64 += f64;
      }
    }
  }
  // the row blocks of the memory plan (one block while it is not known yet)
  const bool have_blocks = (int)ctx->blk_atom.size() == ctx->nblk + 1;
  const int nblk = (kind == 2 && have_blocks) ? ctx->nblk : 1;
  std::vector<int32_t> mblk(nat, 0);
  if (have_blocks)
    for (int b = 0; b < ctx->nblk; b++)
      for (int a = ctx->blk_atom[b]; a < ctx->blk_atom[b + 1]; a++) mblk[a] = b;
  // Problems: groups of middle atoms that share most of their neighbours (atoms
  // consecutive in index order within GROUP_R of the first, in one memory-plan
  // block: the atoms of a molecule).  A group's contraction ranges are
  // concatenated on the K axis, its rows and columns are the union of its
  // members', so the output of the group is added once instead of once per atom.
  // Member k sits at image o_k from the first (its shortest pair); row (A', M)
  // means A' at image M from the first member, i.e. at M - o_k from member k,
  // and the output block of (row (A', M), column (E', N)) is (A', E', N - M).
  struct Member {
    int b;
    int o[3];
  };
  std::vector<std::vector<Member>> groups;
  for (int b = 0; b < nat;) {
    if (!h.use[b]) {
      b++;
      continue;
    }
    std::vector<Member> gm(1, Member{b, {0, 0, 0}});
    int c = b + 1;
    for (; c < nat && (int)gm.size() < GMAX && h.use[c] && mblk[c] == mblk[b]; c++) {
      double best = GROUP_R;
      int64_t qb = -1;
      for (int64_t q = row1[b]; q < row1[b + 1]; q++) {
        if (ctx->pB[q] != c) continue;
        double d2 = 0.0;
        for (int x = 0; x < 3; x++) {
          double sh = 0.0;
          if (ctx->periodic)
            for (int d = 0; d < 3; d++) sh += (double)ctx->pn[3 * q + d] * ctx->cell[3 * d + x];
          const double r = (ctx->xyz[3 * c + x] + sh) - ctx->xyz[3 * b + x];
          d2 += r * r;
        }
        if (std::sqrt(d2) < best) {
          best = std::sqrt(d2);
          qb = q;
        }
      }
      if (qb < 0) break;
      // the member's image relative to the first atom: a neighbour within GROUP_R, so at
      // most one cell away unless a cell edge is shorter than GROUP_R
      bool near = true;
      for (int x = 0; x < 3; x++) near &= ctx->pn[3 * qb + x] >= -1 && ctx->pn[3 * qb + x] <= 1;
      if (!near) break;
      gm.push_back(Member{c, {ctx->pn[3 * qb], ctx->pn[3 * qb + 1], ctx->pn[3 * qb + 2]}});
    }
    h.G = std::max(h.G, (int)gm.size());
    groups.push_back(std::move(gm));
    b = c;
  }
  const int G = h.G;
  const Src absent{-1, -1, 1, 1, 1, -1};
  // (atom, image) as a sortable key; member images are within one cell, so a pair's image
  // shifted by one stays in the key's 8-bit fields unless the pair list's own images reach
  // their limit, which the check below reports
  bool img_ok = true;
  auto node_key = [&img_ok](int a, const int *m) {
    for (int x = 0; x < 3; x++) img_ok &= m[x] > -128 && m[x] < 128;
    return pair_key(0, a, m[0], m[1], m[2]);
  };
  using Slots = std::array<int64_t, GMAX>;
  for (int blk = 0; blk < nblk; blk++)
    for (const auto &gm : groups) {
      const int ng = (int)gm.size();
      // rows: (A', M) from the members' pairs (b_k, A', m), M = m + o_k (terms 3+4 skip
      // the on-site pair: P on B' != A); the pair of each member, or -1
      std::map<int64_t, Slots> rm, cm;
      auto slot = [](std::map<int64_t, Slots> &m, int64_t key) -> Slots & {
        auto it = m.find(key);
        if (it == m.end()) {
          Slots e;
          e.fill(-1);
          it = m.emplace(key, e).first;
        }
        return it->second;
      };
      for (int k = 0; k < ng; k++) {
        const int b = gm[k].b;
        for (int64_t q = row1[b]; q < row1[b + 1]; q++) {
          if (kind == 0 && ctx->onsite[q]) continue;
          if (kind == 2 && mblk[ctx->pB[q]] != blk && nblk > 1) continue;
          int M[3];
          for (int c = 0; c < 3; c++) M[c] = ctx->pn[3 * q + c] + gm[k].o[c];
          slot(rm, node_key(ctx->pB[q], M))[k] = q;
        }
        // columns: (E', N) from the 2-hop blocks Z(b_k, E', n) with products (terms 3+4),
        // or from the pairs (b_k, E', n) that are not on-site (term 2, Z)
        if (kind == 0) {
          for (int64_t z = row2[b]; z < row2[b + 1]; z++) {
            if (ptrZ[z + 1] <= ptrZ[z]) continue;
            int N[3];
            for (int c = 0; c < 3; c++) N[c] = key_n(ctx->keys2[z], c) + gm[k].o[c];
            slot(cm, node_key(key_b(ctx->keys2[z]), N))[k] = z;
          }
        } else {
          for (int64_t q = row1[b]; q < row1[b + 1]; q++) {
            if (ctx->onsite[q]) continue;
            int N[3];
            for (int c = 0; c < 3; c++) N[c] = ctx->pn[3 * q + c] + gm[k].o[c];
            slot(cm, node_key(ctx->pB[q], N))[k] = q;
          }
        }
      }
      if (!img_ok) {
        ctx->last_error = "mixed plan: an image index outside the pair key's range";
        return RIX_EINVAL;
      }
      if (rm.empty()) continue;
      int M = 0, N = 0, K = 0;
      for (const auto &r : rm) {
        const int a = key_b(r.first);
        M += kind == 2 ? ctx->na_at[a] * ctx->nb_at[a] : ctx->nb_at[a];
      }
      for (const auto &c : cm) N += ctx->nb_at[key_b(c.first)];
      int kb[GMAX + 1] = {0};
      for (int k = 0; k < ng; k++) kb[k + 1] = kb[k] + ctx->na_at[gm[k].b] * ctx->nb_at[gm[k].b];
      K = kb[ng];
      const int Mpad = std::max(TM, (M + TM - 1) / TM * TM);
      const int Npad = std::max(TN, (N + TN - 1) / TN * TN);
      const int Kpad = std::max(KC, (K + KC - 1) / KC * KC);
      const int64_t bytes = (int64_t)S * (Mpad + Npad) * Kpad * 2;
      total += bytes;
      maxp = std::max(maxp, bytes);
      // row tiles (the kept blocks of their rows decide, per build, which K stages run)
      std::vector<int2> rt_here, rtq_here;
      {
        // row tile t covers rows [128 t, 128 t + 128): the (pair, member) of the row blocks there
        std::vector<std::pair<int, const Slots *>> blocks;  // (end row, pairs of the members)
        int acc = 0;
        for (const auto &r : rm) {
          const int a = key_b(r.first);
          acc += kind == 2 ? ctx->na_at[a] * ctx->nb_at[a] : ctx->nb_at[a];
          blocks.push_back(std::make_pair(acc, &r.second));
        }
        size_t i0 = 0;
        for (int t = 0; t < Mpad / TM; t++) {
          const int lo = t * TM, hi = std::min(M, lo + TM);
          while (i0 < blocks.size() && blocks[i0].first <= lo) i0++;
          const int first = (int)rtq_here.size();
          for (size_t i = i0; i < blocks.size() && (i == 0 ? 0 : blocks[i - 1].first) < hi; i++)
            for (int k = 0; k < ng; k++) {
              const int64_t q = (*blocks[i].second)[k];
              if (q < 0 || kb[k + 1] == kb[k]) continue;
              // the block's flag: C(A', b_k) (terms 3+4), V(A', G) (term 2), V and D (B, G') (Z)
              const int stages = (kb[k] / KC) | (((kb[k + 1] - 1) / KC) << 16);
              rtq_here.push_back(make_int2(ctx->partner1[q], stages));
            }
          rt_here.push_back(make_int2(first, (int)rtq_here.size() - first));
        }
      }
      const int nkw = (Kpad / KC + 63) / 64;  // mask words per row tile
      // xmap, rowinfo + rowprob + rowsrc + exponent, colinfo + colprob + colsrc + exponent, tiles
      maps += (int64_t)rt_here.size() * (8 + 8 + 1 + 8 * nkw) + (int64_t)rtq_here.size() * 8 +
              (int64_t)rm.size() * cm.size() * 4 + (int64_t)Mpad * (8 + 8 + 32 * G + 4) +
              (int64_t)Npad * (16 + 8 + 32 * G + 4) + (int64_t)(Mpad / TM) * (Npad / TN) * 16 + (int64_t)sizeof(Prob);
      h.tflops += 2.0 * Mpad * Npad * Kpad * npairs;
      if (count_only) continue;
      const int pidx = (int)h.probs.size();
      Prob pr{};
      pr.M = M; pr.N = N; pr.Mpad = Mpad; pr.Npad = Npad; pr.Kpad = Kpad;
      pr.pad_ = K;  // true K (the slicing zero-fills K..Kpad)
      pr.nz = (int32_t)cm.size();
      pr.drop = fixed_point_drop(Kpad, S);
      pr.ng = ng;
      for (int k = 0; k <= GMAX; k++) pr.kb[k] = kb[std::min(k, ng)];
      pr.eaoff = h.eaoff; pr.eboff = h.eboff;
      pr.rowoff = (int64_t)h.rowinfo.size();
      pr.coloff = (int64_t)h.colinfo.size();
      pr.xoff = (int64_t)h.xmap.size();
      h.eaoff += Mpad;
      h.eboff += Npad;
      int qi = 0;
      for (const auto &r : rm) {
        const int a = key_b(r.first);
        const int nbA = ctx->nb_at[a], naA = ctx->na_at[a];
        const int nrow = kind == 2 ? naA * nbA : nbA;
        for (int y = 0; y < nrow; y++) {
          h.rowinfo.push_back(make_int2(qi, y));
          h.rowprob.push_back(pidx);
          for (int k = 0; k < G; k++) {
            const int64_t q = k < ng ? r.second[k] : -1;
            if (q < 0) {
              h.rowsrc.push_back(absent);
              continue;
            }
            const int64_t pq = ctx->partner1[q];  // pair (A', b_k)
            const int nbB = ctx->nb_at[gm[k].b], naB = ctx->na_at[gm[k].b];
            Src sr;
            if (kind == 2) {  // rows (P, j) of V(B,G')[P][.] x D(B,G')[j][.]
              const int P = y / nbA, j = y - P * nbA;
              sr = Src{ctx->offV[pq] + (int64_t)P * naB, ctx->offD[pq] + (int64_t)j * nbB, 1, 0, nbB, (int32_t)pq};
            } else if (kind == 0) {  // C(A,B)[naA + P][i][j]
              sr = Src{ctx->offC[pq] + ((int64_t)naA * nbA + y) * nbB, -1, nbA * nbB, 1, nbB, (int32_t)pq};
            } else {  // U2(A,G)[Q][i][k]
              sr = Src{ctx->offU_h[pq] + (int64_t)y * nbB, -1, nbA * nbB, 1, nbB, (int32_t)pq};
            }
            h.rowsrc.push_back(sr);
          }
        }
        qi++;
      }
      for (int r = M; r < Mpad; r++) {
        h.rowinfo.push_back(make_int2(-1, 0));
        h.rowprob.push_back(pidx);
        for (int k = 0; k < G; k++) h.rowsrc.push_back(absent);
      }
      int zi = 0;
      for (const auto &c : cm) {
        const int e = key_b(c.first);
        const int nbE = ctx->nb_at[e];
        for (int l = 0; l < nbE; l++) {
          h.colinfo.push_back(make_int4(zi, l, nbE, 0));
          h.colprob.push_back(pidx);
          for (int k = 0; k < G; k++) {
            const int64_t z = k < ng ? c.second[k] : -1;
            if (z < 0) {
              h.colsrc.push_back(absent);
              continue;
            }
            const int nbB = ctx->nb_at[gm[k].b];
            if (kind == 0)  // Z(B,E')[P][j][l]
              h.colsrc.push_back(Src{ctx->off2[z] + l, -1, nbB * nbE, nbE, nbB, -1});
            else  // C(G,E')[Q][k][l], Q on G
              h.colsrc.push_back(Src{ctx->offC[z] + l, -1, nbB * nbE, nbE, nbB, (int32_t)z});
          }
        }
        zi++;
      }
      for (int c = N; c < Npad; c++) {
        h.colinfo.push_back(make_int4(-1, 0, 0, 0));
        h.colprob.push_back(pidx);
        for (int k = 0; k < G; k++) h.colsrc.push_back(absent);
      }
      // output block of (row block, column block): a K block, or for kind 2 a Z block of
      // the 2-hop list; -1 where no member meets both (the product is zero there)
      for (const auto &r : rm) {
        const int a = key_b(r.first);
        for (const auto &c : cm) {
          bool meet = false;
          for (int k = 0; k < ng; k++) meet |= r.second[k] >= 0 && c.second[k] >= 0;
          if (!meet) {
            h.xmap.push_back(-1);
            continue;
          }
          const int e = key_b(c.first);
          int nz3[3];
          for (int x = 0; x < 3; x++) nz3[x] = key_n(c.first, x) - key_n(r.first, x);
          const int64_t key = pair_key(a, e, nz3[0], nz3[1], nz3[2]);
          const int64_t x = kind == 2 ? find_sorted(ctx->keys2, row2[a], row2[a + 1], key)
                                      : find_sorted(ctx->keys3, row3[a], row3[a + 1], key);
          if (x < 0 || x >= XHALF) {
            ctx->last_error = "mixed plan: output block outside its list";
            return RIX_EINVAL;
          }
          if (kind == 0)  // term 4 in one orientation of each K block
            h.xmap.push_back(ctx->rep3[x] == 0 ? -1 : ctx->rep3[x] == 2 ? (int32_t)x | XHALF : (int32_t)x);
          else
            h.xmap.push_back((int32_t)x);
        }
      }
      const int rt0 = (int)h.rt.size();
      if (h.rtkw.empty()) h.rtkw.push_back(0);
      for (const int2 &t : rt_here) {
        h.rt.push_back(make_int2((int)h.rtq.size() + t.x, t.y));
        h.rtkw.push_back(h.rtkw.back() + nkw);
      }
      h.rtq.insert(h.rtq.end(), rtq_here.begin(), rtq_here.end());
      {
        // terms 3+4: only the tiles with an output block (one orientation of each K block)
        std::vector<int> rs(1, 0), cs(1, 0);
        for (const auto &r : rm) rs.push_back(rs.back() + ctx->nb_at[key_b(r.first)]);
        for (const auto &c : cm) cs.push_back(cs.back() + ctx->nb_at[key_b(c.first)]);
        const int nq = (int)rm.size(), nzb = (int)cm.size();
        auto live = [&](int mt, int nt) {
          if (kind != 0) return true;
          const int rlo = mt * TM, rhi = std::min(M, rlo + TM), clo = nt * TN, chi = std::min(N, clo + TN);
          if (rlo >= rhi || clo >= chi) return false;
          const int q0 = (int)(std::upper_bound(rs.begin(), rs.end(), rlo) - rs.begin()) - 1;
          const int z0 = (int)(std::upper_bound(cs.begin(), cs.end(), clo) - cs.begin()) - 1;
          for (int q = q0; q < nq && rs[q] < rhi; q++)
            for (int z = z0; z < nzb && cs[z] < chi; z++)
              if (h.xmap[pr.xoff + (int64_t)q * nzb + z] >= 0) return true;
          return false;
        };
        push_tiles_if(h.tiles, pidx, Mpad / TM, Npad / TN, [&](int mt, int) { return rt0 + mt; }, live);
      }
      h.probs.push_back(pr);
      h.pbytes.push_back(bytes);
      // Z of terms 3+4 is resident per block of its middle atoms; kind 2 rows per block
      h.pblk.push_back(kind == 0 ? mblk[gm[0].b] : (kind == 2 ? blk : -1));
    }
  if (maps_out) *maps_out = maps;
  if (maxp_out) *maxp_out = maxp;
  if (total_out) *total_out = total;
  return RIX_OK;
}

// The reusable slice buffer of a plan: the largest problem, or up to 8 GB of them.
int64_t group_budget(int64_t maxp, int64_t total) {
  return total ? std::max(maxp, std::min(total, (int64_t)8 << 30)) : 0;
}

}  // namespace

// Slices per operand when rix_options.n_slices is 0: with balanced digits five
// slices (six for the regrouped plans) keep the mixed build within 1e-8 in K and
// 1e-6 Ha in E_x on the water, ice and perovskite workloads measured (largest
// difference 1.1e-7 Ha, the 1,536-atom perovskite).
constexpr int DEFAULT_SLICES = 5;

// Device bytes the mixed-precision plans will need (their maps plus one slice buffer).
int64_t rix_mixed_bytes(rix_ctx *ctx, const std::vector<int64_t> &ptrZ) {
  ctx->mx_S = ctx->opt.n_slices > 0 ? ctx->opt.n_slices : DEFAULT_SLICES;
  int64_t maps = 0, buf = 0;
  {
    int64_t t1 = 0, tt = 0;
    rix_t1_plan_build(ctx, true, &t1);  // maps plus its slice buffer
    rix_tt_plan_build(ctx, true, &tt);
    maps += t1 + tt;
  }
  for (int kind = 0; kind < 3; kind++) {
    PlanHost h;
    int64_t m = 0, maxp = 0, total = 0;
    plan_host(ctx, kind, ptrZ, h, true, &m, &maxp, &total);
    maps += m + (kind == 2 ? ctx->nat : 0);
    buf = std::max(buf, group_budget(maxp, total));
  }
  // the count is exact for the maps and an upper bound for the slice buffer
  return maps + buf + 4 * (int64_t)ctx->nat + ((int64_t)64 << 10);
}

rix_status rix_mixed_plan(rix_ctx *ctx, const std::vector<int64_t> &ptrZ) {
  using namespace rixtc;
  ctx->mx_S = ctx->opt.n_slices > 0 ? ctx->opt.n_slices : DEFAULT_SLICES;
  if (ctx->mx_S > MAXS) {
    ctx->last_error = "n_slices above 8";
    return RIX_EINVAL;
  }
  int64_t buf = 0;
  double tflops = 0;
  for (int kind = 0; kind < 3; kind++) {
    PlanHost h;
    int64_t maps = 0, maxp = 0, total = 0;
    rix_status s = plan_host(ctx, kind, ptrZ, h, false, &maps, &maxp, &total);
    if (s != RIX_OK) return s;
    rix_mx_plan *pl = new rix_mx_plan;
    pl->kind = kind;
    pl->S = plan_slices(ctx, kind);
    pl->G = h.G;
    (kind == 0 ? ctx->mx34 : kind == 1 ? ctx->mx2 : ctx->mxz) = pl;
    const int64_t budget = group_budget(maxp, total);
    // groups of consecutive problems within the budget and within one memory-plan block
    pl->grp.assign(1, 0);
    int64_t cur = 0, maxgrp = 0;
    const int np = (int)h.probs.size();
    for (int p = 0; p < np; p++) {
      if (p > 0 && (h.pblk[p] != h.pblk[p - 1] || cur + h.pbytes[p] > budget)) {
        pl->grp.push_back(p);
        maxgrp = std::max(maxgrp, cur);
        cur = 0;
      }
      Prob &pr = h.probs[p];
      pr.aoff = cur;
      pr.boff = cur + (int64_t)pl->S * pr.Mpad * pr.Kpad * 2;
      cur += h.pbytes[p];
    }
    maxgrp = std::max(maxgrp, cur);
    pl->grp.push_back(np);
    pl->buf_bytes = np ? maxgrp : 0;
    buf = std::max(buf, pl->buf_bytes);
    const size_t ng = pl->grp.size() - 1;
    pl->grp_blk.assign(ng, -1);
    pl->tile_seg.assign(ng + 1, 0);
    pl->row_seg.assign(ng + 1, 0);
    pl->col_seg.assign(ng + 1, 0);
    {
      size_t ti = 0, ri = 0, ci = 0;
      for (size_t g = 0; g < ng; g++) {
        const int pend = pl->grp[g + 1];
        if (pl->grp[g] < np) pl->grp_blk[g] = h.pblk[pl->grp[g]];
        while (ti < h.tiles.size() && h.tiles[ti].x < pend) ti++;
        while (ri < h.rowprob.size() && h.rowprob[ri] < pend) ri++;
        while (ci < h.colprob.size() && h.colprob[ci] < pend) ci++;
        pl->tile_seg[g + 1] = ti;
        pl->row_seg[g + 1] = ri;
        pl->col_seg[g + 1] = ci;
      }
    }
    pl->tflops = h.tflops;
    pl->fl64 = h.fl64;
    for (const Prob &pr : h.probs) pl->kmax = std::max(pl->kmax, pr.Kpad);
    tflops += h.tflops;
    ctx->stats.tensor_flops_stage[kind == 0 ? 0 : kind == 1 ? 1 : 3] = h.tflops;
    if ((s = rix_upload(ctx, &pl->d_probs, h.probs)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_rowinfo, h.rowinfo)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_colinfo, h.colinfo)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_tiles, h.tiles)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_rowprob, h.rowprob)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_colprob, h.colprob)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_rowsrc, h.rowsrc)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_colsrc, h.colsrc)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_xmap, h.xmap)) != RIX_OK) return s;
    if ((s = rix_alloc(ctx, &pl->d_eA, std::max<int64_t>(h.eaoff, 1))) != RIX_OK) return s;
    if ((s = rix_alloc(ctx, &pl->d_eB, std::max<int64_t>(h.eboff, 1))) != RIX_OK) return s;
    if (!h.rt.empty()) {
      pl->n_rt = (int64_t)h.rt.size();
      if ((s = rix_upload(ctx, &pl->d_rt, h.rt)) != RIX_OK) return s;
      if (!h.rtq.empty() && (s = rix_upload(ctx, &pl->d_rtq, h.rtq)) != RIX_OK) return s;
      if ((s = rix_upload(ctx, &pl->d_rtkw, h.rtkw)) != RIX_OK) return s;
      if ((s = rix_alloc(ctx, &pl->d_kmask, std::max<int64_t>(h.rtkw.back(), 1))) != RIX_OK) return s;
      if ((s = rix_alloc(ctx, &pl->d_rtlive, pl->n_rt)) != RIX_OK) return s;
    }
    if (kind == 2) {
      // middle atoms whose term-4 intermediate runs here: k_Z skips them
      std::vector<int32_t> on;
      for (int g = 0; g < ctx->nat; g++)
        if (h.use[g]) on.push_back(g);
      if ((s = rix_alloc(ctx, &ctx->d_ztc, ctx->nat)) != RIX_OK) return s;
      RIX_CUDA_TRY(ctx, cudaMemset(ctx->d_ztc, 0, ctx->nat));
      if (!on.empty()) {
        int32_t *d_on = nullptr;
        if ((s = rix_upload(ctx, &d_on, on)) != RIX_OK) return s;
        k_flag_set<<<(unsigned)((on.size() + 255) / 256), 256>>>((int)on.size(), d_on, ctx->d_ztc);
        RIX_CUDA_TRY(ctx, cudaDeviceSynchronize());
      }
      ctx->n_ztc = (int)on.size();
      ctx->stats.flops_z_tc = h.fl64;
    }
    if (ctx->opt.verbose)
      fprintf(stderr, "rix mixed %s: %zu GEMM tiles in %zu group(s), slice buffer %.3g GB%s\n",
              kind == 0 ? "terms 3+4" : kind == 1 ? "term 2" : "term-4 intermediate", h.tiles.size(), ng,
              maxgrp * 1e-9, kind == 2 ? (", " + std::to_string(ctx->n_ztc) + " middle atoms").c_str() : "");
  }
  rix_status s;
  {
    int64_t t1buf = 0;
    if ((s = rix_t1_plan_build(ctx, false, &t1buf)) != RIX_OK) return s;
    buf = std::max(buf, t1buf);
    tflops += ctx->stats.tensor_flops_stage[2];
    int64_t ttbuf = 0;
    if ((s = rix_tt_plan_build(ctx, false, &ttbuf)) != RIX_OK) return s;
    buf = std::max(buf, ttbuf);
    tflops += ctx->stats.tensor_flops_stage[4];
  }
  if ((s = rix_dev_alloc(ctx, (void **)&ctx->d_mx_buf, std::max<int64_t>(buf, 16))) != RIX_OK) return s;
  ctx->d_mx_err = ctx->d_err;
  if (ctx->opt.deterministic) {
    if ((s = rix_alloc(ctx, &ctx->d_X128, 2 * ctx->offK[ctx->nk])) != RIX_OK) return s;
  }
  if ((s = rix_alloc(ctx, &ctx->d_gemm_chunks, 1)) != RIX_OK) return s;
  RIX_CUDA_TRY(ctx, cudaMemset(ctx->d_gemm_chunks, 0, sizeof(unsigned long long)));
  ctx->mx_buf_bytes = buf;
  ctx->stats.tensor_flops = tflops;
  ctx->have_mx = true;
  return RIX_OK;
}

// Kernel launches of one rix_build_K: flags, per block T, U2 and Z, terms 1+2 and
// terms 3+4 (FP64 per block) or per group four slicing kernels and a GEMM
// (mixed), symmetrise.
int32_t rix_launch_count(const rix_ctx *ctx) {
  int32_t n = 2 + 3 * ctx->nblk;
  if (ctx->have_mx) {
    // per group: exponents and digits of both operands, then the GEMM
    n += 5 * (int32_t)(ctx->mx34->grp.size() - 1) + 5 * (int32_t)(ctx->mx2->grp.size() - 1) +
         5 * (int32_t)(ctx->mxz->grp.size() - 1) + rix_t1_launches(ctx) + rix_tt_launches(ctx);
    if (ctx->n_t1tc < ctx->nat) n += ctx->nblk;  // k_X12 for the other column atoms
    if (ctx->n_ztc == ctx->nat) n -= ctx->nblk;   // no k_Z: the Z buffer is zeroed by a memset
    // row-tile K-stage masks: once per Z block, once per terms-3+4 block, once for term 2
    if (ctx->mxz->n_rt > 0) n += ctx->nblk;
    if (ctx->mx34->n_rt > 0) n += ctx->nblk;
    if (ctx->mx2->n_rt > 0) n++;
  } else {
    n += 2 * ctx->nblk;  // k_X12, k_X34
  }
  return n;
}

void rix_mixed_free(rix_ctx *ctx) {
  rix_t1_plan_free(ctx);
  rix_tt_plan_free(ctx);
  delete ctx->mx34;
  delete ctx->mx2;
  delete ctx->mxz;
  ctx->mx34 = ctx->mx2 = ctx->mxz = nullptr;
}

namespace {

rix_status launch_gemm(rix_ctx *ctx, GemmArgs ga, int64_t ntiles, int S, cudaStream_t st);

struct Operand {
  const double *x;
  int64_t shift;
  const double *x2;
  const uint8_t *keep, *keep2;
};

// Slice the rows and columns of group g of a plan, then run its GEMM tiles; the
// results go to out + offs[xmap] - oshift (scaled by oscale).
rix_status run_group(rix_ctx *ctx, const rix_mx_plan *pl, size_t g, const Operand &ra, const Operand &cb,
                     const int64_t *offs, double *out, int64_t oshift, double oscale, cudaStream_t st) {
  using namespace rixtc;
  const int S = pl->S;
  const int64_t r0 = pl->row_seg[g], r1 = pl->row_seg[g + 1];
  const int64_t c0 = pl->col_seg[g], c1 = pl->col_seg[g + 1];
  const int64_t t0 = pl->tile_seg[g], t1 = pl->tile_seg[g + 1];
  __nv_bfloat16 *buf = (__nv_bfloat16 *)ctx->d_mx_buf;
  if (r1 > r0) {
    const SrcAcc a{pl->d_rowprob, pl->d_probs, pl->d_rowsrc, pl->G, ra.x, ra.shift, ra.x2, ra.keep, ra.keep2, 0};
    if (pl->kind == 2) {  // Kronecker rows: exponents from the factors' maxima
      k_kron_exp<<<(unsigned)((r1 - r0 + 127) / 128), 128, 0, st>>>(r0, r1 - r0, a, pl->d_eA);
      launch_slice_dig(r0, r1 - r0, a, S, buf, pl->d_eA, st);
    } else {
      slice_rows(r0, r1 - r0, a, S, buf, pl->d_eA, pl->kmax, st);
    }
  }
  if (c1 > c0) {
    const SrcAcc b{pl->d_colprob, pl->d_probs, pl->d_colsrc, pl->G, cb.x, cb.shift, cb.x2, cb.keep, cb.keep2, 1};
    slice_rows(c0, c1 - c0, b, S, buf, pl->d_eB, pl->kmax, st);
  }
  if (t1 > t0) {
    GemmArgs ga{buf, buf, pl->d_eA, pl->d_eB, nullptr, 0, 0, 0, 0, 0, 0, S, 1, 0, ctx->d_mx_err,
                pl->d_tiles + t0, pl->d_probs, pl->d_rowinfo, pl->d_colinfo, pl->d_xmap, offs, out};
    ga.mode = 0;
    ga.oscale = oscale;
    ga.xshift = oshift;
    ga.ntiles = (int)(t1 - t0);
    ga.row_live = pl->d_rtlive;  // row tiles and K stages whose blocks are all screened are skipped
    ga.kmask = pl->d_kmask;
    ga.kmask_off = pl->d_rtkw;
    if (out == ctx->d_X && ctx->d_X128) ga.X128 = ctx->d_X128;  // deterministic: X as 128-bit fixed point
    rix_status ls = launch_gemm(ctx, ga, t1 - t0, S, st);
    if (ls != RIX_OK) return ls;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string("mixed GEMM: ") + cudaGetErrorString(e);
    return RIX_ECUDA;
  }
  return RIX_OK;
}

// One batched GEMM launch of the build; with rix_options.profile >= 2 (and the
// stream not capturing) it is bracketed by a pair of events and counts its K
// stages, for the per-kernel roofline (rix_gemm_profile).
rix_status launch_gemm(rix_ctx *ctx, GemmArgs ga, int64_t ntiles, int S, cudaStream_t st) {
  bool prof = ctx->opt.profile >= 2;
  if (prof) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st != nullptr && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      prof = false;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof) {
    for (cudaEvent_t *e : {&e0, &e1}) {
      if (!ctx->gemm_ev_pool.empty()) {
        *e = ctx->gemm_ev_pool.back();
        ctx->gemm_ev_pool.pop_back();
      } else {
        RIX_CUDA_TRY(ctx, cudaEventCreate(e));
      }
    }
    ga.chunks = (unsigned long long *)ctx->d_gemm_chunks;
    RIX_CUDA_TRY(ctx, cudaEventRecord(e0, st));
  }
  k_gemm_sliced<<<persistent_grid(ntiles), NTHR, smem_bytes(S), st>>>(ga);
  if (prof) {
    RIX_CUDA_TRY(ctx, cudaEventRecord(e1, st));
    ctx->gemm_ev.push_back(e0);
    ctx->gemm_ev.push_back(e1);
  }
  return RIX_OK;
}

void gemm_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(rixtc::k_gemm_sliced, cudaFuncAttributeMaxDynamicSharedMemorySize, rixtc::SMEM_LIMIT);
    done = true;
  }
}

}  // namespace

namespace {
// The K-stage masks and liveness of a plan's row tiles for the current flags (product
// screening applies to the Z plan's (V, D) rows).
void rt_masks(rix_ctx *ctx, const rix_mx_plan *pl, const uint8_t *keep, const uint8_t *keep2, bool pscreen,
              cudaStream_t st) {
  if (pl->n_rt <= 0) return;
  rix::PScreen ps = rix_pscreen(ctx);
  if (!pscreen) ps.tau = 0.f;
  rixtc::k_rt_mask<<<(unsigned)((pl->n_rt + 255) / 256), 256, 0, st>>>(
      pl->n_rt, pl->d_rt, pl->d_rtq, pl->d_rtkw, keep, keep2, ctx->d_pB, ctx->d_maxCatom, ps, pl->d_kmask,
      pl->d_rtlive);
}
}  // namespace

// Terms 3+4 for the middle atoms of memory-plan block blk (Z resident, zbase).
rix_status rix_mixed_x34(rix_ctx *ctx, int blk, int64_t zbase, cudaStream_t st) {
  gemm_attr();
  const rix_mx_plan *pl = ctx->mx34;
  const Operand rows{ctx->d_C, 0, nullptr, ctx->d_keepC, nullptr};
  const Operand cols{ctx->d_Z, zbase, nullptr, nullptr, nullptr};
  rt_masks(ctx, pl, ctx->d_keepC, nullptr, false, st);
  for (size_t g = 0; g + 1 < pl->grp.size(); g++) {
    if (pl->grp_blk[g] != blk) continue;
    // weight 2: term 4 in one orientation of each K block (Z carries the grouping's 1/2)
    rix_status s = run_group(ctx, pl, g, rows, cols, ctx->d_offK, ctx->d_X, 0, 2.0, st);
    if (s != RIX_OK) return s;
  }
  return RIX_OK;
}

// Term 2 for every middle atom (U2 complete).
rix_status rix_mixed_t2(rix_ctx *ctx, cudaStream_t st) {
  gemm_attr();
  const rix_mx_plan *pl = ctx->mx2;
  const Operand rows{ctx->d_U, 0, nullptr, ctx->d_keepV, nullptr};
  const Operand cols{ctx->d_C, 0, nullptr, ctx->d_keepC, nullptr};
  rt_masks(ctx, pl, ctx->d_keepV, nullptr, false, st);
  for (size_t g = 0; g + 1 < pl->grp.size(); g++) {
    rix_status s = run_group(ctx, pl, g, rows, cols, ctx->d_offK, ctx->d_X, 0, 1.0, st);
    if (s != RIX_OK) return s;
  }
  return RIX_OK;
}

// Term-4 intermediate for the rows B of memory-plan block blk (after k_Z stored the
// FP64 part of those Z blocks; Z resident at zbase).
rix_status rix_mixed_z(rix_ctx *ctx, int blk, int64_t zbase, const double *D, cudaStream_t st) {
  gemm_attr();
  const rix_mx_plan *pl = ctx->mxz;
  const Operand rows{ctx->d_V, 0, D, ctx->d_keepV, ctx->d_keepD};
  const Operand cols{ctx->d_C, 0, nullptr, ctx->d_keepC, nullptr};
  rt_masks(ctx, pl, ctx->d_keepV, ctx->d_keepD, true, st);
  for (size_t g = 0; g + 1 < pl->grp.size(); g++) {
    if (pl->grp_blk[g] != blk) continue;
    rix_status s = run_group(ctx, pl, g, rows, cols, ctx->d_off2, ctx->d_Z, zbase, 0.5, st);
    if (s != RIX_OK) return s;
  }
  return RIX_OK;
}

// ==========================================================================
// Term 1 on the tensor cores, one problem per column atom E (and memory-plan
// block of row atoms):
//
//   R(A',E')[(P,i)][(l,Q)] = sum_{G' near E'} sum_k T(A',G')[P][i][k] C(G',E')[Q on E'][k][l]
//   X(A',E')[i][l]        += w sum_{P,Q} V(A',E')[P][Q] R[(P,i)][(l,Q)]
//
// with w = 1 for the pairs (A', E') in their representative orientation, w = 1/2
// for the on-site pair and no row for the others (term 1 is symmetric under the
// transposition of its pair, and K = X + X^T restores the other orientation).
// Rows (A', P, i) over those row atoms A' near E', K = (G', k) over E's
// neighbours G', columns (l, Q).  The V contraction (a few FLOPs per R
// element) runs in the GEMM epilogue in FP64.  This costs about nb_E times
// the FLOPs of the FP64 grouping (which applies V per (A', G', E') triple),
// so a column atom runs here only when its tensor time is estimated lower.
// ==========================================================================
namespace rixtc {

// per-problem segment tables of a term-1 problem
struct T1Ext {
  int64_t koff;    // kmap offset (Kpad entries: (g, k, nbG, -), g < 0 past K)
  int64_t segoff;  // segT offset ([nq][ng]: off2 of T(A'_q, G'_g), -1 if absent)
  int64_t goff;    // segC / gpair offset ([ng])
  int32_t nq, ng;
};

// rows: element (q, P, i ; g, k) = T(A'_q, G'_g)[P][i][k]
struct T1RowAcc {
  const int64_t *prob_of;
  const Prob *probs;
  const T1Ext *ext;
  const int2 *rowinfo;
  const QInfo *qinfo;
  const int4 *kmap;
  const int64_t *segT;
  const double *T;
  int64_t tbase;
  static constexpr int is_b = 0;
  struct Row {
    Prob pr;
    int64_t koff;
    const int64_t *seg;
    int r, P, i, nbA;
  };
  __device__ Row row(int64_t w) const {
    Row R;
    const int64_t pi = prob_of[w];
    R.pr = probs[pi];
    const T1Ext ex = ext[pi];
    R.koff = ex.koff;
    R.r = (int)(w - R.pr.rowoff);
    const int2 ri = rowinfo[w];
    R.seg = nullptr;
    R.P = R.i = 0;
    R.nbA = 1;
    if (ri.x >= 0) {
      R.nbA = qinfo[R.pr.xoff + ri.x].nbA;
      R.P = ri.y / R.nbA;
      R.i = ri.y - R.P * R.nbA;
      R.seg = segT + ex.segoff + (int64_t)ri.x * ex.ng;
    }
    return R;
  }
  __device__ double at(const Row &R, int kk) const {
    if (!R.seg) return 0.0;
    const int4 km = kmap[R.koff + kk];
    if (km.x < 0) return 0.0;
    const int64_t so = R.seg[km.x];
    if (so < 0) return 0.0;
    return T[so - tbase + ((int64_t)R.P * R.nbA + R.i) * km.z + km.y];
  }
};

// columns: element (l, Q ; g, k) = C(G'_g, E')[Q on E'][k][l]
struct T1ColAcc {
  const int64_t *prob_of;
  const Prob *probs;
  const T1Ext *ext;
  const int4 *colinfo;
  const int4 *kmap;
  const int64_t *segC;
  const int32_t *gpair;
  const uint8_t *keepC;
  const double *C;
  static constexpr int is_b = 1;
  struct Row {
    Prob pr;
    int64_t koff, goff;
    int4 ci;
    int r;
  };
  __device__ Row row(int64_t w) const {
    Row R;
    const int64_t pi = prob_of[w];
    R.pr = probs[pi];
    const T1Ext ex = ext[pi];
    R.koff = ex.koff;
    R.goff = ex.goff;
    R.ci = colinfo[w];
    R.r = (int)(w - R.pr.coloff);
    return R;
  }
  __device__ double at(const Row &R, int kk) const {
    if (R.ci.x < 0) return 0.0;
    const int4 km = kmap[R.koff + kk];
    if (km.x < 0 || !keepC[gpair[R.goff + km.x]]) return 0.0;
    return C[segC[R.goff + km.x] + ((int64_t)R.ci.y * km.z + km.y) * R.ci.z + R.ci.x];
  }
};

// Row exponents of the T window once per block: rexp[roff2[t] - rbase + r] = the
// largest exponent of row r of the 2-hop block T(A', G') (its nbG values), one
// CTA per block t in [t0, t1).
__global__ void k_rowexp(int64_t t0, const int64_t *off2, const int64_t *roff2, const int32_t *atomA2,
                         const int32_t *atomB2, const int32_t *nb, const int32_t *na, const double *T,
                         int64_t tbase, int64_t rbase, int *rexp) {
  const int64_t t = t0 + blockIdx.x;
  const int a = atomA2[t], nbG = nb[atomB2[t]];
  const int rows = na[a] * nb[a];
  const double *Tb = T + (off2[t] - tbase);
  int *out = rexp + (roff2[t] - rbase);
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    int m = -2000;
    for (int k = 0; k < nbG; k++) m = max(m, exp_of(fabs(Tb[(int64_t)r * nbG + k])));
    out[r] = m;
  }
}

// Exponents of the term-1 packed rows from the row exponents of their T blocks:
// the row (A'_q, P, i) of a problem spans the blocks T(A'_q, G'_g) of its ng
// neighbours G', so its largest exponent is the largest of theirs (the same value
// the element-wise pass finds: padding and absent blocks hold zeros).
__global__ void k_t1_exp(int64_t n0, int64_t n, T1RowAcc acc, const int64_t *segR, const int *rexp,
                         int64_t rbase, int *e) {
  const int64_t w = n0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n0 + n) return;
  const T1RowAcc::Row R = acc.row(w);
  int m = -2000;
  if (R.seg) {
    const int64_t *rs = segR + (R.seg - acc.segT);
    const int ng = acc.ext[acc.prob_of[w]].ng;
    const int r = R.P * R.nbA + R.i;
    for (int g = lane; g < ng; g += 32) {
      const int64_t so = rs[g];
      if (so >= 0) m = max(m, rexp[so - rbase + r]);
    }
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) e[R.pr.eaoff + R.r] = m;
}

}  // namespace rixtc

struct rix_t1_plan {
  int kmax = 0;                           // longest K (padded) of its problems
  std::vector<int32_t> grp_prob;          // groups of problems [grp_prob[g], grp_prob[g+1])
  std::vector<int32_t> grp_blk;           // memory-plan block of each group
  std::vector<int64_t> tile_seg, row_seg, col_seg;
  int64_t buf_bytes = 0;
  double tflops = 0, fl64 = 0;            // issued tensor FLOPs, FP64 FLOPs of the same work
  Prob *d_probs = nullptr;
  rixtc::T1Ext *d_ext = nullptr;
  int2 *d_rowinfo = nullptr;
  int4 *d_colinfo = nullptr, *d_tiles = nullptr, *d_kmap = nullptr;
  int64_t *d_rowprob = nullptr, *d_colprob = nullptr, *d_segT = nullptr, *d_segC = nullptr;
  int64_t *d_segR = nullptr;              // [nq][ng] like d_segT: row offset of T(A'_q, G'_g) in the row exponents
  int64_t *d_roff2 = nullptr;             // per 2-hop block: its first row among all T rows
  std::vector<int64_t> roff2;
  int32_t *d_gpair = nullptr;
  QInfo *d_qinfo = nullptr;
  int *d_eA = nullptr, *d_eB = nullptr;
};

// Term-1 plan: decide per column atom, build problems (E, block) for the tensor ones.
rix_status rix_t1_plan_build(rix_ctx *ctx, bool count_only, int64_t *bytes_out) {
  using namespace rixtc;
  using rix::key_a;
  using rix::key_b;
  using rix::pair_key;
  const int nat = ctx->nat, S = rix_plan_slices(ctx, 3);
  const int npairs = S * (S + 1) / 2;
  auto &row1 = ctx->row1, &row2 = ctx->row2, &row3 = ctx->row3;
  auto find_sorted = [&](const std::vector<int64_t> &keys, int64_t lo, int64_t hi, int64_t key) {
    auto it = std::lower_bound(keys.begin() + lo, keys.begin() + hi, key);
    return (it == keys.begin() + hi || *it != key) ? (int64_t)-1 : (int64_t)(it - keys.begin());
  };
  // per column atom: FP64 FLOPs of its term 1 and tensor FLOPs of the R form
  std::vector<uint8_t> use(nat, 0);
  double fl64_tc = 0;
  for (int e = 0; e < nat; e++) {
    const int nbE = ctx->nb_at[e], naE = ctx->na_at[e];
    int64_t M = 0, K = 0;
    double f64 = 0;
    for (int64_t q = row1[e]; q < row1[e + 1]; q++) {
      if (!ctx->rep1[ctx->partner1[q]]) continue;  // term 1 of (A', E') in one orientation
      const int a = ctx->pB[q];
      M += (int64_t)ctx->na_at[a] * ctx->nb_at[a];
      for (int64_t g = row1[e]; g < row1[e + 1]; g++) {
        const int gg = ctx->pB[g];
        f64 += 2.0 * naE * ctx->na_at[a] * ctx->nb_at[a] * ctx->nb_at[gg] +
               2.0 * naE * ctx->nb_at[a] * ctx->nb_at[gg] * nbE;
      }
    }
    for (int64_t g = row1[e]; g < row1[e + 1]; g++) K += ctx->nb_at[ctx->pB[g]];
    const double Mp = (double)((M + TM - 1) / TM * TM), Np = (double)((naE * nbE + TN - 1) / TN * TN),
                 Kp = (double)((K + KC - 1) / KC * KC);
    const double tc = 2.0 * Mp * Np * Kp * npairs;
    if (tc / TC_RATE < f64 / FP64_RATE_T1) {
      use[e] = 1;
      fl64_tc += f64;
    }
  }
  // the row blocks of the memory plan (one block while it is not known yet)
  const bool have_blocks = (int)ctx->blk_atom.size() == ctx->nblk + 1;
  const int nblk = have_blocks ? ctx->nblk : 1;
  std::vector<int32_t> blk_of(nat, 0);
  if (have_blocks)
    for (int b = 0; b < nblk; b++)
      for (int a = ctx->blk_atom[b]; a < ctx->blk_atom[b + 1]; a++) blk_of[a] = b;
  std::vector<Prob> probs;
  std::vector<T1Ext> ext;
  std::vector<int2> rowinfo;
  std::vector<int4> colinfo, tiles, kmap;
  std::vector<int64_t> rowprob, colprob, segT, segR, segC, pbytes;
  // rows of every 2-hop block T(A', G') (na_A nb_A each) and their prefix offsets
  std::vector<int64_t> roff2(ctx->n2 + 1, 0);
  for (int64_t t = 0; t < ctx->n2; t++) {
    const int a = key_a(ctx->keys2[t]);
    roff2[t + 1] = roff2[t] + (int64_t)ctx->na_at[a] * ctx->nb_at[a];
  }
  std::vector<int32_t> gpair, pblk;
  std::vector<QInfo> qinfo;
  int64_t eaoff = 0, eboff = 0, maps = 0, maxp = 0, total = 0;
  double tflops = 0;
  std::vector<int64_t> qs;
  for (int b = 0; b < nblk; b++)
    for (int e = 0; e < nat; e++) {
      if (!use[e]) continue;
      qs.clear();
      for (int64_t q = row1[e]; q < row1[e + 1]; q++)
        if (blk_of[ctx->pB[q]] == b && ctx->rep1[ctx->partner1[q]]) qs.push_back(q);
      if (qs.empty()) continue;
      const int nbE = ctx->nb_at[e], naE = ctx->na_at[e];
      const int ng = (int)(row1[e + 1] - row1[e]);
      int M = 0, K = 0;
      for (auto q : qs) M += ctx->na_at[ctx->pB[q]] * ctx->nb_at[ctx->pB[q]];
      for (int64_t g = row1[e]; g < row1[e + 1]; g++) K += ctx->nb_at[ctx->pB[g]];
      const int N = naE * nbE;
      const int Mpad = std::max(TM, (M + TM - 1) / TM * TM), Npad = std::max(TN, (N + TN - 1) / TN * TN);
      const int Kpad = std::max(KC, (K + KC - 1) / KC * KC);
      const int64_t bytes = (int64_t)S * (Mpad + Npad) * Kpad * 2;
      total += bytes;
      maxp = std::max(maxp, bytes);
      maps += (int64_t)Mpad * (8 + 8 + 4) + (int64_t)Npad * (16 + 8 + 4) + (int64_t)Kpad * 16 +
              (int64_t)qs.size() * ng * 16 + (int64_t)ng * 12 + (int64_t)qs.size() * 24 +
              (int64_t)(Mpad / TM) * (Npad / TN) * 16 + (int64_t)(sizeof(Prob) + sizeof(T1Ext));
      tflops += 2.0 * Mpad * Npad * Kpad * npairs;
      if (count_only) continue;
      const int pidx = (int)probs.size();
      Prob pr{};
      pr.M = M; pr.N = N; pr.Mpad = Mpad; pr.Npad = Npad; pr.Kpad = Kpad; pr.pad_ = K;
      pr.nz = ng;
      pr.drop = fixed_point_drop(Kpad, S);
      pr.eaoff = eaoff; pr.eboff = eboff;
      pr.rowoff = (int64_t)rowinfo.size();
      pr.coloff = (int64_t)colinfo.size();
      pr.xoff = (int64_t)qinfo.size();
      eaoff += Mpad;
      eboff += Npad;
      T1Ext ex{(int64_t)kmap.size(), (int64_t)segT.size(), (int64_t)segC.size(), (int32_t)qs.size(), ng};
      // K map and the C segments (G' at image n from E'; C(G',E') is the partner of (E',G',n))
      for (int64_t g = row1[e]; g < row1[e + 1]; g++) {
        const int gg = ctx->pB[g];
        const int64_t p3 = ctx->partner1[g];
        const int nbG = ctx->nb_at[gg];
        const int qE0 = ctx->onsite[p3] ? 0 : ctx->na_at[gg];
        for (int k = 0; k < nbG; k++) kmap.push_back(make_int4((int)(g - row1[e]), k, nbG, 0));
        segC.push_back(ctx->offC[p3] + (int64_t)qE0 * nbG * nbE);
        gpair.push_back((int32_t)p3);
      }
      for (int k = K; k < Kpad; k++) kmap.push_back(make_int4(-1, 0, 1, 0));
      for (int qi = 0; qi < (int)qs.size(); qi++) {
        const int64_t q = qs[qi];
        const int a = ctx->pB[q];
        const int nbA = ctx->nb_at[a], naA = ctx->na_at[a];
        const int64_t vp = ctx->partner1[q];  // pair (A', E', -m)
        int nm[3];
        for (int c = 0; c < 3; c++) nm[c] = -(int)ctx->pn[3 * q + c];
        const int64_t x = find_sorted(ctx->keys3, row3[a], row3[a + 1], pair_key(a, e, nm[0], nm[1], nm[2]));
        if (x < 0) {
          ctx->last_error = "term-1 plan: output block outside the K pattern";
          return RIX_EINVAL;
        }
        qinfo.push_back(QInfo{ctx->offV[vp], (int32_t)x, (int32_t)vp, nbA, ctx->rep1[vp] == 2 ? 1 : 0});
        for (int64_t g = row1[e]; g < row1[e + 1]; g++) {
          int d[3];
          for (int c = 0; c < 3; c++) d[c] = (int)ctx->pn[3 * g + c] - (int)ctx->pn[3 * q + c];
          const int64_t t =
              find_sorted(ctx->keys2, row2[a], row2[a + 1], pair_key(a, ctx->pB[g], d[0], d[1], d[2]));
          segT.push_back(t < 0 ? -1 : ctx->off2[t]);
          segR.push_back(t < 0 ? -1 : roff2[t]);
        }
        for (int r = 0; r < naA * nbA; r++) {
          rowinfo.push_back(make_int2(qi, r));
          rowprob.push_back(pidx);
        }
      }
      for (int r = M; r < Mpad; r++) {
        rowinfo.push_back(make_int2(-1, 0));
        rowprob.push_back(pidx);
      }
      for (int l = 0; l < nbE; l++)
        for (int Q = 0; Q < naE; Q++) {
          colinfo.push_back(make_int4(l, Q, nbE, naE));
          colprob.push_back(pidx);
        }
      for (int c = N; c < Npad; c++) {
        colinfo.push_back(make_int4(-1, 0, 1, 1));
        colprob.push_back(pidx);
      }
      push_tiles(tiles, pidx, Mpad / TM, Npad / TN, [](int, int) { return 0; });
      probs.push_back(pr);
      ext.push_back(ex);
      pbytes.push_back(bytes);
      pblk.push_back(b);
    }
  maps += (ctx->n2 + 1) * 8;  // roff2
  if (count_only) {
    if (bytes_out) *bytes_out = maps + (total ? std::max(maxp, std::min(total, (int64_t)8 << 30)) : 0);
    return RIX_OK;
  }
  rix_t1_plan *pl = new rix_t1_plan;
  ctx->mx1 = pl;
  for (const Prob &pr : probs) pl->kmax = std::max(pl->kmax, pr.Kpad);
  pl->fl64 = fl64_tc;
  pl->tflops = tflops;
  const int64_t budget = std::max(maxp, std::min(total, (int64_t)8 << 30));
  pl->grp_prob.assign(1, 0);
  int64_t cur = 0, maxgrp = 0;
  for (int p = 0; p < (int)probs.size(); p++) {
    if (p > 0 && (pblk[p] != pblk[p - 1] || cur + pbytes[p] > budget)) {
      pl->grp_prob.push_back(p);
      maxgrp = std::max(maxgrp, cur);
      cur = 0;
    }
    probs[p].aoff = cur;
    probs[p].boff = cur + (int64_t)S * probs[p].Mpad * probs[p].Kpad * 2;
    cur += pbytes[p];
  }
  maxgrp = std::max(maxgrp, cur);
  pl->grp_prob.push_back((int)probs.size());
  pl->buf_bytes = probs.empty() ? 0 : maxgrp;
  const size_t ng = pl->grp_prob.size() - 1;
  pl->grp_blk.assign(ng, 0);
  pl->tile_seg.assign(ng + 1, 0);
  pl->row_seg.assign(ng + 1, 0);
  pl->col_seg.assign(ng + 1, 0);
  {
    size_t ti = 0, ri = 0, ci = 0;
    for (size_t g = 0; g < ng; g++) {
      const int pend = pl->grp_prob[g + 1];
      if (pl->grp_prob[g] < (int)pblk.size()) pl->grp_blk[g] = pblk[pl->grp_prob[g]];
      while (ti < tiles.size() && tiles[ti].x < pend) ti++;
      while (ri < rowprob.size() && rowprob[ri] < pend) ri++;
      while (ci < colprob.size() && colprob[ci] < pend) ci++;
      pl->tile_seg[g + 1] = ti;
      pl->row_seg[g + 1] = ri;
      pl->col_seg[g + 1] = ci;
    }
  }
  rix_status s;
  if ((s = rix_upload(ctx, &pl->d_probs, probs)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_ext, ext)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_rowinfo, rowinfo)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_colinfo, colinfo)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_tiles, tiles)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_kmap, kmap)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_rowprob, rowprob)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_colprob, colprob)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_segT, segT)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_segR, segR)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_roff2, roff2)) != RIX_OK) return s;
  pl->roff2.swap(roff2);
  if ((s = rix_upload(ctx, &pl->d_segC, segC)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_gpair, gpair)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_qinfo, qinfo)) != RIX_OK) return s;
  if ((s = rix_alloc(ctx, &pl->d_eA, std::max<int64_t>(eaoff, 1))) != RIX_OK) return s;
  if ((s = rix_alloc(ctx, &pl->d_eB, std::max<int64_t>(eboff, 1))) != RIX_OK) return s;
  // column atoms whose term 1 runs here: k_X12 skips them
  std::vector<int32_t> on;
  for (int e = 0; e < nat; e++)
    if (use[e]) on.push_back(e);
  if ((s = rix_alloc(ctx, &ctx->d_t1tc, nat)) != RIX_OK) return s;
  RIX_CUDA_TRY(ctx, cudaMemset(ctx->d_t1tc, 0, nat));
  if (!on.empty()) {
    int32_t *d_on = nullptr;
    if ((s = rix_upload(ctx, &d_on, on)) != RIX_OK) return s;
    rixtc::k_flag_set<<<(unsigned)((on.size() + 255) / 256), 256>>>((int)on.size(), d_on, ctx->d_t1tc);
    RIX_CUDA_TRY(ctx, cudaDeviceSynchronize());
  }
  ctx->n_t1tc = (int)on.size();
  ctx->stats.tensor_flops_stage[2] = tflops;
  ctx->stats.flops_term1_tc = fl64_tc;
  if (ctx->opt.verbose)
    fprintf(stderr, "rix mixed term 1: %zu of %d column atoms on the tensor cores, %zu GEMM tiles, %zu group(s), "
                    "slice buffer %.3g GB\n", on.size(), nat, tiles.size(), ng, maxgrp * 1e-9);
  if (bytes_out) *bytes_out = maxgrp;
  return RIX_OK;
}

void rix_t1_plan_free(rix_ctx *ctx) {
  delete ctx->mx1;
  ctx->mx1 = nullptr;
}

// Term 1 for the problems of memory-plan block b (T of block b resident at tbase).
rix_status rix_mixed_t1(rix_ctx *ctx, int b, int64_t tbase, cudaStream_t st) {
  using namespace rixtc;
  const rix_t1_plan *pl = ctx->mx1;
  if (!pl) return RIX_OK;
  gemm_attr();
  const int S = rix_plan_slices(ctx, 3);
  __nv_bfloat16 *buf = (__nv_bfloat16 *)ctx->d_mx_buf;
  // row exponents of the block's T window, kept in the Z buffer (Z of this block is
  // built after term 1; the T window has at most as many rows as elements)
  const int64_t w0 = ctx->row2[ctx->blk_atom[b]], w1 = ctx->row2[ctx->blk_atom[b + 1]];
  const int64_t rbase = pl->roff2[w0];
  int *rexp = (int *)ctx->d_Z;
  bool have_rexp = false;
  for (size_t g = 0; g + 1 < pl->grp_prob.size(); g++) {
    if (pl->grp_blk[g] != b || pl->grp_prob[g + 1] == pl->grp_prob[g]) continue;
    const int64_t r0 = pl->row_seg[g], r1 = pl->row_seg[g + 1];
    const int64_t c0 = pl->col_seg[g], c1 = pl->col_seg[g + 1];
    const int64_t t0 = pl->tile_seg[g], t1 = pl->tile_seg[g + 1];
    if (r1 > r0) {
      if (!have_rexp && w1 > w0) {
        k_rowexp<<<(unsigned)(w1 - w0), 128, 0, st>>>(w0, ctx->d_off2, pl->d_roff2, ctx->d_atomA2, ctx->d_atomB2,
                                                      ctx->d_nb, ctx->d_na, ctx->d_T, tbase, rbase, rexp);
        have_rexp = true;
      }
      const T1RowAcc a{pl->d_rowprob, pl->d_probs, pl->d_ext, pl->d_rowinfo, pl->d_qinfo, pl->d_kmap, pl->d_segT,
                       ctx->d_T, tbase};
      k_t1_exp<<<(unsigned)(((r1 - r0) * 32 + 255) / 256), 256, 0, st>>>(r0, r1 - r0, a, pl->d_segR, rexp, rbase,
                                                                          pl->d_eA);
      launch_slice_dig(r0, r1 - r0, a, S, buf, pl->d_eA, st);
    }
    if (c1 > c0) {
      const T1ColAcc b{pl->d_colprob, pl->d_probs, pl->d_ext, pl->d_colinfo, pl->d_kmap, pl->d_segC, pl->d_gpair,
                       ctx->d_keepC, ctx->d_C};
      slice_rows(c0, c1 - c0, b, S, buf, pl->d_eB, pl->kmax, st);
    }
    if (t1 > t0) {
      GemmArgs ga{buf, buf, pl->d_eA, pl->d_eB, nullptr, 0, 0, 0, 0, 0, 0, S, 1, 0, ctx->d_mx_err,
                  pl->d_tiles + t0, pl->d_probs, pl->d_rowinfo, pl->d_colinfo, nullptr, ctx->d_offK, ctx->d_X,
                  1, pl->d_qinfo, ctx->d_V, ctx->d_keepV, 1.0};
      ga.ntiles = (int)(t1 - t0);
      ga.X128 = ctx->d_X128;  // deterministic builds: 128-bit fixed-point additions
      rix_status ls = launch_gemm(ctx, ga, t1 - t0, S, st);
      if (ls != RIX_OK) return ls;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ctx->last_error = std::string("mixed term 1: ") + cudaGetErrorString(e);
      return RIX_ECUDA;
    }
  }
  return RIX_OK;
}

int32_t rix_t1_launches(const rix_ctx *ctx) {
  if (!ctx->mx1) return 0;
  const rix_t1_plan *pl = ctx->mx1;
  int32_t n = 0, last_blk = -1;
  for (size_t g = 0; g + 1 < pl->grp_prob.size(); g++) {
    if (pl->grp_prob[g + 1] == pl->grp_prob[g]) continue;
    n += 5;  // row exponents and digits, column exponents and digits, the GEMM
    if (pl->grp_blk[g] != last_blk) n++;  // k_rowexp, once per block (groups are in block order)
    last_blk = pl->grp_blk[g];
  }
  return n;
}

// ==========================================================================
// T on the tensor cores, one problem per row atom A (for the row atoms where
// it pays): T(A,G')[P][i][k] = sum_{B' near A} C(A,B')[P on A][i][j] D(B',G')[j][k]
// as one GEMM with rows (P, i), K = (B', j) and columns (G', k) over A's 2-hop
// blocks, D(B',G') taken as zero where (B',G') is not a pair.  Results are
// added into the zeroed T buffer of the row block.
// ==========================================================================
namespace rixtc {

struct TTExt {
  int64_t koff;    // kmap offset (Kpad entries: (g, j, nb_B, -), g < 0 past K)
  int64_t p1base;  // first pair (A, .) of the row atom
  int32_t nbA;
  int32_t mbase;   // first K-stage mask word of the problem (column tile nt at mbase + nt * words)
};

// rows: element (P, i ; g, j) = C(A, B'_g)[P][i][j]
struct TTRowAcc {
  const int64_t *prob_of;
  const Prob *probs;
  const TTExt *ext;
  const int2 *rowinfo;
  const int4 *kmap;
  const int64_t *offC;
  const uint8_t *keepC;
  const double *C;
  static constexpr int is_b = 0;
  struct Row {
    Prob pr;
    TTExt ex;
    int r, lrow;
    bool live;
  };
  __device__ Row row(int64_t w) const {
    Row R;
    const int64_t pi = prob_of[w];
    R.pr = probs[pi];
    R.ex = ext[pi];
    R.r = (int)(w - R.pr.rowoff);
    const int2 ri = rowinfo[w];
    R.live = ri.x >= 0;
    R.lrow = ri.y;
    return R;
  }
  __device__ double at(const Row &R, int kk) const {
    if (!R.live) return 0.0;
    const int4 km = kmap[R.ex.koff + kk];
    if (km.x < 0) return 0.0;
    const int64_t p1 = R.ex.p1base + km.x;
    if (!keepC[p1]) return 0.0;
    return C[offC[p1] + (int64_t)R.lrow * km.z + km.y];  // (P nbA + i) nbB + j
  }
};

// columns: element (t, k ; g, j) = D(B'_g, G'_t)[j][k], the pair found among T's products
struct TTColAcc {
  const int64_t *prob_of;
  const Prob *probs;
  const TTExt *ext;
  const int4 *colinfo;  // (z, k, nb_G, t)
  const int4 *kmap;
  const int64_t *ptrT;
  const int2 *LT;       // per T block: (pair (A,B'), pair (B',G')), sorted by the first
  const int64_t *offD;
  const uint8_t *keepD;
  const double *D;
  const unsigned long long *mask;  // K-stage masks of the plan (nullptr: every stage live)
  static constexpr int is_b = 1;
  struct Row {
    Prob pr;
    TTExt ex;
    int4 ci;
    int r;
    int64_t e0, e1;
  };
  // offset of D(B'_g, G') for problem atom pair p1 = (A, B'_g), -1 if that product is absent or screened
  __device__ int64_t dblock(const Row &R, int p1) const {
    int64_t lo = R.e0, hi = R.e1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (LT[mid].x < p1) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= R.e1 || LT[lo].x != p1) return -1;
    const int pD = LT[lo].y;
    return keepD[pD] ? offD[pD] : -1;
  }
  __device__ Row row(int64_t w) const {
    Row R;
    const int64_t pi = prob_of[w];
    R.pr = probs[pi];
    R.ex = ext[pi];
    R.ci = colinfo[w];
    R.r = (int)(w - R.pr.coloff);
    R.e0 = R.ci.x >= 0 ? ptrT[R.ci.w] : 0;
    R.e1 = R.ci.x >= 0 ? ptrT[R.ci.w + 1] : 0;
    return R;
  }
  __device__ double at(const Row &R, int kk) const {
    if (R.ci.x < 0) return 0.0;
    const int4 km = kmap[R.ex.koff + kk];
    if (km.x < 0) return 0.0;
    const int64_t o = dblock(R, (int)(R.ex.p1base + km.x));
    return o < 0 ? 0.0 : D[o + (int64_t)km.y * R.ci.z + R.ci.y];  // j nbG + k
  }
};

// eight consecutive K values of a T column: one search per B' block met (not per value)
__device__ __forceinline__ void load8(const TTColAcc &acc, const TTColAcc::Row &R, int k0, double (&v)[8]) {
  int lastg = -1;
  int64_t o = -1;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    v[j] = 0.0;
    if (R.ci.x < 0) continue;
    const int4 km = acc.kmap[R.ex.koff + k0 + j];
    if (km.x < 0) continue;
    if (km.x != lastg) {
      lastg = km.x;
      o = acc.dblock(R, (int)(R.ex.p1base + km.x));
    }
    if (o >= 0) v[j] = acc.D[o + (int64_t)km.y * R.ci.z + R.ci.y];
  }
}

// the GEMM skips the K stages of a column tile that meet no kept D block
__device__ __forceinline__ bool dig_live(const TTColAcc &acc, const TTColAcc::Row &R, int k0) {
  if (!acc.mask) return true;
  const int c = k0 / KC, words = (R.pr.Kpad / KC + 63) / 64;
  const unsigned long long w = acc.mask[R.ex.mbase + (int64_t)(R.r / TN) * words + (c >> 6)];
  return (w >> (c & 63)) & 1ull;
}

// Column maxima of the D blocks for the T columns' exponents: dcolexp[dcoff[p] + k] =
// the largest exponent of column k of D(pair p) (one warp per pair, lanes over k).
__global__ void k_dcolexp(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *nb, const double *D,
                          const int64_t *offD, const int64_t *dcoff, int *dcolexp) {
  const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= np) return;
  const int nbB = nb[pA[p]], nbG = nb[pB[p]];
  const double *Db = D + offD[p];
  for (int k = lane; k < nbG; k += 32) {
    int m = -2000;
    for (int j = 0; j < nbB; j++) m = max(m, exp_of(fabs(Db[(int64_t)j * nbG + k])));
    dcolexp[dcoff[p] + k] = m;
  }
}

// Exponents of the T plan's columns (G'_t, k): the largest over the kept D blocks
// D(B', G'_t) of the column's T block (its product list) of their column-k maxima,
// which is the largest exponent over the column's K values (the rest are zero).
__global__ void k_tt_colexp(int64_t n0, int64_t n, TTColAcc acc, const int64_t *dcoff, const int *dcolexp,
                            int *e) {
  const int64_t w = n0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n0 + n) return;
  const TTColAcc::Row R = acc.row(w);
  int m = -2000;
  if (R.ci.x >= 0) {
    for (int64_t x = R.e0 + lane; x < R.e1; x += 32) {
      const int pD = acc.LT[x].y;
      if (acc.keepD[pD]) m = max(m, dcolexp[dcoff[pD] + R.ci.y]);
    }
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) e[R.pr.eboff + R.r] = m;
}

// K-stage masks of the T plan: for every product (C(A,B'), D(B',G')) of a T block with kept
// blocks, the stages covering B' in problem A and the column tiles covering G' get their bit.
// One warp per T block.
__global__ void k_tt_mask(int64_t n2, const int64_t *ptrT, const int2 *LT, const int32_t *pB, const int32_t *atomB2,
                          const int32_t *nb, const uint8_t *keepC, const uint8_t *keepD, const int32_t *kpos1,
                          const int2 *tmask, const int32_t *tmw, rix::PScreen ps, unsigned long long *mask) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n2) return;
  const int2 tm = tmask[t];
  if (tm.y < 0) return;
  const int W = tmw[t];
  const int nt0 = tm.x / TN, nt1 = (tm.x + nb[atomB2[t]] - 1) / TN;
  for (int64_t e = ptrT[t] + lane; e < ptrT[t + 1]; e += 32) {
    const int2 en = LT[e];
    if (!keepC[en.x] || !keepD[en.y] || ps.drop2(en.x, en.y)) continue;
    const int k0 = kpos1[en.x];
    const int c0 = k0 / KC, c1 = (k0 + nb[pB[en.x]] - 1) / KC;
    for (int nt = nt0; nt <= nt1; nt++)
      for (int c = c0; c <= c1; c++)
        atomicOr(mask + tm.y + (int64_t)nt * W + (c >> 6), 1ull << (c & 63));
  }
}

__global__ void k_skip_flags(int n, const int32_t *idx, uint8_t *flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) flags[idx[t]] = 1;
}

}  // namespace rixtc

struct rix_tt_plan {
  int kmax = 0;                           // longest K (padded) of its problems
  std::vector<int32_t> grp_prob, grp_blk;
  std::vector<int64_t> tile_seg, row_seg, col_seg;
  int64_t buf_bytes = 0;
  int S = 6;
  Prob *d_probs = nullptr;
  rixtc::TTExt *d_ext = nullptr;
  int2 *d_rowinfo = nullptr;
  int4 *d_colinfo = nullptr, *d_tiles = nullptr, *d_kmap = nullptr;
  int64_t *d_rowprob = nullptr, *d_colprob = nullptr;
  int32_t *d_xmap = nullptr;
  int *d_eA = nullptr, *d_eB = nullptr;
  // K-stage masks: per (problem, column tile) the stages whose D tile is not all zero,
  // set per build from the D screening flags (most (B', G') are not D pairs or are screened)
  int64_t n_mask = 0;
  unsigned long long *d_mask = nullptr;
  int32_t *d_kpos1 = nullptr;   // per pair (A, B'): K offset of B' in problem A (-1: A not here)
  int2 *d_tmask = nullptr;      // per T block (A, G'): (column offset in problem A, mask base), -1 if none
  int32_t *d_tmw = nullptr;     // per T block: mask words per column tile of its problem
  int64_t *d_dcoff = nullptr;   // per pair p: offset of its nb(pB) column exponents
  int *d_dcolexp = nullptr;     // column exponents of the D blocks, per build
};

// T plan: decide per row atom, build one problem per chosen atom (its block is the atom's).
rix_status rix_tt_plan_build(rix_ctx *ctx, bool count_only, int64_t *bytes_out) {
  using namespace rixtc;
  // T feeds every term, so it takes the extra slice as well
  const int nat = ctx->nat, S = rix_plan_slices(ctx, 3);
  const int npairs = S * (S + 1) / 2;
  auto &row1 = ctx->row1, &row2 = ctx->row2;
  std::vector<uint8_t> use(nat, 0);
  double fl64 = 0;
  for (int a = 0; a < nat; a++) {
    const int nbA = ctx->nb_at[a], naA = ctx->na_at[a];
    double f64 = 0;
    int64_t K = 0, N = 0;
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
      const int b = ctx->pB[p1];
      K += ctx->nb_at[b];
      for (int64_t p2 = row1[b]; p2 < row1[b + 1]; p2++)
        f64 += 2.0 * naA * nbA * ctx->nb_at[b] * ctx->nb_at[ctx->pB[p2]];
    }
    for (int64_t t = row2[a]; t < row2[a + 1]; t++) N += ctx->nb_at[rix::key_b(ctx->keys2[t])];
    const double Mp = std::ceil((double)naA * nbA / TM) * TM, Np = std::ceil((double)N / TN) * TN,
                 Kp = std::ceil((double)K / KC) * KC;
    if (2.0 * Mp * Np * Kp * npairs / TC_RATE < f64 / FP64_RATE_T) {
      use[a] = 1;
      fl64 += f64;
    }
  }
  const bool have_blocks = (int)ctx->blk_atom.size() == ctx->nblk + 1;
  std::vector<int32_t> blk_of(nat, 0);
  if (have_blocks)
    for (int b = 0; b < ctx->nblk; b++)
      for (int a = ctx->blk_atom[b]; a < ctx->blk_atom[b + 1]; a++) blk_of[a] = b;
  std::vector<Prob> probs;
  std::vector<TTExt> ext;
  std::vector<int2> rowinfo;
  std::vector<int4> colinfo, tiles, kmap;
  std::vector<int64_t> rowprob, colprob, pbytes;
  std::vector<int32_t> xmap, pblk;
  std::vector<int32_t> kpos1, tmw;
  std::vector<int2> tmask;
  if (!count_only) {
    kpos1.assign(ctx->np, -1);
    tmask.assign(ctx->n2, make_int2(-1, -1));
    tmw.assign(ctx->n2, 0);
  }
  int64_t n_mask = 0;
  int64_t eaoff = 0, eboff = 0, maps = 0, maxp = 0, total = 0;
  double tflops = 0;
  for (int a = 0; a < nat; a++) {
    if (!use[a]) continue;
    const int nbA = ctx->nb_at[a], naA = ctx->na_at[a];
    int K = 0, N = 0;
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) K += ctx->nb_at[ctx->pB[p1]];
    const int nz = (int)(row2[a + 1] - row2[a]);
    for (int64_t t = row2[a]; t < row2[a + 1]; t++) N += ctx->nb_at[rix::key_b(ctx->keys2[t])];
    const int M = naA * nbA;
    const int Mpad = std::max(TM, (M + TM - 1) / TM * TM), Npad = std::max(TN, (N + TN - 1) / TN * TN);
    const int Kpad = std::max(KC, (K + KC - 1) / KC * KC);
    const int64_t bytes = (int64_t)S * (Mpad + Npad) * Kpad * 2;
    total += bytes;
    maxp = std::max(maxp, bytes);
    const int mwords = (Kpad / KC + 63) / 64;
    maps += (int64_t)Mpad * (8 + 8 + 4) + (int64_t)Npad * (16 + 8 + 4) + (int64_t)Kpad * 16 + (int64_t)nz * 4 +
            (int64_t)(Mpad / TM) * (Npad / TN) * 16 + (int64_t)(sizeof(Prob) + sizeof(TTExt)) +
            (int64_t)(Npad / TN) * mwords * 8 + (int64_t)(row1[a + 1] - row1[a]) * 4 + (int64_t)nz * 12;
    tflops += 2.0 * Mpad * Npad * Kpad * npairs;
    if (count_only) continue;
    const int pidx = (int)probs.size();
    Prob pr{};
    pr.M = M; pr.N = N; pr.Mpad = Mpad; pr.Npad = Npad; pr.Kpad = Kpad; pr.pad_ = K;
    pr.nz = nz;
    pr.drop = fixed_point_drop(Kpad, S);
    pr.eaoff = eaoff; pr.eboff = eboff;
    pr.rowoff = (int64_t)rowinfo.size();
    pr.coloff = (int64_t)colinfo.size();
    pr.xoff = (int64_t)xmap.size();
    eaoff += Mpad;
    eboff += Npad;
    const int64_t mbase = n_mask;
    ext.push_back(TTExt{(int64_t)kmap.size(), row1[a], nbA, (int32_t)mbase});
    n_mask += (int64_t)(Npad / TN) * mwords;
    {
      int kp = 0;
      for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
        kpos1[p1] = kp;
        kp += ctx->nb_at[ctx->pB[p1]];
      }
      int np2 = 0;
      for (int64_t t = row2[a]; t < row2[a + 1]; t++) {
        tmask[t] = make_int2(np2, (int)mbase);
        tmw[t] = mwords;
        np2 += ctx->nb_at[rix::key_b(ctx->keys2[t])];
      }
    }
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
      const int nbB = ctx->nb_at[ctx->pB[p1]];
      for (int j = 0; j < nbB; j++) kmap.push_back(make_int4((int)(p1 - row1[a]), j, nbB, 0));
    }
    for (int k = K; k < Kpad; k++) kmap.push_back(make_int4(-1, 0, 1, 0));
    for (int r = 0; r < M; r++) {
      rowinfo.push_back(make_int2(0, r));  // (P nbA + i)
      rowprob.push_back(pidx);
    }
    for (int r = M; r < Mpad; r++) {
      rowinfo.push_back(make_int2(-1, 0));
      rowprob.push_back(pidx);
    }
    for (int64_t t = row2[a]; t < row2[a + 1]; t++) {
      const int nbG = ctx->nb_at[rix::key_b(ctx->keys2[t])];
      for (int k = 0; k < nbG; k++) {
        colinfo.push_back(make_int4((int)(t - row2[a]), k, nbG, (int)t));
        colprob.push_back(pidx);
      }
      xmap.push_back((int32_t)t);
    }
    for (int c = N; c < Npad; c++) {
      colinfo.push_back(make_int4(-1, 0, 1, 0));
      colprob.push_back(pidx);
    }
    push_tiles(tiles, pidx, Mpad / TM, Npad / TN, [&](int, int nt) { return (int)(mbase + nt * mwords); });
    probs.push_back(pr);
    pbytes.push_back(bytes);
    pblk.push_back(blk_of[a]);
  }
  maps += (ctx->np + 1) * 8 + (int64_t)ctx->np * 64 * 4;  // dcoff and (at most) the D column exponents
  if (count_only) {
    if (bytes_out) *bytes_out = maps + (total ? std::max(maxp, std::min(total, (int64_t)8 << 30)) : 0) + nat;
    return RIX_OK;
  }
  rix_tt_plan *pl = new rix_tt_plan;
  ctx->mxt = pl;
  for (const Prob &pr : probs) pl->kmax = std::max(pl->kmax, pr.Kpad);
  pl->S = S;
  const int64_t budget = std::max(maxp, std::min(total, (int64_t)8 << 30));
  pl->grp_prob.assign(1, 0);
  int64_t cur = 0, maxgrp = 0;
  for (int p = 0; p < (int)probs.size(); p++) {
    if (p > 0 && (pblk[p] != pblk[p - 1] || cur + pbytes[p] > budget)) {
      pl->grp_prob.push_back(p);
      maxgrp = std::max(maxgrp, cur);
      cur = 0;
    }
    probs[p].aoff = cur;
    probs[p].boff = cur + (int64_t)S * probs[p].Mpad * probs[p].Kpad * 2;
    cur += pbytes[p];
  }
  maxgrp = std::max(maxgrp, cur);
  pl->grp_prob.push_back((int)probs.size());
  pl->buf_bytes = probs.empty() ? 0 : maxgrp;
  const size_t ng = pl->grp_prob.size() - 1;
  pl->grp_blk.assign(ng, 0);
  pl->tile_seg.assign(ng + 1, 0);
  pl->row_seg.assign(ng + 1, 0);
  pl->col_seg.assign(ng + 1, 0);
  {
    size_t ti = 0, ri = 0, ci = 0;
    for (size_t g = 0; g < ng; g++) {
      const int pend = pl->grp_prob[g + 1];
      if (pl->grp_prob[g] < (int)pblk.size()) pl->grp_blk[g] = pblk[pl->grp_prob[g]];
      while (ti < tiles.size() && tiles[ti].x < pend) ti++;
      while (ri < rowprob.size() && rowprob[ri] < pend) ri++;
      while (ci < colprob.size() && colprob[ci] < pend) ci++;
      pl->tile_seg[g + 1] = ti;
      pl->row_seg[g + 1] = ri;
      pl->col_seg[g + 1] = ci;
    }
  }
  rix_status s;
  if ((s = rix_upload(ctx, &pl->d_probs, probs)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_ext, ext)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_rowinfo, rowinfo)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_colinfo, colinfo)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_tiles, tiles)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_kmap, kmap)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_rowprob, rowprob)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_colprob, colprob)) != RIX_OK) return s;
  if ((s = rix_upload(ctx, &pl->d_xmap, xmap)) != RIX_OK) return s;
  pl->n_mask = n_mask;
  if (n_mask > 0) {
    if ((s = rix_alloc(ctx, &pl->d_mask, n_mask)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_kpos1, kpos1)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_tmask, tmask)) != RIX_OK) return s;
    if ((s = rix_upload(ctx, &pl->d_tmw, tmw)) != RIX_OK) return s;
  }
  if ((s = rix_alloc(ctx, &pl->d_eA, std::max<int64_t>(eaoff, 1))) != RIX_OK) return s;
  if ((s = rix_alloc(ctx, &pl->d_eB, std::max<int64_t>(eboff, 1))) != RIX_OK) return s;
  {
    std::vector<int64_t> dcoff(ctx->np + 1, 0);
    for (int64_t p = 0; p < ctx->np; p++) dcoff[p + 1] = dcoff[p] + ctx->nb_at[ctx->pB[p]];
    if ((s = rix_upload(ctx, &pl->d_dcoff, dcoff)) != RIX_OK) return s;
    if ((s = rix_alloc(ctx, &pl->d_dcolexp, std::max<int64_t>(dcoff[ctx->np], 1))) != RIX_OK) return s;
  }
  std::vector<int32_t> on;
  for (int a = 0; a < nat; a++)
    if (use[a]) on.push_back(a);
  if ((s = rix_alloc(ctx, &ctx->d_ttc, nat)) != RIX_OK) return s;
  RIX_CUDA_TRY(ctx, cudaMemset(ctx->d_ttc, 0, nat));
  if (!on.empty()) {
    int32_t *d_on = nullptr;
    if ((s = rix_upload(ctx, &d_on, on)) != RIX_OK) return s;
    k_skip_flags<<<(unsigned)((on.size() + 255) / 256), 256>>>((int)on.size(), d_on, ctx->d_ttc);
    RIX_CUDA_TRY(ctx, cudaDeviceSynchronize());
  }
  ctx->n_ttc = (int)on.size();
  ctx->stats.tensor_flops_stage[4] = tflops;
  ctx->stats.flops_t_tc = fl64;
  if (ctx->opt.verbose)
    fprintf(stderr, "rix mixed T: %zu of %d row atoms on the tensor cores, %zu GEMM tiles, %zu group(s)\n",
            on.size(), nat, tiles.size(), ng);
  if (bytes_out) *bytes_out = maxgrp;
  return RIX_OK;
}

void rix_tt_plan_free(rix_ctx *ctx) {
  delete ctx->mxt;
  ctx->mxt = nullptr;
}

// T of the tensor-core row atoms of block b (T buffer of the block zeroed, at tbase).
rix_status rix_mixed_T(rix_ctx *ctx, int b, int64_t tbase, const double *D, cudaStream_t st) {
  using namespace rixtc;
  const rix_tt_plan *pl = ctx->mxt;
  if (!pl) return RIX_OK;
  gemm_attr();
  const int S = pl->S;
  __nv_bfloat16 *buf = (__nv_bfloat16 *)ctx->d_mx_buf;
  if (b == 0 && pl->n_mask > 0) {
    // which K stages of every column tile meet a kept D block (D changes every build)
    RIX_CUDA_TRY(ctx, cudaMemsetAsync(pl->d_mask, 0, sizeof(unsigned long long) * pl->n_mask, st));
    k_tt_mask<<<(unsigned)((ctx->n2 * 32 + 255) / 256), 256, 0, st>>>(
        ctx->n2, ctx->d_ptrT, ctx->d_LT, ctx->d_pB, ctx->d_atomB2, ctx->d_nb, ctx->d_keepC, ctx->d_keepD,
        pl->d_kpos1, pl->d_tmask, pl->d_tmw, rix_pscreen(ctx), pl->d_mask);
  }
  if (b == 0 && !pl->grp_blk.empty())
    k_dcolexp<<<(unsigned)((ctx->np * 32 + 255) / 256), 256, 0, st>>>(ctx->np, ctx->d_pA, ctx->d_pB, ctx->d_nb, D,
                                                                      ctx->d_offD, pl->d_dcoff, pl->d_dcolexp);
  for (size_t g = 0; g + 1 < pl->grp_prob.size(); g++) {
    if (pl->grp_blk[g] != b || pl->grp_prob[g + 1] == pl->grp_prob[g]) continue;
    const int64_t r0 = pl->row_seg[g], r1 = pl->row_seg[g + 1];
    const int64_t c0 = pl->col_seg[g], c1 = pl->col_seg[g + 1];
    const int64_t t0 = pl->tile_seg[g], t1 = pl->tile_seg[g + 1];
    if (r1 > r0) {
      const TTRowAcc a{pl->d_rowprob, pl->d_probs, pl->d_ext, pl->d_rowinfo, pl->d_kmap, ctx->d_offC, ctx->d_keepC,
                       ctx->d_C};
      slice_rows(r0, r1 - r0, a, S, buf, pl->d_eA, pl->kmax, st);
    }
    if (c1 > c0) {
      const TTColAcc bb{pl->d_colprob, pl->d_probs, pl->d_ext, pl->d_colinfo, pl->d_kmap, ctx->d_ptrT, ctx->d_LT,
                        ctx->d_offD, ctx->d_keepD, D, pl->n_mask > 0 ? pl->d_mask : nullptr};
      k_tt_colexp<<<(unsigned)(((c1 - c0) * 32 + 255) / 256), 256, 0, st>>>(c0, c1 - c0, bb, pl->d_dcoff,
                                                                             pl->d_dcolexp, pl->d_eB);
      launch_slice_dig(c0, c1 - c0, bb, S, buf, pl->d_eB, st);
    }
    if (t1 > t0) {
      GemmArgs ga{buf, buf, pl->d_eA, pl->d_eB, nullptr, 0, 0, 0, 0, 0, 0, S, 1, 0, ctx->d_mx_err,
                  pl->d_tiles + t0, pl->d_probs, pl->d_rowinfo, pl->d_colinfo, pl->d_xmap, ctx->d_off2, ctx->d_T};
      ga.mode = 0;
      ga.oscale = 1.0;
      ga.xshift = tbase;
      ga.ntiles = (int)(t1 - t0);
      ga.kmask = pl->d_mask;  // skip the K stages whose D tile is all zero
      rix_status ls = launch_gemm(ctx, ga, t1 - t0, S, st);
      if (ls != RIX_OK) return ls;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ctx->last_error = std::string("mixed T: ") + cudaGetErrorString(e);
      return RIX_ECUDA;
    }
  }
  return RIX_OK;
}

int32_t rix_tt_launches(const rix_ctx *ctx) {
  if (!ctx->mxt) return 0;
  const int32_t ng = (int32_t)(ctx->mxt->grp_prob.size() - 1);
  return 5 * ng + (ctx->mxt->n_mask > 0 ? 1 : 0) + (ng > 0 ? 1 : 0);  // + k_tt_mask, k_dcolexp
}

extern "C" rix_status rix_gemm_profile(rix_ctx *ctx, double *ms, int64_t *launches, int64_t *chunks) {
  if (!ctx || !ms || !launches || !chunks) return RIX_EINVAL;
  if (ctx->opt.profile < 2 || !ctx->have_mx) return RIX_EUNSUPPORTED;
  *ms = 0.0;
  *launches = (int64_t)ctx->gemm_ev.size() / 2;
  if (!ctx->gemm_ev.empty()) RIX_CUDA_TRY(ctx, cudaEventSynchronize(ctx->gemm_ev.back()));
  for (size_t i = 0; i + 1 < ctx->gemm_ev.size(); i += 2) {
    float t = 0.f;
    RIX_CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->gemm_ev[i], ctx->gemm_ev[i + 1]));
    *ms += t;
  }
  for (auto e : ctx->gemm_ev) ctx->gemm_ev_pool.push_back(e);
  ctx->gemm_ev.clear();
  unsigned long long c = 0;
  RIX_CUDA_TRY(ctx, cudaMemcpy(&c, ctx->d_gemm_chunks, sizeof c, cudaMemcpyDeviceToHost));
  RIX_CUDA_TRY(ctx, cudaMemset(ctx->d_gemm_chunks, 0, sizeof c));
  *chunks = (int64_t)c;
  return RIX_OK;
}
