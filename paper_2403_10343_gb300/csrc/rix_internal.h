// Internal structures of librix (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/rix.h"

#define RIX_CUDA_TRY(ctx, call)                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(e_);     \
      return RIX_ECUDA;                                                           \
    }                                                                             \
  } while (0)

namespace rix {

// Product screening (rix_options.product_tau): a product of blocks whose max-norms
// multiply to less than tau is skipped.  tau = 0: off.
// 128-bit fixed point in units of 2^-X128_FRAC (deterministic accumulation: integer
// addition does not depend on the order of the additions).  |x| < 2^(127 - X128_FRAC).
constexpr int X128_FRAC = 80;

// x * 2^X128_FRAC as a 128-bit integer (truncated toward minus infinity below the unit)
__device__ __forceinline__ __int128 to_x128(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero and subnormals lie below the unit
  const long long m = (long long)((b & ((1ull << 52) - 1)) | (1ull << 52));
  const int sh = ex - 1075 + X128_FRAC;  // x = m 2^(ex - 1075)
  __int128 v;
  if (sh >= 0) v = sh < 74 ? ((__int128)m << sh) : ((__int128)m << 74);  // beyond the range: saturate
  else v = sh > -64 ? (__int128)(m >> -sh) : 0;
  return (b >> 63) ? -v : v;
}

// the value of a 128-bit fixed-point number (two roundings, the same for the same bits)
__device__ __forceinline__ double from_x128(const unsigned long long *p) {
  const long long hi = (long long)p[1];
  const unsigned long long lo = p[0];
  return (double)hi * 0x1p-16 + (double)lo * 0x1p-80;
}

// *p += v (two 64-bit atomics; the carries out of the low word are counted exactly)
__device__ __forceinline__ void add_x128(unsigned long long *p, __int128 v) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  const unsigned long long old = atomicAdd(p, lo);
  const unsigned long long h = hi + (old + lo < old ? 1ull : 0ull);
  if (h) atomicAdd(p + 1, h);
}

struct PScreen {
  const float *nC, *nV, *nD;
  float tau;
  __device__ __forceinline__ bool drop2(int c, int d) const { return tau > 0.f && nC[c] * nD[d] < tau; }
  __device__ __forceinline__ bool drop3(int v, int d, int c) const {
    return tau > 0.f && nV[v] * nD[d] * nC[c] < tau;
  }
};

// Pair key: A << 44 | B << 24 | (n1+128) << 16 | (n2+128) << 8 | (n3+128).
__host__ __device__ inline int64_t pair_key(int64_t a, int64_t b, int n1, int n2, int n3) {
  return (a << 44) | (b << 24) | ((int64_t)(n1 + 128) << 16) | ((int64_t)(n2 + 128) << 8) |
         (int64_t)(n3 + 128);
}
__host__ __device__ inline int key_a(int64_t k) { return (int)((k >> 44) & 0xFFFFF); }
__host__ __device__ inline int key_b(int64_t k) { return (int)((k >> 24) & 0xFFFFF); }
__host__ __device__ inline int key_n(int64_t k, int c) {
  return (int)((k >> (16 - 8 * c)) & 0xFF) - 128;
}

// One entry of the term-1/2 product list (output = a 2-hop block (A,E)).
struct X12Entry {
  int32_t t;     // T block (A, G') in the 2-hop list
  int32_t p3;    // pair (G', E') carrying C
  int32_t u2;    // pair (A, G') whose U2 block feeds term 2, -1 if no term 2
  int32_t t1;    // 1 if term 1 uses this entry
};

// One entry of the backward term-1/2 list grouped by the C pair (G',E').
struct BX12Entry {
  int32_t t;     // T block (A, G')
  int32_t s;     // output block (A, E') in the 2-hop list (a pair-list block)
  int32_t u2;    // pair (A, G') for term 2, -1 if none
  int32_t t1;    // 1 if term 1
};

// Device allocation tracked for the workspace statistics.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace rix

struct rix_ctx {
  // ------------------------------------------------------------ system
  int32_t nat = 0, nsp = 0;
  bool periodic = false;
  double cell[9] = {0};
  double rc = 0, tau = 0;
  std::vector<double> xyz;
  std::vector<int32_t> sp, nbs, nas;   // species of each atom, per-species sizes
  std::vector<int32_t> nb_at, na_at;   // per atom
  rix_options opt{};
  std::string last_error;
  bool have_cv = false;

  // ------------------------------------------------------------ lists (host)
  int64_t np = 0;                      // 1-hop pairs
  std::vector<int64_t> keys1, offC, offV, offD, row1;
  std::vector<int32_t> pA, pB;
  std::vector<int8_t> pn;              // [np][3]
  std::vector<uint8_t> onsite;
  std::vector<int32_t> partner1;
  int64_t n2 = 0;                      // 2-hop blocks (T and Z)
  std::vector<int64_t> keys2, off2, row2;
  int64_t nk = 0;                      // 3-hop blocks (K and X)
  std::vector<int64_t> keys3, offK, row3;

  // ------------------------------------------------------------ device
  std::vector<rix::DevBuf> bufs;
  size_t dev_bytes = 0;
  // atoms
  int32_t *d_nb = nullptr, *d_na = nullptr;
  // pair list
  int32_t *d_pA = nullptr, *d_pB = nullptr, *d_partner1 = nullptr;
  uint8_t *d_onsite = nullptr;
  // term 1 per pair (A, E', n): 1 = computed (representative orientation), 2 = computed
  // with weight 1/2 (on-site pair), 0 = left to the transpose partner
  std::vector<uint8_t> rep1;
  uint8_t *d_rep1 = nullptr;
  // the same for term 4 per K block (A, E', n) of the 3-hop pattern: 1 = computed with
  // twice the weight of the four-term grouping, 2 = the self block (A, A, 0), weight as
  // in the grouping, 0 = left to the transpose partner
  std::vector<uint8_t> rep3;
  uint8_t *d_rep3 = nullptr;
  int64_t *d_offC = nullptr, *d_offV = nullptr, *d_offD = nullptr, *d_offU = nullptr;
  int32_t *d_map1to2 = nullptr, *d_map1to3 = nullptr;
  // 2-hop and 3-hop lists
  int32_t *d_atomA2 = nullptr, *d_atomB2 = nullptr;   // (A, G) of a 2-hop block
  int64_t *d_off2 = nullptr;
  int32_t *d_map2to1 = nullptr, *d_map2to3 = nullptr;
  int32_t *d_atomA3 = nullptr, *d_atomB3 = nullptr;
  int64_t *d_offK = nullptr;
  int32_t *d_partner3 = nullptr;
  // product lists (CSR over outputs) and launch orders
  int64_t *d_ptrT = nullptr; int2 *d_LT = nullptr;
  int64_t *d_ptrX12 = nullptr; rix::X12Entry *d_LX12 = nullptr;
  int64_t *d_ptrZ = nullptr; int2 *d_LZ = nullptr;
  int64_t *d_ptrX34 = nullptr; int2 *d_LX34 = nullptr;
  // tiled work items: (output, first row) per launch
  int2 *d_itT = nullptr; int64_t n_itT = 0;
  int2 *d_itZ = nullptr; int64_t n_itZ = 0;
  int2 *d_itU = nullptr; int64_t n_itU = 0;
  int32_t *d_ordX12 = nullptr; int64_t n_ordX12 = 0;
  int32_t *d_ordX34 = nullptr; int64_t n_ordX34 = 0;
  // inputs and intermediates
  double *d_C = nullptr, *d_V = nullptr;
  uint8_t *d_keepC = nullptr, *d_keepV = nullptr, *d_keepD = nullptr;
  float *d_normC = nullptr, *d_normV = nullptr, *d_normD = nullptr;  // block max-norms (product screening)
  float *d_maxCatom = nullptr;          // per atom G: the largest norm of its C blocks (G, .)
  double *d_T = nullptr, *d_Z = nullptr, *d_U = nullptr, *d_X = nullptr;
  double *d_epart = nullptr;            // energy partial sums
  unsigned long long *d_X128 = nullptr; // deterministic mixed builds: tensor-core part of X, 128-bit fixed point
  int32_t *d_flag = nullptr;            // device status word
  int64_t n_epart = 0;
  // fold-gamma groups (consecutive K blocks with the same atom pair)
  int64_t n_fold = 0;
  int64_t *d_fold = nullptr;
  int64_t nbasis = 0;
  int64_t *d_bofs = nullptr;            // global basis offset of each atom
  char4 *d_n3 = nullptr;                // image vector (n1, n2, n3) of every K block
  int64_t *d_row1 = nullptr;            // first pair of every atom [nat+1]
  double *d_rvec = nullptr;             // pair vector r_p = x_B + n . cell - x_A of every pair [np][3]
  double *d_gpair = nullptr;            // force chain: dE/dr_p (one Cartesian component) per pair
  double volume = 0.0;                  // cell volume (bohr^3), 0 for a cluster
  // the preceding rix_build_K (rix_options.reuse_forward): its D and K, and whether T, U2 and Z
  // still hold its intermediates (one row block, nothing else has run since)
  const double *fwd_D = nullptr;
  const double *fwd_K = nullptr;
  bool fwd_valid = false;
  // mixed precision: terms 3+4 and term 2 as batched sliced GEMMs on the tensor cores
  bool have_mx = false;
  int32_t mx_S = 5;
  struct rix_mx_plan *mx34 = nullptr, *mx2 = nullptr;
  struct rix_t1_plan *mx1 = nullptr;           // term 1 for the column atoms where it pays
  struct rix_mx_plan *mxz = nullptr;            // term-4 intermediate for the middle atoms where it pays
  struct rix_tt_plan *mxt = nullptr;            // T for the row atoms where it pays
  uint8_t *d_ttc = nullptr;                     // per atom: 1 if its T blocks come from the tensor cores
  int n_ttc = 0;
  uint8_t *d_ztc = nullptr;                     // per atom: 1 if Z's terms through it run on the tensor cores
  int n_ztc = 0;
  uint8_t *d_t1tc = nullptr;                    // per atom: 1 if its term 1 runs on the tensor cores
  int n_t1tc = 0;
  void *d_mx_buf = nullptr;                     // slices of one group of problems
  int64_t mx_buf_bytes = 0;
  int *d_mx_err = nullptr;                      // = d_err (the GEMM kernels' timeout flag)
  // status word of the bounded device waits, in mapped pinned host memory: a kernel
  // that gave up sets it, and the next entry point (or rix_check) reports it
  int *h_err = nullptr, *d_err = nullptr;
  double *noalloc_scratch = nullptr;            // device address of rix_energy_noalloc's fixed array
  std::vector<int64_t> offU_h;                  // U2 offsets per pair (host copy)
  // rix_options.profile >= 2: an event pair around every sliced-GEMM launch, and its K stages
  std::vector<cudaEvent_t> gemm_ev, gemm_ev_pool;
  unsigned long long *d_gemm_chunks = nullptr;

  // memory plan: row blocks of consecutive atoms; item segments per block
  int32_t nblk = 1;
  std::vector<int32_t> blk_atom;                  // [nblk+1]
  std::vector<int64_t> blk_base;                  // off2 of the block's first 2-hop block
  std::vector<int64_t> segT, segU, segX12, segZ;  // [nblk+1] ranges in the item arrays

  // ------------------------------------------------------------ backward plan (opt.backward)
  bool have_bwd = false;
  int64_t *d_ptrBC34 = nullptr; int2 *d_LBC34 = nullptr;   // per pair (A,B'): (pair (A,E'), Z(B,E'))
  int64_t *d_ptrBZ34 = nullptr; int2 *d_LBZ34 = nullptr;   // per Z block: (pair (A,B'), pair (A,E'))
  int64_t *d_ptrBZV = nullptr; int2 *d_LBZV = nullptr;     // per pair (B,G'): (pair (G',E'), Z(B,E'))
  int64_t *d_ptrBZC = nullptr; int2 *d_LBZC = nullptr;     // per pair (G',E'): (pair (B,G'), Z(B,E'))
  int64_t *d_ptrBU2 = nullptr; int2 *d_LBU2 = nullptr;     // per pair (A,G'): (block (A,E'), pair (G',E'))
  int64_t *d_ptrBT1 = nullptr; int2 *d_LBT1 = nullptr;     // per T block: (block (A,E'), pair (G',E'))
  int64_t *d_ptrBC12 = nullptr; rix::BX12Entry *d_LBC12 = nullptr;  // per pair (G',E')
  int64_t *d_ptrBTC = nullptr; int2 *d_LBTC = nullptr;     // per pair (A,B'): (pair (B',G'), T block)
  int4 *d_itB[9] = {nullptr};                              // tiled work items per backward kernel
  int64_t n_itB[9] = {0};
  double *d_U2bar = nullptr, *d_Kbuf = nullptr;   // Tbar and Zbar reuse the T and Z buffers
  double bwd_flops = 0;

  rix_stats_t stats{};

  // shared-memory tile budgets (doubles) of k_X12, k_Z and k_X34; rix_autotune picks them
  int32_t tile_X12 = 12288, tile_Z = 12288, tile_X34 = 12288;

  // stage timing (rix_options.profile): 8 events per build, pooled
  static constexpr int NSTAGE = 8;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<cudaEvent_t> ev_pending;  // NSTAGE + 1 per recorded build
};

// RIX_ETIMEOUT (and the flag cleared) if a bounded device wait of an earlier call gave up
rix_status rix_take_err(rix_ctx *ctx);
// looks up the device address of rix_energy_noalloc's fixed array for this context (rix_noalloc.cu)
rix_status rix_noalloc_attach(rix_ctx *ctx);

// record the stage boundary `i` of the current build (no-op without profiling)
rix_status rix_prof_mark(rix_ctx *ctx, int i, cudaStream_t st);

// helpers shared across translation units
rix_status rix_dev_alloc(rix_ctx *ctx, void **p, size_t bytes);
template <class T>
inline rix_status rix_alloc(rix_ctx *ctx, T **p, size_t n) {
  return rix_dev_alloc(ctx, (void **)p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
}
template <class T>
inline rix_status rix_upload(rix_ctx *ctx, T **p, const std::vector<T> &v) {
  rix_status s = rix_alloc(ctx, p, v.size());
  if (s != RIX_OK) return s;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      ctx->last_error = std::string("upload: ") + cudaGetErrorString(e);
      return RIX_ECUDA;
    }
  }
  return RIX_OK;
}

// mixed precision (rix_tc.cu)
rix_status rix_mixed_plan(rix_ctx *ctx, const std::vector<int64_t> &ptrZ);
int64_t rix_mixed_bytes(rix_ctx *ctx, const std::vector<int64_t> &ptrZ);
rix_status rix_mixed_x34(rix_ctx *ctx, int blk, int64_t zbase, cudaStream_t st);
rix_status rix_mixed_z(rix_ctx *ctx, int blk, int64_t zbase, const double *D, cudaStream_t st);
rix_status rix_mixed_t2(rix_ctx *ctx, cudaStream_t st);
void rix_mixed_free(rix_ctx *ctx);
int32_t rix_launch_count(const rix_ctx *ctx);
rix_status rix_t1_plan_build(rix_ctx *ctx, bool count_only, int64_t *bytes_out);
void rix_t1_plan_free(rix_ctx *ctx);
rix_status rix_mixed_t1(rix_ctx *ctx, int b, int64_t tbase, cudaStream_t st);
int32_t rix_t1_launches(const rix_ctx *ctx);
rix_status rix_tt_plan_build(rix_ctx *ctx, bool count_only, int64_t *bytes_out);
void rix_tt_plan_free(rix_ctx *ctx);
rix_status rix_mixed_T(rix_ctx *ctx, int b, int64_t tbase, const double *D, cudaStream_t st);
int32_t rix_tt_launches(const rix_ctx *ctx);

// FP64 path launches (rix_fp64.cu)
rix_status rix_fp64_build(rix_ctx *ctx, const double *D, double *K, cudaStream_t st, int accumulate = 0);
rix_status rix_launch_T_block(rix_ctx *ctx, const double *D, int b, cudaStream_t st);
rix_status rix_launch_Z_block(rix_ctx *ctx, const double *D, int b, cudaStream_t st);
rix_status rix_launch_flags(rix_ctx *ctx, const double *arr, const int64_t *off, int64_t n,
                            uint8_t *keep, cudaStream_t st, float *norm = nullptr);
rix_status rix_launch_atom_max(rix_ctx *ctx, const float *norm, float *out, cudaStream_t st);
inline rix::PScreen rix_pscreen(const rix_ctx *ctx) {
  return rix::PScreen{ctx->d_normC, ctx->d_normV, ctx->d_normD, (float)ctx->opt.product_tau};
}
rix_status rix_launch_symcheck(rix_ctx *ctx, cudaStream_t st);
rix_status rix_launch_energy(rix_ctx *ctx, const double *D, const double *K, double *Ex,
                             cudaStream_t st);
rix_status rix_launch_fold(rix_ctx *ctx, const double *K, double *Kd, cudaStream_t st);
rix_status rix_launch_pairs(rix_ctx *ctx, const double *d_xyz, const double *d_cell,
                            const int nr[3], int64_t *d_counts, const int64_t *d_rowptr,
                            int64_t *d_keys, cudaStream_t st);
