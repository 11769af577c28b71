// FP64 path of the exchange build and the shared small kernels.
//
// The build runs the paper's grouping of the RI-LVL sum by the atoms that
// carry the two auxiliary functions (Eq. 11, Eqs. 12a-12d).  With i on A, j on B',
// k on G', l on E' it computes
//
//   T(A,G')   = sum_B' C(A,B')^{P on A} D(B',G')                (E = C*D)
//   U2(A,G')  = V(A,G')^T T(A,G')                               (G = E'*V)
//   X(A,E')   = 1/2 sum_G' [V(A,E')^T T(A,G')]^{Q on E'} C(G',E')^{Q on E'}   term 1
//             +     sum_G'!=E' U2(A,G') C(G',E')^{Q on G'}                     term 2
//   Z(B,E')   = 1/2 sum_G'!=E' [V(B,G') C(G',E')^{Q on G'}] applied to D(B,G') (H = F*D)
//   X(A,E')  +=     sum_B'!=A C(A,B')^{P on B'} Z(B,E')                        term 4
//   K(A,E',n) = X(A,E',n) + X(E',A,-n)^T
//
// Term 3 (P on B', Q on E') equals term 2 transposed (the pair symmetry of C,
// V and D stated after Eqs. 12a-12d; the paper's "2G"), and terms 1 and 4 are symmetric by
// themselves, so the last line restores all four terms exactly.
//
// Each kernel is output-stationary: one CTA owns an output block (or a row
// tile of it), walks its product list and keeps the sums in registers, so no
// atomics are needed and every run sums in the same order.
#include <algorithm>
#include <cstdio>
#include <string>

#include "rix_internal.h"

using namespace rix;

namespace {

constexpr int NT = 256;      // threads per CTA
constexpr int MAXE = 32;     // output elements per thread in tiled kernels (NT * MAXE = 8192)
constexpr int XMAXE = 16;    // output elements per thread for K blocks (64 x 64 / 256)
constexpr int SM_MAX = 16384;  // largest shared-memory tile budget in doubles (128 KB)

// ------------------------------------------------------------------ pair list (a1)
__device__ __forceinline__ double d2_raw(const double *xyz, const double *cell, int periodic, int a, int b,
                                         int n1, int n2, int n3) {
  double s[3] = {0.0, 0.0, 0.0};
  if (periodic) {
#pragma unroll
    for (int c = 0; c < 3; c++)
      s[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, cell[c]), __dmul_rn((double)n2, cell[3 + c])),
                       __dmul_rn((double)n3, cell[6 + c]));
  }
  double dx[3];
#pragma unroll
  for (int c = 0; c < 3; c++) dx[c] = __dsub_rn(__dadd_rn(xyz[3 * b + c], s[c]), xyz[3 * a + c]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])), __dmul_rn(dx[2], dx[2]));
}

__device__ __forceinline__ bool is_rep(int a, int b, int n1, int n2, int n3) {
  if (a != b) return a < b;
  if (n1 != 0) return n1 > 0;
  if (n2 != 0) return n2 > 0;
  return n3 >= 0;
}

// One warp per atom A; candidates (B, n1, n2, n3) in lexicographic order, so
// the kept pairs come out sorted.  Pass 1 counts, pass 2 writes the keys.
__global__ void k_pairs(int nat, const double *xyz, const double *cell, int periodic, int nr0, int nr1,
                        int nr2, double rc2, int cut, int64_t *counts, const int64_t *rowptr, int64_t *keys) {
  int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (warp >= nat) return;
  const int a = warp;
  const int N1 = 2 * nr0 + 1, N2 = 2 * nr1 + 1, N3 = 2 * nr2 + 1;
  const int64_t total = (int64_t)nat * N1 * N2 * N3;
  int64_t pos = rowptr ? rowptr[a] : 0;
  int64_t cnt = 0;
  for (int64_t base = 0; base < total; base += 32) {
    int64_t c = base + lane;
    bool keep = false;
    int b = 0, n1 = 0, n2 = 0, n3 = 0;
    if (c < total) {
      int64_t r = c;
      n3 = (int)(r % N3) - nr2; r /= N3;
      n2 = (int)(r % N2) - nr1; r /= N2;
      n1 = (int)(r % N1) - nr0; r /= N1;
      b = (int)r;
      if (!cut) {
        keep = true;
      } else {
        double d2 = is_rep(a, b, n1, n2, n3) ? d2_raw(xyz, cell, periodic, a, b, n1, n2, n3)
                                             : d2_raw(xyz, cell, periodic, b, a, -n1, -n2, -n3);
        keep = d2 < rc2;
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keys && keep) keys[pos + __popc(m & ((1u << lane) - 1u))] = pair_key(a, b, n1, n2, n3);
    pos += __popc(m);
    cnt += __popc(m);
  }
  if (counts && lane == 0) counts[a] = cnt;
}

// ------------------------------------------------------------------ screening flags
// keep[b] = max |block b| >= tau (always 1 when tau <= 0); one warp per block.
// norm (optional): the block's max |x| rounded up to a float (product screening).
__global__ void k_flags(const double *arr, const int64_t *off, int64_t n, double tau, uint8_t *keep, float *norm) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  if (!(tau > 0) && !norm) {
    if (lane == 0) keep[w] = 1;
    return;
  }
  double m = 0;
  for (int64_t i = off[w] + lane; i < off[w + 1]; i += 32) m = fmax(m, fabs(arr[i]));
  for (int s = 16; s; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
  if (lane == 0) {
    keep[w] = !(tau > 0) || m >= tau;
    if (norm) norm[w] = __double2float_ru(m);
  }
}

// ------------------------------------------------------------------ symmetry check of C and V
// C(B,A,-n)[P'][j][i] == C(A,B,n)[P][i][j] with P' the same aux function, and
// V(B,A,-n) == V(A,B,n)^T, bit for bit.  One warp per pair; sets *flag on a mismatch.
__global__ void k_symcheck(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *partner,
                           const uint8_t *onsite, const int32_t *nb, const int32_t *na, const double *C,
                           const int64_t *offC, const double *V, const int64_t *offV, int32_t *flag) {
  int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= np) return;
  int a = pA[p], b = pB[p];
  int64_t q = partner[p];
  int nbA = nb[a], nbB = nb[b], naA = na[a], naB = na[b];
  bool bad = false;
  const double *c = C + offC[p], *cq = C + offC[q];
  int rows = naA + (onsite[p] ? 0 : naB);
  int64_t n = (int64_t)rows * nbA * nbB;
  for (int64_t e = lane; e < n; e += 32) {
    int P = (int)(e / (nbA * nbB));
    int r = (int)(e % (nbA * nbB));
    int i = r / nbB, j = r % nbB;
    int Pq = onsite[p] ? P : (P < naA ? P + naB : P - naA);
    if (c[e] != cq[((int64_t)Pq * nbB + j) * nbA + i]) bad = true;
  }
  const double *v = V + offV[p], *vq = V + offV[q];
  for (int e = lane; e < naA * naB; e += 32) {
    int P = e / naB, Q = e % naB;
    if (v[e] != vq[Q * naA + P]) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1);
}

// ------------------------------------------------------------------ stage T
// T(A,G')[P][i][k] for P in [p0, p0+pt): sum over (C(A,B'), D(B',G')) entries.
__global__ void __launch_bounds__(NT) k_T(const int2 *items, const int64_t *ptrT, const int2 *LT,
                                          const int32_t *atomA2, const int32_t *atomB2, const int64_t *off2,
                                          const int32_t *pB, const int32_t *nb, const int32_t *na,
                                          const double *__restrict__ C, const int64_t *offC,
                                          const double *__restrict__ D, const int64_t *offD,
                                          const uint8_t *keepC, const uint8_t *keepD, double *T,
                                          int64_t tbase, const uint8_t *ttc, PScreen ps) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int2 it = items[blockIdx.x];
  const int t = it.x, p0 = it.y;
  const int a = atomA2[t], g = atomB2[t];
  if (ttc && ttc[a]) return;  // this row atom's T comes from the tensor cores
  const int nbA = nb[a], naA = na[a], nbG = nb[g];
  const int per = nbA * nbG;
  const int pt = max(1, NT * MAXE / per);
  const int pe = min(naA, p0 + pt);
  const int nel = (pe - p0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t e = ptrT[t]; e < ptrT[t + 1]; e++) {
    const int2 en = LT[e];
    if (!keepC[en.x] || !keepD[en.y] || ps.drop2(en.x, en.y)) continue;
    const int nbB = nb[pB[en.x]];
    const double *Dg = D + offD[en.y];
    __syncthreads();
    for (int i = tid; i < nbB * nbG; i += NT) sm[i] = Dg[i];
    __syncthreads();
    const double *Cr = C + offC[en.x] + (int64_t)p0 * nbA * nbB;
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = tid + r * NT;
      if (el < nel) {
        const int row = el / nbG, col = el - row * nbG;
        const double *cr = Cr + (int64_t)row * nbB;
        double s = acc[r];
        for (int j = 0; j < nbB; j++) s = fma(__ldg(cr + j), sm[j * nbG + col], s);
        acc[r] = s;
      }
    }
  }
  double *out = T + (off2[t] - tbase) + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = tid + r * NT;
    if (el < nel) out[el] = acc[r];
  }
}

// ------------------------------------------------------------------ stage U2
// U2(A,G')[Q][i][k] = sum_P V(A,G')[P][Q] T(A,G')[P][i][k] for Q in [q0, q0+qt).
__global__ void __launch_bounds__(NT) k_U2(const int2 *items, const int32_t *pA, const int32_t *pB,
                                           const int32_t *nb, const int32_t *na, const double *__restrict__ V,
                                           const int64_t *offV, const uint8_t *keepV, const int32_t *map1to2,
                                           const double *__restrict__ T, const int64_t *off2,
                                           const int64_t *offU, double *U, int64_t tbase) {
  const int2 it = items[blockIdx.x];
  const int p = it.x, q0 = it.y;
  if (!keepV[p]) return;
  const int a = pA[p], g = pB[p];
  const int nbA = nb[a], naA = na[a], nbG = nb[g], naG = na[g];
  const int per = nbA * nbG;
  const int qt = max(1, NT * MAXE / per);
  const int qe = min(naG, q0 + qt);
  const int nel = (qe - q0) * per;
  const double *Vb = V + offV[p];
  const double *Tt = T + (off2[map1to2[p]] - tbase);
  double *out = U + offU[p] + (int64_t)q0 * per;
  for (int el = threadIdx.x; el < nel; el += NT) {
    const int q = q0 + el / per, c = el % per;
    double s = 0.0;
    for (int P = 0; P < naA; P++) s = fma(__ldg(Vb + P * naG + q), __ldg(Tt + (int64_t)P * per + c), s);
    out[el] = s;
  }
}

// ------------------------------------------------------------------ terms 1 and 2
__global__ void __launch_bounds__(NT) k_X12(const int32_t *ord, const int64_t *ptr, const X12Entry *L,
                                            const int32_t *atomA2, const int32_t *atomB2,
                                            const int32_t *map2to1, const int32_t *map2to3,
                                            const int32_t *pA, const uint8_t *onsite, const int32_t *nb,
                                            const int32_t *na, const double *__restrict__ C,
                                            const int64_t *offC, const double *__restrict__ V,
                                            const int64_t *offV, const uint8_t *keepC, const uint8_t *keepV,
                                            const double *__restrict__ T, const int64_t *off2,
                                            const double *__restrict__ U, const int64_t *offU,
                                            const int64_t *offK, double *X, int64_t tbase, int smb, int t2,
                                            const uint8_t *t1tc, const uint8_t *rep1) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int s = ord[blockIdx.x];
  const int a = atomA2[s], e = atomB2[s];
  const int nbA = nb[a], naA = na[a], nbE = nb[e], naE = na[e];
  const int nel = nbA * nbE;
  const int pae = map2to1[s];
  // term 1 in one orientation of each pair (rep1; else the transpose partner's block
  // carries it), and not for the column atoms whose term 1 runs on the tensor cores
  const bool has1 = pae >= 0 && keepV[pae] && rep1[pae] && !(t1tc && t1tc[e]);
  const double w1 = has1 && rep1[pae] == 2 ? 0.5 : 1.0;
  if (!has1 && !t2) return;
  double acc[XMAXE];
#pragma unroll
  for (int r = 0; r < XMAXE; r++) acc[r] = 0.0;
  for (int64_t it = ptr[s]; it < ptr[s + 1]; it++) {
    const X12Entry en = L[it];
    if (!keepC[en.p3]) continue;
    const int g = pA[en.p3];
    const int nbG = nb[g], naG = na[g];
    const double *Cge = C + offC[en.p3];
    if (en.t1 && has1) {
      // term 1: U1[Q][i][k] = sum_P V(A,E')[P][Q] T(A,G')[P][i][k], Q on E', in tiles of Q
      const int qE0 = onsite[en.p3] ? 0 : naG;
      const double *Tt = T + (off2[en.t] - tbase);
      const double *Vae = V + offV[pae];
      const int per = nbA * nbG;
      const int qt = min(naE, max(1, smb / per));
      for (int q0 = 0; q0 < naE; q0 += qt) {
        const int qn = min(qt, naE - q0);
        __syncthreads();
        for (int el = tid; el < qn * per; el += NT) {
          const int q = el / per, c = el - q * per;
          double u = 0.0;
          for (int P = 0; P < naA; P++) u = fma(__ldg(Vae + P * naE + q0 + q), __ldg(Tt + (int64_t)P * per + c), u);
          sm[el] = u;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < XMAXE; r++) {
          const int el = tid + r * NT;
          if (el < nel) {
            const int i = el / nbE, l = el - i * nbE;
            double v = 0.0;
            for (int q = 0; q < qn; q++) {
              const double *cq = Cge + ((int64_t)(qE0 + q0 + q) * nbG) * nbE + l;
              const double *uq = sm + (q * nbA + i) * nbG;
              for (int k = 0; k < nbG; k++) v = fma(uq[k], __ldg(cq + k * nbE), v);
            }
            acc[r] = fma(w1, v, acc[r]);
          }
        }
      }
    }
    if (t2 && en.u2 >= 0 && keepV[en.u2]) {
      // term 2: X += U2(A,G')[Q][i][k] C(G',E')[Q on G'][k][l] (on the tensor cores in mixed precision)
      const double *U2 = U + offU[en.u2];
#pragma unroll
      for (int r = 0; r < XMAXE; r++) {
        const int el = tid + r * NT;
        if (el < nel) {
          const int i = el / nbE, l = el - i * nbE;
          double v = acc[r];
          for (int q = 0; q < naG; q++) {
            const double *cq = Cge + ((int64_t)q * nbG) * nbE + l;
            const double *uq = U2 + ((int64_t)q * nbA + i) * nbG;
            for (int k = 0; k < nbG; k++) v = fma(__ldg(uq + k), __ldg(cq + k * nbE), v);
          }
          acc[r] = v;
        }
      }
    }
  }
  double *out = X + offK[map2to3[s]];
#pragma unroll
  for (int r = 0; r < XMAXE; r++) {
    const int el = tid + r * NT;
    if (el < nel) out[el] += acc[r];
  }
}

// ------------------------------------------------------------------ term 4 intermediate
// Z(B,E')[P][j][l] = 1/2 sum over (pair (B,G'), pair (G',E') not on-site) of
//   sum_k D(B,G')[j][k] F[P][k][l],  F[P][k][l] = sum_Q V(B,G')[P][Q] C(G',E')[Q on G'][k][l].
__global__ void __launch_bounds__(NT) k_Z(const int2 *items, const int64_t *ptrZ, const int2 *LZ,
                                          const int32_t *atomA2, const int32_t *atomB2, const int64_t *off2,
                                          const int32_t *pB, const int32_t *nb, const int32_t *na,
                                          const double *__restrict__ C, const int64_t *offC,
                                          const double *__restrict__ V, const int64_t *offV,
                                          const double *__restrict__ D, const int64_t *offD,
                                          const uint8_t *keepC, const uint8_t *keepV, const uint8_t *keepD,
                                          double *Z, int64_t zbase, int smb, const uint8_t *ztc, PScreen ps) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int2 it = items[blockIdx.x];
  const int z = it.x, p0 = it.y;
  const int b = atomA2[z], e = atomB2[z];
  const int nbB = nb[b], naB = na[b], nbE = nb[e];
  const int per = nbB * nbE;
  const int pt = max(1, NT * MAXE / per);
  const int pe = min(naB, p0 + pt);
  const int nel = (pe - p0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptrZ[z]; x < ptrZ[z + 1]; x++) {
    const int2 en = LZ[x];
    if (!keepD[en.x] || !keepV[en.x] || !keepC[en.y] || ps.drop3(en.x, en.x, en.y)) continue;
    const int g = pB[en.x];
    if (ztc && ztc[g]) continue;  // this middle atom's part runs on the tensor cores
    const int nbG = nb[g], naG = na[g];
    const double *Dbg = D + offD[en.x];
    const double *Vbg = V + offV[en.x];
    const double *Cge = C + offC[en.y];
    const int fper = nbG * nbE;
    const int ft = max(1, min(pe - p0, smb / fper));
    for (int ps = p0; ps < pe; ps += ft) {
      const int fn = min(ft, pe - ps);
      __syncthreads();
      for (int el = tid; el < fn * fper; el += NT) {
        const int pp = el / fper, c = el - pp * fper;
        const double *vr = Vbg + (int64_t)(ps + pp) * naG;
        double f = 0.0;
        for (int Q = 0; Q < naG; Q++) f = fma(__ldg(vr + Q), __ldg(Cge + (int64_t)Q * fper + c), f);
        sm[el] = f;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = tid + r * NT;
        if (el < nel) {
          const int P = el / per;               // relative to p0
          const int pr = P - (ps - p0);
          if (pr >= 0 && pr < fn) {
            const int rem = el - P * per;
            const int j = rem / nbE, l = rem - j * nbE;
            const double *dj = Dbg + j * nbG;
            const double *fp = sm + pr * fper + l;
            double v = acc[r];
            for (int k = 0; k < nbG; k++) v = fma(__ldg(dj + k), fp[k * nbE], v);
            acc[r] = v;
          }
        }
      }
    }
  }
  double *out = Z + (off2[z] - zbase) + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = tid + r * NT;
    if (el < nel) out[el] = 0.5 * acc[r];
  }
}

// ------------------------------------------------------------------ term 4 (and term 3 via the transpose)
// X(A,E') += sum over (C(A,B') not on-site, Z(B,E'')) of C(A,B')[P on B'][i][j] Z[P][j][l].
__global__ void __launch_bounds__(NT) k_X34(const int32_t *ord, const int64_t *ptr, const int2 *L,
                                            const int32_t *atomA3, const int32_t *atomB3, const int32_t *pB,
                                            const int32_t *nb, const int32_t *na,
                                            const double *__restrict__ C, const int64_t *offC,
                                            const uint8_t *keepC, const double *__restrict__ Z,
                                            const int64_t *off2, const int64_t *offK, double *X, int64_t zbase,
                                            int64_t zlo, int64_t zhi, int smb, const uint8_t *rep3) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int x = ord[blockIdx.x];
  // one orientation of each K block (the transpose partner carries the other), with
  // twice the weight of Z's 1/2; the self block keeps it
  const uint8_t r3 = rep3[x];
  if (!r3) return;
  const double w4 = r3 == 2 ? 1.0 : 2.0;
  const int a = atomA3[x], e = atomB3[x];
  const int nbA = nb[a], naA = na[a], nbE = nb[e];
  const int nel = nbA * nbE;
  double acc[XMAXE];
#pragma unroll
  for (int r = 0; r < XMAXE; r++) acc[r] = 0.0;
  for (int64_t it = ptr[x]; it < ptr[x + 1]; it++) {
    const int2 en = L[it];
    if (!keepC[en.x] || en.y < zlo || en.y >= zhi) continue;
    const int b = pB[en.x];
    const int nbB = nb[b], naB = na[b];
    const double *Cb = C + offC[en.x] + (int64_t)naA * nbA * nbB;
    const double *Zb = Z + (off2[en.y] - zbase);
    const int csz = nbA * nbB, zsz = nbB * nbE;
    const int pc = max(1, min(naB, smb / (csz + zsz)));
    for (int P0 = 0; P0 < naB; P0 += pc) {
      const int pn = min(pc, naB - P0);
      __syncthreads();
      for (int i = tid; i < pn * csz; i += NT) sm[i] = Cb[(int64_t)P0 * csz + i];
      for (int i = tid; i < pn * zsz; i += NT) sm[pn * csz + i] = Zb[(int64_t)P0 * zsz + i];
      __syncthreads();
      const double *Zs = sm + pn * csz;
#pragma unroll
      for (int r = 0; r < XMAXE; r++) {
        const int el = tid + r * NT;
        if (el < nel) {
          const int i = el / nbE, l = el - i * nbE;
          double v = acc[r];
          for (int P = 0; P < pn; P++) {
            const double *cr = sm + (P * nbA + i) * nbB;
            const double *zr = Zs + P * zsz + l;
            for (int j = 0; j < nbB; j++) v = fma(cr[j], zr[j * nbE], v);
          }
          acc[r] = v;
        }
      }
    }
  }
  double *out = X + offK[x];
#pragma unroll
  for (int r = 0; r < XMAXE; r++) {
    const int el = tid + r * NT;
    if (el < nel) out[el] += w4 * acc[r];
  }
}

// ------------------------------------------------------------------ K = X + X^T (image flipped)
// K(A,E,n) = X(A,E,n) + X(E,A,-n)^T (accumulate: added to K); a deterministic mixed
// build keeps the tensor-core part of X in 128-bit fixed point (X128) beside the FP64 part
__global__ void k_sym(int64_t nk, const int32_t *atomA3, const int32_t *atomB3, const int32_t *partner3,
                      const int32_t *nb, const int64_t *offK, const double *__restrict__ X,
                      const unsigned long long *X128, double *K, int accumulate) {
  const int64_t x = blockIdx.x;
  if (x >= nk) return;
  const int nbA = nb[atomA3[x]], nbE = nb[atomB3[x]];
  const int64_t oa = offK[x], ob = offK[partner3[x]];
  double *k = K + oa;
  for (int el = threadIdx.x; el < nbA * nbE; el += blockDim.x) {
    const int i = el / nbE, l = el - i * nbE;
    const int64_t ea = oa + el, eb = ob + l * nbA + i;
    double va = X[ea], vb = X[eb];
    if (X128) {
      va += from_x128(X128 + 2 * ea);
      vb += from_x128(X128 + 2 * eb);
    }
    const double v = va + vb;
    k[el] = accumulate ? k[el] + v : v;
  }
}

// ------------------------------------------------------------------ energy
// Pair p contributes sum_il D(B,A,-n)[l][i] K(A,B,n)[i][l]; each thread owns
// one pair, each CTA reduces its 256 pairs in a fixed tree.
__global__ void k_energy(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *partner,
                         const int32_t *map1to3, const int32_t *nb, const double *__restrict__ D,
                         const int64_t *offD, const uint8_t *keepD, const double *__restrict__ K,
                         const int64_t *offK, double *part) {
  __shared__ double red[256];
  const int64_t p = blockIdx.x * (int64_t)256 + threadIdx.x;
  double s = 0.0;
  if (p < np) {
    const int64_t q = partner[p];
    if (keepD[q]) {
      const int nbA = nb[pA[p]], nbB = nb[pB[p]];
      const double *dq = D + offD[q];
      const double *kb = K + offK[map1to3[p]];
      for (int i = 0; i < nbA; i++)
        for (int l = 0; l < nbB; l++) s = fma(dq[l * nbA + i], kb[i * nbB + l], s);
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// *Ex = scale * sum(part) (accumulate: *Ex += ...); scale -1/4 for the closed-shell energy
__global__ void k_energy_final(int64_t n, const double *part, double *Ex, double scale, int accumulate) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *Ex = accumulate ? *Ex + scale * red[0] : scale * red[0];
}

// ------------------------------------------------------------------ Gamma fold
__global__ void k_fold(int64_t ng, const int64_t *fold, const int32_t *atomA3, const int32_t *atomB3,
                       const int32_t *nb, const int64_t *offK, const int64_t *bofs, int64_t nbasis,
                       const double *__restrict__ K, double *Kd) {
  const int64_t gi = blockIdx.x;
  if (gi >= ng) return;
  const int64_t x0 = fold[gi], x1 = fold[gi + 1];
  const int a = atomA3[x0], e = atomB3[x0];
  const int nbA = nb[a], nbE = nb[e];
  for (int el = threadIdx.x; el < nbA * nbE; el += blockDim.x) {
    double s = 0.0;
    for (int64_t x = x0; x < x1; x++) s += K[offK[x] + el];
    const int i = el / nbE, l = el - i * nbE;
    Kd[(bofs[a] + i) * nbasis + bofs[e] + l] = s;
  }
}

rix_status last(rix_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return RIX_ECUDA;
  }
  return RIX_OK;
}

bool g_attr_done = false;

}  // namespace

rix_status rix_launch_pairs(rix_ctx *ctx, const double *d_xyz, const double *d_cell, const int nr[3],
                            int64_t *d_counts, const int64_t *d_rowptr, int64_t *d_keys, cudaStream_t st) {
  const int nat = ctx->nat;
  const int threads = 256;
  const int64_t blocks = ((int64_t)nat * 32 + threads - 1) / threads;
  k_pairs<<<(unsigned)blocks, threads, 0, st>>>(nat, d_xyz, d_cell, ctx->periodic ? 1 : 0, nr[0], nr[1], nr[2],
                                                ctx->rc * ctx->rc, ctx->rc > 0 ? 1 : 0, d_counts, d_rowptr, d_keys);
  return last(ctx, "k_pairs");
}

rix_status rix_launch_flags(rix_ctx *ctx, const double *arr, const int64_t *off, int64_t n, uint8_t *keep,
                            cudaStream_t st, float *norm) {
  if (n == 0) return RIX_OK;
  const int64_t blocks = (n * 32 + 255) / 256;
  k_flags<<<(unsigned)blocks, 256, 0, st>>>(arr, off, n, ctx->tau, keep, ctx->opt.product_tau > 0 ? norm : nullptr);
  return last(ctx, "k_flags");
}

// out[a] = max over the pairs (a, .) of norm (one thread per atom)
__global__ void k_atom_max(int nat, const int64_t *row1, const float *norm, float *out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nat) return;
  float m = 0.f;
  for (int64_t p = row1[a]; p < row1[a + 1]; p++) m = fmaxf(m, norm[p]);
  out[a] = m;
}

rix_status rix_launch_atom_max(rix_ctx *ctx, const float *norm, float *out, cudaStream_t st) {
  k_atom_max<<<(ctx->nat + 127) / 128, 128, 0, st>>>(ctx->nat, ctx->d_row1, norm, out);
  return last(ctx, "k_atom_max");
}

rix_status rix_launch_symcheck(rix_ctx *ctx, cudaStream_t st) {
  RIX_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int32_t), st));
  const int64_t blocks = (ctx->np * 32 + 255) / 256;
  k_symcheck<<<(unsigned)blocks, 256, 0, st>>>(ctx->np, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_onsite,
                                               ctx->d_nb, ctx->d_na, ctx->d_C, ctx->d_offC, ctx->d_V,
                                               ctx->d_offV, ctx->d_flag);
  return last(ctx, "k_symcheck");
}

namespace {

void set_attrs() {
  if (!g_attr_done) {
    cudaFuncSetAttribute(k_X12, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_MAX * 8);
    cudaFuncSetAttribute(k_Z, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_MAX * 8);
    cudaFuncSetAttribute(k_X34, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_MAX * 8);
    g_attr_done = true;
  }
}

// Z(B;E') for the Z work items [first, first + count) of block b.
rix_status launch_Z_items(rix_ctx *ctx, const double *D, int b, int64_t first, int64_t count, int smb,
                          cudaStream_t st) {
  set_attrs();
  if (!count) return RIX_OK;
  k_Z<<<(unsigned)count, NT, smb * 8, st>>>(ctx->d_itZ + ctx->segZ[b] + first, ctx->d_ptrZ, ctx->d_LZ,
                                            ctx->d_atomA2, ctx->d_atomB2, ctx->d_off2, ctx->d_pB, ctx->d_nb,
                                            ctx->d_na, ctx->d_C, ctx->d_offC, ctx->d_V, ctx->d_offV, D, ctx->d_offD,
                                            ctx->d_keepC, ctx->d_keepV, ctx->d_keepD, ctx->d_Z, ctx->blk_base[b],
                                            smb, ctx->have_mx ? ctx->d_ztc : nullptr, rix_pscreen(ctx));
  return last(ctx, "k_Z");
}

// terms 1+2 for the output blocks [first, first + count) of block b's launch order.
rix_status launch_X12_items(rix_ctx *ctx, int b, int64_t first, int64_t count, int smb, cudaStream_t st) {
  set_attrs();
  if (!count) return RIX_OK;
  k_X12<<<(unsigned)count, NT, smb * 8, st>>>(
      ctx->d_ordX12 + ctx->segX12[b] + first, ctx->d_ptrX12, ctx->d_LX12, ctx->d_atomA2, ctx->d_atomB2,
      ctx->d_map2to1, ctx->d_map2to3, ctx->d_pA, ctx->d_onsite, ctx->d_nb, ctx->d_na, ctx->d_C, ctx->d_offC,
      ctx->d_V, ctx->d_offV, ctx->d_keepC, ctx->d_keepV, ctx->d_T, ctx->d_off2, ctx->d_U, ctx->d_offU, ctx->d_offK,
      ctx->d_X, ctx->blk_base[b], smb, ctx->have_mx ? 0 : 1, ctx->have_mx ? ctx->d_t1tc : nullptr, ctx->d_rep1);
  return last(ctx, "k_X12");
}

// terms 3+4 (FP64) for the K blocks [first, first + count) of the launch order, Z of block b.
rix_status launch_X34_items(rix_ctx *ctx, int b, int64_t first, int64_t count, int smb, cudaStream_t st) {
  set_attrs();
  if (!count) return RIX_OK;
  const int64_t zlo = ctx->row2[ctx->blk_atom[b]], zhi = ctx->row2[ctx->blk_atom[b + 1]];
  k_X34<<<(unsigned)count, NT, smb * 8, st>>>(ctx->d_ordX34 + first, ctx->d_ptrX34, ctx->d_LX34, ctx->d_atomA3,
                                              ctx->d_atomB3, ctx->d_pB, ctx->d_nb, ctx->d_na, ctx->d_C, ctx->d_offC,
                                              ctx->d_keepC, ctx->d_Z, ctx->d_off2, ctx->d_offK, ctx->d_X,
                                              ctx->blk_base[b], zlo, zhi, smb, ctx->d_rep3);
  return last(ctx, "k_X34");
}

}  // namespace

// T(A,G') for the row atoms of block b (T buffer holds that block).  In mixed
// precision the buffer is cleared first and the tensor cores add the T blocks
// of their row atoms; k_T stores the others.
rix_status rix_launch_T_block(rix_ctx *ctx, const double *D, int b, cudaStream_t st) {
  const int64_t nT = ctx->segT[b + 1] - ctx->segT[b];
  const bool tc = ctx->have_mx && ctx->n_ttc > 0;
  if (tc) {
    const int64_t n = ctx->off2[ctx->row2[ctx->blk_atom[b + 1]]] - ctx->blk_base[b];
    RIX_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_T, 0, sizeof(double) * n, st));
  }
  if (nT) {
    k_T<<<(unsigned)nT, NT, 64 * 64 * 8, st>>>(ctx->d_itT + ctx->segT[b], ctx->d_ptrT, ctx->d_LT, ctx->d_atomA2,
                                               ctx->d_atomB2, ctx->d_off2, ctx->d_pB, ctx->d_nb, ctx->d_na,
                                               ctx->d_C, ctx->d_offC, D, ctx->d_offD, ctx->d_keepC, ctx->d_keepD,
                                               ctx->d_T, ctx->blk_base[b], tc ? ctx->d_ttc : nullptr,
                                               rix_pscreen(ctx));
    rix_status s = last(ctx, "k_T");
    if (s != RIX_OK) return s;
  }
  return tc ? rix_mixed_T(ctx, b, ctx->blk_base[b], D, st) : RIX_OK;
}

// Z(B;E') for the middle atoms of block b (Z buffer holds that block): the FP64
// kernel stores its part, then in mixed precision the tensor cores add theirs.
rix_status rix_launch_Z_block(rix_ctx *ctx, const double *D, int b, cudaStream_t st) {
  rix_status s = RIX_OK;
  if (ctx->have_mx && ctx->n_ztc == ctx->nat) {
    // every middle atom runs on the tensor cores: the FP64 kernel would only write zeros
    const int64_t n = ctx->off2[ctx->row2[ctx->blk_atom[b + 1]]] - ctx->blk_base[b];
    RIX_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_Z, 0, sizeof(double) * n, st));
  } else {
    s = launch_Z_items(ctx, D, b, 0, ctx->segZ[b + 1] - ctx->segZ[b], ctx->tile_Z, st);
  }
  if (s == RIX_OK && ctx->have_mx) s = rix_mixed_z(ctx, b, ctx->blk_base[b], D, st);
  return s;
}

rix_status rix_fp64_build(rix_ctx *ctx, const double *D, double *K, cudaStream_t st, int accumulate) {
  set_attrs();
  rix_status s;
  if ((s = rix_prof_mark(ctx, 0, st)) != RIX_OK) return s;
  if ((s = rix_launch_flags(ctx, D, ctx->d_offD, ctx->np, ctx->d_keepD, st, ctx->d_normD)) != RIX_OK) return s;
  if ((s = rix_prof_mark(ctx, 1, st)) != RIX_OK) return s;
  RIX_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_X, 0, sizeof(double) * ctx->offK[ctx->nk], st));
  if (ctx->d_X128)
    RIX_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_X128, 0, 2 * sizeof(unsigned long long) * ctx->offK[ctx->nk], st));
  // terms 1 and 2, one block of row atoms at a time (T resident for the block)
  for (int b = 0; b < ctx->nblk; b++) {
    const int64_t tbase = ctx->blk_base[b];
    if ((s = rix_launch_T_block(ctx, D, b, st)) != RIX_OK) return s;
    if (b == 0 && (s = rix_prof_mark(ctx, 2, st)) != RIX_OK) return s;
    const int64_t nU = ctx->segU[b + 1] - ctx->segU[b];
    if (nU) {
      k_U2<<<(unsigned)nU, NT, 0, st>>>(ctx->d_itU + ctx->segU[b], ctx->d_pA, ctx->d_pB, ctx->d_nb, ctx->d_na,
                                        ctx->d_V, ctx->d_offV, ctx->d_keepV, ctx->d_map1to2, ctx->d_T, ctx->d_off2,
                                        ctx->d_offU, ctx->d_U, tbase);
      if ((s = last(ctx, "k_U2")) != RIX_OK) return s;
    }
    if (b == 0 && (s = rix_prof_mark(ctx, 3, st)) != RIX_OK) return s;
    if ((!ctx->have_mx || ctx->n_t1tc < ctx->nat) &&
        (s = launch_X12_items(ctx, b, 0, ctx->segX12[b + 1] - ctx->segX12[b], ctx->tile_X12, st)) != RIX_OK)
      return s;
    // mixed precision, several row blocks: term 1 on the tensor cores while T of the block is resident
    if (ctx->have_mx && ctx->nblk > 1 && (s = rix_mixed_t1(ctx, b, tbase, st)) != RIX_OK) return s;
  }
  if ((s = rix_prof_mark(ctx, 4, st)) != RIX_OK) return s;
  // mixed precision: term 1 (single block) and term 2 on the tensor cores
  if (ctx->have_mx && ctx->nblk == 1 && (s = rix_mixed_t1(ctx, 0, ctx->blk_base[0], st)) != RIX_OK) return s;
  if (ctx->have_mx && (s = rix_mixed_t2(ctx, st)) != RIX_OK) return s;
  if ((s = rix_prof_mark(ctx, 5, st)) != RIX_OK) return s;
  // terms 3 and 4, one block of middle atoms B at a time (Z resident for the block)
  for (int b = 0; b < ctx->nblk; b++) {
    const int64_t zbase = ctx->blk_base[b];
    if ((s = rix_launch_Z_block(ctx, D, b, st)) != RIX_OK) return s;
    if (b == 0 && (s = rix_prof_mark(ctx, 6, st)) != RIX_OK) return s;
    if (ctx->have_mx) {
      if ((s = rix_mixed_x34(ctx, b, zbase, st)) != RIX_OK) return s;
    } else if ((s = launch_X34_items(ctx, b, 0, ctx->n_ordX34, ctx->tile_X34, st)) != RIX_OK) {
      return s;
    }
  }
  if ((s = rix_prof_mark(ctx, 7, st)) != RIX_OK) return s;
  k_sym<<<(unsigned)ctx->nk, 128, 0, st>>>(ctx->nk, ctx->d_atomA3, ctx->d_atomB3, ctx->d_partner3, ctx->d_nb,
                                           ctx->d_offK, ctx->d_X, ctx->d_X128, K, accumulate);
  if ((s = last(ctx, "k_sym")) != RIX_OK) return s;
  return rix_prof_mark(ctx, 8, st);
}

// ------------------------------------------------------------------ autotuner
// Picks the shared-memory tile budget of k_X12, k_Z and k_X34 (and with it
// their tile shapes and CTAs per SM) by timing each candidate on a slice of
// the real work items of the first memory-plan block; the choice is cached
// per system in a text file.  The analogue of the paper's auto-tuned Fock
// block size (Sec. "Initialization"), at the level of one GPU's tiles.
namespace {

constexpr int N_CAND = 4;
constexpr int CAND[N_CAND] = {4096, 8192, 12288, 16384};

std::string tune_key(const rix_ctx *ctx) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  snprintf(buf, sizeof buf, "%s|nat=%d|np=%lld|n2=%lld|nk=%lld|prec=%d|blk=%d|", prop.name, ctx->nat,
           (long long)ctx->np, (long long)ctx->n2, (long long)ctx->nk, (int)ctx->opt.precision, ctx->nblk);
  std::string k(buf);
  for (char &c : k)
    if (c == ' ') c = '_';
  return k;
}

// time `launch(c)` for every candidate c (one untimed run first); returns the fastest
template <class F>
rix_status pick(rix_ctx *ctx, cudaStream_t st, F launch, int *best, float *best_ms) {
  cudaEvent_t e0, e1;
  RIX_CUDA_TRY(ctx, cudaEventCreate(&e0));
  RIX_CUDA_TRY(ctx, cudaEventCreate(&e1));
  *best_ms = 3.0e38f;
  rix_status s = RIX_OK;
  for (int c = 0; c < N_CAND && s == RIX_OK; c++) {
    if ((s = launch(CAND[c])) != RIX_OK) break;
    cudaEventRecord(e0, st);
    if ((s = launch(CAND[c])) != RIX_OK) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { s = RIX_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < *best_ms) { *best_ms = ms; *best = CAND[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // namespace

extern "C" rix_status rix_autotune(rix_ctx *ctx, const double *D, const char *cache_path, int32_t *chosen,
                                   void *stream) {
  if (!ctx || !D) return RIX_EINVAL;
  if (!ctx->have_cv) return RIX_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    ctx->last_error = "rix_autotune times kernels and cannot run inside a graph capture";
    return RIX_ESTATE;
  }
  ctx->fwd_valid = false;  // the timing runs overwrite the intermediates
  const std::string key = tune_key(ctx);
  if (cache_path && *cache_path) {
    if (FILE *f = fopen(cache_path, "r")) {
      char line[1024];
      while (fgets(line, sizeof line, f)) {
        char k[600];
        int a = 0, b = 0, c = 0;
        if (sscanf(line, "%599s %d %d %d", k, &a, &b, &c) == 4 && key == k && a > 0 && b > 0 && c > 0 &&
            a <= SM_MAX && b <= SM_MAX && c <= SM_MAX) {
          ctx->tile_X12 = a, ctx->tile_Z = b, ctx->tile_X34 = c;
          fclose(f);
          if (chosen) chosen[0] = a, chosen[1] = b, chosen[2] = c;
          return RIX_OK;
        }
      }
      fclose(f);
    }
  }
  rix_status s;
  set_attrs();
  if ((s = rix_launch_flags(ctx, D, ctx->d_offD, ctx->np, ctx->d_keepD, st)) != RIX_OK) return s;
  RIX_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_X, 0, sizeof(double) * ctx->offK[ctx->nk], st));
  const int b = 0;
  const int64_t SAMPLE = 4096;
  // block 0's T and U2 feed the term 1+2 sample
  if ((s = rix_launch_T_block(ctx, D, b, st)) != RIX_OK) return s;
  const int64_t nU = ctx->segU[b + 1] - ctx->segU[b];
  if (nU) {
    k_U2<<<(unsigned)nU, NT, 0, st>>>(ctx->d_itU + ctx->segU[b], ctx->d_pA, ctx->d_pB, ctx->d_nb, ctx->d_na,
                                      ctx->d_V, ctx->d_offV, ctx->d_keepV, ctx->d_map1to2, ctx->d_T, ctx->d_off2,
                                      ctx->d_offU, ctx->d_U, ctx->blk_base[b]);
    if ((s = last(ctx, "k_U2")) != RIX_OK) return s;
  }
  float ms = 0.f;
  {
    const int64_t n = ctx->segX12[b + 1] - ctx->segX12[b], cnt = std::min(n, SAMPLE), first = (n - cnt) / 2;
    if (cnt && (s = pick(ctx, st, [&](int c) { return launch_X12_items(ctx, b, first, cnt, c, st); },
                         &ctx->tile_X12, &ms)) != RIX_OK)
      return s;
  }
  {
    const int64_t n = ctx->segZ[b + 1] - ctx->segZ[b], cnt = std::min(n, SAMPLE), first = (n - cnt) / 2;
    if (cnt && (s = pick(ctx, st, [&](int c) { return launch_Z_items(ctx, D, b, first, cnt, c, st); },
                         &ctx->tile_Z, &ms)) != RIX_OK)
      return s;
  }
  if (!ctx->have_mx && ctx->n_ordX34) {
    if ((s = rix_launch_Z_block(ctx, D, b, st)) != RIX_OK) return s;
    const int64_t n = ctx->n_ordX34, cnt = std::min(n, SAMPLE), first = (n - cnt) / 2;
    if ((s = pick(ctx, st, [&](int c) { return launch_X34_items(ctx, b, first, cnt, c, st); }, &ctx->tile_X34,
                  &ms)) != RIX_OK)
      return s;
  }
  RIX_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (cache_path && *cache_path) {
    if (FILE *f = fopen(cache_path, "a")) {
      fprintf(f, "%s %d %d %d\n", key.c_str(), ctx->tile_X12, ctx->tile_Z, ctx->tile_X34);
      fclose(f);
    }
  }
  if (chosen) chosen[0] = ctx->tile_X12, chosen[1] = ctx->tile_Z, chosen[2] = ctx->tile_X34;
  return RIX_OK;
}

rix_status rix_launch_energy(rix_ctx *ctx, const double *D, const double *K, double *Ex, cudaStream_t st) {
  rix_status s;
  if ((s = rix_launch_flags(ctx, D, ctx->d_offD, ctx->np, ctx->d_keepD, st)) != RIX_OK) return s;
  k_energy<<<(unsigned)ctx->n_epart, 256, 0, st>>>(ctx->np, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_map1to3,
                                                   ctx->d_nb, D, ctx->d_offD, ctx->d_keepD, K, ctx->d_offK,
                                                   ctx->d_epart);
  if ((s = last(ctx, "k_energy")) != RIX_OK) return s;
  k_energy_final<<<1, 1024, 0, st>>>(ctx->n_epart, ctx->d_epart, Ex, -0.25, 0);
  return last(ctx, "k_energy_final");
}

// scale * sum over the D pattern of <D(E,A,-n), K(A,E,n)> into (or added to) *Ex
rix_status rix_launch_energy_scaled(rix_ctx *ctx, const double *D, const double *K, double *Ex, double scale,
                                    int accumulate, cudaStream_t st) {
  rix_status s;
  if ((s = rix_launch_flags(ctx, D, ctx->d_offD, ctx->np, ctx->d_keepD, st)) != RIX_OK) return s;
  k_energy<<<(unsigned)ctx->n_epart, 256, 0, st>>>(ctx->np, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_map1to3,
                                                   ctx->d_nb, D, ctx->d_offD, ctx->d_keepD, K, ctx->d_offK,
                                                   ctx->d_epart);
  if ((s = last(ctx, "k_energy")) != RIX_OK) return s;
  k_energy_final<<<1, 1024, 0, st>>>(ctx->n_epart, ctx->d_epart, Ex, scale, accumulate);
  return last(ctx, "k_energy_final");
}

// Same energy reduction as rix_launch_energy, with the per-CTA partial sums in
// a caller-supplied device buffer of at least ctx->n_epart doubles.
rix_status rix_launch_energy_partials(rix_ctx *ctx, const double *D, const double *K, double *Ex, double *partials,
                                      cudaStream_t st) {
  rix_status s;
  if ((s = rix_launch_flags(ctx, D, ctx->d_offD, ctx->np, ctx->d_keepD, st)) != RIX_OK) return s;
  k_energy<<<(unsigned)ctx->n_epart, 256, 0, st>>>(ctx->np, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_map1to3,
                                                   ctx->d_nb, D, ctx->d_offD, ctx->d_keepD, K, ctx->d_offK,
                                                   partials);
  if ((s = last(ctx, "k_energy")) != RIX_OK) return s;
  k_energy_final<<<1, 1024, 0, st>>>(ctx->n_epart, partials, Ex, -0.25, 0);
  return last(ctx, "k_energy_final");
}

rix_status rix_launch_fold(rix_ctx *ctx, const double *K, double *Kd, cudaStream_t st) {
  RIX_CUDA_TRY(ctx, cudaMemsetAsync(Kd, 0, sizeof(double) * ctx->nbasis * ctx->nbasis, st));
  k_fold<<<(unsigned)ctx->n_fold, 128, 0, st>>>(ctx->n_fold, ctx->d_fold, ctx->d_atomA3, ctx->d_atomB3, ctx->d_nb,
                                                ctx->d_offK, ctx->d_bofs, ctx->nbasis, K, Kd);
  return last(ctx, "k_fold");
}
