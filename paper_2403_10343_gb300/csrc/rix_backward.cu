// rix_backward: gradients of E_x with respect to the stored D, C and V entries.
//
// Reverse mode through the stages of the forward build (rix_fp64.cu).  With
// E = -1/4 sum_p <D(partner p)^T, K(p)> and K = X + X^T, the adjoint of X is
// Xbar(A,E') = -1/2 gEx D(A,E') on the pair list and zero elsewhere, so only
// outputs on the pair list propagate.  The forward intermediates T, U2 and Z
// are recomputed by a forward pass (nothing is kept between calls); when the
// memory plan splits the row atoms into blocks, T and Z are recomputed once
// more per block, and Tbar and Zbar overwrite T and Z in the same buffers
// after their last reader has run.  The
// paper obtains forces and stress by differentiating the same contraction
// (Sec. "EXX force and stress contributions"); dE/dC and dE/dV are the
// quantities those chain through.
//
// Every stored entry is an independent variable for the reverse pass; the
// results are then symmetrised over transpose partners, which yields the
// partial derivatives of the four-index formula itself (for symmetric inputs
// the two agree on every symmetric direction).  dE/dD = -1/2 gEx K exactly.
#include "rix_internal.h"

using namespace rix;


namespace {

constexpr int NT = 256;
constexpr int MAXE = 32;
constexpr int CAP = NT * MAXE;
constexpr int SM_BIG = 12288;

__device__ __forceinline__ int tile_rows(int per) { return max(1, CAP / per); }

// The 2-hop blocks [lo, hi) resident in the T or Z buffer (one block of row
// atoms); block i sits at off2[i] - base in the buffer.
struct Win {
  int64_t lo, hi, base;
};
__device__ __forceinline__ bool in_win(const Win &w, int64_t i) { return i >= w.lo && i < w.hi; }

// ---------------------------------------------------------------- Cbar(A,B')[P on B']
// += sum over (pair (A,E'), Z(B,E')) of sum_l Xbar(A,E')[i][l] Z[P][j][l]
__global__ void __launch_bounds__(NT) kb_C34(const int4 *items, const int64_t *ptr, const int2 *L, const int32_t *pA,
                                             const int32_t *pB, const int32_t *nb, const int32_t *na,
                                             const double *__restrict__ D, const int64_t *offD,
                                             const double *__restrict__ Z, const int64_t *off2, const int64_t *offC,
                                             const uint8_t *keepC, double sX, Win w, double *dC) {
  const int4 it = items[blockIdx.x];
  const int p1 = it.x, p0 = it.y;
  if (!keepC[p1]) return;
  const int a = pA[p1], b = pB[p1];
  const int nbA = nb[a], naA = na[a], nbB = nb[b], naB = na[b];
  const int per = nbA * nbB;
  const int pe = min(naB, p0 + tile_rows(per));
  const int nel = (pe - p0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[p1]; x < ptr[p1 + 1]; x++) {
    const int2 en = L[x];
    if (!in_win(w, en.y)) continue;
    const int e = pB[en.x];
    const int nbE = nb[e];
    const double *Xb = D + offD[en.x];
    const double *Zb = Z + (off2[en.y] - w.base);
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = threadIdx.x + r * NT;
      if (el < nel) {
        const int P = p0 + el / per, rem = el % per;
        const int i = rem / nbB, j = rem - i * nbB;
        const double *xr = Xb + i * nbE;
        const double *zr = Zb + ((int64_t)P * nbB + j) * nbE;
        double v = acc[r];
        for (int l = 0; l < nbE; l++) v = fma(xr[l], zr[l], v);
        acc[r] = v;
      }
    }
  }
  double *out = dC + offC[p1] + ((int64_t)naA + p0) * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] += sX * acc[r];
  }
}

// ---------------------------------------------------------------- Zbar(B,E')
// = sum over (pair (A,B') not on-site, pair (A,E')) of sum_i C(A,B')[P on B'][i][j] Xbar(A,E')[i][l]
__global__ void __launch_bounds__(NT) kb_Z34(const int4 *items, const int64_t *ptr, const int2 *L,
                                             const int32_t *atomA2, const int32_t *atomB2, const int32_t *pA,
                                             const int32_t *nb, const int32_t *na, const double *__restrict__ C,
                                             const int64_t *offC, const uint8_t *keepC,
                                             const double *__restrict__ D, const int64_t *offD,
                                             const int64_t *off2, double sX, Win w, double *Zbar) {
  const int4 it = items[blockIdx.x];
  const int z = it.x, p0 = it.y;
  if (!in_win(w, z)) return;
  const int b = atomA2[z], e = atomB2[z];
  const int nbB = nb[b], naB = na[b], nbE = nb[e];
  const int per = nbB * nbE;
  const int pe = min(naB, p0 + tile_rows(per));
  const int nel = (pe - p0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[z]; x < ptr[z + 1]; x++) {
    const int2 en = L[x];
    if (!keepC[en.x]) continue;
    const int a = pA[en.x];
    const int nbA = nb[a], naA = na[a];
    const double *Cb = C + offC[en.x] + (int64_t)naA * nbA * nbB;
    const double *Xb = D + offD[en.y];
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = threadIdx.x + r * NT;
      if (el < nel) {
        const int P = p0 + el / per, rem = el % per;
        const int j = rem / nbE, l = rem - j * nbE;
        const double *cp = Cb + (int64_t)P * nbA * nbB + j;
        double v = acc[r];
        for (int i = 0; i < nbA; i++) v = fma(cp[i * nbB], Xb[i * nbE + l], v);
        acc[r] = v;
      }
    }
  }
  double *out = Zbar + (off2[z] - w.base) + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] = sX * acc[r];
  }
}

// ---------------------------------------------------------------- Vbar(B,G') from term 4
// Fbar[P][k][l] = 1/2 sum_j D(B,G')[j][k] Zbar(B,E')[P][j][l];  Vbar[P][Q] += sum_kl Fbar C(G',E')[Q on G'][k][l]
__global__ void __launch_bounds__(NT) kb_ZV(const int4 *items, const int64_t *ptr, const int2 *L, const int32_t *pA,
                                            const int32_t *pB, const int32_t *nb, const int32_t *na,
                                            const double *__restrict__ C, const int64_t *offC,
                                            const double *__restrict__ D, const int64_t *offD,
                                            const uint8_t *keepC, const uint8_t *keepV, const uint8_t *keepD,
                                            const double *__restrict__ Zbar, const int64_t *off2,
                                            const int64_t *offV, Win w, double *dV) {
  extern __shared__ double sm[];
  const int4 it = items[blockIdx.x];
  const int p2 = it.x, p0 = it.y;
  if (!keepD[p2] || !keepV[p2]) return;
  const int b = pA[p2], g = pB[p2];
  const int nbB = nb[b], naB = na[b], nbG = nb[g], naG = na[g];
  const int per = naG;
  const int pe = min(naB, p0 + tile_rows(per));
  const int nel = (pe - p0) * per;
  const double *Dbg = D + offD[p2];
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[p2]; x < ptr[p2 + 1]; x++) {
    const int2 en = L[x];
    if (!keepC[en.x] || !in_win(w, en.y)) continue;
    const int e = pB[en.x];
    const int nbE = nb[e];
    const double *Cg = C + offC[en.x];
    const double *Zb = Zbar + (off2[en.y] - w.base);
    const int fper = nbG * nbE;
    const int ft = max(1, min(pe - p0, SM_BIG / fper));
    for (int ps = p0; ps < pe; ps += ft) {
      const int fn = min(ft, pe - ps);
      __syncthreads();
      for (int el = threadIdx.x; el < fn * fper; el += NT) {
        const int pp = el / fper, rem = el - pp * fper;
        const int k = rem / nbE, l = rem - k * nbE;
        const double *zr = Zb + (int64_t)(ps + pp) * nbB * nbE + l;
        double f = 0.0;
        for (int j = 0; j < nbB; j++) f = fma(Dbg[j * nbG + k], zr[j * nbE], f);
        sm[el] = 0.5 * f;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = threadIdx.x + r * NT;
        if (el < nel) {
          const int P = el / per;
          const int pr = P - (ps - p0);
          if (pr >= 0 && pr < fn) {
            const int Q = el - P * per;
            const double *fr = sm + pr * fper;
            const double *cq = Cg + (int64_t)Q * fper;
            double v = acc[r];
            for (int c = 0; c < fper; c++) v = fma(fr[c], cq[c], v);
            acc[r] = v;
          }
        }
      }
    }
  }
  double *out = dV + offV[p2] + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] += acc[r];
  }
}

// ---------------------------------------------------------------- Cbar(G',E')[Q on G'] from term 4
// += sum over (pair (B,G'), Z(B,E')) of sum_P V(B,G')[P][Q] Fbar[P][k][l]
__global__ void __launch_bounds__(NT) kb_ZC(const int4 *items, const int64_t *ptr, const int2 *L, const int32_t *pA,
                                            const int32_t *pB, const int32_t *nb, const int32_t *na,
                                            const double *__restrict__ V, const int64_t *offV,
                                            const double *__restrict__ D, const int64_t *offD,
                                            const uint8_t *keepC, const uint8_t *keepV, const uint8_t *keepD,
                                            const double *__restrict__ Zbar, const int64_t *off2,
                                            const int64_t *offC, Win w, double *dC) {
  extern __shared__ double sm[];
  const int4 it = items[blockIdx.x];
  const int p3 = it.x, q0 = it.y;
  if (!keepC[p3]) return;
  const int g = pA[p3], e = pB[p3];
  const int nbG = nb[g], naG = na[g], nbE = nb[e];
  const int per = nbG * nbE;
  const int qe = min(naG, q0 + tile_rows(per));
  const int nel = (qe - q0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[p3]; x < ptr[p3 + 1]; x++) {
    const int2 en = L[x];
    if (!keepD[en.x] || !keepV[en.x] || !in_win(w, en.y)) continue;
    const int b = pA[en.x];
    const int nbB = nb[b], naB = na[b];
    const double *Dbg = D + offD[en.x];
    const double *Vbg = V + offV[en.x];
    const double *Zb = Zbar + (off2[en.y] - w.base);
    const int pc = max(1, min(naB, SM_BIG / per));
    for (int P0 = 0; P0 < naB; P0 += pc) {
      const int pn = min(pc, naB - P0);
      __syncthreads();
      for (int el = threadIdx.x; el < pn * per; el += NT) {
        const int pp = el / per, rem = el - pp * per;
        const int k = rem / nbE, l = rem - k * nbE;
        const double *zr = Zb + (int64_t)(P0 + pp) * nbB * nbE + l;
        double f = 0.0;
        for (int j = 0; j < nbB; j++) f = fma(Dbg[j * nbG + k], zr[j * nbE], f);
        sm[el] = 0.5 * f;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = threadIdx.x + r * NT;
        if (el < nel) {
          const int Q = q0 + el / per, c = el % per;
          double v = acc[r];
          for (int pp = 0; pp < pn; pp++) v = fma(Vbg[(int64_t)(P0 + pp) * naG + Q], sm[pp * per + c], v);
          acc[r] = v;
        }
      }
    }
  }
  double *out = dC + offC[p3] + (int64_t)q0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] += acc[r];
  }
}

// ---------------------------------------------------------------- U2bar(A,G')
// = sum over (block (A,E') on the pair list, pair (G',E')) of sum_l Xbar(A,E')[i][l] C(G',E')[Q on G'][k][l]
__global__ void __launch_bounds__(NT) kb_U2(const int4 *items, const int64_t *ptr, const int2 *L, const int32_t *pA,
                                            const int32_t *pB, const int32_t *nb, const int32_t *na,
                                            const int32_t *map2to1, const double *__restrict__ C,
                                            const int64_t *offC, const uint8_t *keepC,
                                            const double *__restrict__ D, const int64_t *offD,
                                            const int64_t *offU, double sX, double *U2bar) {
  const int4 it = items[blockIdx.x];
  const int u2 = it.x, q0 = it.y;
  const int a = pA[u2], g = pB[u2];
  const int nbA = nb[a], nbG = nb[g], naG = na[g];
  const int per = nbA * nbG;
  const int qe = min(naG, q0 + tile_rows(per));
  const int nel = (qe - q0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[u2]; x < ptr[u2 + 1]; x++) {
    const int2 en = L[x];
    if (!keepC[en.y]) continue;
    const int pae = map2to1[en.x];
    const int e = pB[en.y];
    const int nbE = nb[e];
    const double *Xb = D + offD[pae];
    const double *Cg = C + offC[en.y];
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = threadIdx.x + r * NT;
      if (el < nel) {
        const int Q = q0 + el / per, rem = el % per;
        const int i = rem / nbG, k = rem - i * nbG;
        const double *xr = Xb + i * nbE;
        const double *cr = Cg + ((int64_t)Q * nbG + k) * nbE;
        double v = acc[r];
        for (int l = 0; l < nbE; l++) v = fma(xr[l], cr[l], v);
        acc[r] = v;
      }
    }
  }
  double *out = U2bar + offU[u2] + (int64_t)q0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] = sX * acc[r];
  }
}

// ---------------------------------------------------------------- Tbar(A,G')
// term 1: Ubar1[Q][i][k] = 1/2 sum_l Xbar(A,E')[i][l] C(G',E')[Q on E'][k][l], Tbar += V(A,E') Ubar1
// term 2: Tbar += V(A,G') U2bar(A,G')
__global__ void __launch_bounds__(NT) kb_T(const int4 *items, const int64_t *ptr, const int2 *L,
                                           const int32_t *atomA2, const int32_t *atomB2, const int32_t *map2to1,
                                           const int32_t *pA, const uint8_t *onsite, const int32_t *nb,
                                           const int32_t *na, const double *__restrict__ C, const int64_t *offC,
                                           const double *__restrict__ V, const int64_t *offV,
                                           const double *__restrict__ D, const int64_t *offD,
                                           const uint8_t *keepC, const uint8_t *keepV, const int64_t *ptrU2,
                                           const double *__restrict__ U2bar, const int64_t *offU,
                                           const int64_t *off2, double sX, Win w, double *Tbar) {
  extern __shared__ double sm[];
  const int4 it = items[blockIdx.x];
  const int t = it.x, p0 = it.y;
  if (!in_win(w, t)) return;
  const int a = atomA2[t], g = atomB2[t];
  const int nbA = nb[a], naA = na[a], nbG = nb[g], naG = na[g];
  const int per = nbA * nbG;
  const int pe = min(naA, p0 + tile_rows(per));
  const int nel = (pe - p0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[t]; x < ptr[t + 1]; x++) {
    const int2 en = L[x];
    const int pae = map2to1[en.x];
    if (!keepC[en.y] || !keepV[pae]) continue;
    const int e = atomB2[en.x];
    const int nbE = nb[e], naE = na[e];
    const int qE0 = onsite[en.y] ? 0 : naG;
    const double *Xb = D + offD[pae];
    const double *Ce = C + offC[en.y] + (int64_t)qE0 * nbG * nbE;
    const double *Vae = V + offV[pae];
    const int qt = max(1, min(naE, SM_BIG / per));
    for (int q0 = 0; q0 < naE; q0 += qt) {
      const int qn = min(qt, naE - q0);
      __syncthreads();
      for (int el = threadIdx.x; el < qn * per; el += NT) {
        const int q = el / per, rem = el - q * per;
        const int i = rem / nbG, k = rem - i * nbG;
        const double *xr = Xb + i * nbE;
        const double *cr = Ce + ((int64_t)(q0 + q) * nbG + k) * nbE;
        double u = 0.0;
        for (int l = 0; l < nbE; l++) u = fma(xr[l], cr[l], u);
        sm[el] = 0.5 * sX * u;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = threadIdx.x + r * NT;
        if (el < nel) {
          const int P = p0 + el / per, c = el % per;
          const double *vr = Vae + (int64_t)P * naE + q0;
          double v = acc[r];
          for (int q = 0; q < qn; q++) v = fma(vr[q], sm[q * per + c], v);
          acc[r] = v;
        }
      }
    }
  }
  const int pag = map2to1[t];
  if (pag >= 0 && keepV[pag] && ptrU2[pag + 1] > ptrU2[pag]) {
    const double *Vag = V + offV[pag];
    const double *Ub = U2bar + offU[pag];
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = threadIdx.x + r * NT;
      if (el < nel) {
        const int P = p0 + el / per, c = el % per;
        double v = acc[r];
        for (int Q = 0; Q < naG; Q++) v = fma(Vag[(int64_t)P * naG + Q], Ub[(int64_t)Q * per + c], v);
        acc[r] = v;
      }
    }
  }
  double *out = Tbar + (off2[t] - w.base) + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] = acc[r];
  }
}

// ---------------------------------------------------------------- Vbar(A,X) from terms 1 and 2
// term 1 (X = E'): Vbar[P][Q] += sum_G' sum_ik T(A,G')[P][i][k] Ubar1[Q][i][k]
// term 2 (X = G'): Vbar[P][Q] += sum_ik T(A,G')[P][i][k] U2bar(A,G')[Q][i][k]
__global__ void __launch_bounds__(NT) kb_V12(const int4 *items, const int64_t *ptrX12, const X12Entry *LX12,
                                             const int32_t *map1to2, const int32_t *pA, const int32_t *pB,
                                             const uint8_t *onsite, const int32_t *nb, const int32_t *na,
                                             const double *__restrict__ C, const int64_t *offC,
                                             const double *__restrict__ D, const int64_t *offD,
                                             const uint8_t *keepC, const uint8_t *keepV,
                                             const double *__restrict__ T, const int64_t *off2,
                                             const int64_t *ptrU2, const double *__restrict__ U2bar,
                                             const int64_t *offU, const int64_t *offV, double sX, Win w,
                                             double *dV) {
  extern __shared__ double sm[];
  const int4 it = items[blockIdx.x];
  const int p = it.x, p0 = it.y;
  // every T block this item reads has the row atom of pair p: it is resident iff T(A,X) is
  const int s = map1to2[p];
  if (!keepV[p] || !in_win(w, s)) return;
  const int a = pA[p], xa = pB[p];
  const int nbA = nb[a], naA = na[a], naX = na[xa], nbX = nb[xa];
  const int per = naX;
  const int pe = min(naA, p0 + tile_rows(per));
  const int nel = (pe - p0) * per;
  (void)naA;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  const double *Xb = D + offD[p];
  for (int64_t x = ptrX12[s]; x < ptrX12[s + 1]; x++) {
    const X12Entry en = LX12[x];
    if (!en.t1 || !keepC[en.p3]) continue;
    const int g = pA[en.p3];
    const int nbG = nb[g], naG = na[g];
    const int qE0 = onsite[en.p3] ? 0 : naG;
    const int uper = nbA * nbG;
    const double *Ce = C + offC[en.p3] + (int64_t)qE0 * nbG * nbX;
    const double *Tt = T + (off2[en.t] - w.base);
    const int qt = max(1, min(naX, SM_BIG / uper));
    for (int q0 = 0; q0 < naX; q0 += qt) {
      const int qn = min(qt, naX - q0);
      __syncthreads();
      for (int el = threadIdx.x; el < qn * uper; el += NT) {
        const int q = el / uper, rem = el - q * uper;
        const int i = rem / nbG, k = rem - i * nbG;
        const double *xr = Xb + i * nbX;
        const double *cr = Ce + ((int64_t)(q0 + q) * nbG + k) * nbX;
        double u = 0.0;
        for (int l = 0; l < nbX; l++) u = fma(xr[l], cr[l], u);
        sm[el] = 0.5 * sX * u;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = threadIdx.x + r * NT;
        if (el < nel) {
          const int P = p0 + el / per, Q = el % per;
          if (Q >= q0 && Q < q0 + qn) {
            const double *tr = Tt + (int64_t)P * uper;
            const double *ur = sm + (Q - q0) * uper;
            double v = acc[r];
            for (int c = 0; c < uper; c++) v = fma(tr[c], ur[c], v);
            acc[r] = v;
          }
        }
      }
    }
  }
  if (ptrU2[p + 1] > ptrU2[p]) {
    const int uper = nbA * nbX;
    const double *Tt = T + (off2[s] - w.base);
    const double *Ub = U2bar + offU[p];
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = threadIdx.x + r * NT;
      if (el < nel) {
        const int P = p0 + el / per, Q = el % per;
        const double *tr = Tt + (int64_t)P * uper;
        const double *ur = Ub + (int64_t)Q * uper;
        double v = acc[r];
        for (int c = 0; c < uper; c++) v = fma(tr[c], ur[c], v);
        acc[r] = v;
      }
    }
  }
  double *out = dV + offV[p] + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] += acc[r];
  }
}

// ---------------------------------------------------------------- Cbar(G',E') from terms 1 and 2
// term 1: Cbar[Q on E'][k][l] += 1/2 sum_i U1[Q][i][k] Xbar(A,E')[i][l], U1 = V(A,E')^T T(A,G')
// term 2: Cbar[Q on G'][k][l] += sum_i U2(A,G')[Q][i][k] Xbar(A,E')[i][l]
__global__ void __launch_bounds__(NT) kb_C12(const int4 *items, const int64_t *ptr, const BX12Entry *L,
                                             const int32_t *atomA2, const int32_t *map2to1, const int32_t *pA,
                                             const int32_t *pB, const uint8_t *onsite, const int32_t *nb,
                                             const int32_t *na, const double *__restrict__ V, const int64_t *offV,
                                             const double *__restrict__ D, const int64_t *offD,
                                             const uint8_t *keepC, const uint8_t *keepV,
                                             const double *__restrict__ T, const int64_t *off2,
                                             const double *__restrict__ U, const int64_t *offU,
                                             const int64_t *offC, double sX, Win w, double *dC) {
  extern __shared__ double sm[];
  const int4 it = items[blockIdx.x];
  const int p3 = it.x, r0 = it.y;
  if (!keepC[p3]) return;
  const int g = pA[p3], e = pB[p3];
  const int nbG = nb[g], naG = na[g], nbE = nb[e], naE = na[e];
  const int qE0 = onsite[p3] ? 0 : naG;
  const int rows = qE0 + naE;
  const int per = nbG * nbE;
  const int rt = max(1, min(CAP / per, SM_BIG / (64 * nbG)));
  const int re = min(rows, r0 + rt);
  const int nel = (re - r0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  // rows of this tile that belong to aux(E') (term 1)
  const int q1lo = max(r0, qE0) - qE0, q1hi = re - qE0;  // Q range [q1lo, q1hi)
  for (int64_t x = ptr[p3]; x < ptr[p3 + 1]; x++) {
    const BX12Entry en = L[x];
    if (!in_win(w, en.t)) continue;  // uniform across the CTA
    const int a = atomA2[en.t];
    const int nbA = nb[a], naA = na[a];
    const int pae = map2to1[en.s];
    const double *Xb = D + offD[pae];
    if (en.t1 && keepV[pae] && q1hi > q1lo) {
      const int uper = nbA * nbG;
      const double *Tt = T + (off2[en.t] - w.base);
      const double *Vae = V + offV[pae];
      const int qn = q1hi - q1lo;
      __syncthreads();
      for (int el = threadIdx.x; el < qn * uper; el += NT) {
        const int q = el / uper, c = el - q * uper;
        double u = 0.0;
        for (int P = 0; P < naA; P++) u = fma(Vae[(int64_t)P * naE + q1lo + q], Tt[(int64_t)P * uper + c], u);
        sm[el] = u;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = threadIdx.x + r * NT;
        if (el < nel) {
          const int row = r0 + el / per, rem = el % per;
          const int q = row - qE0 - q1lo;
          if (row >= qE0 && q >= 0 && q < qn) {
            const int k = rem / nbE, l = rem - k * nbE;
            const double *ur = sm + q * uper + k;
            double v = 0.0;
            for (int i = 0; i < nbA; i++) v = fma(ur[i * nbG], Xb[i * nbE + l], v);
            acc[r] = fma(0.5 * sX, v, acc[r]);
          }
        }
      }
    }
    if (en.u2 >= 0 && keepV[en.u2] && !onsite[p3]) {
      const double *U2 = U + offU[en.u2];
#pragma unroll
      for (int r = 0; r < MAXE; r++) {
        const int el = threadIdx.x + r * NT;
        if (el < nel) {
          const int row = r0 + el / per, rem = el % per;
          if (row < naG) {
            const int k = rem / nbE, l = rem - k * nbE;
            const double *ur = U2 + ((int64_t)row * nbA) * nbG + k;
            double v = 0.0;
            for (int i = 0; i < nbA; i++) v = fma(ur[i * nbG], Xb[i * nbE + l], v);
            acc[r] = fma(sX, v, acc[r]);
          }
        }
      }
    }
  }
  double *out = dC + offC[p3] + (int64_t)r0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] += acc[r];
  }
}

// ---------------------------------------------------------------- Cbar(A,B')[P on A] from T
// += sum over (pair (B',G'), T(A,G')) of sum_k Tbar[P][i][k] D(B',G')[j][k]
__global__ void __launch_bounds__(NT) kb_TC(const int4 *items, const int64_t *ptr, const int2 *L, const int32_t *pA,
                                            const int32_t *pB, const int32_t *nb, const int32_t *na,
                                            const double *__restrict__ D, const int64_t *offD,
                                            const uint8_t *keepC, const uint8_t *keepD,
                                            const double *__restrict__ Tbar, const int64_t *off2,
                                            const int64_t *offC, Win w, double *dC) {
  const int4 it = items[blockIdx.x];
  const int p1 = it.x, p0 = it.y;
  if (!keepC[p1]) return;
  const int a = pA[p1], b = pB[p1];
  const int nbA = nb[a], naA = na[a], nbB = nb[b];
  const int per = nbA * nbB;
  const int pe = min(naA, p0 + tile_rows(per));
  const int nel = (pe - p0) * per;
  double acc[MAXE];
#pragma unroll
  for (int r = 0; r < MAXE; r++) acc[r] = 0.0;
  for (int64_t x = ptr[p1]; x < ptr[p1 + 1]; x++) {
    const int2 en = L[x];
    if (!keepD[en.x] || !in_win(w, en.y)) continue;
    const int g = pB[en.x];
    const int nbG = nb[g];
    const double *Dbg = D + offD[en.x];
    const double *Tb = Tbar + (off2[en.y] - w.base);
#pragma unroll
    for (int r = 0; r < MAXE; r++) {
      const int el = threadIdx.x + r * NT;
      if (el < nel) {
        const int P = p0 + el / per, rem = el % per;
        const int i = rem / nbB, j = rem - i * nbB;
        const double *tr = Tb + ((int64_t)P * nbA + i) * nbG;
        const double *dr = Dbg + j * nbG;
        double v = acc[r];
        for (int k = 0; k < nbG; k++) v = fma(tr[k], dr[k], v);
        acc[r] = v;
      }
    }
  }
  double *out = dC + offC[p1] + (int64_t)p0 * per;
#pragma unroll
  for (int r = 0; r < MAXE; r++) {
    const int el = threadIdx.x + r * NT;
    if (el < nel) out[el] += acc[r];
  }
}

// ---------------------------------------------------------------- symmetrise over transpose partners
// dC: (p, [P][i][j]) <-> (partner, [P'][j][i]);  dV: (p, [P][Q]) <-> (partner, [Q][P]).
__global__ void kb_symC(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *partner,
                        const uint8_t *onsite, const int32_t *nb, const int32_t *na, const int64_t *offC, double *dC) {
  const int64_t p = blockIdx.x;
  if (p >= np) return;
  const int64_t q = partner[p];
  if (q < p) return;
  const int a = pA[p], b = pB[p];
  const int nbA = nb[a], nbB = nb[b], naA = na[a], naB = na[b];
  const int rows = naA + (onsite[p] ? 0 : naB);
  const int64_t n = (int64_t)rows * nbA * nbB;
  double *c = dC + offC[p], *cq = dC + offC[q];
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int P = (int)(e / (nbA * nbB));
    const int r = (int)(e % (nbA * nbB));
    const int i = r / nbB, j = r % nbB;
    if (onsite[p]) {
      if (i > j) continue;
      const int64_t e2 = ((int64_t)P * nbA + j) * nbB + i;
      const double v = 0.5 * (c[e] + c[e2]);
      c[e] = v;
      c[e2] = v;
    } else {
      const int Pq = P < naA ? P + naB : P - naA;
      const int64_t e2 = ((int64_t)Pq * nbB + j) * nbA + i;
      const double v = 0.5 * (c[e] + cq[e2]);
      c[e] = v;
      cq[e2] = v;
    }
  }
}

__global__ void kb_symV(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *partner,
                        const int32_t *na, const int64_t *offV, double *dV) {
  const int64_t p = blockIdx.x;
  if (p >= np) return;
  const int64_t q = partner[p];
  if (q < p) return;
  const int naA = na[pA[p]], naB = na[pB[p]];
  double *v = dV + offV[p], *vq = dV + offV[q];
  for (int e = threadIdx.x; e < naA * naB; e += blockDim.x) {
    const int P = e / naB, Q = e % naB;
    if (q == p && P > Q) continue;
    const double s = 0.5 * (v[e] + vq[Q * naA + P]);
    v[e] = s;
    vq[Q * naA + P] = s;
  }
}

// dD = -1/2 gEx K on the pair list (K is symmetric, so no further symmetrisation)
__global__ void kb_dD(int64_t np, const int32_t *pA, const int32_t *pB, const int32_t *map1to3, const int32_t *nb,
                      const int64_t *offD, const int64_t *offK, const double *__restrict__ K, double s,
                      double *dD) {
  const int64_t p = blockIdx.x;
  if (p >= np) return;
  const int n = nb[pA[p]] * nb[pB[p]];
  const double *k = K + offK[map1to3[p]];
  double *d = dD + offD[p];
  for (int e = threadIdx.x; e < n; e += blockDim.x) d[e] = s * k[e];
}

rix_status last_err(rix_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return RIX_ECUDA;
  }
  return RIX_OK;
}

bool g_bwd_attr = false;

}  // namespace

extern "C" rix_status rix_backward(rix_ctx *ctx, const double *D, double gEx, double *dD, double *dC, double *dV,
                                   void *stream) {
  if (!ctx || !D) return RIX_EINVAL;
  if (!ctx->have_cv) return RIX_ESTATE;
  if (!ctx->have_bwd) {
    ctx->last_error = "context set up without rix_options.backward";
    return RIX_ESTATE;
  }
  if (rix_status s0 = rix_take_err(ctx)) return s0;
  cudaStream_t st = (cudaStream_t)stream;
  if (!g_bwd_attr) {
    cudaFuncSetAttribute(kb_ZV, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_BIG * 8);
    cudaFuncSetAttribute(kb_ZC, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_BIG * 8);
    cudaFuncSetAttribute(kb_T, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_BIG * 8);
    cudaFuncSetAttribute(kb_V12, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_BIG * 8);
    cudaFuncSetAttribute(kb_C12, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_BIG * 8);
    g_bwd_attr = true;
  }
  // forward recompute: flags, T, U2, Z and K (U2 stays complete; T and Z hold the last block),
  // unless the preceding build of this D left them resident and the caller asked to reuse them
  const double *Kf = ctx->d_Kbuf;
  rix_status s = RIX_OK;
  if (ctx->opt.reuse_forward && ctx->fwd_valid && ctx->fwd_D == D && ctx->nblk == 1) {
    Kf = ctx->fwd_K;
  } else {
    s = rix_fp64_build(ctx, D, ctx->d_Kbuf, st);
    if (s != RIX_OK) return s;
  }
  ctx->fwd_valid = false;  // the adjoint overwrites T and Z below
  const double sX = -0.5 * gEx;
  const int64_t np = ctx->np;
  if (dD) {
    kb_dD<<<(unsigned)np, 128, 0, st>>>(np, ctx->d_pA, ctx->d_pB, ctx->d_map1to3, ctx->d_nb, ctx->d_offD,
                                        ctx->d_offK, Kf, -0.5 * gEx, dD);
    if ((s = last_err(ctx, "kb_dD")) != RIX_OK) return s;
  }
  if (!dC && !dV) return RIX_OK;
  // U2bar (term 2 adjoint) is per pair and needs no T
  if (ctx->n_itB[4]) {
    kb_U2<<<(unsigned)ctx->n_itB[4], NT, 0, st>>>(ctx->d_itB[4], ctx->d_ptrBU2, ctx->d_LBU2, ctx->d_pA, ctx->d_pB,
                                                  ctx->d_nb, ctx->d_na, ctx->d_map2to1, ctx->d_C, ctx->d_offC,
                                                  ctx->d_keepC, D, ctx->d_offD, ctx->d_offU, sX, ctx->d_U2bar);
    if ((s = last_err(ctx, "kb_U2")) != RIX_OK) return s;
  }
  if (dC) RIX_CUDA_TRY(ctx, cudaMemsetAsync(dC, 0, sizeof(double) * ctx->offC[np], st));
  if (dV) RIX_CUDA_TRY(ctx, cudaMemsetAsync(dV, 0, sizeof(double) * ctx->offV[np], st));
  const int nblk = ctx->nblk;
  // terms 1 and 2, one block of row atoms at a time: T (recomputed when the plan
  // has several blocks), its consumers, then Tbar into the same buffer
  for (int b = 0; b < nblk; b++) {
    const Win w{ctx->row2[ctx->blk_atom[b]], ctx->row2[ctx->blk_atom[b + 1]], ctx->blk_base[b]};
    if (nblk > 1 && (s = rix_launch_T_block(ctx, D, b, st)) != RIX_OK) return s;
    if (dC && ctx->n_itB[7]) {
      kb_C12<<<(unsigned)ctx->n_itB[7], NT, SM_BIG * 8, st>>>(
          ctx->d_itB[7], ctx->d_ptrBC12, ctx->d_LBC12, ctx->d_atomA2, ctx->d_map2to1, ctx->d_pA, ctx->d_pB,
          ctx->d_onsite, ctx->d_nb, ctx->d_na, ctx->d_V, ctx->d_offV, D, ctx->d_offD, ctx->d_keepC, ctx->d_keepV,
          ctx->d_T, ctx->d_off2, ctx->d_U, ctx->d_offU, ctx->d_offC, sX, w, dC);
      if ((s = last_err(ctx, "kb_C12")) != RIX_OK) return s;
    }
    if (dV && ctx->n_itB[6]) {
      kb_V12<<<(unsigned)ctx->n_itB[6], NT, SM_BIG * 8, st>>>(
          ctx->d_itB[6], ctx->d_ptrX12, ctx->d_LX12, ctx->d_map1to2, ctx->d_pA, ctx->d_pB, ctx->d_onsite, ctx->d_nb,
          ctx->d_na, ctx->d_C, ctx->d_offC, D, ctx->d_offD, ctx->d_keepC, ctx->d_keepV, ctx->d_T, ctx->d_off2,
          ctx->d_ptrBU2, ctx->d_U2bar, ctx->d_offU, ctx->d_offV, sX, w, dV);
      if ((s = last_err(ctx, "kb_V12")) != RIX_OK) return s;
    }
    if (dC && ctx->n_itB[5]) {
      kb_T<<<(unsigned)ctx->n_itB[5], NT, SM_BIG * 8, st>>>(
          ctx->d_itB[5], ctx->d_ptrBT1, ctx->d_LBT1, ctx->d_atomA2, ctx->d_atomB2, ctx->d_map2to1, ctx->d_pA,
          ctx->d_onsite, ctx->d_nb, ctx->d_na, ctx->d_C, ctx->d_offC, ctx->d_V, ctx->d_offV, D, ctx->d_offD,
          ctx->d_keepC, ctx->d_keepV, ctx->d_ptrBU2, ctx->d_U2bar, ctx->d_offU, ctx->d_off2, sX, w, ctx->d_T);
      if ((s = last_err(ctx, "kb_T")) != RIX_OK) return s;
      if (ctx->n_itB[8]) {
        kb_TC<<<(unsigned)ctx->n_itB[8], NT, 0, st>>>(ctx->d_itB[8], ctx->d_ptrBTC, ctx->d_LBTC, ctx->d_pA,
                                                      ctx->d_pB, ctx->d_nb, ctx->d_na, D, ctx->d_offD, ctx->d_keepC,
                                                      ctx->d_keepD, ctx->d_T, ctx->d_off2, ctx->d_offC, w, dC);
        if ((s = last_err(ctx, "kb_TC")) != RIX_OK) return s;
      }
    }
  }
  // terms 3 and 4, one block of middle atoms at a time: Z, its consumer, then Zbar
  for (int b = 0; b < nblk; b++) {
    const Win w{ctx->row2[ctx->blk_atom[b]], ctx->row2[ctx->blk_atom[b + 1]], ctx->blk_base[b]};
    if (nblk > 1 && (s = rix_launch_Z_block(ctx, D, b, st)) != RIX_OK) return s;
    if (dC && ctx->n_itB[0]) {
      kb_C34<<<(unsigned)ctx->n_itB[0], NT, 0, st>>>(ctx->d_itB[0], ctx->d_ptrBC34, ctx->d_LBC34, ctx->d_pA,
                                                     ctx->d_pB, ctx->d_nb, ctx->d_na, D, ctx->d_offD, ctx->d_Z,
                                                     ctx->d_off2, ctx->d_offC, ctx->d_keepC, sX, w, dC);
      if ((s = last_err(ctx, "kb_C34")) != RIX_OK) return s;
    }
    if (ctx->n_itB[1]) {
      kb_Z34<<<(unsigned)ctx->n_itB[1], NT, 0, st>>>(ctx->d_itB[1], ctx->d_ptrBZ34, ctx->d_LBZ34, ctx->d_atomA2,
                                                     ctx->d_atomB2, ctx->d_pA, ctx->d_nb, ctx->d_na, ctx->d_C,
                                                     ctx->d_offC, ctx->d_keepC, D, ctx->d_offD, ctx->d_off2, sX, w,
                                                     ctx->d_Z);
      if ((s = last_err(ctx, "kb_Z34")) != RIX_OK) return s;
    }
    if (dC && ctx->n_itB[3]) {
      kb_ZC<<<(unsigned)ctx->n_itB[3], NT, SM_BIG * 8, st>>>(
          ctx->d_itB[3], ctx->d_ptrBZC, ctx->d_LBZC, ctx->d_pA, ctx->d_pB, ctx->d_nb, ctx->d_na, ctx->d_V,
          ctx->d_offV, D, ctx->d_offD, ctx->d_keepC, ctx->d_keepV, ctx->d_keepD, ctx->d_Z, ctx->d_off2,
          ctx->d_offC, w, dC);
      if ((s = last_err(ctx, "kb_ZC")) != RIX_OK) return s;
    }
    if (dV && ctx->n_itB[2]) {
      kb_ZV<<<(unsigned)ctx->n_itB[2], NT, SM_BIG * 8, st>>>(
          ctx->d_itB[2], ctx->d_ptrBZV, ctx->d_LBZV, ctx->d_pA, ctx->d_pB, ctx->d_nb, ctx->d_na, ctx->d_C,
          ctx->d_offC, D, ctx->d_offD, ctx->d_keepC, ctx->d_keepV, ctx->d_keepD, ctx->d_Z, ctx->d_off2,
          ctx->d_offV, w, dV);
      if ((s = last_err(ctx, "kb_ZV")) != RIX_OK) return s;
    }
  }
  if (dC) {
    kb_symC<<<(unsigned)np, 128, 0, st>>>(np, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_onsite, ctx->d_nb,
                                         ctx->d_na, ctx->d_offC, dC);
    if ((s = last_err(ctx, "kb_symC")) != RIX_OK) return s;
  }
  if (dV) {
    kb_symV<<<(unsigned)np, 128, 0, st>>>(np, ctx->d_pA, ctx->d_pB, ctx->d_partner1, ctx->d_na, ctx->d_offV, dV);
    if ((s = last_err(ctx, "kb_symV")) != RIX_OK) return s;
  }
  return RIX_OK;
}
