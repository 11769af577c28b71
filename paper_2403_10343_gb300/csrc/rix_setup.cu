// rix_setup / layout / set_CV / stats / destroy: system setup and the product plan.
//
// The pair list (the paper's sparse bookkeeping of overlapping atom pairs,
// Sec. "General concepts") is built on the device; the 2-hop and 3-hop block
// lists and the per-output product lists are derived on the host once per
// geometry (the analogue of the paper's "Initialization" stage, which is not
// part of the per-iteration exchange build).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <omp.h>

#include "rix_internal.h"

using namespace rix;

rix_status rix_dev_alloc(rix_ctx *ctx, void **p, size_t bytes) {
  if (ctx->opt.max_workspace_bytes > 0 &&
      (int64_t)(ctx->dev_bytes + bytes) > ctx->opt.max_workspace_bytes) {
    ctx->last_error = "workspace limit exceeded";
    return RIX_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RIX_ENOMEM : RIX_ECUDA;
  }
  ctx->bufs.push_back({*p, bytes});
  ctx->dev_bytes += bytes;
  return RIX_OK;
}

#define TRY(x)                       \
  do {                               \
    rix_status s_ = (x);             \
    if (s_ != RIX_OK) return s_;     \
  } while (0)

namespace {

int64_t find_in(const std::vector<int64_t> &keys, int64_t lo, int64_t hi, int64_t key) {
  auto it = std::lower_bound(keys.begin() + lo, keys.begin() + hi, key);
  if (it == keys.begin() + hi || *it != key) return -1;
  return it - keys.begin();
}

inline int64_t key_add(int64_t a, int64_t b_atom, const int8_t *m1, const int8_t *m2, bool *ok) {
  int n[3];
  for (int c = 0; c < 3; c++) {
    n[c] = (int)m1[c] + (int)m2[c];
    if (n[c] < -127 || n[c] > 127) *ok = false;
  }
  return pair_key(a, b_atom, n[0], n[1], n[2]);
}

void decode_n(int64_t key, int8_t *n) {
  for (int c = 0; c < 3; c++) n[c] = (int8_t)key_n(key, c);
}

// image range with a one-cell margin: |n_i| <= floor(rc / h_i + w_i) + 1
void image_range(const rix_ctx *ctx, int nr[3]) {
  nr[0] = nr[1] = nr[2] = 0;
  if (!ctx->periodic) return;
  const double *a = ctx->cell;
  double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
               a[2] * (a[3] * a[7] - a[4] * a[6]);
  double inv[9] = {(a[4] * a[8] - a[5] * a[7]) / det, (a[2] * a[7] - a[1] * a[8]) / det,
                   (a[1] * a[5] - a[2] * a[4]) / det, (a[5] * a[6] - a[3] * a[8]) / det,
                   (a[0] * a[8] - a[2] * a[6]) / det, (a[2] * a[3] - a[0] * a[5]) / det,
                   (a[3] * a[7] - a[4] * a[6]) / det, (a[1] * a[6] - a[0] * a[7]) / det,
                   (a[0] * a[4] - a[1] * a[3]) / det};
  for (int d = 0; d < 3; d++) {
    const double *u = a + 3 * ((d + 1) % 3), *v = a + 3 * ((d + 2) % 3);
    double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    double h = std::fabs(det) / std::sqrt(cx * cx + cy * cy + cz * cz);
    double fmin = 1e300, fmax = -1e300;
    for (int i = 0; i < ctx->nat; i++) {
      double f = ctx->xyz[3 * i] * inv[0 * 3 + d] + ctx->xyz[3 * i + 1] * inv[1 * 3 + d] +
                 ctx->xyz[3 * i + 2] * inv[2 * 3 + d];
      fmin = std::min(fmin, f);
      fmax = std::max(fmax, f);
    }
    nr[d] = (int)std::floor(ctx->rc / h + (fmax - fmin)) + 1;
  }
}

// Stable counting sort of (key, payload) records whose keys lie in [lo, hi).
template <class P>
void group_by(int64_t lo, int64_t hi, const std::vector<int64_t> &keys, const std::vector<P> &pay,
              int64_t *ptr_out /* [hi-lo] starts, relative */, P *dst) {
  std::vector<int64_t> cnt(hi - lo + 1, 0);
  for (int64_t k : keys) cnt[k - lo + 1]++;
  for (int64_t i = 0; i < hi - lo; i++) cnt[i + 1] += cnt[i];
  for (int64_t i = 0; i < hi - lo; i++) ptr_out[i] = cnt[i];
  for (size_t e = 0; e < keys.size(); e++) dst[cnt[keys[e] - lo]++] = pay[e];
}

}  // namespace

// --------------------------------------------------------------------------
// Group (key, payload) records into CSR order, keeping input order within a key.
template <class P>
static void csr_group(int64_t nkeys, const std::vector<int64_t> &key, const std::vector<P> &pay,
                      std::vector<int64_t> &ptr, std::vector<P> &out) {
  ptr.assign(nkeys + 1, 0);
  for (int64_t k : key) ptr[k + 1]++;
  for (int64_t i = 0; i < nkeys; i++) ptr[i + 1] += ptr[i];
  std::vector<int64_t> pos(ptr.begin(), ptr.end() - 1);
  out.resize(key.size());
  for (size_t e = 0; e < key.size(); e++) out[pos[key[e]]++] = pay[e];
}

// Work items (output, first row) over `rows` rows of `per` elements each, rows per item
// chosen by the same rule as the kernels.
static void add_items(std::vector<int4> &it, int64_t out, int64_t rows, int64_t rt) {
  for (int64_t r0 = 0; r0 < rows; r0 += rt) it.push_back(make_int4((int)out, (int)r0, 0, 0));
}

// Product lists of the adjoint (reverse order of the stages of rix_build_K).  Only
// output blocks (A,E') on the pair list carry a nonzero adjoint, so every list is
// restricted to them.
static rix_status build_backward_lists(rix_ctx *ctx, const std::vector<int2> &LT, const std::vector<int64_t> &ptrT,
                                       const std::vector<X12Entry> &LX12, const std::vector<int64_t> &ptrX12,
                                       const std::vector<int2> &LZ, const std::vector<int64_t> &ptrZ,
                                       const std::vector<int32_t> &map1to2, const std::vector<int32_t> &map2to1,
                                       const std::vector<int32_t> &atomA2, const std::vector<int32_t> &atomB2) {
  const int nat = ctx->nat;
  const int64_t np = ctx->np, n2 = ctx->n2;
  auto &pA = ctx->pA, &pB = ctx->pB;
  auto &pn = ctx->pn;
  auto &row1 = ctx->row1, &row2 = ctx->row2;
  auto &keys2 = ctx->keys2;
  auto NB = [&](int a) { return (int64_t)ctx->nb_at[a]; };
  auto NA = [&](int a) { return (int64_t)ctx->na_at[a]; };
  auto find2 = [&](int64_t key) { int a = key_a(key); return find_in(keys2, row2[a], row2[a + 1], key); };
  const int64_t CAP = 8192, SMB = 12288;
  double fl = 0;

  // (pair (A,B') not on-site, pair (A,E')) -> Z(B, E'-n1)
  std::vector<int64_t> kBC, kBZ;
  std::vector<int2> vBC, vBZ;
  for (int a = 0; a < nat; a++)
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
      if (ctx->onsite[p1]) continue;
      int b = pB[p1];
      for (int64_t pae = row1[a]; pae < row1[a + 1]; pae++) {
        int e = pB[pae];
        int8_t m[3];
        bool ok = true;
        for (int c = 0; c < 3; c++) m[c] = (int8_t)(pn[3 * pae + c] - pn[3 * p1 + c]);
        int64_t z = find2(pair_key(b, e, m[0], m[1], m[2]));
        if (z < 0 || ptrZ[z + 1] == ptrZ[z] || !ok) continue;
        kBC.push_back(p1); vBC.push_back(make_int2((int)pae, (int)z));
        kBZ.push_back(z); vBZ.push_back(make_int2((int)p1, (int)pae));
        fl += 4.0 * NA(b) * NB(a) * NB(b) * NB(e);
      }
    }
  std::vector<int64_t> ptrBC, ptrBZ;
  std::vector<int2> LBC, LBZ;
  csr_group(np, kBC, vBC, ptrBC, LBC);
  csr_group(n2, kBZ, vBZ, ptrBZ, LBZ);
  std::vector<int64_t>().swap(kBC); std::vector<int2>().swap(vBC);
  std::vector<int64_t>().swap(kBZ); std::vector<int2>().swap(vBZ);

  // (pair (B,G'), pair (G',E') not on-site) for Z blocks that carry an adjoint
  std::vector<int64_t> kZV, kZC;
  std::vector<int2> vZV, vZC;
  for (int64_t z = 0; z < n2; z++) {
    if (ptrBZ[z + 1] == ptrBZ[z]) continue;
    int b = atomA2[z], e = atomB2[z];
    for (int64_t x = ptrZ[z]; x < ptrZ[z + 1]; x++) {
      int2 en = LZ[x];
      int g = pB[en.x];
      kZV.push_back(en.x); vZV.push_back(make_int2(en.y, (int)z));
      kZC.push_back(en.y); vZC.push_back(make_int2(en.x, (int)z));
      fl += 2.0 * NA(b) * NA(g) * NB(g) * NB(e) * 2 + 2.0 * NA(b) * NB(b) * NB(g) * NB(e) * 2;
    }
  }
  std::vector<int64_t> ptrZV, ptrZC;
  std::vector<int2> LZV, LZC;
  csr_group(np, kZV, vZV, ptrZV, LZV);
  csr_group(np, kZC, vZC, ptrZC, LZC);
  std::vector<int64_t>().swap(kZV); std::vector<int2>().swap(vZV);
  std::vector<int64_t>().swap(kZC); std::vector<int2>().swap(vZC);

  // terms 1 and 2, outputs on the pair list only
  std::vector<int64_t> kU2, kT1, kC12;
  std::vector<int2> vU2, vT1;
  std::vector<BX12Entry> vC12;
  std::vector<uint8_t> hasT1(np, 0);
  for (int64_t s = 0; s < n2; s++) {
    int64_t pae = map2to1[s];
    if (pae < 0) continue;
    int a = atomA2[s], e = atomB2[s];
    for (int64_t x = ptrX12[s]; x < ptrX12[s + 1]; x++) {
      const X12Entry &en = LX12[x];
      int g = pA[en.p3];
      if (en.u2 >= 0) {
        kU2.push_back(en.u2); vU2.push_back(make_int2((int)s, en.p3));
        fl += 2.0 * NA(g) * NB(a) * NB(g) * NB(e) * 2;
      }
      if (en.t1) {
        kT1.push_back(en.t); vT1.push_back(make_int2((int)s, en.p3));
        hasT1[pae] = 1;
        fl += 2.0 * NA(e) * NB(a) * NB(g) * NB(e) * 2 + 2.0 * NA(a) * NA(e) * NB(a) * NB(g) * 3;
      }
      kC12.push_back(en.p3); vC12.push_back({en.t, (int32_t)s, en.u2, en.t1});
    }
  }
  std::vector<int64_t> ptrU2, ptrT1, ptrC12;
  std::vector<int2> LU2, LT1;
  std::vector<BX12Entry> LC12;
  csr_group(np, kU2, vU2, ptrU2, LU2);
  csr_group(n2, kT1, vT1, ptrT1, LT1);
  csr_group(np, kC12, vC12, ptrC12, LC12);
  std::vector<int64_t>().swap(kU2); std::vector<int2>().swap(vU2);
  std::vector<int64_t>().swap(kT1); std::vector<int2>().swap(vT1);
  std::vector<int64_t>().swap(kC12); std::vector<BX12Entry>().swap(vC12);

  // T adjoint -> C(A,B') own block: (pair (B',G'), T block)
  std::vector<int64_t> kTC;
  std::vector<int2> vTC;
  for (int64_t t = 0; t < n2; t++)
    for (int64_t x = ptrT[t]; x < ptrT[t + 1]; x++) {
      kTC.push_back(LT[x].x); vTC.push_back(make_int2(LT[x].y, (int)t));
      int a = atomA2[t], g = atomB2[t], b = pB[LT[x].x];
      fl += 2.0 * NA(a) * NB(a) * NB(b) * NB(g);
    }
  std::vector<int64_t> ptrTC;
  std::vector<int2> LTC;
  csr_group(np, kTC, vTC, ptrTC, LTC);
  std::vector<int64_t>().swap(kTC); std::vector<int2>().swap(vTC);

  // ------------------------------------------------------------ tiled work items
  std::vector<int4> it[9];
  for (int64_t p = 0; p < np; p++) {
    int a = pA[p], x = pB[p];
    if (ptrBC[p + 1] > ptrBC[p]) add_items(it[0], p, NA(x), std::max<int64_t>(1, CAP / (NB(a) * NB(x))));
    if (ptrZV[p + 1] > ptrZV[p]) add_items(it[2], p, NA(a), std::max<int64_t>(1, CAP / NA(x)));
    if (ptrZC[p + 1] > ptrZC[p]) add_items(it[3], p, NA(a), std::max<int64_t>(1, CAP / (NB(a) * NB(x))));
    if (ptrU2[p + 1] > ptrU2[p]) add_items(it[4], p, NA(x), std::max<int64_t>(1, CAP / (NB(a) * NB(x))));
    if (hasT1[p] || ptrU2[p + 1] > ptrU2[p]) add_items(it[6], p, NA(a), std::max<int64_t>(1, CAP / NA(x)));
    if (ptrC12[p + 1] > ptrC12[p]) {
      int64_t rows = NA(a) + (ctx->onsite[p] ? 0 : NA(x));
      int64_t per = NB(a) * NB(x);
      add_items(it[7], p, rows, std::max<int64_t>(1, std::min(CAP / per, SMB / (64 * NB(a)))));
    }
    if (ptrTC[p + 1] > ptrTC[p]) add_items(it[8], p, NA(a), std::max<int64_t>(1, CAP / (NB(a) * NB(x))));
  }
  for (int64_t z = 0; z < n2; z++) {
    int b = atomA2[z], e = atomB2[z];
    if (ptrBZ[z + 1] > ptrBZ[z]) add_items(it[1], z, NA(b), std::max<int64_t>(1, CAP / (NB(b) * NB(e))));
    bool needT = ptrT1[z + 1] > ptrT1[z];
    int64_t pag = map2to1[z];
    if (pag >= 0 && ptrU2[pag + 1] > ptrU2[pag]) needT = true;
    if (needT) add_items(it[5], z, NA(b), std::max<int64_t>(1, CAP / (NB(b) * NB(e))));
  }
  (void)map1to2;
  ctx->bwd_flops = fl;

  TRY(rix_upload(ctx, &ctx->d_ptrBC34, ptrBC)); TRY(rix_upload(ctx, &ctx->d_LBC34, LBC));
  TRY(rix_upload(ctx, &ctx->d_ptrBZ34, ptrBZ)); TRY(rix_upload(ctx, &ctx->d_LBZ34, LBZ));
  TRY(rix_upload(ctx, &ctx->d_ptrBZV, ptrZV)); TRY(rix_upload(ctx, &ctx->d_LBZV, LZV));
  TRY(rix_upload(ctx, &ctx->d_ptrBZC, ptrZC)); TRY(rix_upload(ctx, &ctx->d_LBZC, LZC));
  TRY(rix_upload(ctx, &ctx->d_ptrBU2, ptrU2)); TRY(rix_upload(ctx, &ctx->d_LBU2, LU2));
  TRY(rix_upload(ctx, &ctx->d_ptrBT1, ptrT1)); TRY(rix_upload(ctx, &ctx->d_LBT1, LT1));
  TRY(rix_upload(ctx, &ctx->d_ptrBC12, ptrC12)); TRY(rix_upload(ctx, &ctx->d_LBC12, LC12));
  TRY(rix_upload(ctx, &ctx->d_ptrBTC, ptrTC)); TRY(rix_upload(ctx, &ctx->d_LBTC, LTC));
  for (int k = 0; k < 9; k++) {
    TRY(rix_upload(ctx, &ctx->d_itB[k], it[k]));
    ctx->n_itB[k] = it[k].size();
  }
  int64_t nU = 0;
  for (int64_t p = 0; p < np; p++) nU += NA(pB[p]) * NB(pA[p]) * NB(pB[p]);
  TRY(rix_alloc(ctx, &ctx->d_U2bar, nU));
  TRY(rix_alloc(ctx, &ctx->d_Kbuf, ctx->offK[ctx->nk]));
  ctx->have_bwd = true;
  return RIX_OK;
}

static rix_status build_lists(rix_ctx *ctx) {
  const int nat = ctx->nat;
  const int64_t np = ctx->np;
  auto &pA = ctx->pA, &pB = ctx->pB;
  auto &pn = ctx->pn;
  auto &row1 = ctx->row1;
  auto NB = [&](int a) { return (int64_t)ctx->nb_at[a]; };
  auto NA = [&](int a) { return (int64_t)ctx->na_at[a]; };

  // ---------------------------------------------------------------- 2-hop and 3-hop nodes
  std::vector<std::vector<int64_t>> k2(nat), k3(nat);
  bool ok = true;
#pragma omp parallel for schedule(dynamic, 1) reduction(&& : ok)
  for (int a = 0; a < nat; a++) {
    std::vector<int64_t> v;
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
      int b = pB[p1];
      for (int64_t p2 = row1[b]; p2 < row1[b + 1]; p2++)
        v.push_back(key_add(a, pB[p2], &pn[3 * p1], &pn[3 * p2], &ok));
    }
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    std::vector<int64_t> w;
    for (int64_t k : v) {
      int g = key_b(k);
      int8_t m[3];
      decode_n(k, m);
      for (int64_t p3 = row1[g]; p3 < row1[g + 1]; p3++) w.push_back(key_add(a, pB[p3], m, &pn[3 * p3], &ok));
    }
    std::sort(w.begin(), w.end());
    w.erase(std::unique(w.begin(), w.end()), w.end());
    k2[a].swap(v);
    k3[a].swap(w);
  }
  if (!ok) {
    ctx->last_error = "lattice images beyond +-127 cells";
    return RIX_EINVAL;
  }
  ctx->row2.assign(nat + 1, 0);
  ctx->row3.assign(nat + 1, 0);
  for (int a = 0; a < nat; a++) {
    ctx->row2[a + 1] = ctx->row2[a] + k2[a].size();
    ctx->row3[a + 1] = ctx->row3[a] + k3[a].size();
  }
  ctx->n2 = ctx->row2[nat];
  ctx->nk = ctx->row3[nat];
  ctx->keys2.resize(ctx->n2);
  ctx->keys3.resize(ctx->nk);
  for (int a = 0; a < nat; a++) {
    std::copy(k2[a].begin(), k2[a].end(), ctx->keys2.begin() + ctx->row2[a]);
    std::copy(k3[a].begin(), k3[a].end(), ctx->keys3.begin() + ctx->row3[a]);
    std::vector<int64_t>().swap(k2[a]);
    std::vector<int64_t>().swap(k3[a]);
  }
  const int64_t n2 = ctx->n2, nk = ctx->nk;
  auto &keys1 = ctx->keys1, &keys2 = ctx->keys2, &keys3 = ctx->keys3;
  auto &row2 = ctx->row2, &row3 = ctx->row3;
  auto find1 = [&](int64_t key) { int a = key_a(key); return find_in(keys1, row1[a], row1[a + 1], key); };
  auto find2 = [&](int64_t key) { int a = key_a(key); return find_in(keys2, row2[a], row2[a + 1], key); };
  auto find3 = [&](int64_t key) { int a = key_a(key); return find_in(keys3, row3[a], row3[a + 1], key); };

  // ---------------------------------------------------------------- offsets and maps
  std::vector<int32_t> atomA2(n2), atomB2(n2), map2to1(n2), map2to3(n2);
  ctx->off2.assign(n2 + 1, 0);
  std::vector<int64_t> sz2(n2);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < n2; t++) {
    int a = key_a(keys2[t]), g = key_b(keys2[t]);
    atomA2[t] = a; atomB2[t] = g;
    sz2[t] = NA(a) * NB(a) * NB(g);
    map2to1[t] = (int32_t)find1(keys2[t]);
    map2to3[t] = (int32_t)find3(keys2[t]);
  }
  for (int64_t t = 0; t < n2; t++) ctx->off2[t + 1] = ctx->off2[t] + sz2[t];
  std::vector<int32_t> atomA3(nk), atomB3(nk), partner3(nk);
  ctx->offK.assign(nk + 1, 0);
  std::vector<int64_t> szk(nk);
  bool sym_ok = true;
#pragma omp parallel for schedule(static) reduction(&& : sym_ok)
  for (int64_t x = 0; x < nk; x++) {
    int a = key_a(keys3[x]), e = key_b(keys3[x]);
    atomA3[x] = a; atomB3[x] = e;
    szk[x] = NB(a) * NB(e);
    int64_t q = find3(pair_key(e, a, -key_n(keys3[x], 0), -key_n(keys3[x], 1), -key_n(keys3[x], 2)));
    if (q < 0) sym_ok = false;
    partner3[x] = (int32_t)q;
  }
  if (!sym_ok) {
    ctx->last_error = "K pattern not symmetric (pair list asymmetric)";
    return RIX_EINVAL;
  }
  for (int64_t x = 0; x < nk; x++) ctx->offK[x + 1] = ctx->offK[x] + szk[x];
  // Term 4 (like term 1) is symmetric under (A, E', n) -> (E', A, -n) with
  // transposition: it is computed for one orientation of each K block (twice the 1/2
  // of the grouping), the self block (A, A, 0) being its own partner.
  ctx->rep3.assign(nk, 0);
  for (int64_t x = 0; x < nk; x++) {
    const int a = key_a(keys3[x]), e = key_b(keys3[x]);
    const int n0 = key_n(keys3[x], 0), n1 = key_n(keys3[x], 1), n2 = key_n(keys3[x], 2);
    const bool pos = n0 > 0 || (n0 == 0 && (n1 > 0 || (n1 == 0 && n2 > 0)));
    ctx->rep3[x] = partner3[x] == x ? 2 : (a < e || (a == e && pos)) ? 1 : 0;
  }
  std::vector<int32_t> map1to2(np), map1to3(np);
  std::vector<int64_t> offU(np + 1, 0);
  for (int64_t p = 0; p < np; p++) {
    map1to2[p] = (int32_t)find2(keys1[p]);
    map1to3[p] = (int32_t)find3(keys1[p]);
    offU[p + 1] = offU[p] + NA(pB[p]) * NB(pA[p]) * NB(pB[p]);
  }

  // ---------------------------------------------------------------- T list: T(A,G') <- (C(A,B'), D(B',G'))
  std::vector<int64_t> ptrT(n2 + 1, 0);
  std::vector<int64_t> cntT(nat + 1, 0);
  for (int a = 0; a < nat; a++) {
    int64_t c = 0;
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) c += row1[pB[p1] + 1] - row1[pB[p1]];
    cntT[a + 1] = cntT[a] + c;
  }
  std::vector<int2> LT(cntT[nat]);
  double flT = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : flT)
  for (int a = 0; a < nat; a++) {
    std::vector<int64_t> key;
    std::vector<int2> pay;
    bool lok = true;
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
      int b = pB[p1];
      for (int64_t p2 = row1[b]; p2 < row1[b + 1]; p2++) {
        int64_t t = find2(key_add(a, pB[p2], &pn[3 * p1], &pn[3 * p2], &lok));
        key.push_back(t);
        pay.push_back(make_int2((int)p1, (int)p2));
        flT += 2.0 * NA(a) * NB(a) * NB(b) * NB(pB[p2]);
      }
    }
    std::vector<int64_t> rel(row2[a + 1] - row2[a]);
    group_by(row2[a], row2[a + 1], key, pay, rel.data(), LT.data() + cntT[a]);
    for (int64_t i = 0; i < (int64_t)rel.size(); i++) ptrT[row2[a] + i] = cntT[a] + rel[i];
  }
  ptrT[n2] = cntT[nat];

  // ---------------------------------------------------------------- X12 list (terms 1 and 2)
  std::vector<std::vector<X12Entry>> lx(nat);
  std::vector<std::vector<int64_t>> lxk(nat);
  double flX12 = 0, flU2 = 0, flT2 = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : flX12, flT2)
  for (int a = 0; a < nat; a++) {
    struct Rec { int64_t s; int32_t t, p3, u2, t1; };
    std::vector<Rec> r;
    bool lok = true;
    // term 1: P on A, Q on E'; (A,E') in the pair list
    for (int64_t pae = row1[a]; pae < row1[a + 1]; pae++) {
      int64_t s = map1to2[pae];
      int e = pB[pae];
      for (int64_t pq = row1[e]; pq < row1[e + 1]; pq++) {
        int g = pB[pq];
        int64_t t = find2(key_add(a, g, &pn[3 * pae], &pn[3 * pq], &lok));
        r.push_back({s, (int32_t)t, ctx->partner1[pq], -1, 1});
      }
    }
    // term 2: P on A, Q on G' != E'; (A,G') in the pair list
    for (int64_t pag = row1[a]; pag < row1[a + 1]; pag++) {
      int64_t t = map1to2[pag];
      int g = pB[pag];
      for (int64_t p3 = row1[g]; p3 < row1[g + 1]; p3++) {
        if (ctx->onsite[p3]) continue;
        int64_t s = find2(key_add(a, pB[p3], &pn[3 * pag], &pn[3 * p3], &lok));
        r.push_back({s, (int32_t)t, (int32_t)p3, (int32_t)pag, 0});
      }
    }
    std::sort(r.begin(), r.end(), [](const Rec &x, const Rec &y) {
      if (x.s != y.s) return x.s < y.s;
      if (x.t != y.t) return x.t < y.t;
      return x.p3 < y.p3;
    });
    std::vector<X12Entry> out;
    std::vector<int64_t> outk;
    for (size_t i = 0; i < r.size();) {
      size_t j = i;
      X12Entry en{r[i].t, r[i].p3, -1, 0};
      while (j < r.size() && r[j].s == r[i].s && r[j].t == r[i].t && r[j].p3 == r[i].p3) {
        if (r[j].u2 >= 0) en.u2 = r[j].u2;
        en.t1 |= r[j].t1;
        j++;
      }
      int e = pB[en.p3], g = pA[en.p3];
      // term 1 runs in one orientation of each pair (the list keeps both for the adjoint)
      if (en.t1 && ctx->rep1[map2to1[r[i].s]])
        flX12 += 2.0 * NA(e) * NA(a) * NB(a) * NB(g) + 2.0 * NA(e) * NB(a) * NB(g) * NB(e);
      if (en.u2 >= 0) {
        flX12 += 2.0 * NA(g) * NB(a) * NB(g) * NB(e);
        flT2 += 2.0 * NA(g) * NB(a) * NB(g) * NB(e);
      }
      out.push_back(en);
      outk.push_back(r[i].s);
      i = j;
    }
    lx[a].swap(out);
    lxk[a].swap(outk);
  }
  std::vector<int64_t> ptrX12(n2 + 1, 0);
  std::vector<int64_t> baseX(nat + 1, 0);
  for (int a = 0; a < nat; a++) baseX[a + 1] = baseX[a] + lx[a].size();
  std::vector<X12Entry> LX12(baseX[nat]);
  for (int a = 0; a < nat; a++) {
    std::copy(lx[a].begin(), lx[a].end(), LX12.begin() + baseX[a]);
    int64_t e = 0;
    for (int64_t s = row2[a]; s < row2[a + 1]; s++) {
      ptrX12[s] = baseX[a] + e;
      while (e < (int64_t)lxk[a].size() && lxk[a][e] == s) e++;
    }
    std::vector<X12Entry>().swap(lx[a]);
    std::vector<int64_t>().swap(lxk[a]);
  }
  ptrX12[n2] = baseX[nat];
  for (int64_t p = 0; p < np; p++) flU2 += 2.0 * NA(pA[p]) * NA(pB[p]) * NB(pA[p]) * NB(pB[p]);

  // ---------------------------------------------------------------- Z list (term 4): Z(B,E') <- (pair (B,G'), pair (G',E'))
  // and the X34 list: X(A,E') <- (C(A,B') not on-site, Z(B,E'-n1)).  Z blocks that no
  // product reaches (possible only without neighbours) are left out of the X34 list.
  std::vector<std::vector<int2>> lz(nat), lxx(nat);
  std::vector<std::vector<int64_t>> lzp(nat), lxp(nat);
  double flZ = 0, flX34 = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : flZ)
  for (int b = 0; b < nat; b++) {
    std::vector<int64_t> key;
    std::vector<int2> pay;
    bool lok = true;
    for (int64_t p2 = row1[b]; p2 < row1[b + 1]; p2++) {
      int g = pB[p2];
      for (int64_t p3 = row1[g]; p3 < row1[g + 1]; p3++) {
        if (ctx->onsite[p3]) continue;
        int e = pB[p3];
        key.push_back(find2(key_add(b, e, &pn[3 * p2], &pn[3 * p3], &lok)));
        pay.push_back(make_int2((int)p2, (int)p3));
        flZ += 2.0 * NA(b) * NA(g) * NB(g) * NB(e) + 2.0 * NA(b) * NB(b) * NB(g) * NB(e);
      }
    }
    std::vector<int64_t> rel(row2[b + 1] - row2[b] + 1);
    lz[b].resize(key.size());
    group_by(row2[b], row2[b + 1], key, pay, rel.data(), lz[b].data());
    rel[row2[b + 1] - row2[b]] = key.size();
    lzp[b].swap(rel);
  }
  std::vector<int64_t> ptrZ(n2 + 1, 0);
  std::vector<int2> LZ;
  {
    int64_t tot = 0;
    for (int b = 0; b < nat; b++) tot += lz[b].size();
    LZ.resize(tot);
    int64_t base = 0;
    for (int b = 0; b < nat; b++) {
      for (int64_t z = row2[b]; z < row2[b + 1]; z++) ptrZ[z] = base + lzp[b][z - row2[b]];
      std::copy(lz[b].begin(), lz[b].end(), LZ.begin() + base);
      base += lz[b].size();
      std::vector<int2>().swap(lz[b]);
      std::vector<int64_t>().swap(lzp[b]);
    }
    ptrZ[n2] = base;
  }
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : flX34)
  for (int a = 0; a < nat; a++) {
    std::vector<int64_t> key;
    std::vector<int2> pay;
    bool lok = true;
    for (int64_t p1 = row1[a]; p1 < row1[a + 1]; p1++) {
      if (ctx->onsite[p1]) continue;
      int b = pB[p1];
      for (int64_t z = row2[b]; z < row2[b + 1]; z++) {
        if (ptrZ[z + 1] == ptrZ[z]) continue;
        int e = key_b(keys2[z]);
        int8_t m[3];
        decode_n(keys2[z], m);
        const int64_t x3 = find3(key_add(a, e, &pn[3 * p1], m, &lok));
        key.push_back(x3);
        pay.push_back(make_int2((int)p1, (int)z));
        if (x3 >= 0 && ctx->rep3[x3]) flX34 += 2.0 * NA(b) * NB(b) * NB(a) * NB(e);  // one orientation
      }
    }
    std::vector<int64_t> rel(row3[a + 1] - row3[a] + 1);
    lxx[a].resize(key.size());
    group_by(row3[a], row3[a + 1], key, pay, rel.data(), lxx[a].data());
    rel[row3[a + 1] - row3[a]] = key.size();
    lxp[a].swap(rel);
  }
  std::vector<int64_t> ptrX34(nk + 1, 0);
  std::vector<int2> LX34;
  {
    int64_t tot = 0;
    for (int a = 0; a < nat; a++) tot += lxx[a].size();
    LX34.resize(tot);
    int64_t base = 0;
    for (int a = 0; a < nat; a++) {
      for (int64_t x = row3[a]; x < row3[a + 1]; x++) ptrX34[x] = base + lxp[a][x - row3[a]];
      std::copy(lxx[a].begin(), lxx[a].end(), LX34.begin() + base);
      base += lxx[a].size();
      std::vector<int2>().swap(lxx[a]);
      std::vector<int64_t>().swap(lxp[a]);
    }
    ptrX34[nk] = base;
  }

  // ---------------------------------------------------------------- backward plan
  if (ctx->opt.backward) {
    rix_status sb = build_backward_lists(ctx, LT, ptrT, LX12, ptrX12, LZ, ptrZ, map1to2, map2to1, atomA2,
                                         atomB2);
    if (sb != RIX_OK) return sb;
  }

  // ---------------------------------------------------------------- work items and launch orders
  const int64_t CAP = 8192;  // output elements per work item (256 threads x 32)
  std::vector<int2> itT, itZ, itU;
  std::vector<double> cT, cZ;
  for (int64_t t = 0; t < n2; t++) {
    int a = atomA2[t], g = atomB2[t];
    int64_t per = NB(a) * NB(g);
    int64_t pt = std::max<int64_t>(1, CAP / per);
    double len = (double)(ptrT[t + 1] - ptrT[t]);
    for (int64_t p0 = 0; p0 < NA(a); p0 += pt) {
      itT.push_back(make_int2((int)t, (int)p0));
      cT.push_back(len * std::min(pt, NA(a) - p0) * per);
    }
  }
  for (int64_t z = 0; z < n2; z++) {
    int b = atomA2[z], e = atomB2[z];
    int64_t per = NB(b) * NB(e);
    int64_t pt = std::max<int64_t>(1, CAP / per);
    double len = (double)(ptrZ[z + 1] - ptrZ[z]);
    if (len == 0) continue;
    for (int64_t p0 = 0; p0 < NA(b); p0 += pt) {
      itZ.push_back(make_int2((int)z, (int)p0));
      cZ.push_back(len * std::min(pt, NA(b) - p0) * per);
    }
  }
  for (int64_t p = 0; p < np; p++) {
    int a = pA[p], g = pB[p];
    int64_t per = NB(a) * NB(g);
    int64_t qt = std::max<int64_t>(1, CAP / per);
    for (int64_t q0 = 0; q0 < NA(g); q0 += qt) itU.push_back(make_int2((int)p, (int)q0));
  }
  // launch order: most expensive first (longest processing time first)
  auto order_by = [](std::vector<int2> &it, const std::vector<double> &cost) {
    std::vector<int64_t> idx(it.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return cost[x] > cost[y]; });
    std::vector<int2> o(it.size());
    for (size_t i = 0; i < idx.size(); i++) o[i] = it[idx[i]];
    it.swap(o);
  };
  order_by(itT, cT);
  order_by(itZ, cZ);
  std::vector<int32_t> ordX12, ordX34;
  std::vector<double> cX12;
  for (int64_t s = 0; s < n2; s++)
    if (ptrX12[s + 1] > ptrX12[s]) {
      ordX12.push_back((int32_t)s);
      cX12.push_back((double)(ptrX12[s + 1] - ptrX12[s]) * NA(atomA2[s]) * NB(atomA2[s]));
    }
  {
    std::vector<int64_t> idx(ordX12.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return cX12[x] > cX12[y]; });
    std::vector<int32_t> o(idx.size());
    for (size_t i = 0; i < idx.size(); i++) o[i] = ordX12[idx[i]];
    ordX12.swap(o);
  }
  {
    std::vector<double> c;
    for (int64_t x = 0; x < nk; x++)
      if (ptrX34[x + 1] > ptrX34[x]) {
        ordX34.push_back((int32_t)x);
        c.push_back((double)(ptrX34[x + 1] - ptrX34[x]) * NB(atomA3[x]) * NB(atomB3[x]));
      }
    std::vector<int64_t> idx(ordX34.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return c[x] > c[y]; });
    std::vector<int32_t> o(idx.size());
    for (size_t i = 0; i < idx.size(); i++) o[i] = ordX34[idx[i]];
    ordX34.swap(o);
  }
  // fold groups: consecutive K blocks of one atom pair
  std::vector<int64_t> fold;
  for (int64_t x = 0; x < nk; x++)
    if (x == 0 || (keys3[x] >> 24) != (keys3[x - 1] >> 24)) fold.push_back(x);
  fold.push_back(nk);
  std::vector<int64_t> bofs(nat + 1, 0);
  for (int a = 0; a < nat; a++) bofs[a + 1] = bofs[a] + NB(a);
  ctx->nbasis = bofs[nat];

  // ---------------------------------------------------------------- stats
  rix_stats_t &st = ctx->stats;
  st.n_atoms = nat; st.n_pairs = np; st.n_pairs2 = n2; st.n_kblocks = nk;
  st.c_elems = ctx->offC[np]; st.v_elems = ctx->offV[np]; st.d_elems = ctx->offD[np];
  st.k_elems = ctx->offK[nk];
  st.flops_stage[0] = flT; st.flops_stage[1] = flU2; st.flops_stage[2] = flX12;
  st.flops_stage[3] = flZ; st.flops_stage[4] = flX34; st.flops_stage[5] = (double)ctx->offK[nk];
  st.flops_fp64 = flT + flU2 + flX12 + flZ + flX34 + st.flops_stage[5];
  st.flops_term2 = flT2;
  st.min_bytes = 8.0 * (st.c_elems + st.v_elems + st.d_elems) + 8.0 * st.k_elems;
  if (ctx->opt.verbose)
    fprintf(stderr, "rix: %lld pairs, %lld 2-hop, %lld K blocks; lists T %zu X12 %zu Z %zu X34 %zu; %.3g FLOP\n",
            (long long)np, (long long)n2, (long long)nk, LT.size(), LX12.size(), LZ.size(), LX34.size(),
            st.flops_fp64);

  // ---------------------------------------------------------------- upload
  TRY(rix_upload(ctx, &ctx->d_map1to2, map1to2));
  TRY(rix_upload(ctx, &ctx->d_map1to3, map1to3));
  TRY(rix_upload(ctx, &ctx->d_offU, offU));
  ctx->offU_h = offU;
  TRY(rix_upload(ctx, &ctx->d_atomA2, atomA2));
  TRY(rix_upload(ctx, &ctx->d_atomB2, atomB2));
  TRY(rix_upload(ctx, &ctx->d_off2, ctx->off2));
  TRY(rix_upload(ctx, &ctx->d_map2to1, map2to1));
  TRY(rix_upload(ctx, &ctx->d_map2to3, map2to3));
  TRY(rix_upload(ctx, &ctx->d_atomA3, atomA3));
  TRY(rix_upload(ctx, &ctx->d_rep3, ctx->rep3));
  TRY(rix_upload(ctx, &ctx->d_atomB3, atomB3));
  TRY(rix_upload(ctx, &ctx->d_offK, ctx->offK));
  TRY(rix_upload(ctx, &ctx->d_partner3, partner3));
  TRY(rix_upload(ctx, &ctx->d_ptrT, ptrT));
  TRY(rix_upload(ctx, &ctx->d_LT, LT));
  TRY(rix_upload(ctx, &ctx->d_ptrX12, ptrX12));
  TRY(rix_upload(ctx, &ctx->d_LX12, LX12));
  TRY(rix_upload(ctx, &ctx->d_ptrZ, ptrZ));
  TRY(rix_upload(ctx, &ctx->d_LZ, LZ));
  TRY(rix_upload(ctx, &ctx->d_ptrX34, ptrX34));
  TRY(rix_upload(ctx, &ctx->d_LX34, LX34));
  TRY(rix_upload(ctx, &ctx->d_fold, fold)); ctx->n_fold = (int64_t)fold.size() - 1;
  TRY(rix_upload(ctx, &ctx->d_bofs, bofs));
  {
    // image vector of every K block (the Bloch phases of rix_bloch)
    std::vector<char4> n3(nk);
    for (int64_t x = 0; x < nk; x++)
      n3[x] = make_char4((signed char)key_n(keys3[x], 0), (signed char)key_n(keys3[x], 1),
                         (signed char)key_n(keys3[x], 2), 0);
    TRY(rix_upload(ctx, &ctx->d_n3, n3));
  }
  TRY(rix_alloc(ctx, &ctx->d_U, offU[np]));
  TRY(rix_alloc(ctx, &ctx->d_X, ctx->offK[nk]));
  ctx->n_epart = (np + 255) / 256;
  TRY(rix_alloc(ctx, &ctx->d_epart, ctx->n_epart + 1));
  TRY(rix_alloc(ctx, &ctx->d_flag, 4));

  // ---------------------------------------------------------------- memory plan (row blocks)
  // T and Z need off2[n2] doubles each.  If both do not fit in what is left, the
  // rows are processed in blocks of consecutive atoms (the paper's Fock-matrix
  // blocks): T, U2 and terms 1+2 per block of row atoms A, Z and terms 3+4 per
  // block of middle atoms B, with T and Z buffers sized for the largest block.
  std::vector<int64_t> asz(nat);
  for (int a = 0; a < nat; a++) asz[a] = ctx->off2[row2[a + 1]] - ctx->off2[row2[a]];
  int64_t avail0;
  {
    size_t fr = 0, to = 0;
    cudaMemGetInfo(&fr, &to);
    avail0 = (int64_t)fr - ((int64_t)4 << 30);
    if (ctx->opt.max_workspace_bytes > 0)
      avail0 = std::min<int64_t>(avail0, ctx->opt.max_workspace_bytes - (int64_t)ctx->dev_bytes);
    // still to come besides T and Z: the work-item arrays and a little slack
    const int64_t items = (int64_t)(itT.size() + itZ.size() + itU.size()) * (int64_t)sizeof(int2) +
                          (int64_t)(ordX12.size() + ordX34.size()) * (int64_t)sizeof(int32_t);
    avail0 -= items + ((int64_t)64 << 10);
  }
  // blocks for a T/Z budget; in mixed precision the plans' size depends on the
  // blocks (their problems split by block), so the split is redone until the
  // plans fit beside the buffers
  const bool mixed = ctx->opt.precision == RIX_MIXED_BF16;
  ctx->nblk = 1;
  ctx->blk_atom.clear();
  int64_t mx_est = mixed ? rix_mixed_bytes(ctx, ptrZ) : 0;
  for (int iter = 0;; iter++) {
    const int64_t per_buf = std::max<int64_t>(0, (avail0 - mx_est) / 2 / (int64_t)sizeof(double));
    ctx->blk_atom.assign(1, 0);
    int64_t cur = 0;
    for (int a = 0; a < nat; a++) {
      if (asz[a] > per_buf) {
        ctx->last_error = "workspace too small for the intermediates of one atom";
        return RIX_ENOMEM;
      }
      const bool full = ctx->opt.block_atoms > 0 && a - ctx->blk_atom.back() >= ctx->opt.block_atoms;
      if (cur + asz[a] > per_buf || full) {
        ctx->blk_atom.push_back(a);
        cur = 0;
      }
      cur += asz[a];
    }
    ctx->blk_atom.push_back(nat);
    ctx->nblk = (int)ctx->blk_atom.size() - 1;
    if (!mixed || iter == 4) break;
    const int64_t need = rix_mixed_bytes(ctx, ptrZ);
    if (need <= mx_est) break;
    mx_est = need;
  }
  const int nblk = ctx->nblk;
  std::vector<int> blk_of(nat);
  int64_t maxbuf = 0;
  ctx->blk_base.assign(nblk, 0);
  for (int b = 0; b < nblk; b++) {
    for (int a = ctx->blk_atom[b]; a < ctx->blk_atom[b + 1]; a++) blk_of[a] = b;
    ctx->blk_base[b] = ctx->off2[row2[ctx->blk_atom[b]]];
    maxbuf = std::max(maxbuf, ctx->off2[row2[ctx->blk_atom[b + 1]]] - ctx->blk_base[b]);
  }
  // items of one block are contiguous, in cost order within the block
  auto seg_sort = [&](std::vector<int2> &it, auto blk_of_item, std::vector<int64_t> &seg) {
    std::stable_sort(it.begin(), it.end(), [&](const int2 &x, const int2 &y) { return blk_of_item(x) < blk_of_item(y); });
    seg.assign(nblk + 1, 0);
    for (auto &v : it) seg[blk_of_item(v) + 1]++;
    for (int b = 0; b < nblk; b++) seg[b + 1] += seg[b];
  };
  seg_sort(itT, [&](const int2 &v) { return blk_of[atomA2[v.x]]; }, ctx->segT);
  seg_sort(itZ, [&](const int2 &v) { return blk_of[atomA2[v.x]]; }, ctx->segZ);
  seg_sort(itU, [&](const int2 &v) { return blk_of[pA[v.x]]; }, ctx->segU);
  {
    std::stable_sort(ordX12.begin(), ordX12.end(),
                     [&](int32_t x, int32_t y) { return blk_of[atomA2[x]] < blk_of[atomA2[y]]; });
    ctx->segX12.assign(nblk + 1, 0);
    for (auto v : ordX12) ctx->segX12[blk_of[atomA2[v]] + 1]++;
    for (int b = 0; b < nblk; b++) ctx->segX12[b + 1] += ctx->segX12[b];
  }
  ctx->nblk = nblk;
  TRY(rix_upload(ctx, &ctx->d_itT, itT)); ctx->n_itT = itT.size();
  TRY(rix_upload(ctx, &ctx->d_itZ, itZ)); ctx->n_itZ = itZ.size();
  TRY(rix_upload(ctx, &ctx->d_itU, itU)); ctx->n_itU = itU.size();
  TRY(rix_upload(ctx, &ctx->d_ordX12, ordX12)); ctx->n_ordX12 = ordX12.size();
  TRY(rix_upload(ctx, &ctx->d_ordX34, ordX34)); ctx->n_ordX34 = ordX34.size();
  TRY(rix_alloc(ctx, &ctx->d_T, maxbuf));
  TRY(rix_alloc(ctx, &ctx->d_Z, maxbuf));
  ctx->stats.tz_bytes = 2 * maxbuf * (int64_t)sizeof(double);
  if (ctx->opt.precision == RIX_MIXED_BF16) TRY(rix_mixed_plan(ctx, ptrZ));
  if (ctx->opt.verbose) fprintf(stderr, "rix: %d row block(s), T/Z buffers %.3g GB each\n", nblk, maxbuf * 8e-9);
  return RIX_OK;
}

// --------------------------------------------------------------------------
extern "C" rix_status rix_setup(const rix_system *sys, const rix_options *opt, rix_ctx **out) {
  if (!out) return RIX_EINVAL;
  *out = nullptr;
  if (!sys || !sys->xyz_bohr || !sys->species || !sys->nbas_per_species || !sys->naux_per_species)
    return RIX_EINVAL;
  if (sys->n_atoms <= 0 || sys->n_atoms >= (1 << 20) || sys->n_species <= 0) return RIX_EINVAL;
  if (sys->cell_bohr && !(sys->cutoff_bohr > 0)) return RIX_EINVAL;
  for (int s = 0; s < sys->n_species; s++) {
    if (sys->nbas_per_species[s] < 1 || sys->nbas_per_species[s] > 64) return RIX_EINVAL;
    if (sys->naux_per_species[s] < 1 || sys->naux_per_species[s] > 256) return RIX_EINVAL;
  }
  for (int i = 0; i < sys->n_atoms; i++)
    if (sys->species[i] < 0 || sys->species[i] >= sys->n_species) return RIX_EINVAL;
  for (int i = 0; i < 3 * sys->n_atoms; i++)
    if (!std::isfinite(sys->xyz_bohr[i])) return RIX_EINVAL;
  if (opt && opt->precision != RIX_FP64 && opt->precision != RIX_MIXED_BF16) return RIX_EINVAL;
  if (opt && (opt->n_slices < 0 || opt->n_slices > 8 || opt->n_slices_regrouped < 0 || opt->n_slices_regrouped > 8))
    return RIX_EINVAL;
  if (opt && !(opt->product_tau >= 0.0)) return RIX_EINVAL;

  rix_ctx *ctx = new rix_ctx();
  if (opt) ctx->opt = *opt;
  ctx->nat = sys->n_atoms;
  ctx->nsp = sys->n_species;
  ctx->xyz.assign(sys->xyz_bohr, sys->xyz_bohr + 3 * sys->n_atoms);
  ctx->sp.assign(sys->species, sys->species + sys->n_atoms);
  ctx->nbs.assign(sys->nbas_per_species, sys->nbas_per_species + sys->n_species);
  ctx->nas.assign(sys->naux_per_species, sys->naux_per_species + sys->n_species);
  ctx->periodic = sys->cell_bohr != nullptr;
  if (ctx->periodic) memcpy(ctx->cell, sys->cell_bohr, sizeof(double) * 9);
  ctx->rc = sys->cutoff_bohr;
  ctx->tau = sys->screen_tau;
  ctx->nb_at.resize(ctx->nat);
  ctx->na_at.resize(ctx->nat);
  for (int i = 0; i < ctx->nat; i++) {
    ctx->nb_at[i] = ctx->nbs[ctx->sp[i]];
    ctx->na_at[i] = ctx->nas[ctx->sp[i]];
  }
  auto fail = [&](rix_status s) {
    if (ctx->opt.verbose) fprintf(stderr, "rix_setup: %s\n", ctx->last_error.c_str());
    rix_destroy(ctx);
    return s;
  };

  rix_status s;
  const bool user_pairs = sys->pairs != nullptr || sys->n_pairs != 0;
  if (user_pairs) {
    // ---------------------------------------------- the caller's pair list (host, validated here)
    if (!sys->pairs || sys->n_pairs <= 0 || sys->n_pairs >= INT32_MAX) {
      ctx->last_error = "pairs: need n_pairs > 0 entries";
      return fail(RIX_EINVAL);
    }
    std::vector<int64_t> keys((size_t)sys->n_pairs);
    for (int64_t p = 0; p < sys->n_pairs; p++) {
      const int32_t *e = sys->pairs + 5 * p;
      bool ok = e[0] >= 0 && e[0] < ctx->nat && e[1] >= 0 && e[1] < ctx->nat;
      for (int c = 0; c < 3; c++) ok = ok && e[2 + c] >= -42 && e[2 + c] <= 42 && (ctx->periodic || e[2 + c] == 0);
      if (!ok) {
        ctx->last_error = "pairs: atom out of range, or an image beyond +-42 (three hops must stay within +-127), "
                          "or an image in a cluster";
        return fail(RIX_EINVAL);
      }
      keys[p] = pair_key(e[0], e[1], e[2], e[3], e[4]);
    }
    std::sort(keys.begin(), keys.end());
    if (std::adjacent_find(keys.begin(), keys.end()) != keys.end()) {
      ctx->last_error = "pairs: duplicate entry";
      return fail(RIX_EINVAL);
    }
    ctx->keys1.swap(keys);
    ctx->np = (int64_t)ctx->keys1.size();
    ctx->row1.assign(ctx->nat + 1, 0);
    for (int64_t p = 0; p < ctx->np; p++) ctx->row1[key_a(ctx->keys1[p]) + 1]++;
    for (int a = 0; a < ctx->nat; a++) ctx->row1[a + 1] += ctx->row1[a];
  } else {
  // ------------------------------------------------ pair list on the device
  int nr[3];
  image_range(ctx, nr);
  for (int d = 0; d < 3; d++)
    if (3 * nr[d] > 127) {
      ctx->last_error = "cutoff too large for the cell (images beyond +-127)";
      return fail(RIX_EINVAL);
    }
  double *d_xyz = nullptr, *d_cell = nullptr;
  int64_t *d_counts = nullptr, *d_rowptr = nullptr, *d_keys = nullptr;
  if ((s = rix_alloc(ctx, &d_xyz, 3 * (size_t)ctx->nat)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &d_cell, 9)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &d_counts, ctx->nat + 1)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &d_rowptr, ctx->nat + 1)) != RIX_OK) return fail(s);
  if (cudaMemcpy(d_xyz, ctx->xyz.data(), sizeof(double) * 3 * ctx->nat, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_cell, ctx->cell, sizeof(double) * 9, cudaMemcpyHostToDevice) != cudaSuccess) {
    ctx->last_error = "upload geometry";
    return fail(RIX_ECUDA);
  }
  if ((s = rix_launch_pairs(ctx, d_xyz, d_cell, nr, d_counts, nullptr, nullptr, 0)) != RIX_OK) return fail(s);
  std::vector<int64_t> counts(ctx->nat);
  if (cudaMemcpy(counts.data(), d_counts, sizeof(int64_t) * ctx->nat, cudaMemcpyDeviceToHost) != cudaSuccess) {
    ctx->last_error = std::string("pair count: ") + cudaGetErrorString(cudaGetLastError());
    return fail(RIX_ECUDA);
  }
  ctx->row1.assign(ctx->nat + 1, 0);
  for (int a = 0; a < ctx->nat; a++) ctx->row1[a + 1] = ctx->row1[a] + counts[a];
  ctx->np = ctx->row1[ctx->nat];
  if (ctx->np >= INT32_MAX) { ctx->last_error = "too many pairs"; return fail(RIX_EUNSUPPORTED); }
  if ((s = rix_alloc(ctx, &d_keys, ctx->np)) != RIX_OK) return fail(s);
  cudaMemcpy(d_rowptr, ctx->row1.data(), sizeof(int64_t) * (ctx->nat + 1), cudaMemcpyHostToDevice);
  if ((s = rix_launch_pairs(ctx, d_xyz, d_cell, nr, nullptr, d_rowptr, d_keys, 0)) != RIX_OK) return fail(s);
  ctx->keys1.resize(ctx->np);
  if (cudaMemcpy(ctx->keys1.data(), d_keys, sizeof(int64_t) * ctx->np, cudaMemcpyDeviceToHost) != cudaSuccess) {
    ctx->last_error = std::string("pair fill: ") + cudaGetErrorString(cudaGetLastError());
    return fail(RIX_ECUDA);
  }
  }
  // decode
  const int64_t np = ctx->np;
  ctx->pA.resize(np); ctx->pB.resize(np); ctx->pn.resize(3 * np); ctx->onsite.resize(np);
  ctx->partner1.resize(np);
  ctx->offC.assign(np + 1, 0); ctx->offV.assign(np + 1, 0); ctx->offD.assign(np + 1, 0);
  for (int64_t p = 0; p < np; p++) {
    int64_t k = ctx->keys1[p];
    int a = key_a(k), b = key_b(k);
    ctx->pA[p] = a; ctx->pB[p] = b;
    for (int c = 0; c < 3; c++) ctx->pn[3 * p + c] = (int8_t)key_n(k, c);
    ctx->onsite[p] = (a == b && key_n(k, 0) == 0 && key_n(k, 1) == 0 && key_n(k, 2) == 0);
    int64_t rows = ctx->na_at[a] + (ctx->onsite[p] ? 0 : ctx->na_at[b]);
    ctx->offC[p + 1] = ctx->offC[p] + rows * ctx->nb_at[a] * ctx->nb_at[b];
    ctx->offV[p + 1] = ctx->offV[p] + (int64_t)ctx->na_at[a] * ctx->na_at[b];
    ctx->offD[p + 1] = ctx->offD[p] + (int64_t)ctx->nb_at[a] * ctx->nb_at[b];
  }
  for (int64_t p = 0; p < np; p++) {
    int64_t k = pair_key(ctx->pB[p], ctx->pA[p], -ctx->pn[3 * p], -ctx->pn[3 * p + 1], -ctx->pn[3 * p + 2]);
    int b = ctx->pB[p];
    int64_t q = find_in(ctx->keys1, ctx->row1[b], ctx->row1[b + 1], k);
    if (q < 0) { ctx->last_error = "pair list not symmetric"; return fail(RIX_EINVAL); }
    ctx->partner1[p] = (int32_t)q;
  }
  if ((s = rix_upload(ctx, &ctx->d_nb, ctx->nb_at)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_na, ctx->na_at)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_pA, ctx->pA)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_pB, ctx->pB)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_partner1, ctx->partner1)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_onsite, ctx->onsite)) != RIX_OK) return fail(s);
  // Term 1 is symmetric under (A, E', n) -> (E', A, -n) with transposition (C, V and D
  // are pair-symmetric), and K = X + X^T adds the transpose of every block of X; so
  // term 1 is computed for one orientation of each pair only, with weight 1 instead
  // of the 1/2 of the four-term grouping (weight 1/2 on the on-site pair, its own
  // partner).  Representative: A < E', or A == E' with n lexicographically positive.
  ctx->rep1.assign(np, 0);
  for (int64_t p = 0; p < np; p++) {
    const int a = ctx->pA[p], b = ctx->pB[p];
    const int n0 = ctx->pn[3 * p], n1 = ctx->pn[3 * p + 1], n2 = ctx->pn[3 * p + 2];
    const bool pos = n0 > 0 || (n0 == 0 && (n1 > 0 || (n1 == 0 && n2 > 0)));
    ctx->rep1[p] = ctx->onsite[p] ? 2 : (a < b || (a == b && pos)) ? 1 : 0;
  }
  if ((s = rix_upload(ctx, &ctx->d_rep1, ctx->rep1)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_offC, ctx->offC)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_offV, ctx->offV)) != RIX_OK) return fail(s);
  if ((s = rix_upload(ctx, &ctx->d_offD, ctx->offD)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_C, ctx->offC[np])) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_V, ctx->offV[np])) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_keepC, np)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_keepV, np)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_keepD, np)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_normC, np)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_normV, np)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_normD, np)) != RIX_OK) return fail(s);
  if ((s = rix_alloc(ctx, &ctx->d_maxCatom, ctx->nat)) != RIX_OK) return fail(s);
  {
    // pair vectors (the geometry the force and stress chain differentiates through)
    std::vector<double> rv(3 * (size_t)np);
    for (int64_t p = 0; p < np; p++)
      for (int c = 0; c < 3; c++) {
        double sh = 0.0;
        if (ctx->periodic)
          for (int d = 0; d < 3; d++) sh += (double)ctx->pn[3 * p + d] * ctx->cell[3 * d + c];
        rv[3 * p + c] = (ctx->xyz[3 * ctx->pB[p] + c] + sh) - ctx->xyz[3 * ctx->pA[p] + c];
      }
    if ((s = rix_upload(ctx, &ctx->d_rvec, rv)) != RIX_OK) return fail(s);
    if ((s = rix_upload(ctx, &ctx->d_row1, ctx->row1)) != RIX_OK) return fail(s);
    if ((s = rix_alloc(ctx, &ctx->d_gpair, np)) != RIX_OK) return fail(s);
    if (ctx->periodic) {
      const double *a = ctx->cell;
      ctx->volume = std::fabs(a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                              a[2] * (a[3] * a[7] - a[4] * a[6]));
    }
  }
  if (cudaHostAlloc((void **)&ctx->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&ctx->d_err, ctx->h_err, 0) != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = "mapped status word";
    return fail(RIX_ECUDA);
  }
  *(volatile int *)ctx->h_err = 0;
  if ((s = rix_noalloc_attach(ctx)) != RIX_OK) return fail(s);
  if ((s = build_lists(ctx)) != RIX_OK) return fail(s);
  ctx->stats.workspace_bytes = (int64_t)ctx->dev_bytes;
  *out = ctx;
  return RIX_OK;
}

extern "C" rix_status rix_layout(const rix_ctx *ctx, int32_t which, int64_t *n_blocks,
                                 const int64_t **keys, const int64_t **offsets) {
  if (!ctx || !n_blocks || !keys || !offsets) return RIX_EINVAL;
  switch (which) {
    case RIX_LIST_C: *n_blocks = ctx->np; *keys = ctx->keys1.data(); *offsets = ctx->offC.data(); break;
    case RIX_LIST_V: *n_blocks = ctx->np; *keys = ctx->keys1.data(); *offsets = ctx->offV.data(); break;
    case RIX_LIST_D: *n_blocks = ctx->np; *keys = ctx->keys1.data(); *offsets = ctx->offD.data(); break;
    case RIX_LIST_K: *n_blocks = ctx->nk; *keys = ctx->keys3.data(); *offsets = ctx->offK.data(); break;
    default: return RIX_EINVAL;
  }
  return RIX_OK;
}

extern "C" rix_status rix_layout_sizes(const rix_ctx *ctx, int64_t *c, int64_t *v, int64_t *d, int64_t *k) {
  if (!ctx) return RIX_EINVAL;
  if (c) *c = ctx->offC[ctx->np];
  if (v) *v = ctx->offV[ctx->np];
  if (d) *d = ctx->offD[ctx->np];
  if (k) *k = ctx->offK[ctx->nk];
  return RIX_OK;
}

extern "C" rix_status rix_set_CV(rix_ctx *ctx, const double *C, const double *V, void *stream) {
  if (!ctx || !C || !V) return RIX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // host or device sources: the direction follows from the (unified) address
  RIX_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_C, C, sizeof(double) * ctx->offC[ctx->np], cudaMemcpyDefault, st));
  RIX_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_V, V, sizeof(double) * ctx->offV[ctx->np], cudaMemcpyDefault, st));
  rix_status s = rix_launch_symcheck(ctx, st);
  if (s != RIX_OK) return s;
  int32_t bad = 0;
  RIX_CUDA_TRY(ctx, cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RIX_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if ((s = rix_take_err(ctx)) != RIX_OK) return s;
  if (bad) {
    ctx->have_cv = false;
    ctx->last_error = "C or V blocks differ from their transposed partners";
    return RIX_ENOTSYM;
  }
  ctx->fwd_valid = false;
  if ((s = rix_launch_flags(ctx, ctx->d_C, ctx->d_offC, ctx->np, ctx->d_keepC, st, ctx->d_normC)) != RIX_OK) return s;
  if ((s = rix_launch_flags(ctx, ctx->d_V, ctx->d_offV, ctx->np, ctx->d_keepV, st, ctx->d_normV)) != RIX_OK) return s;
  if (ctx->opt.product_tau > 0 && (s = rix_launch_atom_max(ctx, ctx->d_normC, ctx->d_maxCatom, st)) != RIX_OK)
    return s;
  ctx->have_cv = true;
  return RIX_OK;
}

rix_status rix_take_err(rix_ctx *ctx) {
  if (ctx->h_err && *(volatile int *)ctx->h_err) {
    *(volatile int *)ctx->h_err = 0;
    ctx->last_error = "a bounded device wait of an earlier call ran out; its results are invalid";
    return RIX_ETIMEOUT;
  }
  return RIX_OK;
}

extern "C" rix_status rix_check(rix_ctx *ctx, void *stream) {
  if (!ctx) return RIX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    ctx->last_error = "rix_check synchronises the stream and cannot run inside a graph capture";
    return RIX_ESTATE;
  }
  RIX_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return rix_take_err(ctx);
}

extern "C" rix_status rix_build_K(rix_ctx *ctx, const double *D, double *K, void *stream) {
  if (!ctx || !D || !K) return RIX_EINVAL;
  if (!ctx->have_cv) return RIX_ESTATE;
  rix_status s = rix_take_err(ctx);
  if (s != RIX_OK) return s;
  ctx->fwd_valid = false;
  s = rix_fp64_build(ctx, D, K, (cudaStream_t)stream);
  if (s == RIX_OK && ctx->nblk == 1) {
    ctx->fwd_D = D;
    ctx->fwd_K = K;
    ctx->fwd_valid = true;
  }
  return s;
}

extern "C" rix_status rix_build_K_delta(rix_ctx *ctx, const double *dD, double *K, void *stream) {
  if (!ctx || !dD || !K) return RIX_EINVAL;
  if (!ctx->have_cv) return RIX_ESTATE;
  rix_status s = rix_take_err(ctx);
  if (s != RIX_OK) return s;
  ctx->fwd_valid = false;
  return rix_fp64_build(ctx, dD, K, (cudaStream_t)stream, 1);
}

extern "C" rix_status rix_energy(rix_ctx *ctx, const double *D, const double *K, double *Ex, void *stream) {
  if (!ctx || !D || !K || !Ex) return RIX_EINVAL;
  rix_status s = rix_take_err(ctx);
  if (s != RIX_OK) return s;
  if (D != ctx->fwd_D) ctx->fwd_valid = false;  // the D screening flags follow this D
  return rix_launch_energy(ctx, D, K, Ex, (cudaStream_t)stream);
}

extern "C" rix_status rix_fold_gamma(rix_ctx *ctx, const double *K, double *Kd, void *stream) {
  if (!ctx || !K || !Kd) return RIX_EINVAL;
  return rix_launch_fold(ctx, K, Kd, (cudaStream_t)stream);
}

extern "C" rix_status rix_stats(const rix_ctx *ctx, rix_stats_t *out) {
  if (!ctx || !out) return RIX_EINVAL;
  *out = ctx->stats;
  out->workspace_bytes = (int64_t)ctx->dev_bytes;
  out->n_row_blocks = ctx->nblk;
  out->launches_build = rix_launch_count(ctx);
  out->nbasis = ctx->nbasis;
  return RIX_OK;
}

extern "C" const char *rix_strerror(rix_status s) {
  switch (s) {
    case RIX_OK: return "ok";
    case RIX_EINVAL: return "invalid argument";
    case RIX_ENOMEM: return "out of memory";
    case RIX_ECUDA: return "CUDA error";
    case RIX_ENOTSYM: return "C or V not pair-symmetric";
    case RIX_ETIMEOUT: return "device wait timed out";
    case RIX_EUNSUPPORTED: return "unsupported";
    case RIX_ESTATE: return "call out of order";
  }
  return "unknown status";
}

extern "C" const char *rix_last_error(const rix_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

rix_status rix_prof_mark(rix_ctx *ctx, int i, cudaStream_t st) {
  if (!ctx->opt.profile) return RIX_OK;
  // no stage events inside a CUDA graph capture (replays would not refresh them)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st != nullptr && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return RIX_OK;
  // at most 4096 builds are kept between two reads
  if (i == 0 && ctx->ev_pending.size() >= (size_t)4096 * (rix_ctx::NSTAGE + 1)) return RIX_OK;
  if (i != 0 && ctx->ev_pending.size() % (rix_ctx::NSTAGE + 1) == 0) return RIX_OK;
  cudaEvent_t e;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else {
    RIX_CUDA_TRY(ctx, cudaEventCreate(&e));
  }
  RIX_CUDA_TRY(ctx, cudaEventRecord(e, st));
  ctx->ev_pending.push_back(e);
  return RIX_OK;
}

extern "C" rix_status rix_stage_times(rix_ctx *ctx, double *ms, int32_t n, int32_t *n_builds) {
  if (!ctx || !ms || n < 0) return RIX_EINVAL;
  if (!ctx->opt.profile) return RIX_EUNSUPPORTED;
  const int W = rix_ctx::NSTAGE + 1;
  for (int i = 0; i < n; i++) ms[i] = 0.0;
  size_t full = ctx->ev_pending.size() / W * W;
  int nb = (int)(full / W);
  if (full) RIX_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev_pending[full - 1]));
  for (int b = 0; b < nb; b++)
    for (int s = 0; s < rix_ctx::NSTAGE && s < n; s++) {
      float t = 0.f;
      RIX_CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->ev_pending[b * W + s], ctx->ev_pending[b * W + s + 1]));
      ms[s] += t;
    }
  for (auto e : ctx->ev_pending) ctx->ev_pool.push_back(e);
  ctx->ev_pending.clear();
  if (n_builds) *n_builds = nb;
  return RIX_OK;
}

extern "C" void rix_destroy(rix_ctx *ctx) {
  if (!ctx) return;
  rix_mixed_free(ctx);
  for (auto e : ctx->ev_pending) cudaEventDestroy(e);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  for (auto e : ctx->gemm_ev) cudaEventDestroy(e);
  for (auto e : ctx->gemm_ev_pool) cudaEventDestroy(e);
  for (auto &b : ctx->bufs) cudaFree(b.p);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  delete ctx;
}
