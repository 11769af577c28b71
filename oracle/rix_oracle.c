/*
 * rix oracle -- plain, slow, FP64 CPU reference of the RI-LVL exchange build.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code with the CUDA library.
 *
 * What it computes (paper, Sec. "Description of the real-space formalism"):
 *
 *   K_il = sum_{jk} sum_{PQ} C^P_ij V_PQ C^Q_kl D_jk            (Eq. 4)
 *   E_x  = -1/4 sum_il D_li K_il                                   (-1/4 Tr(D K))
 *
 * with the RI-LVL restriction C^P_ij = 0 unless P sits on the atom of i or the
 * atom of j (Eqs. 6-7), image-resolved lattice sums (Eq. 4) and the
 * translational symmetry C^{mu(R')}_{i(0) k(R')} = C^{mu(0)}_{k(0) i(-R')}.
 *
 * The sum is taken in the paper's grouping by which atom carries P and which
 * carries Q (Eq. 11 with the intermediates of Eqs. 12a-12d; i on A, j on B,
 * k on G, l on E):
 *   term 1  P on A, Q on E         : T = C D (E = C*D), U = V^T T, K += U C
 *   term 2  P on A, Q on G (G!=E)  : U = V(A,G)^T T,   K += U C
 *   term 3  P on B (B!=A), Q on E  : S = D C, Z3 = V S, K += C Z3
 *   term 4  P on B (B!=A), Q on G (G!=E): Y = D C, Z4 = sum_G V Y, K += C Z4
 * (the paper's H = F D, 2G and F E pieces; term 3 is computed directly here,
 * not as the transpose of term 2).  Every loop is explicit; no BLAS.
 *
 * Atoms in other cells are nodes (atom, n1, n2, n3).  A pair (X, Y, n) links
 * node (X, 0) to node (Y, n); blocks between (X, a) and (Y, b) are the pair
 * (X, Y, b - a).  Input screening (paper Sec. "Initialization": compression
 * below 1e-10): a C, V or D block with max |x| < tau is treated as zero.
 *
 * Canonical packed layout of the inputs:
 *   C(A,B,n) [P][i][j], P over aux(A) then aux(B) (aux(A) only on-site)
 *   V(A,B,n) [P][Q];  D(A,B,n) [i][j];  K(A,E,n) [i][l]
 * blocks back to back in lexicographic (A, B, n1, n2, n3) order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EMPTY UINT64_MAX

/* ------------------------------------------------------------------ keys */
static uint64_t pair_key(int64_t a, int64_t b, int n1, int n2, int n3) {
    return ((uint64_t)a << 44) | ((uint64_t)b << 24) | ((uint64_t)(n1 + 128) << 16) |
           ((uint64_t)(n2 + 128) << 8) | (uint64_t)(n3 + 128);
}
static uint64_t node_key(int64_t a, int n1, int n2, int n3) {
    return ((uint64_t)a << 24) | ((uint64_t)(n1 + 128) << 16) | ((uint64_t)(n2 + 128) << 8) |
           (uint64_t)(n3 + 128);
}

/* ----------------------------------------------- open-addressing hash map */
typedef struct { uint64_t *k; int64_t *v; int64_t cap, n; } hmap;

static void hm_init(hmap *h, int64_t expect) {
    int64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    h->cap = cap; h->n = 0;
    h->k = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    h->v = (int64_t *)malloc(sizeof(int64_t) * cap);
    for (int64_t i = 0; i < cap; i++) h->k[i] = EMPTY;
}
static void hm_free(hmap *h) { free(h->k); free(h->v); h->k = NULL; h->v = NULL; }
static int64_t hm_slot(const hmap *h, uint64_t key) {
    uint64_t x = key * 0x9E3779B97F4A7C15ull;
    int64_t s = (int64_t)(x >> 17) & (h->cap - 1);
    while (h->k[s] != EMPTY && h->k[s] != key) s = (s + 1) & (h->cap - 1);
    return s;
}
static int64_t hm_get(const hmap *h, uint64_t key) {
    int64_t s = hm_slot(h, key);
    return h->k[s] == key ? h->v[s] : -1;
}
static void hm_grow(hmap *h) {
    hmap g; hm_init(&g, h->cap);
    for (int64_t i = 0; i < h->cap; i++)
        if (h->k[i] != EMPTY) { int64_t s = hm_slot(&g, h->k[i]); g.k[s] = h->k[i]; g.v[s] = h->v[i]; g.n++; }
    hm_free(h); *h = g;
}
/* returns existing value, or inserts val and returns -1 - (new index) convention: here insert-if-absent */
static int64_t hm_get_or_put(hmap *h, uint64_t key, int64_t val) {
    if (2 * (h->n + 1) > h->cap) hm_grow(h);
    int64_t s = hm_slot(h, key);
    if (h->k[s] == key) return h->v[s];
    h->k[s] = key; h->v[s] = val; h->n++;
    return val;
}

/* ------------------------------------------------------------ the system */
typedef struct {
    int nat, nsp, periodic;
    double *xyz, cell[9], rc, tau;
    int *sp, *nbs, *nas;
    /* pair list (own construction) */
    int64_t np;
    int32_t *pA, *pB, *pn;     /* pn: [np][3] */
    uint8_t *onsite;
    int64_t *partner, *rowptr;  /* rowptr[nat+1] */
    int64_t *offC, *offV, *offD;
    hmap pairs;
    /* data */
    const double *C, *V, *D;
    uint8_t *keepC, *keepV, *keepD;
    /* K pattern for the selected rows */
    int nrows; int32_t *rows;
    int64_t nk; uint64_t *kkeys; int64_t *offK; int64_t *krow; /* krow[nrows+1] */
    int terms;  /* bit t-1 enables term t (all four by default) */
    int dry;    /* 1: count the multiply-adds of a build without doing them */
    double flops;  /* FLOPs (2 per multiply-add) of the last build */
    int sampled;   /* 1: K only for the blocks listed in kkeys (orc_kpattern_blocks) */
    hmap needZ;    /* sampled mode: Z blocks (B, E', m) some listed K block uses */
} orc;

static inline int NB(const orc *o, int a) { return o->nbs[o->sp[a]]; }
static inline int NA(const orc *o, int a) { return o->nas[o->sp[a]]; }

/* squared distance of pair (a, b, n) in the exact operation order of the
 * canonical format, evaluated in the representative orientation */
static double d2_raw(const orc *o, int a, int b, int n1, int n2, int n3) {
    double s[3] = {0, 0, 0};
    if (o->periodic) {
        for (int c = 0; c < 3; c++)
            s[c] = ((double)n1 * o->cell[0 * 3 + c] + (double)n2 * o->cell[1 * 3 + c]) + (double)n3 * o->cell[2 * 3 + c];
    }
    double dx[3];
    for (int c = 0; c < 3; c++) dx[c] = (o->xyz[3 * b + c] + s[c]) - o->xyz[3 * a + c];
    return (dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2];
}
static int is_rep(int a, int b, int n1, int n2, int n3) {
    if (a < b) return 1;
    if (a > b) return 0;
    if (n1 != 0) return n1 > 0;
    if (n2 != 0) return n2 > 0;
    return n3 >= 0; /* n == 0 (on-site) counts as its own representative */
}
static double pair_d2(const orc *o, int a, int b, int n1, int n2, int n3) {
    if (is_rep(a, b, n1, n2, n3)) return d2_raw(o, a, b, n1, n2, n3);
    return d2_raw(o, b, a, -n1, -n2, -n3);
}

static void inv3(const double *m, double *r) {
    double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) + m[2] * (m[3] * m[7] - m[4] * m[6]);
    r[0] = (m[4] * m[8] - m[5] * m[7]) / det; r[1] = (m[2] * m[7] - m[1] * m[8]) / det; r[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    r[3] = (m[5] * m[6] - m[3] * m[8]) / det; r[4] = (m[0] * m[8] - m[2] * m[6]) / det; r[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    r[6] = (m[3] * m[7] - m[4] * m[6]) / det; r[7] = (m[1] * m[6] - m[0] * m[7]) / det; r[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

/* Build the pair list: brute force over atoms and over every image that can
 * come within the cutoff (plane spacing h_i, fractional spread w_i:
 * |n_i| <= floor(rc/h_i + w_i)).  Rows come out sorted (B, then n). */
static int build_pairs(orc *o) {
    int nr[3] = {0, 0, 0};
    if (o->periodic) {
        double inv[9];
        inv3(o->cell, inv);
        double vol = fabs(o->cell[0] * (o->cell[4] * o->cell[8] - o->cell[5] * o->cell[7]) -
                          o->cell[1] * (o->cell[3] * o->cell[8] - o->cell[5] * o->cell[6]) +
                          o->cell[2] * (o->cell[3] * o->cell[7] - o->cell[4] * o->cell[6]));
        for (int d = 0; d < 3; d++) {
            const double *u = o->cell + 3 * ((d + 1) % 3), *v = o->cell + 3 * ((d + 2) % 3);
            double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
            double h = vol / sqrt(cx * cx + cy * cy + cz * cz);
            double fmin = 1e300, fmax = -1e300;
            for (int a = 0; a < o->nat; a++) {
                double f = o->xyz[3 * a] * inv[0 * 3 + d] + o->xyz[3 * a + 1] * inv[1 * 3 + d] + o->xyz[3 * a + 2] * inv[2 * 3 + d];
                if (f < fmin) fmin = f;
                if (f > fmax) fmax = f;
            }
            nr[d] = (int)floor(o->rc / h + (fmax - fmin));
        }
    }
    double rc2 = o->rc * o->rc;
    int cut = o->rc > 0;
    int64_t *cnt = (int64_t *)calloc(o->nat + 1, sizeof(int64_t));
    /* pass 1: count */
    #pragma omp parallel for schedule(dynamic, 4)
    for (int a = 0; a < o->nat; a++) {
        int64_t c = 0;
        for (int b = 0; b < o->nat; b++)
            for (int n1 = -nr[0]; n1 <= nr[0]; n1++)
                for (int n2 = -nr[1]; n2 <= nr[1]; n2++)
                    for (int n3 = -nr[2]; n3 <= nr[2]; n3++)
                        if (!cut || pair_d2(o, a, b, n1, n2, n3) < rc2) c++;
        cnt[a + 1] = c;
    }
    o->rowptr = (int64_t *)malloc(sizeof(int64_t) * (o->nat + 1));
    o->rowptr[0] = 0;
    for (int a = 0; a < o->nat; a++) o->rowptr[a + 1] = o->rowptr[a] + cnt[a + 1];
    free(cnt);
    o->np = o->rowptr[o->nat];
    o->pA = (int32_t *)malloc(sizeof(int32_t) * o->np);
    o->pB = (int32_t *)malloc(sizeof(int32_t) * o->np);
    o->pn = (int32_t *)malloc(sizeof(int32_t) * 3 * o->np);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int a = 0; a < o->nat; a++) {
        int64_t c = o->rowptr[a];
        for (int b = 0; b < o->nat; b++)
            for (int n1 = -nr[0]; n1 <= nr[0]; n1++)
                for (int n2 = -nr[1]; n2 <= nr[1]; n2++)
                    for (int n3 = -nr[2]; n3 <= nr[2]; n3++)
                        if (!cut || pair_d2(o, a, b, n1, n2, n3) < rc2) {
                            o->pA[c] = a; o->pB[c] = b;
                            o->pn[3 * c] = n1; o->pn[3 * c + 1] = n2; o->pn[3 * c + 2] = n3;
                            c++;
                        }
    }
    hm_init(&o->pairs, o->np);
    for (int64_t p = 0; p < o->np; p++)
        hm_get_or_put(&o->pairs, pair_key(o->pA[p], o->pB[p], o->pn[3 * p], o->pn[3 * p + 1], o->pn[3 * p + 2]), p);
    o->onsite = (uint8_t *)malloc(o->np);
    o->partner = (int64_t *)malloc(sizeof(int64_t) * o->np);
    o->offC = (int64_t *)malloc(sizeof(int64_t) * (o->np + 1));
    o->offV = (int64_t *)malloc(sizeof(int64_t) * (o->np + 1));
    o->offD = (int64_t *)malloc(sizeof(int64_t) * (o->np + 1));
    o->offC[0] = o->offV[0] = o->offD[0] = 0;
    for (int64_t p = 0; p < o->np; p++) {
        int a = o->pA[p], b = o->pB[p];
        const int32_t *n = o->pn + 3 * p;
        o->onsite[p] = (a == b && n[0] == 0 && n[1] == 0 && n[2] == 0);
        o->partner[p] = hm_get(&o->pairs, pair_key(b, a, -n[0], -n[1], -n[2]));
        if (o->partner[p] < 0) return -1;
        int64_t rows = NA(o, a) + (o->onsite[p] ? 0 : NA(o, b));
        o->offC[p + 1] = o->offC[p] + rows * NB(o, a) * NB(o, b);
        o->offV[p + 1] = o->offV[p] + (int64_t)NA(o, a) * NA(o, b);
        o->offD[p + 1] = o->offD[p] + (int64_t)NB(o, a) * NB(o, b);
    }
    return 0;
}

static int64_t find_pair(const orc *o, int a, int b, int n1, int n2, int n3) {
    if (n1 < -127 || n1 > 127 || n2 < -127 || n2 > 127 || n3 < -127 || n3 > 127) return -1;
    return hm_get(&o->pairs, pair_key(a, b, n1, n2, n3));
}

/* ------------------------------------------------------------- public API */
void *orc_create(int nat, const double *xyz, const int *species, int nsp, const int *nbas,
                 const int *naux, const double *cell, double cutoff, double tau) {
    orc *o = (orc *)calloc(1, sizeof(orc));
    o->nat = nat; o->nsp = nsp;
    o->xyz = (double *)malloc(sizeof(double) * 3 * nat); memcpy(o->xyz, xyz, sizeof(double) * 3 * nat);
    o->sp = (int *)malloc(sizeof(int) * nat); memcpy(o->sp, species, sizeof(int) * nat);
    o->nbs = (int *)malloc(sizeof(int) * nsp); memcpy(o->nbs, nbas, sizeof(int) * nsp);
    o->nas = (int *)malloc(sizeof(int) * nsp); memcpy(o->nas, naux, sizeof(int) * nsp);
    o->periodic = cell != NULL;
    if (cell) memcpy(o->cell, cell, sizeof(double) * 9);
    o->rc = cutoff; o->tau = tau;
    if (o->periodic && cutoff <= 0) { free(o); return NULL; }
    o->terms = 15;
    if (build_pairs(o) != 0) return NULL;
    return o;
}

/* Restrict the sum to a subset of the four terms (bit t-1 = term t); for tests. */
void orc_set_terms(void *h, int mask) { ((orc *)h)->terms = mask; }

int64_t orc_npairs(void *h) { return ((orc *)h)->np; }
void orc_pairs(void *h, int64_t *keys) {
    orc *o = (orc *)h;
    for (int64_t p = 0; p < o->np; p++)
        keys[p] = (int64_t)pair_key(o->pA[p], o->pB[p], o->pn[3 * p], o->pn[3 * p + 1], o->pn[3 * p + 2]);
}
int64_t orc_size(void *h, int which) {
    orc *o = (orc *)h;
    return which == 0 ? o->offC[o->np] : which == 1 ? o->offV[o->np] : o->offD[o->np];
}

static double blockmax(const double *x, int64_t n) {
    double m = 0;
    for (int64_t i = 0; i < n; i++) { double a = fabs(x[i]); if (a > m) m = a; }
    return m;
}

/* Attach the packed inputs and derive the screening flags. */
void orc_set_data(void *h, const double *C, const double *V, const double *D) {
    orc *o = (orc *)h;
    o->C = C; o->V = V; o->D = D;
    free(o->keepC); free(o->keepV); free(o->keepD);
    o->keepC = (uint8_t *)malloc(o->np); o->keepV = (uint8_t *)malloc(o->np); o->keepD = (uint8_t *)malloc(o->np);
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < o->np; p++) {
        if (o->tau > 0) {
            o->keepC[p] = blockmax(C + o->offC[p], o->offC[p + 1] - o->offC[p]) >= o->tau;
            o->keepV[p] = blockmax(V + o->offV[p], o->offV[p + 1] - o->offV[p]) >= o->tau;
            o->keepD[p] = blockmax(D + o->offD[p], o->offD[p + 1] - o->offD[p]) >= o->tau;
        } else {
            o->keepC[p] = o->keepV[p] = o->keepD[p] = 1;
        }
    }
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* K pattern for the chosen row atoms: every node reachable from the row atom
 * by at most three pair hops (the furthest reach of term 4). */
int64_t orc_kpattern(void *h, int nrows, const int32_t *rows) {
    orc *o = (orc *)h;
    free(o->rows); free(o->kkeys); free(o->offK); free(o->krow);
    if (o->sampled) { hm_free(&o->needZ); o->sampled = 0; }
    if (nrows < 0) {
        o->nrows = o->nat;
        o->rows = (int32_t *)malloc(sizeof(int32_t) * o->nat);
        for (int a = 0; a < o->nat; a++) o->rows[a] = a;
    } else {
        o->nrows = nrows;
        o->rows = (int32_t *)malloc(sizeof(int32_t) * (nrows + 1));
        memcpy(o->rows, rows, sizeof(int32_t) * nrows);
    }
    uint64_t **lists = (uint64_t **)calloc(o->nrows, sizeof(uint64_t *));
    int64_t *lens = (int64_t *)calloc(o->nrows, sizeof(int64_t));
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < o->nrows; r++) {
        int a = o->rows[r];
        hmap seen; hm_init(&seen, 4096);
        /* frontier expansion, three hops; nodes stored as (atom, n) */
        int64_t cap = 4096, n = 0;
        uint64_t *nodes = (uint64_t *)malloc(sizeof(uint64_t) * cap);
        int32_t *na_ = (int32_t *)malloc(sizeof(int32_t) * cap * 4);
        nodes[n] = node_key(a, 0, 0, 0); na_[0] = a; na_[1] = na_[2] = na_[3] = 0;
        hm_get_or_put(&seen, nodes[0], 0); n = 1;
        int64_t lo = 0, hi = 1;
        for (int hop = 0; hop < 3; hop++) {
            for (int64_t x = lo; x < hi; x++) {
                int xa = na_[4 * x]; int m1 = na_[4 * x + 1], m2 = na_[4 * x + 2], m3 = na_[4 * x + 3];
                for (int64_t p = o->rowptr[xa]; p < o->rowptr[xa + 1]; p++) {
                    int yb = o->pB[p];
                    int q1 = m1 + o->pn[3 * p], q2 = m2 + o->pn[3 * p + 1], q3 = m3 + o->pn[3 * p + 2];
                    uint64_t k = node_key(yb, q1, q2, q3);
                    if (hm_get(&seen, k) >= 0) continue;
                    if (n == cap) {
                        cap *= 2;
                        nodes = (uint64_t *)realloc(nodes, sizeof(uint64_t) * cap);
                        na_ = (int32_t *)realloc(na_, sizeof(int32_t) * cap * 4);
                    }
                    nodes[n] = k; na_[4 * n] = yb; na_[4 * n + 1] = q1; na_[4 * n + 2] = q2; na_[4 * n + 3] = q3;
                    hm_get_or_put(&seen, k, n);
                    n++;
                }
            }
            lo = hi; hi = n;
        }
        uint64_t *pk = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int64_t x = 0; x < n; x++)
            pk[x] = pair_key(a, na_[4 * x], na_[4 * x + 1], na_[4 * x + 2], na_[4 * x + 3]);
        qsort(pk, n, sizeof(uint64_t), cmp_u64);
        lists[r] = pk; lens[r] = n;
        free(nodes); free(na_); hm_free(&seen);
    }
    o->krow = (int64_t *)malloc(sizeof(int64_t) * (o->nrows + 1));
    o->krow[0] = 0;
    for (int r = 0; r < o->nrows; r++) o->krow[r + 1] = o->krow[r] + lens[r];
    o->nk = o->krow[o->nrows];
    o->kkeys = (uint64_t *)malloc(sizeof(uint64_t) * (o->nk + 1));
    o->offK = (int64_t *)malloc(sizeof(int64_t) * (o->nk + 1));
    for (int r = 0; r < o->nrows; r++) {
        memcpy(o->kkeys + o->krow[r], lists[r], sizeof(uint64_t) * lens[r]);
        free(lists[r]);
    }
    free(lists); free(lens);
    o->offK[0] = 0;
    for (int64_t x = 0; x < o->nk; x++) {
        int a = (int)((o->kkeys[x] >> 44) & 0xFFFFF), e = (int)((o->kkeys[x] >> 24) & 0xFFFFF);
        o->offK[x + 1] = o->offK[x] + (int64_t)NB(o, a) * NB(o, e);
    }
    return o->nk;
}
/* K pattern = an explicit list of blocks (A, E', n) (sampled mode): only these
 * blocks are computed, with T and Z restricted to what they need.  Returns the
 * number of blocks; their order follows orc_kkeys (sorted). */
static int cmp_u64b(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}
int64_t orc_kpattern_blocks(void *h, int64_t n, const int64_t *keys) {
    orc *o = (orc *)h;
    free(o->rows); free(o->kkeys); free(o->offK); free(o->krow);
    if (o->sampled) hm_free(&o->needZ);
    o->sampled = 1;
    o->kkeys = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    memcpy(o->kkeys, keys, sizeof(uint64_t) * n);
    qsort(o->kkeys, n, sizeof(uint64_t), cmp_u64b);
    o->nk = n;
    o->rows = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    o->krow = (int64_t *)malloc(sizeof(int64_t) * (n + 2));
    o->nrows = 0;
    for (int64_t x = 0; x < n; x++) {
        int a = (int)((o->kkeys[x] >> 44) & 0xFFFFF);
        if (o->nrows == 0 || o->rows[o->nrows - 1] != a) { o->rows[o->nrows] = a; o->krow[o->nrows] = x; o->nrows++; }
    }
    o->krow[o->nrows] = n;
    o->offK = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    o->offK[0] = 0;
    hm_init(&o->needZ, 4096);
    for (int64_t x = 0; x < n; x++) {
        int a = (int)((o->kkeys[x] >> 44) & 0xFFFFF), e = (int)((o->kkeys[x] >> 24) & 0xFFFFF);
        int m1 = (int)((o->kkeys[x] >> 16) & 0xFF) - 128, m2 = (int)((o->kkeys[x] >> 8) & 0xFF) - 128,
            m3 = (int)(o->kkeys[x] & 0xFF) - 128;
        o->offK[x + 1] = o->offK[x] + (int64_t)NB(o, a) * NB(o, e);
        for (int64_t p = o->rowptr[a]; p < o->rowptr[a + 1]; p++) {
            const int32_t *n1 = o->pn + 3 * p;
            hm_get_or_put(&o->needZ, pair_key(o->pB[p], e, m1 - n1[0], m2 - n1[1], m3 - n1[2]), 1);
        }
    }
    return n;
}

void orc_kkeys(void *h, int64_t *keys) {
    orc *o = (orc *)h;
    memcpy(keys, o->kkeys, sizeof(int64_t) * o->nk);
}
int64_t orc_ksize(void *h) { orc *o = (orc *)h; return o->offK[o->nk]; }

/* --------------------------------------------------------- node storage */
/* A growable set of dense blocks keyed by node: used for T (per row atom),
 * Z and S (per B atom). */
typedef struct { hmap map; int64_t n, cap, used, bcap; int64_t *off; int32_t *atom; int32_t *img; double *buf; } nodestore;

static void ns_init(nodestore *s) {
    hm_init(&s->map, 256); s->n = 0; s->cap = 256; s->used = 0; s->bcap = 1 << 16;
    s->off = (int64_t *)malloc(sizeof(int64_t) * s->cap);
    s->atom = (int32_t *)malloc(sizeof(int32_t) * s->cap);
    s->img = (int32_t *)malloc(sizeof(int32_t) * 3 * s->cap);
    s->buf = (double *)calloc(s->bcap, sizeof(double));
}
static void ns_free(nodestore *s) { hm_free(&s->map); free(s->off); free(s->atom); free(s->img); free(s->buf); }
/* offset of the block of node (atom, m) of size sz, created zeroed if absent */
static int64_t ns_block(nodestore *s, int atom, int m1, int m2, int m3, int64_t sz) {
    uint64_t k = node_key(atom, m1, m2, m3);
    int64_t id = hm_get(&s->map, k);
    if (id >= 0) return s->off[id];
    if (s->n == s->cap) {
        s->cap *= 2;
        s->off = (int64_t *)realloc(s->off, sizeof(int64_t) * s->cap);
        s->atom = (int32_t *)realloc(s->atom, sizeof(int32_t) * s->cap);
        s->img = (int32_t *)realloc(s->img, sizeof(int32_t) * 3 * s->cap);
    }
    while (s->used + sz > s->bcap) {
        int64_t nc = s->bcap * 2;
        s->buf = (double *)realloc(s->buf, sizeof(double) * nc);
        memset(s->buf + s->bcap, 0, sizeof(double) * (nc - s->bcap));
        s->bcap = nc;
    }
    id = s->n++;
    s->off[id] = s->used; s->atom[id] = atom;
    s->img[3 * id] = m1; s->img[3 * id + 1] = m2; s->img[3 * id + 2] = m3;
    s->used += sz;
    hm_get_or_put(&s->map, k, id);
    return s->off[id];
}
static int64_t ns_find(const nodestore *s, int atom, int m1, int m2, int m3) {
    int64_t id = hm_get(&s->map, node_key(atom, m1, m2, m3));
    return id < 0 ? -1 : s->off[id];
}

/* ------------------------------------------------------- terms 3 and 4 */
/* Z(B; E') [P in aux(B)][j in B][l in E'] for every node E' two hops from B:
 *   term 3: Z += V(B,E') S(B,E'),  S^Q_jl = sum_{G'} sum_k D(B,G')_jk C(G',E')^{Q on E'}_kl
 *   term 4: Z += sum_{G' != E'} V(B,G') Y,  Y^Q_jl = sum_k D(B,G')_jk C(G',E')^{Q on G'}_kl
 * (the paper's H = F D and G pieces for P on the second atom). */
static void build_Z(const orc *o, int b, nodestore *Z, double *fl) {
    int nbB = NB(o, b), naB = NA(o, b);
    nodestore S; ns_init(&S);
    double *Y = NULL; int64_t ycap = 0;
    for (int64_t p2 = o->rowptr[b]; p2 < o->rowptr[b + 1]; p2++) {
        if (!o->keepD[p2]) continue;
        int g = o->pB[p2]; const int32_t *n2 = o->pn + 3 * p2;
        int nbG = NB(o, g), naG = NA(o, g);
        const double *Dbg = o->D + o->offD[p2];
        const double *Vbg = o->V + o->offV[p2];
        for (int64_t p3 = o->rowptr[g]; p3 < o->rowptr[g + 1]; p3++) {
            if (!o->keepC[p3]) continue;
            int e = o->pB[p3]; const int32_t *n3 = o->pn + 3 * p3;
            int nbE = NB(o, e), naE = NA(o, e);
            int m1 = n2[0] + n3[0], m2 = n2[1] + n3[1], m3 = n2[2] + n3[2];
            const double *Cge = o->C + o->offC[p3];
            int qE0 = o->onsite[p3] ? 0 : naG;  /* first row of aux(E') in C(G',E') */
            if (o->sampled && hm_get(&o->needZ, pair_key(b, e, m1, m2, m3)) < 0) continue;
            /* term 3: S(B,E') if V(B,E') is present */
            int64_t pbe = find_pair(o, b, e, m1, m2, m3);
            if ((o->terms & 4) && pbe >= 0 && o->keepV[pbe]) {
                int64_t so = ns_block(&S, e, m1, m2, m3, (int64_t)naE * nbB * nbE);
                double *s = S.buf + so;
                *fl += 2.0 * naE * nbB * nbE * nbG;
                if (!o->dry)
                for (int q = 0; q < naE; q++)
                    for (int j = 0; j < nbB; j++)
                        for (int l = 0; l < nbE; l++) {
                            double acc = 0;
                            for (int k = 0; k < nbG; k++)
                                acc += Dbg[j * nbG + k] * Cge[((int64_t)(qE0 + q) * nbG + k) * nbE + l];
                            s[((int64_t)q * nbB + j) * nbE + l] += acc;
                        }
            }
            /* term 4: Q on G' != E', needs V(B,G') */
            if ((o->terms & 8) && !o->onsite[p3] && o->keepV[p2]) {
                int64_t ysz = (int64_t)naG * nbB * nbE;
                if (ysz > ycap) { free(Y); ycap = ysz; Y = (double *)malloc(sizeof(double) * ycap); }
                *fl += 2.0 * naG * nbB * nbE * nbG + 2.0 * naB * nbB * nbE * naG;
                if (!o->dry)
                for (int q = 0; q < naG; q++)
                    for (int j = 0; j < nbB; j++)
                        for (int l = 0; l < nbE; l++) {
                            double acc = 0;
                            for (int k = 0; k < nbG; k++)
                                acc += Dbg[j * nbG + k] * Cge[((int64_t)q * nbG + k) * nbE + l];
                            Y[((int64_t)q * nbB + j) * nbE + l] = acc;
                        }
                int64_t zo = ns_block(Z, e, m1, m2, m3, (int64_t)naB * nbB * nbE);
                double *z = Z->buf + zo;
                if (!o->dry)
                for (int pp = 0; pp < naB; pp++)
                    for (int j = 0; j < nbB; j++)
                        for (int l = 0; l < nbE; l++) {
                            double acc = 0;
                            for (int q = 0; q < naG; q++)
                                acc += Vbg[(int64_t)pp * naG + q] * Y[((int64_t)q * nbB + j) * nbE + l];
                            z[((int64_t)pp * nbB + j) * nbE + l] += acc;
                        }
            }
        }
    }
    /* term 3: Z += V(B,E') S */
    for (int64_t id = 0; id < S.n; id++) {
        int e = S.atom[id]; const int32_t *m = S.img + 3 * id;
        int nbE = NB(o, e), naE = NA(o, e);
        int64_t pbe = find_pair(o, b, e, m[0], m[1], m[2]);
        const double *Vbe = o->V + o->offV[pbe];
        const double *s = S.buf + S.off[id];
        int64_t zo = ns_block(Z, e, m[0], m[1], m[2], (int64_t)naB * nbB * nbE);
        double *z = Z->buf + zo;
        *fl += 2.0 * naB * nbB * nbE * naE;
        if (!o->dry)
        for (int pp = 0; pp < naB; pp++)
            for (int j = 0; j < nbB; j++)
                for (int l = 0; l < nbE; l++) {
                    double acc = 0;
                    for (int q = 0; q < naE; q++)
                        acc += Vbe[(int64_t)pp * naE + q] * s[((int64_t)q * nbB + j) * nbE + l];
                    z[((int64_t)pp * nbB + j) * nbE + l] += acc;
                }
    }
    free(Y);
    ns_free(&S);
}

/* index of a K block in a row (the pattern holds every node the terms reach) */
static int64_t kfind(const orc *o, int64_t lo, int64_t hi, uint64_t key) {
    const int64_t end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (o->kkeys[mid] < key) lo = mid + 1; else hi = mid;
    }
    if (lo < end && o->kkeys[lo] == key) return lo;
    return o->sampled ? -1 : lo;  /* a full pattern contains every node the terms reach */
}

/* ---------------------------------------------------------- one K row */
static void k_row(const orc *o, int r, nodestore *Zs, const uint8_t *haveZ, double *K, double *fl) {
    int a = o->rows[r];
    int nbA = NB(o, a), naA = NA(o, a);
    int64_t k0 = o->krow[r], k1 = o->krow[r + 1];
    /* K blocks of this row: binary search in the sorted row keys */
#define KBLOCK(E, M1, M2, M3) kfind(o, k0, k1, pair_key(a, (E), (M1), (M2), (M3)))
    /* sampled mode: T only for the nodes G' next to a listed E' of this row */
    hmap needT; hm_init(&needT, 64);
    if (o->sampled)
        for (int64_t x = k0; x < k1; x++) {
            int e = (int)((o->kkeys[x] >> 24) & 0xFFFFF);
            int m1 = (int)((o->kkeys[x] >> 16) & 0xFF) - 128, m2 = (int)((o->kkeys[x] >> 8) & 0xFF) - 128,
                m3 = (int)(o->kkeys[x] & 0xFF) - 128;
            for (int64_t q = o->rowptr[e]; q < o->rowptr[e + 1]; q++) {
                const int32_t *nq = o->pn + 3 * q;
                hm_get_or_put(&needT, node_key(o->pB[q], m1 + nq[0], m2 + nq[1], m3 + nq[2]), 1);
            }
        }
    /* term 1/2 intermediate T(A,G') [P in aux(A)][i][k] = sum_{B'} C(A,B')^{P on A} D(B',G') */
    nodestore T; ns_init(&T);
    for (int64_t p1 = o->rowptr[a]; p1 < o->rowptr[a + 1]; p1++) {
        if (!o->keepC[p1]) continue;
        int b = o->pB[p1]; const int32_t *n1 = o->pn + 3 * p1;
        int nbB = NB(o, b);
        const double *Cab = o->C + o->offC[p1];
        for (int64_t p2 = o->rowptr[b]; p2 < o->rowptr[b + 1]; p2++) {
            if (!o->keepD[p2]) continue;
            int g = o->pB[p2]; const int32_t *n2 = o->pn + 3 * p2;
            int nbG = NB(o, g);
            const double *Dbg = o->D + o->offD[p2];
            if (o->sampled && hm_get(&needT, node_key(g, n1[0] + n2[0], n1[1] + n2[1], n1[2] + n2[2])) < 0) continue;
            int64_t to = ns_block(&T, g, n1[0] + n2[0], n1[1] + n2[1], n1[2] + n2[2], (int64_t)naA * nbA * nbG);
            double *t = T.buf + to;
            *fl += 2.0 * naA * nbA * nbG * nbB;
            if (!o->dry)
            for (int pp = 0; pp < naA; pp++)
                for (int i = 0; i < nbA; i++)
                    for (int k = 0; k < nbG; k++) {
                        double acc = 0;
                        for (int j = 0; j < nbB; j++)
                            acc += Cab[((int64_t)pp * nbA + i) * nbB + j] * Dbg[j * nbG + k];
                        t[((int64_t)pp * nbA + i) * nbG + k] += acc;
                    }
        }
    }
    /* terms 1 and 2 */
    double *U1 = NULL, *U2 = NULL; int64_t u1cap = 0, u2cap = 0;
    for (int64_t id = 0; id < T.n; id++) {
        int g = T.atom[id]; const int32_t *m = T.img + 3 * id;
        int nbG = NB(o, g), naG = NA(o, g);
        const double *t = T.buf + T.off[id];
        /* U2 = V(A,G')^T T, Q on G' */
        int have2 = 0;
        int64_t pag = find_pair(o, a, g, m[0], m[1], m[2]);
        if ((o->terms & 2) && pag >= 0 && o->keepV[pag]) {
            have2 = 1;
            int64_t sz = (int64_t)naG * nbA * nbG;
            if (sz > u2cap) { free(U2); u2cap = sz; U2 = (double *)malloc(sizeof(double) * sz); }
            const double *Vag = o->V + o->offV[pag];
            *fl += 2.0 * naG * nbA * nbG * naA;
            if (!o->dry)
            for (int q = 0; q < naG; q++)
                for (int i = 0; i < nbA; i++)
                    for (int k = 0; k < nbG; k++) {
                        double acc = 0;
                        for (int pp = 0; pp < naA; pp++)
                            acc += Vag[(int64_t)pp * naG + q] * t[((int64_t)pp * nbA + i) * nbG + k];
                        U2[((int64_t)q * nbA + i) * nbG + k] = acc;
                    }
        }
        for (int64_t p3 = o->rowptr[g]; p3 < o->rowptr[g + 1]; p3++) {
            if (!o->keepC[p3]) continue;
            int e = o->pB[p3]; const int32_t *n3 = o->pn + 3 * p3;
            int nbE = NB(o, e), naE = NA(o, e);
            int e1 = m[0] + n3[0], e2 = m[1] + n3[1], e3 = m[2] + n3[2];
            const double *Cge = o->C + o->offC[p3];
            const int64_t kx = KBLOCK(e, e1, e2, e3);
            if (kx < 0) continue;
            double *kb = K + o->offK[kx];
            /* term 1: P on A, Q on E' */
            int64_t pae = find_pair(o, a, e, e1, e2, e3);
            if ((o->terms & 1) && pae >= 0 && o->keepV[pae]) {
                int64_t sz = (int64_t)naE * nbA * nbG;
                if (sz > u1cap) { free(U1); u1cap = sz; U1 = (double *)malloc(sizeof(double) * sz); }
                const double *Vae = o->V + o->offV[pae];
                *fl += 2.0 * naE * nbA * nbG * naA + 2.0 * nbA * nbE * naE * nbG;
                if (!o->dry)
                for (int q = 0; q < naE; q++)
                    for (int i = 0; i < nbA; i++)
                        for (int k = 0; k < nbG; k++) {
                            double acc = 0;
                            for (int pp = 0; pp < naA; pp++)
                                acc += Vae[(int64_t)pp * naE + q] * t[((int64_t)pp * nbA + i) * nbG + k];
                            U1[((int64_t)q * nbA + i) * nbG + k] = acc;
                        }
                int qE0 = o->onsite[p3] ? 0 : naG;
                if (!o->dry)
                for (int i = 0; i < nbA; i++)
                    for (int l = 0; l < nbE; l++) {
                        double acc = 0;
                        for (int q = 0; q < naE; q++)
                            for (int k = 0; k < nbG; k++)
                                acc += U1[((int64_t)q * nbA + i) * nbG + k] * Cge[((int64_t)(qE0 + q) * nbG + k) * nbE + l];
                        kb[i * nbE + l] += acc;
                    }
            }
            /* term 2: P on A, Q on G' != E' */
            if (have2 && !o->onsite[p3]) {
                *fl += 2.0 * nbA * nbE * naG * nbG;
                if (!o->dry)
                for (int i = 0; i < nbA; i++)
                    for (int l = 0; l < nbE; l++) {
                        double acc = 0;
                        for (int q = 0; q < naG; q++)
                            for (int k = 0; k < nbG; k++)
                                acc += U2[((int64_t)q * nbA + i) * nbG + k] * Cge[((int64_t)q * nbG + k) * nbE + l];
                        kb[i * nbE + l] += acc;
                    }
            }
        }
    }
    free(U1); free(U2);
    ns_free(&T);
    /* terms 3 and 4: K(A,E') += C(A,B')^{P on B'} Z(B; E' - n1), B' != A */
    for (int64_t p1 = o->rowptr[a]; p1 < o->rowptr[a + 1]; p1++) {
        if (!o->keepC[p1] || o->onsite[p1]) continue;
        int b = o->pB[p1]; const int32_t *n1 = o->pn + 3 * p1;
        int nbB = NB(o, b), naB = NA(o, b);
        if (!haveZ[b]) continue;
        const nodestore *Z = Zs + b;
        const double *Cab = o->C + o->offC[p1];
        for (int64_t id = 0; id < Z->n; id++) {
            int e = Z->atom[id]; const int32_t *m = Z->img + 3 * id;
            int nbE = NB(o, e);
            const double *z = Z->buf + Z->off[id];
            const int64_t kx = KBLOCK(e, n1[0] + m[0], n1[1] + m[1], n1[2] + m[2]);
            if (kx < 0) continue;
            double *kb = K + o->offK[kx];
            *fl += 2.0 * nbA * nbE * naB * nbB;
            if (!o->dry)
            for (int i = 0; i < nbA; i++)
                for (int l = 0; l < nbE; l++) {
                    double acc = 0;
                    for (int pp = 0; pp < naB; pp++)
                        for (int j = 0; j < nbB; j++)
                            acc += Cab[((int64_t)(naA + pp) * nbA + i) * nbB + j] * z[((int64_t)pp * nbB + j) * nbE + l];
                    kb[i * nbE + l] += acc;
                }
        }
    }
    hm_free(&needT);
#undef KBLOCK
}

/* Exchange matrix rows for the pattern set by orc_kpattern; K is [ksize].
 * With dry = 1 the loops only count their multiply-adds (K is left zero). */
int orc_build_K_ex(void *h, double *K, int dry) {
    orc *o = (orc *)h;
    if (!o->C || !o->kkeys) return -1;
    o->dry = dry;
    memset(K, 0, sizeof(double) * o->offK[o->nk]);
    /* Z(B;.) for every B adjacent to a selected row */
    uint8_t *need = (uint8_t *)calloc(o->nat, 1);
    for (int r = 0; r < o->nrows; r++) {
        int a = o->rows[r];
        for (int64_t p = o->rowptr[a]; p < o->rowptr[a + 1]; p++) need[o->pB[p]] = 1;
    }
    nodestore *Zs = (nodestore *)calloc(o->nat, sizeof(nodestore));
    double fl = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(+ : fl)
    for (int b = 0; b < o->nat; b++) {
        if (!need[b]) continue;
        ns_init(&Zs[b]);
        build_Z(o, b, &Zs[b], &fl);
    }
    #pragma omp parallel for schedule(dynamic, 1) reduction(+ : fl)
    for (int r = 0; r < o->nrows; r++) k_row(o, r, Zs, need, K, &fl);
    for (int b = 0; b < o->nat; b++) if (need[b]) ns_free(&Zs[b]);
    free(Zs); free(need);
    o->flops = fl;
    o->dry = 0;
    return 0;
}
int orc_build_K(void *h, double *K) { return orc_build_K_ex(h, K, 0); }
double orc_flops(void *h) { return ((orc *)h)->flops; }

/* Per-row energy contributions e_r = -1/4 sum_{l} sum_{i in row atom} D_li K_il,
 * D_li taken from the block D(E,A,-n) (the transpose partner of D(A,E,n));
 * returns the sum over the selected rows. */
double orc_energy(void *h, const double *K, double *per_row) {
    orc *o = (orc *)h;
    double tot = 0;
    for (int r = 0; r < o->nrows; r++) {
        int a = o->rows[r];
        int nbA = NB(o, a);
        double e = 0;
        for (int64_t p = o->rowptr[a]; p < o->rowptr[a + 1]; p++) {
            int64_t q = o->partner[p];
            if (!o->keepD[q]) continue;
            int b = o->pB[p]; const int32_t *n = o->pn + 3 * p;
            int nbB = NB(o, b);
            int64_t x = kfind(o, o->krow[r], o->krow[r + 1], pair_key(a, b, n[0], n[1], n[2]));
            if (x < 0) continue;  /* sampled mode: block not listed */
            const double *kb = K + o->offK[x];
            const double *dq = o->D + o->offD[q];   /* D(B,A,-n) [l][i] */
            for (int i = 0; i < nbA; i++)
                for (int l = 0; l < nbB; l++) e += dq[l * nbA + i] * kb[i * nbB + l];
        }
        e *= -0.25;
        if (per_row) per_row[r] = e;
        tot += e;
    }
    return tot;
}

void orc_destroy(void *h) {
    orc *o = (orc *)h;
    if (!o) return;
    free(o->xyz); free(o->sp); free(o->nbs); free(o->nas);
    free(o->pA); free(o->pB); free(o->pn); free(o->onsite); free(o->partner); free(o->rowptr);
    free(o->offC); free(o->offV); free(o->offD); hm_free(&o->pairs);
    free(o->keepC); free(o->keepV); free(o->keepD);
    free(o->rows); free(o->kkeys); free(o->offK); free(o->krow);
    free(o);
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the OpenMP loops over rows (n <= 0: every processor); the
 * arithmetic of each row does not depend on it. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}
