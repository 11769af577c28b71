/*
 * Fast fill of the synthetic C and V blocks (input generation only; no part of
 * the exchange computation).  Same definitions as rix_inputs.rng / blocks:
 *
 *   normal(seed, stream, c): SplitMix64 of (seed*K1 + stream*K2 + 2c) and of
 *   (... + 2c + 1) give two 53-bit uniforms u1, u2; N = sqrt(-2 ln(1-u1)) cos(2 pi u2).
 *   C block of a representative pair p: element e = normal(counter = offC[p] + e)
 *   times exp(-0.8 r_p); on-site blocks symmetrised from the upper triangle;
 *   the transpose partner gets the transposed block with its aux blocks swapped.
 *   V block: short-range Coulomb of two s-Gaussians, series below R < 1e-3 g1.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ull, M1 = 0xBF58476D1CE4E5B9ull, M2 = 0x94D049BB133111EBull;
static const uint64_t KSEED = 0xD1B54A32D192ED03ull, KSTREAM = 0x8CB92BA72F3D8DD7ull;

static inline uint64_t splitmix(uint64_t x) {
    uint64_t z = x + GOLDEN;
    z = (z ^ (z >> 30)) * M1;
    z = (z ^ (z >> 27)) * M2;
    return z ^ (z >> 31);
}
static inline double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

static inline double normal_at(uint64_t base, uint64_t c) {
    const double u1 = 1.0 - u01(splitmix(base + 2 * c));
    const double u2 = u01(splitmix(base + 2 * c + 1));
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

/* C for every pair; rep[p] marks representatives (the others are mirrored). */
void fill_C(int64_t np, const int64_t *offC, const uint8_t *rep, const uint8_t *onsite, const int64_t *partner,
            const int32_t *naA, const int32_t *naB, const int32_t *nbA, const int32_t *nbB, const double *dist,
            uint64_t seed, uint64_t stream, double *C) {
    const uint64_t base = seed * KSEED + stream * KSTREAM;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < np; p++) {
        if (!rep[p]) continue;
        const int na = naA[p], nb = naB[p], ia = nbA[p], jb = nbB[p];
        const int rows = na + (onsite[p] ? 0 : nb);
        const int64_t size = (int64_t)rows * ia * jb;
        const double amp = exp(-0.8 * dist[p]);
        double *blk = C + offC[p];
        for (int64_t e = 0; e < size; e++) blk[e] = normal_at(base, (uint64_t)(offC[p] + e)) * amp;
        if (onsite[p]) {
            for (int P = 0; P < rows; P++)
                for (int i = 0; i < ia; i++)
                    for (int j = 0; j < i; j++)
                        blk[((int64_t)P * ia + i) * jb + j] = blk[((int64_t)P * ia + j) * jb + i];
        } else {
            double *q = C + offC[partner[p]];
            for (int P = 0; P < rows; P++) {
                const int Pq = P < na ? P + nb : P - na;
                for (int i = 0; i < ia; i++)
                    for (int j = 0; j < jb; j++)
                        q[((int64_t)Pq * jb + j) * ia + i] = blk[((int64_t)P * ia + i) * jb + j];
            }
        }
    }
}

/* V for every representative pair and its transpose partner. sig* point at the
 * aux widths of the two atoms of pair p (sigoff[p], sigoffB[p] into sig). */
void fill_V(int64_t np, const int64_t *offV, const uint8_t *rep, const int64_t *partner, const int32_t *naA,
            const int32_t *naB, const int64_t *sigA, const int64_t *sigB, const double *sig, const double *dist,
            double omega, double *V) {
    const double two_sqrt_pi = 1.1283791670955126;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < np; p++) {
        if (!rep[p]) continue;
        const int na = naA[p], nb = naB[p];
        const double R = dist[p];
        double *v = V + offV[p];
        double *vq = V + offV[partner[p]];
        for (int P = 0; P < na; P++)
            for (int Q = 0; Q < nb; Q++) {
                const double sP = sig[sigA[p] + P], sQ = sig[sigB[p] + Q];
                const double g1 = sqrt(2.0 * (sP * sP + sQ * sQ));
                double x;
                if (omega > 0) {
                    const double g2 = sqrt(g1 * g1 + 1.0 / (omega * omega));
                    if (R < 1e-3 * g1)
                        x = two_sqrt_pi * ((1.0 / g1 - 1.0 / g2) - (R * R / 3.0) * (1.0 / (g1 * g1 * g1) - 1.0 / (g2 * g2 * g2)));
                    else
                        x = (erf(R / g1) - erf(R / g2)) / R;
                } else {  /* full range (PBE0): the omega -> 0 limit, plain Coulomb of two Gaussians */
                    if (R < 1e-3 * g1)
                        x = two_sqrt_pi * ((1.0 / g1) - (R * R / 3.0) * (1.0 / (g1 * g1 * g1)));
                    else
                        x = erf(R / g1) / R;
                }
                v[(int64_t)P * nb + Q] = x;
                vq[(int64_t)Q * na + P] = x;
            }
    }
}
