/*
 * Plain FP64 CPU oracle for the FMG-MLMC method of Liu, Li, Sun & Yu,
 * "A full multigrid multilevel (quasi-) Monte Carlo method for the
 * single-phase subsurface flow with random coefficients" (arXiv 1910.04727).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * Everything here is written to be checked against the paper by eye:
 * one sample at a time, cell by cell, in the order the method states it.
 *
 *   - Philox4x64-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), used for the
 *     MC points, the Sobol' initial direction numbers and the digital shifts.
 *   - Inverse standard-normal CDF by bisection then Newton on
 *     Phi(x) = erfc(-x/sqrt2)/2.
 *   - Sobol' points (Bratley & Fox construction: primitive polynomials over
 *     GF(2), direction-number recurrence), Gray-code index, digital shift
 *     (the randomized QMC of Sec. 2.4).
 *   - Cell-centred finite volumes for -div(k grad u) = 0 (Eq. 1) on the
 *     unit square, both cases of Table 1.  Case II: Dirichlet u=pW on the
 *     west edge, u=pE on the east edge, zero flux on north and south; QoI =
 *     outflux through the east edge.  Case I: Dirichlet data on all four
 *     edges (pW, pE, pS, pN); QoI = u(0.5, 0.5), the mean of the four cells
 *     that meet at the centre.
 *   - Red-black Gauss-Seidel V(nu1,nu2) cycles, full multigrid over the
 *     same grid hierarchy as the MLMC levels (Sec. 2.5), coefficient
 *     coarsening by injection k^c_{I,J} = k^f_{2I-1,2J-1} (Sec. 2.5, written
 *     0-indexed as [2I][2J]), exact solve on the 4x4 grid, and the coarse
 *     QoI Q^c taken from the FMG stage one grid below the finest (Sec. 2.5,
 *     Algorithm 3).
 *
 * Grid layout: an n x n grid is stored row-major with x fastest,
 * a[j*n + i] for cell (i, j), i = 0 at the west edge, j = 0 at the south edge.
 * All cells are squares, so a face transmissibility does not depend on h.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (SC'11): 10 rounds of the Philox S-box on a 4x64-bit counter */
/* with a 2x64-bit key bumped by the Weyl constants between rounds.          */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        unsigned __int128 prod0 = (unsigned __int128)PHILOX_M0 * c0;
        unsigned __int128 prod1 = (unsigned __int128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(prod0 >> 64), lo0 = (uint64_t)prod0;
        uint64_t hi1 = (uint64_t)(prod1 >> 64), lo1 = (uint64_t)prod1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream purposes: the high 32 bits of key[1]. */
#define OR_PURPOSE_MC 1u
#define OR_PURPOSE_SHIFT 2u
#define OR_PURPOSE_SOBOL_DIR 3u
#define OR_SOBOL_DIR_SEED 0x1910047270ULL

/* Word `w` of the stream (key0, key1): counter (w/4, index, 0, 0), lane w%4. */
uint64_t or_philox_word(uint64_t key0, uint64_t key1, uint64_t index, uint64_t w)
{
    uint64_t ctr[4] = {w / 4, index, 0, 0};
    uint64_t key[2] = {key0, key1};
    uint64_t out[4];
    or_philox4x64_10(ctr, key, out);
    return out[w % 4];
}

/* ------------------------------------------------------------------------ */
/* Inverse normal CDF.  Phi(x) = erfc(-x/sqrt(2))/2.  For u < 1/2 bracket   */
/* the root of Phi(x) = u on [-40, 0] by bisection, then polish by Newton    */
/* steps x <- x - (Phi(x) - u)/phi(x).  For u > 1/2 use the symmetry         */
/* Phi^{-1}(u) = -Phi^{-1}(1 - u), where 1 - u is exact for u in [1/2, 1).    */
/* ------------------------------------------------------------------------ */
static double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }
static double std_normal_pdf(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * M_PI); }

static double norminv_lower(double u) /* 0 < u <= 1/2 */
{
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (std_normal_cdf(mid) < u) lo = mid; else hi = mid;
        if (hi - lo <= 1e-6 * fabs(hi)) break;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 8; ++it) {
        double step = (std_normal_cdf(x) - u) / std_normal_pdf(x);
        double xn = x - step;
        if (xn == x) break;
        x = xn;
    }
    return x;
}

double or_norminv(double u)
{
    if (u <= 0.0) return -INFINITY;
    if (u >= 1.0) return INFINITY;
    if (u == 0.5) return 0.0;
    if (u < 0.5) return norminv_lower(u);
    return -norminv_lower(1.0 - u);
}

/* MC points (Sec. 2.3): xi[s*dim + k] = Phi^{-1}(u), u = ((w >> 11) + 1/2) 2^-53,
 * w = word k of the stream (seed, MC<<32 | level) at sample index first + s.  */
void or_mc_normals(uint64_t seed, uint32_t level, uint64_t first, uint32_t n,
                   uint32_t dim, double* xi)
{
    uint64_t key1 = ((uint64_t)OR_PURPOSE_MC << 32) | level;
    for (uint32_t s = 0; s < n; ++s)
        for (uint32_t k = 0; k < dim; ++k) {
            uint64_t w = or_philox_word(seed, key1, first + s, k);
            double u = ((double)(w >> 11) + 0.5) * 0x1p-53;
            xi[(size_t)s * dim + k] = or_norminv(u);
        }
}

/* The 64-bit words behind or_mc_normals: w[s*dim + k] = word k of the
 * stream (seed, MC<<32 | level) at sample index first + s. */
void or_mc_words(uint64_t seed, uint32_t level, uint64_t first, uint32_t n, uint32_t dim, uint64_t* w)
{
    uint64_t key1 = ((uint64_t)OR_PURPOSE_MC << 32) | level;
    for (uint32_t s = 0; s < n; ++s)
        for (uint32_t k = 0; k < dim; ++k)
            w[(size_t)s * dim + k] = or_philox_word(seed, key1, first + s, k);
}

/* ------------------------------------------------------------------------ */
/* Sobol' points (Sec. 2.4, Sobol' sequence; Bratley & Fox, ACM TOMS 1988).  */
/* ------------------------------------------------------------------------ */

/* Polynomials over GF(2) as bit masks: bit d is the coefficient of x^d. */
static uint64_t gf2_mulmod(uint64_t a, uint64_t b, uint64_t p, int deg)
{
    uint64_t r = 0;
    while (b) {
        if (b & 1) r ^= a;
        b >>= 1;
        a <<= 1;
        if (a & (1ULL << deg)) a ^= p;
    }
    return r;
}

static uint64_t gf2_powmod_x(uint64_t e, uint64_t p, int deg)
{
    uint64_t base = 2; /* the polynomial x, reduced mod p */
    if (base >> deg & 1) base ^= p;
    uint64_t result = 1;
    while (e) {
        if (e & 1) result = gf2_mulmod(result, base, p, deg);
        base = gf2_mulmod(base, base, p, deg);
        e >>= 1;
    }
    return result;
}

/* p (degree deg, constant term 1) is primitive iff x has multiplicative
 * order exactly 2^deg - 1 modulo p: x^(2^deg-1) = 1 and x^((2^deg-1)/q) != 1
 * for every prime q dividing 2^deg - 1. */
int or_gf2_is_primitive(uint64_t p, int deg)
{
    if (!(p & 1) || !(p >> deg & 1)) return 0;
    uint64_t order = (1ULL << deg) - 1;
    if (gf2_powmod_x(order, p, deg) != 1) return 0;
    uint64_t m = order;
    for (uint64_t q = 2; q * q <= m; ++q) {
        if (m % q) continue;
        if (gf2_powmod_x(order / q, p, deg) == 1) return 0;
        while (m % q == 0) m /= q;
    }
    if (m > 1 && gf2_powmod_x(order / m, p, deg) == 1) return 0;
    return 1;
}

/* The first `count` primitive polynomials in ascending degree, ascending
 * bit-mask order within a degree.  Returns how many were written. */
int or_primitive_polys(int count, uint64_t* polys, int* degrees)
{
    int found = 0;
    for (int deg = 1; deg <= 31 && found < count; ++deg)
        for (uint64_t p = (1ULL << deg) | 1; p < (1ULL << (deg + 1)) && found < count; p += 2)
            if (or_gf2_is_primitive(p, deg)) {
                polys[found] = p;
                degrees[found] = deg;
                ++found;
            }
    return found;
}

/* Direction numbers V[d*32 + (k-1)] = m_k 2^(32-k), k = 1..32.
 * Dimension 0 is van der Corput (m_k = 1).  Dimension d >= 1 uses the d-th
 * primitive polynomial x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1; its initial
 * m_1..m_s are odd, m_k < 2^k, drawn as m_k = 2 (w mod 2^(k-1)) + 1 from the
 * Philox stream (SOBOL_DIR_SEED, SOBOL_DIR<<32), index d, word k-1; beyond
 * that  m_k = m_(k-s) ^ 2^s m_(k-s) ^ XOR_{i=1}^{s-1} 2^i a_i m_(k-i).     */
int or_sobol_direction_numbers(uint32_t dim, uint32_t* V)
{
    uint64_t* polys = (uint64_t*)malloc(sizeof(uint64_t) * (dim + 1));
    int* degs = (int*)malloc(sizeof(int) * (dim + 1));
    int have = or_primitive_polys((int)dim, polys, degs);
    if (dim > 1 && have < (int)dim - 1) { free(polys); free(degs); return -1; }
    uint64_t key1 = (uint64_t)OR_PURPOSE_SOBOL_DIR << 32;
    for (uint32_t d = 0; d < dim; ++d) {
        uint64_t m[33];
        if (d == 0) {
            for (int k = 1; k <= 32; ++k) m[k] = 1;
        } else {
            uint64_t p = polys[d - 1];
            int s = degs[d - 1];
            for (int k = 1; k <= s && k <= 32; ++k) {
                uint64_t w = or_philox_word(OR_SOBOL_DIR_SEED, key1, d, (uint64_t)(k - 1));
                m[k] = 2 * (w % (1ULL << (k - 1))) + 1;
            }
            for (int k = s + 1; k <= 32; ++k) {
                uint64_t v = m[k - s] ^ (m[k - s] << s);
                for (int i = 1; i < s; ++i) {
                    int a_i = (int)((p >> (s - i)) & 1);
                    if (a_i) v ^= m[k - i] << i;
                }
                m[k] = v;
            }
        }
        for (int k = 1; k <= 32; ++k) V[d * 32 + (k - 1)] = (uint32_t)(m[k] << (32 - k));
    }
    free(polys);
    free(degs);
    return 0;
}

/* Digital shift words: shift[r*dim + d] = high 32 bits of word d of the
 * Philox stream (seed, SHIFT<<32 | level) at index r.                       */
void or_sobol_shifts(uint64_t seed, uint32_t level, uint32_t n_shifts, uint32_t dim,
                     uint32_t* shift)
{
    uint64_t key1 = ((uint64_t)OR_PURPOSE_SHIFT << 32) | level;
    for (uint32_t r = 0; r < n_shifts; ++r)
        for (uint32_t d = 0; d < dim; ++d)
            shift[(size_t)r * dim + d] = (uint32_t)(or_philox_word(seed, key1, r, d) >> 32);
}

/* Point n in Gray-code order: x_d = XOR over set bits b of gray(n) of
 * V[d][b], then XOR the digital shift.  out[(r*n + s)*dim + d]; xi the same
 * layout with u = (x + 1/2) 2^-32 mapped through Phi^{-1} (nullable).       */
void or_sobol_points(const uint32_t* V, uint32_t dim, uint64_t first, uint32_t n,
                     uint32_t n_shifts, const uint32_t* shift, uint32_t* out, double* xi)
{
    for (uint32_t r = 0; r < n_shifts; ++r)
        for (uint32_t s = 0; s < n; ++s) {
            uint64_t idx = first + s;
            uint64_t gray = idx ^ (idx >> 1);
            for (uint32_t d = 0; d < dim; ++d) {
                uint32_t x = 0;
                for (int b = 0; b < 32; ++b)
                    if ((gray >> b) & 1) x ^= V[d * 32 + b];
                if (shift) x ^= shift[(size_t)r * dim + d];
                size_t o = ((size_t)r * n + s) * dim + d;
                if (out) out[o] = x;
                if (xi) xi[o] = or_norminv(((double)x + 0.5) * 0x1p-32);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Randomized QMC rules (Sec. 2.4: random shift of a lattice rule, scramble   */
/* of the Sobol' sequence).                                                  */
/* ------------------------------------------------------------------------ */
#define OR_PURPOSE_LATTICE_SHIFT 4u
#define OR_PURPOSE_OWEN 5u

/* omega(x) = B_2(x) = x^2 - x + 1/6, the shift-invariant kernel of the
 * unanchored Sobolev space of first-order mixed smoothness. */
static double bernoulli2(double x) { return x * x - x + 1.0 / 6.0; }

/* Rank-1 lattice generating vector for the embedded point sets of 2^m
 * points, m = m_min .. m_max, component by component: z_1 = 1; component s
 * is the odd z < 2^(m_max - 1) minimising
 *   C(z) = sum_m e^2_m(z_1..z_(s-1), z) / e^2_m(z_1..z_(s-1)),
 * with the shift-averaged squared worst-case error of the 2^m-point lattice
 * e^2_m = -1 + 2^-m sum_k prod_j (1 + gamma_j omega({k z_j / 2^m})) and
 * product weights gamma_j = 1 / j^2.  With P_m = sum_k p_k and
 * E_m(z) = sum_k p_k omega({k z / 2^m}), p_k the product over the chosen
 * components, e^2_m(z) = -1 + (P_m + gamma_s E_m(z)) / 2^m.  Sums run over
 * k in increasing order; ties go to the smaller z (z and 2^m - z give the
 * same lattice).  Plain O(dim 2^(2 m_max)) evaluation. */
int or_lattice_cbc(uint32_t dim, int m_min, int m_max, uint32_t* z)
{
    if (m_min < 1 || m_max < m_min || m_max > 24 || dim < 1) return -1;
    int nm = m_max - m_min + 1;
    double** p = (double**)calloc((size_t)nm, sizeof(double*));
    double* e2 = (double*)calloc((size_t)nm, sizeof(double));
    double* P = (double*)calloc((size_t)nm, sizeof(double));
    for (int a = 0; a < nm; ++a) {
        uint32_t n = 1u << (m_min + a);
        p[a] = (double*)malloc(sizeof(double) * n);
        double sum = 0.0;
        for (uint32_t k = 0; k < n; ++k) {
            p[a][k] = 1.0 + 1.0 * bernoulli2((double)k / n);   /* z_1 = 1, gamma_1 = 1 */
            sum += p[a][k];
        }
        e2[a] = -1.0 + sum / n;
    }
    z[0] = 1;
    uint32_t half = 1u << (m_max - 1);
    for (uint32_t s = 1; s < dim; ++s) {
        double gamma = 1.0 / ((double)(s + 1) * (s + 1));
        for (int a = 0; a < nm; ++a) {
            uint32_t n = 1u << (m_min + a);
            double sum = 0.0;
            for (uint32_t k = 0; k < n; ++k) sum += p[a][k];
            P[a] = sum;
        }
        uint32_t best = 1;
        double bestC = INFINITY;
        for (uint32_t c = 1; c < half; c += 2) {
            double C = 0.0;
            for (int a = 0; a < nm; ++a) {
                uint32_t n = 1u << (m_min + a);
                double E = 0.0;
                for (uint32_t k = 0; k < n; ++k)
                    E += p[a][k] * bernoulli2((double)(((uint64_t)k * c) & (n - 1)) / n);
                C += (-1.0 + (P[a] + gamma * E) / n) / e2[a];
            }
            if (C < bestC) { bestC = C; best = c; }
        }
        z[s] = best;
        for (int a = 0; a < nm; ++a) {
            uint32_t n = 1u << (m_min + a);
            double sum = 0.0;
            for (uint32_t k = 0; k < n; ++k) {
                p[a][k] *= 1.0 + gamma * bernoulli2((double)(((uint64_t)k * best) & (n - 1)) / n);
                sum += p[a][k];
            }
            e2[a] = -1.0 + sum / n;
        }
    }
    for (int a = 0; a < nm; ++a) free(p[a]);
    free(p); free(e2); free(P);
    return 0;
}

/* Shift-averaged squared worst-case error e^2 of the 2^m-point lattice with
 * generating vector z (the quantity the construction above works with). */
double or_lattice_e2(const uint32_t* z, uint32_t dim, int m)
{
    uint32_t n = 1u << m;
    double sum = 0.0;
    for (uint32_t k = 0; k < n; ++k) {
        double prod = 1.0;
        for (uint32_t j = 0; j < dim; ++j)
            prod *= 1.0 + bernoulli2((double)(((uint64_t)k * z[j]) & (n - 1)) / n) / ((double)(j + 1) * (j + 1));
        sum += prod;
    }
    return -1.0 + sum / n;
}

/* Points of the randomly shifted lattice sequence, 32-bit fixed point:
 * point index i is taken in radical-inverse order (its m_max low bits
 * reversed), so the first 2^m points are the 2^m-point lattice, and
 * x[r][s][d] = (z_d phi(i) 2^(32 - m_max) + Delta_(r,d)) mod 2^32 with the
 * shift Delta = the high 32 bits of word d of the Philox stream
 * (seed, LATTICE_SHIFT << 32 | level) at index r.  u = (x + 1/2) 2^-32. */
void or_lattice_points(const uint32_t* z, uint32_t dim, int m_max, uint64_t seed, uint32_t level,
                       uint64_t first, uint32_t n, uint32_t first_shift, uint32_t n_shifts, uint32_t* x)
{
    uint64_t key1 = ((uint64_t)OR_PURPOSE_LATTICE_SHIFT << 32) | level;
    for (uint32_t r = 0; r < n_shifts; ++r)
        for (uint32_t s = 0; s < n; ++s) {
            uint64_t i = first + s;
            uint32_t rev = 0;
            for (int b = 0; b < m_max; ++b)
                if ((i >> b) & 1) rev |= 1u << (m_max - 1 - b);
            for (uint32_t d = 0; d < dim; ++d) {
                uint32_t delta = (uint32_t)(or_philox_word(seed, key1, first_shift + r, d) >> 32);
                uint32_t t = (uint32_t)((uint64_t)z[d] * rev) & ((m_max == 32) ? 0xFFFFFFFFu : ((1u << m_max) - 1));
                x[((size_t)r * n + s) * dim + d] = (t << (32 - m_max)) + delta;
            }
        }
}

/* Nested uniform scrambling (Owen 1995) of a 32-bit coordinate: output bit
 * b (b = 0 the most significant) is input bit b XOR a random bit that
 * depends on the scramble r, the dimension d, b and the input's b leading
 * bits.  The random bit of that tree node is the low bit of word 0 of
 * Philox4x64-10 with key (seed, OWEN << 32 | level) at counter
 * (prefix, r << 32 | d, b, 0). */
uint32_t or_owen_scramble(uint64_t seed, uint32_t level, uint32_t r, uint32_t d, uint32_t x)
{
    uint64_t key[2] = {seed, ((uint64_t)OR_PURPOSE_OWEN << 32) | level};
    uint32_t y = 0;
    for (int b = 0; b < 32; ++b) {
        uint64_t prefix = b == 0 ? 0 : (uint64_t)(x >> (32 - b));
        uint64_t ctr[4] = {prefix, ((uint64_t)r << 32) | d, (uint64_t)b, 0};
        uint64_t out[4];
        or_philox4x64_10(ctr, key, out);
        uint32_t bit = ((x >> (31 - b)) & 1u) ^ (uint32_t)(out[0] & 1u);
        y |= bit << (31 - b);
    }
    return y;
}

/* Owen-scrambled Sobol' points: the plain Gray-code point (no digital
 * shift), then the nested scramble of scramble r = first_shift + r'. */
void or_sobol_owen_points(const uint32_t* V, uint32_t dim, uint64_t seed, uint32_t level, uint64_t first,
                          uint32_t n, uint32_t first_shift, uint32_t n_shifts, uint32_t* x)
{
    for (uint32_t r = 0; r < n_shifts; ++r)
        for (uint32_t s = 0; s < n; ++s) {
            uint64_t idx = first + s, gray = idx ^ (idx >> 1);
            for (uint32_t d = 0; d < dim; ++d) {
                uint32_t v = 0;
                for (int b = 0; b < 32; ++b)
                    if ((gray >> b) & 1) v ^= V[(size_t)d * 32 + b];
                x[((size_t)r * n + s) * dim + d] = or_owen_scramble(seed, level, first_shift + r, d, v);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Finite volumes, Eq. 1 / Table 1.                                          */
/* Interior face: harmonic mean 2 k_a k_b / (k_a + k_b) (unit face over unit */
/* centre distance on square cells).  Dirichlet boundary face: the centre is */
/* h/2 from the face, T = 2 k.  West/east faces are Dirichlet in both cases; */
/* north/south are no-flow (T = 0) in Case II and Dirichlet in Case I (the   */
/* flag `ns` below).                                                         */
/* Cell equation: sum_faces T (u_c - u_other) = 0, u_other = boundary value   */
/* on a Dirichlet face.                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double pW, pE;   /* Dirichlet values on the west and east edges */
    int nu0;         /* V-cycles per FMG stage (fixed mode) */
    int nu1, nu2;    /* pre- and post-smoothing RB-GS sweeps */
    int converged;   /* 1: V-cycles at each stage until ||r||/||b|| <= tol */
    double tol;
    int max_cycles;
    int coarse_op;   /* coefficients of the V-cycle's coarse-grid correction
                        operators: 0 the injected field itself, 1 the geometric
                        mean of the four children of the injected field one
                        grid finer */
    int energy_step; /* 1: scale each prolongated correction d by the step
                        (r, d) / (d, A d) that minimises the energy error
                        along d (r the residual it corrects) */
    int bc_case;     /* Table 1: 2 (default) Case II, 1 Case I */
    double pS, pN;   /* Case I: Dirichlet values on the south and north edges */
} or_params;

/* Boundary data of one problem: g[0..3] = west, east, south, north values,
 * ns = 1 when the north and south edges are Dirichlet (Case I). */
typedef struct {
    double g[4];
    int ns;
} or_bc;

static or_bc bc_of(const or_params* P)
{
    or_bc b;
    b.g[0] = P->pW;
    b.g[1] = P->pE;
    b.ns = (P->bc_case == 1);
    b.g[2] = b.ns ? P->pS : 0.0;
    b.g[3] = b.ns ? P->pN : 0.0;
    return b;
}

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

static void cell_faces(int n, const double* K, int ns, int i, int j,
                       double* tw, double* te, double* ts, double* tn)
{
    double k = K[j * n + i];
    double tb = ns ? 2.0 * k : 0.0; /* north / south boundary face */
    *tw = (i > 0) ? harmonic(K[j * n + i - 1], k) : 2.0 * k;
    *te = (i < n - 1) ? harmonic(k, K[j * n + i + 1]) : 2.0 * k;
    *ts = (j > 0) ? harmonic(K[(j - 1) * n + i], k) : tb;
    *tn = (j < n - 1) ? harmonic(k, K[(j + 1) * n + i]) : tb;
}

/* y = A x (boundary values enter the rhs, not A). */
void or_apply_A_bc(int n, const double* K, int ns, const double* x, double* y)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double tw, te, ts, tn;
            cell_faces(n, K, ns, i, j, &tw, &te, &ts, &tn);
            double v = (tw + te + ts + tn) * x[j * n + i];
            if (i > 0) v -= tw * x[j * n + i - 1];
            if (i < n - 1) v -= te * x[j * n + i + 1];
            if (j > 0) v -= ts * x[(j - 1) * n + i];
            if (j < n - 1) v -= tn * x[(j + 1) * n + i];
            y[j * n + i] = v;
        }
}

void or_apply_A(int n, const double* K, const double* x, double* y) { or_apply_A_bc(n, K, 0, x, y); }

/* rhs of the stage problem: the Dirichlet data moved to the right side,
 * T g on every Dirichlet boundary face. */
void or_stage_rhs_bc(int n, const double* K, const double* g, int ns, double* b)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double k = K[j * n + i];
            double v = 0.0;
            if (i == 0) v += 2.0 * k * g[0];
            if (i == n - 1) v += 2.0 * k * g[1];
            if (ns && j == 0) v += 2.0 * k * g[2];
            if (ns && j == n - 1) v += 2.0 * k * g[3];
            b[j * n + i] = v;
        }
}

void or_stage_rhs(int n, const double* K, double pW, double pE, double* b)
{
    double g[4] = {pW, pE, 0.0, 0.0};
    or_stage_rhs_bc(n, K, g, 0, b);
}

/* One red-black Gauss-Seidel sweep: red cells ((i+j) even) then black. */
void or_rbgs_sweep_bc(int n, const double* K, int ns, const double* b, double* x)
{
    for (int color = 0; color < 2; ++color)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                if (((i + j) & 1) != color) continue;
                double tw, te, ts, tn;
                cell_faces(n, K, ns, i, j, &tw, &te, &ts, &tn);
                double s = b[j * n + i];
                if (i > 0) s += tw * x[j * n + i - 1];
                if (i < n - 1) s += te * x[j * n + i + 1];
                if (j > 0) s += ts * x[(j - 1) * n + i];
                if (j < n - 1) s += tn * x[(j + 1) * n + i];
                x[j * n + i] = s / (tw + te + ts + tn);
            }
}

void or_rbgs_sweep(int n, const double* K, const double* b, double* x) { or_rbgs_sweep_bc(n, K, 0, b, x); }

/* r = b - A x */
void or_residual_bc(int n, const double* K, int ns, const double* b, const double* x, double* r)
{
    or_apply_A_bc(n, K, ns, x, r);
    for (int c = 0; c < n * n; ++c) r[c] = b[c] - r[c];
}

void or_residual(int n, const double* K, const double* b, const double* x, double* r)
{
    or_residual_bc(n, K, 0, b, x, r);
}

/* Coarse rhs = sum of the four fine residuals of each coarse cell. */
void or_restrict_sum(int nc, const double* rf, double* bc)
{
    int nf = 2 * nc;
    for (int J = 0; J < nc; ++J)
        for (int I = 0; I < nc; ++I)
            bc[J * nc + I] = rf[(2 * J) * nf + 2 * I] + rf[(2 * J) * nf + 2 * I + 1] +
                             rf[(2 * J + 1) * nf + 2 * I] + rf[(2 * J + 1) * nf + 2 * I + 1];
}

/* Coarse value with ghost cells.  A Dirichlet face with value g on it
 * extrapolates 2 g - u from the edge cell (west / east always, north /
 * south in Case I); a no-flow face mirrors the edge cell (north / south in
 * Case II).  A ghost in a corner takes the x rule on the y ghost. */
static double coarse_value(int nc, const double* uc, int I, int J, const double* g, int ns)
{
    if (J < 0 || J > nc - 1) {
        int Je = J < 0 ? 0 : nc - 1;
        double ge = J < 0 ? g[2] : g[3];
        double edge = coarse_value(nc, uc, I, Je, g, ns);
        return ns ? 2.0 * ge - edge : edge;
    }
    if (I < 0) return 2.0 * g[0] - uc[J * nc + 0];
    if (I > nc - 1) return 2.0 * g[1] - uc[J * nc + nc - 1];
    return uc[J * nc + I];
}

/* Bilinear cell-centred interpolation: 9/16 parent, 3/16 each of the two
 * nearest coarse neighbours in x and y, 1/16 the diagonal one.             */
static double bilinear(int nc, const double* uc, int i, int j, const double* g, int ns)
{
    int I = i / 2, J = j / 2;
    int Ix = (i & 1) ? I + 1 : I - 1;
    int Jy = (j & 1) ? J + 1 : J - 1;
    return (9.0 * coarse_value(nc, uc, I, J, g, ns) + 3.0 * coarse_value(nc, uc, Ix, J, g, ns) +
            3.0 * coarse_value(nc, uc, I, Jy, g, ns) + 1.0 * coarse_value(nc, uc, Ix, Jy, g, ns)) /
           16.0;
}

/* x_f += P e_c (the error vanishes on the Dirichlet faces). */
void or_prolong_add_bc(int nc, const double* ec, int ns, double* xf)
{
    static const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    int nf = 2 * nc;
    for (int j = 0; j < nf; ++j)
        for (int i = 0; i < nf; ++i) xf[j * nf + i] += bilinear(nc, ec, i, j, zero, ns);
}

void or_prolong_add(int nc, const double* ec, double* xf) { or_prolong_add_bc(nc, ec, 0, xf); }

/* FMG start of a stage: x_f = P u_c with the Dirichlet data as ghosts. */
void or_fmg_interpolate_bc(int nc, const double* uc, const double* g, int ns, double* xf)
{
    int nf = 2 * nc;
    for (int j = 0; j < nf; ++j)
        for (int i = 0; i < nf; ++i) xf[j * nf + i] = bilinear(nc, uc, i, j, g, ns);
}

void or_fmg_interpolate(int nc, const double* uc, double pW, double pE, double* xf)
{
    double g[4] = {pW, pE, 0.0, 0.0};
    or_fmg_interpolate_bc(nc, uc, g, 0, xf);
}

/* Coefficient coarsening by injection: K_c[J][I] = K_f[2J][2I]. */
void or_inject(int nc, const double* Kf, double* Kc)
{
    int nf = 2 * nc;
    for (int J = 0; J < nc; ++J)
        for (int I = 0; I < nc; ++I) Kc[J * nc + I] = Kf[(2 * J) * nf + 2 * I];
}

/* Exact solve on a small grid: assemble the dense SPD matrix and factor it
 * by Cholesky, A = L L^T, then two triangular solves. */
void or_exact_solve_bc(int n, const double* K, int ns, const double* b, double* x)
{
    int m = n * n;
    double* A = (double*)calloc((size_t)m * m, sizeof(double));
    double* e = (double*)calloc((size_t)m, sizeof(double));
    double* col = (double*)calloc((size_t)m, sizeof(double));
    for (int c = 0; c < m; ++c) { /* column c of A is A e_c */
        e[c] = 1.0;
        or_apply_A_bc(n, K, ns, e, col);
        for (int r = 0; r < m; ++r) A[r * m + c] = col[r];
        e[c] = 0.0;
    }
    for (int c = 0; c < m; ++c) { /* in-place Cholesky, lower triangle */
        double d = A[c * m + c];
        for (int k = 0; k < c; ++k) d -= A[c * m + k] * A[c * m + k];
        d = sqrt(d);
        A[c * m + c] = d;
        for (int r = c + 1; r < m; ++r) {
            double v = A[r * m + c];
            for (int k = 0; k < c; ++k) v -= A[r * m + k] * A[c * m + k];
            A[r * m + c] = v / d;
        }
    }
    for (int r = 0; r < m; ++r) { /* L y = b */
        double v = b[r];
        for (int k = 0; k < r; ++k) v -= A[r * m + k] * col[k];
        col[r] = v / A[r * m + r];
    }
    for (int r = m - 1; r >= 0; --r) { /* L^T x = y */
        double v = col[r];
        for (int k = r + 1; k < m; ++k) v -= A[k * m + r] * x[k];
        x[r] = v / A[r * m + r];
    }
    free(A);
    free(e);
    free(col);
}

void or_exact_solve(int n, const double* K, const double* b, double* x) { or_exact_solve_bc(n, K, 0, b, x); }

/* QoI of Case I: u(0.5, 0.5).  For even n the centre is the corner shared by
 * cells (n/2-1 .. n/2, n/2-1 .. n/2); bilinear interpolation from their
 * centres gives the mean of the four. */
double or_centre_value(int n, const double* x)
{
    int h = n / 2;
    return 0.25 * (x[(h - 1) * n + h - 1] + x[(h - 1) * n + h] + x[h * n + h - 1] + x[h * n + h]);
}

/* QoI of Case II: outflux through the east edge,
 * Q = sum_j 2 k_(n-1,j) (u_(n-1,j) - pE). */
double or_outflux(int n, const double* K, const double* x, double pE)
{
    double q = 0.0;
    for (int j = 0; j < n; ++j) q += 2.0 * K[j * n + n - 1] * (x[j * n + n - 1] - pE);
    return q;
}

/* Influx through the west edge (mass balance check). */
double or_influx(int n, const double* K, const double* x, double pW)
{
    double q = 0.0;
    for (int j = 0; j < n; ++j) q += 2.0 * K[j * n] * (pW - x[j * n]);
    return q;
}

double or_norm2(int m, const double* v)
{
    double s = 0.0;
    for (int c = 0; c < m; ++c) s += v[c] * v[c];
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Multigrid over the hierarchy n_k = n0 2^k, k = 0..m (n0 = coarsest).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int m;           /* finest index */
    int n0;          /* coarsest grid size */
    double* K[32];   /* injected coefficients per grid (the stage problems) */
    double* Kop[32]; /* coefficients of the correction operators below the top */
    double* Kavg[32];
    double* x[32];   /* iterate per grid */
    double* b[32];   /* rhs per grid */
    double* r[32];   /* residual work per grid */
    double* d[32];   /* prolongated correction and A d (energy step), 2 cells per cell */
    int energy_step;
    int ns;          /* north / south edges Dirichlet (Case I) */
} hierarchy;

static int grid_n(const hierarchy* H, int k) { return H->n0 << k; }

/* K_c[J][I] = (K_f[2J][2I] K_f[2J][2I+1] K_f[2J+1][2I] K_f[2J+1][2I+1])^(1/4) */
void or_geometric_children(int nc, const double* Kf, double* Kc)
{
    int nf = 2 * nc;
    for (int J = 0; J < nc; ++J)
        for (int I = 0; I < nc; ++I)
            Kc[J * nc + I] = exp(0.25 * (log(Kf[(2 * J) * nf + 2 * I]) + log(Kf[(2 * J) * nf + 2 * I + 1]) +
                                         log(Kf[(2 * J + 1) * nf + 2 * I]) + log(Kf[(2 * J + 1) * nf + 2 * I + 1])));
}

static void hierarchy_init(hierarchy* H, int n_fine, int n0, const double* K_fine, int coarse_op,
                           int energy_step, int ns)
{
    memset(H, 0, sizeof(*H));
    H->energy_step = energy_step;
    H->ns = ns;
    H->n0 = n0;
    int m = 0;
    while ((n0 << m) < n_fine) ++m;
    H->m = m;
    for (int k = 0; k <= m; ++k) {
        size_t cells = (size_t)grid_n(H, k) * grid_n(H, k);
        H->K[k] = (double*)malloc(sizeof(double) * cells);
        H->x[k] = (double*)calloc(cells, sizeof(double));
        H->b[k] = (double*)calloc(cells, sizeof(double));
        H->r[k] = (double*)calloc(cells, sizeof(double));
        if (energy_step) H->d[k] = (double*)calloc(2 * cells, sizeof(double));
    }
    memcpy(H->K[m], K_fine, sizeof(double) * (size_t)n_fine * n_fine);
    for (int k = m; k >= 1; --k) or_inject(grid_n(H, k - 1), H->K[k], H->K[k - 1]);
    for (int k = 0; k <= m; ++k) {
        H->Kop[k] = H->K[k];
        if (coarse_op == 1 && k < m) {
            H->Kavg[k] = (double*)malloc(sizeof(double) * (size_t)grid_n(H, k) * grid_n(H, k));
            or_geometric_children(grid_n(H, k), H->K[k + 1], H->Kavg[k]);
            H->Kop[k] = H->Kavg[k];
        }
    }
}

static void hierarchy_free(hierarchy* H)
{
    for (int k = 0; k <= H->m; ++k) {
        free(H->K[k]); free(H->x[k]); free(H->b[k]); free(H->r[k]); free(H->Kavg[k]); free(H->d[k]);
    }
}

/* One V(nu1, nu2) cycle for A_k x_k = b_k; grid `top` carries the stage
 * operator (injected K), the grids below it the correction operators. */
static void vcycle(hierarchy* H, int k, int top, int nu1, int nu2)
{
    int n = grid_n(H, k);
    const double* K = (k == top) ? H->K[k] : H->Kop[k];
    if (k == 0) {
        or_exact_solve_bc(n, K, H->ns, H->b[0], H->x[0]);
        return;
    }
    for (int s = 0; s < nu1; ++s) or_rbgs_sweep_bc(n, K, H->ns, H->b[k], H->x[k]);
    or_residual_bc(n, K, H->ns, H->b[k], H->x[k], H->r[k]);
    or_restrict_sum(n / 2, H->r[k], H->b[k - 1]);
    memset(H->x[k - 1], 0, sizeof(double) * (size_t)(n / 2) * (n / 2));
    vcycle(H, k - 1, top, nu1, nu2);
    if (!H->energy_step) {
        or_prolong_add_bc(n / 2, H->x[k - 1], H->ns, H->x[k]);
    } else {
        /* d = P e_c; x += alpha d with alpha = (r, d) / (d, A d), the exact
           line minimum of the energy error (A symmetric positive definite) */
        size_t cells = (size_t)n * n;
        double* d = H->d[k];
        double* Ad = d + cells;
        memset(d, 0, sizeof(double) * cells);
        or_prolong_add_bc(n / 2, H->x[k - 1], H->ns, d);
        or_apply_A_bc(n, K, H->ns, d, Ad);
        double rd = 0.0, dAd = 0.0;
        for (size_t c = 0; c < cells; ++c) {
            rd += H->r[k][c] * d[c];
            dAd += d[c] * Ad[c];
        }
        double alpha = dAd > 0.0 ? rd / dAd : 0.0;
        for (size_t c = 0; c < cells; ++c) H->x[k][c] += alpha * d[c];
    }
    for (int s = 0; s < nu2; ++s) or_rbgs_sweep_bc(n, K, H->ns, H->b[k], H->x[k]);
}

/* Relative residual ||b - A x|| / ||b|| on grid k. */
static double rel_residual(hierarchy* H, int k)
{
    int n = grid_n(H, k);
    or_residual_bc(n, H->K[k], H->ns, H->b[k], H->x[k], H->r[k]);
    double nb = or_norm2(n * n, H->b[k]);
    return or_norm2(n * n, H->r[k]) / (nb > 0 ? nb : 1.0);
}

/* Cycles for one FMG stage: nu0 V-cycles (fixed mode), or V-cycles until the
 * relative residual is <= tol (converged mode, the literal reading of "the
 * solutions are exact" at the end of each stage). Returns the cycles used. */
static int stage_cycles(hierarchy* H, int k, const or_params* P)
{
    if (!P->converged) {
        for (int it = 0; it < P->nu0; ++it) vcycle(H, k, k, P->nu1, P->nu2);
        return P->nu0;
    }
    int it = 0;
    while (it < P->max_cycles && rel_residual(H, k) > P->tol) {
        vcycle(H, k, k, P->nu1, P->nu2);
        ++it;
    }
    return it;
}

/* QoI of a stage solution: Case II the east outflux, Case I u(0.5, 0.5). */
static double stage_qoi(const or_bc* bc, int n, const double* K, const double* x)
{
    return bc->ns ? or_centre_value(n, x) : or_outflux(n, K, x, bc->g[1]);
}

/* Full multigrid for one sample: exact solve on the coarsest grid, then for
 * each finer grid interpolate the previous stage's solution and run the
 * stage's V-cycles.  Q^c is the outflux of the stage one below the finest
 * (the by-product of Algorithm 3), Q^f the outflux of the finest stage.
 * p_out (nullable) receives the finest solution.  qc is NaN when the finest
 * grid is the coarsest.  Returns total V-cycles. */
int or_fmg_solve(int n_fine, int n0, const double* K_fine, const or_params* P,
                 double* p_out, double* qf, double* qc)
{
    hierarchy H;
    or_bc bc = bc_of(P);
    hierarchy_init(&H, n_fine, n0, K_fine, P->coarse_op, P->energy_step, bc.ns);
    int cycles = 0;
    *qc = NAN;
    or_stage_rhs_bc(n0, H.K[0], bc.g, bc.ns, H.b[0]);
    or_exact_solve_bc(n0, H.K[0], bc.ns, H.b[0], H.x[0]);
    if (H.m == 1) *qc = stage_qoi(&bc, n0, H.K[0], H.x[0]);
    for (int k = 1; k <= H.m; ++k) {
        int n = grid_n(&H, k);
        or_fmg_interpolate_bc(n / 2, H.x[k - 1], bc.g, bc.ns, H.x[k]);
        or_stage_rhs_bc(n, H.K[k], bc.g, bc.ns, H.b[k]);
        cycles += stage_cycles(&H, k, P);
        if (k == H.m - 1) *qc = stage_qoi(&bc, n, H.K[k], H.x[k]);
    }
    *qf = stage_qoi(&bc, n_fine, H.K[H.m], H.x[H.m]);
    if (p_out) memcpy(p_out, H.x[H.m], sizeof(double) * (size_t)n_fine * n_fine);
    hierarchy_free(&H);
    return cycles;
}

/* V-cycles on a given problem A x = b from the given x (for convergence-factor
 * checks).  res_hist[c] = ||b - A x|| after cycle c (c = 0 before any). */
void or_vcycle_solve(int n, int n0, const double* K, const double* b, double* x,
                     int nu1, int nu2, int ncycles, int coarse_op, int energy_step, int ns, double* res_hist)
{
    hierarchy H;
    hierarchy_init(&H, n, n0, K, coarse_op, energy_step, ns);
    memcpy(H.b[H.m], b, sizeof(double) * (size_t)n * n);
    memcpy(H.x[H.m], x, sizeof(double) * (size_t)n * n);
    for (int c = 0; c <= ncycles; ++c) {
        if (c > 0) vcycle(&H, H.m, H.m, nu1, nu2);
        if (res_hist) {
            or_residual_bc(n, H.K[H.m], ns, H.b[H.m], H.x[H.m], H.r[H.m]);
            res_hist[c] = or_norm2(n * n, H.r[H.m]);
        }
    }
    memcpy(x, H.x[H.m], sizeof(double) * (size_t)n * n);
    hierarchy_free(&H);
}

/* Batch of independent samples, one thread per sample when OpenMP is on.
 * K[s*n*n ...], qf[s], qc[s]; p (nullable) [s][n][n]. Returns threads used. */
int or_fmg_solve_batch(int n_fine, int n0, int S, const double* K, const or_params* P,
                       double* p, double* qf, double* qc, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int s = 0; s < S; ++s) {
        size_t off = (size_t)s * n_fine * n_fine;
        or_fmg_solve(n_fine, n0, K + off, P, p ? p + off : NULL, qf + s, qc + s);
    }
#ifdef _OPENMP
    used = nthreads;
#endif
    (void)nthreads;
    return used;
}
