// Rank-1 lattice sequence for randomized QMC (Sec. 2.4: "random shift" of a
// lattice rule): the generating vector, built component by component on the
// host by the fast construction of Nuyens & Cools (FFT over the
// multiplicative group of the odd residues), for the embedded point sets of
// 2^m points, m = m_min .. m_max.
//
// Criterion (the same as the test oracle's plain construction): component s
// is the odd z < 2^(m_max - 1) minimising
//   C(z) = sum_m e^2_m(z_1..z_(s-1), z) / e^2_m(z_1..z_(s-1)),
//   e^2_m = -1 + 2^-m sum_k prod_j (1 + gamma_j omega({k z_j / 2^m})),
// omega = B_2 (the shift-averaged worst-case error of the unanchored
// Sobolev space), gamma_j = 1 / j^2, z_1 = 1.  With p_k the product over
// the chosen components, e^2_m(z) = -1 + (P_m + gamma_s E_m(z)) / 2^m,
// E_m(z) = sum_k p_k omega({k z / 2^m}): a matrix-vector product for all z
// at once.
//
// Fast evaluation of E_m for every odd z: split k = 2^v u with u odd; then
// {k z / 2^m} = {u z' / 2^r}, r = m - v, z' = z mod 2^r, and
//   E_m(z) = omega(0) p_0 + sum_v sum_{u in U_r} omega(u z' / 2^r) p_(2^v u),
// U_r the odd residues mod 2^r.  For r >= 3, U_r = {(-1)^a 5^b mod 2^r},
// a in {0, 1}, b mod 2^(r-2) (Gauss), so the inner sum is a cyclic
// correlation over Z_2 x Z_(2^(r-2)): four length-2^(r-2) correlations,
// done by FFT.  r = 1, 2 are summed directly.  O(2^m m) per component and
// size instead of O(4^m).
//
// The FFT rounds differently from a plain sum, so the decision is taken on
// the plain sums: every candidate within a small margin of the fast minimum
// is re-evaluated term by term, in the oracle's operation order (IEEE
// double, no fused multiply-adds: the library's host code is compiled with
// contraction off), and the smallest z with the least criterion wins.  The
// generating vector is therefore the plain construction's, bit for bit.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace fm {
namespace {

using cplx = std::complex<double>;

double bernoulli2(double x) { return x * x - x + 1.0 / 6.0; }

// Roots e^(-2 pi i k / L), k < L/2, for fft below.
std::vector<cplx> fft_roots(size_t L) {
    const double pi = 3.14159265358979323846;
    std::vector<cplx> w(std::max<size_t>(L / 2, 1));
    for (size_t k = 0; k < L / 2; ++k) w[k] = cplx(std::cos(2.0 * pi * k / L), -std::sin(2.0 * pi * k / L));
    return w;
}

// In-place iterative radix-2 FFT of length L = 2^p, X_k = sum_j x_j e^(-+2 pi i jk/L)
// (sign -1: forward, +1: inverse, unnormalised); roots from fft_roots(L).
void fft(std::vector<cplx>& a, int sign, const std::vector<cplx>& roots) {
    const size_t L = a.size();
    for (size_t i = 1, j = 0; i < L; ++i) {   // bit-reversal permutation
        size_t bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= L; len <<= 1) {
        const size_t step = L / len;
        for (size_t i = 0; i < L; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                // complex arithmetic written out (finite values only)
                const double wr = roots[k * step].real(), wi = sign < 0 ? roots[k * step].imag()
                                                                      : -roots[k * step].imag();
                const double xr = a[i + k + len / 2].real(), xi = a[i + k + len / 2].imag();
                const double vr = xr * wr - xi * wi, vi = xr * wi + xi * wr;
                const double ur = a[i + k].real(), ui = a[i + k].imag();
                a[i + k] = cplx(ur + vr, ui + vi);
                a[i + k + len / 2] = cplx(ur - vr, ui - vi);
            }
    }
}

// The group U_r (r >= 3) as Z_2 x Z_L, L = 2^(r-2): elem[a L + b] = (-1)^a 5^b mod 2^r,
// index[w] = a L + b for odd w; Ff[a] = DFT of omega(elem[a L + b] / 2^r) over b.
struct Group {
    int r = 0;
    uint32_t L = 0;
    std::vector<uint32_t> elem;
    std::vector<int32_t> index;
    std::vector<cplx> roots;
    std::vector<cplx> Ff[2];
};

Group make_group(int r) {
    Group g;
    g.r = r;
    const uint32_t n = 1u << r, mask = n - 1;
    g.L = 1u << (r - 2);
    g.elem.resize(2 * g.L);
    g.index.assign(n, -1);
    uint32_t w = 1;
    for (uint32_t b = 0; b < g.L; ++b) {
        g.elem[b] = w;
        g.elem[g.L + b] = (n - w) & mask;
        w = (w * 5u) & mask;
    }
    for (uint32_t e = 0; e < 2 * g.L; ++e) g.index[g.elem[e]] = (int32_t)e;
    g.roots = fft_roots(g.L);
    for (int a = 0; a < 2; ++a) {
        g.Ff[a].resize(g.L);
        for (uint32_t b = 0; b < g.L; ++b) g.Ff[a][b] = bernoulli2((double)g.elem[a * g.L + b] / n);
        fft(g.Ff[a], -1, g.roots);
    }
    return g;
}

// E[w] += sum_{u in U_r} omega(u w / 2^r) q[u] for every odd w < 2^r (q indexed by odd u).
void group_correlation(const Group& g, const std::vector<double>& q, std::vector<double>& E) {
    const uint32_t L = g.L;
    std::vector<cplx> Q[2];
    for (int a = 0; a < 2; ++a) {
        Q[a].resize(L);
        for (uint32_t b = 0; b < L; ++b) Q[a][b] = q[g.elem[a * L + b]];
        fft(Q[a], -1, g.roots);
    }
    std::vector<cplx> R0(L), R1(L);
    auto mulc = [](cplx f, cplx q) {   // f * conj(q)
        return cplx(f.real() * q.real() + f.imag() * q.imag(), f.imag() * q.real() - f.real() * q.imag());
    };
    for (uint32_t k = 0; k < L; ++k) {
        const cplx a0 = mulc(g.Ff[0][k], Q[0][k]), a1 = mulc(g.Ff[1][k], Q[1][k]);
        const cplx b0 = mulc(g.Ff[1][k], Q[0][k]), b1 = mulc(g.Ff[0][k], Q[1][k]);
        R0[k] = cplx(a0.real() + a1.real(), a0.imag() + a1.imag());   // alpha = 0
        R1[k] = cplx(b0.real() + b1.real(), b0.imag() + b1.imag());   // alpha = 1
    }
    fft(R0, +1, g.roots);
    fft(R1, +1, g.roots);
    for (uint32_t b = 0; b < L; ++b) {
        E[g.elem[b]] += R0[b].real() / L;
        E[g.elem[L + b]] += R1[b].real() / L;
    }
}

struct Cbc {
    int m_min, m_max;
    std::vector<std::vector<double>> p;   // p[a][k], a = m - m_min
    std::vector<double> e2, P;

    // The criterion of candidate z summed term by term (the plain construction's order).
    double plain(uint32_t z, double gamma) const {
        double C = 0.0;
        for (int a = 0; a <= m_max - m_min; ++a) {
            const uint32_t n = 1u << (m_min + a);
            double E = 0.0;
            for (uint32_t k = 0; k < n; ++k)
                E += p[a][k] * bernoulli2((double)(((uint64_t)k * z) & (n - 1)) / n);
            C += (-1.0 + (P[a] + gamma * E) / n) / e2[a];
        }
        return C;
    }
};

}  // namespace

int lattice_cbc_host(uint32_t dim, int m_min, int m_max, uint32_t* z) {
    if (m_min < 1 || m_max < m_min || m_max > 24 || dim < 1) return -1;
    const int nm = m_max - m_min + 1;
    Cbc c;
    c.m_min = m_min;
    c.m_max = m_max;
    c.p.resize(nm);
    c.e2.resize(nm);
    c.P.resize(nm);
    for (int a = 0; a < nm; ++a) {
        const uint32_t n = 1u << (m_min + a);
        c.p[a].resize(n);
        double sum = 0.0;
        for (uint32_t k = 0; k < n; ++k) {
            c.p[a][k] = 1.0 + 1.0 * bernoulli2((double)k / n);   // z_1 = 1, gamma_1 = 1
            sum += c.p[a][k];
        }
        c.e2[a] = -1.0 + sum / n;
    }
    std::vector<Group> groups(m_max + 1);
    for (int r = 3; r <= m_max; ++r) groups[r] = make_group(r);
    z[0] = 1;
    const uint32_t half = 1u << (m_max - 1);
    std::vector<double> Cfast(half, 0.0);
    std::vector<double> q, E;
    for (uint32_t s = 1; s < dim; ++s) {
        const double gamma = 1.0 / ((double)(s + 1) * (s + 1));
        for (int a = 0; a < nm; ++a) {
            const uint32_t n = 1u << (m_min + a);
            double sum = 0.0;
            for (uint32_t k = 0; k < n; ++k) sum += c.p[a][k];
            c.P[a] = sum;
        }
        std::fill(Cfast.begin(), Cfast.end(), 0.0);
        for (int a = 0; a < nm; ++a) {
            const int m = m_min + a;
            const uint32_t n = 1u << m;
            E.assign(n, 0.0);   // E[w] for odd w < n
            const double e0 = bernoulli2(0.0) * c.p[a][0];
            for (int v = 0; v < m; ++v) {
                const int r = m - v;
                const uint32_t nr = 1u << r;
                // q[u] = p_(2^v u), u odd < 2^r; its correlation lands on E mod 2^r
                q.assign(nr, 0.0);
                for (uint32_t u = 1; u < nr; u += 2) q[u] = c.p[a][(size_t)u << v];
                std::vector<double> Er(nr, 0.0);
                if (r >= 3) {
                    group_correlation(groups[r], q, Er);
                } else if (r == 2) {
                    Er[1] = bernoulli2(1.0 / 4) * q[1] + bernoulli2(3.0 / 4) * q[3];
                    Er[3] = bernoulli2(3.0 / 4) * q[1] + bernoulli2(1.0 / 4) * q[3];
                } else {
                    Er[1] = bernoulli2(0.5) * q[1];
                }
                for (uint32_t w = 1; w < n; w += 2) E[w] += Er[w & (nr - 1)];
            }
            for (uint32_t zc = 1; zc < half; zc += 2)
                Cfast[zc] += (-1.0 + (c.P[a] + gamma * (e0 + E[zc & (n - 1)])) / n) / c.e2[a];
        }
        double cmin = INFINITY;
        for (uint32_t zc = 1; zc < half; zc += 2) cmin = std::min(cmin, Cfast[zc]);
        const double margin = 1e-7 * std::fabs(cmin) + 1e-12;
        uint32_t best = 0;
        double bestC = INFINITY;
        for (uint32_t zc = 1; zc < half; zc += 2) {
            if (Cfast[zc] > cmin + margin) continue;
            const double C = c.plain(zc, gamma);
            if (C < bestC) {
                bestC = C;
                best = zc;
            }
        }
        z[s] = best;
        for (int a = 0; a < nm; ++a) {
            const uint32_t n = 1u << (m_min + a);
            double sum = 0.0;
            for (uint32_t k = 0; k < n; ++k) {
                c.p[a][k] *= 1.0 + gamma * bernoulli2((double)(((uint64_t)k * best) & (n - 1)) / n);
                sum += c.p[a][k];
            }
            c.e2[a] = -1.0 + sum / n;
        }
    }
    return 0;
}

// The vector for (dim, m_min, m_max), built once per process.
const std::vector<uint32_t>* lattice_vector_cached(uint32_t dim, int m_min, int m_max) {
    static std::mutex mu;
    static std::map<std::tuple<uint32_t, int, int>, std::vector<uint32_t>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(dim, m_min, m_max);
    auto it = cache.find(key);
    if (it != cache.end()) return &it->second;
    std::vector<uint32_t> z(dim);
    if (lattice_cbc_host(dim, m_min, m_max, z.data()) != 0) return nullptr;
    return &(cache[key] = std::move(z));
}

}  // namespace fm

extern "C" fm_status fm_lattice_cbc(uint32_t dim, int32_t m_min, int32_t m_max, uint32_t* z) {
    if (!z || dim < 1 || dim > 4096 || m_min < 1 || m_max < m_min || m_max > 24) return FM_EINVAL;
    return fm::lattice_cbc_host(dim, m_min, m_max, z) == 0 ? FM_OK : FM_EINVAL;
}
