// MC and randomized-QMC points (Sec. 2.3, Sec. 2.4, Sec. 3.1).
//
// One thread produces four consecutive dimensions of one sample: a single
// Philox4x64-10 block gives the four 64-bit words, so no word is computed
// twice.  Output is written x-fastest ([sample][dim]), coalesced across the
// warp.  Integer work (Philox words, Sobol' points, shifts) is bit-exact;
// Phi^{-1} is CUDA's normcdfinv.
#include "common.cuh"

namespace fm {

// xi (nullable): the normals; words (nullable): the raw 64-bit Philox words
// they come from, in the same [sample][dim] layout.
__global__ void k_mc_points(uint64_t seed, uint32_t level, uint64_t first, uint32_t n,
                            uint32_t dim, double* __restrict__ xi, uint64_t* __restrict__ words) {
    const uint32_t blocks = (dim + 3) / 4;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * blocks) return;
    const uint32_t s = (uint32_t)(t / blocks);
    const uint32_t b = (uint32_t)(t % blocks);
    u64x4 c = {{b, first + s, 0, 0}};
    u64x4 w = philox4x64(c, seed, (kPurposeMC << 32) | level);
#pragma unroll
    for (int lane = 0; lane < 4; ++lane) {
        uint32_t k = 4 * b + lane;
        if (k < dim) {
            if (words) words[(size_t)s * dim + k] = w.v[lane];
            if (xi) {
                const double u = ((double)(w.v[lane] >> 11) + 0.5) * 0x1p-53;
                xi[(size_t)s * dim + k] = normcdfinv(u);
            }
        }
    }
}

// Sobol' point x_d(idx) = XOR_{b : bit b of gray(idx)} V[d][b], shifted.
__global__ void k_sobol_points(const uint32_t* __restrict__ V, uint64_t seed, uint32_t level,
                               uint32_t dim, uint64_t first, uint32_t n, uint32_t first_shift,
                               uint32_t n_shifts, uint32_t* __restrict__ out,
                               double* __restrict__ xi) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)n_shifts * n * dim;
    if (t >= total) return;
    const uint32_t d = (uint32_t)(t % dim);
    const uint64_t sn = t / dim;
    const uint32_t s = (uint32_t)(sn % n);
    const uint32_t r = (uint32_t)(sn / n);
    const uint64_t idx = first + s;
    const uint64_t gray = idx ^ (idx >> 1);
    uint32_t x = 0;
    const uint32_t* Vd = V + (size_t)d * 32;
#pragma unroll 4
    for (int b = 0; b < 32; ++b)
        if ((gray >> b) & 1) x ^= __ldg(Vd + b);
    // digital shift of (level, shift first_shift + r, dimension d)
    u64x4 c = {{d / 4, first_shift + r, 0, 0}};
    u64x4 w = philox4x64(c, seed, (kPurposeShift << 32) | level);
    x ^= (uint32_t)(w.v[d % 4] >> 32);
    if (out) out[t] = x;
    if (xi) xi[t] = normcdfinv(((double)x + 0.5) * 0x1p-32);
}

// Nested uniform scrambling (Owen 1995) of one 32-bit coordinate: output
// bit b (b = 0 the most significant) is input bit b XOR the random bit of
// the tree node (b, leading b input bits): the low bit of word 0 of the
// Philox stream (seed, OWEN << 32 | level) at counter (prefix, r << 32 | d, b, 0).
__device__ __forceinline__ uint32_t owen_scramble(uint64_t seed, uint32_t level, uint32_t r, uint32_t d,
                                                  uint32_t x) {
    const uint64_t k1 = (kPurposeOwen << 32) | level;
    uint32_t y = 0;
#pragma unroll 1
    for (int b = 0; b < 32; ++b) {
        const uint64_t prefix = b == 0 ? 0 : (uint64_t)(x >> (32 - b));
        const u64x4 c = {{prefix, ((uint64_t)r << 32) | d, (uint64_t)b, 0}};
        const u64x4 w = philox4x64(c, seed, k1);
        y |= (((x >> (31 - b)) & 1u) ^ (uint32_t)(w.v[0] & 1u)) << (31 - b);
    }
    return y;
}

// Owen-scrambled Sobol' points: the plain Gray-code point, then the nested
// scramble of scramble first_shift + r.  Same layout as k_sobol_points.
__global__ void k_sobol_owen_points(const uint32_t* __restrict__ V, uint64_t seed, uint32_t level, uint32_t dim,
                                    uint64_t first, uint32_t n, uint32_t first_shift, uint32_t n_shifts,
                                    uint32_t* __restrict__ out, double* __restrict__ xi) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)n_shifts * n * dim;
    if (t >= total) return;
    const uint32_t d = (uint32_t)(t % dim);
    const uint64_t sn = t / dim;
    const uint32_t s = (uint32_t)(sn % n);
    const uint32_t r = (uint32_t)(sn / n);
    const uint64_t idx = first + s;
    const uint64_t gray = idx ^ (idx >> 1);
    uint32_t x = 0;
    const uint32_t* Vd = V + (size_t)d * 32;
#pragma unroll 4
    for (int b = 0; b < 32; ++b)
        if ((gray >> b) & 1) x ^= __ldg(Vd + b);
    x = owen_scramble(seed, level, first_shift + r, d, x);
    if (out) out[t] = x;
    if (xi) xi[t] = normcdfinv(((double)x + 0.5) * 0x1p-32);
}

// Randomly shifted rank-1 lattice sequence (32-bit fixed point): point index
// i in radical-inverse order over m_max bits (the first 2^m points are the
// 2^m-point lattice), x = (z_d phi(i) 2^(32 - m_max) + Delta) mod 2^32, the
// shift Delta the high 32 bits of word d of the Philox stream
// (seed, LATTICE_SHIFT << 32 | level) at index first_shift + r.
__global__ void k_lattice_points(const uint32_t* __restrict__ z, int m_max, uint64_t seed, uint32_t level,
                                 uint32_t dim, uint64_t first, uint32_t n, uint32_t first_shift, uint32_t n_shifts,
                                 uint32_t* __restrict__ out, double* __restrict__ xi) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)n_shifts * n * dim;
    if (t >= total) return;
    const uint32_t d = (uint32_t)(t % dim);
    const uint64_t sn = t / dim;
    const uint32_t s = (uint32_t)(sn % n);
    const uint32_t r = (uint32_t)(sn / n);
    const uint32_t i = (uint32_t)(first + s);
    const uint32_t rev = __brev(i) >> (32 - m_max);
    const uint32_t mask = m_max == 32 ? 0xFFFFFFFFu : ((1u << m_max) - 1u);
    const uint32_t tq = (uint32_t)((uint64_t)__ldg(z + d) * rev) & mask;
    const u64x4 c = {{d / 4, first_shift + r, 0, 0}};
    const u64x4 w = philox4x64(c, seed, (kPurposeLatticeShift << 32) | level);
    const uint32_t x = (tq << (32 - m_max)) + (uint32_t)(w.v[d % 4] >> 32);
    if (out) out[t] = x;
    if (xi) xi[t] = normcdfinv(((double)x + 0.5) * 0x1p-32);
}

// ------------------------------------------------------------------ host
// Bratley & Fox: primitive polynomials over GF(2) in ascending degree and
// bit-mask order; initial odd m_k < 2^k from Philox; the recurrence
// m_k = m_(k-s) ^ (m_(k-s) << s) ^ XOR_{i<s} a_i (m_(k-i) << i).
static uint64_t gf2_mulmod(uint64_t a, uint64_t b, uint64_t p, int deg) {
    uint64_t r = 0;
    for (; b; b >>= 1) {
        if (b & 1) r ^= a;
        a <<= 1;
        if ((a >> deg) & 1) a ^= p;
    }
    return r;
}

static uint64_t gf2_pow_x(uint64_t e, uint64_t p, int deg) {
    uint64_t base = 2;
    if ((base >> deg) & 1) base ^= p;
    uint64_t r = 1;
    for (; e; e >>= 1) {
        if (e & 1) r = gf2_mulmod(r, base, p, deg);
        base = gf2_mulmod(base, base, p, deg);
    }
    return r;
}

static bool gf2_primitive(uint64_t p, int deg) {
    const uint64_t order = (1ULL << deg) - 1;
    if (gf2_pow_x(order, p, deg) != 1) return false;
    uint64_t m = order;
    for (uint64_t q = 2; q * q <= m; ++q) {
        if (m % q) continue;
        if (gf2_pow_x(order / q, p, deg) == 1) return false;
        while (m % q == 0) m /= q;
    }
    return !(m > 1 && gf2_pow_x(order / m, p, deg) == 1);
}

int sobol_direction_numbers_host(uint32_t dim, std::vector<uint32_t>& V) {
    V.assign((size_t)dim * 32, 0);
    std::vector<uint64_t> polys;
    std::vector<int> degs;
    for (int deg = 1; deg <= 31 && polys.size() + 1 < dim; ++deg)
        for (uint64_t p = (1ULL << deg) | 1; p < (1ULL << (deg + 1)) && polys.size() + 1 < dim; p += 2)
            if (gf2_primitive(p, deg)) {
                polys.push_back(p);
                degs.push_back(deg);
            }
    if (dim > 1 && polys.size() + 1 < dim) return -1;
    for (uint32_t d = 0; d < dim; ++d) {
        uint64_t m[33];
        if (d == 0) {
            for (int k = 1; k <= 32; ++k) m[k] = 1;
        } else {
            const uint64_t p = polys[d - 1];
            const int s = degs[d - 1];
            for (int k = 1; k <= s && k <= 32; ++k) {
                u64x4 c = {{(uint64_t)(k - 1) / 4, d, 0, 0}};
                u64x4 w = philox4x64(c, kSobolDirSeed, kPurposeSobolDir << 32);
                m[k] = 2 * (w.v[(k - 1) % 4] % (1ULL << (k - 1))) + 1;
            }
            for (int k = s + 1; k <= 32; ++k) {
                uint64_t v = m[k - s] ^ (m[k - s] << s);
                for (int i = 1; i < s; ++i)
                    if ((p >> (s - i)) & 1) v ^= m[k - i] << i;
                m[k] = v;
            }
        }
        for (int k = 1; k <= 32; ++k) V[(size_t)d * 32 + k - 1] = (uint32_t)(m[k] << (32 - k));
    }
    return 0;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status mc_points(fm_ctx* ctx, uint32_t level, uint64_t first, uint32_t n,
                               uint32_t dim, double* d_xi, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "mc_points: null context");
    FM_CHECK_ARG(ctx, dim >= 1 && dim <= 4096, "mc_points: dim must be in [1, 4096]");
    FM_CHECK_ARG(ctx, n == 0 || d_xi != nullptr, "mc_points: null output");
    if (n == 0) return FM_OK;
    const uint64_t threads = (uint64_t)n * ((dim + 3) / 4);
    const int bs = 256;
    FM_TIMED(ctx, kFamPoints, as_stream(stream), 8.0 * n * dim, 0.0,
             k_mc_points<<<(unsigned)((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
                 ctx->cfg.seed, level, first, n, dim, d_xi, nullptr));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status mc_words(fm_ctx* ctx, uint32_t level, uint64_t first, uint32_t n, uint32_t dim,
                              uint64_t* d_words, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "mc_words: null context");
    FM_CHECK_ARG(ctx, dim >= 1 && dim <= 4096, "mc_words: dim must be in [1, 4096]");
    FM_CHECK_ARG(ctx, n == 0 || d_words != nullptr, "mc_words: null output");
    if (n == 0) return FM_OK;
    const uint64_t threads = (uint64_t)n * ((dim + 3) / 4);
    const int bs = 256;
    FM_TIMED(ctx, kFamPoints, as_stream(stream), 8.0 * n * dim, 0.0,
             k_mc_points<<<(unsigned)((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
                 ctx->cfg.seed, level, first, n, dim, nullptr, d_words));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status sobol_points(fm_ctx* ctx, uint32_t level, uint32_t dim, uint64_t first,
                                  uint32_t n, uint32_t first_shift, uint32_t n_shifts,
                                  uint32_t* d_x, double* d_xi, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "sobol_points: null context");
    FM_CHECK_ARG(ctx, dim >= 1 && (int)dim <= ctx->cfg.M,
                 "sobol_points: dim must be in [1, M]");
    FM_CHECK_ARG(ctx, first + n <= (1ULL << 32), "sobol_points: point index beyond 2^32");
    if (n == 0 || n_shifts == 0) return FM_OK;
    const uint64_t total = (uint64_t)n_shifts * n * dim;
    const int bs = 256;
    FM_TIMED(ctx, kFamPoints, as_stream(stream), 12.0 * total, 0.0,
             k_sobol_points<<<(unsigned)((total + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
                 ctx->d_sobol_V, ctx->cfg.seed, level, dim, first, n, first_shift, n_shifts, d_x, d_xi));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status sobol_direction_numbers(const fm_ctx* ctx, uint32_t* V) {
    if (!ctx || !V) return FM_EINVAL;
    std::copy(ctx->h_sobol_V.begin(), ctx->h_sobol_V.end(), V);
    return FM_OK;
}

extern "C" fm_status qmc_points(fm_ctx* ctx, int32_t rule, uint32_t level, uint32_t dim, uint64_t first, uint32_t n,
                                uint32_t first_shift, uint32_t n_shifts, uint32_t* d_x, double* d_xi, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "qmc_points: null context");
    FM_CHECK_ARG(ctx, rule == FM_QMC_SOBOL_SHIFT || rule == FM_QMC_SOBOL_OWEN || rule == FM_QMC_LATTICE,
                 "qmc_points: unknown rule");
    if (rule == FM_QMC_SOBOL_SHIFT)
        return sobol_points(ctx, level, dim, first, n, first_shift, n_shifts, d_x, d_xi, stream);
    FM_CHECK_ARG(ctx, dim >= 1 && (int)dim <= ctx->cfg.M, "qmc_points: dim must be in [1, M]");
    if (n == 0 || n_shifts == 0) return FM_OK;
    const uint64_t total = (uint64_t)n_shifts * n * dim;
    const int bs = 256;
    if (rule == FM_QMC_SOBOL_OWEN) {
        FM_CHECK_ARG(ctx, first + n <= (1ULL << 32), "qmc_points: point index beyond 2^32");
        FM_TIMED(ctx, kFamPoints, as_stream(stream), 12.0 * total, 0.0,
                 k_sobol_owen_points<<<(unsigned)((total + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
                     ctx->d_sobol_V, ctx->cfg.seed, level, dim, first, n, first_shift, n_shifts, d_x, d_xi));
    } else {
        FM_CHECK_ARG(ctx, ctx->d_lattice_z != nullptr,
                     "qmc_points: the lattice rule needs a context created with qmc_rule = FM_QMC_LATTICE");
        const int m_max = ctx->cfg.lattice_m;
        FM_CHECK_ARG(ctx, first + n <= (1ULL << m_max),
                     "qmc_points: point index beyond the lattice sequence's 2^lattice_m points");
        FM_TIMED(ctx, kFamPoints, as_stream(stream), 12.0 * total, 0.0,
                 k_lattice_points<<<(unsigned)((total + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
                     ctx->d_lattice_z, m_max, ctx->cfg.seed, level, dim, first, n, first_shift, n_shifts, d_x,
                     d_xi));
    }
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status lattice_generating_vector(const fm_ctx* ctx, uint32_t* z) {
    if (!ctx || !z) return FM_EINVAL;
    FM_CHECK_ARG(ctx, !ctx->h_lattice_z.empty(), "lattice_generating_vector: no lattice rule in this context");
    std::copy(ctx->h_lattice_z.begin(), ctx->h_lattice_z.end(), z);
    return FM_OK;
}
