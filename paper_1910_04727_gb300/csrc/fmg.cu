// Batched full multigrid for the Case II Darcy problem (Eq. 1, Table 1,
// Sec. 2.5): one FMG hierarchy per sample, all samples of a batch advanced
// level by level, every kernel covering every cell of every sample of one
// grid (x fastest, so a warp touches consecutive cells of one row).
//
// Per grid k (n_k = n_coarsest << k) and sample the scratch holds
//   K   coefficients (injected from the finer grid; the finest is the input)
//   Te  east-face transmissibility of each cell (2K on the east edge)
//   Tn  north-face transmissibility (0 on the north edge)
//   D   diagonal: sum of the four face transmissibilities (2K on the west edge)
//   p   iterate, b right-hand side
// and for the coarsest grid the inverse of its dense operator, so each exact
// solve is one small matrix-vector product.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace fm {

constexpr int kBlock = 256;

inline unsigned blocks_for(size_t threads) { return (unsigned)((threads + kBlock - 1) / kBlock); }

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

// K_c[J][I] = K_f[2J][2I] (Sec. 2.5, the lower-left child in 0-indexed form).
__global__ void k_inject(int nc, size_t S, const double* __restrict__ Kf, double* __restrict__ Kc) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)nc * nc;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    const int c = (int)(t % cells);
    const int I = c % nc, J = c / nc, nf = 2 * nc;
    Kc[t] = Kf[s * (size_t)nf * nf + (size_t)(2 * J) * nf + 2 * I];
}

// Face transmissibilities: harmonic mean inside, 2K on the Dirichlet edges,
// none on the no-flow edges.
__global__ void k_coefficients(int n, size_t S, const double* __restrict__ K, double* __restrict__ Te,
                               double* __restrict__ Tn, double* __restrict__ D) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)n * n;
    if (t >= S * cells) return;
    const int c = (int)(t % cells);
    const int i = c % n, j = c / n;
    const double k = K[t];
    const double tw = (i > 0) ? harmonic(K[t - 1], k) : 2.0 * k;
    const double te = (i < n - 1) ? harmonic(k, K[t + 1]) : 2.0 * k;
    const double ts = (j > 0) ? harmonic(K[t - n], k) : 0.0;
    const double tn = (j < n - 1) ? harmonic(k, K[t + n]) : 0.0;
    Te[t] = te;
    Tn[t] = tn;
    D[t] = tw + te + ts + tn;
}

// Right-hand side of a stage problem: the Dirichlet data moved to the rhs.
__global__ void k_stage_rhs(int n, size_t S, const double* __restrict__ K, double pW, double pE,
                            double* __restrict__ b) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)n * n;
    if (t >= S * cells) return;
    const int i = (int)(t % cells) % n;
    double v = 0.0;
    if (i == 0) v += 2.0 * K[t] * pW;
    if (i == n - 1) v += 2.0 * K[t] * pE;
    b[t] = v;
}

// One colour of a red-black Gauss-Seidel sweep: cells with (i + j) % 2 == color.
__global__ void k_rbgs_color(int n, size_t S, int color, const double* __restrict__ b,
                             const double* __restrict__ Te, const double* __restrict__ Tn,
                             const double* __restrict__ D, double* __restrict__ p) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t half = (size_t)n * n / 2;
    if (t >= S * half) return;
    const size_t s = t / half;
    const int h = (int)(t % half);
    const int j = h / (n / 2);
    const int i = 2 * (h % (n / 2)) + ((j + color) & 1);
    const size_t c = s * (size_t)n * n + (size_t)j * n + i;
    double acc = b[c];
    if (i > 0) acc += Te[c - 1] * p[c - 1];
    if (i < n - 1) acc += Te[c] * p[c + 1];
    if (j > 0) acc += Tn[c - n] * p[c - n];
    if (j < n - 1) acc += Tn[c] * p[c + n];
    p[c] = acc / D[c];
}

__device__ __forceinline__ double residual_at(int n, size_t c, int i, int j, const double* b,
                                              const double* Te, const double* Tn, const double* D,
                                              const double* p) {
    double v = D[c] * p[c];
    if (i > 0) v -= Te[c - 1] * p[c - 1];
    if (i < n - 1) v -= Te[c] * p[c + 1];
    if (j > 0) v -= Tn[c - n] * p[c - n];
    if (j < n - 1) v -= Tn[c] * p[c + n];
    return b[c] - v;
}

// Fused residual + restriction: b_c = sum of the four fine residuals; p_c = 0.
__global__ void k_residual_restrict(int nc, size_t S, const double* __restrict__ bf,
                                    const double* __restrict__ Te, const double* __restrict__ Tn,
                                    const double* __restrict__ D, const double* __restrict__ pf,
                                    double* __restrict__ bc, double* __restrict__ pc) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)nc * nc;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    const int C = (int)(t % cells);
    const int I = C % nc, J = C / nc, nf = 2 * nc;
    const size_t base = s * (size_t)nf * nf;
    const int i0 = 2 * I, j0 = 2 * J;
    const size_t c00 = base + (size_t)j0 * nf + i0;
    const double r00 = residual_at(nf, c00, i0, j0, bf, Te, Tn, D, pf);
    const double r10 = residual_at(nf, c00 + 1, i0 + 1, j0, bf, Te, Tn, D, pf);
    const double r01 = residual_at(nf, c00 + nf, i0, j0 + 1, bf, Te, Tn, D, pf);
    const double r11 = residual_at(nf, c00 + nf + 1, i0 + 1, j0 + 1, bf, Te, Tn, D, pf);
    bc[t] = r00 + r10 + r01 + r11;
    pc[t] = 0.0;
}

// Coarse value with ghosts: mirror across the no-flow edges, 2g - u across
// the Dirichlet edges (g = 0 for an error).
__device__ __forceinline__ double coarse_ghost(int nc, const double* uc, int I, int J, double gW,
                                               double gE) {
    J = J < 0 ? 0 : (J > nc - 1 ? nc - 1 : J);
    if (I < 0) return 2.0 * gW - uc[(size_t)J * nc];
    if (I > nc - 1) return 2.0 * gE - uc[(size_t)J * nc + nc - 1];
    return uc[(size_t)J * nc + I];
}

__device__ __forceinline__ double bilinear_at(int nc, const double* uc, int i, int j, double gW,
                                              double gE) {
    const int I = i >> 1, J = j >> 1;
    const int Ix = (i & 1) ? I + 1 : I - 1;
    const int Jy = (j & 1) ? J + 1 : J - 1;
    return (9.0 * coarse_ghost(nc, uc, I, J, gW, gE) + 3.0 * coarse_ghost(nc, uc, Ix, J, gW, gE) +
            3.0 * coarse_ghost(nc, uc, I, Jy, gW, gE) + 1.0 * coarse_ghost(nc, uc, Ix, Jy, gW, gE)) /
           16.0;
}

// p_f += P e_c (add = 1, boundary values 0) or p_f = P u_c (add = 0, FMG start).
__global__ void k_prolong(int nc, size_t S, const double* __restrict__ uc, double gW, double gE,
                          int add, double* __restrict__ pf) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = 2 * nc;
    const size_t cells = (size_t)nf * nf;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    const int c = (int)(t % cells);
    const double v = bilinear_at(nc, uc + s * (size_t)nc * nc, c % nf, c / nf, gW, gE);
    pf[t] = add ? pf[t] + v : v;
}

// Inverse of the dense operator of the coarsest grid (m = n0^2 unknowns), by
// Gauss-Jordan elimination on [A | I]; A is SPD so no pivoting is needed.
// One thread per sample; m <= 16.
__global__ void k_coarse_inverse(int n0, size_t S, const double* __restrict__ Te,
                                 const double* __restrict__ Tn, const double* __restrict__ D,
                                 double* __restrict__ Ainv) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int m = n0 * n0;
    double A[16][16], X[16][16];
    const double* te = Te + s * m;
    const double* tn = Tn + s * m;
    const double* d = D + s * m;
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) {
            A[r][c] = 0.0;
            X[r][c] = (r == c) ? 1.0 : 0.0;
        }
    for (int c = 0; c < m; ++c) {
        const int i = c % n0, j = c / n0;
        A[c][c] = d[c];
        if (i < n0 - 1) { A[c][c + 1] = -te[c]; A[c + 1][c] = -te[c]; }
        if (j < n0 - 1) { A[c][c + n0] = -tn[c]; A[c + n0][c] = -tn[c]; }
    }
    for (int k = 0; k < m; ++k) {
        const double inv = 1.0 / A[k][k];
        for (int c = 0; c < m; ++c) { A[k][c] *= inv; X[k][c] *= inv; }
        for (int r = 0; r < m; ++r) {
            if (r == k) continue;
            const double f = A[r][k];
            if (f == 0.0) continue;
            for (int c = 0; c < m; ++c) { A[r][c] -= f * A[k][c]; X[r][c] -= f * X[k][c]; }
        }
    }
    double* out = Ainv + s * (size_t)m * m;
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) out[r * m + c] = X[r][c];
}

// p = A^{-1} b on the coarsest grid; one thread per (sample, unknown).
__global__ void k_coarse_solve(int m, size_t S, const double* __restrict__ Ainv,
                               const double* __restrict__ b, double* __restrict__ p) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S * m) return;
    const size_t s = t / m;
    const int r = (int)(t % m);
    const double* row = Ainv + s * (size_t)m * m + (size_t)r * m;
    const double* bs = b + s * m;
    double acc = 0.0;
    for (int c = 0; c < m; ++c) acc += row[c] * bs[c];
    p[t] = acc;
}

// Q = sum_j 2 K_(n-1,j) (p_(n-1,j) - pE), one warp per sample, shuffle reduction.
__global__ void k_outflux(int n, size_t S, const double* __restrict__ K, const double* __restrict__ p,
                          double pE, double* __restrict__ q) {
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (warp >= S) return;
    const size_t base = warp * (size_t)n * n + (n - 1);
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc += 2.0 * K[base + (size_t)j * n] * (p[base + (size_t)j * n] - pE);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) q[warp] = acc;
}

__global__ void k_fill(size_t count, double v, double* __restrict__ x) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) x[t] = v;
}

// ------------------------------------------------------------------ driver
struct GridBufs {
    int n;
    const double* K;
    double *Te, *Tn, *D, *p, *b;
};

struct Hierarchy {
    fm_ctx* ctx;
    int m;   // finest index
    int n0;
    size_t S;
    GridBufs g[FM_MAX_LEVELS + 8];
    double* Ainv;
};

static size_t hierarchy_doubles(int n_fine, int n0, size_t S) {
    size_t total = 0;
    for (int n = n0; n <= n_fine; n *= 2) total += (size_t)6 * n * n;  // K, Te, Tn, D, p, b
    total += (size_t)n0 * n0 * n0 * n0;                                 // Ainv
    return total * S;
}

int64_t batch_limit(const fm_ctx* ctx, int n) {
    const size_t per = hierarchy_doubles(n, std::max(ctx->cfg.n_coarsest, 4), 1) * sizeof(double) +
                       (size_t)n * n * sizeof(double) + (size_t)ctx->cfg.M * sizeof(double);
    const size_t budget = (size_t)8 << 30;   // 8 GiB of scratch per batch
    int64_t lim = (int64_t)(budget / per);
    if (ctx->cfg.max_batch > 0) lim = std::min<int64_t>(lim, ctx->cfg.max_batch);
    return std::max<int64_t>(lim, 1);
}

static fm_status carve(fm_ctx* ctx, Hierarchy& H, int n_fine, int n0, size_t S, const double* d_K) {
    const size_t need = hierarchy_doubles(n_fine, n0, S) * sizeof(double) + 64 * 256;
    if (ctx->arena.capacity < need) {
        if (ctx->arena.base) cudaFree(ctx->arena.base);
        ctx->arena.base = nullptr;
        ctx->arena.capacity = 0;
        if (cudaMalloc((void**)&ctx->arena.base, need) != cudaSuccess) {
            set_error(ctx, "fmg scratch allocation of " + std::to_string(need) + " bytes failed");
            return FM_ENOMEM;
        }
        ctx->arena.capacity = need;
    }
    char* cur = ctx->arena.base;
    auto take = [&](size_t count) {
        double* p = reinterpret_cast<double*>(cur);
        cur += ((count * sizeof(double) + 255) / 256) * 256;
        return p;
    };
    H.ctx = ctx;
    H.n0 = n0;
    H.S = S;
    H.m = 0;
    while ((n0 << H.m) < n_fine) ++H.m;
    for (int k = 0; k <= H.m; ++k) {
        const int n = n0 << k;
        const size_t cnt = S * (size_t)n * n;
        GridBufs& g = H.g[k];
        g.n = n;
        g.K = (k == H.m) ? d_K : take(cnt);
        g.Te = take(cnt);
        g.Tn = take(cnt);
        g.D = take(cnt);
        g.p = take(cnt);
        g.b = take(cnt);
    }
    H.Ainv = take(S * (size_t)n0 * n0 * n0 * n0);
    return FM_OK;
}

static void vcycle(const Hierarchy& H, int k, const fm_solve_params& prm, cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    const size_t S = H.S;
    const GridBufs& g = H.g[k];
    if (k == 0) {
        const int m = H.n0 * H.n0;
        FM_TIMED(ctx, kFamCoarseSolve, st, (double)S * (m * m + 2 * m) * 8.0, 2.0 * S * m * m,
                 k_coarse_solve<<<blocks_for(S * m), kBlock, 0, st>>>(m, S, H.Ainv, g.b, g.p));
        return;
    }
    const int n = g.n;
    const size_t cells = S * (size_t)n * n;
    const size_t half = cells / 2;
    // algorithmic bytes of one colour: half of a single-pass sweep that reads
    // p, b, Te, Tn, D and writes p (48 B per cell in FP64)
    const double sweep_half_bytes = 24.0 * cells, sweep_half_flops = 5.0 * cells;
    for (int it = 0; it < prm.nu1; ++it)
        for (int color = 0; color < 2; ++color)
            FM_TIMED(ctx, kFamSmoother, st, sweep_half_bytes, sweep_half_flops,
                     k_rbgs_color<<<blocks_for(half), kBlock, 0, st>>>(n, S, color, g.b, g.Te, g.Tn, g.D, g.p));
    const GridBufs& c = H.g[k - 1];
    FM_TIMED(ctx, kFamResidualRestrict, st, 44.0 * cells, 10.0 * cells,
             k_residual_restrict<<<blocks_for(S * (size_t)c.n * c.n), kBlock, 0, st>>>(
                 c.n, S, g.b, g.Te, g.Tn, g.D, g.p, c.b, c.p));
    vcycle(H, k - 1, prm, st);
    FM_TIMED(ctx, kFamProlong, st, 18.0 * cells, 8.0 * cells,
             k_prolong<<<blocks_for(cells), kBlock, 0, st>>>(c.n, S, c.p, 0.0, 0.0, 1, g.p));
    for (int it = 0; it < prm.nu2; ++it)
        for (int color = 0; color < 2; ++color)
            FM_TIMED(ctx, kFamSmoother, st, sweep_half_bytes, sweep_half_flops,
                     k_rbgs_color<<<blocks_for(half), kBlock, 0, st>>>(n, S, color, g.b, g.Te, g.Tn, g.D, g.p));
}

static void outflux(const Hierarchy& H, int k, double pE, double* q, cudaStream_t st) {
    const GridBufs& g = H.g[k];
    FM_TIMED(H.ctx, kFamOutflux, st, 16.0 * H.S * g.n, 3.0 * H.S * g.n,
             k_outflux<<<blocks_for(H.S * 32), kBlock, 0, st>>>(g.n, H.S, g.K, g.p, pE, q));
}

static void fmg_batch(const Hierarchy& H, const fm_solve_params& prm, double* qf, double* qc,
                      double* p_out, cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    const size_t S = H.S;
    // coefficient hierarchy: inject, then faces and diagonals on every grid
    for (int k = H.m; k >= 1; --k) {
        const int nc = H.g[k - 1].n;
        const size_t cc = S * (size_t)nc * nc;
        FM_TIMED(ctx, kFamInject, st, 16.0 * cc, 0.0,
                 k_inject<<<blocks_for(cc), kBlock, 0, st>>>(nc, S, H.g[k].K, const_cast<double*>(H.g[k - 1].K)));
    }
    for (int k = 0; k <= H.m; ++k) {
        const GridBufs& g = H.g[k];
        const size_t cells = S * (size_t)g.n * g.n;
        FM_TIMED(ctx, kFamCoefficients, st, 32.0 * cells, 16.0 * cells,
                 k_coefficients<<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, g.K, g.Te, g.Tn, g.D));
    }
    {
        const int m = H.n0 * H.n0;
        FM_TIMED(ctx, kFamCoarseInverse, st, (double)S * (3 * m + m * m) * 8.0, 2.0 * S * m * m * m,
                 k_coarse_inverse<<<blocks_for(S), 64, 0, st>>>(H.n0, S, H.g[0].Te, H.g[0].Tn, H.g[0].D, H.Ainv));
    }
    // stage 0: exact solve of the coarsest stage problem
    {
        const GridBufs& g = H.g[0];
        const size_t cells = S * (size_t)g.n * g.n;
        FM_TIMED(ctx, kFamStageRhs, st, 16.0 * cells, 2.0 * cells,
                 k_stage_rhs<<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, g.K, prm.pW, prm.pE, g.b));
        vcycle(H, 0, prm, st);
        if (H.m == 1 && qc) outflux(H, 0, prm.pE, qc, st);
    }
    for (int k = 1; k <= H.m; ++k) {
        const GridBufs& g = H.g[k];
        const size_t cells = S * (size_t)g.n * g.n;
        FM_TIMED(ctx, kFamFmgInterp, st, 10.0 * cells, 8.0 * cells,
                 k_prolong<<<blocks_for(cells), kBlock, 0, st>>>(H.g[k - 1].n, S, H.g[k - 1].p, prm.pW, prm.pE, 0, g.p));
        FM_TIMED(ctx, kFamStageRhs, st, 16.0 * cells, 2.0 * cells,
                 k_stage_rhs<<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, g.K, prm.pW, prm.pE, g.b));
        for (int it = 0; it < prm.nu0; ++it) vcycle(H, k, prm, st);
        if (k == H.m - 1 && qc) outflux(H, k, prm.pE, qc, st);
    }
    if (H.m == 0 && qc) k_fill<<<blocks_for(S), kBlock, 0, st>>>(S, std::nan(""), qc);
    outflux(H, H.m, prm.pE, qf, st);
    if (p_out)
        cudaMemcpyAsync(p_out, H.g[H.m].p, sizeof(double) * S * H.g[H.m].n * H.g[H.m].n,
                        cudaMemcpyDeviceToDevice, st);
}

fm_status fmg_solve_impl(fm_ctx* ctx, int n_fine, uint32_t S, const double* d_K,
                         const fm_solve_params& prm, double* d_qf, double* d_qc, double* d_p,
                         cudaStream_t st) {
    const int n0 = prm.n_coarsest;
    FM_CHECK_ARG(ctx, n0 >= 2 && n0 <= 4, "fmg_solve_batch: n_coarsest must be 2..4");
    FM_CHECK_ARG(ctx, n_fine >= n0 && n_fine <= 8192, "fmg_solve_batch: bad n_fine");
    int m = 0;
    while ((n0 << m) < n_fine) ++m;
    FM_CHECK_ARG(ctx, (n0 << m) == n_fine, "fmg_solve_batch: n_fine must be n_coarsest * 2^m");
    FM_CHECK_ARG(ctx, prm.nu0 >= 1 && prm.nu1 >= 0 && prm.nu2 >= 0 && prm.nu1 + prm.nu2 >= 1,
                 "fmg_solve_batch: need nu0 >= 1 and nu1 + nu2 >= 1");
    FM_CHECK_ARG(ctx, prm.precision == FM_PREC_FP64, "fmg_solve_batch: unknown precision");
    FM_CHECK_ARG(ctx, S == 0 || (d_K && d_qf), "fmg_solve_batch: null input or output");
    if (S == 0) return FM_OK;
    const int64_t lim = batch_limit(ctx, n_fine);
    for (uint64_t first = 0; first < S; first += (uint64_t)lim) {
        const size_t cnt = (size_t)std::min<uint64_t>((uint64_t)lim, S - first);
        const size_t off = first * (size_t)n_fine * n_fine;
        Hierarchy H;
        FM_TRY(carve(ctx, H, n_fine, n0, cnt, d_K + off));
        fmg_batch(H, prm, d_qf + first, d_qc ? d_qc + first : nullptr, d_p ? d_p + off : nullptr, st);
        FM_CUDA_TRY(ctx, cudaGetLastError());
    }
    return FM_OK;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fmg_solve_batch(fm_ctx* ctx, int32_t n_fine, uint32_t n, const double* d_K,
                                     const fm_solve_params* prm, double* d_qf, double* d_qc,
                                     double* d_p, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fmg_solve_batch: null context");
    FM_CHECK_ARG(ctx, prm != nullptr, "fmg_solve_batch: null parameters");
    return fmg_solve_impl(ctx, n_fine, n, d_K, *prm, d_qf, d_qc, d_p, as_stream(stream));
}
