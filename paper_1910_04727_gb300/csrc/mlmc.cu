// MLMC / MLQMC level sums and the host controller (Sec. 2.2-2.5,
// Algorithms 1-3).
//
// Sums are deterministic: a fixed block size and a fixed sample-to-block map
// give each block a Neumaier-compensated partial sum in a fixed order, and a
// single thread folds the partials into the running (sum, compensation)
// pairs in block order.  Repeating a run repeats its sums bit for bit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace fm {

constexpr int kSumBlock = 256;
constexpr double kMaxSamplesPerLevel = 1e9;   // guard against a runaway sample-size rule
constexpr int kSumItems = 2048;   // samples per block

struct Pair {
    double s, c;
};

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// partial[block][4][2]: (sum, comp) of y, y^2, qf, qc over the block's samples.
__global__ void __launch_bounds__(kSumBlock) k_level_partials(size_t S, const double* __restrict__ qf,
                                                             const double* __restrict__ qc, int coarse,
                                                             double* __restrict__ partial) {
    __shared__ double sh[kSumBlock][8];
    const size_t begin = (size_t)blockIdx.x * kSumItems;
    const size_t end = min(S, begin + kSumItems);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t i = begin + threadIdx.x; i < end; i += kSumBlock) {
        const double f = qf[i];
        const double c = coarse ? qc[i] : 0.0;
        const double y = f - c;
        neumaier_add(acc[0], acc[1], y);
        neumaier_add(acc[2], acc[3], y * y);
        neumaier_add(acc[4], acc[5], f);
        neumaier_add(acc[6], acc[7], coarse ? c : 0.0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int width = kSumBlock / 2; width > 0; width >>= 1) {
        if (threadIdx.x < width) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double s = sh[threadIdx.x][2 * q], c = sh[threadIdx.x][2 * q + 1];
                neumaier_add(s, c, sh[threadIdx.x + width][2 * q]);
                c += sh[threadIdx.x + width][2 * q + 1];
                sh[threadIdx.x][2 * q] = s;
                sh[threadIdx.x][2 * q + 1] = c;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) partial[(size_t)blockIdx.x * 8 + threadIdx.x] = sh[0][threadIdx.x];
}

__global__ void k_level_fold(int nblocks, size_t S, const double* __restrict__ partial,
                             fm_level_sums* __restrict__ sums) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* dst[4] = {sums->sum_y, sums->sum_y2, sums->sum_qf, sums->sum_qc};
    for (int q = 0; q < 4; ++q) {
        double s = dst[q][0], c = dst[q][1];
        for (int b = 0; b < nblocks; ++b) {
            neumaier_add(s, c, partial[(size_t)b * 8 + 2 * q]);
            c += partial[(size_t)b * 8 + 2 * q + 1];
        }
        dst[q][0] = s;
        dst[q][1] = c;
    }
    sums->count += (double)S;
}

fm_status level_sums_add(fm_ctx* ctx, uint32_t S, const double* d_qf, const double* d_qc, int coarse,
                         fm_level_sums* d_sums, cudaStream_t st) {
    if (S == 0) return FM_OK;
    const int nb = (int)((S + kSumItems - 1) / kSumItems);
    FM_TRY(ensure(ctx, &ctx->d_partials, &ctx->partial_capacity, (size_t)nb * 8));
    FM_TIMED(ctx, kFamLevelSums, st, 16.0 * S, 8.0 * S,
             k_level_partials<<<nb, kSumBlock, 0, st>>>(S, d_qf, d_qc, coarse, ctx->d_partials);
             k_level_fold<<<1, 32, 0, st>>>(nb, S, ctx->d_partials, d_sums));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

static fm_solve_params solve_params(const fm_ctx* ctx) {
    fm_solve_params p{};
    p.pW = ctx->cfg.pW;
    p.pE = ctx->cfg.pE;
    p.n_coarsest = ctx->cfg.n_coarsest;
    p.nu0 = ctx->cfg.nu0;
    p.nu1 = ctx->cfg.nu1;
    p.nu2 = ctx->cfg.nu2;
    p.precision = ctx->cfg.precision;
    p.kernel = FM_KERNEL_AUTO;
    p.converged = ctx->cfg.converged;
    p.tol = ctx->cfg.tol;
    p.qtol = ctx->cfg.qtol;
    p.max_cycles = ctx->cfg.max_cycles;
    return p;
}

static double fold(const double* pair) { return pair[0] + pair[1]; }

// least-squares slope of -log2|v_l| over l = 1..L (NaN if undefined)
static double fit_rate(const double* v, int L) {
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    int cnt = 0;
    for (int l = 1; l <= L; ++l) {
        if (!(std::fabs(v[l]) > 0)) return NAN;
        const double y = std::log2(std::fabs(v[l]));
        sx += l; sy += y; sxx += (double)l * l; sxy += l * y;
        ++cnt;
    }
    if (cnt < 2) return NAN;
    return -(cnt * sxy - sx * sy) / (cnt * sxx - sx * sx);
}

}  // namespace fm

using namespace fm;

extern "C" fm_status mlmc_sample_level(fm_ctx* ctx, int32_t level, uint64_t first, uint32_t n,
                                       int32_t shift, fm_level_sums* d_sums, double* d_qf, double* d_qc,
                                       void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "mlmc_sample_level: null context");
    FM_CHECK_ARG(ctx, (level >= 0 || (level == -1 && ctx->surrogate_on)) && level < ctx->cfg.n_levels,
                 "mlmc_sample_level: bad level (-1, the surrogate level, needs surrogate_enable)");
    FM_CHECK_ARG(ctx, ctx->basis_ready, "mlmc_sample_level: no KL basis installed");
    FM_CHECK_ARG(ctx, shift < ctx->cfg.n_shifts, "mlmc_sample_level: shift out of range");
    FM_CHECK_ARG(ctx, d_sums != nullptr || d_qf != nullptr, "mlmc_sample_level: no output");
    if (n == 0) return FM_OK;
    cudaStream_t st = as_stream(stream);
    const bool s_level = (level == -1);
    const bool with_s = ctx->surrogate_on && level <= 0;   // S(xi) needed: level -1, or Y_0 = Q_0 - S
    const int N = grid_of_level(ctx, s_level ? 0 : level), M = ctx->cfg.M;
    const uint32_t stream_level = s_level ? kSurrogateLevelStream : (uint32_t)level;
    const fm_solve_params prm = solve_params(ctx);
    // MC surrogate samples need no FP64 points: S is evaluated from the Philox words
    const bool s_mc = s_level && shift < 0;
    const int64_t lim = s_level ? (int64_t)1 << 22 : std::min<int64_t>(batch_limit(ctx, N), (int64_t)65535 * 64);
    const size_t cap = (size_t)std::min<int64_t>(lim, n);
    if (!s_mc) FM_TRY(ensure(ctx, &ctx->d_xi, &ctx->xi_capacity, cap * M));
    if (!s_level) FM_TRY(ensure(ctx, &ctx->d_K, &ctx->K_capacity, cap * (size_t)N * N));
    FM_TRY(ensure(ctx, &ctx->d_q, &ctx->q_capacity, 2 * cap));
    for (uint64_t off = 0; off < n; off += cap) {
        const uint32_t cnt = (uint32_t)std::min<uint64_t>(cap, n - off);
        if (shift >= 0) {
            FM_TRY(sobol_points(ctx, stream_level, (uint32_t)M, first + off, cnt, (uint32_t)shift, 1, nullptr,
                                ctx->d_xi, stream));
        } else if (!s_mc) {
            FM_TRY(mc_points(ctx, stream_level, first + off, cnt, (uint32_t)M, ctx->d_xi, stream));
        }
        double* qf = ctx->d_q;
        double* qc = ctx->d_q + cap;
        // S(omega): from the Philox words of the sample for MC, from its QMC point otherwise
        auto eval_s = [&](double* out) -> fm_status {
            return shift < 0 ? surrogate_eval_mc_impl(ctx, stream_level, first + off, cnt, out, st)
                             : surrogate_eval_impl(ctx, cnt, ctx->d_xi, out, st);
        };
        if (s_level) {
            // the surrogate level: Y = S
            FM_TRY(eval_s(qf));
        } else {
            FM_TRY(kl_field_batch(ctx, level, cnt, ctx->d_xi, ctx->d_K, stream));
            FM_TRY(fmg_solve_impl(ctx, N, cnt, ctx->d_K, prm, qf, qc, nullptr, nullptr, st));
            // level 0 with the surrogate: Y = Q_0 - S, S in the Q^c slot
            if (with_s) FM_TRY(eval_s(qc));
        }
        if (d_sums) FM_TRY(level_sums_add(ctx, cnt, qf, qc, (level > 0 || (with_s && !s_level)) ? 1 : 0, d_sums, st));
        if (d_qf) FM_CUDA_TRY(ctx, cudaMemcpyAsync(d_qf + off, qf, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (d_qc) FM_CUDA_TRY(ctx, cudaMemcpyAsync(d_qc + off, qc, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    return FM_OK;
}

extern "C" fm_status mlmc_estimate(fm_ctx* ctx, const fm_estimate_opts* opts, fm_result* out) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "mlmc_estimate: null context");
    FM_CHECK_ARG(ctx, opts && out, "mlmc_estimate: null argument");
    FM_CHECK_ARG(ctx, opts->eps > 0, "mlmc_estimate: eps must be positive");
    FM_CHECK_ARG(ctx, opts->n_pilot >= 2, "mlmc_estimate: n_pilot must be >= 2");
    FM_CHECK_ARG(ctx, !opts->qmc || ctx->cfg.n_shifts >= 2, "mlmc_estimate: QMC needs n_shifts >= 2");
    const auto t0 = std::chrono::steady_clock::now();
    FM_CHECK_ARG(ctx, !opts->surrogate || (ctx->mlp && opts->surrogate_cost > 0),
                 "mlmc_estimate: the surrogate level needs a trained network and surrogate_cost > 0");
    // Extended levels e = 0 .. L_e: with the surrogate, e = 0 is the S level
    // and e = l + 1 MLMC level l; without it e = l.
    const int off = opts->surrogate ? 1 : 0;
    const int Lr = ctx->cfg.n_levels - 1;
    const int L = Lr + off;
    const int R = opts->qmc ? ctx->cfg.n_shifts : 1;
    const int max_rounds = opts->max_rounds > 0 ? opts->max_rounds : 100;
    const size_t cells = (size_t)(L + 1) * R;
    std::vector<fm_level_sums> h(cells);
    FM_CUDA_TRY(ctx, cudaMemset(ctx->d_sums, 0, cells * sizeof(fm_level_sums)));
    double C[FM_MAX_LEVELS + 1];
    for (int e = 0; e <= L; ++e) {
        const double n = grid_of_level(ctx, std::max(0, e - off));
        C[e] = n * n * 4.0 / 3.0;
    }
    if (off) C[0] *= opts->surrogate_cost;   // S-level cost relative to a level-0 sample
    std::memset(out, 0, sizeof(*out));
    int64_t N[FM_MAX_LEVELS + 1] = {};
    int64_t dN[FM_MAX_LEVELS + 1];
    for (int l = 0; l <= L; ++l) dN[l] = opts->n_pilot;
    double mean[FM_MAX_LEVELS + 1] = {}, var[FM_MAX_LEVELS + 1] = {};
    int rounds = 0;
    const int saved_on = ctx->surrogate_on;
    ctx->surrogate_on = opts->surrogate ? 1 : 0;
    struct Restore {
        fm_ctx* c;
        int v;
        ~Restore() { c->surrogate_on = v; }
    } restore{ctx, saved_on};

    // device time per extended level: an event pair around each level's
    // sampling, read back at the next synchronisation
    struct LevelTimer {
        std::vector<cudaEvent_t> ev;
        std::vector<int> lev;
        size_t used = 0;
        ~LevelTimer() {
            for (cudaEvent_t e : ev) cudaEventDestroy(e);
        }
    } lt;
    double lsec[FM_MAX_LEVELS + 1] = {};
    auto event = [&]() -> cudaEvent_t {
        if (lt.used == lt.ev.size()) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            lt.ev.push_back(e);
        }
        return lt.ev[lt.used++];
    };
    auto collect = [&]() {
        for (size_t i = 0; i + 1 < lt.used; i += 2) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, lt.ev[i], lt.ev[i + 1]) == cudaSuccess) lsec[lt.lev[i / 2]] += ms * 1e-3;
        }
        lt.used = 0;
        lt.lev.clear();
    };

    auto refresh = [&]() -> fm_status {
        FM_TRY(fm_sync(ctx));
        collect();
        FM_CUDA_TRY(ctx, cudaMemcpy(h.data(), ctx->d_sums, cells * sizeof(fm_level_sums), cudaMemcpyDeviceToHost));
        for (int l = 0; l <= L; ++l) {
            if (!opts->qmc) {
                const fm_level_sums& s = h[l];
                const double n = s.count;
                const double sy = fold(s.sum_y), sy2 = fold(s.sum_y2);
                if (!std::isfinite(sy) || !std::isfinite(sy2)) {
                    set_error(ctx, "mlmc_estimate: non-finite samples on level " + std::to_string(l));
                    return FM_ENOTCONV;
                }
                mean[l] = sy / n;
                var[l] = n > 1 ? std::max(0.0, (sy2 - sy * sy / n) / (n - 1)) : 0.0;
            } else {
                double m[64];
                double mm = 0.0;
                for (int r = 0; r < R; ++r) {
                    const fm_level_sums& s = h[(size_t)l * R + r];
                    m[r] = fold(s.sum_y) / s.count;
                    if (!std::isfinite(m[r])) {
                        set_error(ctx, "mlmc_estimate: non-finite samples on level " + std::to_string(l));
                        return FM_ENOTCONV;
                    }
                    mm += m[r];
                }
                mm /= R;
                double v = 0.0;
                for (int r = 0; r < R; ++r) v += (m[r] - mm) * (m[r] - mm);
                mean[l] = mm;
                var[l] = v / ((double)R * (R - 1));
            }
        }
        return FM_OK;
    };

    auto run = [&](int l, int64_t first, int64_t cnt) -> fm_status {
        cudaEvent_t e0 = event(), e1 = event();
        lt.lev.push_back(l);
        cudaEventRecord(e0, nullptr);
        for (int r = 0; r < R; ++r)
            FM_TRY(mlmc_sample_level(ctx, l - off, (uint64_t)first, (uint32_t)cnt, opts->qmc ? r : -1,
                                     ctx->d_sums + (size_t)l * R + r, nullptr, nullptr, nullptr));
        cudaEventRecord(e1, nullptr);
        return FM_OK;
    };

    if (!opts->qmc) {
        // Algorithm 1 / 3 at fixed L: evaluate dN, update V_l and the optimal N_l, repeat.
        while (rounds < max_rounds) {
            bool any = false;
            for (int l = 0; l <= L; ++l)
                if (dN[l] > 0) {
                    FM_TRY(run(l, N[l], dN[l]));
                    N[l] += dN[l];
                    any = true;
                }
            if (!any) break;
            ++rounds;
            FM_TRY(refresh());
            double tot = 0.0;
            for (int l = 0; l <= L; ++l) tot += std::sqrt(var[l] * C[l]);
            for (int l = 0; l <= L; ++l) {
                const double opt = std::ceil(2.0 / (opts->eps * opts->eps) * std::sqrt(var[l] / C[l]) * tot);
                if (!std::isfinite(opt) || opt > kMaxSamplesPerLevel) {
                    set_error(ctx, "mlmc_estimate: level " + std::to_string(l) + " would need " +
                                       std::to_string(opt) + " samples (variance " + std::to_string(var[l]) +
                                       "); beyond the per-level cap");
                    return FM_ENOTCONV;
                }
                dN[l] = std::max<int64_t>(0, (int64_t)opt - N[l]);
            }
        }
        double v = 0.0;
        for (int l = 0; l <= L; ++l) v += var[l] / (double)N[l];
        out->var_estimator = v;
    } else {
        // Algorithm 2 at fixed L: pilot, then double N_l at argmax V[Y_l]/(N_l C_l).
        for (int l = 0; l <= L; ++l) {
            FM_TRY(run(l, 0, opts->n_pilot));
            N[l] = opts->n_pilot;
        }
        FM_TRY(refresh());
        while (rounds < max_rounds) {
            double tot = 0.0;
            for (int l = 0; l <= L; ++l) tot += var[l];
            if (tot <= opts->eps * opts->eps / 2) break;
            int best = 0;
            double bv = -1.0;
            for (int l = 0; l <= L; ++l) {
                const double v = var[l] / ((double)N[l] * C[l]);
                if (v > bv) { bv = v; best = l; }
            }
            FM_CHECK_ARG(ctx, N[best] <= ((int64_t)1 << 31), "mlmc_estimate: QMC point budget exhausted");
            FM_TRY(run(best, N[best], N[best]));
            N[best] *= 2;
            ++rounds;
            FM_TRY(refresh());
        }
        double v = 0.0;
        for (int l = 0; l <= L; ++l) v += var[l];
        out->var_estimator = v;
    }
    double est = 0.0;
    for (int e = 0; e <= L; ++e) est += mean[e];
    for (int l = 0; l <= Lr; ++l) {
        out->mean[l] = mean[l + off];
        out->var[l] = var[l + off];
        out->N[l] = N[l + off];
    }
    for (int l = 0; l <= Lr; ++l) out->level_seconds[l] = lsec[l + off];
    out->seconds_s = off ? lsec[0] : 0.0;
    if (off) {
        out->mean_s = mean[0];
        out->var_s = var[0];
        out->N_s = N[0];
    }
    out->estimate = est;
    out->alpha = fit_rate(out->mean, Lr);
    out->beta = fit_rate(out->var, Lr);
    out->bias = (std::isfinite(out->alpha) && out->alpha > 0)
                    ? std::fabs(out->mean[Lr]) / (std::pow(2.0, out->alpha) - 1.0) : NAN;
    out->rounds = rounds;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return FM_OK;
}
