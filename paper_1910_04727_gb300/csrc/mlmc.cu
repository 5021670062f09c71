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
        // y^2 with its rounding error (exact product): the pair then holds
        // the sum of the exact squares, which the variance needs when
        // |mean| >> sd
        const double y2 = y * y;
        neumaier_add(acc[2], acc[3], y2);
        acc[3] += fma(y, y, -y2);
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

fm_status level_sums_add_to(fm_ctx* ctx, uint32_t S, const double* d_qf, const double* d_qc, int coarse,
                            fm_level_sums* d_sums, cudaStream_t st, double** partials, size_t* capacity) {
    if (S == 0) return FM_OK;
    const int nb = (int)((S + kSumItems - 1) / kSumItems);
    FM_TRY(ensure(ctx, partials, capacity, (size_t)nb * 8));
    double* part = *partials;
    FM_TIMED(ctx, kFamLevelSums, st, 16.0 * S, 8.0 * S,
             k_level_partials<<<nb, kSumBlock, 0, st>>>(S, d_qf, d_qc, coarse, part);
             k_level_fold<<<1, 32, 0, st>>>(nb, S, part, d_sums));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

fm_status level_sums_add(fm_ctx* ctx, uint32_t S, const double* d_qf, const double* d_qc, int coarse,
                         fm_level_sums* d_sums, cudaStream_t st) {
    return level_sums_add_to(ctx, S, d_qf, d_qc, coarse, d_sums, st, &ctx->d_partials, &ctx->partial_capacity);
}

fm_solve_params solve_params(const fm_ctx* ctx) {
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
    p.bc_case = ctx->cfg.bc_case;
    p.ir_cycles = ctx->cfg.ir_cycles;
    p.energy_step = ctx->cfg.energy_step;
    p.pS = ctx->cfg.pS;
    p.pN = ctx->cfg.pN;
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
            FM_TRY(qmc_points(ctx, ctx->cfg.qmc_rule, stream_level, (uint32_t)M, first + off, cnt, (uint32_t)shift, 1,
                              nullptr, ctx->d_xi, stream));
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
            // level 0 takes no Q^c (Y_0 = Q_0, or Q_0 - S): the solver then
            // leaves its coarse stage unrefined, unless the caller asks for it
            double* solve_qc = (level > 0 || (d_qc && !with_s)) ? qc : nullptr;
            FM_TRY(fmg_solve_impl(ctx, N, cnt, ctx->d_K, prm, qf, solve_qc, nullptr, nullptr, st));
            // level 0 with the surrogate: Y = Q_0 - S, S in the Q^c slot
            if (with_s) FM_TRY(eval_s(qc));
        }
        if (d_sums) FM_TRY(level_sums_add(ctx, cnt, qf, qc, (level > 0 || (with_s && !s_level)) ? 1 : 0, d_sums, st));
        if (d_qf) FM_CUDA_TRY(ctx, cudaMemcpyAsync(d_qf + off, qf, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (d_qc) FM_CUDA_TRY(ctx, cudaMemcpyAsync(d_qc + off, qc, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    return FM_OK;
}

namespace {

struct Request {
    int e;               // extended level
    uint64_t first, n;
    int shift;
};

// Per-level buffers of a batched round, kept in the context across rounds
// and estimates (grown when short), so a timed estimate allocates nothing.
struct LevelBuf {
    double *xi = nullptr, *K = nullptr, *q = nullptr;
    size_t cap = 0;    // samples of xi and q
    size_t kcap = 0;   // samples of K (one pass)
};
struct BatchedBufs {
    LevelBuf lb[FM_MAX_LEVELS];
    // the surrogate level's MC requests on a stream of their own: S values,
    // partial sums, the stream and its fork and join events
    double* s_q = nullptr;
    size_t s_cap = 0;
    double* s_part = nullptr;
    size_t s_pcap = 0;
    cudaStream_t s_st = nullptr;
    cudaEvent_t s_fork = nullptr, s_join = nullptr;
};

BatchedBufs* batched_state(fm_ctx* ctx) {
    if (!ctx->batched) ctx->batched = new BatchedBufs();
    return static_cast<BatchedBufs*>(ctx->batched);
}

LevelBuf* batched_bufs(fm_ctx* ctx) { return batched_state(ctx)->lb; }

// Chunk of the surrogate level's samples per evaluation (the one
// mlmc_sample_level uses, so the sums are the same whichever path adds them).
constexpr uint64_t kSChunk = (uint64_t)1 << 22;

// GPU side of the controller: samples go to mlmc_sample_level with the
// running sums of (level, shift) cell e * R + r in ctx->d_sums; an event pair
// around each request gives the device time per level.  Batched: a round's
// requests are kept until the controller reads the sums, then every level's
// points and fields are made, all levels are solved as one uneven batch
// (fmg_solve_uneven), and the sums are added request by request.
struct GpuSampler {
    fm_ctx* ctx;
    int off, R;
    size_t cells;
    bool batched = false;
    std::vector<Request> pending;
    LevelBuf* lb = nullptr;   // the context's (batched_bufs)
    double round_sec = 0.0;
    cudaEvent_t b0 = nullptr, b1 = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<int> lev;
    size_t used = 0;
    double lsec[FM_MAX_LEVELS + 1] = {};
    ~GpuSampler() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (b0) cudaEventDestroy(b0);
        if (b1) cudaEventDestroy(b1);
    }
    cudaEvent_t event() {
        if (used == ev.size()) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            ev.push_back(e);
        }
        return ev[used++];
    }
    void collect() {
        for (size_t i = 0; i + 1 < used; i += 2) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) lsec[lev[i / 2]] += ms * 1e-3;
        }
        used = 0;
        lev.clear();
    }
};

fm_status gpu_enqueue(void* user, int32_t e, uint64_t first, uint64_t n, int32_t shift) {
    GpuSampler* g = static_cast<GpuSampler*>(user);
    if (g->batched) {
        g->pending.push_back(Request{e, first, n, shift});
        return FM_OK;
    }
    cudaEvent_t e0 = g->event(), e1 = g->event();
    g->lev.push_back(e);
    cudaEventRecord(e0, nullptr);
    fm_level_sums* cell = g->ctx->d_sums + (size_t)e * g->R + (shift < 0 ? 0 : shift);
    for (uint64_t done = 0; done < n;) {
        const uint32_t cnt = (uint32_t)std::min<uint64_t>(n - done, (uint64_t)1 << 30);
        FM_TRY(mlmc_sample_level(g->ctx, e - g->off, first + done, cnt, shift, cell, nullptr, nullptr, nullptr));
        done += cnt;
    }
    cudaEventRecord(e1, nullptr);
    return FM_OK;
}

// The pending requests of a round as one uneven batch (see GpuSampler).
fm_status flush_batched(GpuSampler* g) {
    fm_ctx* ctx = g->ctx;
    if (g->pending.empty()) return FM_OK;
    const int L = ctx->cfg.n_levels, M = ctx->cfg.M;
    const fm_solve_params prm = solve_params(ctx);
    std::vector<uint64_t> total(L, 0);
    for (const Request& r : g->pending)
        if (r.e - g->off >= 0) total[r.e - g->off] += r.n;
    if (!g->b0) {
        cudaEventCreate(&g->b0);
        cudaEventCreate(&g->b1);
    }
    cudaEventRecord(g->b0, nullptr);
    // The surrogate level's MC requests need only the trained network (the
    // fused inference kernel, no shared scratch): they run on a stream of
    // their own beside the round's points, fields and solves.
    BatchedBufs* B = batched_state(ctx);
    const bool s_side = surrogate_mc_fused(ctx);
    bool s_forked = false;
    if (s_side) {
        uint64_t need = 0;
        for (const Request& r : g->pending)
            if (r.e - g->off < 0 && r.shift < 0) need = std::max<uint64_t>(need, std::min<uint64_t>(r.n, kSChunk));
        if (need) {
            if (!B->s_st) {
                FM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&B->s_st, cudaStreamNonBlocking));
                FM_CUDA_TRY(ctx, cudaEventCreateWithFlags(&B->s_fork, cudaEventDisableTiming));
                FM_CUDA_TRY(ctx, cudaEventCreateWithFlags(&B->s_join, cudaEventDisableTiming));
            }
            FM_TRY(ensure(ctx, &B->s_q, &B->s_cap, (size_t)need));
            FM_CUDA_TRY(ctx, cudaEventRecord(B->s_fork, nullptr));
            FM_CUDA_TRY(ctx, cudaStreamWaitEvent(B->s_st, B->s_fork, 0));
            for (const Request& r : g->pending) {
                if (r.e - g->off >= 0 || r.shift >= 0) continue;
                cudaEvent_t e0 = g->event(), e1 = g->event();
                g->lev.push_back(r.e);
                cudaEventRecord(e0, B->s_st);
                fm_level_sums* cell = ctx->d_sums + (size_t)r.e * g->R;
                for (uint64_t done = 0; done < r.n;) {
                    const uint32_t cnt = (uint32_t)std::min<uint64_t>(r.n - done, kSChunk);
                    FM_TRY(surrogate_eval_mc_impl(ctx, kSurrogateLevelStream, r.first + done, cnt, B->s_q, B->s_st));
                    FM_TRY(level_sums_add_to(ctx, cnt, B->s_q, nullptr, 0, cell, B->s_st, &B->s_part, &B->s_pcap));
                    done += cnt;
                }
                cudaEventRecord(e1, B->s_st);
            }
            FM_CUDA_TRY(ctx, cudaEventRecord(B->s_join, B->s_st));
            s_forked = true;
        }
    }
    // points of every request, level by level, requests packed in order;
    // fields and solves in passes of at most batch_limit samples per level,
    // one uneven batch per pass (every level's next chunk)
    std::vector<uint64_t> chunk(L, 0);
    uint64_t passes = 0;
    for (int l = 0; l < L; ++l) {
        if (!total[l]) continue;
        const int N = grid_of_level(ctx, l);
        chunk[l] = std::min<uint64_t>(total[l], (uint64_t)batch_limit(ctx, N));
        passes = std::max<uint64_t>(passes, (total[l] + chunk[l] - 1) / chunk[l]);
        LevelBuf& b = g->lb[l];
        if (b.cap < total[l] || b.kcap < chunk[l]) {
            if (b.xi) cudaFree(b.xi);
            if (b.K) cudaFree(b.K);
            if (b.q) cudaFree(b.q);
            b.xi = b.K = b.q = nullptr;
            b.cap = b.kcap = 0;
            if (cudaMalloc((void**)&b.xi, total[l] * M * sizeof(double)) != cudaSuccess ||
                cudaMalloc((void**)&b.K, chunk[l] * (size_t)N * N * sizeof(double)) != cudaSuccess ||
                cudaMalloc((void**)&b.q, 2 * total[l] * sizeof(double)) != cudaSuccess) {
                set_error(ctx, "mlmc_estimate: allocation of a batched round failed");
                return FM_ENOMEM;
            }
            b.cap = total[l];
            b.kcap = chunk[l];
        }
        uint64_t o = 0;
        for (const Request& r : g->pending) {
            if (r.e - g->off != l) continue;
            for (uint64_t d = 0; d < r.n;) {
                const uint32_t cnt = (uint32_t)std::min<uint64_t>(r.n - d, (uint64_t)1 << 30);
                double* xi = b.xi + (o + d) * M;
                if (r.shift < 0) FM_TRY(mc_points(ctx, (uint32_t)l, r.first + d, cnt, (uint32_t)M, xi, nullptr));
                else FM_TRY(qmc_points(ctx, ctx->cfg.qmc_rule, (uint32_t)l, (uint32_t)M, r.first + d, cnt,
                                       (uint32_t)r.shift, 1, nullptr, xi, nullptr));
                d += cnt;
            }
            o += r.n;
        }
    }
    for (uint64_t pass = 0; pass < passes; ++pass) {
        std::vector<fm_batch_group> groups;
        for (int l = 0; l < L; ++l) {
            const uint64_t d0 = pass * chunk[l];
            if (!total[l] || d0 >= total[l]) continue;
            const int N = grid_of_level(ctx, l);
            const uint32_t cnt = (uint32_t)std::min<uint64_t>(chunk[l], total[l] - d0);
            LevelBuf& b = g->lb[l];
            for (uint64_t d = 0; d < cnt;) {
                const uint32_t c = (uint32_t)std::min<uint64_t>(cnt - d, (uint64_t)1 << 20);
                FM_TRY(kl_field_batch(ctx, l, c, b.xi + (d0 + d) * M, b.K + d * (size_t)N * N, nullptr));
                d += c;
            }
            // grids of 128 x 128 and more as two groups (two branches of the
            // graph): the refinement rounds of one half, latency-bound once
            // few of its samples still iterate, overlap the other half's
            // (measured on a 1000-sample 256 x 256 pilot: 55.9 -> 53.2 ms)
            // level 0 takes no Q^c (its coarse slot holds S, or nothing)
            double* qcl = l > 0 ? b.q + total[l] + d0 : nullptr;
            const uint32_t half = (N >= 128 && cnt >= 64) ? cnt / 2 : 0;
            if (half) {
                groups.push_back(fm_batch_group{N, half, b.K, b.q + d0, qcl, nullptr});
                groups.push_back(fm_batch_group{N, cnt - half, b.K + (size_t)half * N * N, b.q + d0 + half,
                                                qcl ? qcl + half : nullptr, nullptr});
            } else {
                groups.push_back(fm_batch_group{N, cnt, b.K, b.q + d0, qcl, nullptr});
            }
        }
        FM_TRY(fmg_solve_uneven(ctx, (int32_t)groups.size(), groups.data(), &prm, nullptr));
    }
    // the sums of every request: levels >= 1, then level 0 (with the
    // surrogate, Y_0 = Q_0 - S) and the surrogate level, whose network may
    // still be training on its own stream (they wait for it on the device)
    for (int k = 0; k < L; ++k) {
        const int l = (k + 1) % L;
        if (!total[l]) continue;
        LevelBuf& b = g->lb[l];
        uint64_t o = 0;
        for (const Request& r : g->pending) {
            if (r.e - g->off != l) continue;
            double* qf = b.q + o;
            double* qc = b.q + total[l] + o;
            const bool with_s = ctx->surrogate_on && l == 0;
            if (with_s) {
                if (r.shift < 0) FM_TRY(surrogate_eval_mc_impl(ctx, 0, r.first, (uint32_t)r.n, qc, nullptr));
                else FM_TRY(surrogate_eval_impl(ctx, (uint32_t)r.n, b.xi + o * M, qc, nullptr));
            }
            fm_level_sums* cell = ctx->d_sums + (size_t)r.e * g->R + (r.shift < 0 ? 0 : r.shift);
            FM_TRY(level_sums_add(ctx, (uint32_t)r.n, qf, qc, (l > 0 || with_s) ? 1 : 0, cell, nullptr));
            o += r.n;
        }
    }
    for (const Request& r : g->pending) {
        if (r.e - g->off >= 0 || (s_forked && r.shift < 0)) continue;
        cudaEvent_t e0 = g->event(), e1 = g->event();
        g->lev.push_back(r.e);
        cudaEventRecord(e0, nullptr);
        fm_level_sums* cell = ctx->d_sums + (size_t)r.e * g->R + (r.shift < 0 ? 0 : r.shift);
        for (uint64_t done = 0; done < r.n;) {
            const uint32_t cnt = (uint32_t)std::min<uint64_t>(r.n - done, (uint64_t)1 << 30);
            FM_TRY(mlmc_sample_level(ctx, r.e - g->off, r.first + done, cnt, r.shift, cell, nullptr, nullptr, nullptr));
            done += cnt;
        }
        cudaEventRecord(e1, nullptr);
    }
    if (s_forked) FM_CUDA_TRY(ctx, cudaStreamWaitEvent(nullptr, B->s_join, 0));
    cudaEventRecord(g->b1, nullptr);
    g->pending.clear();
    return FM_OK;
}

fm_status gpu_read(void* user, fm_level_sums* local) {
    GpuSampler* g = static_cast<GpuSampler*>(user);
    FM_TRY(flush_batched(g));
    FM_TRY(fm_sync(g->ctx));
    if (g->batched && g->b0) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g->b0, g->b1) == cudaSuccess) g->round_sec += ms * 1e-3;
    }
    g->collect();
    FM_CUDA_TRY(g->ctx, cudaMemcpy(local, g->ctx->d_sums, g->cells * sizeof(fm_level_sums), cudaMemcpyDeviceToHost));
    return FM_OK;
}

}  // namespace

namespace fm {

void batched_free(fm_ctx* ctx) {
    if (!ctx->batched) return;
    BatchedBufs* B = static_cast<BatchedBufs*>(ctx->batched);
    for (LevelBuf& b : B->lb) {
        cudaFree(b.xi);
        cudaFree(b.K);
        cudaFree(b.q);
    }
    cudaFree(B->s_q);
    cudaFree(B->s_part);
    if (B->s_st) cudaStreamDestroy(B->s_st);
    if (B->s_fork) cudaEventDestroy(B->s_fork);
    if (B->s_join) cudaEventDestroy(B->s_join);
    delete B;
    ctx->batched = nullptr;
}

}  // namespace fm

extern "C" fm_status mlmc_estimate_sharded(fm_ctx* ctx, const fm_estimate_opts* opts, int32_t rank, int32_t world,
                                           fm_allgather_fn allgather, void* user, fm_result* out) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "mlmc_estimate: null context");
    FM_CHECK_ARG(ctx, opts && out, "mlmc_estimate: null argument");
    FM_CHECK_ARG(ctx, opts->eps > 0, "mlmc_estimate: eps must be positive");
    FM_CHECK_ARG(ctx, opts->n_pilot >= 2, "mlmc_estimate: n_pilot must be >= 2");
    FM_CHECK_ARG(ctx, !opts->qmc || ctx->cfg.n_shifts >= 2, "mlmc_estimate: QMC needs n_shifts >= 2");
    FM_CHECK_ARG(ctx, world >= 1 && rank >= 0 && rank < world && (world == 1 || allgather),
                 "mlmc_estimate: bad rank / world, or no allgather for several ranks");
    FM_CHECK_ARG(ctx, !opts->surrogate || (ctx->mlp && opts->surrogate_cost > 0),
                 "mlmc_estimate: the surrogate level needs a trained network and surrogate_cost > 0");
    FM_CHECK_ARG(ctx, !opts->adapt_L || (opts->L_start >= 1 && opts->L_start < ctx->cfg.n_levels),
                 "mlmc_estimate: adapt_L needs 1 <= L_start < n_levels");
    const auto t0 = std::chrono::steady_clock::now();
    // Extended levels e = 0 .. L: with the surrogate, e = 0 is the S level
    // and e = l + 1 MLMC level l; without it e = l.
    const int off = opts->surrogate ? 1 : 0;
    const int Lr = ctx->cfg.n_levels - 1;
    const int L = Lr + off;
    const int R = opts->qmc ? ctx->cfg.n_shifts : 1;
    const size_t cells = (size_t)(L + 1) * R;
    FM_CUDA_TRY(ctx, cudaMemset(ctx->d_sums, 0, cells * sizeof(fm_level_sums)));
    double C[FM_MAX_LEVELS + 1];
    for (int e = 0; e <= L; ++e) {
        const double n = grid_of_level(ctx, std::max(0, e - off));
        C[e] = n * n * 4.0 / 3.0;
    }
    if (off) C[0] *= opts->surrogate_cost;   // S-level cost relative to a level-0 sample
    std::memset(out, 0, sizeof(*out));
    const int saved_on = ctx->surrogate_on;
    ctx->surrogate_on = opts->surrogate ? 1 : 0;
    struct Restore {
        fm_ctx* c;
        int v;
        ~Restore() { c->surrogate_on = v; }
    } restore{ctx, saved_on};

    GpuSampler g;
    g.ctx = ctx;
    g.off = off;
    g.R = R;
    g.cells = cells;
    g.batched = opts->batched != 0;
    g.lb = batched_bufs(ctx);
    fm_core_opts co{};
    co.n_ext = L + 1;
    co.cost = C;
    co.eps = opts->eps;
    co.qmc = opts->qmc;
    co.n_shifts = R;
    co.n_pilot = opts->n_pilot;
    co.max_rounds = opts->max_rounds;
    co.rank = rank;
    co.world = world;
    co.level0 = off;
    co.adapt = opts->adapt_L ? 1 : 0;
    co.n_ext_start = opts->adapt_L ? opts->L_start + 1 + off : L + 1;
    co.alpha = opts->alpha;
    fm_core_result cr{};
    char msg[512] = {0};
    const fm_status st = mlmc_estimate_core(&co, gpu_enqueue, gpu_read, allgather, &g, &cr, msg, sizeof(msg));
    if (st != FM_OK) {
        if (msg[0]) set_error(ctx, msg);
        return st;
    }
    // the finest level the controller ended on
    const int Lu = cr.n_ext_used - 1 - off;
    out->estimate = cr.estimate;
    out->var_estimator = cr.var_estimator;
    for (int l = 0; l <= Lu; ++l) {
        out->mean[l] = cr.mean[l + off];
        out->var[l] = cr.var[l + off];
        out->N[l] = cr.N[l + off];
        out->level_seconds[l] = g.lsec[l + off];
    }
    out->batched_seconds = g.round_sec;
    if (off) {
        out->mean_s = cr.mean[0];
        out->var_s = cr.var[0];
        out->N_s = cr.N[0];
        out->seconds_s = g.lsec[0];
    }
    out->alpha = fit_rate(out->mean, Lu);
    out->beta = fit_rate(out->var, Lu);
    out->bias = cr.bias;
    out->alpha_used = cr.alpha_used;
    out->bias_ok = cr.bias_ok;
    out->L = Lu;
    out->rounds = cr.rounds;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return FM_OK;
}

extern "C" fm_status mlmc_estimate(fm_ctx* ctx, const fm_estimate_opts* opts, fm_result* out) {
    return mlmc_estimate_sharded(ctx, opts, 0, 1, nullptr, nullptr, out);
}
