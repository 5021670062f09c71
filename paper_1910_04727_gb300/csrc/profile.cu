// Event-pair timing of kernel families for roofline reports.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fm {

static const char* kFamilyNames[kFamilyCount] = {
    "points", "kl_gemm_exp", "inject", "coefficients", "stage_rhs", "rbgs_smoother",
    "residual_restrict", "prolong_correct", "fmg_interpolate", "coarse_inverse",
    "coarse_solve", "outflux", "level_sums", "fmg_resident", "mlp_gemm", "mlp_train_graph",
    "uneven_graph", "rbgs_tile", "rbgs_strip", "vcycle_tail"};

int prof_start(fm_ctx* ctx, int family, cudaStream_t st) {
    Profiler& P = ctx->prof;
    if (!P.active || !((P.mask >> family) & 1u)) return -1;
    while (P.pool.size() < P.pool_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        P.pool.push_back(e);
    }
    ProfRecord r;
    r.family = family;
    r.start = P.pool[P.pool_used++];
    r.stop = P.pool[P.pool_used++];
    cudaEventRecord(r.start, st);
    P.records.push_back(r);
    return (int)P.records.size() - 1;
}

constexpr int kMaxCounters = 1 << 14;

double* prof_counter(fm_ctx* ctx, int idx) {
    Profiler& P = ctx->prof;
    if (idx < 0 || P.counters_used + kCountersPerRecord > kMaxCounters) return nullptr;
    if (!P.counters) {
        if (cudaMalloc((void**)&P.counters, kMaxCounters * sizeof(double)) != cudaSuccess) {
            P.counters = nullptr;
            return nullptr;
        }
        cudaMemset(P.counters, 0, kMaxCounters * sizeof(double));
    }
    P.records[idx].counter = P.counters_used;
    double* c = P.counters + P.counters_used;
    P.counters_used += kCountersPerRecord;
    return c;
}

void prof_stop(fm_ctx* ctx, int idx, cudaStream_t st, double bytes, double flops) {
    if (idx < 0) return;
    ProfRecord& r = ctx->prof.records[idx];
    cudaEventRecord(r.stop, st);
    r.bytes = bytes;
    r.flops = flops;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_profile_begin(fm_ctx* ctx, uint32_t family_mask) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_profile_begin: null context");
    ctx->prof.active = true;
    ctx->prof.mask = family_mask;
    ctx->prof.records.clear();
    ctx->prof.pool_used = 0;
    if (ctx->prof.counters) cudaMemset(ctx->prof.counters, 0, kMaxCounters * sizeof(double));
    ctx->prof.counters_used = 0;
    return FM_OK;
}

extern "C" fm_status fm_profile_end(fm_ctx* ctx, fm_kernel_stat* stats, int32_t max_stats,
                                    int32_t* n_stats) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_profile_end: null context");
    ctx->prof.active = false;
    FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    fm_kernel_stat acc[kFamilyCount];
    for (int f = 0; f < kFamilyCount; ++f) acc[f] = fm_kernel_stat{f, 0, 0.0, 0.0, 0.0, 0.0};
    std::vector<double> counted(ctx->prof.counters_used);
    if (!counted.empty())
        FM_CUDA_TRY(ctx, cudaMemcpy(counted.data(), ctx->prof.counters, counted.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost));
    for (const ProfRecord& r : ctx->prof.records) {
        float ms = 0.0f;
        FM_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, r.start, r.stop));
        fm_kernel_stat& a = acc[r.family];
        a.launches += 1;
        a.ms += ms;
        if (r.counter >= 0) {
            // counted by the kernel: [flops, of which FP64, model bytes]
            const double* c = &counted[r.counter];
            a.flops += r.flops + c[0];
            a.flops_fp64 += c[1];
            a.bytes += c[2] > 0.0 ? c[2] : r.bytes;
        } else {
            a.flops += r.flops;
            a.bytes += r.bytes;
        }
    }
    int out = 0;
    for (int f = 0; f < kFamilyCount; ++f)
        if (acc[f].launches > 0 && out < max_stats && stats) stats[out++] = acc[f];
    if (n_stats) *n_stats = out;
    ctx->prof.records.clear();
    return FM_OK;
}

extern "C" const char* fm_kernel_family_name(int32_t family) {
    return (family >= 0 && family < kFamilyCount) ? kFamilyNames[family] : nullptr;
}
