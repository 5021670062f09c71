// Context lifetime and error reporting of the C ABI.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace fm {

static thread_local std::string g_create_error;

void set_error(const fm_ctx* ctx, const std::string& msg) {
    if (ctx) const_cast<fm_ctx*>(ctx)->last_error = msg;
    else g_create_error = msg;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_create(const fm_config* cfg, fm_ctx** out) {
    FM_CHECK_ARG(nullptr, cfg && out, "fm_create: null argument");
    FM_CHECK_ARG(nullptr, cfg->n_levels >= 1 && cfg->n_levels <= FM_MAX_LEVELS, "fm_create: n_levels out of range");
    FM_CHECK_ARG(nullptr, cfg->n_coarsest >= 2 && cfg->n_coarsest <= 4, "fm_create: n_coarsest must be 2..4");
    int m = 0;
    while ((cfg->n_coarsest << m) < cfg->n_level0) ++m;
    FM_CHECK_ARG(nullptr, (cfg->n_coarsest << m) == cfg->n_level0,
                 "fm_create: n_level0 must be n_coarsest times a power of two");
    FM_CHECK_ARG(nullptr, ((int64_t)cfg->n_level0 << (cfg->n_levels - 1)) <= 8192, "fm_create: finest grid above 8192");
    FM_CHECK_ARG(nullptr, cfg->M >= 1 && cfg->M <= 4096, "fm_create: M must be in [1, 4096]");
    FM_CHECK_ARG(nullptr, cfg->sigma2 > 0 && cfg->lambda > 0, "fm_create: sigma2 and lambda must be positive");
    FM_CHECK_ARG(nullptr, cfg->nu0 >= 1 && cfg->nu1 >= 0 && cfg->nu2 >= 0 && cfg->nu1 + cfg->nu2 >= 1,
                 "fm_create: need nu0 >= 1 and nu1 + nu2 >= 1");
    FM_CHECK_ARG(nullptr, cfg->precision == FM_PREC_FP64 || cfg->precision == FM_PREC_MIXED,
                 "fm_create: unknown precision");
    FM_CHECK_ARG(nullptr, cfg->precision != FM_PREC_MIXED || cfg->converged,
                 "fm_create: the mixed form refines to a tolerance (converged = 1)");
    FM_CHECK_ARG(nullptr, !cfg->converged || (cfg->tol > 0 && cfg->max_cycles >= 1),
                 "fm_create: converged mode needs tol > 0 and max_cycles >= 1");
    FM_CHECK_ARG(nullptr, cfg->n_shifts >= 0 && cfg->n_shifts <= 64, "fm_create: n_shifts must be in [0, 64]");
    FM_CHECK_ARG(nullptr, cfg->kl_mode >= FM_KL_AUTO && cfg->kl_mode <= FM_KL_BF16X3, "fm_create: unknown kl_mode");
    FM_CHECK_ARG(nullptr, cfg->bc_case == 0 || cfg->bc_case == FM_CASE_I || cfg->bc_case == FM_CASE_II,
                 "fm_create: bc_case must be FM_CASE_I or FM_CASE_II");
    FM_CHECK_ARG(nullptr, cfg->nu == 0.0 || cfg->nu == 0.5 || cfg->nu == 1.0 || cfg->nu == 1.5 || cfg->nu == 2.5,
                 "fm_create: nu must be 0.5, 1, 1.5 or 2.5");
    FM_CHECK_ARG(nullptr, cfg->qmc_rule >= FM_QMC_SOBOL_SHIFT && cfg->qmc_rule <= FM_QMC_LATTICE,
                 "fm_create: unknown qmc_rule");
    FM_CHECK_ARG(nullptr, cfg->lattice_m == 0 || (cfg->lattice_m >= 5 && cfg->lattice_m <= 24),
                 "fm_create: lattice_m must be 5 .. 24");
    FM_CHECK_ARG(nullptr, cfg->ir_cycles >= 0 && cfg->ir_cycles <= 64, "fm_create: ir_cycles must be 0 .. 64");
    FM_CHECK_ARG(nullptr, !cfg->energy_step || cfg->converged,
                 "fm_create: the energy-optimal step runs in converged mode");
    fm_ctx* ctx = new (std::nothrow) fm_ctx();
    if (!ctx) {
        set_error(nullptr, "fm_create: host allocation failed");
        return FM_ENOMEM;
    }
    ctx->cfg = *cfg;
    if (ctx->cfg.lattice_m == 0) ctx->cfg.lattice_m = 16;
    cudaGetDevice(&ctx->device);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (sobol_direction_numbers_host((uint32_t)cfg->M, ctx->h_sobol_V) != 0) {
        delete ctx;
        set_error(nullptr, "fm_create: Sobol' direction numbers unavailable for this M");
        return FM_EINVAL;
    }
    const size_t vbytes = ctx->h_sobol_V.size() * sizeof(uint32_t);
    const size_t sums = (size_t)(cfg->n_levels + 1) * (cfg->n_shifts > 0 ? cfg->n_shifts : 1);
    if (cudaMalloc((void**)&ctx->d_sobol_V, vbytes) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_sums, sums * sizeof(fm_level_sums)) != cudaSuccess) {
        fm_destroy(ctx);
        set_error(nullptr, "fm_create: device allocation failed");
        return FM_ENOMEM;
    }
    if (cudaMemcpy(ctx->d_sobol_V, ctx->h_sobol_V.data(), vbytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        fm_destroy(ctx);
        set_error(nullptr, "fm_create: copy of the direction numbers failed");
        return FM_ECUDA;
    }
    if (cfg->qmc_rule == FM_QMC_LATTICE) {
        const int mm = ctx->cfg.lattice_m;
        const std::vector<uint32_t>* z = lattice_vector_cached((uint32_t)cfg->M, lattice_m_min(mm), mm);
        if (!z || cudaMalloc((void**)&ctx->d_lattice_z, z->size() * sizeof(uint32_t)) != cudaSuccess ||
            cudaMemcpy(ctx->d_lattice_z, z->data(), z->size() * sizeof(uint32_t), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            fm_destroy(ctx);
            set_error(nullptr, "fm_create: lattice generating vector unavailable");
            return FM_ENOMEM;
        }
        ctx->h_lattice_z = *z;
    }
    cudaDeviceGetStreamPriorityRange(&ctx->prio_lo, &ctx->prio_hi);
    ctx->prio_lo = std::min(ctx->prio_lo, ctx->prio_hi + fm_ctx::kPrioLevels - 1);
    for (int p = ctx->prio_hi; p <= ctx->prio_lo; ++p) {
        if (cudaStreamCreateWithPriority(&ctx->body_stream[p - ctx->prio_hi], cudaStreamNonBlocking, p) !=
            cudaSuccess) {
            fm_destroy(ctx);
            set_error(nullptr, "fm_create: stream creation failed");
            return FM_ECUDA;
        }
    }
    fmg_init_attributes();
    resident_init_attributes();
    *out = ctx;
    return FM_OK;
}

extern "C" void fm_destroy(fm_ctx* ctx) {
    if (!ctx) return;
    for (int l = 0; l < FM_MAX_LEVELS; ++l) cudaFree(ctx->d_basis[l]);
    cudaFree(ctx->d_sobol_V);
    cudaFree(ctx->d_lattice_z);
    cudaFree(ctx->arena.base);
    cudaFree(ctx->d_xi);
    cudaFree(ctx->d_K);
    cudaFree(ctx->d_q);
    cudaFree(ctx->d_sums);
    cudaFree(ctx->d_partials);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    cudaFree(ctx->prof.counters);
    mlp_free(ctx);
    uneven_free(ctx);
    batched_free(ctx);
    for (cudaStream_t s : ctx->body_stream)
        if (s) cudaStreamDestroy(s);
    for (int l = 0; l < FM_MAX_LEVELS; ++l) cudaFree(ctx->tc.basis[l]);
    cudaFree(ctx->tc.xi);
    cudaFree(ctx->tc.err);
    delete ctx;
}

extern "C" fm_status surrogate_enable(fm_ctx* ctx, int32_t on) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "surrogate_enable: null context");
    ctx->surrogate_on = on ? 1 : 0;
    return FM_OK;
}

extern "C" fm_status fm_sync(fm_ctx* ctx) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_sync: null context");
    FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (ctx->tc.err) {
        int e = 0;
        FM_CUDA_TRY(ctx, cudaMemcpy(&e, ctx->tc.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            // reported once: the flag is cleared for the calls that follow
            FM_CUDA_TRY(ctx, cudaMemset(ctx->tc.err, 0, sizeof(int)));
            set_error(ctx, "a bounded device-side wait of the tensor-core kernels ran out");
            return FM_ETIMEOUT;
        }
    }
    if (surrogate_err_flag(ctx)) {
        set_error(ctx, "a bounded device-side wait of the surrogate network ran out");
        return FM_ETIMEOUT;
    }
    return FM_OK;
}

extern "C" const char* fm_last_error(const fm_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}
