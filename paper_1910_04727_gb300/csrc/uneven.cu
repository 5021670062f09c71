// Uneven batches: groups of samples with different grid sizes solved in one
// CUDA graph.
//
// Every group gets a branch of its own (fork and join events around it):
// groups where FM_KERNEL_AUTO takes the resident kernel run it (a
// persistent grid, one sample per CTA or warp), the others the level-wise
// schedule with its scratch in an arena of the group's own.  The converged
// stages of the level-wise schedule loop on the device (a conditional WHILE
// node per refined stage), so nothing in the graph waits for the host.
// Branches run concurrently: one group's latency-bound coarse grids and
// residual tests overlap another group's bandwidth-bound fine grids, and
// the graph removes the gaps between the thousands of small launches.
//
// Executable graphs are kept in the context by shape (groups, grids,
// schedule), a few of them: a later call with a kept shape only updates the
// kernel parameters (cudaGraphExecUpdate), a new shape is instantiated.  An
// estimator's rounds alternate between shapes (the pilot round solves every
// level, later rounds a few), so keeping one graph per shape saves an
// instantiation per round.
#include <algorithm>
#include <functional>
#include <vector>

#include "common.cuh"

namespace fm {

struct UnevenState {
    std::vector<Arena> arenas;        // level-wise scratch, one per group
    // branch streams by priority (index: priority - prio_hi), a branch per group
    std::vector<cudaStream_t> side[fm_ctx::kPrioLevels];
    std::vector<cudaEvent_t> join;    // one per group
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;       // capture origin
    struct Kept {
        std::vector<int64_t> key;
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    std::vector<Kept> kept;           // at most kKeptGraphs, the least recently used replaced
    uint64_t tick = 0;
    int64_t instantiations = 0, updates = 0, launches = 0;
};

constexpr size_t kKeptGraphs = 8;

static UnevenState* uneven_state(fm_ctx* ctx) { return static_cast<UnevenState*>(ctx->uneven); }

void uneven_free(fm_ctx* ctx) {
    UnevenState* U = uneven_state(ctx);
    if (!U) return;
    for (Arena& a : U->arenas) cudaFree(a.base);
    for (const std::vector<cudaStream_t>& v : U->side)
        for (cudaStream_t s : v) cudaStreamDestroy(s);
    for (cudaEvent_t e : U->join) cudaEventDestroy(e);
    if (U->fork) cudaEventDestroy(U->fork);
    if (U->cap) cudaStreamDestroy(U->cap);
    for (UnevenState::Kept& k : U->kept) cudaGraphExecDestroy(k.exec);
    delete U;
    ctx->uneven = nullptr;
}

// Branch priorities: the group of the largest grid (the batch's longest
// chain of launches) one below the device's greatest priority (the greatest
// is the surrogate's training stream), the next grid size one lower, and so
// on to the least priority.  A branch's kernel nodes, its refinement loops'
// bodies included, carry its priority, so the longest branch's launches are
// scheduled first and the shorter branches fill the SMs around them.
static std::vector<int> branch_priorities(const fm_ctx* ctx, int n_groups, const fm_batch_group* groups) {
    std::vector<int> sizes;
    for (int g = 0; g < n_groups; ++g) sizes.push_back(groups[g].n_fine);
    std::sort(sizes.begin(), sizes.end(), std::greater<int>());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    std::vector<int> prio(n_groups);
    for (int g = 0; g < n_groups; ++g) {
        const int r = (int)(std::find(sizes.begin(), sizes.end(), groups[g].n_fine) - sizes.begin());
        prio[g] = std::min(ctx->prio_hi + 1 + r, ctx->prio_lo);
    }
    return prio;
}

// Streams and events for n_groups branches of the given priorities: side
// stream of group g = the j-th stream of its priority, j counting the
// groups of that priority before g.
static fm_status uneven_prepare(fm_ctx* ctx, int n_groups, const std::vector<int>& prio,
                                std::vector<cudaStream_t>* branch) {
    if (!ctx->uneven) ctx->uneven = new UnevenState();
    UnevenState* U = uneven_state(ctx);
    if (!U->cap) {
        FM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&U->cap, cudaStreamNonBlocking));
        FM_CUDA_TRY(ctx, cudaEventCreateWithFlags(&U->fork, cudaEventDisableTiming));
    }
    while ((int)U->join.size() < n_groups) {
        cudaEvent_t e;
        FM_CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        U->join.push_back(e);
        U->arenas.emplace_back();
    }
    int used[fm_ctx::kPrioLevels] = {};
    branch->assign(n_groups, nullptr);
    for (int g = 0; g < n_groups; ++g) {
        const int pi = prio[g] - ctx->prio_hi;
        std::vector<cudaStream_t>& pool = U->side[pi];
        if (used[pi] == (int)pool.size()) {
            cudaStream_t s;
            FM_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio[g]));
            pool.push_back(s);
        }
        (*branch)[g] = pool[used[pi]++];
    }
    return FM_OK;
}

// Groups on the resident kernel: where FM_KERNEL_AUTO would take it.
static bool resident_grid(const fm_ctx* ctx, const fm_batch_group& G, const fm_solve_params& prm) {
    return prm.kernel != FM_KERNEL_LEVELWISE && auto_resident(G.n_fine, G.count, ctx->sms, prm);
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fmg_solve_uneven(fm_ctx* ctx, int32_t n_groups, const fm_batch_group* groups,
                                      const fm_solve_params* prm, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fmg_solve_uneven: null context");
    FM_CHECK_ARG(ctx, prm != nullptr && groups != nullptr, "fmg_solve_uneven: null argument");
    FM_CHECK_ARG(ctx, n_groups >= 1 && n_groups <= 64, "fmg_solve_uneven: 1 .. 64 groups");
    FM_CHECK_ARG(ctx, prm->kernel != FM_KERNEL_RESIDENT, "fmg_solve_uneven: the schedule is chosen per group");
    const int n0 = prm->n_coarsest;
    for (int g = 0; g < n_groups; ++g) {
        const fm_batch_group& G = groups[g];
        int m = 0;
        while (m < 16 && (n0 << m) < G.n_fine) ++m;
        FM_CHECK_ARG(ctx, n0 >= 2 && n0 <= 4 && G.n_fine >= n0 && (n0 << m) == G.n_fine && G.n_fine <= 8192,
                     "fmg_solve_uneven: group " + std::to_string(g) + ": n_fine must be n_coarsest * 2^m");
        FM_CHECK_ARG(ctx, G.count == 0 || (G.d_K && G.d_qf),
                     "fmg_solve_uneven: group " + std::to_string(g) + ": null input or output");
    }
    const std::vector<int> prio = branch_priorities(ctx, n_groups, groups);
    std::vector<cudaStream_t> branch;
    FM_TRY(uneven_prepare(ctx, n_groups, prio, &branch));
    UnevenState* U = uneven_state(ctx);
    // level-wise scratch is sized before the capture (no allocation inside it)
    for (int g = 0; g < n_groups; ++g) {
        const fm_batch_group& G = groups[g];
        if (G.count == 0 || resident_grid(ctx, G, *prm)) continue;
        const size_t need = fmg_levelwise_scratch(ctx, G.n_fine, G.count, *prm);
        Arena& a = U->arenas[g];
        if (a.capacity < need) {
            if (a.base) cudaFree(a.base);
            a.base = nullptr;
            a.capacity = 0;
            if (cudaMalloc((void**)&a.base, need) != cudaSuccess) {
                set_error(ctx, "fmg_solve_uneven: scratch allocation of " + std::to_string(need) + " bytes failed");
                return FM_ENOMEM;
            }
            a.capacity = need;
        }
    }
    FM_CUDA_TRY(ctx, cudaGetLastError());
    // capture: fork, one branch per group, join
    const bool prof = ctx->prof.active;
    ctx->prof.active = false;
    fm_status st = FM_OK;
    cudaGraph_t graph = nullptr;
    FM_CUDA_TRY(ctx, cudaStreamBeginCapture(U->cap, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(U->fork, U->cap);
    for (int g = 0; g < n_groups && st == FM_OK; ++g) {
        const fm_batch_group& G = groups[g];
        if (G.count == 0) continue;
        cudaStreamWaitEvent(branch[g], U->fork, 0);
        fm_solve_params p = *prm;
        p.kernel = resident_grid(ctx, G, *prm) ? FM_KERNEL_AUTO : FM_KERNEL_LEVELWISE;
        st = fmg_solve_with(ctx, U->arenas[g], G.n_fine, G.count, G.d_K, p, G.d_qf, G.d_qc, nullptr, G.d_status,
                            branch[g]);
        cudaEventRecord(U->join[g], branch[g]);
        cudaStreamWaitEvent(U->cap, U->join[g], 0);
    }
    const cudaError_t ce = cudaStreamEndCapture(U->cap, &graph);
    ctx->prof.active = prof;
    if (st != FM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error(ctx, std::string("fmg_solve_uneven: graph capture failed: ") + cudaGetErrorString(ce));
        cudaGetLastError();
        return FM_ECUDA;
    }
    // a kept graph of the same shape: update its parameters; otherwise instantiate
    std::vector<int64_t> key = {n_groups, prm->precision, prm->converged, prm->energy_step, prm->nu0, prm->nu1,
                                prm->nu2, prm->n_coarsest, prm->bc_case, prm->kernel, prm->ir_cycles};
    // per group: grid, non-empty, schedule, and whether Q^c is asked for (a
    // converged solve refines its coarse stage only then)
    for (int g = 0; g < n_groups; ++g)
        key.insert(key.end(), {groups[g].n_fine, groups[g].count > 0, resident_grid(ctx, groups[g], *prm),
                               groups[g].d_qc != nullptr});
    cudaGraphExec_t exec = nullptr;
    for (size_t i = 0; i < U->kept.size() && !exec; ++i) {
        if (U->kept[i].key != key) continue;
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(U->kept[i].exec, graph, &info) == cudaSuccess) {
            exec = U->kept[i].exec;
            U->kept[i].used = ++U->tick;
            ++U->updates;
        } else {   // same key, other topology (a changed smoother shape, say): replace it
            cudaGetLastError();
            cudaGraphExecDestroy(U->kept[i].exec);
            U->kept.erase(U->kept.begin() + (long)i);
        }
    }
    if (!exec) {
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(graph);
            set_error(ctx, std::string("fmg_solve_uneven: graph instantiation failed: ") + cudaGetErrorString(ie));
            return FM_ECUDA;
        }
        ++U->instantiations;
        if (U->kept.size() >= kKeptGraphs) {
            auto lru = std::min_element(U->kept.begin(), U->kept.end(),
                                        [](const UnevenState::Kept& a, const UnevenState::Kept& b) { return a.used < b.used; });
            cudaGraphExecDestroy(lru->exec);
            U->kept.erase(lru);
        }
        U->kept.push_back(UnevenState::Kept{key, exec, ++U->tick});
    }
    cudaGraphDestroy(graph);
    cudaStream_t s = as_stream(stream);
    double cells = 0.0;
    for (int g = 0; g < n_groups; ++g) cells += (double)groups[g].count * groups[g].n_fine * groups[g].n_fine;
    FM_TIMED(ctx, kFamUnevenGraph, s, 8.0 * cells, 0.0, cudaGraphLaunch(exec, s));
    ++U->launches;
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status fmg_uneven_stats(const fm_ctx* ctx, int64_t* instantiations, int64_t* updates,
                                      int64_t* launches) {
    if (!ctx) return FM_EINVAL;
    const UnevenState* U = static_cast<const UnevenState*>(ctx->uneven);
    if (instantiations) *instantiations = U ? U->instantiations : 0;
    if (updates) *updates = U ? U->updates : 0;
    if (launches) *launches = U ? U->launches : 0;
    return FM_OK;
}
