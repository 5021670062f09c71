// Internal definitions shared by the translation units of libfmgmlmc.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "fmgmlmc.h"

namespace fm {

// ------------------------------------------------------------------ Philox
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
// (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2, c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0),
// with the key bumped by the Weyl constants between rounds.
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ULL;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ULL;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73BULL;

// Stream purposes (high half of key[1]).
constexpr uint64_t kPurposeMC = 1;
constexpr uint64_t kPurposeShift = 2;
constexpr uint64_t kPurposeSobolDir = 3;
constexpr uint64_t kPurposeLatticeShift = 4;
constexpr uint64_t kPurposeOwen = 5;
constexpr uint64_t kSobolDirSeed = 0x1910047270ULL;

struct u64x4 {
    uint64_t v[4];
};

__host__ __device__ inline void mulhilo64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
    hi = __umul64hi(a, b);
    lo = a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

__host__ __device__ inline u64x4 philox4x64(u64x4 c, uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(kPhiloxM0, c.v[0], hi0, lo0);
        mulhilo64(kPhiloxM1, c.v[2], hi1, lo1);
        u64x4 n = {{hi1 ^ c.v[1] ^ k0, lo1, hi0 ^ c.v[3] ^ k1, lo0}};
        c = n;
    }
    return c;
}

// ------------------------------------------------------------------ boundary data
// Boundary data of a problem (Table 1): Dirichlet values g[0..3] on the
// west, east, south and north edges; ns = 1 when the north and south edges
// are Dirichlet (Case I), 0 when they are no-flow (Case II, where g[2] and
// g[3] are unused).
struct Bnd {
    double g[4];
    int ns;
};

// Ghost values of a prolongation: the boundary data of the function being
// interpolated (zero for an error), in its arithmetic U.
template <typename U>
struct Ghost {
    U w, e, s, n;
    int ns;
};

// The schedule FM_KERNEL_AUTO takes for a grid: the resident kernel where it
// is the faster one on GB300 (up to 32 x 32 in the mixed form, 16 x 16 in
// FP64), the level-wise schedule (with its V-cycle tail below 32 x 32) above
// and for the energy-optimal step, which the resident kernel lacks.
// Measured per grid, samples per second of resident over level-wise:
// 16 x 16 2.0x (mixed), 1.1x (FP64, two cycles per stage), 1.2x (FP64
// converged); 64 x 64 0.82x, 0.89x, 1.04x; 32 x 32 0.93x and 0.84x in FP64,
// level in the mixed form (0.97x alone, ahead inside the five-level estimate).
// The resident kernel for grids up to 32 x 32 in the mixed form (16 x 16 in
// FP64); also for a converged mixed 64 x 64 batch of at most two samples per
// SM: one CTA per sample then finishes in one or two waves, where the
// level-wise schedule is a latency-bound chain of small launches.
inline bool auto_resident(int n_fine, size_t S, int sms, const fm_solve_params& prm) {
    if (prm.energy_step) return false;
    if (prm.precision == FM_PREC_MIXED && prm.converged && n_fine == 64 && S <= 2 * (size_t)sms) return true;
    return n_fine <= (prm.precision == FM_PREC_MIXED ? 32 : 16);
}

// V-cycles between residual tests of a converged stage.
inline int cycles_per_test(const fm_solve_params& prm) { return prm.ir_cycles > 0 ? prm.ir_cycles : prm.nu0; }

inline Bnd bnd_of(const fm_solve_params& prm) {
    Bnd b;
    b.ns = prm.bc_case == FM_CASE_I ? 1 : 0;
    b.g[0] = prm.pW;
    b.g[1] = prm.pE;
    b.g[2] = b.ns ? prm.pS : 0.0;
    b.g[3] = b.ns ? prm.pN : 0.0;
    return b;
}

// The Dirichlet data of cell (i, j) of an n x n grid moved to the right-hand
// side: 2 k g for every Dirichlet boundary face of the cell (coefficient k).
__host__ __device__ inline double dirichlet_rhs(const Bnd& b, int n, int i, int j, double k) {
    double v = 0.0;
    if (i == 0) v += 2.0 * k * b.g[0];
    if (i == n - 1) v += 2.0 * k * b.g[1];
    if (b.ns && j == 0) v += 2.0 * k * b.g[2];
    if (b.ns && j == n - 1) v += 2.0 * k * b.g[3];
    return v;
}

// ------------------------------------------------------------------ covariance (Sec. 3.1)
// x K_1(x), x >= 0, the shape of the Matern nu = 1 covariance (K_1 the
// modified Bessel function of the second kind; the limit at 0 is 1).
//   x <= 2: the ascending series (DLMF 10.31.1 with n = 1),
//     x K_1(x) = 1 + x ln(x/2) I_1(x)
//                - (x^2/4) sum_k (psi(k+1) + psi(k+2)) (x^2/4)^k / (k! (k+1)!),
//     I_1(x) = (x/2) sum_k (x^2/4)^k / (k! (k+1)!), psi(k+1) = H_k - gamma;
//   x > 2: the integral K_1(x) = int_0^inf exp(-x cosh t) cosh t dt (DLMF
//     10.32.9) by the trapezoidal rule, which converges exponentially for
//     this analytic, rapidly decaying integrand; the step follows the
//     integrand's width near t = 0, about 1 / sqrt(x).
// Relative error below 2e-14 on [0, 200] against an independent evaluation.
__host__ __device__ inline double xk1(double x) {
    if (x <= 0.0) return 1.0;
    if (x <= 2.0) {
        const double z = 0.25 * x * x;
        const double gamma = 0.57721566490153286061;
        double term = 1.0, i1 = 0.0, s = 0.0, H = 0.0;
        for (int k = 0; k < 40; ++k) {
            const double psi1 = H - gamma, psi2 = H + 1.0 / (k + 1) - gamma;
            i1 += term;
            s += (psi1 + psi2) * term;
            H += 1.0 / (k + 1);
            term *= z / ((double)(k + 1) * (k + 2));
            if (term < 1e-18 * i1) break;
        }
        return 1.0 + x * log(0.5 * x) * (0.5 * x * i1) - z * s;
    }
    const double h = fmin(0.25, 0.5 / sqrt(x));
    double acc = 0.5;   // t = 0, half weight
    for (int j = 1; j < 4096; ++j) {
        const double t = j * h, c = cosh(t);
        const double v = exp(-x * (c - 1.0)) * c;
        acc += v;
        if (v < 1e-18 * acc) break;
    }
    return x * exp(-x) * acc * h;
}

// Matern covariance of Sec. 3.1 at distance d >= 0 for the smoothness values
// this library builds bases for: nu = 1/2 (exponential), 1 (through x K_1),
// 3/2 and 5/2 (their closed forms); 0 for any other nu.
__host__ __device__ inline double matern(double nu, double sigma2, double lambda, double d) {
    if (nu == 0.5) return sigma2 * exp(-d / lambda);
    if (nu == 1.0) return sigma2 * xk1(sqrt(2.0) * d / lambda);
    if (nu == 1.5) {
        const double x = sqrt(3.0) * d / lambda;
        return sigma2 * (1.0 + x) * exp(-x);
    }
    if (nu == 2.5) {
        const double x = sqrt(5.0) * d / lambda;
        return sigma2 * (1.0 + x + x * x / 3.0) * exp(-x);
    }
    return 0.0;
}

// ------------------------------------------------------------------ errors
#define FM_CUDA_TRY(ctx, expr)                                                        \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            fm::set_error((ctx), std::string(#expr) + ": " + cudaGetErrorString(e_)); \
            return FM_ECUDA;                                                          \
        }                                                                             \
    } while (0)

#define FM_CHECK_ARG(ctx, cond, msg)                   \
    do {                                               \
        if (!(cond)) {                                 \
            fm::set_error((ctx), std::string(msg));    \
            return FM_EINVAL;                          \
        }                                              \
    } while (0)

#define FM_TRY(expr)                 \
    do {                             \
        fm_status s_ = (expr);       \
        if (s_ != FM_OK) return s_;  \
    } while (0)

void set_error(const fm_ctx* ctx, const std::string& msg);

// ------------------------------------------------------------------ profiling
enum Family {
    kFamPoints = 0, kFamKlGemm, kFamInject, kFamCoefficients, kFamStageRhs, kFamSmoother,
    kFamResidualRestrict, kFamProlong, kFamFmgInterp, kFamCoarseInverse, kFamCoarseSolve,
    kFamOutflux, kFamLevelSums, kFamResidentFmg, kFamMlp, kFamMlpTrain, kFamUnevenGraph, kFamSmootherTile,
    kFamSmootherStrip, kFamVcycleTail, kFamilyCount
};

struct ProfRecord {
    int family;
    cudaEvent_t start, stop;
    double bytes = 0.0, flops = 0.0;
    int counter = -1;   // device flop counter the kernel adds to (-1: none)
};

struct Profiler {
    bool active = false;
    uint32_t mask = 0;
    std::vector<ProfRecord> records;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    double* counters = nullptr;   // device flop counters of kernels that count their own work
    int counters_used = 0;
};

// ------------------------------------------------------------------ arena
// A grow-only device buffer the context hands out in 256-byte-aligned pieces.
struct Arena {
    char* base = nullptr;
    size_t capacity = 0;
    size_t used = 0;
};

// Smoother launch shape per (precision, grid): chosen by fm_autotune.
struct TuneTable {
    int32_t n[2][16] = {};        // grid the entry was tuned for (0: none)
    int32_t tile[2][16] = {};     // tile interior (0: one launch per colour, -1: column strips)
    int32_t threads[2][16] = {};
};

// Tensor-core KL synthesis state (kl_tc.cu).
struct TcState {
    bool ready = false;
    int split = 0, Mpad = 0, Kp = 0;
    void* basis[FM_MAX_LEVELS] = {};   // BF16 [cells][Kp] per level
    CUtensorMap mapA[FM_MAX_LEVELS];
    CUtensorMap mapB;
    void* xi = nullptr;                // BF16 [capacity][Kp]
    size_t xi_capacity = 0, mapB_rows = 0;
    int* err = nullptr;                // device flag: a bounded wait ran out
};

}  // namespace fm

struct fm_ctx {
    fm_config cfg{};
    int device = 0;
    int sms = 0;   // multiprocessors of the device
    std::string last_error;
    // KL basis per MLMC level: [n_l^2][M] FP64, row-subsets of the finest grid's basis.
    double* d_basis[FM_MAX_LEVELS] = {};
    bool basis_ready = false;
    // Sobol' direction numbers [M][32] (device and host copies).
    uint32_t* d_sobol_V = nullptr;
    std::vector<uint32_t> h_sobol_V;
    // lattice generating vector [M] (device and host copies; FM_QMC_LATTICE)
    uint32_t* d_lattice_z = nullptr;
    std::vector<uint32_t> h_lattice_z;
    // scratch
    fm::Arena arena;
    double* d_xi = nullptr;          // points of the current batch
    size_t xi_capacity = 0;
    double* d_K = nullptr;           // fields of the current batch
    size_t K_capacity = 0;
    double* d_q = nullptr;           // Q^f, Q^c of the current batch
    size_t q_capacity = 0;
    fm_level_sums* d_sums = nullptr; // [n_levels][max(1, n_shifts)] for mlmc_estimate
    double* d_partials = nullptr;    // per-block partial sums of the level-sum kernel
    size_t partial_capacity = 0;
    fm::Profiler prof;
    fm::TcState tc;
    void* mlp = nullptr;             // surrogate network state (mlp.cu)
    int surrogate_on = 0;            // level -1 = S(xi), level 0 = Q_0 - S(xi)
    // Streams that capture the bodies of device-side refinement loops, one
    // per stream priority (index: priority - prio_hi), so that a loop body's
    // kernel nodes carry the priority of the branch that captured it.
    static constexpr int kPrioLevels = 8;
    cudaStream_t body_stream[kPrioLevels] = {};
    int prio_hi = 0, prio_lo = 0;   // greatest (numerically lowest) and least stream priority
    fm::TuneTable tune;              // smoother launch shapes (fm_autotune)
    void* uneven = nullptr;          // uneven-batch executor state (uneven.cu)
    void* batched = nullptr;         // buffers of batched estimator rounds, kept across estimates (mlmc.cu)
    int fused_infer = 1;             // MC surrogate evaluation in one fused kernel (inputs up to 256 wide)
    int tail_max = 32;               // level-wise V-cycles: grids <= tail_max below the top run as one
                                     // resident tail kernel (0: per-grid launches throughout)
};

namespace fm {

// Grows *buf to hold `count` elements of T; previous contents are dropped.
template <typename T>
fm_status ensure(fm_ctx* ctx, T** buf, size_t* capacity, size_t count) {
    if (*capacity >= count && *buf) return FM_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *capacity = 0;
    if (cudaMalloc((void**)buf, sizeof(T) * count) != cudaSuccess) {
        set_error(ctx, "device allocation of " + std::to_string(sizeof(T) * count) + " bytes failed");
        return FM_ENOMEM;
    }
    *capacity = count;
    return FM_OK;
}

inline int grid_of_level(const fm_ctx* ctx, int level) { return ctx->cfg.n_level0 << level; }
// Matern smoothness of the configured field (0 is read as 1/2, the exponential covariance).
inline double matern_nu(const fm_config& cfg) { return cfg.nu > 0.0 ? cfg.nu : 0.5; }
inline int finest_grid(const fm_ctx* ctx) { return grid_of_level(ctx, ctx->cfg.n_levels - 1); }

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Event-pair timing around one launch of `family` (no-op unless profiling).
int prof_start(fm_ctx* ctx, int family, cudaStream_t st);
void prof_stop(fm_ctx* ctx, int idx, cudaStream_t st, double bytes, double flops);
// Zeroed device doubles for record idx that the launched kernel adds its own
// counts to (read at fm_profile_end): [0] flops, [1] the FP64 part of them,
// [2] algorithmic bytes of the work it ran (0: keep the launch's figure).
// Null when not profiling.
constexpr int kCountersPerRecord = 3;
double* prof_counter(fm_ctx* ctx, int idx);

#define FM_TIMED(ctx, family, st, bytes, flops, ...)          \
    do {                                                       \
        const int pi_ = fm::prof_start((ctx), (family), (st)); \
        __VA_ARGS__;                                           \
        fm::prof_stop((ctx), pi_, (st), (bytes), (flops));     \
    } while (0)

// The solver parameters of the context's configuration (mlmc.cu).
fm_solve_params solve_params(const fm_ctx* ctx);

// Samples per device batch for grid n (memory of the FMG hierarchy and field).
int64_t batch_limit(const fm_ctx* ctx, int n);

// FMG solve into caller-provided outputs (used by mlmc_sample_level too).
// The same with the level-wise scratch taken from `ar` (grown when short,
// which must not happen during stream capture: see fmg_levelwise_scratch).
fm_status fmg_solve_with(fm_ctx* ctx, Arena& ar, int n_fine, uint32_t S, const double* d_K,
                         const fm_solve_params& prm, double* d_qf, double* d_qc, double* d_p,
                         int32_t* d_status, cudaStream_t st);
size_t fmg_levelwise_scratch(const fm_ctx* ctx, int n_fine, uint32_t S, const fm_solve_params& prm);
void fmg_init_attributes();
void resident_init_attributes();
void uneven_free(fm_ctx* ctx);
void batched_free(fm_ctx* ctx);
fm_status fmg_solve_impl(fm_ctx* ctx, int n_fine, uint32_t S, const double* d_K,
                         const fm_solve_params& prm, double* d_qf, double* d_qc, double* d_p,
                         int32_t* d_status, cudaStream_t stream);

// Sample-resident FMG (fmg_resident.cu); false if the grid does not fit.
bool fmg_resident_launch(fm_ctx* ctx, int n_fine, int n0, size_t S, const double* d_K,
                         const fm_solve_params& prm, double* qf, double* qc, double* p_out,
                         int32_t* status, cudaStream_t st);

// Tensor-core KL synthesis (kl_tc.cu): install the BF16 basis, then fields.
fm_status kl_tc_install(fm_ctx* ctx, int split);
fm_status kl_tc_field(fm_ctx* ctx, int level, uint32_t n, const double* d_xi, double* d_K, cudaStream_t st);
// Nystrom interpolation of the KL basis on the tensor cores (kl_tc.cu).
fm_status kl_tc_nystrom(fm_ctx* ctx, int q, const double* dVt, const double* d_inv_sqrt_theta, double* d_out);

// KL arithmetic of the context: 1 FP64, 2 BF16, 3 BF16 split (bf16x3).
int kl_mode_of(const fm_ctx* ctx);

// Surrogate network (mlp.cu).
constexpr uint32_t kSurrogateLevelStream = 12;   // Philox level id of the S-level samples
constexpr uint32_t kSurrogateTrainStream = 13;   // Philox level id of the training samples
fm_status surrogate_eval_impl(fm_ctx* ctx, uint32_t n, const double* d_xi, double* d_s, cudaStream_t st);
// S for MC samples first .. first+n-1 of Philox stream `level`, from the
// Philox words directly (FP32 inverse normal, BF16 input).
fm_status surrogate_eval_mc_impl(fm_ctx* ctx, uint32_t level, uint64_t first, uint32_t n, double* d_s,
                                 cudaStream_t st);
int surrogate_err_flag(const fm_ctx* ctx);
// surrogate_eval_mc_impl runs the fused inference kernel (no scratch shared
// with the context's other surrogate evaluations).
bool surrogate_mc_fused(const fm_ctx* ctx);
void mlp_free(fm_ctx* ctx);

// Level sums of a batch (mlmc.cu).
fm_status level_sums_add(fm_ctx* ctx, uint32_t S, const double* d_qf, const double* d_qc,
                         int coarse, fm_level_sums* d_sums, cudaStream_t stream);
// The same with partial-sum scratch of the caller's (*partials, grown when
// short), for sums that run beside others on another stream.
fm_status level_sums_add_to(fm_ctx* ctx, uint32_t S, const double* d_qf, const double* d_qc, int coarse,
                            fm_level_sums* d_sums, cudaStream_t stream, double** partials, size_t* capacity);

// Host-side Sobol' direction numbers (points.cu).
int sobol_direction_numbers_host(uint32_t dim, std::vector<uint32_t>& V);

// Lattice generating vector of the embedded 2^m point sets (lattice.cu).
int lattice_cbc_host(uint32_t dim, int m_min, int m_max, uint32_t* z);
const std::vector<uint32_t>* lattice_vector_cached(uint32_t dim, int m_min, int m_max);
// The smallest embedded size of the lattice sequence: 2^5 points (the QMC pilot).
inline int lattice_m_min(int m_max) { return m_max < 5 ? m_max : 5; }

}  // namespace fm
