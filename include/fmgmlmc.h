/*
 * fmgmlmc.h - C ABI of the GB300 full-multigrid multilevel (quasi-) Monte
 * Carlo library.
 *
 * Method: Liu, Li, Sun & Yu, "A full multigrid multilevel (quasi-) Monte
 * Carlo method for the single-phase subsurface flow with random
 * coefficients", arXiv 1910.04727.  The model problem is Eq. 1 on the unit
 * square with the boundary data and QoI of Table 1: Case II (the default:
 * Dirichlet p_W / p_E on the west / east edges, no flow north and south,
 * QoI = outflux through the east edge) or Case I (Dirichlet data on all
 * four edges, QoI = u(0.5, 0.5)); the permeability is k = exp(g), g a Gaussian field
 * with the exponential Matern covariance of Sec. 3.1, represented by its
 * truncated KL expansion.  The MLMC levels (Sec. 2.2, Algorithm 1) share
 * their grid hierarchy with the full multigrid solver (Sec. 2.5): one FMG
 * solve of level l gives both Q^f_l and Q^c_l (Algorithm 3), the coarse
 * coefficients coming from the fine ones by injection (Sec. 2.5).
 *
 * Conventions
 *   - Every pointer named d_* is DEVICE memory owned by the caller; the
 *     library never frees it and keeps no reference after the call returns.
 *     Every other pointer is host memory owned by the caller.
 *   - Grids are n x n cells, stored row-major with x fastest: cell (i, j)
 *     (i = 0 at the west edge, j = 0 at the south edge) is element j*n + i.
 *     A batch of S grids is S consecutive grids ([S][n][n]).
 *   - Calls that take a cudaStream_t (passed as void*, NULL = the legacy
 *     default stream) are asynchronous on that stream; the return status
 *     covers argument checks and launch errors only.
 *   - A context is not thread-safe; use one per host thread.
 *   - No C++ exception crosses this interface.
 */
#ifndef FMGMLMC_H
#define FMGMLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fm_status;
#define FM_OK 0
#define FM_EINVAL 1        /* bad argument (message in fm_last_error) */
#define FM_ENOMEM 2        /* device or host allocation failed */
#define FM_ECUDA 3         /* a CUDA call failed */
#define FM_ENOTCONV 4      /* a solve did not reach its tolerance */
#define FM_ETIMEOUT 5      /* a bounded device wait ran out */
#define FM_EUNSUPPORTED 6  /* valid request the library does not implement */

#define FM_MAX_LEVELS 12

/* Arithmetic of the solver.
 * FP64:  every step in FP64.
 * MIXED: FP32 smoothing, restriction, prolongation and coarsest solve inside
 *        an FP64 iterative-refinement loop on the stages that give Q^c and
 *        Q^f; FP64 only for the finest-grid residual, the iterate those
 *        stages update and the outflux.  Needs converged = 1. */
#define FM_PREC_FP64 0
#define FM_PREC_MIXED 1

/* Arithmetic of the KL field synthesis.
 * AUTO: FP64 in the FP64 form, BF16X3 in the mixed form.
 * FP64: FP64 SIMT contraction.
 * BF16: tcgen05 tensor cores, BF16 basis and coefficients, FP32 accumulation
 *       (relative error of g about 2^-8).
 * BF16X3: tcgen05 tensor cores on the split products hi*hi + hi*lo + lo*hi
 *       (relative error of g about 2^-16). */
#define FM_KL_AUTO 0
#define FM_KL_FP64 1
#define FM_KL_BF16 2
#define FM_KL_BF16X3 3

typedef struct fm_ctx fm_ctx;

/* Problem and method parameters of one FMG-MLMC run. */
typedef struct {
    int32_t n_levels;     /* MLMC levels L + 1 (1 .. FM_MAX_LEVELS) */
    int32_t n_level0;     /* finest grid of level 0; level l uses n_level0 << l */
    int32_t n_coarsest;   /* coarsest FMG grid (the exact-solve grid); 4 */
    int32_t M;            /* KL modes (1 .. 4096) */
    double sigma2;        /* variance of g (Sec. 3.1) */
    double lambda;        /* correlation length (Sec. 3.1) */
    double pW, pE;        /* Dirichlet data on the west / east edges (Table 1) */
    int32_t nu0;          /* V-cycles per FMG stage */
    int32_t nu1, nu2;     /* pre- / post-smoothing red-black Gauss-Seidel sweeps */
    int32_t precision;    /* FM_PREC_* */
    int32_t converged;    /* 0: nu0 V-cycles per stage; 1: the stages giving Q^c and Q^f
                             iterate until ||b - A p||_2 <= tol ||b||_2 */
    double tol;           /* relative residual target of converged stages */
    double qtol;          /* converged stages also stop once an iteration changes the
                             stage's outflux by <= qtol |Q| (0: residual test only) */
    int32_t max_cycles;   /* cycle cap of a converged stage */
    int32_t kl_mode;      /* FM_KL_*: arithmetic of the field synthesis */
    int32_t n_shifts;     /* QMC digital shifts R */
    uint64_t seed;        /* key of the Philox streams (MC points, QMC shifts) */
    int64_t max_batch;    /* most samples per device batch (0: library's choice) */
    int32_t bc_case;      /* Table 1: FM_CASE_II (0 is read as Case II) or FM_CASE_I */
    double pS, pN;        /* Case I: Dirichlet data on the south / north edges */
    double nu;            /* Matern smoothness of the field (Sec. 3.1, Table 2): 0.5 (exponential;
                             0 is read as 0.5), 1, 1.5 or 2.5 */
    int32_t qmc_rule;     /* randomized QMC points of the MLQMC estimator (FM_QMC_*) */
    int32_t lattice_m;    /* FM_QMC_LATTICE: the sequence holds 2^lattice_m points (5 .. 24;
                             0 is read as 16) */
    int32_t ir_cycles;    /* converged stages: V-cycles between residual tests (0: nu0) */
    int32_t energy_step;  /* 1: the energy-optimal correction step in every solve (see
                             fm_solve_params; the level-wise schedule) */
} fm_config;

/* Randomized QMC rules (Sec. 2.4).
 * FM_QMC_SOBOL_SHIFT: Sobol' points, XOR with a random digital shift.
 * FM_QMC_SOBOL_OWEN:  Sobol' points, nested uniform (Owen) scrambling.
 * FM_QMC_LATTICE:     rank-1 lattice sequence (generating vector from
 *                     fm_lattice_cbc for the embedded sets of 2^5 ..
 *                     2^lattice_m points, built when the context is
 *                     created), shifted modulo 1 by a random vector. */
#define FM_QMC_SOBOL_SHIFT 0
#define FM_QMC_SOBOL_OWEN 1
#define FM_QMC_LATTICE 2

/* Boundary conditions and QoI (Table 1).
 * FM_CASE_II: p = pW on the west edge, pE on the east edge, no flow through
 *             the north and south edges; QoI = the outflux through the east
 *             edge, sum_j 2 K_(n-1,j) (p_(n-1,j) - pE).
 * FM_CASE_I:  Dirichlet data pW, pE, pS, pN on the west, east, south and
 *             north edges; QoI = u(0.5, 0.5).  The centre is the corner of
 *             the four middle cells of every grid, and the bilinear
 *             interpolation of their centre values there is their mean. */
#define FM_CASE_I 1
#define FM_CASE_II 2

/* Kernel schedule of a batched FMG solve (same arithmetic, same result up
 * to rounding order). */
#define FM_KERNEL_AUTO 0       /* resident where it is the faster schedule (up to 32 x 32 in
                                  the mixed form, 16 x 16 in FP64, and a converged mixed
                                  64 x 64 batch of at most two samples per SM; not with the
                                  energy step), else levelwise */
#define FM_KERNEL_LEVELWISE 1  /* one kernel per grid operation over all samples */
#define FM_KERNEL_RESIDENT 2   /* one CTA per sample, hierarchy in shared memory
                                  (n_fine <= 64 in FP64) */

/* Parameters of one batched FMG solve. */
typedef struct {
    double pW, pE;        /* Dirichlet data */
    int32_t n_coarsest;   /* coarsest grid (4) */
    int32_t nu0, nu1, nu2;
    int32_t precision;    /* FM_PREC_* */
    int32_t kernel;       /* FM_KERNEL_* */
    int32_t converged;    /* 0: nu0 V-cycles on every stage (the end of a stage's
                             cycles is its "exact" solution); 1: stages n_fine/2 and
                             n_fine iterate to ||b - A p||_2 <= tol ||b||_2, testing
                             after every nu0 V-cycles (in the mixed form: nu0 FP32
                             V-cycles on the correction per FP64 residual) */
    double tol;
    double qtol;          /* also stop once a cycle changes the outflux by <= qtol |Q| */
    int32_t max_cycles;   /* cap per converged stage; a sample that reaches it gets
                             status FM_ENOTCONV */
    int32_t energy_step;  /* 1 (converged mode, level-wise schedule): add each V-cycle's
                             coarse-grid correction d = P e_c as alpha d, alpha = (r, d) /
                             (d, A d) per sample, the energy minimum along d, so no cycle
                             raises the energy error (robust at high contrast) */
    int32_t bc_case;      /* FM_CASE_II (0 is read as Case II) or FM_CASE_I */
    double pS, pN;        /* Case I: Dirichlet data on the south / north edges */
    int32_t ir_cycles;    /* converged mode: V-cycles between residual tests (in the mixed form:
                             FP32 V-cycles per FP64 residual); 0: nu0 */
} fm_solve_params;

/* ---------------------------------------------------------------- context */

/* Create a context on the current CUDA device.  Checks cfg, computes the
 * Sobol' direction numbers for M dimensions and allocates the level-sum
 * buffers.  *out is set only on FM_OK. */
fm_status fm_create(const fm_config* cfg, fm_ctx** out);

/* Release every device and host resource of ctx (NULL is a no-op). */
void fm_destroy(fm_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed fm_create
 * on this thread when ctx is NULL).  Valid until the next call. */
const char* fm_last_error(const fm_ctx* ctx);

/* ---------------------------------------------------------------- points */

/* MC points (Sec. 2.3): d_xi[s*dim + k] = Phi^{-1}(u),
 * u = ((w >> 11) + 1/2) 2^-53, where w is 64-bit word k of the Philox4x64-10
 * stream keyed (seed, 1<<32 | level) at counter (k/4, first + s, 0, 0),
 * lane k%4.  n samples; dim <= 4096.  Phi^{-1} is CUDA's normcdfinv. */
fm_status mc_points(fm_ctx* ctx, uint32_t level, uint64_t first, uint32_t n, uint32_t dim,
                    double* d_xi, void* stream);

/* The raw 64-bit Philox4x64-10 words behind mc_points (Sec. 2.3):
 * d_words[s*dim + k] = word k of the stream keyed (seed, 1<<32 | level) at
 * counter (k/4, first + s, 0, 0), lane k%4, written by the same kernel that
 * mc_points runs, so the normals are Phi^{-1}(((w >> 11) + 1/2) 2^-53) of
 * exactly these words.  n samples; dim <= 4096; d_words device [n][dim]. */
fm_status mc_words(fm_ctx* ctx, uint32_t level, uint64_t first, uint32_t n, uint32_t dim,
                   uint64_t* d_words, void* stream);

/* Randomized Sobol' points (Sec. 2.4 / 3.1): point index first + s (Gray-code
 * order, x = XOR of the direction numbers selected by the bits of
 * (n XOR n>>1)), XOR a digital shift per (level, shift r, dimension) drawn
 * from the Philox stream (seed, 2<<32 | level) at counter (d/4, r, 0, 0),
 * lane d%4, high 32 bits.  d_x (nullable) receives the uint32 points
 * [n_shifts][n][dim]; d_xi (nullable) Phi^{-1}((x + 1/2) 2^-32) in the same
 * layout.  dim <= the context's M. */
fm_status sobol_points(fm_ctx* ctx, uint32_t level, uint32_t dim, uint64_t first, uint32_t n,
                       uint32_t first_shift, uint32_t n_shifts, uint32_t* d_x, double* d_xi,
                       void* stream);

/* Host copy of the Sobol' direction numbers V[d*32 + b] (d < M, b < 32). */
fm_status sobol_direction_numbers(const fm_ctx* ctx, uint32_t* V);

/* Randomized QMC points of rule `rule` (FM_QMC_*), point indices first ..
 * first+n-1, randomizations first_shift .. first_shift+n_shifts-1, 32-bit
 * fixed point x in d_x (nullable) and Phi^{-1}((x + 1/2) 2^-32) in d_xi
 * (nullable), both [n_shifts][n][dim], dim <= M.
 *   FM_QMC_SOBOL_SHIFT: as sobol_points.
 *   FM_QMC_SOBOL_OWEN:  the Gray-code Sobol' point x, then output bit b
 *       (b = 0 the leading bit) = input bit b XOR the random bit of tree node
 *       (b, the b leading input bits): the low bit of word 0 of Philox4x64-10
 *       keyed (seed, 5 << 32 | level) at counter (prefix, r << 32 | d, b, 0).
 *   FM_QMC_LATTICE:     point index i in radical-inverse order over
 *       lattice_m bits, x = (z_d phi(i) 2^(32 - lattice_m) + Delta) mod 2^32,
 *       Delta = high 32 bits of word d of the Philox stream (seed, 4 << 32 |
 *       level) at index r; first + n <= 2^lattice_m.  Needs a context created
 *       with qmc_rule = FM_QMC_LATTICE (FM_EINVAL otherwise). */
fm_status qmc_points(fm_ctx* ctx, int32_t rule, uint32_t level, uint32_t dim, uint64_t first, uint32_t n,
                     uint32_t first_shift, uint32_t n_shifts, uint32_t* d_x, double* d_xi, void* stream);

/* Generating vector of a rank-1 lattice sequence for the embedded point sets
 * of 2^m points, m = m_min .. m_max (Sec. 2.4 lattice rules; host only, no
 * CUDA call).  Component by component: z_1 = 1; component s is the odd
 * z < 2^(m_max-1) minimising sum_m e^2_m(z_1..z_(s-1), z) / e^2_m(z_1..z_(s-1)),
 * e^2_m = -1 + 2^-m sum_k prod_j (1 + gamma_j B_2({k z_j / 2^m})) the
 * shift-averaged squared worst-case error with product weights
 * gamma_j = 1/j^2 (ties to the smaller z).  Evaluated by the fast
 * construction of Nuyens and Cools (FFTs over the group of odd residues
 * mod 2^m), the minimum confirmed on plain sums.  z: host [dim], dim <= 4096,
 * 1 <= m_min <= m_max <= 24. */
fm_status fm_lattice_cbc(uint32_t dim, int32_t m_min, int32_t m_max, uint32_t* z);

/* Host copy of the context's lattice generating vector [M] (FM_QMC_LATTICE). */
fm_status lattice_generating_vector(const fm_ctx* ctx, uint32_t* z);

/* ---------------------------------------------------------------- KL field */

/* Install a KL basis (Sec. 3.1): basis_ref[c*M + k] = sqrt(theta_k) phi_k(x_c)
 * at the cells c of the finest grid n_ref = n_level0 << (n_levels - 1).  Grid
 * n of a coarser level samples the field at the finest-grid points that
 * injection keeps (cell (i,j) of grid n -> cell (s i, s j) of grid n_ref,
 * s = n_ref / n), so the coarse coefficients of level l and the fine ones of
 * level l-1 coincide.  basis_ref is device memory if on_device, else host. */
fm_status kl_basis_set(fm_ctx* ctx, const double* basis_ref, int32_t on_device);

/* Build the KL basis of the Matern covariance of Sec. 3.1 (smoothness cfg.nu,
 * see fm_matern_covariance) on the GPU by the Nystrom method: midpoint quadrature on a q x q grid
 * (q = 0: smallest q >= 32 with q^2 >= 8 M), a dense symmetric eigensolve
 * (cuSOLVER) of the weighted covariance matrix, and Nystrom interpolation
 * of the top M eigenfunctions to the field points.  theta_out (nullable,
 * host) receives the M eigenvalues, captured_out (nullable, host)
 * sum_{k<=M} theta_k / (sigma2 meas(Omega)).  Synchronous. */
fm_status kl_basis_build(fm_ctx* ctx, int32_t q, double* theta_out, double* captured_out);

/* Arithmetic of the Nystrom interpolation B = C_x V / sqrt(theta) (2 n_ref^2
 * q^2 M flops) in kl_basis_build_ex.
 * AUTO:   FP64 (cuBLAS DGEMM) up to 2e12 flops, the tensor cores above.
 * FP64:   FP64 DGEMM over chunks of field points.
 * TENSOR: one tcgen05 BF16x3 GEMM per chunk of field points (covariance tile
 *         and eigenvectors split into BF16 hi + lo, products hi*hi + hi*lo +
 *         lo*hi, FP32 accumulation: entries to about 1e-5 relative), the
 *         finest grid's basis written in place (the large high-contrast
 *         configuration: 2048^2 points, 1024 modes, q = 96). */
#define FM_INTERP_AUTO 0
#define FM_INTERP_FP64 1
#define FM_INTERP_TENSOR 2

/* kl_basis_build with the interpolation arithmetic chosen (FM_INTERP_*). */
fm_status kl_basis_build_ex(fm_ctx* ctx, int32_t q, int32_t interp, double* theta_out, double* captured_out);

/* The Matern covariance of Sec. 3.1 at n distances (host memory, no CUDA
 * call): C(d) = sigma2 2^(1-nu) / Gamma(nu) (sqrt(2 nu) d / lambda)^nu
 * K_nu(sqrt(2 nu) d / lambda), C(0) = sigma2, for nu = 0.5 (sigma2
 * exp(-d/lambda)), 1 (sigma2 x K_1(x), x = sqrt 2 d / lambda, K_1 by its
 * ascending series for x <= 2 and the trapezoidal rule on its integral
 * representation above), 1.5 and 2.5 (closed forms).  FM_EINVAL for another
 * nu, non-positive sigma2 or lambda, or a negative distance. */
fm_status fm_matern_covariance(double nu, double sigma2, double lambda, const double* d, int64_t n, double* c);

/* Copy the installed basis of the finest grid (the layout kl_basis_set takes)
 * to basis_ref_out: device memory if on_device, else host.  Synchronous. */
fm_status kl_basis_get(const fm_ctx* ctx, double* basis_ref_out, int32_t on_device);

/* Field synthesis (Sec. 3.1): d_K[s][c] = exp(sum_k B_l[c][k] d_xi[s*M + k])
 * for the n samples of MLMC level `level` (grid n_level0 << level), in the
 * context's kl_mode; d_K is [n][N_l][N_l] doubles.  The tensor-core forms
 * report a device-side wait that ran out through fm_sync. */
fm_status kl_field_batch(fm_ctx* ctx, int32_t level, uint32_t n, const double* d_xi,
                         double* d_K, void* stream);

/* ---------------------------------------------------------------- solver */

/* Full multigrid (Sec. 2.5) for n independent problems on an n_fine x n_fine
 * grid with coefficients d_K [n][n_fine][n_fine] (boundary data and QoI of
 * prm->bc_case, Table 1): coefficients coarsened by
 * injection K^c[I][J] = K^f[2I][2J] down to the coarsest grid, exact solve
 * there, then per finer grid bilinear interpolation of the previous stage's
 * solution and nu0 V(nu1,nu2) cycles (red-black Gauss-Seidel, residual
 * restricted by summing the 2x2 children, bilinear cell-centred
 * prolongation).  Outputs: d_qf[s] QoI of the finest stage; d_qc[s]
 * (nullable) QoI of the stage one grid coarser (the Q^c by-product;
 * NaN if n_fine == n_coarsest).  In converged mode that stage is refined
 * to the tolerance only when d_qc is given; without it the stage only
 * starts the finest one, and Q^f agrees with the d_qc run to within the
 * tolerance, not bit for bit.  d_p (nullable) the finest solution
 * [n][n_fine][n_fine]; d_status (nullable) per-sample FM_OK / FM_ENOTCONV.
 * n_fine must be n_coarsest times a power of two.  Scratch is owned by the
 * context.  prm->kernel picks the schedule: the resident one (the whole
 * hierarchy of a sample in shared memory, n_fine <= 64) or the level-wise
 * one (any n_fine up to 8192); both run FP64 and mixed, fixed and converged
 * (the energy step: level-wise only). */
fm_status fmg_solve_batch(fm_ctx* ctx, int32_t n_fine, uint32_t n, const double* d_K,
                          const fm_solve_params* prm, double* d_qf, double* d_qc,
                          double* d_p, int32_t* d_status, void* stream);

/* The same FP64 fixed-cycle solve on the level-wise schedule as
 * fmg_solve_batch, for callers that must not allocate device memory during a
 * solve: code that runs under a memory budget fixed up front, inside a
 * memory pool owned by someone else, or on a path where a cudaMalloc would
 * stall the device or fail.  It allocates nothing (no cudaMalloc, cudaFree
 * or allocating library routine; profiling must be off): its scratch is one
 * static device array of 32 MiB that the library holds on every device that
 * loads it until the process exits.  The paper has no counterpart; this is
 * an interface for callers that cannot allocate.
 *   - Inputs and outputs stay the caller's: d_K [n][n_fine][n_fine], d_qf
 *     [n], d_qc [n] (nullable), as in fmg_solve_batch.
 *   - prm must ask for FM_PREC_FP64 with converged = 0; prm->kernel is not
 *     read.  A batch whose hierarchy needs more than 32 MiB (about 6 samples
 *     of 256 x 256, 25 of 128 x 128, 100 of 64 x 64) is rejected with
 *     FM_EINVAL and a message giving the bytes it needs: split it.
 *   - The first call on each device looks up the array's device address with
 *     that device current (cudaGetSymbolAddress) and keeps it; make that
 *     first call before any stream capture.
 *   - Every call uses the same array, which keeps whatever the last call left
 *     in it; the solve writes every scratch entry before reading it.  Calls
 *     whose work overlaps on the GPU (other streams, other host threads) race
 *     on the array: serialise them. */
fm_status fmg_solve_batch_static(fm_ctx* ctx, int32_t n_fine, uint32_t n, const double* d_K,
                                 const fm_solve_params* prm, double* d_qf, double* d_qc, void* stream);

/* ---------------------------------------------------------------- uneven batches */

/* One group of an uneven batch: `count` samples of one grid size. */
typedef struct {
    int32_t n_fine;        /* finest grid n_coarsest * 2^m */
    uint32_t count;        /* samples */
    const double* d_K;     /* device [count][n_fine][n_fine] coefficients */
    double* d_qf;          /* device [count] outflux of the finest grid */
    double* d_qc;          /* device [count] outflux of grid n_fine / 2 (nullable; without it a
                              converged solve leaves that stage unrefined, as fmg_solve_batch) */
    int32_t* d_status;     /* device [count] per-sample FM_OK / FM_ENOTCONV (nullable) */
} fm_batch_group;

/* FMG solves of groups with different grid sizes as one CUDA graph: one
 * branch per group, the resident kernel where FM_KERNEL_AUTO takes it and the
 * level-wise schedule above, the refined stages of the converged mode
 * looping on the device (conditional graph nodes), so the graph runs without
 * the host.  Each sample's results are those fmg_solve_batch gives it.
 * Branches carry stream priorities by grid size, the largest grid's highest
 * (below the surrogate's training stream).  The executable graphs stay in
 * ctx, one per shape (grids, schedules and which groups ask for Q^c; up to
 * 8, the least recently used replaced), and a call with a kept shape updates
 * that graph in place.
 * prm->kernel: FM_KERNEL_AUTO or FM_KERNEL_LEVELWISE
 * (every group level-wise).  Asynchronous on `stream`; one call at a time
 * per ctx.  Scratch is allocated before the capture (FM_ENOMEM). */
fm_status fmg_solve_uneven(fm_ctx* ctx, int32_t n_groups, const fm_batch_group* groups,
                           const fm_solve_params* prm, void* stream);

/* Graph bookkeeping of fmg_solve_uneven: instantiations, in-place updates and
 * launches so far (host only). */
fm_status fmg_uneven_stats(const fm_ctx* ctx, int64_t* instantiations, int64_t* updates, int64_t* launches);

/* ---------------------------------------------------------------- autotuning */

/* One tuned grid: the smoother launch shape chosen for it. */
typedef struct {
    int32_t n;            /* grid n x n */
    int32_t tile;         /* tile interior staged in shared memory (0: one launch per colour and sweep;
                             -1: column strips) */
    int32_t threads;      /* 0: register-blocked tile kernel (only p in shared memory); else threads
                             per CTA of the tile kernel that stages every operand in shared memory */
    double ms_best;       /* one smoothing call (nsweeps sweeps) with the chosen shape, milliseconds */
    double ms_default;    /* the same with the built-in default shape */
    int64_t samples;      /* samples of the timing batch (about 64 Mi cells) */
} fm_tune_entry;

/* Times the red-black smoother's launch shapes (one launch per colour,
 * column strips, or tiles of 8, 16, 32, 64 cells with a 2 nsweeps halo, either register-blocked
 * with only the iterate in shared memory or with every operand staged there
 * at 128 or 256 threads) for the grids n_min, 2 n_min, ..., <= n_max on a
 * synthetic batch of about 64 Mi cells per grid, and keeps the fastest in
 * ctx for that precision (FM_PREC_FP64: the FP64 grids; FM_PREC_MIXED: the
 * FP32 ones).  Every later solve on ctx uses the choice; the sweeps' results
 * are the same whichever shape runs.  Synchronous; entries (nullable) gets up
 * to max_entries rows. */
fm_status fm_autotune(fm_ctx* ctx, int32_t precision, int32_t nsweeps, int32_t n_min, int32_t n_max,
                      fm_tune_entry* entries, int32_t max_entries, int32_t* n_entries);

/* Sets the smoother launch shape of grid n (a power of two) for one
 * precision, as fm_autotune would set it: tile = 0 one launch per colour
 * and sweep; -1 column strips (one warp per 64-column strip marching up the
 * rows, 1 or 2 sweeps); 8, 16, 32 or 64 tiles with threads = 0
 * (register-blocked) or 128 / 256 (staged in shared memory); tile = -2
 * removes the entry so the built-in default applies.  A shape that cannot
 * run a solve's sweeps (sweep counts, shared memory) falls back to colour
 * launches; every shape gives the same results.  FM_EINVAL otherwise. */
fm_status fm_set_smoother_shape(fm_ctx* ctx, int32_t precision, int32_t n, int32_t tile, int32_t threads);

/* Level-wise V-cycles: the part below a correction grid of at most n_max x
 * n_max cells (a power of two up to 32; default 32) runs as one resident
 * launch per cycle (every listed sample's tail in shared memory) instead of
 * several launches per grid; 0 launches grid by grid throughout.  Same
 * arithmetic in the same order: the results do not change.  The
 * energy-optimal step always runs grid by grid. */
fm_status fm_set_vcycle_tail(fm_ctx* ctx, int32_t n_max);

/* ---------------------------------------------------------------- MLMC */

/* Running sums of one (level, shift) cell: Neumaier-compensated FP64 pairs
 * (sum, compensation) of Y, Y^2, Q^f, Q^c, and the sample count.  Y = Q^f on
 * level 0 and Q^f - Q^c above (Sec. 2.2). */
typedef struct {
    double sum_y[2];
    double sum_y2[2];
    double sum_qf[2];
    double sum_qc[2];
    double count;
    double pad[7];
} fm_level_sums;

/* Statistics of one fm_level_sums cell (host memory; no CUDA call). */
typedef struct {
    double count;         /* samples */
    double mean;          /* sum Y / count */
    double var;           /* Bessel-corrected sample variance of Y (0 for count < 2) */
    double sum_qf, sum_qc;
} fm_level_stat;

/* Mean and variance of the samples behind one cell (Sec. 2.2: the sample
 * mean of Y_l and the estimate V_l of its variance).  The compensated sums
 * of Y and of the exact Y^2 are read as double-double numbers and
 * S2 - S1^2 / n is formed in double-double arithmetic, so the variance keeps
 * its accuracy when |mean| is much larger than the standard deviation.
 * FM_EINVAL for a null pointer. */
fm_status fm_level_stats(const fm_level_sums* sums, fm_level_stat* out);

/* Draw samples first .. first+n-1 of level `level` (MC if shift < 0, else
 * QMC shift `shift`), synthesise their fields, run the FMG solve and add Y,
 * Y^2, Q^f, Q^c to *d_sums (device).  With the surrogate enabled
 * (surrogate_enable) level -1 is the surrogate level (Y = S(xi), no solve, on
 * a point stream of its own) and level 0 gives Y = Q_0 - S(xi) with S in the
 * Q^c sums.  d_qf / d_qc (nullable, device [n]) receive the per-sample QoIs.
 * Level 0 needs no Q^c, so its solves leave the coarse stage unrefined
 * (fmg_solve_batch without d_qc) unless d_qc asks for it without the
 * surrogate.  Processes the samples in batches of at most the context's
 * max_batch. */
fm_status mlmc_sample_level(fm_ctx* ctx, int32_t level, uint64_t first, uint32_t n,
                            int32_t shift, fm_level_sums* d_sums, double* d_qf, double* d_qc,
                            void* stream);

typedef struct {
    double eps;           /* target RMSE */
    int32_t qmc;          /* 0: MLMC (Algorithm 1/3), 1: MLQMC (Algorithm 2) */
    int64_t n_pilot;      /* initial samples per level (per shift for QMC) */
    int32_t max_rounds;
    int32_t surrogate;    /* 1: add the surrogate control-variate level below level 0 */
    double surrogate_cost; /* cost of an S-level sample relative to a level-0 sample */
    int32_t batched;      /* 1: each round's solves of all levels as one uneven batch (fmg_solve_uneven);
                             the surrogate level's MC samples on a stream of their own beside it */
    int32_t adapt_L;      /* 1: grow the finest level from L_start (bias test of Algorithms 1-3) up to
                             n_levels - 1; 0: use every level of the context */
    int32_t L_start;      /* adapt_L: the first finest level, 1 .. n_levels - 1 (the paper starts at 2) */
    double alpha;         /* weak rate of the bias test; <= 0: fitted on the level means, floored at 1/2 */
} fm_estimate_opts;

typedef struct {
    double estimate;                 /* sum_l mean(Y_l) */
    double var_estimator;            /* sum_l V_l / N_l (MC) or sum_l Var(Y^_l) (QMC) */
    double mean[FM_MAX_LEVELS];      /* mean(Y_l) */
    double var[FM_MAX_LEVELS];       /* MC: V_l; QMC: variance of the level estimate */
    int64_t N[FM_MAX_LEVELS];        /* samples per level (per shift for QMC) */
    double alpha, beta;              /* fitted rates of |E Y_l| and V_l, l = 1 .. L */
    double bias;                     /* |mean(Y_L)| / (2^alpha_used - 1) (Algorithm 1) */
    int32_t rounds;
    double seconds;                  /* wall time of the call */
    double mean_s, var_s;            /* surrogate level: mean(S), V[S] (or its level-estimate variance) */
    int64_t N_s;                     /* surrogate-level samples */
    double level_seconds[FM_MAX_LEVELS]; /* device time spent sampling each level (CUDA events) */
    double seconds_s;                /* device time spent on the surrogate level */
    double batched_seconds;          /* batched mode: device time of the rounds' uneven batches */
    int32_t L;                       /* finest level used (n_levels - 1 unless adapt_L stopped earlier) */
    int32_t bias_ok;                 /* bias < eps / sqrt(2) */
    double alpha_used;               /* opts alpha if > 0, else max(alpha, 1/2) (1/2 if not fitted) */
} fm_result;

/* The host controller (Algorithm 3 with the MC rule N_l = (2/eps^2)
 * sqrt(V_l/C_l) sum_k sqrt(V_k C_k), or Algorithm 2's doubling rule for
 * QMC), at the fixed finest level n_levels - 1 or, with adapt_L, growing
 * the finest level until the bias test passes (mlmc_estimate_core), with
 * the cost model C_l = (4/3) (n_level0 << l)^2.  Uses the default stream,
 * synchronous. */
fm_status mlmc_estimate(fm_ctx* ctx, const fm_estimate_opts* opts, fm_result* out);

/* ---------------------------------------------------------------- controller over ranks */

/* Callbacks of the sample-size controller.  `ext_level` counts the levels
 * the controller sees (with the surrogate, 0 is the surrogate level and
 * l + 1 MLMC level l).  enqueue: add samples first .. first+n-1 of
 * ext_level (QMC shift `shift`, or -1 for MC) to this rank's running sums,
 * asynchronously if it likes.  read: finish the queued work and copy this
 * rank's running sums, [n_ext][R] cells (R = 1 for MC), to `local`.
 * allgather: place every rank's `local` (bytes_per_rank each) into `all`,
 * rank r at offset r * bytes_per_rank, on every rank.  Each returns FM_OK or
 * an error status, which ends the estimate with that status. */
typedef fm_status (*fm_enqueue_fn)(void* user, int32_t ext_level, uint64_t first, uint64_t n, int32_t shift);
typedef fm_status (*fm_read_fn)(void* user, fm_level_sums* local);
typedef fm_status (*fm_allgather_fn)(void* user, const fm_level_sums* local, fm_level_sums* all,
                                     size_t bytes_per_rank);

typedef struct {
    int32_t n_ext;         /* levels seen by the controller, 1 .. FM_MAX_LEVELS + 1 */
    const double* cost;    /* [n_ext] cost of one sample of each level (> 0) */
    double eps;            /* target RMSE */
    int32_t qmc;           /* 0: MC rule (Algorithm 3); 1: QMC doubling rule (Algorithm 2) */
    int32_t n_shifts;      /* R for QMC (2 .. 64) */
    int64_t n_pilot;       /* initial samples per level (per shift for QMC), >= 2 */
    int32_t max_rounds;    /* controller rounds (<= 0: 100) */
    int32_t rank, world;   /* this rank and the number of ranks (world 1: no allgather) */
    int32_t level0;        /* extended index of MLMC level 0 (1 with a surrogate level below it, else 0) */
    int32_t adapt;         /* 1: grow the finest level (the bias test of Algorithms 1-3) up to n_ext - 1 */
    int32_t n_ext_start;   /* adapt: extended levels in use at the start, level0 + 2 .. n_ext */
    double alpha;          /* weak rate of the bias test; <= 0: the fitted rate of |mean(Y_l)|, l >= 1,
                              floored at 1/2 */
} fm_core_opts;

typedef struct {
    double estimate, var_estimator;
    double mean[FM_MAX_LEVELS + 1], var[FM_MAX_LEVELS + 1];
    int64_t N[FM_MAX_LEVELS + 1];    /* samples per level over all ranks (per shift for QMC) */
    int32_t rounds;
    int32_t n_ext_used;              /* extended levels in use at the end (n_ext unless adapt) */
    int32_t bias_ok;                 /* bias < eps / sqrt(2) */
    double bias, alpha_used;         /* Richardson estimate |mean(Y_L)| / (2^alpha - 1) and its alpha
                                        (NaN when no level >= 1 is in use) */
} fm_core_result;

/* Rank `rank`'s contiguous share of samples first .. first+n-1 among `world`
 * ranks: floor(n / world) each, the remainder one apiece to the lowest
 * ranks.  Host only. */
void fm_shard_range(uint64_t first, uint64_t n, int32_t rank, int32_t world, uint64_t* my_first, uint64_t* my_n);

/* The controller of mlmc_estimate over callbacks (Algorithms 1-3; sample
 * sizes as in mlmc_estimate).  With adapt the finest level grows: starting
 * from n_ext_start levels, once the sample sizes are met (MC: no level needs
 * extra samples; QMC: sum of the level-estimate variances <= eps^2/2) the
 * run stops if the Richardson bias estimate is below eps/sqrt(2) or every
 * level is in use, else the next level gets n_pilot samples (per shift) and
 * the rounds go on.  Without adapt all n_ext levels are used from the start
 * and the bias estimate is only reported.  Every request is split
 * by fm_shard_range; the ranks' sums are folded in rank order (Neumaier), so
 * all ranks compute the same schedule and the same estimate.  Host only: it
 * makes no CUDA call.  On an error status `err` (nullable, errlen bytes)
 * holds a message. */
fm_status mlmc_estimate_core(const fm_core_opts* opts, fm_enqueue_fn enqueue, fm_read_fn read,
                             fm_allgather_fn allgather, void* user, fm_core_result* out, char* err, size_t errlen);

/* mlmc_estimate with the samples of every request shared among `world`
 * ranks (one context per rank, each on its own GPU): rank r solves its
 * contiguous share, and `allgather` (with `user`) exchanges the level sums
 * once per controller round.  world = 1 is mlmc_estimate.  Synchronous. */
fm_status mlmc_estimate_sharded(fm_ctx* ctx, const fm_estimate_opts* opts, int32_t rank, int32_t world,
                                fm_allgather_fn allgather, void* user, fm_result* out);

/* Synchronise the device and report device-side failures of earlier
 * asynchronous calls on ctx: FM_ETIMEOUT if a bounded wait inside a kernel
 * ran out (its output is then invalid; the flag is cleared once reported),
 * FM_ECUDA for a CUDA error.  Every wait of the tensor-core kernels on an
 * mbarrier (TMA tiles, MMA completion) gives up after 50 ms of wall time;
 * the kernel then waits, again bounded, for the copies it issued, frees its
 * tensor memory and returns. */
fm_status fm_sync(fm_ctx* ctx);

/* Check of the failure path above, not part of the method: one CTA waits,
 * with the same bounded wait, on an mbarrier that nothing arrives on, for
 * budget_ns (0 .. 1e9) of wall time.  The wait runs out, the kernel sets the
 * context's device flag and returns, and the next fm_sync reports
 * FM_ETIMEOUT; the context stays usable.  Asynchronous on `stream`. */
fm_status fm_wait_check(fm_ctx* ctx, int64_t budget_ns, void* stream);

/* ---------------------------------------------------------------- surrogate */

/* Control-variate level below the coarsest grid (the project's addition to
 * the telescoping sum of Eq. 2): E[Q_L] = E[S] + E[Q_0 - S] + sum_{l>=1}
 * E[Y_l], unbiased for any S.  S(xi) = mu + sd f(xi), f an MLP M -> 256 ->
 * 256 -> 256 -> 1 with GELU(z) = z (1 + erf(z/sqrt 2))/2; hidden layers run
 * on tcgen05 tensor cores with BF16 operands (weights, input, activations,
 * back-propagated pre-activation gradients) and FP32 accumulation; FP32
 * master parameters and Adam.  Flat FP32 parameter layout: W1 [256][M], b1
 * [256], W2 [256][256], b2, W3 [256][256], b3, w4 [256], b4 [1]. */
typedef struct {
    int32_t n_train;      /* training pairs (xi, Q_0) drawn from level 0 (>= 256) */
    int32_t epochs;
    double lr;            /* Adam step, cosine-decayed to 0 over the run */
    uint64_t seed;        /* parameter initialisation and shuffling */
    int32_t batch;        /* mini-batch rows: a multiple of 128, at most 4096 (0: 256) */
    int32_t async_run;    /* 1: return once the training steps are launched (see surrogate_train) */
    double target_tol;    /* > 0: residual and outflux-change tolerance of the training pairs'
                             level-0 solves (converged forms); <= 0: the context's own.  Any S
                             leaves the estimator unbiased, so the targets need no more
                             accuracy than the network's fit */
} fm_train_opts;

typedef struct {
    double loss_first, loss_last;   /* mini-batch MSE of the standardised target */
    double mu, sd;                  /* target standardisation */
    double corr;                    /* correlation of S with Q_0 on the training set */
    double var_q, var_residual;     /* V[Q_0] and V[Q_0 - S] on the training set */
    int32_t steps;
    double seconds;
} fm_train_report;

/* Turn the surrogate level of mlmc_sample_level on (1) or off (0). */
fm_status surrogate_enable(fm_ctx* ctx, int32_t on);

/* Number of FP32 parameters of the network for the context's M. */
int64_t surrogate_param_count(const fm_ctx* ctx);

/* Copy the FP32 parameters to (set = 0) or from (set = 1) host memory. */
fm_status surrogate_params(fm_ctx* ctx, float* host_params, int32_t set);

/* Set the target standardisation (S = mu + sd f). */
fm_status surrogate_set_scale(fm_ctx* ctx, double mu, double sd);

/* One forward and backward pass of the MSE loss on a batch of 256 rows:
 * d_xi [256][M] FP64 inputs, d_target [256] FP32 standardised targets;
 * host_grads (nullable) receives the gradient in the parameter layout,
 * host_loss (nullable) the mean squared error.  Synchronous. */
fm_status surrogate_loss_grad(fm_ctx* ctx, const double* d_xi, const float* d_target, float* host_grads,
                              double* host_loss);

/* Train from scratch on n_train level-0 samples of the method (points on a
 * stream of their own, the context's field and solver).  The training pairs
 * are formed synchronously; the training steps run on the network's own
 * stream.  async_run = 0: returns when training is done, with the whole
 * report.  async_run = 1: returns once the steps are launched; the report
 * then holds mu, sd, var_q and steps (the losses, corr and var_residual are
 * NaN) and surrogate_train_finish gives the rest.  Meanwhile other work runs
 * beside the steps (an estimator round solving levels >= 1, say), and every
 * use of the network (surrogate_eval*, the surrogate level of
 * mlmc_sample_level and mlmc_estimate, surrogate_params, a new training)
 * waits for the steps to end: on the device where it is asynchronous, on the
 * host otherwise.  The network's state is the same either way. */
fm_status surrogate_train(fm_ctx* ctx, const fm_train_opts* opts, fm_train_report* report);

/* End of a training run launched with async_run = 1: waits for its steps
 * and fills the whole report (report nullable).  FM_EINVAL if no run is in
 * flight. */
fm_status surrogate_train_finish(fm_ctx* ctx, fm_train_report* report);

/* Schedule of surrogate_eval_mc (and of the surrogate level in MC mode):
 * on = 1 (the default), for M <= 256 the whole network runs in one kernel per
 * 128 rows (inputs formed in shared memory, the hidden layers back to back on
 * the tensor cores, activations never leaving the SM); on = 0, layer by layer
 * through device memory.  Both give the same S bit for bit. */
fm_status surrogate_set_fused(fm_ctx* ctx, int32_t on);

/* d_s[s] = S(d_xi[s]) for n rows of FP64 KL coefficients [n][M]. */
fm_status surrogate_eval(fm_ctx* ctx, uint32_t n, const double* d_xi, double* d_s, void* stream);

/* S for the MC samples first .. first+n-1 of Philox stream `stream_level`
 * (the `level` argument of mc_points; the surrogate level draws from stream
 * 12), evaluated from the samples' Philox words: u from the top 23 bits of
 * each word, FP32 inverse normal, BF16 network input.  This is the map the
 * estimator applies on both levels where S enters in MC mode, so S is the
 * same function of the sample there.  d_s: device [n] FP64.  Asynchronous on
 * `stream`; FM_EINVAL without an installed network. */
fm_status surrogate_eval_mc(fm_ctx* ctx, uint32_t stream_level, uint64_t first, uint32_t n, double* d_s,
                            void* stream);

/* ---------------------------------------------------------------- profiling */

/* Per-kernel-family timing for roofline reports (not part of the method).
 * While a profile is open, the library records a CUDA event pair on the
 * launching stream around every launch of the families in `family_mask`
 * (bit f = family f, see fm_kernel_family_name) and notes the algorithmic
 * bytes and flops of each launch. */
fm_status fm_profile_begin(fm_ctx* ctx, uint32_t family_mask);

typedef struct {
    int32_t family;       /* family index */
    int64_t launches;
    double ms;            /* sum of event-timed launch durations */
    double bytes;         /* sum of algorithmic bytes (the resident FMG: the byte model of the
                             V-cycles and residual tests it ran, as if each grid operation
                             streamed its operands through HBM) */
    double flops;         /* sum of algorithmic flops */
    double flops_fp64;    /* the part of flops done in FP64 (kernels that count their own work) */
} fm_kernel_stat;

/* Close the profile: synchronises the device, returns one entry per family
 * with at least one launch (at most max_stats) and the count in *n_stats. */
fm_status fm_profile_end(fm_ctx* ctx, fm_kernel_stat* stats, int32_t max_stats, int32_t* n_stats);

/* Name of kernel family f (NULL when out of range). */
const char* fm_kernel_family_name(int32_t family);

#ifdef __cplusplus
}
#endif
#endif /* FMGMLMC_H */
