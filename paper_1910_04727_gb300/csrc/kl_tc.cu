// Tensor-core KL field synthesis (Sec. 3.1) for the mixed form:
//   K[s][c] = exp( sum_k A[c][k] B[s][k] ),
// A = the level's basis sqrt(theta_k) phi_k(x_c) and B = the KL coefficients,
// both BF16 and K-major, FP32 accumulation in tensor memory.
//
// One CTA computes a 128-cell x 256-sample tile: warp 0 (one thread) streams
// 64-wide K blocks of A and B into shared memory with TMA (128-byte
// swizzle), warp 1 (one thread) issues tcgen05.mma into a 128 x 256 FP32
// accumulator in TMEM, and all four warps drain TMEM with tcgen05.ld, apply
// exp and store FP64 fields (consecutive cells across a warp: coalesced).
//
// Split precision ("bf16x3"): the host lays out A' = [A_hi | A_hi | A_lo] and
// B' = [B_hi | B_lo | B_hi] along an extended K, so one GEMM gives
// A_hi B_hi + A_hi B_lo + A_lo B_hi, the product to about 2^-16 relative
// instead of BF16's 2^-8, still on the tensor cores.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "tc.cuh"

namespace fm {

constexpr int kTcM = 128;     // cells per tile (MMA M)
constexpr int kTcN = 256;     // samples per tile (MMA N)
constexpr int kTcK = 64;      // K elements per stage (one 128-byte swizzle row)
constexpr int kTcStages = 2;
constexpr uint32_t kTcABytes = kTcM * kTcK * 2;   // 16 KiB
constexpr uint32_t kTcBBytes = kTcN * kTcK * 2;   // 32 KiB
constexpr size_t kTcSmem = 1024 + kTcStages * (kTcABytes + kTcBBytes) + 256;

// EPI 0 (field synthesis): K[s][c] = exp(D[c][s]).  EPI 1 (Nystrom
// interpolation of the KL basis): K[c][s] = D[c][s] colscale[s], row-major
// [cells][S] in FP64.
template <int EPI>
__global__ void __launch_bounds__(128, 1)
    k_kl_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int cells,
                 int S, int kblocks, double* __restrict__ K, int* __restrict__ err,
                 const double* __restrict__ colscale) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    uint8_t* base = smem_raw + ((1024 - (raw & 1023)) & 1023);   // 1024-byte aligned tiles
    uint8_t* sA = base;
    uint8_t* sB = base + kTcStages * kTcABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kTcStages * kTcBBytes);
    uint64_t* empty = full + kTcStages;
    uint64_t* done = empty + kTcStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * kTcM, s0 = blockIdx.y * kTcN;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::prefetch_tensormap(&mapA);
        tc::prefetch_tensormap(&mapB);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, kTcN);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: K blocks through a kTcStages-deep ring
        int issued = 0;
        for (int kb = 0; kb < kblocks; ++kb) {
            const int st = kb % kTcStages, round = kb / kTcStages;
            if (round > 0 && !tc::mbar_wait(&empty[st], (round - 1) & 1, err)) break;
            tc::mbar_arrive_expect_tx(&full[st], kTcABytes + kTcBBytes);
            tc::tma_load_2d(sA + st * kTcABytes, &mapA, &full[st], kb * kTcK, c0);
            tc::tma_load_2d(sB + st * kTcBBytes, &mapB, &full[st], kb * kTcK, s0);
            ++issued;
        }
        tc::drain_loads(full, kTcStages, issued, err);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four K=16 steps per stage, accumulate after the first
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, kTcN);
        for (int kb = 0; kb < kblocks; ++kb) {
            const int st = kb % kTcStages, round = kb / kTcStages;
            if (!tc::mbar_wait(&full[st], round & 1, err)) break;
            tc::fence_after_sync();
            const uint32_t a = tc::smem_u32(sA + st * kTcABytes), b = tc::smem_u32(sB + st * kTcBBytes);
#pragma unroll
            for (int j = 0; j < kTcK / 16; ++j)
                tc::mma_bf16(tmem, tc::sdesc_kmajor_sw128(a + 32 * j), tc::sdesc_kmajor_sw128(b + 32 * j), idesc,
                             (kb | j) != 0);
            tc::mma_commit(&empty[st]);   // frees the stage once these MMAs have read it
        }
        tc::mma_commit(done);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait(done, 0, err);
    __syncwarp();
    tc::fence_after_sync();
    if (ok) {
        const int c = c0 + warp * 32 + lane;
        const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int chunk = 0; chunk < kTcN / 32; ++chunk) {
            uint32_t r[32];
            tc::tmem_ld_32x32b_x32(row + chunk * 32, r);
            if (c < cells) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int s = s0 + chunk * 32 + i;
                    if (s >= S) continue;
                    if (EPI == 0) K[(size_t)s * cells + c] = (double)expf(__uint_as_float(r[i]));
                    else K[(size_t)c * S + s] = (double)__uint_as_float(r[i]) * colscale[s];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcN);
}

// One CTA waits, with the bounded wait of the kernels above, on an mbarrier
// that no thread ever arrives on: the wait runs out after budget_ns, sets
// *err and the kernel returns.
__global__ void k_wait_check(uint64_t budget_ns, int* __restrict__ err) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
    tc::mbar_wait(&bar, 0, err, budget_ns);
}

// A operand of the Nystrom interpolation: field points r0 .. r0+rows-1 (cell
// centres of the n_ref grid, row-major) against the q x q quadrature nodes:
// sqrt(w) C(|x - x_j|), w = 1/q^2, in the split layout (hi, hi, lo) of row
// length 3 Kpad (columns beyond q^2 are zero).
__global__ void k_nystrom_cross_bf16(int n_ref, size_t r0, size_t rows, int q, int Kpad, double nu, double sigma2,
                                     double lambda, __nv_bfloat16* __restrict__ out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * Kpad) return;
    const size_t rr = t / Kpad;
    const int jq = (int)(t % Kpad);
    const int nq = q * q;
    double v = 0.0;
    if (jq < nq) {
        const size_t r = r0 + rr;
        const double x = ((double)(r % n_ref) + 0.5) / n_ref, y = ((double)(r / n_ref) + 0.5) / n_ref;
        const double xq = ((double)(jq % q) + 0.5) / q, yq = ((double)(jq / q) + 0.5) / q;
        const double d = sqrt((x - xq) * (x - xq) + (y - yq) * (y - yq));
        v = matern(nu, sigma2, lambda, d) / q;
    }
    const __nv_bfloat16 hi = __double2bfloat16(v);
    __nv_bfloat16* o = out + rr * (size_t)(3 * Kpad);
    o[jq] = hi;
    o[Kpad + jq] = hi;
    o[2 * Kpad + jq] = __double2bfloat16(v - (double)__bfloat162float(hi));
}

// x [n][M] FP64 -> [n][Kp] BF16 in the split layout (hi, lo, hi) or plain (hi).
__global__ void k_xi_to_bf16(size_t n, int M, int Mpad, int split, const double* __restrict__ x,
                             __nv_bfloat16* __restrict__ out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * Mpad) return;
    const size_t s = t / Mpad;
    const int k = (int)(t % Mpad);
    const double v = (k < M) ? x[s * M + k] : 0.0;
    const __nv_bfloat16 hi = __double2bfloat16(v);
    const int Kp = split ? 3 * Mpad : Mpad;
    __nv_bfloat16* o = out + s * Kp;
    o[k] = hi;
    if (split) {
        o[Mpad + k] = __double2bfloat16(v - (double)__bfloat162float(hi));
        o[2 * Mpad + k] = hi;
    }
}

// basis [cells][M] FP64 -> [cells][Kp] BF16, split layout (hi, hi, lo).
__global__ void k_basis_to_bf16(size_t cells, int M, int Mpad, int split, const double* __restrict__ B,
                                __nv_bfloat16* __restrict__ out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cells * Mpad) return;
    const size_t c = t / Mpad;
    const int k = (int)(t % Mpad);
    const double v = (k < M) ? B[c * M + k] : 0.0;
    const __nv_bfloat16 hi = __double2bfloat16(v);
    const int Kp = split ? 3 * Mpad : Mpad;
    __nv_bfloat16* o = out + c * Kp;
    o[k] = hi;
    if (split) {
        o[Mpad + k] = hi;
        o[2 * Mpad + k] = __double2bfloat16(v - (double)__bfloat162float(hi));
    }
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// [rows][Kp] BF16, box 64 x box_rows, 128-byte swizzle, zero fill outside.
static bool make_map(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t Kp, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {Kp, rows};
    cuuint64_t strides[1] = {Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static unsigned nblk(size_t threads) { return (unsigned)((threads + 255) / 256); }

fm_status kl_tc_install(fm_ctx* ctx, int split) {
    const int M = ctx->cfg.M, Mpad = (M + kTcK - 1) / kTcK * kTcK, Kp = split ? 3 * Mpad : Mpad;
    ctx->tc.split = split;
    ctx->tc.Mpad = Mpad;
    ctx->tc.Kp = Kp;
    for (int l = 0; l < ctx->cfg.n_levels; ++l) {
        const int n = grid_of_level(ctx, l);
        const size_t cells = (size_t)n * n;
        cudaFree(ctx->tc.basis[l]);
        ctx->tc.basis[l] = nullptr;
        if (cudaMalloc((void**)&ctx->tc.basis[l], cells * Kp * 2) != cudaSuccess) {
            set_error(ctx, "tensor-core basis allocation failed");
            return FM_ENOMEM;
        }
        k_basis_to_bf16<<<nblk(cells * Mpad), 256>>>(cells, M, Mpad, split, ctx->d_basis[l],
                                                     (__nv_bfloat16*)ctx->tc.basis[l]);
        if (!make_map(&ctx->tc.mapA[l], ctx->tc.basis[l], cells, Kp, kTcM)) {
            set_error(ctx, "cuTensorMapEncodeTiled failed for the basis");
            return FM_ECUDA;
        }
    }
    FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    ctx->tc.ready = true;
    return FM_OK;
}

fm_status kl_tc_field(fm_ctx* ctx, int level, uint32_t n, const double* d_xi, double* d_K, cudaStream_t st) {
    const int N = grid_of_level(ctx, level), cells = N * N, M = ctx->cfg.M;
    const int Mpad = ctx->tc.Mpad, Kp = ctx->tc.Kp;
    if (ctx->tc.xi_capacity < (size_t)n) {
        cudaFree(ctx->tc.xi);
        ctx->tc.xi = nullptr;
        ctx->tc.xi_capacity = 0;
        if (cudaMalloc((void**)&ctx->tc.xi, (size_t)n * Kp * 2) != cudaSuccess) {
            set_error(ctx, "tensor-core coefficient buffer allocation failed");
            return FM_ENOMEM;
        }
        ctx->tc.xi_capacity = n;
        if (!make_map(&ctx->tc.mapB, ctx->tc.xi, n, Kp, kTcN)) {
            set_error(ctx, "cuTensorMapEncodeTiled failed for the coefficients");
            return FM_ECUDA;
        }
        ctx->tc.mapB_rows = n;
    }
    if (!ctx->tc.err) {
        // the flag stays set until fm_sync reports it
        FM_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->tc.err, sizeof(int)));
        FM_CUDA_TRY(ctx, cudaMemset(ctx->tc.err, 0, sizeof(int)));
    }
    static bool attr = false;
    if (!attr) {
        FM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_kl_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kTcSmem));
        FM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_kl_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kTcSmem));
        attr = true;
    }
    k_xi_to_bf16<<<nblk((size_t)n * Mpad), 256, 0, st>>>(n, M, Mpad, ctx->tc.split, d_xi,
                                                        (__nv_bfloat16*)ctx->tc.xi);
    // the coefficient map covers the buffer's capacity; rows >= n are never stored
    dim3 grid((cells + kTcM - 1) / kTcM, (n + kTcN - 1) / kTcN);
    const double flops = 2.0 * (double)n * cells * Kp;
    const double bytes = 2.0 * ((double)cells * Kp + (double)n * Kp) + 8.0 * (double)n * cells;
    FM_TIMED(ctx, kFamKlGemm, st, bytes, flops,
             k_kl_gemm_tc<0><<<grid, 128, kTcSmem, st>>>(ctx->tc.mapA[level],
                                                        ctx->tc.mapB, cells, (int)n,
                                                        Kp / kTcK, d_K, ctx->tc.err, nullptr));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

}  // namespace fm

namespace fm {

// Nystrom interpolation of the KL basis on the tensor cores:
// out[x][k] = inv_sqrt_theta[k] sum_j sqrt(w) C(x, x_j) V[j][k] over the
// n_ref^2 field points, with dVt = V^T [M][q^2] FP64, as one BF16x3 GEMM per
// chunk of field points (products to about 2^-16 relative, FP32
// accumulation in tensor memory).  Synchronous; the bounded waits report
// FM_ETIMEOUT.
fm_status kl_tc_nystrom(fm_ctx* ctx, int q, const double* dVt, const double* d_inv_sqrt_theta, double* d_out) {
    const int M = ctx->cfg.M, n_ref = finest_grid(ctx), nq = q * q;
    const int Kpad = (nq + kTcK - 1) / kTcK * kTcK, Kp = 3 * Kpad;
    const size_t rows = (size_t)n_ref * n_ref;
    size_t chunk = std::max<size_t>(kTcM, ((size_t)2 << 30) / ((size_t)Kp * 2));   // about 2 GiB of A
    chunk = std::min(rows, chunk / kTcM * kTcM);
    void *A = nullptr, *B = nullptr;
    fm_status st = FM_OK;
    if (!ctx->tc.err) {
        FM_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->tc.err, sizeof(int)));
        FM_CUDA_TRY(ctx, cudaMemset(ctx->tc.err, 0, sizeof(int)));
    }
    static bool attr = false;
    if (!attr) {
        FM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_kl_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kTcSmem));
        attr = true;
    }
    do {
        if (cudaMalloc(&A, chunk * Kp * 2) != cudaSuccess || cudaMalloc(&B, (size_t)M * Kp * 2) != cudaSuccess) {
            set_error(ctx, "kl_basis_build: tensor-core interpolation buffers");
            st = FM_ENOMEM;
            break;
        }
        // B operand: V^T, split (hi, lo, hi)
        k_xi_to_bf16<<<nblk((size_t)M * Kpad), 256>>>((size_t)M, nq, Kpad, 1, dVt, (__nv_bfloat16*)B);
        CUtensorMap mapB, mapA;
        if (!make_map(&mapB, B, M, Kp, kTcN) || !make_map(&mapA, A, chunk, Kp, kTcM)) {
            set_error(ctx, "kl_basis_build: cuTensorMapEncodeTiled failed");
            st = FM_ECUDA;
            break;
        }
        const double nu = matern_nu(ctx->cfg), sigma2 = ctx->cfg.sigma2, lambda = ctx->cfg.lambda;
        for (size_t r0 = 0; r0 < rows; r0 += chunk) {
            const size_t nr = std::min(chunk, rows - r0);
            k_nystrom_cross_bf16<<<nblk(nr * Kpad), 256>>>(n_ref, r0, nr, q, Kpad, nu, sigma2, lambda,
                                                           (__nv_bfloat16*)A);
            dim3 grid((unsigned)((nr + kTcM - 1) / kTcM), (unsigned)((M + kTcN - 1) / kTcN));
            k_kl_gemm_tc<1><<<grid, 128, kTcSmem>>>(mapA, mapB, (int)nr, M, Kp / kTcK, d_out + r0 * M, ctx->tc.err,
                                                   d_inv_sqrt_theta);
        }
        if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            set_error(ctx, "kl_basis_build: tensor-core interpolation failed");
            st = FM_ECUDA;
            break;
        }
        int e = 0;
        cudaMemcpy(&e, ctx->tc.err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e) {
            cudaMemset(ctx->tc.err, 0, sizeof(int));
            set_error(ctx, "kl_basis_build: a bounded device-side wait ran out");
            st = FM_ETIMEOUT;
        }
    } while (0);
    cudaFree(A);
    cudaFree(B);
    return st;
}

}  // namespace fm

extern "C" fm_status fm_wait_check(fm_ctx* ctx, int64_t budget_ns, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_wait_check: null context");
    FM_CHECK_ARG(ctx, budget_ns >= 0 && budget_ns <= 1000000000LL, "fm_wait_check: budget must be 0 .. 1e9 ns");
    if (!ctx->tc.err) {
        FM_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->tc.err, sizeof(int)));
        FM_CUDA_TRY(ctx, cudaMemset(ctx->tc.err, 0, sizeof(int)));
    }
    cudaStream_t st = fm::as_stream(stream);
    fm::k_wait_check<<<1, 32, 0, st>>>((uint64_t)budget_ns, ctx->tc.err);
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}
