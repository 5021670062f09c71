// Karhunen-Loeve field synthesis (Sec. 3.1) and the one-time basis setup.
//
// kl_field_batch is the contraction K[s][c] = exp(sum_k B[c][k] xi[s][k]):
// cells x modes by modes x samples.  The FP64 form below is a register-tiled
// SIMT GEMM (FP64 has no fast tensor-core path on this part) with the
// exponential fused into the epilogue, so g is never written to memory.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace fm {

// 64 samples x 64 cells per CTA, 16 x 16 threads, 4 x 4 outputs per thread,
// modes staged through shared memory 16 at a time.
constexpr int kTS = 64, kTC = 64, kTK = 16;

__global__ void __launch_bounds__(256) k_kl_gemm_exp_f64(int cells, int M, int S,
                                                        const double* __restrict__ xi,
                                                        const double* __restrict__ B,
                                                        double* __restrict__ K) {
    __shared__ double sx[kTK][kTS + 1];
    __shared__ double sb[kTK][kTC + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int s0 = blockIdx.y * kTS, c0 = blockIdx.x * kTC;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < M; k0 += kTK) {
        // each thread loads 4 elements of each tile (64 rows x 16 modes)
        for (int e = threadIdx.x; e < kTS * kTK; e += 256) {
            const int r = e / kTK, kk = e % kTK;
            const int s = s0 + r, c = c0 + r, k = k0 + kk;
            sx[kk][r] = (s < S && k < M) ? xi[(size_t)s * M + k] : 0.0;
            sb[kk][r] = (c < cells && k < M) ? B[(size_t)c * M + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = sx[kk][ty + 16 * u];
                bb[u] = sb[kk][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int s = s0 + ty + 16 * u;
        if (s >= S) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = c0 + tx + 16 * v;
            if (c < cells) K[(size_t)s * cells + c] = exp(acc[u][v]);
        }
    }
}

// rows of the finest-grid basis kept by grid n: cell (i, j) -> (s i, s j)
__global__ void k_gather_rows(int n, int n_ref, int M, const double* __restrict__ Bref,
                              double* __restrict__ Bl) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * n * M) return;
    const int k = (int)(t % M);
    const size_t c = t / M;
    const int i = (int)(c % n), j = (int)(c / n), s = n_ref / n;
    Bl[t] = Bref[((size_t)(s * j) * n_ref + (size_t)s * i) * M + k];
}

// Weighted covariance matrix of the Nystrom method on the q x q midpoint grid.
__global__ void k_nystrom_matrix(int q, double nu, double sigma2, double lambda, double* __restrict__ A) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)q * q;
    if (t >= n * n) return;
    const size_t a = t / n, b = t % n;
    const double xa = ((double)(a % q) + 0.5) / q, ya = ((double)(a / q) + 0.5) / q;
    const double xb = ((double)(b % q) + 0.5) / q, yb = ((double)(b / q) + 0.5) / q;
    const double d = sqrt((xa - xb) * (xa - xb) + (ya - yb) * (ya - yb));
    A[t] = matern(nu, sigma2, lambda, d) / (double)n;
}

// Covariance between field points (rows) and quadrature nodes (columns),
// times sqrt(w): C[x][j] = sqrt(w) C_nu(|x - x_j|).
__global__ void k_nystrom_cross(int n_ref, size_t first, size_t rows, int q, double nu, double sigma2,
                                double lambda, double* __restrict__ C) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nq = (size_t)q * q;
    if (t >= rows * nq) return;
    const size_t r = first + t / nq, jq = t % nq;
    const double x = ((double)(r % n_ref) + 0.5) / n_ref, y = ((double)(r / n_ref) + 0.5) / n_ref;
    const double xq = ((double)(jq % q) + 0.5) / q, yq = ((double)(jq / q) + 0.5) / q;
    const double d = sqrt((x - xq) * (x - xq) + (y - yq) * (y - yq));
    C[t] = matern(nu, sigma2, lambda, d) / sqrt((double)nq);
}

// B[x][k] *= 1/sqrt(theta_k)
__global__ void k_scale_cols(size_t rows, int M, const double* __restrict__ inv_sqrt_theta,
                             double* __restrict__ B) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * M) return;
    B[t] *= inv_sqrt_theta[t % M];
}

static unsigned nblocks(size_t threads, int bs = 256) { return (unsigned)((threads + bs - 1) / bs); }

static fm_status install_basis(fm_ctx* ctx, const double* d_Bref) {
    const int L = ctx->cfg.n_levels, M = ctx->cfg.M, n_ref = finest_grid(ctx);
    for (int l = 0; l < L; ++l) {
        const int n = grid_of_level(ctx, l);
        const size_t cnt = (size_t)n * n * M;
        if (!ctx->d_basis[l]) {
            if (cudaMalloc((void**)&ctx->d_basis[l], cnt * sizeof(double)) != cudaSuccess) {
                set_error(ctx, "kl basis allocation failed");
                return FM_ENOMEM;
            }
        }
        if (ctx->d_basis[l] != d_Bref)   // the finest grid may have been built in place
            k_gather_rows<<<nblocks(cnt), 256>>>(n, n_ref, M, d_Bref, ctx->d_basis[l]);
        FM_CUDA_TRY(ctx, cudaGetLastError());
    }
    FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    const int mode = kl_mode_of(ctx);
    if (mode == FM_KL_BF16 || mode == FM_KL_BF16X3) FM_TRY(kl_tc_install(ctx, mode == FM_KL_BF16X3));
    ctx->basis_ready = true;
    return FM_OK;
}

int kl_mode_of(const fm_ctx* ctx) {
    if (ctx->cfg.kl_mode != FM_KL_AUTO) return ctx->cfg.kl_mode;
    return ctx->cfg.precision == FM_PREC_MIXED ? FM_KL_BF16X3 : FM_KL_FP64;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status kl_basis_set(fm_ctx* ctx, const double* basis_ref, int32_t on_device) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "kl_basis_set: null context");
    FM_CHECK_ARG(ctx, basis_ref != nullptr, "kl_basis_set: null basis");
    const int n_ref = finest_grid(ctx);
    const size_t cnt = (size_t)n_ref * n_ref * ctx->cfg.M;
    if (on_device) return install_basis(ctx, basis_ref);
    double* tmp = nullptr;
    if (cudaMalloc((void**)&tmp, cnt * sizeof(double)) != cudaSuccess) {
        set_error(ctx, "kl_basis_set: staging allocation failed");
        return FM_ENOMEM;
    }
    fm_status st = FM_OK;
    if (cudaMemcpy(tmp, basis_ref, cnt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error(ctx, "kl_basis_set: host-to-device copy failed");
        st = FM_ECUDA;
    } else {
        st = install_basis(ctx, tmp);
    }
    cudaFree(tmp);
    return st;
}

extern "C" fm_status kl_basis_build(fm_ctx* ctx, int32_t q, double* theta_out, double* captured_out) {
    return kl_basis_build_ex(ctx, q, FM_INTERP_AUTO, theta_out, captured_out);
}

extern "C" fm_status kl_basis_build_ex(fm_ctx* ctx, int32_t q, int32_t interp, double* theta_out,
                                       double* captured_out) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "kl_basis_build: null context");
    FM_CHECK_ARG(ctx, interp >= FM_INTERP_AUTO && interp <= FM_INTERP_TENSOR, "kl_basis_build: unknown interp");
    const int M = ctx->cfg.M;
    if (q <= 0) {
        q = 32;
        while ((int64_t)q * q < 8LL * M) q += 8;
    }
    const int nq = q * q;
    FM_CHECK_ARG(ctx, nq >= M, "kl_basis_build: q^2 must be >= M");
    FM_CHECK_ARG(ctx, nq <= 16384, "kl_basis_build: q^2 must be <= 16384");
    const int n_ref = finest_grid(ctx);
    const size_t rows = (size_t)n_ref * n_ref;
    const double sigma2 = ctx->cfg.sigma2, lambda = ctx->cfg.lambda, nu = matern_nu(ctx->cfg);
    // the interpolation B = C_x V costs 2 n_ref^2 q^2 M flops: FP64 up to 2e12,
    // the tensor cores (BF16x3) above, unless the caller chooses
    const bool tensor = interp == FM_INTERP_TENSOR ||
                        (interp == FM_INTERP_AUTO && 2.0 * (double)rows * nq * M > 2e12);

    double *dA = nullptr, *dW = nullptr, *dV = nullptr, *dC = nullptr, *dB = nullptr, *dInv = nullptr,
           *dWork = nullptr;
    int* dInfo = nullptr;
    cusolverDnHandle_t sol = nullptr;
    cublasHandle_t blas = nullptr;
    fm_status st = FM_OK;
    const size_t chunk = std::min<size_t>(rows, std::max<size_t>(1, ((size_t)1 << 28) / nq));
    auto fail = [&](fm_status s, const char* msg) {
        set_error(ctx, std::string("kl_basis_build: ") + msg);
        st = s;
    };
    do {
        if (cudaMalloc((void**)&dA, sizeof(double) * nq * nq) != cudaSuccess ||
            cudaMalloc((void**)&dW, sizeof(double) * nq) != cudaSuccess ||
            cudaMalloc((void**)&dV, sizeof(double) * (size_t)nq * M) != cudaSuccess ||
            (!tensor && cudaMalloc((void**)&dC, sizeof(double) * chunk * nq) != cudaSuccess) ||
            (!tensor && cudaMalloc((void**)&dB, sizeof(double) * rows * M) != cudaSuccess) ||
            cudaMalloc((void**)&dInv, sizeof(double) * M) != cudaSuccess ||
            cudaMalloc((void**)&dInfo, sizeof(int)) != cudaSuccess) {
            fail(FM_ENOMEM, "allocation failed");
            break;
        }
        k_nystrom_matrix<<<nblocks((size_t)nq * nq), 256>>>(q, nu, sigma2, lambda, dA);
        if (cusolverDnCreate(&sol) != CUSOLVER_STATUS_SUCCESS || cublasCreate(&blas) != CUBLAS_STATUS_SUCCESS) {
            fail(FM_ECUDA, "library handle creation failed");
            break;
        }
        int lwork = 0;
        if (cusolverDnDsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nq, dA, nq,
                                        dW, &lwork) != CUSOLVER_STATUS_SUCCESS) {
            fail(FM_ECUDA, "syevd workspace query failed");
            break;
        }
        if (cudaMalloc((void**)&dWork, sizeof(double) * (size_t)lwork) != cudaSuccess) {
            fail(FM_ENOMEM, "syevd workspace allocation failed");
            break;
        }
        if (cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nq, dA, nq, dW, dWork,
                             lwork, dInfo) != CUSOLVER_STATUS_SUCCESS) {
            fail(FM_ECUDA, "syevd failed");
            break;
        }
        int info = 0;
        std::vector<double> w(nq), V((size_t)nq * M);
        if (cudaMemcpy(&info, dInfo, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || info != 0) {
            fail(FM_ECUDA, "syevd did not converge");
            break;
        }
        cudaMemcpy(w.data(), dW, sizeof(double) * nq, cudaMemcpyDeviceToHost);
        // eigenvalues ascend; column c of dA (column-major) is eigenvector c.
        // Keep the top M, descending, each with its largest entry positive.
        std::vector<double> col(nq), theta(M), inv(M), Vt(tensor ? (size_t)nq * M : 0);
        double trace = 0.0;
        for (int a = 0; a < nq; ++a) trace += w[a];
        for (int k = 0; k < M; ++k) {
            const int c = nq - 1 - k;
            cudaMemcpy(col.data(), dA + (size_t)c * nq, sizeof(double) * nq, cudaMemcpyDeviceToHost);
            int arg = 0;
            for (int a = 1; a < nq; ++a)
                if (std::fabs(col[a]) > std::fabs(col[arg])) arg = a;
            const double sgn = col[arg] < 0 ? -1.0 : 1.0;
            for (int a = 0; a < nq; ++a) V[(size_t)a * M + k] = sgn * col[a];   // V[j][k]
            if (tensor)
                for (int a = 0; a < nq; ++a) Vt[(size_t)k * nq + a] = sgn * col[a];   // V^T[k][j]
            theta[k] = w[c];
            inv[k] = 1.0 / std::sqrt(w[c]);
        }
        cudaMemcpy(dV, tensor ? Vt.data() : V.data(), sizeof(double) * (size_t)nq * M, cudaMemcpyHostToDevice);
        cudaMemcpy(dInv, inv.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
        if (tensor) {
            // the finest grid's basis is interpolated in place; coarser grids gather from it
            double*& fine = ctx->d_basis[ctx->cfg.n_levels - 1];
            if (!fine && cudaMalloc((void**)&fine, sizeof(double) * rows * M) != cudaSuccess) {
                fail(FM_ENOMEM, "allocation of the finest basis failed");
                break;
            }
            st = kl_tc_nystrom(ctx, q, dV, dInv, fine);
            if (st == FM_OK) st = install_basis(ctx, fine);
            if (st == FM_OK) {
                if (theta_out) std::copy(theta.begin(), theta.end(), theta_out);
                if (captured_out) {
                    double kept = 0.0;
                    for (double t : theta) kept += t;
                    *captured_out = kept / trace;
                }
            }
            break;
        }
        // B = Cx V (row-major [rows][M]) in chunks of field points, via the
        // column-major identity B^T = V^T Cx^T.
        const double one = 1.0, zero = 0.0;
        for (size_t r0 = 0; r0 < rows && st == FM_OK; r0 += chunk) {
            const size_t nr = std::min(chunk, rows - r0);
            k_nystrom_cross<<<nblocks(nr * nq), 256>>>(n_ref, r0, nr, q, nu, sigma2, lambda, dC);
            if (cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, M, (int)nr, nq, &one, dV, M, dC, nq, &zero,
                            dB + r0 * M, M) != CUBLAS_STATUS_SUCCESS)
                fail(FM_ECUDA, "dgemm failed");
        }
        if (st != FM_OK) break;
        k_scale_cols<<<nblocks(rows * M), 256>>>(rows, M, dInv, dB);
        if (cudaDeviceSynchronize() != cudaSuccess) {
            fail(FM_ECUDA, "kernel failure");
            break;
        }
        st = install_basis(ctx, dB);
        if (st == FM_OK) {
            if (theta_out) std::copy(theta.begin(), theta.end(), theta_out);
            if (captured_out) {
                double kept = 0.0;
                for (double t : theta) kept += t;
                *captured_out = kept / trace;
            }
        }
    } while (0);
    if (sol) cusolverDnDestroy(sol);
    if (blas) cublasDestroy(blas);
    cudaFree(dA); cudaFree(dW); cudaFree(dV); cudaFree(dC); cudaFree(dB); cudaFree(dInv);
    cudaFree(dWork); cudaFree(dInfo);
    return st;
}

extern "C" fm_status kl_basis_get(const fm_ctx* ctx, double* basis_ref_out, int32_t on_device) {
    FM_CHECK_ARG(ctx, ctx != nullptr && basis_ref_out != nullptr, "kl_basis_get: null argument");
    FM_CHECK_ARG(ctx, ctx->basis_ready, "kl_basis_get: no KL basis installed");
    const int n_ref = finest_grid(ctx);
    const size_t bytes = (size_t)n_ref * n_ref * ctx->cfg.M * sizeof(double);
    FM_CUDA_TRY(ctx, cudaMemcpy(basis_ref_out, ctx->d_basis[ctx->cfg.n_levels - 1], bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return FM_OK;
}

extern "C" fm_status kl_field_batch(fm_ctx* ctx, int32_t level, uint32_t n, const double* d_xi,
                                    double* d_K, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "kl_field_batch: null context");
    FM_CHECK_ARG(ctx, level >= 0 && level < ctx->cfg.n_levels, "kl_field_batch: bad level");
    FM_CHECK_ARG(ctx, ctx->basis_ready, "kl_field_batch: no KL basis installed");
    FM_CHECK_ARG(ctx, n == 0 || (d_xi && d_K), "kl_field_batch: null pointer");
    if (n == 0) return FM_OK;
    const int mode = kl_mode_of(ctx);
    if (mode == FM_KL_BF16 || mode == FM_KL_BF16X3)
        return kl_tc_field(ctx, level, n, d_xi, d_K, as_stream(stream));
    const int N = grid_of_level(ctx, level);
    const int cells = N * N;
    dim3 grid((cells + kTC - 1) / kTC, (n + kTS - 1) / kTS);
    FM_CHECK_ARG(ctx, grid.y <= 65535, "kl_field_batch: too many samples in one call");
    const double M = ctx->cfg.M;
    FM_TIMED(ctx, kFamKlGemm, as_stream(stream), 8.0 * ((double)n * M + (double)cells * M + (double)n * cells),
             2.0 * n * (double)cells * M,
             k_kl_gemm_exp_f64<<<grid, 256, 0, as_stream(stream)>>>(cells, ctx->cfg.M, (int)n, d_xi,
                                                                  ctx->d_basis[level], d_K));
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status fm_matern_covariance(double nu, double sigma2, double lambda, const double* d, int64_t n,
                                          double* c) {
    if (!(nu == 0.5 || nu == 1.0 || nu == 1.5 || nu == 2.5) || !(sigma2 > 0) || !(lambda > 0) || n < 0 ||
        (n > 0 && (!d || !c)))
        return FM_EINVAL;
    for (int64_t k = 0; k < n; ++k) {
        if (!(d[k] >= 0)) return FM_EINVAL;
        c[k] = fm::matern(nu, sigma2, lambda, d[k]);
    }
    return FM_OK;
}
