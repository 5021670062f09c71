// Surrogate control-variate level: an MLP S(xi) = mu + sd * f(xi), f a
// 4-layer perceptron M -> 256 -> 256 -> 256 -> 1 with GELU, trained by MSE
// and Adam on outflux samples the method itself produces, and used as one
// more estimator level below the coarsest grid:
//   E[Q_L] = E[S] + E[Q_0 - S] + sum_{l>=1} E[Q_l - Q_(l-1)]
// (unbiased for any S; a good S lowers the variance of Q_0 - S).
//
// Every hidden-layer contraction runs on the tcgen05 tensor cores: BF16
// operands staged by TMA (128-byte swizzle), FP32 accumulation in TMEM, and
// fused epilogues: forward bias + GELU writing the next layer's BF16 operand
// both row-major (next forward GEMM) and transposed (weight-gradient GEMM);
// backward GELU' writing the BF16 pre-activation gradient both ways; weight
// gradients in FP32.  The output layer (256 -> 1), bias gradients and Adam
// are small FP32 kernels.  Operands are BF16 exactly where the FP64 oracle
// rounds: weights, input, hidden activations, pre-activation gradients.
//
// Training runs as one CUDA graph per step (batch gather, forward, backward,
// Adam with the BF16 refresh, step counter) replayed for the whole run; the
// step number lives on the device, so every replay is the same graph.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <random>

#include "common.cuh"
#include "tc.cuh"

namespace fm {

constexpr int kH = 256;          // hidden width
constexpr int kGm = 128;         // GEMM tile rows (MMA M)
constexpr int kGk = 64;          // K per stage
constexpr int kGStages = 2;
constexpr int kMaxBatch = 4096;  // training mini-batch capacity (leading dimension of transposed operands)
constexpr int kLossBatch = 256;  // rows of surrogate_loss_grad
constexpr int kTrainBN = 64;     // N tile of the training GEMMs (more CTAs on small problems)
constexpr int kEvalBN = 256;     // N tile of the inference GEMMs
constexpr int kEvalChunk = 1 << 16;

enum EpiKind { kEpiFwdGelu = 0, kEpiBwdGelu = 1, kEpiF32 = 2 };

struct EpiArgs {
    int M, N;                       // valid rows / columns of D
    const float* bias;              // forward: [N]
    float* Z;                       // forward: pre-activation out; backward: pre-activation in
    int ldz;
    __nv_bfloat16* H;               // BF16 out, row-major [M][ldh]
    int ldh;
    __nv_bfloat16* HT;              // BF16 out, transposed [N][ldt] (nullable)
    int ldt;
    float* F;                       // FP32 out [M][ldf]
    int ldf;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Programmatic dependent launch: wait until the preceding kernel of the
// stream has completed (and its writes are visible), then let the next one be
// scheduled.  No-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// n consecutive FP32 / BF16 values of one row: 16-byte stores when the row
// chunk is whole and aligned, element stores otherwise.
__device__ __forceinline__ void store_row_f32(float* p, const float (&a)[32], int n) {
    if (n == 32 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            reinterpret_cast<float4*>(p)[i] = make_float4(a[4 * i], a[4 * i + 1], a[4 * i + 2], a[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i < n) p[i] = a[i];
    }
}

__device__ __forceinline__ void store_row_bf16(__nv_bfloat16* p, const __nv_bfloat16 (&h)[32], int n) {
    if (n == 32 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) reinterpret_cast<uint4*>(p)[i] = reinterpret_cast<const uint4*>(h)[i];
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i < n) p[i] = h[i];
    }
}

__device__ __forceinline__ void load_row_f32(const float* p, float (&a)[32], int n) {
    if (n == 32 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 v = reinterpret_cast<const float4*>(p)[i];
            a[4 * i] = v.x;
            a[4 * i + 1] = v.y;
            a[4 * i + 2] = v.z;
            a[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) a[i] = i < n ? p[i] : 0.0f;
    }
}

// D[m][n] = sum_k A[m][k] B[n][k]: A [M][K] and B [N][K] BF16 K-major, one
// 128 x BN tile per CTA, then the EPI epilogue on D.  Warp 0 lane 0 issues
// the TMA loads, warp 1 lane 0 the MMAs; all four warps drain TMEM (warp w
// owns rows 32w .. 32w+31 of the tile, one row per thread).
template <int BN, int EPI>
__global__ void __launch_bounds__(128, 1)
    k_gemm_bf16_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int kblocks,
                   EpiArgs e, int* __restrict__ err) {
    constexpr uint32_t kA = kGm * kGk * 2, kB = BN * kGk * 2;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    uint8_t* base = smem_raw + ((1024 - (raw & 1023)) & 1023);
    uint8_t* sA = base;
    uint8_t* sB = base + kGStages * kA;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kGStages * kB);
    uint64_t* empty = full + kGStages;
    uint64_t* done = empty + kGStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kGm, n0 = blockIdx.y * BN;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kGStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::prefetch_tensormap(&mapA);
        tc::prefetch_tensormap(&mapB);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, BN);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // the setup above overlaps the previous kernel; its outputs are read below
    pdl_wait_then_release();
    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int kb = 0; kb < kblocks; ++kb) {
            const int st = kb % kGStages, round = kb / kGStages;
            if (round > 0 && !tc::mbar_wait(&empty[st], (round - 1) & 1, err)) break;
            tc::mbar_arrive_expect_tx(&full[st], kA + kB);
            tc::tma_load_2d(sA + st * kA, &mapA, &full[st], kb * kGk, m0);
            tc::tma_load_2d(sB + st * kB, &mapB, &full[st], kb * kGk, n0);
            ++issued;
        }
        tc::drain_loads(full, kGStages, issued, err);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kGm, BN);
        for (int kb = 0; kb < kblocks; ++kb) {
            const int st = kb % kGStages, round = kb / kGStages;
            if (!tc::mbar_wait(&full[st], round & 1, err)) break;
            tc::fence_after_sync();
            const uint32_t a = tc::smem_u32(sA + st * kA), b = tc::smem_u32(sB + st * kB);
#pragma unroll
            for (int j = 0; j < kGk / 16; ++j)
                tc::mma_bf16(tmem, tc::sdesc_kmajor_sw128(a + 32 * j), tc::sdesc_kmajor_sw128(b + 32 * j), idesc,
                             (kb | j) != 0);
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(done);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait(done, 0, err);
    __syncwarp();
    tc::fence_after_sync();
    if (ok) {
        const int r = m0 + warp * 32 + lane;
        const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int chunk = 0; chunk < BN / 32; ++chunk) {
            uint32_t v[32];
            tc::tmem_ld_32x32b_x32(row + chunk * 32, v);
            const int c0 = n0 + chunk * 32;
            if (r >= e.M || c0 >= e.N) continue;
            const int n = min(32, e.N - c0);
            float a[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) a[i] = __uint_as_float(v[i]);
            if (EPI == kEpiF32) {
                store_row_f32(e.F + (size_t)r * e.ldf + c0, a, n);
                continue;
            }
            __nv_bfloat16 h[32];
            if (EPI == kEpiFwdGelu) {
#pragma unroll
                for (int i = 0; i < 32; ++i) a[i] += (i < n) ? __ldg(e.bias + c0 + i) : 0.0f;
                if (e.Z) store_row_f32(e.Z + (size_t)r * e.ldz + c0, a, n);
#pragma unroll
                for (int i = 0; i < 32; ++i) h[i] = __float2bfloat16_rn(gelu_f(a[i]));
            } else {
                float z[32];
                load_row_f32(e.Z + (size_t)r * e.ldz + c0, z, n);
#pragma unroll
                for (int i = 0; i < 32; ++i) h[i] = __float2bfloat16_rn(a[i] * gelu_grad_f(z[i]));
            }
            store_row_bf16(e.H + (size_t)r * e.ldh + c0, h, n);
            if (e.HT) {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (i < n) e.HT[(size_t)(c0 + i) * e.ldt + r] = h[i];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

template <int BN>
constexpr size_t gemm_smem() {
    return 1024 + kGStages * ((size_t)kGm * kGk * 2 + (size_t)BN * kGk * 2) + 256;
}

// ------------------------------------------------------------------ fused MC inference
// S for MC samples in one kernel, one 128-row tile per CTA (eight warps):
// the tile's BF16 inputs are formed from the samples' Philox words straight
// into shared memory (k_surrogate_x_mc's map), the three hidden layers run
// back to back on the tensor cores with the activations kept in shared
// memory between them (TMEM accumulator, bias + GELU + BF16 epilogue written
// as the next layer's A operand), and the output layer and S = mu + sd f
// close the tile.  Every value is formed as the layer-by-layer path forms it
// (same MMA sequence, same epilogue, k_mlp_out's summation order), so S is
// bit-identical to it; what goes away is the activations' round trips
// through HBM and five launches per 65536 rows.  Inputs up to 256 wide.
// Weights stream in blocks of 64 inputs x 128 outputs (16 KB, two MMAs of
// N = 128 per 64-input block), so a CTA takes 97 KB of shared memory and two
// CTAs share an SM: one's epilogue runs beside the other's loads and MMAs.
constexpr int kFusedRows = 128;
constexpr int kFusedThreads = 256;
constexpr uint32_t kFusedKBlock = kFusedRows * kGk * 2;   // 16 KB: 128 rows x 64 columns BF16
constexpr uint32_t kFusedWStage = (kH / 2) * kGk * 2;     // 16 KB: half the rows (128 outputs) x 64 columns BF16
constexpr int kFusedH3Stride = kH * 2 + 16;               // bytes per row of the staged last layer

__host__ __device__ constexpr size_t fused_smem_bytes() {
    return 1024 + 4 * (size_t)kFusedKBlock + 2 * (size_t)kFusedWStage + 128;
}

// Byte offset of element (r, k) of a 128 x 256 BF16 A operand stored as four
// K-blocks of 64 columns, each 128 rows of 128 bytes with the 128-byte
// swizzle (16-byte chunk c of row r at chunk c ^ (r mod 8)), the layout TMA
// writes for the tensor-core descriptors.
__device__ __forceinline__ uint32_t fused_a_offset(int r, int k) {
    const int kb = k >> 6, kk = k & 63;
    return (uint32_t)kb * kFusedKBlock + (uint32_t)r * 128u + (uint32_t)((((kk >> 3) ^ (r & 7)) << 4) | ((kk & 7) << 1));
}

struct FusedArgs {
    uint64_t seed, first;
    uint32_t level;
    int n, M, D;
    const float *b1, *b2, *b3, *b4;
    const __nv_bfloat16* w4;
    double mu, sd;
    double* s;
    int* err;
};

__global__ void __launch_bounds__(kFusedThreads, 2)
    k_mlp_infer_mc(const __grid_constant__ CUtensorMap mapW1, const __grid_constant__ CUtensorMap mapW2,
                   const __grid_constant__ CUtensorMap mapW3, FusedArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    uint8_t* base = smem_raw + ((1024 - (raw & 1023)) & 1023);
    uint8_t* sAct = base;                                   // the layer's A operand (4 K-blocks)
    uint8_t* sW = base + 4 * kFusedKBlock;                  // weight K-blocks, two stages
    uint64_t* full = reinterpret_cast<uint64_t*>(sW + 2 * kFusedWStage);
    uint64_t* empty = full + 2;
    uint64_t* done = empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * kFusedRows;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::prefetch_tensormap(&mapW1);
        tc::prefetch_tensormap(&mapW2);
        tc::prefetch_tensormap(&mapW3);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, kH);
    // the tile's inputs: 4 columns per Philox call, as k_surrogate_x_mc forms them
    {
        const int groups = a.D / 4;
        for (int t = threadIdx.x; t < kFusedRows * groups; t += kFusedThreads) {
            const int r = t / groups, g = t % groups;
            __align__(8) __nv_bfloat16 h[4];
            if (r0 + r < a.n && 4 * g < a.M) {
                u64x4 c = {{(uint64_t)g, a.first + (uint64_t)(r0 + r), 0, 0}};
                const u64x4 w = philox4x64(c, a.seed, (kPurposeMC << 32) | a.level);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float u = ((float)(w.v[q] >> 41) + 0.5f) * 0x1p-23f;
                    h[q] = __float2bfloat16_rn(4 * g + q < a.M ? normcdfinvf(u) : 0.0f);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = __float2bfloat16_rn(0.0f);
            }
            *reinterpret_cast<uint2*>(sAct + fused_a_offset(r, 4 * g)) = *reinterpret_cast<const uint2*>(h);
        }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // weight blocks (64 inputs x 128 outputs) in one sequence over the three
    // layers (W1: 2 D / 64, W2 and W3: 8 each; output half fastest), through
    // a two-stage ring: block q in stage q % 2
    const int kb1 = 2 * (a.D / kGk);
    const int lstart[4] = {0, kb1, kb1 + 8, kb1 + 16};
    const CUtensorMap* maps[3] = {&mapW1, &mapW2, &mapW3};
    const float* biases[3] = {a.b1, a.b2, a.b3};
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kFusedRows, kH / 2);
    int issued = 0;   // producer (warp 0 lane 0): weight blocks issued so far
    bool ok = true;
    const int qd = warp & 3, ch = warp >> 2;   // TMEM lane quadrant, column half of the epilogue
    const int r = 32 * qd + lane;               // the tile row this thread drains
    for (int L = 0; L < 3 && ok; ++L) {
        if (warp == 0 && lane == 0) {
            // this layer's blocks and up to two of the next one (their stages
            // free up as this layer's MMAs complete, without the epilogue)
            const int upto = L < 2 ? min(lstart[L + 1] + 2, lstart[L + 2]) : lstart[3];
            while (issued < upto) {
                const int q = issued, st = q & 1, lq = q < lstart[1] ? 0 : (q < lstart[2] ? 1 : 2);
                if (q >= 2 && !tc::mbar_wait(&empty[st], ((q >> 1) - 1) & 1, a.err)) break;
                const int u = q - lstart[lq];   // input block u / 2, output half u % 2
                tc::mbar_arrive_expect_tx(&full[st], kFusedWStage);
                tc::tma_load_2d(sW + st * kFusedWStage, maps[lq], &full[st], (u >> 1) * kGk, (u & 1) * (kH / 2));
                ++issued;
            }
        } else if (warp == 1 && lane == 0) {
            for (int q = lstart[L]; q < lstart[L + 1]; ++q) {
                const int st = q & 1, u = q - lstart[L], kb = u >> 1;
                if (!tc::mbar_wait(&full[st], (q >> 1) & 1, a.err)) break;
                tc::fence_after_sync();
                const uint32_t aa = tc::smem_u32(sAct + kb * kFusedKBlock), bb = tc::smem_u32(sW + st * kFusedWStage);
                const uint32_t dst = tmem + (uint32_t)((u & 1) * (kH / 2));   // the output half's TMEM columns
#pragma unroll
                for (int j = 0; j < kGk / 16; ++j)
                    tc::mma_bf16(dst, tc::sdesc_kmajor_sw128(aa + 32 * j), tc::sdesc_kmajor_sw128(bb + 32 * j), idesc,
                                 (kb | j) != 0);
                tc::mma_commit(&empty[st]);
            }
            tc::mma_commit(done);
        }
        __syncwarp();
        // every thread goes on alike: a wait that ran out anywhere ends the
        // layers for the whole CTA (the error flag is already set)
        ok = __syncthreads_and(tc::mbar_wait(done, L & 1, a.err)) != 0;
        tc::fence_after_sync();
        if (ok) {
            // bias + GELU + BF16, as the layer-by-layer epilogue forms it: the
            // next layer's A operand in place, the last layer's rows plainly
            const uint32_t trow = tmem + ((uint32_t)(32 * qd) << 16);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int c0 = ch * 128 + c * 32;
                uint32_t v[32];
                tc::tmem_ld_32x32b_x32(trow + c0, v);
                float x[32];
                __align__(16) __nv_bfloat16 h[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    x[i] = __uint_as_float(v[i]) + __ldg(biases[L] + c0 + i);
                    h[i] = __float2bfloat16_rn(gelu_f(x[i]));
                }
                if (L < 2) {
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        *reinterpret_cast<uint4*>(sAct + fused_a_offset(r, c0 + 8 * m)) =
                            reinterpret_cast<const uint4*>(h)[m];
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        *reinterpret_cast<uint4*>(base + (size_t)r * kFusedH3Stride + (c0 + 8 * m) * 2) =
                            reinterpret_cast<const uint4*>(h)[m];
                }
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (warp == 0 && lane == 0) tc::drain_loads(full, 2, issued, a.err);
    if (ok) {
        // output layer, one warp per row in k_mlp_out's order, then S = mu + sd f
        for (int rr = warp; rr < kFusedRows; rr += kFusedThreads / 32) {
            const __nv_bfloat16* h3 = reinterpret_cast<const __nv_bfloat16*>(base + (size_t)rr * kFusedH3Stride);
            float acc = 0.0f;
            for (int j = lane; j < kH; j += 32) acc += __bfloat162float(h3[j]) * __bfloat162float(a.w4[j]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
            if (lane == 0 && r0 + rr < a.n) {
                const float o = acc + a.b4[0];
                a.s[r0 + rr] = a.mu + a.sd * (double)o;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kH);
}

// ------------------------------------------------------------------ small kernels
// Rows of xi (FP64 [B][M]) -> BF16 X [B][D] (zero padded) and, if XT, XT [D][ldt].
__global__ void k_gather_x(int B, int M, int D, const double* __restrict__ xi, __nv_bfloat16* __restrict__ X,
                           __nv_bfloat16* __restrict__ XT, int ldt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * D) return;
    const int b = t / D, k = t % D;
    const __nv_bfloat16 v = __float2bfloat16_rn((float)(k < M ? xi[(size_t)b * M + k] : 0.0));
    X[(size_t)b * D + k] = v;
    if (XT) XT[(size_t)k * ldt + b] = v;
}

// out[b] = H3[b] . w4 + b4 (FP32), one warp per row; training: dout[b] =
// 2 (out[b] - t[b]) / B and the squared error.
__global__ void k_mlp_out(int B, const __nv_bfloat16* __restrict__ H3, const __nv_bfloat16* __restrict__ w4,
                          const float* __restrict__ b4, const float* __restrict__ t, float* __restrict__ out,
                          float* __restrict__ dout, float* __restrict__ sq) {
    pdl_wait_then_release();
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= B) return;
    float acc = 0.0f;
    for (int j = lane; j < kH; j += 32)
        acc += __bfloat162float(H3[(size_t)b * kH + j]) * __bfloat162float(w4[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        const float o = acc + b4[0];
        out[b] = o;
        if (t) {
            const float d = o - t[b];
            dout[b] = 2.0f * d / (float)B;
            sq[b] = d * d;
        }
    }
}

// Training: the output layer and its gradient in one pass, one warp per row:
// out, dout and the squared error as k_mlp_out forms them, then the
// pre-activation gradient dZ3 = bf16((dout w4) * gelu'(Z3)), row-major and
// transposed [kH][ldt].
__global__ void k_mlp_out_train(int B, int ldt, const __nv_bfloat16* __restrict__ H3,
                                const __nv_bfloat16* __restrict__ w4, const float* __restrict__ b4,
                                const float* __restrict__ t, float* __restrict__ out, float* __restrict__ dout,
                                float* __restrict__ sq, const float* __restrict__ Z3, __nv_bfloat16* __restrict__ dZ,
                                __nv_bfloat16* __restrict__ dZT) {
    pdl_wait_then_release();
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= B) return;
    float acc = 0.0f;
    for (int j = lane; j < kH; j += 32)
        acc += __bfloat162float(H3[(size_t)b * kH + j]) * __bfloat162float(w4[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    float dv = 0.0f;
    if (lane == 0) {
        const float o = acc + b4[0];
        out[b] = o;
        const float d = o - t[b];
        dv = 2.0f * d / (float)B;
        dout[b] = dv;
        sq[b] = d * d;
    }
    dv = __shfl_sync(0xffffffffu, dv, 0);
    for (int j = lane; j < kH; j += 32) {
        const float d = dv * __bfloat162float(w4[j]) * gelu_grad_f(Z3[(size_t)b * kH + j]);
        const __nv_bfloat16 v = __float2bfloat16_rn(d);
        dZ[(size_t)b * kH + j] = v;
        dZT[(size_t)j * ldt + b] = v;
    }
}

// Row sums of a transposed operand, one warp per row j (lanes over the batch,
// fixed order): gb[j] = sum_b w[b] T[j][b], with w = 1 when null.  With
// ones_row, warp N also writes gb[N] = sum_b w[b] (the output bias).
__global__ void k_row_sums(int N, int B, int ldt, const __nv_bfloat16* __restrict__ T, const float* __restrict__ w,
                           float* __restrict__ gb, float* __restrict__ ones_row) {
    pdl_wait_then_release();
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j > N || (j == N && !ones_row)) return;
    float acc = 0.0f;
    for (int b = lane; b < B; b += 32) {
        const float x = (j < N) ? __bfloat162float(T[(size_t)j * ldt + b]) : 1.0f;
        acc += w ? w[b] * x : x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        if (j < N) gb[j] = acc;
        else ones_row[0] = acc;
    }
}

// W [rows][cols] FP32 -> BF16 [rows][ld] (zero padded) and, if WT, [cols][rows].
__global__ void k_weight_bf16(int rows, int cols, int ld, const float* __restrict__ W, __nv_bfloat16* __restrict__ Wb,
                              __nv_bfloat16* __restrict__ WT) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * ld) return;
    const int r = t / ld, c = t % ld;
    const __nv_bfloat16 v = __float2bfloat16_rn(c < cols ? W[(size_t)r * cols + c] : 0.0f);
    Wb[t] = v;
    if (WT && c < cols) WT[(size_t)c * rows + r] = v;
}

__global__ void k_surrogate_value(int n, const float* __restrict__ out, double mu, double sd, double* __restrict__ s) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) s[t] = mu + sd * (double)out[t];
}

// Mini-batch `*step` of a training run: rows perm[(step / spe) * n + (step %
// spe) * B + b] of xi (FP64 [n][M]) and of the standardised targets tt, as
// the BF16 operands X [B][D] (zero padded) and XT [D][ldt] and the FP32 t [B].
__global__ void k_train_batch(int B, int M, int D, int ldt, int n, int spe, const int* __restrict__ step,
                              const int32_t* __restrict__ perm, const double* __restrict__ xi,
                              const float* __restrict__ tt, __nv_bfloat16* __restrict__ X,
                              __nv_bfloat16* __restrict__ XT, float* __restrict__ t) {
    pdl_wait_then_release();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * D) return;
    const int b = i / D, k = i % D;
    const int s = *step;
    const size_t row = (size_t)perm[(size_t)(s / spe) * n + (size_t)(s % spe) * B + b];
    const __nv_bfloat16 v = __float2bfloat16_rn((float)(k < M ? xi[row * M + k] : 0.0));
    X[(size_t)b * D + k] = v;
    XT[(size_t)k * ldt + b] = v;
    if (k == 0) t[b] = tt[row];
}

// One Adam step (Kingma & Ba) at step number *step of `total`, learning rate
// lr0 (1 + cos(pi step / total)) / 2, followed by the BF16 operand copies of
// the updated weights (row-major and, for W2 / W3, transposed); the step
// counter then advances (`done` counts finished blocks, zero between steps).
struct AdamArgs {
    size_t np;
    float *P, *m, *v;
    const float* g;
    int* step;
    int* done;
    int total;
    float lr0, b1, b2, eps;
    size_t off[8];
    int M, D;
    __nv_bfloat16 *W1b, *W2b, *W3b, *W2T, *W3T, *w4b;
};

// One parameter's Adam update at step s, and its BF16 operand copies.
__device__ __forceinline__ void adam_update(const AdamArgs& a, size_t t, int s) {
    const float k = (float)(s + 1);
    const float lr = a.lr0 * 0.5f * (1.0f + cospif((float)s / (float)a.total));
    const float c1 = 1.0f - powf(a.b1, k), c2 = 1.0f - powf(a.b2, k);
    const float gt = a.g[t];
    const float mt = a.b1 * a.m[t] + (1.0f - a.b1) * gt;
    const float vt = a.b2 * a.v[t] + (1.0f - a.b2) * gt * gt;
    a.m[t] = mt;
    a.v[t] = vt;
    const float p = a.P[t] - lr * (mt / c1) / (sqrtf(vt / c2) + a.eps);
    a.P[t] = p;
    const __nv_bfloat16 h = __float2bfloat16_rn(p);
    if (t < a.off[1]) {
        a.W1b[(t / a.M) * a.D + t % a.M] = h;
    } else if (t >= a.off[2] && t < a.off[3]) {
        const size_t u = t - a.off[2];
        a.W2b[u] = h;
        a.W2T[(u % kH) * kH + u / kH] = h;
    } else if (t >= a.off[4] && t < a.off[5]) {
        const size_t u = t - a.off[4];
        a.W3b[u] = h;
        a.W3T[(u % kH) * kH + u / kH] = h;
    } else if (t >= a.off[6] && t < a.off[7]) {
        a.w4b[t - a.off[6]] = h;
    }
}

__global__ void k_adam_step(AdamArgs a) {
    pdl_wait_then_release();
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = *a.step;
    if (t < a.np) adam_update(a, t, s);
    // the last block to finish advances the step counter (every block has
    // read it by then) and re-arms the block count for the next step
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.done, 1) == (int)gridDim.x - 1) {
            *a.step = s + 1;
            *a.done = 0;
        }
    }
}

// X[b][k] = bf16(Phi^-1(u)) for the MC sample first + b of Philox stream
// `level` (the words of the FP64 points: u from the top 23 bits of word k,
// Phi^-1 in FP32), zero for k >= M.  The surrogate sees its input in BF16,
// so this FP32 map from the same Philox words is its input on both estimator
// levels that use it.
__global__ void k_surrogate_x_mc(uint64_t seed, uint32_t level, uint64_t first, int n, int M, int D,
                                 __nv_bfloat16* __restrict__ X) {
    const int blocks = D / 4;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * blocks) return;
    const int s = (int)(t / blocks), b = (int)(t % blocks);
    __align__(8) __nv_bfloat16 h[4];
    if (4 * b < M) {
        u64x4 c = {{(uint64_t)b, first + s, 0, 0}};
        const u64x4 w = philox4x64(c, seed, (kPurposeMC << 32) | level);
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            // 23 bits keep (k + 1/2) exact in FP32, so 0 < u < 1 strictly
            const float u = ((float)(w.v[lane] >> 41) + 0.5f) * 0x1p-23f;
            h[lane] = __float2bfloat16_rn(4 * b + lane < M ? normcdfinvf(u) : 0.0f);
        }
    } else {
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) h[lane] = __float2bfloat16_rn(0.0f);
    }
    *reinterpret_cast<uint2*>(X + (size_t)s * D + 4 * b) = *reinterpret_cast<const uint2*>(h);
}

// ------------------------------------------------------------------ host state
static unsigned nb(size_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

struct MlpState {
    bool ready = false;
    int M = 0, D = 0;                  // KL modes, padded input width
    size_t np = 0;                     // FP32 parameters
    size_t off[8] = {};                // W1 b1 W2 b2 W3 b3 w4 b4
    float *P = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2T = nullptr, *W3T = nullptr, *w4b = nullptr;
    // training batch (capacity kMaxBatch rows; transposed operands [*][kMaxBatch])
    __nv_bfloat16 *X = nullptr, *XT = nullptr, *H[3] = {}, *HT[3] = {}, *dZ[3] = {}, *dZT[3] = {};
    float *Z[3] = {}, *t = nullptr, *out = nullptr, *dout = nullptr, *sq = nullptr;
    // training maps: A operands (box 128 rows), B operands (box kTrainBN rows)
    CUtensorMap mX, mH1, mH2, mdZ2, mdZ3, mdZ1T, mdZ2T, mdZ3T;
    CUtensorMap tW1, tW2, tW3, tW2T, tW3T, tXT, tH1T, tH2T;
    // inference
    __nv_bfloat16 *eX = nullptr, *eH[3] = {};
    float* eout = nullptr;
    CUtensorMap meX, meH1, meH2, eW1, eW2, eW3;
    CUtensorMap fW1, fW2, fW3;         // the weights in 128-row boxes (fused inference)
    double mu = 0.0, sd = 1.0;
    int* err = nullptr;
    int* step = nullptr;               // device step counter of a training run; step[1]: Adam's block count
    cudaStream_t st = nullptr;         // training stream (graph capture)
    // the weight- and bias-gradient kernels of a step run on `side`, beside
    // the back-propagation chain on the step's stream (fork / join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_dz2 = nullptr, ev_dz1 = nullptr, ev_join = nullptr;
    // A training run whose steps may still be running on `st` (launched with
    // fm_train_opts.async_run): every use of the network waits for `trained`
    // on its stream, host-side uses wait on the host.  The run's buffers and
    // graph live until surrogate_train_finish (or the next run) ends the run;
    // the buffers stay for the next run.
    struct Run {
        bool pending = false;          // steps launched, not yet finished
        cudaEvent_t trained = nullptr; // recorded after the last step
        double* xi = nullptr;          // training inputs [n][M] (the fit report evaluates on them)
        float* tt = nullptr;           // standardised targets
        int32_t* perm = nullptr;       // shuffles of every epoch
        float* sq0 = nullptr;          // squared errors of the first step's batch
        // capacities (elements) of the buffers above and of the training
        // solves' fields and outputs: kept across runs, grown when short
        size_t xi_cap = 0, tt_cap = 0, perm_cap = 0, sq0_cap = 0, K_cap = 0, q_cap = 0;
        double *K = nullptr, *q = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        std::vector<double> hq;        // targets Q_0 on the host
        int n = 0, batch = 0;
        fm_train_report rep{};         // fields known at launch
        std::chrono::steady_clock::time_point t0;
    } run;
};

static MlpState* state(fm_ctx* ctx) { return reinterpret_cast<MlpState*>(ctx->mlp); }

// Device-side ordering after a training run still in flight: work on `st`
// that reads the network waits for its last step (no host wait).
static void wait_trained(MlpState* S, cudaStream_t st) {
    if (S && S->run.pending) cudaStreamWaitEvent(st, S->run.trained, 0);
}

// Host-side: wait until a training run in flight has finished its steps.
static void settle(MlpState* S) {
    if (S && S->run.pending) cudaEventSynchronize(S->run.trained);
}

static fm_status train_finish(fm_ctx* ctx, fm_train_report* rep);

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn_mlp() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// BF16 [rows][K] K-major, box (64 x box_rows), 128-byte swizzle.
static bool map_bf16(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t K, uint32_t box_rows) {
    auto fn = encode_fn_mlp();
    if (!fn) return false;
    cuuint64_t dims[2] = {K, rows};
    cuuint64_t strides[1] = {K * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGk, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch, with programmatic stream serialisation when pdl (the training
// graph: each kernel's launch and prologue overlap the previous kernel).
template <typename... KArgs, typename... Args>
static void launch(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   Args... args) {
    if (!pdl) {
        k<<<grid, block, smem, st>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

template <int BN, int EPI>
static bool gemm_attr() {
    return cudaFuncSetAttribute(k_gemm_bf16_tc<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gemm_smem<BN>()) == cudaSuccess;
}

// D = A B^T over K (a multiple of 64): M x N outputs in 128 x BN tiles.
template <int BN, int EPI>
static void gemm(fm_ctx* ctx, const CUtensorMap& A, const CUtensorMap& B, int M, int N, int K, const EpiArgs& e,
                 cudaStream_t st, bool pdl = false) {
    dim3 grid((M + kGm - 1) / kGm, (N + BN - 1) / BN);
    FM_TIMED(ctx, kFamMlp, st, 2.0 * ((double)M * K + (double)N * K) + 4.0 * (double)M * N,
             2.0 * (double)M * N * K,
             launch(pdl, k_gemm_bf16_tc<BN, EPI>, grid, dim3(128), gemm_smem<BN>(), st, A, B, K / kGk, e,
                    state(ctx)->err));
}

static fm_status mlp_alloc(fm_ctx* ctx) {
    if (ctx->mlp) return FM_OK;
    MlpState* S = new MlpState();
    ctx->mlp = S;
    // inputs padded to a multiple of 128 (whole K blocks and N tiles)
    const int M = ctx->cfg.M, D = (M + 127) / 128 * 128, L = kMaxBatch;
    S->M = M;
    S->D = D;
    size_t o = 0;
    const size_t sizes[8] = {(size_t)kH * M, kH, (size_t)kH * kH, kH, (size_t)kH * kH, kH, kH, 1};
    for (int i = 0; i < 8; ++i) {
        S->off[i] = o;
        o += sizes[i];
    }
    S->np = o;
    bool ok = true;
    auto al = [&](void** p, size_t bytes) {
        if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
        if (ok) cudaMemset(*p, 0, bytes);
    };
    al((void**)&S->P, o * 4);
    al((void**)&S->G, o * 4);
    al((void**)&S->Am, o * 4);
    al((void**)&S->Av, o * 4);
    al((void**)&S->W1b, (size_t)kH * D * 2);
    al((void**)&S->W2b, (size_t)kH * kH * 2);
    al((void**)&S->W3b, (size_t)kH * kH * 2);
    al((void**)&S->W2T, (size_t)kH * kH * 2);
    al((void**)&S->W3T, (size_t)kH * kH * 2);
    al((void**)&S->w4b, (size_t)kH * 2);
    al((void**)&S->X, (size_t)L * D * 2);
    al((void**)&S->XT, (size_t)D * L * 2);
    for (int l = 0; l < 3; ++l) {
        al((void**)&S->H[l], (size_t)L * kH * 2);
        al((void**)&S->HT[l], (size_t)kH * L * 2);
        al((void**)&S->dZ[l], (size_t)L * kH * 2);
        al((void**)&S->dZT[l], (size_t)kH * L * 2);
        al((void**)&S->Z[l], (size_t)L * kH * 4);
        al((void**)&S->eH[l], (size_t)kEvalChunk * kH * 2);
    }
    al((void**)&S->t, L * 4);
    al((void**)&S->out, L * 4);
    al((void**)&S->dout, L * 4);
    al((void**)&S->sq, L * 4);
    al((void**)&S->eX, (size_t)kEvalChunk * D * 2);
    al((void**)&S->eout, (size_t)kEvalChunk * 4);
    al((void**)&S->err, 4);
    al((void**)&S->step, 8);
    // the training stream at the highest priority: a run beside an estimator
    // round gets its small, latency-bound steps scheduled ahead of the
    // round's wide launches instead of queueing behind them
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (ok && cudaStreamCreateWithPriority(&S->st, cudaStreamNonBlocking, hi) != cudaSuccess) ok = false;
    if (ok && cudaStreamCreateWithPriority(&S->side, cudaStreamNonBlocking, hi) != cudaSuccess) ok = false;
    for (cudaEvent_t* e : {&S->ev_fork, &S->ev_dz2, &S->ev_dz1, &S->ev_join})
        if (ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (!ok) {
        set_error(ctx, "surrogate: device allocation failed");
        return FM_ENOMEM;
    }
    if (!(gemm_attr<kTrainBN, kEpiFwdGelu>() && gemm_attr<kTrainBN, kEpiBwdGelu>() &&
          gemm_attr<kTrainBN, kEpiF32>() && gemm_attr<kEvalBN, kEpiFwdGelu>() &&
          cudaFuncSetAttribute(k_mlp_infer_mc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fused_smem_bytes()) == cudaSuccess)) {
        set_error(ctx, "surrogate: cannot raise the GEMM kernels' shared-memory limit");
        return FM_ECUDA;
    }
    const uint32_t bn = kTrainBN;
    ok = map_bf16(&S->mX, S->X, L, D, kGm) && map_bf16(&S->mH1, S->H[0], L, kH, kGm) &&
         map_bf16(&S->mH2, S->H[1], L, kH, kGm) && map_bf16(&S->mdZ2, S->dZ[1], L, kH, kGm) &&
         map_bf16(&S->mdZ3, S->dZ[2], L, kH, kGm) && map_bf16(&S->mdZ1T, S->dZT[0], kH, L, kGm) &&
         map_bf16(&S->mdZ2T, S->dZT[1], kH, L, kGm) && map_bf16(&S->mdZ3T, S->dZT[2], kH, L, kGm) &&
         map_bf16(&S->tW1, S->W1b, kH, D, bn) && map_bf16(&S->tW2, S->W2b, kH, kH, bn) &&
         map_bf16(&S->tW3, S->W3b, kH, kH, bn) && map_bf16(&S->tW2T, S->W2T, kH, kH, bn) &&
         map_bf16(&S->tW3T, S->W3T, kH, kH, bn) && map_bf16(&S->tXT, S->XT, D, L, bn) &&
         map_bf16(&S->tH1T, S->HT[0], kH, L, bn) && map_bf16(&S->tH2T, S->HT[1], kH, L, bn) &&
         map_bf16(&S->meX, S->eX, kEvalChunk, D, kGm) && map_bf16(&S->meH1, S->eH[0], kEvalChunk, kH, kGm) &&
         map_bf16(&S->meH2, S->eH[1], kEvalChunk, kH, kGm) && map_bf16(&S->eW1, S->W1b, kH, D, kEvalBN) &&
         map_bf16(&S->eW2, S->W2b, kH, kH, kEvalBN) && map_bf16(&S->eW3, S->W3b, kH, kH, kEvalBN) &&
         map_bf16(&S->fW1, S->W1b, kH, D, kH / 2) && map_bf16(&S->fW2, S->W2b, kH, kH, kH / 2) &&
         map_bf16(&S->fW3, S->W3b, kH, kH, kH / 2);
    if (!ok) {
        set_error(ctx, "surrogate: cuTensorMapEncodeTiled failed");
        return FM_ECUDA;
    }
    return FM_OK;
}

// BF16 operand copies of the FP32 master parameters.
static void refresh_bf16(fm_ctx* ctx, cudaStream_t st) {
    MlpState* S = state(ctx);
    const int M = S->M, D = S->D;
    k_weight_bf16<<<nb((size_t)kH * D), 256, 0, st>>>(kH, M, D, S->P + S->off[0], S->W1b, nullptr);
    k_weight_bf16<<<nb((size_t)kH * kH), 256, 0, st>>>(kH, kH, kH, S->P + S->off[2], S->W2b, S->W2T);
    k_weight_bf16<<<nb((size_t)kH * kH), 256, 0, st>>>(kH, kH, kH, S->P + S->off[4], S->W3b, S->W3T);
    k_weight_bf16<<<nb(kH), 256, 0, st>>>(1, kH, kH, S->P + S->off[6], S->w4b, nullptr);
}

// Forward + backward of one batch of B rows (a multiple of 128, <= kMaxBatch)
// already in S->X / S->XT / S->t; gradients into S->G.  The chain that
// back-propagates (dZ3 -> dZ2 -> dZ1 -> dW1) runs on st; the other weight
// and bias gradients, which nothing downstream reads but Adam, run beside it
// on S->side (forked after the output layer, joined at the end), so a
// training step's critical path is 9 kernels (batch gather, three forward
// GEMMs, the output layer with its gradient, dZ2, dZ1, dW1, Adam with the
// step counter) instead of 17.
static void train_step_grads(fm_ctx* ctx, int B, cudaStream_t st, bool pdl = false) {
    MlpState* S = state(ctx);
    const int D = S->D, L = kMaxBatch;
    constexpr int BN = kTrainBN;
    cudaStream_t sd = S->side;
    EpiArgs e{};
    // forward: Z_l = H_(l-1) W_l^T + b_l, H_l = bf16(gelu(Z_l))
    e = EpiArgs{B, kH, S->P + S->off[1], S->Z[0], kH, S->H[0], kH, S->HT[0], L, nullptr, 0};
    gemm<BN, kEpiFwdGelu>(ctx, S->mX, S->tW1, B, kH, D, e, st, pdl);
    e = EpiArgs{B, kH, S->P + S->off[3], S->Z[1], kH, S->H[1], kH, S->HT[1], L, nullptr, 0};
    gemm<BN, kEpiFwdGelu>(ctx, S->mH1, S->tW2, B, kH, kH, e, st, pdl);
    e = EpiArgs{B, kH, S->P + S->off[5], S->Z[2], kH, S->H[2], kH, S->HT[2], L, nullptr, 0};
    gemm<BN, kEpiFwdGelu>(ctx, S->mH2, S->tW3, B, kH, kH, e, st, pdl);
    // output layer and dZ3 = bf16(dout w4 gelu'(Z3)) on st; gw4 = dout^T H3, gb4 = sum dout beside it
    launch(pdl, k_mlp_out_train, dim3(nb((size_t)B * 32)), dim3(256), 0, st, B, L, S->H[2], S->w4b,
           S->P + S->off[7], S->t, S->out, S->dout, S->sq, S->Z[2], S->dZ[2], S->dZT[2]);
    cudaEventRecord(S->ev_fork, st);
    cudaStreamWaitEvent(sd, S->ev_fork, 0);
    launch(pdl, k_row_sums, dim3(nb((size_t)(kH + 1) * 32)), dim3(256), 0, sd, kH, B, L, S->HT[2], S->dout,
           S->G + S->off[6], S->G + S->off[7]);
    // layer 3: dW3 = dZ3^T H2, db3 beside; dZ2 = bf16((dZ3 W3) gelu'(Z2)) on st
    e = EpiArgs{kH, kH, nullptr, nullptr, 0, nullptr, 0, nullptr, 0, S->G + S->off[4], kH};
    gemm<BN, kEpiF32>(ctx, S->mdZ3T, S->tH2T, kH, kH, B, e, sd, pdl);
    launch(pdl, k_row_sums, dim3(nb((size_t)kH * 32)), dim3(256), 0, sd, kH, B, L, S->dZT[2], nullptr,
           S->G + S->off[5], nullptr);
    e = EpiArgs{B, kH, nullptr, S->Z[1], kH, S->dZ[1], kH, S->dZT[1], L, nullptr, 0};
    gemm<BN, kEpiBwdGelu>(ctx, S->mdZ3, S->tW3T, B, kH, kH, e, st, pdl);
    // layer 2: dW2, db2 beside; dZ1 on st
    cudaEventRecord(S->ev_dz2, st);
    cudaStreamWaitEvent(sd, S->ev_dz2, 0);
    e = EpiArgs{kH, kH, nullptr, nullptr, 0, nullptr, 0, nullptr, 0, S->G + S->off[2], kH};
    gemm<BN, kEpiF32>(ctx, S->mdZ2T, S->tH1T, kH, kH, B, e, sd, pdl);
    launch(pdl, k_row_sums, dim3(nb((size_t)kH * 32)), dim3(256), 0, sd, kH, B, L, S->dZT[1], nullptr,
           S->G + S->off[3], nullptr);
    e = EpiArgs{B, kH, nullptr, S->Z[0], kH, S->dZ[0], kH, S->dZT[0], L, nullptr, 0};
    gemm<BN, kEpiBwdGelu>(ctx, S->mdZ2, S->tW2T, B, kH, kH, e, st, pdl);
    // layer 1: db1 beside; dW1 = dZ1^T X on st (N = D input columns; the FP32
    // gradient keeps the M real ones)
    cudaEventRecord(S->ev_dz1, st);
    cudaStreamWaitEvent(sd, S->ev_dz1, 0);
    launch(pdl, k_row_sums, dim3(nb((size_t)kH * 32)), dim3(256), 0, sd, kH, B, L, S->dZT[0], nullptr,
           S->G + S->off[1], nullptr);
    e = EpiArgs{kH, S->M, nullptr, nullptr, 0, nullptr, 0, nullptr, 0, S->G + S->off[0], S->M};
    gemm<BN, kEpiF32>(ctx, S->mdZ1T, S->tXT, kH, D, B, e, st, pdl);
    cudaEventRecord(S->ev_join, sd);
    cudaStreamWaitEvent(st, S->ev_join, 0);
}

// Forward of n rows, chunked: fill(o, cnt, st) writes rows o .. o+cnt-1 of
// the input as BF16 into S->eX; S = mu + sd f lands in d_s.
template <class Fill>
static void eval_chunks(fm_ctx* ctx, uint32_t n, Fill fill, double* d_s, cudaStream_t st) {
    MlpState* S = state(ctx);
    wait_trained(S, st);
    for (uint32_t o = 0; o < n; o += kEvalChunk) {
        const int cnt = (int)std::min<uint32_t>(kEvalChunk, n - o);
        fill(o, cnt, st);
        EpiArgs e{cnt, kH, S->P + S->off[1], nullptr, 0, S->eH[0], kH, nullptr, 0, nullptr, 0};
        gemm<kEvalBN, kEpiFwdGelu>(ctx, S->meX, S->eW1, cnt, kH, S->D, e, st);
        e = EpiArgs{cnt, kH, S->P + S->off[3], nullptr, 0, S->eH[1], kH, nullptr, 0, nullptr, 0};
        gemm<kEvalBN, kEpiFwdGelu>(ctx, S->meH1, S->eW2, cnt, kH, kH, e, st);
        e = EpiArgs{cnt, kH, S->P + S->off[5], nullptr, 0, S->eH[2], kH, nullptr, 0, nullptr, 0};
        gemm<kEvalBN, kEpiFwdGelu>(ctx, S->meH2, S->eW3, cnt, kH, kH, e, st);
        k_mlp_out<<<nb((size_t)cnt * 32), 256, 0, st>>>(cnt, S->eH[2], S->w4b, S->P + S->off[7], nullptr, S->eout,
                                                        nullptr, nullptr);
        k_surrogate_value<<<nb(cnt), 256, 0, st>>>(cnt, S->eout, S->mu, S->sd, d_s + o);
    }
}

// S(xi) for n rows of xi (FP64 [n][M]).
static void eval_forward(fm_ctx* ctx, uint32_t n, const double* d_xi, double* d_s, cudaStream_t st) {
    MlpState* S = state(ctx);
    eval_chunks(ctx, n, [&](uint32_t o, int cnt, cudaStream_t s2) {
        k_gather_x<<<nb((size_t)cnt * S->D), 256, 0, s2>>>(cnt, S->M, S->D, d_xi + (size_t)o * S->M, S->eX, nullptr,
                                                           0);
    }, d_s, st);
}

fm_status surrogate_eval_mc_impl(fm_ctx* ctx, uint32_t level, uint64_t first, uint32_t n, double* d_s,
                                 cudaStream_t st) {
    FM_CHECK_ARG(ctx, ctx->mlp && state(ctx)->ready, "surrogate: no trained or installed network");
    if (n == 0) return FM_OK;
    MlpState* S = state(ctx);
    const uint64_t seed = ctx->cfg.seed;
    if (S->D <= kH && ctx->fused_infer) {
        // inputs up to 256 wide: the whole network in one kernel per 128 rows
        wait_trained(S, st);
        FusedArgs fa{seed, first, level, (int)n, S->M, S->D, S->P + S->off[1], S->P + S->off[3], S->P + S->off[5],
                     S->P + S->off[7], S->w4b, S->mu, S->sd, d_s, S->err};
        const double flops = 2.0 * n * ((double)S->D * kH + 2.0 * kH * kH + kH);
        FM_TIMED(ctx, kFamMlp, st, 8.0 * n, flops,
                 k_mlp_infer_mc<<<(unsigned)((n + kFusedRows - 1) / kFusedRows), kFusedThreads, fused_smem_bytes(),
                                  st>>>(S->fW1, S->fW2, S->fW3, fa));
        FM_CUDA_TRY(ctx, cudaGetLastError());
        return FM_OK;
    }
    eval_chunks(ctx, n, [&](uint32_t o, int cnt, cudaStream_t s2) {
        FM_TIMED(ctx, kFamPoints, s2, (double)cnt * S->D * 2, 0.0,
                 k_surrogate_x_mc<<<nb((size_t)cnt * (S->D / 4)), 256, 0, s2>>>(seed, level, first + o, cnt, S->M,
                                                                                 S->D, S->eX));
    }, d_s, st);
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

fm_status surrogate_eval_impl(fm_ctx* ctx, uint32_t n, const double* d_xi, double* d_s, cudaStream_t st) {
    FM_CHECK_ARG(ctx, ctx->mlp && state(ctx)->ready, "surrogate: no trained or installed network");
    if (n == 0) return FM_OK;
    eval_forward(ctx, n, d_xi, d_s, st);
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

bool surrogate_mc_fused(const fm_ctx* ctx) {
    const MlpState* S = reinterpret_cast<const MlpState*>(ctx->mlp);
    return S && S->ready && S->D <= kH && ctx->fused_infer;
}

int surrogate_err_flag(const fm_ctx* ctx) {
    if (!ctx->mlp) return 0;
    int e = 0;
    cudaMemcpy(&e, reinterpret_cast<MlpState*>(ctx->mlp)->err, sizeof(int), cudaMemcpyDeviceToHost);
    return e;
}

void mlp_free(fm_ctx* ctx) {
    MlpState* S = state(ctx);
    if (!S) return;
    train_finish(ctx, nullptr);
    if (S->run.trained) cudaEventDestroy(S->run.trained);
    for (void* p : {(void*)S->run.xi, (void*)S->run.tt, (void*)S->run.perm, (void*)S->run.sq0, (void*)S->run.K,
                    (void*)S->run.q})
        cudaFree(p);
    void* ptrs[] = {S->P, S->G, S->Am, S->Av, S->W1b, S->W2b, S->W3b, S->W2T, S->W3T, S->w4b, S->X, S->XT,
                    S->t, S->out, S->dout, S->sq, S->eX, S->eout, S->err, S->step};
    if (S->st) cudaStreamDestroy(S->st);
    if (S->side) cudaStreamDestroy(S->side);
    for (cudaEvent_t e : {S->ev_fork, S->ev_dz2, S->ev_dz1, S->ev_join})
        if (e) cudaEventDestroy(e);
    for (void* p : ptrs) cudaFree(p);
    for (int l = 0; l < 3; ++l) {
        cudaFree(S->H[l]); cudaFree(S->HT[l]); cudaFree(S->dZ[l]); cudaFree(S->dZT[l]); cudaFree(S->Z[l]);
        cudaFree(S->eH[l]);
    }
    delete S;
    ctx->mlp = nullptr;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status surrogate_params(fm_ctx* ctx, float* host_params, int32_t set) {
    FM_CHECK_ARG(ctx, ctx != nullptr && host_params != nullptr, "surrogate_params: null argument");
    FM_TRY(mlp_alloc(ctx));
    MlpState* S = state(ctx);
    settle(S);
    if (set) {
        FM_CUDA_TRY(ctx, cudaMemcpy(S->P, host_params, S->np * 4, cudaMemcpyHostToDevice));
        refresh_bf16(ctx, nullptr);
        FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
        S->ready = true;
    } else {
        FM_CUDA_TRY(ctx, cudaMemcpy(host_params, S->P, S->np * 4, cudaMemcpyDeviceToHost));
    }
    return FM_OK;
}

extern "C" int64_t surrogate_param_count(const fm_ctx* ctx) {
    if (!ctx) return -1;
    const int64_t M = ctx->cfg.M;
    return kH * M + kH + 2 * ((int64_t)kH * kH + kH) + kH + 1;
}

extern "C" fm_status surrogate_set_scale(fm_ctx* ctx, double mu, double sd) {
    FM_CHECK_ARG(ctx, ctx != nullptr && sd > 0, "surrogate_set_scale: bad argument");
    FM_TRY(mlp_alloc(ctx));
    settle(state(ctx));
    state(ctx)->mu = mu;
    state(ctx)->sd = sd;
    return FM_OK;
}

extern "C" fm_status surrogate_loss_grad(fm_ctx* ctx, const double* d_xi, const float* d_target, float* host_grads,
                                         double* host_loss) {
    FM_CHECK_ARG(ctx, ctx != nullptr && d_xi && d_target, "surrogate_loss_grad: null argument");
    FM_TRY(mlp_alloc(ctx));
    MlpState* S = state(ctx);
    settle(S);
    FM_CUDA_TRY(ctx, cudaMemset(S->err, 0, 4));
    k_gather_x<<<nb((size_t)kLossBatch * S->D), 256>>>(kLossBatch, S->M, S->D, d_xi, S->X, S->XT, kMaxBatch);
    FM_CUDA_TRY(ctx, cudaMemcpy(S->t, d_target, kLossBatch * 4, cudaMemcpyDeviceToDevice));
    train_step_grads(ctx, kLossBatch, nullptr);
    FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (surrogate_err_flag(ctx)) {
        set_error(ctx, "surrogate_loss_grad: a bounded tensor-core wait ran out");
        return FM_ETIMEOUT;
    }
    if (host_grads) FM_CUDA_TRY(ctx, cudaMemcpy(host_grads, S->G, S->np * 4, cudaMemcpyDeviceToHost));
    if (host_loss) {
        std::vector<float> sq(kLossBatch);
        FM_CUDA_TRY(ctx, cudaMemcpy(sq.data(), S->sq, kLossBatch * 4, cudaMemcpyDeviceToHost));
        double l = 0.0;
        for (float v : sq) l += v;
        *host_loss = l / kLossBatch;
    }
    return FM_OK;
}

namespace fm {

// The end of a training run: wait for its steps, read the first and last
// mini-batch losses, evaluate the fit on the training set, destroy the run's
// graph (its buffers stay for the next run).  rep (nullable) receives the
// whole report.
static fm_status train_finish(fm_ctx* ctx, fm_train_report* rep) {
    MlpState* S = state(ctx);
    if (!S || !S->run.pending) return FM_OK;
    MlpState::Run& R = S->run;
    fm_status stt = FM_OK;
    if (cudaEventSynchronize(R.trained) != cudaSuccess) stt = FM_ECUDA;
    const int n = R.n, batch = R.batch;
    auto mean_sq = [&](const float* d) {
        std::vector<float> sq(batch);
        cudaMemcpy(sq.data(), d, batch * 4, cudaMemcpyDeviceToHost);
        double l = 0.0;
        for (float v : sq) l += v;
        return l / batch;
    };
    double first_loss = NAN, last_loss = NAN, corr = NAN, var_res = NAN;
    if (stt == FM_OK) {
        first_loss = mean_sq(R.sq0);
        last_loss = mean_sq(S->sq);
    }
    R.pending = false;   // the network is final from here on
    if (stt == FM_OK && surrogate_err_flag(ctx)) {
        set_error(ctx, "surrogate_train: a bounded tensor-core wait ran out");
        stt = FM_ETIMEOUT;
    }
    if (stt == FM_OK) {
        S->ready = true;
        // fit on the training set: correlation of S with Q_0
        double* sv = nullptr;
        if (cudaMalloc((void**)&sv, (size_t)n * 8) != cudaSuccess) {
            stt = FM_ENOMEM;
        } else {
            eval_forward(ctx, n, R.xi, sv, nullptr);
            std::vector<double> hs(n);
            cudaMemcpy(hs.data(), sv, (size_t)n * 8, cudaMemcpyDeviceToHost);
            cudaFree(sv);
            const std::vector<double>& hq = R.hq;
            double ms = 0.0, mu = 0.0, cov = 0.0, vs = 0.0, vq = 0.0, vr = 0.0;
            for (int i = 0; i < n; ++i) {
                ms += hs[i];
                mu += hq[i];
            }
            ms /= n;
            mu /= n;
            for (int i = 0; i < n; ++i) {
                cov += (hs[i] - ms) * (hq[i] - mu);
                vs += (hs[i] - ms) * (hs[i] - ms);
                vq += (hq[i] - mu) * (hq[i] - mu);
                vr += (hq[i] - hs[i]) * (hq[i] - hs[i]);
            }
            corr = cov / std::sqrt(vs * vq + 1e-300);
            var_res = vr / (n - 1);
        }
    }
    if (rep) {
        *rep = R.rep;
        rep->loss_first = first_loss;
        rep->loss_last = last_loss;
        rep->corr = corr;
        rep->var_residual = var_res;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - R.t0).count();
    }
    if (R.exec) cudaGraphExecDestroy(R.exec);
    if (R.graph) cudaGraphDestroy(R.graph);
    R.exec = nullptr;
    R.graph = nullptr;
    R.hq.clear();
    return stt;
}

}  // namespace fm

extern "C" fm_status surrogate_train(fm_ctx* ctx, const fm_train_opts* opts, fm_train_report* rep) {
    FM_CHECK_ARG(ctx, ctx != nullptr && opts != nullptr, "surrogate_train: null argument");
    FM_CHECK_ARG(ctx, ctx->basis_ready, "surrogate_train: no KL basis installed");
    const int batch = opts->batch > 0 ? opts->batch : 256;
    FM_CHECK_ARG(ctx, batch % 128 == 0 && batch <= kMaxBatch,
                 "surrogate_train: batch must be a multiple of 128 and at most 4096");
    FM_CHECK_ARG(ctx, opts->n_train >= batch && opts->epochs >= 1 && opts->lr > 0,
                 "surrogate_train: need n_train >= batch, epochs >= 1, lr > 0");
    const auto t0 = std::chrono::steady_clock::now();
    FM_TRY(mlp_alloc(ctx));
    FM_TRY(train_finish(ctx, nullptr));   // a run still in flight ends first
    MlpState* S = state(ctx);
    MlpState::Run& R = S->run;
    const int n = opts->n_train, M = ctx->cfg.M;
    // training pairs (xi, Q_0) from the method: level-0 FMG solves on a stream of their own
    const int N0 = grid_of_level(ctx, 0);
    const uint32_t chunk = 65536;
    FM_TRY(ensure(ctx, &R.xi, &R.xi_cap, (size_t)n * M));
    FM_TRY(ensure(ctx, &R.q, &R.q_cap, (size_t)n));
    FM_TRY(ensure(ctx, &R.K, &R.K_cap, (size_t)std::min<uint32_t>(chunk, (uint32_t)n) * N0 * N0));
    double *xi = R.xi, *q = R.q, *K = R.K;
    fm_status stt = FM_OK;
    {
        fm_solve_params prm = solve_params(ctx);
        if (opts->target_tol > 0 && prm.converged) {
            prm.tol = opts->target_tol;
            prm.qtol = opts->target_tol;
        }
        for (uint32_t o = 0; stt == FM_OK && o < (uint32_t)n; o += chunk) {
            const uint32_t c = std::min<uint32_t>(chunk, n - o);
            stt = mc_points(ctx, kSurrogateTrainStream, o, c, M, xi + (size_t)o * M, nullptr);
            if (stt == FM_OK) stt = kl_field_batch(ctx, 0, c, xi + (size_t)o * M, K, nullptr);
            if (stt == FM_OK) stt = fmg_solve_impl(ctx, N0, c, K, prm, q + o, nullptr, nullptr, nullptr, nullptr);
        }
    }
    // The host's part while the device forms the pairs: initial parameters
    // U(-1/sqrt(fan_in), 1/sqrt(fan_in)) (Adam state zero) and the shuffles.
    std::mt19937_64 gen(opts->seed);
    std::uniform_real_distribution<double> uni(0.0, 1.0);
    std::vector<float> hp(S->np);
    const int fan[8] = {M, M, kH, kH, kH, kH, kH, kH};
    for (int i = 0; i < 8; ++i) {
        const size_t end = (i == 7) ? S->np : S->off[i + 1];
        const double a = 1.0 / std::sqrt((double)fan[i]);
        for (size_t k = S->off[i]; k < end; ++k) hp[k] = (float)((2.0 * uni(gen) - 1.0) * a);
    }
    // one shuffled permutation per epoch, all uploaded before the run
    const int spe = n / batch;
    const int total = spe * opts->epochs;
    std::vector<int32_t> perm((size_t)n * opts->epochs);
    for (int ep = 0; ep < opts->epochs; ++ep) {
        int32_t* pe = perm.data() + (size_t)ep * n;
        std::iota(pe, pe + n, 0);
        std::shuffle(pe, pe + n, gen);
    }
    std::vector<double> hq(n);
    if (stt == FM_OK && cudaMemcpy(hq.data(), q, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) stt = FM_ECUDA;
    if (stt != FM_OK) return stt;
    double mu = 0.0, var = 0.0;
    for (double v : hq) mu += v;
    mu /= n;
    for (double v : hq) var += (v - mu) * (v - mu);
    const double sd = std::sqrt(var / (n - 1));
    S->mu = mu;
    S->sd = sd > 0 ? sd : 1.0;
    std::vector<float> ht(n);
    for (int i = 0; i < n; ++i) ht[i] = (float)((hq[i] - mu) / S->sd);
    // the run's state: from here on train_finish ends it
    R.hq = std::move(hq);
    R.n = n;
    R.batch = batch;
    R.t0 = t0;
    R.rep = fm_train_report{};
    R.rep.mu = mu;
    R.rep.sd = S->sd;
    R.rep.var_q = var / (n - 1);
    R.rep.steps = total;
    if (!R.trained) FM_CUDA_TRY(ctx, cudaEventCreateWithFlags(&R.trained, cudaEventDisableTiming));
    cudaStream_t ts = S->st;
    auto launch_run = [&]() -> fm_status {
        FM_TRY(ensure(ctx, &R.tt, &R.tt_cap, (size_t)n));
        FM_TRY(ensure(ctx, &R.perm, &R.perm_cap, perm.size()));
        FM_TRY(ensure(ctx, &R.sq0, &R.sq0_cap, (size_t)batch));
        FM_CUDA_TRY(ctx, cudaMemcpy(R.tt, ht.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
        FM_CUDA_TRY(ctx, cudaMemcpy(R.perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice));
        FM_CUDA_TRY(ctx, cudaMemcpy(S->P, hp.data(), S->np * 4, cudaMemcpyHostToDevice));
        FM_CUDA_TRY(ctx, cudaMemset(S->Am, 0, S->np * 4));
        FM_CUDA_TRY(ctx, cudaMemset(S->Av, 0, S->np * 4));
        FM_CUDA_TRY(ctx, cudaMemset(S->err, 0, 4));
        FM_CUDA_TRY(ctx, cudaMemset(S->step, 0, 8));
        refresh_bf16(ctx, nullptr);
        FM_CUDA_TRY(ctx, cudaDeviceSynchronize());
        // one training step as a CUDA graph: batch gather, forward, backward,
        // Adam + BF16 refresh, step counter; replayed `total` times
        AdamArgs aa{S->np, S->P, S->Am, S->Av, S->G, S->step, S->step + 1, total, (float)opts->lr, 0.9f, 0.999f, 1e-8f,
                    {}, M, S->D, S->W1b, S->W2b, S->W3b, S->W2T, S->W3T, S->w4b};
        for (int i = 0; i < 8; ++i) aa.off[i] = S->off[i];
        const bool prof_on = ctx->prof.active;
        ctx->prof.active = false;    // no event records inside the captured graph
        FM_CUDA_TRY(ctx, cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal));
        // programmatic dependent launches: every kernel's launch and setup
        // overlap its predecessor (kernels wait for it before touching data)
        launch(true, k_train_batch, dim3(nb((size_t)batch * S->D)), dim3(256), 0, ts, batch, M, S->D, kMaxBatch, n,
               spe, (const int*)S->step, (const int32_t*)R.perm, (const double*)R.xi, (const float*)R.tt, S->X,
               S->XT, S->t);
        train_step_grads(ctx, batch, ts, true);
        launch(true, k_adam_step, dim3(nb(S->np)), dim3(256), 0, ts, aa);
        const cudaError_t ce = cudaStreamEndCapture(ts, &R.graph);
        ctx->prof.active = prof_on;
        FM_CUDA_TRY(ctx, ce);
        FM_CUDA_TRY(ctx, cudaGraphInstantiate(&R.exec, R.graph, 0));
        const int pidx = prof_start(ctx, kFamMlpTrain, ts);
        FM_CUDA_TRY(ctx, cudaGraphLaunch(R.exec, ts));
        // the first step's batch errors, for the report
        FM_CUDA_TRY(ctx, cudaMemcpyAsync(R.sq0, S->sq, (size_t)batch * 4, cudaMemcpyDeviceToDevice, ts));
        for (int k = 1; k < total; ++k) FM_CUDA_TRY(ctx, cudaGraphLaunch(R.exec, ts));
        const double D = S->D;
        prof_stop(ctx, pidx, ts, 0.0, (double)total * 2.0 * batch * (2.0 * D * kH + 6.0 * kH * kH));
        FM_CUDA_TRY(ctx, cudaEventRecord(R.trained, ts));
        return FM_OK;
    };
    R.pending = true;   // train_finish ends the run whatever launch_run got to
    S->ready = true;    // users of the network wait for R.trained
    stt = launch_run();
    if (stt != FM_OK) {
        cudaStreamSynchronize(ts);
        train_finish(ctx, nullptr);
        return stt;
    }
    if (opts->async_run) {
        if (rep) {   // the fields known now; surrogate_train_finish gives the rest
            *rep = R.rep;
            rep->loss_first = rep->loss_last = rep->corr = rep->var_residual = NAN;
            rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
        return FM_OK;
    }
    return train_finish(ctx, rep);
}

extern "C" fm_status surrogate_set_fused(fm_ctx* ctx, int32_t on) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "surrogate_set_fused: null context");
    ctx->fused_infer = on ? 1 : 0;
    return FM_OK;
}

extern "C" fm_status surrogate_train_finish(fm_ctx* ctx, fm_train_report* rep) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "surrogate_train_finish: null context");
    FM_CHECK_ARG(ctx, ctx->mlp && state(ctx)->run.pending, "surrogate_train_finish: no training run in flight");
    return train_finish(ctx, rep);
}

extern "C" fm_status surrogate_eval(fm_ctx* ctx, uint32_t n, const double* d_xi, double* d_s, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "surrogate_eval: null context");
    FM_CHECK_ARG(ctx, n == 0 || (d_xi && d_s), "surrogate_eval: null pointer");
    return surrogate_eval_impl(ctx, n, d_xi, d_s, as_stream(stream));
}

extern "C" fm_status surrogate_eval_mc(fm_ctx* ctx, uint32_t stream_level, uint64_t first, uint32_t n, double* d_s,
                                       void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "surrogate_eval_mc: null context");
    FM_CHECK_ARG(ctx, n == 0 || d_s, "surrogate_eval_mc: null pointer");
    return surrogate_eval_mc_impl(ctx, stream_level, first, n, d_s, as_stream(stream));
}
