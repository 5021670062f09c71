// Batched full multigrid for the Case II Darcy problem (Eq. 1, Table 1,
// Sec. 2.5), level-wise schedule: one FMG hierarchy per sample, all samples
// of a batch advanced together, every kernel covering every cell of every
// (active) sample of one grid, x fastest so a warp touches consecutive cells
// of one row.  Used for grids whose hierarchy does not fit in one CTA's
// shared memory (n > 64); smaller grids take the resident schedule.
//
// Per grid k (n_k = n_coarsest << k) and sample the scratch holds
//   K   FP64 coefficients (injected from the finer grid; the finest is the input)
//   Te  east-face transmissibility of each cell (2K on the east edge)
//   Tn  north-face transmissibility (0 on the north edge)
//   D   diagonal: sum of the four face transmissibilities (2K on the west edge)
//   p   iterate, b right-hand side
// in the V-cycle type T (FP64, or FP32 in the mixed form), and for the
// coarsest grid the inverse of its dense operator, so each exact solve is a
// small matrix-vector product.  The mixed form adds FP64 p, Te, Tn, D on the
// two refined grids (n/2 and n, which give Q^c and Q^f).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace fm {

constexpr int kBlock = 256;

inline unsigned blocks_for(size_t threads) { return (unsigned)((threads + kBlock - 1) / kBlock); }

template <typename C>
__device__ __forceinline__ C harmonic(C a, C b) { return C(2) * a * b / (a + b); }

// Sample of a flat thread index and whether it still iterates.
__device__ __forceinline__ bool inactive(const int32_t* active, size_t s) { return active && !active[s]; }

// K_c[J][I] = K_f[2J][2I] (Sec. 2.5, the lower-left child in 0-indexed form).
__global__ void k_inject(int nc, size_t S, const double* __restrict__ Kf, double* __restrict__ Kc) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)nc * nc;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    const int c = (int)(t % cells);
    const int I = c % nc, J = c / nc, nf = 2 * nc;
    Kc[t] = Kf[s * (size_t)nf * nf + (size_t)(2 * J) * nf + 2 * I];
}

// Correction-grid coefficients: K_c[J][I] = geometric mean of the four
// children K_f[2J+dj][2I+di] on the injected grid one level finer, computed
// in C (FP32 for the FP32 correction operators of the mixed form: they steer
// the iteration only, the refined stage operators stay FP64).
template <typename C>
__global__ void k_child_geomean(int nc, size_t S, const double* __restrict__ Kf, double* __restrict__ Kc) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)nc * nc;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    const int c = (int)(t % cells);
    const int I = c % nc, J = c / nc, nf = 2 * nc;
    const double* k = Kf + s * (size_t)nf * nf + (size_t)(2 * J) * nf + 2 * I;
    Kc[t] = (double)exp(C(0.25) * (log((C)k[0]) + log((C)k[1]) + log((C)k[nf]) + log((C)k[nf + 1])));
}

// Face transmissibilities: harmonic mean inside, 2K on the Dirichlet edges
// (west / east; north / south too when ns, Table 1 Case I), none on the
// no-flow edges, in arithmetic C; optional FP64 copies for refined grids
// (which take C = double).  Te of the east column and Tn of the north row
// hold the boundary faces: every kernel couples neighbours only across
// interior faces, so these enter through D alone.  Each face is formed once
// (the east and north faces of its cell); k_diagonal then sums them.
template <typename T, typename C>
__global__ void k_faces(int n, size_t S, int ns, const double* __restrict__ K, T* __restrict__ Te,
                        T* __restrict__ Tn, double* __restrict__ Te64, double* __restrict__ Tn64) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)n * n;
    if (t >= S * cells) return;
    const int c = (int)(t % cells);
    const int i = c % n, j = c / n;
    const C k = (C)K[t];
    const C te = (i < n - 1) ? harmonic<C>(k, (C)K[t + 1]) : C(2) * k;
    const C tn = (j < n - 1) ? harmonic<C>(k, (C)K[t + n]) : (ns ? C(2) * k : C(0));
    Te[t] = (T)te;
    Tn[t] = (T)tn;
    if (Te64) {
        Te64[t] = (double)te;
        Tn64[t] = (double)tn;
    }
}

// D = tw + te + ts + tn from the faces in their arithmetic C (the FP64 copies
// where they exist): the west face of a cell is its west neighbour's east
// face, the same harmonic mean of the same two values, so D equals the sum
// of four freshly formed faces bit for bit.  Boundary faces: 2K west, 2K
// south when ns, else 0.
template <typename T, typename C>
__global__ void k_diagonal(int n, size_t S, int ns, const double* __restrict__ K, const T* __restrict__ Te,
                           const T* __restrict__ Tn, const double* __restrict__ Te64,
                           const double* __restrict__ Tn64, T* __restrict__ D, double* __restrict__ D64) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)n * n;
    if (t >= S * cells) return;
    const int c = (int)(t % cells);
    const int i = c % n, j = c / n;
    auto fe = [&](size_t u) { return Te64 ? (C)Te64[u] : (C)Te[u]; };
    auto fn = [&](size_t u) { return Tn64 ? (C)Tn64[u] : (C)Tn[u]; };
    const C k = (C)K[t];
    const C tw = (i > 0) ? fe(t - 1) : C(2) * k;
    const C ts = (j > 0) ? fn(t - n) : (ns ? C(2) * k : C(0));
    const C d = tw + fe(t) + ts + fn(t);
    D[t] = (T)d;
    if (D64) D64[t] = (double)d;
}

// Right-hand side of a stage problem: the Dirichlet data moved to the rhs.
template <typename T>
__global__ void k_stage_rhs(int n, size_t S, const double* __restrict__ K, Bnd bd, T* __restrict__ b) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)n * n;
    if (t >= S * cells) return;
    const int c = (int)(t % cells);
    const int i = c % n, j = c / n;
    b[t] = (T)dirichlet_rhs(bd, n, i, j, K[t]);
}

// One colour of a red-black Gauss-Seidel sweep: cells with (i + j) % 2 == color.
template <typename T>
__global__ void k_rbgs_color(int n, size_t S, int color, const T* __restrict__ b, const T* __restrict__ Te,
                             const T* __restrict__ Tn, const T* __restrict__ D, T* __restrict__ p,
                             const int32_t* __restrict__ active) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t half = (size_t)n * n / 2;
    if (t >= S * half) return;
    const size_t s = t / half;
    if (inactive(active, s)) return;
    const int h = (int)(t % half);
    const int j = h / (n / 2);
    const int i = 2 * (h % (n / 2)) + ((j + color) & 1);
    const size_t c = s * (size_t)n * n + (size_t)j * n + i;
    T acc = b[c];
    if (i > 0) acc += Te[c - 1] * p[c - 1];
    if (i < n - 1) acc += Te[c] * p[c + 1];
    if (j > 0) acc += Tn[c - n] * p[c - n];
    if (j < n - 1) acc += Tn[c] * p[c + n];
    p[c] = acc * (T(1) / D[c]);
}

// Coarse value with ghosts: 2g - u across the Dirichlet edges (g = 0 for an
// error), the edge value mirrored across the no-flow edges; a corner ghost
// takes the x rule on the y ghost.
template <typename U>
__device__ __forceinline__ U coarse_ghost_x(int nc, const U* uc, int I, int J, const Ghost<U>& g) {
    if (I < 0) return U(2) * g.w - uc[(size_t)J * nc];
    if (I > nc - 1) return U(2) * g.e - uc[(size_t)J * nc + nc - 1];
    return uc[(size_t)J * nc + I];
}
template <typename U>
__device__ __forceinline__ U coarse_ghost(int nc, const U* uc, int I, int J, const Ghost<U>& g) {
    if (J < 0) {
        const U edge = coarse_ghost_x(nc, uc, I, 0, g);
        return g.ns ? U(2) * g.s - edge : edge;
    }
    if (J > nc - 1) {
        const U edge = coarse_ghost_x(nc, uc, I, nc - 1, g);
        return g.ns ? U(2) * g.n - edge : edge;
    }
    return coarse_ghost_x(nc, uc, I, J, g);
}

// (P u_c) at fine cell (i, j): bilinear cell-centred (9, 3, 3, 1) / 16 with
// the ghosts above.  One expression for every kernel that prolongs.
// The weights on the four coarse values: own cell (I, J), its x neighbour
// Ix, its y neighbour Jy, and the diagonal one.
template <typename U>
__device__ __forceinline__ U prolong_vals(U own, U nx, U ny, U nxy) {
    return (U(9) * own + U(3) * nx + U(3) * ny + U(1) * nxy) / U(16);
}
template <typename U>
__device__ __forceinline__ U prolong_at(int nc, const U* u, int i, int j, const Ghost<U>& g) {
    const int I = i >> 1, J = j >> 1;
    const int Ix = (i & 1) ? I + 1 : I - 1;
    const int Jy = (j & 1) ? J + 1 : J - 1;
    return prolong_vals(coarse_ghost(nc, u, I, J, g), coarse_ghost(nc, u, Ix, J, g), coarse_ghost(nc, u, I, Jy, g),
                        coarse_ghost(nc, u, Ix, Jy, g));
}
// an error's ghosts: zero boundary data
template <typename U>
__device__ __forceinline__ U prolong_err(int nc, const U* u, int i, int j, int ns) {
    const Ghost<U> g{U(0), U(0), U(0), U(0), ns};
    return prolong_at(nc, u, i, j, g);
}

// nsweeps red-black sweeps (colour 0 then 1) on tiles of TI x TI cells of
// one sample, staged in shared memory with a halo of hh = 2 nsweeps cells:
// each half-sweep leaves one more ring at the halo's edge stale, so after
// 2 nsweeps half-sweeps exactly the interior is current.  Every cell update
// is the colour kernel's, in the same order, so the result is bit-identical
// to 2 nsweeps k_rbgs_color launches while p, b and the coefficients cross
// HBM once.  The iterate is read from p_in and written to p_out (another
// buffer): a tile's halo is its neighbours' interior, which must still hold
// the values from before the call whatever order the CTAs run in.  Grid:
// S * tiles^2 CTAs, tile index fastest; inactive samples are not written.
template <typename T>
__global__ void __launch_bounds__(256) k_rbgs_tile(int n, size_t S, int TI, int hh, int nsweeps,
                                                   const T* __restrict__ b, const T* __restrict__ Te,
                                                   const T* __restrict__ Tn, const T* __restrict__ D,
                                                   const T* __restrict__ p_in, T* __restrict__ p_out,
                                                   const int32_t* __restrict__ active, const T* __restrict__ ec,
                                                   int ns) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    const int tiles = (n + TI - 1) / TI;
    const size_t s = blockIdx.x / ((unsigned)tiles * tiles);
    if (s >= S || inactive(active, s)) return;
    const int tid = (int)(blockIdx.x % ((unsigned)tiles * tiles));
    const int ti = tid % tiles, tj = tid / tiles;
    const int xa = max(ti * TI - hh, 0), ya = max(tj * TI - hh, 0);
    const int xb = min(ti * TI + TI + hh, n), yb = min(tj * TI + TI + hh, n);
    const int RW = xb - xa, RH = yb - ya, R = RW * RH;
    T* sp = reinterpret_cast<T*>(tile_smem);
    T* sb = sp + R;
    T* se = sb + R;
    T* sn = se + R;
    T* sd = sn + R;
    const size_t base = s * (size_t)n * n;
    for (int e = threadIdx.x; e < R; e += blockDim.x) {
        const int r = e / RW, q = e % RW;
        const size_t g = base + (size_t)(ya + r) * n + xa + q;
        // with ec: the coarse-grid correction p + (P e) as k_prolong forms it
        sp[e] = ec ? p_in[g] + prolong_err(n / 2, ec + s * (size_t)(n / 2) * (n / 2), xa + q, ya + r, ns)
                   : p_in[g];
        sb[e] = b[g];
        se[e] = Te[g];
        sn[e] = Tn[g];
        sd[e] = D[g];
    }
    __syncthreads();
    const int W2 = (RW + 1) / 2;
    for (int hs = 0; hs < 2 * nsweeps; ++hs) {
        const int color = hs & 1;
        for (int h = threadIdx.x; h < RH * W2; h += blockDim.x) {
            const int r = h / W2;
            const int q = 2 * (h % W2) + ((color + xa + ya + r) & 1);
            if (q >= RW) continue;
            const int i = xa + q, j = ya + r;
            // a cell whose in-domain neighbour lies outside the region is not updated
            if ((i > 0 && q == 0) || (i < n - 1 && q == RW - 1) || (j > 0 && r == 0) || (j < n - 1 && r == RH - 1))
                continue;
            const int e = r * RW + q;
            T acc = sb[e];
            if (i > 0) acc += se[e - 1] * sp[e - 1];
            if (i < n - 1) acc += se[e] * sp[e + 1];
            if (j > 0) acc += sn[e - RW] * sp[e - RW];
            if (j < n - 1) acc += sn[e] * sp[e + RW];
            sp[e] = acc * (T(1) / sd[e]);
        }
        __syncthreads();
    }
    const int x0 = ti * TI, y0 = tj * TI;
    const int IW = min(TI, n - x0), IH = min(TI, n - y0);
    for (int e = threadIdx.x; e < IW * IH; e += blockDim.x) {
        const int r = e / IW, q = e % IW;
        p_out[base + (size_t)(y0 + r) * n + x0 + q] = sp[(y0 - ya + r) * RW + (x0 - xa + q)];
    }
}

// The tile smoother with every operand but the iterate in registers.  Thread
// (c, g) owns the column pair 2c, 2c+1 and rows g RPT .. g RPT + RPT - 1 of an
// R x R region (tile interior plus halo, clipped at the domain edge) for all
// sweeps: in every row one of its two cells has the colour being updated, so
// every lane updates RPT cells per half-sweep with no divergence.  b, 1/D and
// the four faces of its cells are loaded once (a face that does not exist is
// zero, and the zero-padded shared array keeps every neighbour read in
// bounds); only p goes through shared memory, and neighbours inside the
// thread's own cells come from registers.  Same halo argument, same update
// order and reciprocal as the colour kernel: bit-identical sweeps (a missing
// face adds an exact zero).
template <typename T, int R, int RPT>
__global__ void __launch_bounds__((R / 2) * (R / RPT)) k_rbgs_tile_reg(int n, size_t S, int TI, int hh, int nsweeps,
                                                                      const T* __restrict__ b,
                                                                      const T* __restrict__ Te,
                                                                      const T* __restrict__ Tn,
                                                                      const T* __restrict__ D,
                                                                      const T* __restrict__ p_in, T* __restrict__ p_out,
                                                                      const int32_t* __restrict__ active,
                                                                      const T* __restrict__ ec, int ns) {
    static_assert(R % 2 == 0 && R % RPT == 0, "region must split into column pairs and row strips");
    constexpr int C = R / 2, P = R + 2;   // column pairs; padded row pitch
    __shared__ T sp[P * P];
    const int tiles = (n + TI - 1) / TI;
    const size_t s = blockIdx.x / ((unsigned)tiles * tiles);
    if (s >= S || inactive(active, s)) return;
    const int tid = (int)(blockIdx.x % ((unsigned)tiles * tiles));
    const int ti = tid % tiles, tj = tid / tiles;
    const int xa = max(ti * TI - hh, 0), ya = max(tj * TI - hh, 0);
    const int RW = min(ti * TI + TI + hh, n) - xa, RH = min(tj * TI + TI + hh, n) - ya;
    const int c = threadIdx.x % C, y0 = (threadIdx.x / C) * RPT;
    const size_t base = s * (size_t)n * n;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) sp[e] = T(0);
    __syncthreads();
    T rb[RPT][2], rr[RPT][2], re[RPT][2], rw[RPT][2], rn[RPT][2], rs[RPT][2], rp[RPT][2];
    bool up[RPT][2];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = 2 * c + j, y = y0 + k, gx = xa + x, gy = ya + y;
            rb[k][j] = rr[k][j] = re[k][j] = rw[k][j] = rn[k][j] = rs[k][j] = rp[k][j] = T(0);
            up[k][j] = false;
            if (x < RW && y < RH) {
                const size_t g = base + (size_t)gy * n + gx;
                // with ec: the coarse-grid correction p + (P e) as k_prolong forms it
                rp[k][j] = ec ? p_in[g] + prolong_err(n / 2, ec + s * (size_t)(n / 2) * (n / 2), gx, gy, ns)
                              : p_in[g];
                rb[k][j] = b[g];
                rr[k][j] = T(1) / D[g];
                if (gx < n - 1) re[k][j] = Te[g];
                if (gy < n - 1) rn[k][j] = Tn[g];
                if (gx > 0) rw[k][j] = Te[g - 1];
                if (gy > 0) rs[k][j] = Tn[g - n];
                // a cell whose in-domain neighbour lies outside the region is not updated
                up[k][j] = !((gx > 0 && x == 0) || (gx < n - 1 && x == RW - 1) || (gy > 0 && y == 0) ||
                             (gy < n - 1 && y == RH - 1));
                sp[(y + 1) * P + x + 1] = rp[k][j];
            }
        }
    }
    __syncthreads();
    for (int hs = 0; hs < 2 * nsweeps; ++hs) {
        const int color = hs & 1;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int y = y0 + k;
            // the cell of this colour in row y: column 2c + j (selects, so the
            // register arrays are never indexed at run time)
            const bool j = ((color + xa + ya + y) & 1) != 0;
            const int x = 2 * c + (j ? 1 : 0);
            const T* row = sp + (y + 1) * P + x + 1;
            const T p0 = rp[k][0], p1 = rp[k][1];
            const T pw = j ? p0 : row[-1];
            const T pe = j ? row[1] : p1;
            const T ps = k > 0 ? (j ? rp[k - 1][1] : rp[k - 1][0]) : row[-P];
            const T pn = k < RPT - 1 ? (j ? rp[k + 1][1] : rp[k + 1][0]) : row[P];
            T acc = j ? rb[k][1] : rb[k][0];
            acc += (j ? rw[k][1] : rw[k][0]) * pw;
            acc += (j ? re[k][1] : re[k][0]) * pe;
            acc += (j ? rs[k][1] : rs[k][0]) * ps;
            acc += (j ? rn[k][1] : rn[k][0]) * pn;
            const bool u = j ? up[k][1] : up[k][0];
            const T v = u ? acc * (j ? rr[k][1] : rr[k][0]) : (j ? p1 : p0);
            if (j) rp[k][1] = v;
            else rp[k][0] = v;
            if (x < RW && y < RH) sp[(y + 1) * P + x + 1] = v;
        }
        __syncthreads();
    }
    const int x0 = ti * TI, y0i = tj * TI;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = 2 * c + j, y = y0 + k, gx = xa + x, gy = ya + y;
            if (x < RW && y < RH && gx >= x0 && gx < min(x0 + TI, n) && gy >= y0i && gy < min(y0i + TI, n))
                p_out[base + (size_t)gy * n + gx] = rp[k][j];
        }
    }
}

// Asynchronous global -> shared copies of B = 4, 8 or 16 bytes (cp.async, both
// addresses B-aligned), commit groups, and the wait until at most N groups
// of this thread are still in flight.
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    static_assert(B == 4 || B == 8 || B == 16, "cp.async of 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "n"(B)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A product the compiler may not fuse into a neighbouring add.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Column-strip wavefront smoother: nsweeps red-black sweeps (HS = 2 nsweeps
// half-sweeps) by one warp over a window of 64 columns of one sample,
// marching up the rows.  Lane l owns columns 2l, 2l+1 of the window, so in
// every row it holds one cell of each colour; W / E neighbours in other
// lanes come by warp shuffles, N / S neighbours from the rows the lane keeps
// in registers.  At step y the warp takes in row y and runs half-sweep k on
// row y - k for k = 1 .. HS: row y - k + 1 has just had half-sweep k - 1 and
// row y - k - 1 had it one step earlier, so every update sees the values the
// sweep order prescribes, and row y - HS is final and is written out.  The
// HS + 2 rows being swept stay in registers (a ring whose slots are fixed by
// the unrolled step index); the rows ahead of them arrive through a
// per-warp shared-memory ring filled by cp.async (strip_depth rows deep:
// each lane copies and later reads back only its own pairs).  A cell with an
// in-domain neighbour outside the window (first or last column, first or
// last row of a segment) is not updated, so after HS half-sweeps the window
// minus HS columns and rows on each side is exact.  Every update is the
// colour kernel's in the same order with the reciprocal of D, so the sweeps
// are bit-identical to the other shapes (a missing face adds an exact zero).
// Operands cross HBM once per call, as float2 / double2 pairs per lane.
// p_in -> p_out as for the tiles; with ec the iterate is p_in + P ec: the
// coarse row a fine row needs comes through the same ring (each lane's
// coarse column, plus the columns left and right of the window), and the
// three coarse rows in use stay in registers, so the correction adds no
// dependent loads.
//
// With FUSE (pre-smoothing of a V-cycle) the warp also forms the residual
// b - A p of each final row once the row above it is final, and the
// restriction to the coarse grid: the lane's column pair is one coarse
// column, so it sums its four fine residuals over two rows in
// k_residual_restrict's order and writes b_c (and p_c = 0).  The residual
// needs exact neighbours, so the strip and segment halos grow by two.
// Strips overlap by 2 XH columns and row segments by 2 VH rows; one unit
// (sample, row segment, strip) per warp, strip index fastest.
constexpr int kStripWarps = 4;

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

// Rows in flight per warp of the strip shapes (shared-memory ring of 40 KB per CTA).
template <typename T>
__host__ __device__ constexpr int strip_depth() { return sizeof(T) == 4 ? 8 : 4; }

// Window offset (columns left of the output columns) and halo rows of the strip shapes.
__host__ __device__ constexpr int strip_xh(int HS, bool fuse) { return fuse ? HS + 2 : HS; }
__host__ __device__ constexpr int strip_ow(int HS, bool fuse) { return 64 - 2 * strip_xh(HS, fuse); }

template <typename T, int HS, bool FUSE>
__global__ void __launch_bounds__(32 * kStripWarps, sizeof(T) == 4 ? 4 : 1) k_rbgs_strip(int n, size_t S_all, int strips, int seg_all, int segs_all,
                                                                 const T* __restrict__ b, const T* __restrict__ Te,
                                                                 const T* __restrict__ Tn, const T* __restrict__ D,
                                                                 const T* __restrict__ p_in, T* __restrict__ p_out,
                                                                 const int32_t* __restrict__ active,
                                                                 const T* __restrict__ ec, T* __restrict__ bc,
                                                                 T* __restrict__ pc, const int32_t* __restrict__ order,
                                                                 int ns, const int32_t* __restrict__ dcount,
                                                                 int resident) {
    using V2 = typename Pair<T>::type;
    constexpr int R = HS + 2;                       // rows in registers: y - HS - 1 .. y
    constexpr int XH = strip_xh(HS, FUSE), VH = XH;  // halo columns and rows (even)
    constexpr int OW = strip_ow(HS, FUSE);          // output columns of a strip
    constexpr int DEPTH = strip_depth<T>();         // rows in flight in the shared-memory ring
    static_assert(HS % 2 == 0 && XH % 2 == 0, "even half-sweep count and halos");
    // Each lane copies its own float2 / double2 of the five operands of a row
    // into its own slot of the warp's ring (cp.async, one commit group per
    // row) and reads back only what it copied, so no lane waits for another.
    __shared__ V2 ring[kStripWarps][DEPTH][5][32];
    __shared__ T cring[kStripWarps][DEPTH][34];   // with ec: [0] left of lane 0, [1 + l] lane l, [33] right of lane 31
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // the samples enumerated and their row segments: as launched, or (dcount:
    // inside a device-side refinement loop) the count of listed samples the
    // last residual test left, with segments short enough to fill one wave
    // of warps when those samples are few
    size_t S = S_all;
    int seg = seg_all, segs = segs_all;
    if (dcount) {
        S = (size_t)*dcount;
        if (S * strips < (size_t)resident) {
            int sg = n;
            while (sg / 2 >= 16 && S * strips * (size_t)((n + sg / 2 - 1) / (sg / 2)) <= (size_t)resident) sg /= 2;
            seg = sg;
            segs = (n + sg - 1) / sg;
        }
    }
    const size_t unit = (size_t)blockIdx.x * kStripWarps + (threadIdx.x >> 5);
    if (unit >= S * (size_t)segs * strips) return;   // S: the samples enumerated (listed by order, if given)
    const int sx = (int)(unit % strips);
    const size_t rest = unit / strips;
    const int sy = (int)(rest % segs);
    const size_t s = order ? (size_t)order[rest / segs] : rest / segs;
    if (inactive(active, s)) return;
    const int ox = sx * OW, oy = sy * seg, oye = min(oy + seg, n);
    const int gx = ox - XH + 2 * lane;   // even, so (n even) both cells are in the domain or neither
    const bool in_x = gx >= 0 && gx < n;
    const int ys = max(oy - VH, 0), ye = min(oye + VH, n);   // rows taken in; ys even
    const bool updL = in_x && !(gx > 0 && lane == 0);
    const bool updR = in_x && !(gx + 1 < n - 1 && lane == 31);
    const bool out_x = in_x && gx >= ox && gx < ox + OW;
    const size_t base = s * (size_t)n * n;
    const T* ecs = ec ? ec + s * (size_t)(n / 2) * (n / 2) : nullptr;
    const V2 zero2{T(0), T(0)}, one2{T(1), T(1)};

    V2(*my)[5][32] = ring[threadIdx.x >> 5];
    T(*myc)[34] = cring[threadIdx.x >> 5];
    const int nc = n / 2, I = gx >> 1;   // the lane's coarse column
    // row y into ring slot (y - ys) % DEPTH, with ec also coarse row
    // min((y + 1) / 2, nc - 1), the highest one fine row y needs; every step
    // commits one group
    auto fetch = [&](int y) {
        if (y < ye) {
            const int slot = (y - ys) % DEPTH;
            if (in_x) {
                const size_t g = base + (size_t)y * n + gx;
                V2* v = &my[slot][0][lane];
                constexpr int B = (int)sizeof(V2);
                cp_async<B>(v + 0 * 32, p_in + g);
                cp_async<B>(v + 1 * 32, b + g);
                cp_async<B>(v + 2 * 32, D + g);
                cp_async<B>(v + 3 * 32, Te + g);
                cp_async<B>(v + 4 * 32, Tn + g);
            }
            if (ecs) {
                const T* crow = ecs + (size_t)min((y + 1) >> 1, nc - 1) * nc;
                if (in_x) cp_async<(int)sizeof(T)>(&myc[slot][1 + lane], crow + I);
                if (lane == 0 && I - 1 >= 0 && I - 1 < nc) cp_async<(int)sizeof(T)>(&myc[slot][0], crow + I - 1);
                if (lane == 31 && I + 1 >= 0 && I + 1 < nc) cp_async<(int)sizeof(T)>(&myc[slot][33], crow + I + 1);
            }
        }
        cp_async_commit();
    };
    // with ec: coarse values (own column, left and right neighbours with the
    // Dirichlet ghosts of coarse_ghost) of the coarse rows taken in at the
    // last three steps
    T cs0[3] = {T(0), T(0), T(0)}, cs1[3] = {T(0), T(0), T(0)}, cs2[3] = {T(0), T(0), T(0)};
    auto coarse3 = [&](T own, T left, T right, T (&dst)[3]) {
        dst[0] = own;
        dst[1] = I == 0 ? T(2) * T(0) - own : left;
        dst[2] = I == nc - 1 ? T(2) * T(0) - own : right;
    };
    if (ecs && in_x && ys > 0) {   // coarse row ys / 2 - 1, the lower y neighbour of fine row ys
        const T* crow = ecs + (size_t)(ys / 2 - 1) * nc;
        coarse3(crow[I], I > 0 ? crow[I - 1] : T(0), I + 1 < nc ? crow[I + 1] : T(0), cs1);
    }
    T p[R][2], bb[R][2], rr[R][2], ee[R][2], nf[R][2], wl[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
        p[c][0] = p[c][1] = bb[c][0] = bb[c][1] = ee[c][0] = ee[c][1] = nf[c][0] = nf[c][1] = wl[c] = T(0);
        rr[c][0] = rr[c][1] = T(0);
    }
    // FUSE: the row leaving the ring (p and north faces) and the partial coarse sum
    T pq[2] = {T(0), T(0)}, nq[2] = {T(0), T(0)}, rsum = T(0);
    for (int q = 0; q < DEPTH; ++q) fetch(ys + q);
    const int steps = ye - ys + HS + (FUSE ? 1 : 0);
    for (int y0 = ys; y0 < ys + steps; y0 += R) {
#pragma unroll
        for (int J = 0; J < R; ++J) {
            const int y = y0 + J;
            if (FUSE) {   // keep row y - R (the S neighbour of the residual row y - HS - 1)
                pq[0] = p[J][0];
                pq[1] = p[J][1];
                nq[0] = nf[J][0];
                nq[1] = nf[J][1];
            }
            {   // take in row y (register slot J), then start the copy of row y + DEPTH
                cp_async_wait<DEPTH - 1>();   // this lane's copies of row y have landed
                V2 fp = zero2, fb = zero2, fd = one2, fe = zero2, fn = zero2;
                if (in_x && y < ye) {
                    const V2* slot = &my[(y - ys) % DEPTH][0][lane];
                    fp = slot[0 * 32];
                    fb = slot[1 * 32];
                    fd = slot[2 * 32];
                    fe = slot[3 * 32];
                    fn = slot[4 * 32];
                }
                T a0 = fp.x, a1 = fp.y;
                if (ecs) {   // the coarse-grid correction p + (P e) as k_prolong forms it
                    __syncwarp();   // the neighbouring lanes' coarse copies have landed too
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        cs2[q] = cs1[q];
                        cs1[q] = cs0[q];
                    }
                    if (in_x && y < ye) {
                        const T* cv = myc[(y - ys) % DEPTH];
                        coarse3(cv[1 + lane], cv[lane], cv[2 + lane], cs0);
                        // fine row y: coarse row y / 2 and its y neighbour (one row down for
                        // even y, one up for odd y); the step index J has the parity of y.
                        // Past the south / north edge the neighbour is the ghost row: the
                        // edge row itself across a no-flow edge, its negative across a
                        // Dirichlet one (ns: -own, and -(the x ghosts) in the corners)
                        const T* uJ = (J & 1) ? cs1 : cs0;
                        const bool edge = (J & 1) ? y == n - 1 : y == 0;
                        const T* uJy = (J & 1) ? (edge ? cs1 : cs0) : (edge ? cs0 : cs2);
                        const T sg = (edge && ns) ? T(-1) : T(1);
                        a0 = a0 + prolong_vals(uJ[0], uJ[1], sg * uJy[0], sg * uJy[1]);
                        a1 = a1 + prolong_vals(uJ[0], uJ[2], sg * uJy[0], sg * uJy[2]);
                    }
                }
                p[J][0] = a0;
                p[J][1] = a1;
                bb[J][0] = fb.x;
                bb[J][1] = fb.y;
                rr[J][0] = T(1) / fd.x;
                rr[J][1] = T(1) / fd.y;
                ee[J][0] = fe.x;
                ee[J][1] = gx + 1 < n - 1 ? fe.y : T(0);
                nf[J][0] = y < n - 1 ? fn.x : T(0);
                nf[J][1] = y < n - 1 ? fn.y : T(0);
                wl[J] = __shfl_up_sync(kAll, ee[J][1], 1);   // W face of the left cell
                if (ecs) __syncwarp();   // every lane has read the coarse slot before it is refilled
                fetch(y + DEPTH);
            }
#pragma unroll
            for (int k = 1; k <= HS; ++k) {
                // half-sweep k (colour (k - 1) & 1) on row r: the left cell
                // (even column) has that colour iff y is odd
                const int r = y - k;
                const int c = (J - k + 4 * R) % R, lo = (J - k - 1 + 4 * R) % R, hi = (J - k + 1 + 4 * R) % R;
                const bool row_ok = r >= ys && r < ye && (r > ys || ys == 0) && (r < ye - 1 || ye == n);
                if (J & 1) {
                    const T pw = __shfl_up_sync(kAll, p[c][1], 1);
                    T acc = bb[c][0];
                    acc += wl[c] * pw;
                    acc += ee[c][0] * p[c][1];
                    acc += nf[lo][0] * p[lo][0];
                    acc += nf[c][0] * p[hi][0];
                    const T v = acc * rr[c][0];
                    p[c][0] = (row_ok && updL) ? v : p[c][0];
                } else {
                    const T pe = __shfl_down_sync(kAll, p[c][0], 1);
                    T acc = bb[c][1];
                    acc += ee[c][0] * p[c][0];
                    acc += ee[c][1] * pe;
                    acc += nf[lo][1] * p[lo][1];
                    acc += nf[c][1] * p[hi][1];
                    const T v = acc * rr[c][1];
                    p[c][1] = (row_ok && updR) ? v : p[c][1];
                }
            }
            {
                const int r = y - HS;
                if (out_x && r >= oy && r < oye) {
                    const int c = (J - HS + 4 * R) % R;
                    *reinterpret_cast<V2*>(p_out + base + (size_t)r * n + gx) = V2{p[c][0], p[c][1]};
                }
            }
            if (FUSE) {
                // residual of row q = y - HS - 1 (rows q - 1, q + 1 final), as residual_at forms it
                const int q = y - HS - 1;
                const int c = (J - HS - 1 + 4 * R) % R, hi = (J - HS + 4 * R) % R;
                const T pw = __shfl_up_sync(kAll, p[c][1], 1);
                const T pe = __shfl_down_sync(kAll, p[c][0], 1);
                if (out_x && q >= oy && q < oye) {
                    const V2 dq = *reinterpret_cast<const V2*>(D + base + (size_t)q * n + gx);
                    T v0 = mul_rn(dq.x, p[c][0]);
                    v0 = fma(-wl[c], pw, v0);
                    v0 = fma(-ee[c][0], p[c][1], v0);
                    v0 = fma(-nq[0], pq[0], v0);
                    v0 = fma(-nf[c][0], p[hi][0], v0);
                    const T r0 = bb[c][0] - v0;
                    T v1 = mul_rn(dq.y, p[c][1]);
                    v1 = fma(-ee[c][0], p[c][0], v1);
                    v1 = fma(-ee[c][1], pe, v1);
                    v1 = fma(-nq[1], pq[1], v1);
                    v1 = fma(-nf[c][1], p[hi][1], v1);
                    const T r1 = bb[c][1] - v1;
                    if ((J & 1) == 0) {   // q odd: the coarse cell's upper row
                        const size_t cc = s * (size_t)(n / 2) * (n / 2) + (size_t)(q / 2) * (n / 2) + gx / 2;
                        bc[cc] = rsum + r0 + r1;
                        pc[cc] = T(0);
                    } else {
                        rsum = r0 + r1;
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
}

// r = b - A p at cell c: D p rounded, then one fused multiply-add per face
// (W, E, S, N), spelled out so that every kernel forming a residual rounds
// the same way whatever the compiler would contract.
template <typename T>
__device__ __forceinline__ T residual_at(int n, size_t c, int i, int j, const T* b, const T* Te, const T* Tn,
                                         const T* D, const T* p) {
    T v = mul_rn(D[c], p[c]);
    if (i > 0) v = fma(-Te[c - 1], p[c - 1], v);
    if (i < n - 1) v = fma(-Te[c], p[c + 1], v);
    if (j > 0) v = fma(-Tn[c - n], p[c - n], v);
    if (j < n - 1) v = fma(-Tn[c], p[c + n], v);
    return b[c] - v;
}

// Fused residual + restriction: b_c = sum of the four fine residuals; p_c = 0.
template <typename T>
__global__ void k_residual_restrict(int nc, size_t S, const T* __restrict__ bf, const T* __restrict__ Te,
                                    const T* __restrict__ Tn, const T* __restrict__ D, const T* __restrict__ pf,
                                    T* __restrict__ bc, T* __restrict__ pc, const int32_t* __restrict__ active) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cells = (size_t)nc * nc;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    if (inactive(active, s)) return;
    const int C = (int)(t % cells);
    const int I = C % nc, J = C / nc, nf = 2 * nc;
    const size_t base = s * (size_t)nf * nf;
    const int i0 = 2 * I, j0 = 2 * J;
    const size_t c00 = base + (size_t)j0 * nf + i0;
    const T r00 = residual_at(nf, c00, i0, j0, bf, Te, Tn, D, pf);
    const T r10 = residual_at(nf, c00 + 1, i0 + 1, j0, bf, Te, Tn, D, pf);
    const T r01 = residual_at(nf, c00 + nf, i0, j0 + 1, bf, Te, Tn, D, pf);
    const T r11 = residual_at(nf, c00 + nf + 1, i0 + 1, j0 + 1, bf, Te, Tn, D, pf);
    bc[t] = r00 + r10 + r01 + r11;
    pc[t] = T(0);
}

// p_f += P e_c (add = 1, boundary values 0) or p_f = P u_c (add = 0, FMG start,
// the Dirichlet data as ghost values).
template <typename U>
__global__ void k_prolong(int nc, size_t S, const U* __restrict__ uc, Ghost<U> gh, int add, U* __restrict__ pf,
                          const int32_t* __restrict__ active) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = 2 * nc;
    const size_t cells = (size_t)nf * nf;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    if (inactive(active, s)) return;
    const int c = (int)(t % cells);
    const int i = c % nf, j = c / nf;
    const U v = prolong_at(nc, uc + s * (size_t)nc * nc, i, j, gh);
    pf[t] = add ? pf[t] + v : v;
}

// Energy-optimal step of a coarse-grid correction: the correction d = P e_c
// is added as alpha d with alpha = (r, d) / (d, A d), r = b - A x the
// residual it answers, the exact line minimum of the energy error for the
// symmetric positive definite A (so a cycle never raises the energy error,
// whatever the correction operators).  Per (sample, chunk) of grid n: the
// partial sums of (r, d) and (d, A d) in FP64, with d formed on the fly by
// the prolongation (A d takes it at the four neighbours too); entries 0 and
// 1 of the sample's 3-double slots in partial.
template <typename T>
__global__ void k_energy_partials(int n, size_t S, int chunks, const T* __restrict__ b, const T* __restrict__ Te,
                                  const T* __restrict__ Tn, const T* __restrict__ D, const T* __restrict__ x,
                                  const T* __restrict__ ec, const int32_t* __restrict__ active,
                                  const int32_t* __restrict__ order, double* __restrict__ partial, int ns) {
    __shared__ double red[2][32];
    if (blockIdx.x / chunks >= S) return;   // S: the samples enumerated (listed by order, if given)
    const size_t s = order ? (size_t)order[blockIdx.x / chunks] : blockIdx.x / chunks;
    const int ch = (int)(blockIdx.x % chunks);
    if (inactive(active, s)) return;
    const int nc = n / 2;
    const size_t base = s * (size_t)n * n;
    const T* e = ec + s * (size_t)nc * nc;
    const int cells = n * n, per = (cells + chunks - 1) / chunks;
    const int c0 = ch * per, c1 = min(cells, c0 + per);
    double rd = 0.0, dad = 0.0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const int i = c % n, j = c / n;
        const size_t g = base + c;
        const T r = residual_at(n, g, i, j, b, Te, Tn, D, x);
        const T d = prolong_err(nc, e, i, j, ns);
        T ad = mul_rn(D[g], d);
        if (i > 0) ad = fma(-Te[g - 1], prolong_err(nc, e, i - 1, j, ns), ad);
        if (i < n - 1) ad = fma(-Te[g], prolong_err(nc, e, i + 1, j, ns), ad);
        if (j > 0) ad = fma(-Tn[g - n], prolong_err(nc, e, i, j - 1, ns), ad);
        if (j < n - 1) ad = fma(-Tn[g], prolong_err(nc, e, i, j + 1, ns), ad);
        rd += (double)r * (double)d;
        dad += (double)d * (double)ad;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rd += __shfl_down_sync(0xffffffffu, rd, off);
        dad += __shfl_down_sync(0xffffffffu, dad, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = rd;
        red[1][threadIdx.x >> 5] = dad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, q = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            q += red[1][w];
        }
        double* out = partial + ((size_t)s * chunks + ch) * 3;
        out[0] = a;
        out[1] = q;
    }
}

// alpha[s] = (r, d) / (d, A d) from the chunks' partial sums (0 when d = 0).
__global__ void k_energy_alpha(size_t S, int chunks, const double* __restrict__ partial, double* __restrict__ alpha,
                               const int32_t* __restrict__ active) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || inactive(active, s)) return;
    double rd = 0.0, dad = 0.0;
    for (int ch = 0; ch < chunks; ++ch) {
        rd += partial[((size_t)s * chunks + ch) * 3];
        dad += partial[((size_t)s * chunks + ch) * 3 + 1];
    }
    alpha[s] = dad > 0.0 ? rd / dad : 0.0;
}

// p_f += alpha[s] P e_c, the stepped correction (in FP64, rounded once to T).
template <typename T>
__global__ void k_prolong_step(int nc, size_t S, const T* __restrict__ uc, const double* __restrict__ alpha,
                               T* __restrict__ pf, const int32_t* __restrict__ active, int ns) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = 2 * nc;
    const size_t cells = (size_t)nf * nf;
    if (t >= S * cells) return;
    const size_t s = t / cells;
    if (inactive(active, s)) return;
    const int c = (int)(t % cells);
    const T v = prolong_err(nc, uc + s * (size_t)nc * nc, c % nf, c / nf, ns);
    pf[t] = (T)((double)pf[t] + alpha[s] * (double)v);
}

// The first colour (0) of post-smoothing fused with the coarse-grid
// correction p += P e: a red cell's update reads only its black neighbours,
// so they are read as p + (P e) on the fly and the red cell's own correction
// is never needed (its value is replaced); the next colour launch then
// replaces every black cell from the updated red ones.  Each corrected value
// is k_prolong's and each update k_rbgs_color's, so the sweep is
// bit-identical to a prolongation pass followed by the colour launches.
template <typename T>
__global__ void k_rbgs_color0_prolong(int n, size_t S, const T* __restrict__ b, const T* __restrict__ Te,
                                      const T* __restrict__ Tn, const T* __restrict__ D, T* __restrict__ p,
                                      const T* __restrict__ ec, const int32_t* __restrict__ active, int ns) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t half = (size_t)n * n / 2;
    if (t >= S * half) return;
    const size_t s = t / half;
    if (inactive(active, s)) return;
    const int h = (int)(t % half);
    const int j = h / (n / 2);
    const int i = 2 * (h % (n / 2)) + (j & 1);
    const size_t base = s * (size_t)n * n;
    const size_t c = base + (size_t)j * n + i;
    const int nc = n / 2;
    const T* e = ec + s * (size_t)nc * nc;
    T acc = b[c];
    if (i > 0) acc += Te[c - 1] * (p[c - 1] + prolong_err(nc, e, i - 1, j, ns));
    if (i < n - 1) acc += Te[c] * (p[c + 1] + prolong_err(nc, e, i + 1, j, ns));
    if (j > 0) acc += Tn[c - n] * (p[c - n] + prolong_err(nc, e, i, j - 1, ns));
    if (j < n - 1) acc += Tn[c] * (p[c + n] + prolong_err(nc, e, i, j + 1, ns));
    p[c] = acc * (T(1) / D[c]);
}

// Inverse of the dense operator of the coarsest grid (m = n0^2 <= 16
// unknowns), Gauss-Jordan on [A | I] in FP64 (A is SPD, so no pivoting).
// One warp per sample with [A | X] in shared memory: lane c < 16 owns column
// c of A, lane 16 + c column c of X.
constexpr int kInvWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kInvWarps) k_coarse_inverse(int n0, size_t S, const double* __restrict__ K,
                                                                   T* __restrict__ Ainv, int ns) {
    __shared__ double sh[kInvWarps][2][16][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t s = (size_t)blockIdx.x * kInvWarps + warp;
    if (s >= S) return;   // whole warps leave together
    const int m = n0 * n0;
    double(*A)[16] = sh[warp][0];
    double(*X)[16] = sh[warp][1];
    const double* k = K + s * m;
    for (int r = lane; r < m; r += 32) {   // row r: the equation of cell r
        for (int c = 0; c < m; ++c) {
            A[r][c] = 0.0;
            X[r][c] = (r == c) ? 1.0 : 0.0;
        }
        const int i = r % n0, j = r / n0;
        const double tw = (i > 0) ? harmonic(k[r - 1], k[r]) : 2.0 * k[r];
        const double te = (i < n0 - 1) ? harmonic(k[r], k[r + 1]) : 2.0 * k[r];
        const double tb = ns ? 2.0 * k[r] : 0.0;   // north / south boundary face
        const double ts = (j > 0) ? harmonic(k[r - n0], k[r]) : tb;
        const double tn = (j < n0 - 1) ? harmonic(k[r], k[r + n0]) : tb;
        A[r][r] = tw + te + ts + tn;
        if (i > 0) A[r][r - 1] = -tw;
        if (i < n0 - 1) A[r][r + 1] = -te;
        if (j > 0) A[r][r - n0] = -ts;
        if (j < n0 - 1) A[r][r + n0] = -tn;
    }
    __syncwarp();
    const bool ownA = lane < m, ownX = lane >= 16 && lane - 16 < m;
    const int col = lane & 15;
    for (int p = 0; p < m; ++p) {
        const double piv = A[p][p];
        double f[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) f[r] = (r < m) ? A[r][p] : 0.0;
        __syncwarp();
        // scale row p, then eliminate column p from every other row
        if (ownA) A[p][col] /= piv;
        if (ownX) X[p][col] /= piv;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (r >= m || r == p) continue;
            if (ownA) A[r][col] -= f[r] * A[p][col];
            if (ownX) X[r][col] -= f[r] * X[p][col];
        }
        __syncwarp();
    }
    T* out = Ainv + s * (size_t)m * m;
    for (int e = lane; e < m * m; e += 32) out[e] = (T)X[e / m][e % m];
}

// p = A^{-1} b on the coarsest grid; one thread per (sample, unknown).
template <typename T>
__global__ void k_coarse_solve(int m, size_t S, const T* __restrict__ Ainv, const T* __restrict__ b,
                               T* __restrict__ p, const int32_t* __restrict__ active) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S * m) return;
    const size_t s = t / m;
    if (inactive(active, s)) return;
    const int r = (int)(t % m);
    const T* row = Ainv + s * (size_t)m * m + (size_t)r * m;
    const T* bs = b + s * m;
    T acc = T(0);
    for (int c = 0; c < m; ++c) acc += row[c] * bs[c];
    p[t] = acc;
}

// The QoI of Table 1, one warp per sample.  Case II: the east outflux
// Q = sum_j 2 K_(n-1,j) (p_(n-1,j) - pE), shuffle reduction.  Case I:
// u(0.5, 0.5), the mean of the four cells at the centre.
template <typename P>
__global__ void k_outflux(int n, size_t S, const double* __restrict__ K, const P* __restrict__ p, Bnd bd,
                          double* __restrict__ q) {
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (warp >= S) return;
    if (bd.ns) {
        if (lane == 0) {
            const size_t c = warp * (size_t)n * n + (size_t)(n / 2 - 1) * n + n / 2 - 1;
            q[warp] = 0.25 * (((double)p[c] + (double)p[c + 1]) + ((double)p[c + n] + (double)p[c + n + 1]));
        }
        return;
    }
    const size_t base = warp * (size_t)n * n + (n - 1);
    double acc = 0.0;
    for (int j = lane; j < n; j += 32)
        acc += 2.0 * K[base + (size_t)j * n] * ((double)p[base + (size_t)j * n] - bd.g[1]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) q[warp] = acc;
}

__global__ void k_fill(size_t count, double v, double* __restrict__ x) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) x[t] = v;
}

// ------------------------------------------------------------------ refinement kernels
// Per-sample convergence test of the stage problem, split over `chunks`
// CTAs per sample (grid S * chunks, chunk index fastest): each CTA forms the
// residual of its band of rows and writes its partial sums of ||r||^2,
// ||b||^2 and the outflux to partial[(s * chunks + ch) * 3 + 0..2]; the
// mixed form (p64 != null) forms the residual in FP64 from the FP64 grid and
// writes it, rounded, into the FP32 rhs bT with the FP32 correction pT
// zeroed.  k_stage_decide then folds the partials in chunk order.  b / bT
// and p / pT are the same arrays, hence no __restrict__ on them.
// Threads walk rows (a column each, or several rows per pass on grids
// narrower than the block), so no cell index is divided.  The rhs of a stage
// problem is zero off the Dirichlet edges: interior cells take r = -A p with
// no K load, and only edge cells form the Dirichlet term and add to ||b||^2.
// On GB300 the FP64 pipe (1/58 of the FP32 rate) bounds this kernel, so the
// interior FP64 work is the residual's product and four FMAs, the square
// and one rounding.
template <typename T>
__global__ void k_stage_partials(int n, size_t S, int chunks, const double* __restrict__ K, Bnd bd,
                                 const T* b, const T* __restrict__ Te, const T* __restrict__ Tn,
                                 const T* __restrict__ D, const T* p, const double* __restrict__ p64,
                                 const double* __restrict__ Te64, const double* __restrict__ Tn64,
                                 const double* __restrict__ D64, T* bT, T* pT, const int32_t* __restrict__ active,
                                 double* __restrict__ partial, const int32_t* __restrict__ order) {
    __shared__ double red[3][32];
    // S: the samples enumerated (listed by order, if given)
    if (blockIdx.x / chunks >= S) return;
    const size_t s = order ? (size_t)order[blockIdx.x / chunks] : blockIdx.x / chunks;
    const int ch = (int)(blockIdx.x % chunks);
    if (inactive(active, s)) return;
    const size_t base = s * (size_t)n * n;
    const int rows = (n + chunks - 1) / chunks;
    const int j0 = ch * rows, j1 = min(n, j0 + rows);
    // thread -> first column i0 and row offset jo; a pass covers rpi rows
    const int nt = (int)blockDim.x;
    const bool wide = n >= nt;
    const int rpi = wide ? 1 : nt / n;
    const int i0 = wide ? (int)threadIdx.x : (int)threadIdx.x % n;
    const int jo = wide ? 0 : (int)threadIdx.x / n;
    const int istep = wide ? nt : n;
    const int h0 = n / 2 - 1, h1 = n / 2;   // Case I: the four centre cells
    double rr = 0.0, bb = 0.0, qq = 0.0;
    if (jo < rpi) {
        for (int j = j0 + jo; j < j1; j += rpi) {
            const bool row_edge = bd.ns && (j == 0 || j == n - 1);
            const bool row_centre = bd.ns && (j == h0 || j == h1);
            for (int i = i0; i < n; i += istep) {
                const size_t g = base + (size_t)j * n + i;
                const bool edge = row_edge || i == 0 || i == n - 1;
                double r, pv;
                if (p64) {
                    pv = p64[g];
                    double v = D64[g] * pv;
                    if (i > 0) v -= Te64[g - 1] * p64[g - 1];
                    if (i < n - 1) v -= Te64[g] * p64[g + 1];
                    if (j > 0) v -= Tn64[g - n] * p64[g - n];
                    if (j < n - 1) v -= Tn64[g] * p64[g + n];
                    if (edge) {
                        const double f = dirichlet_rhs(bd, n, i, j, K[g]);
                        r = f - v;
                        bb += f * f;
                    } else {
                        r = -v;
                    }
                    bT[g] = (T)r;
                    pT[g] = T(0);
                } else {
                    pv = (double)p[g];
                    r = (double)residual_at(n, g, i, j, b, Te, Tn, D, p);
                    if (edge) {
                        const double f = dirichlet_rhs(bd, n, i, j, K[g]);
                        bb += f * f;
                    }
                }
                rr += r * r;
                if (bd.ns) {
                    if (row_centre && (i == h0 || i == h1)) qq += 0.25 * pv;
                } else if (i == n - 1) {
                    qq += 2.0 * K[g] * (pv - bd.g[1]);
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, off);
        bb += __shfl_down_sync(0xffffffffu, bb, off);
        qq += __shfl_down_sync(0xffffffffu, qq, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = rr;
        red[1][threadIdx.x >> 5] = bb;
        red[2][threadIdx.x >> 5] = qq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b2 = 0.0, q = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b2 += red[1][w];
            q += red[2][w];
        }
        double* out = partial + ((size_t)s * chunks + ch) * 3;
        out[0] = a;
        out[1] = b2;
        out[2] = q;
    }
}

// The test itself, one thread per sample: active[s] = ||b - A p|| > tol ||b||
// and the last pass moved the outflux by more than qtol |Q|; counted in *left.
__global__ void k_stage_decide(size_t S, int chunks, const double* __restrict__ partial, double tol, double qtol,
                               double* __restrict__ qprev, int32_t* __restrict__ active, int32_t* __restrict__ left,
                               int32_t* __restrict__ order) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || inactive(active, s)) return;
    double a = 0.0, b2 = 0.0, q = 0.0;
    for (int ch = 0; ch < chunks; ++ch) {
        const double* v = partial + ((size_t)s * chunks + ch) * 3;
        a += v[0];
        b2 += v[1];
        q += v[2];
    }
    const bool done = a <= tol * tol * b2 || (qtol > 0 && fabs(q - qprev[s]) <= qtol * fabs(q));
    qprev[s] = q;
    active[s] = done ? 0 : 1;
    if (!done) {   // count it and list it (in no particular order) for launches over the active samples
        const int i = atomicAdd(left, 1);
        if (order) order[i] = (int32_t)s;
    }
}

// Mixed form: the FP64 refinement update p64 += e (the FP32 correction).
template <typename T>
// Grid-stride over the enumerated cells: S samples (listed by order, if
// given), or with dcount (inside a graph's refinement loop) the count the
// last residual test left, so a launch sized for every sample does little
// work once few of them still iterate.
__global__ void k_ir_update(size_t cells, size_t S, const T* __restrict__ e, double* __restrict__ p64,
                            const int32_t* __restrict__ active, const int32_t* __restrict__ order,
                            const int32_t* __restrict__ dcount) {
    const size_t total = (dcount ? (size_t)*dcount : S) * cells;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t s = order ? (size_t)order[t / cells] : t / cells;
        if (inactive(active, s)) continue;
        const size_t g = s * cells + t % cells;
        p64[g] += (double)e[g];
    }
}

template <typename T>
__global__ void k_widen(size_t count, const T* __restrict__ x, double* __restrict__ y) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = (double)x[t];
}

__global__ void k_status(size_t S, const int32_t* __restrict__ active, int32_t* __restrict__ status) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S && active[s]) status[s] = FM_ENOTCONV;
}

// ------------------------------------------------------------------ V-cycle tail
// The part of a level-wise V-cycle below a correction grid of at most 32 x 32
// cells, per sample in shared memory: pre-smoothing, residual and restriction
// down to the coarsest grid, its solve, then prolongation and post-smoothing
// back up.  One CTA per listed sample replaces the per-grid launches of those
// grids (several tiny launches per grid and cycle).  Every operation is the
// level-wise kernels' own, in their order and rounding: sweeps in colour
// order with the faces W, E, S, N fused into the accumulator and the
// reciprocal of D, residuals as residual_at forms them, restriction sums in
// k_residual_restrict's order, the coarse product as k_coarse_solve sums it,
// corrections as prolong_vals forms them; so the result is the per-grid
// schedule's bit for bit (up to the sign of a zero).
constexpr int kTailMaxN = 32;
constexpr int kTailThreads = 128;

template <typename T>
struct TailArgs {
    int kt, n0, nu1, nu2, ns;               // grids 0 .. kt, n_j = n0 << j; ns: Dirichlet north / south
    size_t S;                               // samples enumerated (the listed ones, with order)
    const T* Te[8];                         // correction operators of grids 0 .. kt
    const T* Tn[8];
    const T* D[8];
    const T* b;                             // rhs of grid kt [..][n_kt^2]
    T* p;                                   // out: the correction on grid kt
    const T* Ainv;                          // coarsest correction operator's inverse [..][m][m]
    const int32_t* active;
    const int32_t* order;
};

template <typename T>
__host__ __device__ inline size_t tail_smem_bytes(int kt, int n0) {
    size_t cells = 0;
    for (int j = 0; j <= kt; ++j) cells += (size_t)(n0 << j) * (n0 << j);
    return (6 * cells + (size_t)n0 * n0 * n0 * n0) * sizeof(T);
}

// The largest tail footprint over every coarsest size (2, 3, 4) and the
// deepest correction grid of at most kTailMaxN cells a side above it.
template <typename T>
inline size_t tail_smem_max() {
    size_t m = 0;
    for (int n0 = 2; n0 <= 4; ++n0) {
        int kt = 0;
        while ((n0 << (kt + 1)) <= kTailMaxN) ++kt;
        m = std::max(m, tail_smem_bytes<T>(kt, n0));
    }
    return m;
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(TailArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    const size_t u = blockIdx.x;
    if (u >= a.S) return;
    const size_t s = a.order ? (size_t)a.order[u] : u;
    if (inactive(a.active, s)) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    // Grid j holds six arrays of n_j^2 = m0 4^j values (te, tn, d, 1/d, b, p)
    // from 6 m0 (4^j - 1) / 3 values into shared memory; the coarsest
    // operator's inverse follows the last grid.  Addresses are formed in
    // registers (no per-grid pointer tables in local memory).
    T* const sm = reinterpret_cast<T*>(tail_smem);
    const int m0 = a.n0 * a.n0;
    auto arr = [&](int j, int q) -> T* { return sm + 2 * m0 * ((1 << (2 * j)) - 1) + q * (m0 << (2 * j)); };
    for (int j = 0; j <= a.kt; ++j) {
        const int c = m0 << (2 * j);
        const T* gte = a.Te[j] + s * (size_t)c;
        const T* gtn = a.Tn[j] + s * (size_t)c;
        const T* gd = a.D[j] + s * (size_t)c;
        T* te = arr(j, 0);
        T* tn = arr(j, 1);
        T* dd = arr(j, 2);
        T* rd = arr(j, 3);
#pragma unroll 4
        for (int e = tid; e < c; e += nt) {
            const T d = gd[e];
            te[e] = gte[e];
            tn[e] = gtn[e];
            dd[e] = d;
            rd[e] = T(1) / d;
        }
    }
    T* const ainv = arr(a.kt + 1, 0);
    {
        const int c = m0 << (2 * a.kt);
        const T* gb = a.b + s * (size_t)c;
        T* bt = arr(a.kt, 4);
        T* pt = arr(a.kt, 5);
#pragma unroll 4
        for (int e = tid; e < c; e += nt) {
            bt[e] = gb[e];
            pt[e] = T(0);   // the restriction left a zero correction
        }
        const T* gA = a.Ainv + s * (size_t)m0 * m0;
        for (int e = tid; e < m0 * m0; e += nt) ainv[e] = gA[e];
    }
    __syncthreads();
    // Red-black sweeps on grid j: thread -> column pair xh of rows y0, y0 + ry, ...
    auto sweeps = [&](int j, int nsw) {
        const int n = a.n0 << j, hn = n >> 1, ry = nt / hn;
        const int xh = tid % hn, y0 = tid / hn;
        const T* te = arr(j, 0);
        const T* tn = arr(j, 1);
        const T* rd = arr(j, 3);
        const T* bb = arr(j, 4);
        T* pp = arr(j, 5);
        for (int it = 0; it < nsw; ++it)
            for (int color = 0; color < 2; ++color) {
                for (int y = y0; y < n && y0 < ry; y += ry) {
                    const int x = 2 * xh + ((y + color) & 1), c = y * n + x;
                    T acc = bb[c];
                    if (x > 0) acc = fma(te[c - 1], pp[c - 1], acc);
                    if (x < n - 1) acc = fma(te[c], pp[c + 1], acc);
                    if (y > 0) acc = fma(tn[c - n], pp[c - n], acc);
                    if (y < n - 1) acc = fma(tn[c], pp[c + n], acc);
                    pp[c] = acc * rd[c];
                }
                __syncthreads();
            }
    };
    for (int j = a.kt; j >= 1; --j) {
        sweeps(j, a.nu1);
        const int nf = a.n0 << j, nc = nf / 2, rc = nt / nc;
        const int I = tid % nc, J0 = tid / nc;
        const T* te = arr(j, 0);
        const T* tn = arr(j, 1);
        const T* dd = arr(j, 2);
        const T* bf = arr(j, 4);
        const T* pf = arr(j, 5);
        T* bc = arr(j - 1, 4);
        T* pc = arr(j - 1, 5);
        for (int J = J0; J < nc && J0 < rc; J += rc) {
            const int i0 = 2 * I, j0 = 2 * J;
            const size_t c00 = (size_t)j0 * nf + i0;
            const T r00 = residual_at(nf, c00, i0, j0, bf, te, tn, dd, pf);
            const T r10 = residual_at(nf, c00 + 1, i0 + 1, j0, bf, te, tn, dd, pf);
            const T r01 = residual_at(nf, c00 + nf, i0, j0 + 1, bf, te, tn, dd, pf);
            const T r11 = residual_at(nf, c00 + nf + 1, i0 + 1, j0 + 1, bf, te, tn, dd, pf);
            bc[J * nc + I] = r00 + r10 + r01 + r11;
            pc[J * nc + I] = T(0);
        }
        __syncthreads();
    }
    if (tid < m0) {
        const T* b0 = arr(0, 4);
        T acc = T(0);
        for (int c = 0; c < m0; ++c) acc = fma(ainv[tid * m0 + c], b0[c], acc);
        arr(0, 5)[tid] = acc;
    }
    __syncthreads();
    for (int j = 1; j <= a.kt; ++j) {
        const int nf = a.n0 << j, nc = nf / 2, rf = nt / nf;
        const int i = tid % nf, y0 = tid / nf;
        const T* pc = arr(j - 1, 5);
        T* pf = arr(j, 5);
        for (int y = y0; y < nf && y0 < rf; y += rf) pf[y * nf + i] = pf[y * nf + i] + prolong_err(nc, pc, i, y, a.ns);
        __syncthreads();
        sweeps(j, a.nu2);
    }
    const int c = m0 << (2 * a.kt);
    const T* pt = arr(a.kt, 5);
    T* gp = a.p + s * (size_t)c;
#pragma unroll 4
    for (int e = tid; e < c; e += nt) gp[e] = pt[e];
}

// ------------------------------------------------------------------ driver
template <typename T>
struct GridBufs {
    int n;
    const double* K;
    T *Te, *Tn, *D, *p, *b;
    T* p2;                             // second iterate buffer of the tile smoother
    double* Kc;                        // correction-grid coefficients (k < m)
    T *TeC, *TnC, *DC;                 // their faces and diagonal
    double *p64, *Te64, *Tn64, *D64;   // refined grids of the mixed form only
};

template <typename T>
struct Hierarchy {
    fm_ctx* ctx;
    int m;
    int n0;
    size_t S;
    GridBufs<T> g[FM_MAX_LEVELS + 8];
    T* Ainv;           // coarsest stage operator (injected K)
    T* AinvC;          // coarsest correction operator (child means)
    int32_t* active;   // per-sample iterate flags of converged stages
    int32_t* left;     // count of samples still iterating
    int32_t* iter;     // residual tests done in the current refined stage (graph loops)
    double* qprev;     // outflux of the previous iteration per sample
    double* partial;   // per-(sample, chunk) partial sums of the residual tests
    int32_t* order;    // the samples still iterating, as listed by the last residual test
    double* alpha;     // per-sample step of the energy-optimal coarse-grid correction
    // Host-side count of the samples still iterating in a refined stage (the
    // host loop reads it after every test; S otherwise): the strip smoother
    // sizes its row segments for it, so that a launch with few active samples
    // does not march long columns.
    mutable size_t busy = 0;
    // Device-side count of the samples still iterating (the refinement loop
    // of a graph, where the host cannot read it): the strip smoother then
    // enumerates the listed samples itself.
    mutable const int32_t* dcount = nullptr;
    // launches may enumerate only the listed samples
    bool listed() const { return order && busy > 0 && busy < S; }
};

// CTAs per sample of a residual test on grid n (about 8192 cells each).
inline int check_chunks(int n) { return std::max(1, std::min(128, n * n / 8192)); }

static size_t hierarchy_bytes(int n_fine, int n0, size_t S, size_t tsize, bool mixed, bool converged) {
    size_t total = 0;
    int m = 0;
    while ((n0 << m) < n_fine) ++m;
    for (int k = 0; k <= m; ++k) {
        const size_t c = (size_t)(n0 << k) * (n0 << k);
        total += c * (8 + 6 * tsize) + 6 * 256;
        if (k < m) total += c * (8 + 3 * tsize) + 4 * 256;
        if (mixed && k >= m - 1) total += c * 32 + 4 * 256;
    }
    total += 2 * ((size_t)n0 * n0 * n0 * n0 * tsize + 256);
    if (converged) total += 4 * 4 + 16 + (size_t)check_chunks(n_fine) * 24 + 7 * 256;
    return total * S + 4096;
}

int64_t batch_limit(const fm_ctx* ctx, int n) {
    const bool mixed = ctx->cfg.precision == FM_PREC_MIXED;
    const size_t per = hierarchy_bytes(n, std::max(ctx->cfg.n_coarsest, 4), 1, mixed ? 4 : 8, mixed, true) +
                       (size_t)n * n * sizeof(double) + (size_t)ctx->cfg.M * sizeof(double);
    const size_t budget = (size_t)8 << 30;   // 8 GiB of scratch per batch
    int64_t lim = (int64_t)(budget / per);
    if (ctx->cfg.max_batch > 0) lim = std::min<int64_t>(lim, ctx->cfg.max_batch);
    return std::max<int64_t>(lim, 1);
}

// Scratch of a level-wise batch of S samples: grows `ar` when it is too small
// (never while a stream is being captured: callers size it first).
template <typename T>
static fm_status carve(fm_ctx* ctx, Arena& ar, Hierarchy<T>& H, int n_fine, int n0, size_t S, const double* d_K,
                       bool mixed, bool converged) {
    const size_t need = hierarchy_bytes(n_fine, n0, S, sizeof(T), mixed, converged);
    if (ar.capacity < need) {
        if (ar.base) cudaFree(ar.base);
        ar.base = nullptr;
        ar.capacity = 0;
        if (cudaMalloc((void**)&ar.base, need) != cudaSuccess) {
            set_error(ctx, "fmg scratch allocation of " + std::to_string(need) + " bytes failed");
            return FM_ENOMEM;
        }
        ar.capacity = need;
    }
    char* cur = ar.base;
    auto take = [&](size_t bytes) {
        char* p = cur;
        cur += ((bytes + 255) / 256) * 256;
        return p;
    };
    H.ctx = ctx;
    H.n0 = n0;
    H.S = S;
    H.m = 0;
    while ((n0 << H.m) < n_fine) ++H.m;
    for (int k = 0; k <= H.m; ++k) {
        const int n = n0 << k;
        const size_t cnt = S * (size_t)n * n;
        GridBufs<T>& g = H.g[k];
        g.n = n;
        g.K = (k == H.m) ? d_K : (double*)take(cnt * 8);
        g.Te = (T*)take(cnt * sizeof(T));
        g.Tn = (T*)take(cnt * sizeof(T));
        g.D = (T*)take(cnt * sizeof(T));
        g.p = (T*)take(cnt * sizeof(T));
        g.b = (T*)take(cnt * sizeof(T));
        g.p2 = (T*)take(cnt * sizeof(T));
        g.Kc = nullptr;
        g.TeC = g.TnC = g.DC = nullptr;
        if (k < H.m) {
            g.Kc = (double*)take(cnt * 8);
            g.TeC = (T*)take(cnt * sizeof(T));
            g.TnC = (T*)take(cnt * sizeof(T));
            g.DC = (T*)take(cnt * sizeof(T));
        }
        g.p64 = g.Te64 = g.Tn64 = g.D64 = nullptr;
        if (mixed && k >= H.m - 1) {
            g.p64 = (double*)take(cnt * 8);
            g.Te64 = (double*)take(cnt * 8);
            g.Tn64 = (double*)take(cnt * 8);
            g.D64 = (double*)take(cnt * 8);
        }
    }
    H.Ainv = (T*)take(S * (size_t)n0 * n0 * n0 * n0 * sizeof(T));
    H.AinvC = (T*)take(S * (size_t)n0 * n0 * n0 * n0 * sizeof(T));
    H.active = converged ? (int32_t*)take(S * 4) : nullptr;
    H.left = converged ? (int32_t*)take(4) : nullptr;
    H.iter = converged ? (int32_t*)take(4) : nullptr;
    H.qprev = converged ? (double*)take(S * 8) : nullptr;
    H.partial = converged ? (double*)take(S * (size_t)check_chunks(n_fine) * 24) : nullptr;
    H.order = converged ? (int32_t*)take(S * 4) : nullptr;
    H.alpha = converged ? (double*)take(S * 8) : nullptr;
    return FM_OK;
}

constexpr size_t kMaxSmem = 200 * 1024;   // dynamic shared memory of the tile smoother

// Resident warps of the strip smoother on the whole GPU, [FP64, FP32][1 or 2 sweeps][fused residual].
static int g_strip_warps[2][2][2] = {};

template <typename T, int HS, bool FUSE>
static void strip_occupancy(int sms) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_rbgs_strip<T, HS, FUSE>, 32 * kStripWarps, 0) !=
        cudaSuccess)
        blocks = 1;
    g_strip_warps[sizeof(T) == 4 ? 1 : 0][HS / 2 - 1][FUSE ? 1 : 0] =
        std::max(1, blocks) * kStripWarps * std::max(1, sms);
}

// Kernel attributes and occupancies, set once per process before any launch
// or capture.
void fmg_init_attributes() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_rbgs_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        cudaFuncSetAttribute(k_rbgs_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        cudaFuncSetAttribute(k_vcycle_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tail_smem_max<float>());
        cudaFuncSetAttribute(k_vcycle_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tail_smem_max<double>());
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        strip_occupancy<float, 2, false>(sms);
        strip_occupancy<float, 4, false>(sms);
        strip_occupancy<double, 2, false>(sms);
        strip_occupancy<double, 4, false>(sms);
        strip_occupancy<float, 2, true>(sms);
        strip_occupancy<float, 4, true>(sms);
        strip_occupancy<double, 2, true>(sms);
        strip_occupancy<double, 4, true>(sms);
        cudaGetLastError();
    });
}

// Rows per segment of the strip smoother: the power-of-two fraction of n (at
// least 16 rows) that minimises the waves of units over the resident warps
// times the steps of one unit (segment plus 2 VH halo rows plus the steps
// that drain the wavefront).
static int strip_segment(int n, size_t S, int strips, int HS, int VH, int resident) {
    int best = n;
    double best_cost = 1e300;
    for (int seg = n; seg >= 16; seg /= 2) {
        const size_t units = S * (size_t)strips * ((n + seg - 1) / seg);
        const double waves = std::ceil((double)units / std::max(1, resident));
        const double cost = waves * (std::min(seg + (seg < n ? 2 * VH : 0), n) + HS + 1);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = seg;
        }
    }
    return best;
}

// One strip-smoother launch (bc, pc: with the fused residual and restriction
// to the coarse grid).  nsweeps is 1 or 2 and n even (smooth_shape).
template <typename T, int HS, bool FUSE>
static void strip_launch(fm_ctx* ctx, int n, size_t S, const T* b, const T* Te, const T* Tn, const T* D,
                         const T* p_in, T* p_out, const int32_t* active, const T* ec, T* bc, T* pc,
                         cudaStream_t st, size_t busy, const int32_t* order, int ns, const int32_t* dcount) {
    constexpr int OW = strip_ow(HS, FUSE), VH = strip_xh(HS, FUSE);
    const int strips = (n + OW - 1) / OW;
    const int resident = g_strip_warps[sizeof(T) == 4 ? 1 : 0][HS / 2 - 1][FUSE];
    // with the host's count of active samples and their list, enumerate only
    // those; with a device-side count (dcount, refinement loops inside a
    // graph) the kernel enumerates the listed samples itself, and the grid
    // covers the most units it can form (all samples, or one wave)
    const bool dev = dcount && order;
    const bool listed = !dev && order && busy > 0 && busy < S;
    const size_t sb = listed ? busy : S;
    const int seg = strip_segment(n, sb, strips, HS, VH, resident);
    const int segs = (n + seg - 1) / seg;
    size_t units = sb * (size_t)strips * segs;
    if (dev) units = std::max(units, (size_t)resident);
    const size_t cells = sb * (size_t)n * n;
    const unsigned grid = (unsigned)((units + kStripWarps - 1) / kStripWarps);
    const double bytes = (6.0 + (FUSE ? 0.5 : 0.0)) * sizeof(T) * cells;
    const double flops = 5.0 * HS * cells + (FUSE ? 12.0 * cells : 0.0);
    FM_TIMED(ctx, kFamSmootherStrip, st, bytes, flops,
             k_rbgs_strip<T, HS, FUSE><<<grid, 32 * kStripWarps, 0, st>>>(
                 n, sb, strips, seg, segs, b, Te, Tn, D, p_in, p_out, active, ec, bc, pc,
                 (listed || dev) ? order : nullptr, ns, dev ? dcount : nullptr, resident));
}

// Launch shape code of the column-strip smoother (tile codes are > 0, colour
// launches 0).  It runs 1 or 2 sweeps on even grids of at least 16 cells.
constexpr int kShapeStrip = -1;
static bool strip_fits(int n, int nu1, int nu2) {
    return n >= 16 && n % 2 == 0 && nu1 >= 1 && nu1 <= 2 && nu2 >= 1 && nu2 <= 2;
}

static size_t tile_smem_bytes(int tile, int n, int nsweeps, size_t tsize) {
    const int TI = std::min(tile, n);
    const int hh = TI >= n ? 0 : 2 * nsweeps;
    const int RW = std::min(TI + 2 * hh, n);
    return 5 * (size_t)RW * RW * tsize;
}

// Launch shape `tile` (tile interior staged in shared memory, p_in -> p_out;
// 0: one launch per colour and sweep, in place on p_in) with `threads` per
// CTA.  Returns the buffer that holds the result.  With ec (tile shapes
// only), the iterate is p_in + P ec, the coarse-grid correction added as
// the tiles load.
template <typename T>
static T* smooth_with(fm_ctx* ctx, int tile, int threads, int n, size_t S, int nsweeps, const T* b, const T* Te,
                      const T* Tn, const T* D, T* p_in, T* p_out, const int32_t* active, cudaStream_t st,
                      const T* ec = nullptr, size_t busy = 0, const int32_t* order = nullptr, int ns = 0,
                      const int32_t* dcount = nullptr) {
    if (nsweeps <= 0) return p_in;
    const size_t cells = S * (size_t)n * n;
    if (tile == kShapeStrip) {
        if (nsweeps == 2)
            strip_launch<T, 4, false>(ctx, n, S, b, Te, Tn, D, p_in, p_out, active, ec, nullptr, nullptr, st, busy,
                                      order, ns, dcount);
        else
            strip_launch<T, 2, false>(ctx, n, S, b, Te, Tn, D, p_in, p_out, active, ec, nullptr, nullptr, st, busy,
                                      order, ns, dcount);
        return p_out;
    }
    if (tile > 0) {
        const int TI = std::min(tile, n);
        const int hh = TI >= n ? 0 : 2 * nsweeps;
        const int tiles = (n + TI - 1) / TI;
        const unsigned grid = (unsigned)(S * tiles * tiles);
        const double bytes = 6.0 * sizeof(T) * cells, flops = 10.0 * nsweeps * cells;
        // register-blocked regions (threads == 0): whole grids of 8, 16, 32
        // (and, FP32, 64) cells, or 32 (and, FP32, 64) interiors with a halo of
        // up to 4 (nsweeps <= 2); FP64 copies of the large regions would spill
        constexpr bool f32 = sizeof(T) == 4;
        if (threads == 0 && hh == 0 && (n == 8 || n == 16 || n == 32 || (f32 && n == 64))) {
            if (n == 8)
                FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops, k_rbgs_tile_reg<T, 8, 1><<<grid, 4 * 8, 0, st>>>(
                    n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
            else if (n == 16)
                FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops, k_rbgs_tile_reg<T, 16, 2><<<grid, 8 * 8, 0, st>>>(
                    n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
            else if (n == 32)
                FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops, k_rbgs_tile_reg<T, 32, 4><<<grid, 16 * 8, 0, st>>>(
                    n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
            else if constexpr (f32)
                FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops, k_rbgs_tile_reg<T, 64, 8><<<grid, 32 * 8, 0, st>>>(
                    n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
            return p_out;
        }
        if (threads == 0 && hh > 0 && hh <= 4 && (TI == 32 || (f32 && TI == 64))) {
            if (TI == 32)
                FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops, k_rbgs_tile_reg<T, 40, 5><<<grid, 20 * 8, 0, st>>>(
                    n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
            else if constexpr (f32)
                FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops, k_rbgs_tile_reg<T, 72, 9><<<grid, 36 * 8, 0, st>>>(
                    n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
            return p_out;
        }
        FM_TIMED(ctx, kFamSmootherTile, st, bytes, flops,
                 k_rbgs_tile<T><<<grid, threads > 0 ? threads : 256, tile_smem_bytes(tile, n, nsweeps, sizeof(T)),
                                  st>>>(n, S, TI, hh, nsweeps, b, Te, Tn, D, p_in, p_out, active, ec, ns));
        return p_out;
    }
    T* p = p_in;
    const size_t half = cells / 2;
    for (int it = 0; it < nsweeps; ++it)
        for (int color = 0; color < 2; ++color)
            FM_TIMED(ctx, kFamSmoother, st, 3.0 * sizeof(T) * cells, 5.0 * cells,
                     k_rbgs_color<T><<<blocks_for(half), kBlock, 0, st>>>(n, S, color, b, Te, Tn, D, p, active));
    return p;
}

static int tune_slot(int n) { return std::min(15, 31 - __builtin_clz((unsigned)n)); }

// Smoother launch shape of grid n.  Untuned defaults (fm_autotune's choices
// on GB300 for two sweeps): register-blocked regions up to 32 x 32, then FP32
// column strips; FP64 keeps one launch per colour up to 512 (its strips and
// tiles are bound by the FP64 divide) and strips above.  An fm_autotune or
// fm_set_smoother_shape entry for this grid and precision replaces the
// default.  Tiles and strips need both smoothing phases of the V-cycle (so
// the iterate goes p -> p2 -> p); tiles need their staged region in shared
// memory, strips 1 or 2 sweeps.
template <typename T>
static void smooth_shape(const fm_ctx* ctx, int n, const fm_solve_params& prm, int* tile, int* threads) {
    const int pi = sizeof(T) == 4 ? 1 : 0, slot = tune_slot(n);
    const bool f32 = sizeof(T) == 4;
    *tile = 0;
    *threads = 0;
    if (n <= 32) *tile = 32;   // one register-blocked region per sample
    else if (f32 || n > 512) *tile = kShapeStrip;
    if (ctx->tune.n[pi][slot] == n) {
        *tile = ctx->tune.tile[pi][slot];
        *threads = ctx->tune.threads[pi][slot];
    }
    if (*tile > 0 && (prm.nu1 < 1 || prm.nu2 < 1 ||
                      tile_smem_bytes(*tile, n, std::max(prm.nu1, prm.nu2), sizeof(T)) > kMaxSmem))
        *tile = 0;
    if (*tile == kShapeStrip && !strip_fits(n, prm.nu1, prm.nu2)) *tile = 0;
}

// The V-cycle below correction grid kt (<= 32 x 32) as one resident tail
// launch over the listed samples (k_vcycle_tail).
template <typename T>
static void vcycle_tail(const Hierarchy<T>& H, int kt, const fm_solve_params& prm, const int32_t* active,
                        cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    TailArgs<T> a{};
    a.kt = kt;
    a.n0 = H.n0;
    a.nu1 = prm.nu1;
    a.nu2 = prm.nu2;
    a.ns = prm.bc_case == FM_CASE_I ? 1 : 0;
    const bool listed = H.listed();
    a.S = listed ? H.busy : H.S;
    double cells = 0.0;
    for (int j = 0; j <= kt; ++j) {
        a.Te[j] = H.g[j].TeC;
        a.Tn[j] = H.g[j].TnC;
        a.D[j] = H.g[j].DC;
        cells += (double)H.g[j].n * H.g[j].n;
    }
    a.b = H.g[kt].b;
    a.p = H.g[kt].p;
    a.Ainv = H.AinvC;
    a.active = active;
    a.order = listed ? H.order : nullptr;
    const size_t smem = tail_smem_bytes<T>(kt, H.n0);
    const double top = (double)H.g[kt].n * H.g[kt].n;
    FM_TIMED(ctx, kFamVcycleTail, st, (3.0 * cells + 2.0 * top) * sizeof(T) * a.S,
             (10.0 * (prm.nu1 + prm.nu2) + 18.0) * cells * a.S,
             k_vcycle_tail<T><<<(unsigned)a.S, kTailThreads, smem, st>>>(a));
}

// One V(nu1, nu2) cycle on grid k; grid `top` carries the stage operator
// (injected K), the grids below it the correction operators (child means).
template <typename T>
static void vcycle(const Hierarchy<T>& H, int k, int top, const fm_solve_params& prm, const int32_t* active,
                   cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    const size_t S = H.S;
    const GridBufs<T>& g = H.g[k];
    const double ts = sizeof(T);
    const bool stage_op = (k == top);
    const int ns = prm.bc_case == FM_CASE_I ? 1 : 0;   // Dirichlet north / south edges (Table 1, Case I)
    const T* Te = stage_op ? g.Te : g.TeC;
    const T* Tn = stage_op ? g.Tn : g.TnC;
    const T* D = stage_op ? g.D : g.DC;
    if (k == 0) {
        const int m = H.n0 * H.n0;
        FM_TIMED(ctx, kFamCoarseSolve, st, (double)S * (m * m + 2 * m) * ts, 2.0 * S * m * m,
                 k_coarse_solve<T><<<blocks_for(S * m), kBlock, 0, st>>>(m, S, stage_op ? H.Ainv : H.AinvC, g.b,
                                                                         g.p, active));
        return;
    }
    const int n = g.n;
    const size_t cells = S * (size_t)n * n;
    int tile, threads;
    smooth_shape<T>(ctx, n, prm, &tile, &threads);
    // pre-smoothing p -> p2 (tiles, strips) or in place; post-smoothing back into p
    const GridBufs<T>& c = H.g[k - 1];
    T* cur;
    if (tile == kShapeStrip) {
        // strips form the residual and its restriction in the same pass
        if (prm.nu1 == 2)
            strip_launch<T, 4, true>(ctx, n, S, g.b, Te, Tn, D, g.p, g.p2, active, nullptr, c.b, c.p, st, H.busy,
                                     H.order, ns, H.dcount);
        else
            strip_launch<T, 2, true>(ctx, n, S, g.b, Te, Tn, D, g.p, g.p2, active, nullptr, c.b, c.p, st, H.busy,
                                     H.order, ns, H.dcount);
        cur = g.p2;
    } else {
        cur = smooth_with<T>(ctx, tile, threads, n, S, prm.nu1, g.b, Te, Tn, D, g.p, g.p2, active, st, nullptr,
                             H.busy, H.order, ns, H.dcount);
        FM_TIMED(ctx, kFamResidualRestrict, st, 5.5 * ts * cells, 10.0 * cells,
                 k_residual_restrict<T><<<blocks_for(S * (size_t)c.n * c.n), kBlock, 0, st>>>(
                     c.n, S, g.b, Te, Tn, D, cur, c.b, c.p, active));
    }
    // the V-cycle below: the resident tail for correction grids up to
    // ctx->tail_max, else grid by grid
    if (k - 1 >= 1 && c.n <= ctx->tail_max && !prm.energy_step && S > 0)
        vcycle_tail(H, k - 1, prm, active, st);
    else
        vcycle(H, k - 1, top, prm, active, st);
    if (prm.energy_step) {
        // the stepped correction (converged mode: partials and alpha in the hierarchy)
        const int chunks = check_chunks(n);
        const bool listed = H.listed();
        const size_t nl = listed ? H.busy : S;
        FM_TIMED(ctx, kFamProlong, st, (5.0 * ts + 1.25 * ts) * nl * n * n + 2.0 * ts * cells, 40.0 * nl * n * n,
                 k_energy_partials<T><<<(unsigned)(nl * chunks), kBlock, 0, st>>>(
                     n, nl, chunks, g.b, Te, Tn, D, cur, c.p, active, listed ? H.order : nullptr, H.partial, ns);
                 k_energy_alpha<<<blocks_for(S), kBlock, 0, st>>>(S, chunks, H.partial, H.alpha, active);
                 k_prolong_step<T><<<blocks_for(cells), kBlock, 0, st>>>(c.n, S, c.p, H.alpha, cur, active, ns));
        smooth_with<T>(ctx, tile, threads, n, S, prm.nu2, g.b, Te, Tn, D, cur, g.p, active, st, nullptr, H.busy,
                       H.order, ns, H.dcount);
        return;
    }
    if (tile == 0 && prm.nu2 >= 1) {
        // colour launches: the correction rides in the first post-smoothing colour
        FM_TIMED(ctx, kFamSmoother, st, 3.0 * ts * cells + ts * S * c.n * c.n, 5.0 * cells,
                 k_rbgs_color0_prolong<T><<<blocks_for(cells / 2), kBlock, 0, st>>>(n, S, g.b, Te, Tn, D, cur, c.p,
                                                                                    active, ns));
        FM_TIMED(ctx, kFamSmoother, st, 3.0 * ts * cells, 5.0 * cells,
                 k_rbgs_color<T><<<blocks_for(cells / 2), kBlock, 0, st>>>(n, S, 1, g.b, Te, Tn, D, cur, active));
        smooth_with<T>(ctx, 0, 0, n, S, prm.nu2 - 1, g.b, Te, Tn, D, cur, g.p, active, st);
        return;
    }
    if (tile != 0 && prm.nu2 >= 1) {
        // tiles and strips: the correction is added as they load the iterate
        smooth_with<T>(ctx, tile, threads, n, S, prm.nu2, g.b, Te, Tn, D, cur, g.p, active, st, c.p, H.busy,
                       H.order, ns, H.dcount);
        return;
    }
    const Ghost<T> zero{T(0), T(0), T(0), T(0), ns};
    FM_TIMED(ctx, kFamProlong, st, 2.25 * ts * cells, 8.0 * cells,
             k_prolong<T><<<blocks_for(cells), kBlock, 0, st>>>(c.n, S, c.p, zero, 1, cur, active));
    smooth_with<T>(ctx, tile, threads, n, S, prm.nu2, g.b, Te, Tn, D, cur, g.p, active, st, nullptr, H.busy,
                   H.order, ns, H.dcount);
}

template <typename P>
static void outflux(fm_ctx* ctx, int n, size_t S, const double* K, const P* p, const Bnd& bd, double* q,
                    cudaStream_t st) {
    FM_TIMED(ctx, kFamOutflux, st, 16.0 * S * n, 3.0 * S * n,
             k_outflux<P><<<blocks_for(S * 32), kBlock, 0, st>>>(n, S, K, p, bd, q));
}

// One residual test of the refined stage on grid k (partials, then the decision).
template <typename T>
static void stage_test(const Hierarchy<T>& H, int k, const fm_solve_params& prm, bool mixed, cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    const GridBufs<T>& g = H.g[k];
    const size_t S = H.S, cells = (size_t)g.n * g.n;
    const int chunks = check_chunks(g.n);
    const size_t ns = H.listed() ? H.busy : S;
    FM_TIMED(ctx, kFamResidualRestrict, st, (mixed ? 48.0 : 40.0) * ns * cells, 12.0 * ns * cells,
             k_stage_partials<T><<<(unsigned)(ns * chunks), kBlock, 0, st>>>(
                 g.n, ns, chunks, g.K, bnd_of(prm), g.b, g.Te, g.Tn, g.D, g.p, g.p64, g.Te64, g.Tn64, g.D64, g.b,
                 g.p, H.active, H.partial, H.listed() ? H.order : nullptr);
             k_stage_decide<<<blocks_for(S), kBlock, 0, st>>>(S, chunks, H.partial, prm.tol, prm.qtol, H.qprev,
                                                              H.active, H.left, H.order));
}

// Blocks of a refinement update over `work` cells: enough to fill the GPU a
// few times over, the grid-stride loop takes the rest.
static unsigned ir_update_blocks(const fm_ctx* ctx, size_t work) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    return (unsigned)std::max<size_t>(1, std::min<size_t>(blocks_for(work), (size_t)sms * 16));
}

// Loop control of a refined stage inside a CUDA graph: after residual test
// number *it, another pass runs while a sample is still active and fewer than
// max_cycles tests have been made; the bound ends every loop.
__global__ void k_refine_cond(const int32_t* __restrict__ left, int32_t* __restrict__ it, int max_cycles,
                              cudaGraphConditionalHandle h) {
    const int i = *it;
    *it = i + 1;
    cudaGraphSetConditional(h, (*left > 0 && i < max_cycles) ? 1u : 0u);
}

// The refined stage as a device-side loop of the graph being captured on
// st: a residual test, then a conditional WHILE node whose body is nu0
// V-cycles (masked to the active samples), the FP64 update of the mixed form
// and the next test.  No host synchronisation; the same tests and updates in
// the same order as the host loop of refine_stage.
template <typename T>
static fm_status refine_stage_graph(const Hierarchy<T>& H, int k, const fm_solve_params& prm, bool mixed,
                                    int32_t* status, cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    const GridBufs<T>& g = H.g[k];
    const size_t S = H.S, cells = (size_t)g.n * g.n;
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    FM_CUDA_TRY(ctx, cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h;
    FM_CUDA_TRY(ctx, cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault));
    auto test = [&](cudaStream_t s) {
        cudaMemsetAsync(H.left, 0, sizeof(int32_t), s);
        stage_test(H, k, prm, mixed, s);
        k_refine_cond<<<1, 1, 0, s>>>(H.left, H.iter, prm.max_cycles, h);
    };
    FM_CUDA_TRY(ctx, cudaMemsetAsync(H.active, 0xff, S * sizeof(int32_t), st));   // all active (-1)
    FM_CUDA_TRY(ctx, cudaMemsetAsync(H.qprev, 0xff, S * sizeof(double), st));     // NaN
    FM_CUDA_TRY(ctx, cudaMemsetAsync(H.iter, 0, sizeof(int32_t), st));
    test(st);
    FM_CUDA_TRY(ctx, cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    FM_CUDA_TRY(ctx, cudaGraphAddNode(&node, graph, deps, nullptr, nd, &np));
    FM_CUDA_TRY(ctx, cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    // the body is captured on a stream of the branch's own priority
    int prio = 0;
    FM_CUDA_TRY(ctx, cudaStreamGetPriority(st, &prio));
    prio = std::min(std::max(prio, ctx->prio_hi), ctx->prio_lo);
    cudaStream_t bs = ctx->body_stream[prio - ctx->prio_hi];
    FM_CUDA_TRY(ctx, cudaStreamBeginCaptureToGraph(bs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed));
    // the body's strips enumerate the samples the last test listed
    H.dcount = H.order ? H.left : nullptr;
    for (int v = 0; v < cycles_per_test(prm); ++v) vcycle(H, k, k, prm, H.active, bs);
    H.dcount = nullptr;
    if (mixed)
        k_ir_update<T><<<ir_update_blocks(ctx, S * cells), kBlock, 0, bs>>>(cells, S, g.p, g.p64, H.active,
                                                                              H.order, H.order ? H.left : nullptr);
    test(bs);
    cudaGraph_t body = nullptr;
    FM_CUDA_TRY(ctx, cudaStreamEndCapture(bs, &body));
    if (status) k_status<<<blocks_for(S), kBlock, 0, st>>>(S, H.active, status);
    return FM_OK;
}

// Cycles of one refined stage until every sample passes its residual test.
template <typename T>
static fm_status refine_stage(const Hierarchy<T>& H, int k, const fm_solve_params& prm, bool mixed,
                              int32_t* status, cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    FM_CUDA_TRY(ctx, cudaStreamIsCapturing(st, &capturing));
    if (capturing == cudaStreamCaptureStatusActive) return refine_stage_graph(H, k, prm, mixed, status, st);
    const GridBufs<T>& g = H.g[k];
    const size_t S = H.S, cells = (size_t)g.n * g.n;
    FM_CUDA_TRY(ctx, cudaMemsetAsync(H.active, 0xff, S * sizeof(int32_t), st));   // all active (-1)
    FM_CUDA_TRY(ctx, cudaMemsetAsync(H.qprev, 0xff, S * sizeof(double), st));     // NaN
    int32_t left = 0;
    for (int it = 0;; ++it) {
        FM_CUDA_TRY(ctx, cudaMemsetAsync(H.left, 0, sizeof(int32_t), st));
        stage_test(H, k, prm, mixed, st);
        FM_CUDA_TRY(ctx, cudaMemcpyAsync(&left, H.left, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        H.busy = left > 0 ? (size_t)left : S;
        if (left == 0) break;
        if (it >= prm.max_cycles) {
            if (status) k_status<<<blocks_for(S), kBlock, 0, st>>>(S, H.active, status);
            break;
        }
        for (int v = 0; v < cycles_per_test(prm); ++v) vcycle(H, k, k, prm, H.active, st);
        if (mixed)
            k_ir_update<T><<<ir_update_blocks(ctx, (H.listed() ? H.busy : S) * cells), kBlock, 0, st>>>(
                cells, H.listed() ? H.busy : S, g.p, g.p64, H.active, H.listed() ? H.order : nullptr, nullptr);
    }
    H.busy = 0;   // later stages run every sample
    return FM_OK;
}

template <typename T>
static fm_status fmg_batch(const Hierarchy<T>& H, const fm_solve_params& prm, double* qf, double* qc,
                           double* p_out, int32_t* status, cudaStream_t st) {
    fm_ctx* ctx = H.ctx;
    const size_t S = H.S;
    const bool mixed = prm.precision == FM_PREC_MIXED;
    const bool conv = prm.converged != 0;
    const double ts = sizeof(T);
    const Bnd bd = bnd_of(prm);
    if (status) FM_CUDA_TRY(ctx, cudaMemsetAsync(status, 0, sizeof(int32_t) * S, st));
    // coefficient hierarchy: inject, then faces and diagonals on every grid
    for (int k = H.m; k >= 1; --k) {
        const int nc = H.g[k - 1].n;
        const size_t cc = S * (size_t)nc * nc;
        FM_TIMED(ctx, kFamInject, st, 16.0 * cc, 0.0,
                 k_inject<<<blocks_for(cc), kBlock, 0, st>>>(nc, S, H.g[k].K, const_cast<double*>(H.g[k - 1].K)));
    }
    for (int k = 0; k <= H.m; ++k) {
        const GridBufs<T>& g = H.g[k];
        const size_t cells = S * (size_t)g.n * g.n;
        // FP64 arithmetic for FP64 grids and for the refined grids' FP64 copies
        if (sizeof(T) == 8 || g.Te64)
            FM_TIMED(ctx, kFamCoefficients, st, (8.0 + 3.0 * ts + (g.Te64 ? 24.0 : 0.0)) * cells, 16.0 * cells,
                     k_faces<T, double><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, bd.ns, g.K, g.Te, g.Tn,
                                                                              g.Te64, g.Tn64);
                     k_diagonal<T, double><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, bd.ns, g.K, g.Te, g.Tn,
                                                                                 g.Te64, g.Tn64, g.D, g.D64));
        else
            FM_TIMED(ctx, kFamCoefficients, st, (8.0 + 3.0 * ts) * cells, 16.0 * cells,
                     k_faces<T, T><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, bd.ns, g.K, g.Te, g.Tn, nullptr,
                                                                         nullptr);
                     k_diagonal<T, T><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, bd.ns, g.K, g.Te, g.Tn, nullptr,
                                                                            nullptr, g.D, nullptr));
    }
    for (int k = 0; k < H.m; ++k) {
        const GridBufs<T>& g = H.g[k];
        const size_t cells = S * (size_t)g.n * g.n;
        FM_TIMED(ctx, kFamCoefficients, st, (32.0 + 8.0 + 3.0 * ts) * cells, 40.0 * cells,
                 k_child_geomean<T><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, H.g[k + 1].K, g.Kc);
                 k_faces<T, T><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, bd.ns, g.Kc, g.TeC, g.TnC, nullptr,
                                                                     nullptr);
                 k_diagonal<T, T><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, bd.ns, g.Kc, g.TeC, g.TnC, nullptr,
                                                                        nullptr, g.DC, nullptr));
    }
    if (H.m >= 1) {
        const int m = H.n0 * H.n0;
        FM_TIMED(ctx, kFamCoarseInverse, st, (double)S * (8 * m + ts * m * m), 2.0 * S * m * m * m,
                 k_coarse_inverse<T><<<(unsigned)((S + kInvWarps - 1) / kInvWarps), 32 * kInvWarps, 0, st>>>(
                     H.n0, S, H.g[0].Kc, H.AinvC, bd.ns));
    }
    {
        const int m = H.n0 * H.n0;
        FM_TIMED(ctx, kFamCoarseInverse, st, (double)S * (8 * m + ts * m * m), 2.0 * S * m * m * m,
                 k_coarse_inverse<T><<<(unsigned)((S + kInvWarps - 1) / kInvWarps), 32 * kInvWarps, 0, st>>>(H.n0, S, H.g[0].K, H.Ainv,
                                                                                                 bd.ns));
    }
    // the stage one grid coarser is refined only where its QoI is asked for:
    // otherwise it just gives the finest stage its starting guess
    const bool refine_c = conv && qc != nullptr;
    for (int k = 0; k <= H.m; ++k) {
        const GridBufs<T>& g = H.g[k];
        const size_t cells = S * (size_t)g.n * g.n;
        const bool refined = conv && (k == H.m || (k == H.m - 1 && refine_c));
        if (k > 0) {
            const GridBufs<T>& c = H.g[k - 1];
            if (mixed && refined && k == H.m && H.m >= 1 && refine_c) {
                FM_TIMED(ctx, kFamFmgInterp, st, 10.0 * cells, 8.0 * cells,
                         k_prolong<double><<<blocks_for(cells), kBlock, 0, st>>>(
                             c.n, S, c.p64, Ghost<double>{bd.g[0], bd.g[1], bd.g[2], bd.g[3], bd.ns}, 0, g.p64,
                             nullptr));
            } else {
                FM_TIMED(ctx, kFamFmgInterp, st, 1.25 * ts * cells, 8.0 * cells,
                         k_prolong<T><<<blocks_for(cells), kBlock, 0, st>>>(
                             c.n, S, c.p, Ghost<T>{(T)bd.g[0], (T)bd.g[1], (T)bd.g[2], (T)bd.g[3], bd.ns}, 0, g.p,
                             nullptr));
            }
        }
        FM_TIMED(ctx, kFamStageRhs, st, (8.0 + ts) * cells, 2.0 * cells,
                 k_stage_rhs<T><<<blocks_for(cells), kBlock, 0, st>>>(g.n, S, g.K, bd, g.b));
        if (k == 0) vcycle(H, 0, 0, prm, nullptr, st);
        if (!refined) {
            if (k > 0)
                for (int it = 0; it < prm.nu0; ++it) vcycle(H, k, k, prm, nullptr, st);
        } else {
            if (mixed && !(k == H.m && H.m >= 1 && refine_c))
                k_widen<T><<<blocks_for(cells), kBlock, 0, st>>>(cells, g.p, g.p64);
            FM_TRY(refine_stage(H, k, prm, mixed, status, st));
        }
        if (k == H.m - 1 && qc) {
            if (mixed && refined) outflux(ctx, g.n, S, g.K, g.p64, bd, qc, st);
            else outflux(ctx, g.n, S, g.K, g.p, bd, qc, st);
        }
    }
    const GridBufs<T>& f = H.g[H.m];
    const bool fine64 = mixed && conv;
    if (H.m == 0 && qc) k_fill<<<blocks_for(S), kBlock, 0, st>>>(S, std::nan(""), qc);
    if (fine64) outflux(ctx, f.n, S, f.K, f.p64, bd, qf, st);
    else outflux(ctx, f.n, S, f.K, f.p, bd, qf, st);
    if (p_out) {
        const size_t cells = S * (size_t)f.n * f.n;
        if (fine64)
            FM_CUDA_TRY(ctx, cudaMemcpyAsync(p_out, f.p64, sizeof(double) * cells, cudaMemcpyDeviceToDevice, st));
        else
            k_widen<T><<<blocks_for(cells), kBlock, 0, st>>>(cells, f.p, p_out);
    }
    return FM_OK;
}

template <typename T>
static fm_status levelwise(fm_ctx* ctx, Arena& ar, int n_fine, int n0, uint32_t S, const double* d_K,
                           const fm_solve_params& prm, double* d_qf, double* d_qc, double* d_p,
                           int32_t* d_status, cudaStream_t st) {
    const bool mixed = prm.precision == FM_PREC_MIXED;
    const int64_t lim = batch_limit(ctx, n_fine);
    for (uint64_t first = 0; first < S; first += (uint64_t)lim) {
        const size_t cnt = (size_t)std::min<uint64_t>((uint64_t)lim, S - first);
        const size_t off = first * (size_t)n_fine * n_fine;
        Hierarchy<T> H;
        FM_TRY(carve(ctx, ar, H, n_fine, n0, cnt, d_K + off, mixed, prm.converged != 0));
        FM_TRY(fmg_batch(H, prm, d_qf + first, d_qc ? d_qc + first : nullptr, d_p ? d_p + off : nullptr,
                         d_status ? d_status + first : nullptr, st));
        FM_CUDA_TRY(ctx, cudaGetLastError());
    }
    return FM_OK;
}

// Scratch bytes a level-wise solve of S samples of grid n_fine takes (one batch).
size_t fmg_levelwise_scratch(const fm_ctx* ctx, int n_fine, uint32_t S, const fm_solve_params& prm) {
    const bool mixed = prm.precision == FM_PREC_MIXED;
    const size_t cnt = (size_t)std::min<int64_t>(batch_limit(ctx, n_fine), S);
    return hierarchy_bytes(n_fine, prm.n_coarsest, cnt, mixed ? 4 : 8, mixed, prm.converged != 0);
}

fm_status fmg_solve_impl(fm_ctx* ctx, int n_fine, uint32_t S, const double* d_K,
                         const fm_solve_params& prm, double* d_qf, double* d_qc, double* d_p,
                         int32_t* d_status, cudaStream_t st) {
    return fmg_solve_with(ctx, ctx->arena, n_fine, S, d_K, prm, d_qf, d_qc, d_p, d_status, st);
}

fm_status fmg_solve_with(fm_ctx* ctx, Arena& ar, int n_fine, uint32_t S, const double* d_K,
                         const fm_solve_params& prm, double* d_qf, double* d_qc, double* d_p,
                         int32_t* d_status, cudaStream_t st) {
    const int n0 = prm.n_coarsest;
    FM_CHECK_ARG(ctx, n0 >= 2 && n0 <= 4, "fmg_solve_batch: n_coarsest must be 2..4");
    FM_CHECK_ARG(ctx, n_fine >= n0 && n_fine <= 8192, "fmg_solve_batch: bad n_fine");
    int m = 0;
    while ((n0 << m) < n_fine) ++m;
    FM_CHECK_ARG(ctx, (n0 << m) == n_fine, "fmg_solve_batch: n_fine must be n_coarsest * 2^m");
    FM_CHECK_ARG(ctx, prm.nu0 >= 1 && prm.nu1 >= 0 && prm.nu2 >= 0 && prm.nu1 + prm.nu2 >= 1,
                 "fmg_solve_batch: need nu0 >= 1 and nu1 + nu2 >= 1");
    FM_CHECK_ARG(ctx, prm.precision == FM_PREC_FP64 || prm.precision == FM_PREC_MIXED,
                 "fmg_solve_batch: unknown precision");
    FM_CHECK_ARG(ctx, prm.precision != FM_PREC_MIXED || prm.converged,
                 "fmg_solve_batch: the mixed form refines to a tolerance (converged = 1)");
    FM_CHECK_ARG(ctx, !prm.converged || (prm.tol > 0 && prm.max_cycles >= 1),
                 "fmg_solve_batch: converged mode needs tol > 0 and max_cycles >= 1");
    FM_CHECK_ARG(ctx, S == 0 || (d_K && d_qf), "fmg_solve_batch: null input or output");
    FM_CHECK_ARG(ctx, prm.kernel >= FM_KERNEL_AUTO && prm.kernel <= FM_KERNEL_RESIDENT,
                 "fmg_solve_batch: unknown kernel schedule");
    FM_CHECK_ARG(ctx, prm.ir_cycles >= 0 && prm.ir_cycles <= 64, "fmg_solve_batch: ir_cycles must be 0 .. 64");
    FM_CHECK_ARG(ctx, prm.bc_case == 0 || prm.bc_case == FM_CASE_I || prm.bc_case == FM_CASE_II,
                 "fmg_solve_batch: bc_case must be FM_CASE_I or FM_CASE_II");
    FM_CHECK_ARG(ctx, !prm.energy_step || (prm.converged && prm.kernel != FM_KERNEL_RESIDENT),
                 "fmg_solve_batch: the energy-optimal correction step runs in converged mode on the level-wise "
                 "schedule");
    if (S == 0) return FM_OK;
    if (prm.kernel == FM_KERNEL_RESIDENT || (prm.kernel == FM_KERNEL_AUTO && auto_resident(n_fine, S, ctx->sms, prm))) {
        if (fmg_resident_launch(ctx, n_fine, n0, S, d_K, prm, d_qf, d_qc, d_p, d_status, st)) {
            FM_CUDA_TRY(ctx, cudaGetLastError());
            return FM_OK;
        }
        FM_CHECK_ARG(ctx, prm.kernel == FM_KERNEL_AUTO,
                     "fmg_solve_batch: the resident schedule needs the hierarchy in shared memory "
                     "(n_fine <= 64) and a power-of-two coarsest grid (2 or 4)");
    }
    if (prm.precision == FM_PREC_MIXED)
        return levelwise<float>(ctx, ar, n_fine, n0, S, d_K, prm, d_qf, d_qc, d_p, d_status, st);
    return levelwise<double>(ctx, ar, n_fine, n0, S, d_K, prm, d_qf, d_qc, d_p, d_status, st);
}

// ------------------------------------------------------------------ allocation-free variant
// Scratch of fmg_solve_batch_static: one file-scope device array, present on
// every device that loads the library for as long as the process lives.
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
static __device__ __align__(256) char g_static_scratch[kStaticScratchBytes];

// Device address of the array on the current device.  Host code only sees a
// stand-in symbol, so the address is asked for once per device, with that
// device current, and kept.
static char* static_scratch_address(fm_ctx* ctx, fm_status* status) {
    static std::mutex mu;
    static char* addr[128] = {};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        set_error(ctx, "fmg_solve_batch_static: no current CUDA device");
        *status = FM_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error(ctx, std::string("fmg_solve_batch_static: cudaGetSymbolAddress failed: ") +
                               cudaGetErrorString(e));
            *status = FM_ECUDA;
            return nullptr;
        }
        addr[dev] = static_cast<char*>(p);
    }
    *status = FM_OK;
    return addr[dev];
}

// The level-wise FP64 hierarchy of carve(), laid out in a caller-given buffer.
static void carve_into(fm_ctx* ctx, Hierarchy<double>& H, char* base, int n_fine, int n0, size_t S,
                       const double* d_K) {
    char* cur = base;
    auto take = [&](size_t bytes) {
        char* p = cur;
        cur += ((bytes + 255) / 256) * 256;
        return p;
    };
    H.ctx = ctx;
    H.n0 = n0;
    H.S = S;
    H.m = 0;
    while ((n0 << H.m) < n_fine) ++H.m;
    for (int k = 0; k <= H.m; ++k) {
        const int n = n0 << k;
        const size_t cnt = S * (size_t)n * n;
        GridBufs<double>& g = H.g[k];
        g.n = n;
        g.K = (k == H.m) ? d_K : (double*)take(cnt * 8);
        g.Te = (double*)take(cnt * 8);
        g.Tn = (double*)take(cnt * 8);
        g.D = (double*)take(cnt * 8);
        g.p = (double*)take(cnt * 8);
        g.b = (double*)take(cnt * 8);
        g.p2 = (double*)take(cnt * 8);
        g.Kc = nullptr;
        g.TeC = g.TnC = g.DC = nullptr;
        if (k < H.m) {
            g.Kc = (double*)take(cnt * 8);
            g.TeC = (double*)take(cnt * 8);
            g.TnC = (double*)take(cnt * 8);
            g.DC = (double*)take(cnt * 8);
        }
        g.p64 = g.Te64 = g.Tn64 = g.D64 = nullptr;
    }
    H.Ainv = (double*)take(S * (size_t)n0 * n0 * n0 * n0 * 8);
    H.AinvC = (double*)take(S * (size_t)n0 * n0 * n0 * n0 * 8);
    H.active = nullptr;
    H.left = nullptr;
    H.iter = nullptr;
    H.qprev = nullptr;
    H.partial = nullptr;
    H.order = nullptr;
    H.alpha = nullptr;
}

// ------------------------------------------------------------------ autotuning
// Synthetic smoothing problem for timing: faces in (0.5, 1.5), a diagonal
// that dominates them, rhs and iterate in (-1, 1) (a hash of the index).
template <typename T>
__global__ void k_tune_fill(size_t count, T* __restrict__ b, T* __restrict__ Te, T* __restrict__ Tn,
                            T* __restrict__ D, T* __restrict__ p) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    uint64_t h = t * 0x9E3779B97F4A7C15ULL;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ULL;
    h ^= h >> 29;
    const double u0 = (double)(h & 0xFFFFF) / 1048576.0, u1 = (double)((h >> 20) & 0xFFFFF) / 1048576.0;
    const double u2 = (double)((h >> 40) & 0xFFFFF) / 1048576.0;
    Te[t] = (T)(0.5 + u0);
    Tn[t] = (T)(0.5 + u1);
    D[t] = (T)(4.5 + u2);
    b[t] = (T)(2.0 * u2 - 1.0);
    p[t] = (T)(2.0 * u0 - 1.0);
}

template <typename T>
static fm_status autotune_grid(fm_ctx* ctx, int n, int nsweeps, fm_tune_entry* e) {
    // about 64 Mi cells per call (well beyond L2), at least one sample
    const size_t S = std::max<size_t>(1, ((size_t)64 << 20) / ((size_t)n * n));
    const size_t cells = S * (size_t)n * n;
    T* buf = nullptr;
    FM_CUDA_TRY(ctx, cudaMalloc((void**)&buf, 6 * cells * sizeof(T)));
    T *b = buf, *Te = b + cells, *Tn = Te + cells, *D = Tn + cells, *p = D + cells, *p2 = p + cells;
    k_tune_fill<T><<<blocks_for(cells), kBlock>>>(cells, b, Te, Tn, D, p);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = ctx->prof.active;
    ctx->prof.active = false;
    auto time_shape = [&](int tile, int threads) -> double {
        if (tile > 0 && tile_smem_bytes(tile, n, nsweeps, sizeof(T)) > kMaxSmem) return 1e30;
        smooth_with<T>(ctx, tile, threads, n, S, nsweeps, b, Te, Tn, D, p, p2, nullptr, nullptr);   // warm-up
        cudaEventRecord(e0);
        for (int r = 0; r < 4; ++r)   // p -> p2 -> p for tiles
            smooth_with<T>(ctx, tile, threads, n, S, nsweeps, b, Te, Tn, D, r & 1 ? p2 : p, r & 1 ? p : p2, nullptr,
                           nullptr);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 4.0;
    };
    fm_solve_params dp{};
    dp.nu1 = dp.nu2 = nsweeps;
    int def_tile = 0, def_threads = 0;
    const int pi = sizeof(T) == 4 ? 1 : 0, slot = tune_slot(n);
    ctx->tune.n[pi][slot] = 0;   // the untuned default
    smooth_shape<T>(ctx, n, dp, &def_tile, &def_threads);
    double best = 1e30;
    int bt = def_tile, bth = def_threads;
    e->ms_default = time_shape(def_tile, def_threads);
    const int tiles[] = {0, kShapeStrip, 8, 16, 32, 64};
    const int thr[] = {0, 128, 256};   // 0: register-blocked regions (fixed thread count)
    for (int tile : tiles) {
        if (tile > 0 && tile > n && tile != 8) continue;   // one whole-grid candidate is enough
        if (tile == kShapeStrip && !strip_fits(n, nsweeps, nsweeps)) continue;
        for (int th : thr) {
            if (tile <= 0 && th != 0) continue;               // colour launches and strips have a fixed shape
            const double ms = time_shape(tile, th);
            if (ms < best) {
                best = ms;
                bt = tile;
                bth = th;
            }
        }
    }
    if (e->ms_default <= best) {   // the default, timed first, stays unless beaten
        best = e->ms_default;
        bt = def_tile;
        bth = def_threads;
    }
    ctx->prof.active = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    FM_CUDA_TRY(ctx, cudaGetLastError());
    ctx->tune.n[pi][slot] = n;
    ctx->tune.tile[pi][slot] = bt;
    ctx->tune.threads[pi][slot] = bth;
    e->n = n;
    e->tile = bt;
    e->threads = bth;
    e->ms_best = best;
    e->samples = (int64_t)S;
    return FM_OK;
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_autotune(fm_ctx* ctx, int32_t precision, int32_t nsweeps, int32_t n_min, int32_t n_max,
                                 fm_tune_entry* entries, int32_t max_entries, int32_t* n_entries) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_autotune: null context");
    FM_CHECK_ARG(ctx, precision == FM_PREC_FP64 || precision == FM_PREC_MIXED, "fm_autotune: unknown precision");
    FM_CHECK_ARG(ctx, nsweeps >= 1 && nsweeps <= 8, "fm_autotune: nsweeps must be 1..8");
    FM_CHECK_ARG(ctx, n_min >= 2 && n_max >= n_min && n_max <= 8192, "fm_autotune: bad grid range");
    int count = 0;
    for (int n = n_min; n <= n_max; n *= 2) {
        fm_tune_entry e{};
        if (precision == FM_PREC_MIXED) FM_TRY(autotune_grid<float>(ctx, n, nsweeps, &e));
        else FM_TRY(autotune_grid<double>(ctx, n, nsweeps, &e));
        if (entries && count < max_entries) entries[count] = e;
        ++count;
    }
    if (n_entries) *n_entries = std::min(count, max_entries);
    return FM_OK;
}

extern "C" fm_status fm_set_vcycle_tail(fm_ctx* ctx, int32_t n_max) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_set_vcycle_tail: null context");
    FM_CHECK_ARG(ctx, n_max == 0 || (n_max >= 2 && n_max <= kTailMaxN && (n_max & (n_max - 1)) == 0),
                 "fm_set_vcycle_tail: n_max must be 0 or a power of two up to 32");
    ctx->tail_max = n_max;
    return FM_OK;
}

extern "C" fm_status fm_set_smoother_shape(fm_ctx* ctx, int32_t precision, int32_t n, int32_t tile,
                                          int32_t threads) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fm_set_smoother_shape: null context");
    FM_CHECK_ARG(ctx, precision == FM_PREC_FP64 || precision == FM_PREC_MIXED,
                 "fm_set_smoother_shape: unknown precision");
    FM_CHECK_ARG(ctx, n >= 2 && n <= 8192 && (n & (n - 1)) == 0, "fm_set_smoother_shape: n must be a power of two");
    const bool tile_ok = tile == 8 || tile == 16 || tile == 32 || tile == 64;
    FM_CHECK_ARG(ctx, tile == -2 || tile == 0 || tile == kShapeStrip || tile_ok,
                 "fm_set_smoother_shape: tile must be -2, -1, 0, 8, 16, 32 or 64");
    FM_CHECK_ARG(ctx, (tile_ok && (threads == 0 || threads == 128 || threads == 256)) || (!tile_ok && threads == 0),
                 "fm_set_smoother_shape: threads must be 0 (or 128, 256 for tiles)");
    const int pi = precision == FM_PREC_MIXED ? 1 : 0, slot = tune_slot(n);
    if (tile == -2) {
        if (ctx->tune.n[pi][slot] == n) ctx->tune.n[pi][slot] = 0;
        return FM_OK;
    }
    ctx->tune.n[pi][slot] = n;
    ctx->tune.tile[pi][slot] = tile;
    ctx->tune.threads[pi][slot] = threads;
    return FM_OK;
}

extern "C" fm_status fmg_solve_batch_static(fm_ctx* ctx, int32_t n_fine, uint32_t n, const double* d_K,
                                            const fm_solve_params* prm, double* d_qf, double* d_qc,
                                            void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fmg_solve_batch_static: null context");
    FM_CHECK_ARG(ctx, prm != nullptr, "fmg_solve_batch_static: null parameters");
    const int n0 = prm->n_coarsest;
    FM_CHECK_ARG(ctx, n0 >= 2 && n0 <= 4, "fmg_solve_batch_static: n_coarsest must be 2..4");
    FM_CHECK_ARG(ctx, n_fine >= n0 && n_fine <= 8192, "fmg_solve_batch_static: bad n_fine");
    int m = 0;
    while ((n0 << m) < n_fine) ++m;
    FM_CHECK_ARG(ctx, (n0 << m) == n_fine, "fmg_solve_batch_static: n_fine must be n_coarsest * 2^m");
    FM_CHECK_ARG(ctx, prm->nu0 >= 1 && prm->nu1 >= 0 && prm->nu2 >= 0 && prm->nu1 + prm->nu2 >= 1,
                 "fmg_solve_batch_static: need nu0 >= 1 and nu1 + nu2 >= 1");
    FM_CHECK_ARG(ctx, prm->precision == FM_PREC_FP64 && !prm->converged,
                 "fmg_solve_batch_static: only the FP64 fixed-cycle schedule (converged = 0)");
    // the energy step keeps per-sample dot products and step lengths that the
    // static hierarchy has no room for
    FM_CHECK_ARG(ctx, !prm->energy_step, "fmg_solve_batch_static: the energy-optimal step is not available here");
    FM_CHECK_ARG(ctx, prm->bc_case == 0 || prm->bc_case == FM_CASE_I || prm->bc_case == FM_CASE_II,
                 "fmg_solve_batch_static: bc_case must be FM_CASE_I or FM_CASE_II");
    FM_CHECK_ARG(ctx, n == 0 || (d_K && d_qf), "fmg_solve_batch_static: null input or output");
    if (n == 0) return FM_OK;
    const size_t need = hierarchy_bytes(n_fine, n0, n, 8, false, false);
    FM_CHECK_ARG(ctx, need <= kStaticScratchBytes,
                 "fmg_solve_batch_static: " + std::to_string(n) + " samples of " + std::to_string(n_fine) + "x" +
                     std::to_string(n_fine) + " need " + std::to_string(need) + " bytes of scratch; the static "
                     "scratch holds " + std::to_string(kStaticScratchBytes) + " bytes: split the batch");
    fm_status st = FM_OK;
    char* base = static_scratch_address(ctx, &st);
    if (!base) return st;
    Hierarchy<double> H;
    carve_into(ctx, H, base, n_fine, n0, n, d_K);
    // per-launch profiling creates events and counters: off for this call
    const bool prof = ctx->prof.active;
    ctx->prof.active = false;
    const fm_status rs = fmg_batch(H, *prm, d_qf, d_qc, nullptr, nullptr, as_stream(stream));
    ctx->prof.active = prof;
    FM_TRY(rs);
    FM_CUDA_TRY(ctx, cudaGetLastError());
    return FM_OK;
}

extern "C" fm_status fmg_solve_batch(fm_ctx* ctx, int32_t n_fine, uint32_t n, const double* d_K,
                                     const fm_solve_params* prm, double* d_qf, double* d_qc,
                                     double* d_p, int32_t* d_status, void* stream) {
    FM_CHECK_ARG(ctx, ctx != nullptr, "fmg_solve_batch: null context");
    FM_CHECK_ARG(ctx, prm != nullptr, "fmg_solve_batch: null parameters");
    return fmg_solve_impl(ctx, n_fine, n, d_K, *prm, d_qf, d_qc, d_p, d_status, as_stream(stream));
}
