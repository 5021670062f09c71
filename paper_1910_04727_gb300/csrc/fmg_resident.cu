// Sample-resident full multigrid: one CTA owns one sample at a time and keeps
// its entire FMG hierarchy (Sec. 2.5) in shared memory.  HBM traffic is the
// fine coefficient field in and two QoIs out, so small grids (the level-0
// work of an MLMC run, hundreds of thousands of 16x16 .. 64x64 samples) run
// at shared-memory speed instead of streaming every sweep through L2/HBM.
// CTAs are persistent: each loops over samples blockIdx.x, +gridDim.x, ...
//
// Shared layout per grid k (n = n0 << k), type T of the V-cycle arithmetic:
//   p    iterate (a correction inside iterative refinement)
//   te   east-face transmissibility (2K on the east edge)
//   tn   north-face transmissibility (0 on the north edge)
//   tw   west-edge transmissibility 2K of each row (n values)
//   ts   south-edge transmissibility of each column (n values: 2K in Case I of
//        Table 1, where the south and north edges are Dirichlet, else 0; tn
//        of the north row likewise holds the north-edge face)
//   dinv reciprocal diagonal (FP64 form, and the mixed form up to 16 x 16;
//        otherwise the FP32 smoother divides by D formed from the faces)
//   b    right-hand side.  In the FP64 form the finest grid has none: it only
//        ever solves its stage problem, whose right-hand side (the Dirichlet
//        data) is formed on the fly from tw, te, p_W and p_E.
// Mixed form (T = float): the grids of the two refined stages (n_fine/2 and
// n_fine, which give Q^c and Q^f) also hold FP64 p, te, tn, tw; the FP64
// residual of the stage problem is the right-hand side of an FP32 V-cycle
// for the correction, which is added to the FP64 iterate.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace fm {

// Grids are n = 2^lg cells a side (the resident schedule takes power-of-two
// hierarchies), so cell c = j n + i splits by shifts and masks.
template <typename T>
struct RGrid {
    int n, lg;
    T *p, *te, *tn, *dinv, *tw, *ts, *b;   // dinv and b may be null
};

struct HGrid {
    int n, lg;
    double *p, *te, *tn, *tw, *ts;
};

__host__ __device__ inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

template <typename T>
struct RLayout {
    int m, n0;
    RGrid<T> g[8];
    HGrid h[2];      // mixed form: h[0] = grid m-1 (m >= 1), h[1] = grid m
    T* ainv;         // inverse of the coarsest operator
    T* work;         // Gauss-Jordan scratch
    double* red;     // block-reduction scratch (80 doubles)
    size_t bytes;
};

// Carve the shared buffer (or count its size when base == nullptr).  warp:
// one sample per warp (its reductions are shuffles, no block scratch).
template <typename T>
__host__ __device__ inline RLayout<T> resident_layout(char* base, int n_fine, int n0, bool mixed, bool warp) {
    RLayout<T> L;
    L.n0 = n0;
    L.m = 0;
    while ((n0 << L.m) < n_fine) ++L.m;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base + off;
        off += ((bytes + 15) / 16) * 16;
        return p;
    };
    for (int k = 0; k <= L.m; ++k) {
        const int n = n0 << k;
        const size_t c = (size_t)n * n;
        RGrid<T>& g = L.g[k];
        g.n = n;
        g.lg = ilog2(n);
        g.p = (T*)take(c * sizeof(T));
        g.te = (T*)take(c * sizeof(T));
        g.tn = (T*)take(c * sizeof(T));
        g.tw = (T*)take(n * sizeof(T));
        g.ts = (T*)take(n * sizeof(T));
        // the mixed form keeps 1/D only for hierarchies up to 16 x 16 (one
        // sample per warp), where it costs no occupancy; larger ones form D
        // from the faces and divide
        g.dinv = (mixed && n_fine > 16) ? nullptr : (T*)take(c * sizeof(T));
        g.b = (mixed || k < L.m) ? (T*)take(c * sizeof(T)) : nullptr;
    }
    for (int q = 0; q < 2; ++q) {
        const int k = L.m - 1 + q;
        HGrid& h = L.h[q];
        h.n = (k >= 0) ? (n0 << k) : 0;
        h.lg = ilog2(h.n);
        h.p = h.te = h.tn = h.tw = h.ts = nullptr;
        if (!mixed || k < 0) continue;
        const size_t c = (size_t)h.n * h.n;
        h.p = (double*)take(c * 8);
        h.te = (double*)take(c * 8);
        h.tn = (double*)take(c * 8);
        h.tw = (double*)take(h.n * 8);
        h.ts = (double*)take(h.n * 8);
    }
    L.ainv = (T*)take((size_t)n0 * n0 * n0 * n0 * sizeof(T));
    // Gauss-Jordan scratch of the coarse inverses (formed before the stage
    // loop and at stage 1): the finest grid's iterate (FP64 copy in the mixed
    // form), which nothing touches before stage m >= 2
    const size_t wbytes = (size_t)n0 * n0 * n0 * n0 * sizeof(T);
    if (L.m >= 2 && mixed && L.h[1].p)
        L.work = (T*)L.h[1].p;
    else if (L.m >= 2 && !mixed && (size_t)n_fine * n_fine * sizeof(T) >= wbytes)
        L.work = L.g[L.m].p;
    else
        L.work = (T*)take(wbytes);
    L.red = warp ? nullptr : (double*)take(80 * 8);
    L.bytes = off;
    return L;
}

template <typename C>
__device__ __forceinline__ C harm(C a, C b) {
    return C(2) * a * b / (a + b);
}

// All per-sample routines of the resident schedule, for one group of threads
// that owns a sample: the whole CTA (WARP = false) or a single warp (WARP =
// true, several samples per CTA, __syncwarp instead of CTA barriers).
template <typename T, bool WARP>
struct Res {
    static __device__ __forceinline__ int rank() { return WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x; }
    static __device__ __forceinline__ int size() { return WARP ? 32 : (int)blockDim.x; }
    static __device__ __forceinline__ void sync() {
        if (WARP) __syncwarp();
        else __syncthreads();
    }

// ------------------------------------------------------------------ setup
// Face transmissibilities of grid n, K injected from the fine field at
// stride s = n_fine / n (read from global memory; L1/L2 serve the reuse).
static __device__ void resident_setup_grid(const RGrid<T>& g, const HGrid* h, const double* __restrict__ Kf,
                                    int n_fine, int ns) {
    // FP64 faces where an FP64 copy is kept (or T is FP64); otherwise the
    // FP32 correction-solver coefficients are formed in FP32
    const int n = g.n, s = n_fine / n;
    auto K = [&](int i, int j) { return __ldg(Kf + (size_t)(s * j) * n_fine + (size_t)s * i); };
    for (int c = rank(); c < n * n; c += size()) {
        const int i = c & (n - 1), j = c >> g.lg;
        if (h || sizeof(T) == 8) {
            const double k = K(i, j);
            const double tb = ns ? 2.0 * k : 0.0;   // south / north edge face
            const double te = (i < n - 1) ? harm(k, K(i + 1, j)) : 2.0 * k;
            const double tn = (j < n - 1) ? harm(k, K(i, j + 1)) : tb;
            g.te[c] = (T)te;
            g.tn[c] = (T)tn;
            if (i == 0) g.tw[j] = (T)(2.0 * k);
            if (j == 0) g.ts[i] = (T)tb;
            if (h) {
                h->te[c] = te;
                h->tn[c] = tn;
                if (i == 0) h->tw[j] = 2.0 * k;
                if (j == 0) h->ts[i] = tb;
            }
        } else {
            const T k = (T)K(i, j);
            const T tb = ns ? T(2) * k : T(0);
            const T te = (i < n - 1) ? harm(k, (T)K(i + 1, j)) : T(2) * k;
            const T tn = (j < n - 1) ? harm(k, (T)K(i, j + 1)) : tb;
            g.te[c] = te;
            g.tn[c] = tn;
            if (i == 0) g.tw[j] = T(2) * k;
            if (j == 0) g.ts[i] = tb;
        }
    }
}

// Reciprocal diagonal of grid n from its stored faces, once every face of the
// grid is in place (each face is formed once: the west face of a cell is its
// west neighbour's east face, the same harmonic mean of the same two values),
// in the arithmetic of the V-cycles that use it (FP32 in the mixed form, also
// on the refined grids whose FP64 faces serve the residual only).
static __device__ void resident_setup_diag(const RGrid<T>& g) {
    if (!g.dinv) return;
    const int n = g.n;
    for (int c = rank(); c < n * n; c += size()) {
        const int i = c & (n - 1), j = c >> g.lg;
        const T tw = (i > 0) ? g.te[c - 1] : g.tw[j];
        const T ts = (j > 0) ? g.tn[c - n] : g.ts[i];
        g.dinv[c] = T(1) / (tw + g.te[c] + ts + g.tn[c]);
    }
}

// Coefficients of grid n as a correction grid: K of each cell is the
// geometric mean of its four children on the injected grid 2n, i.e. of the
// fine field at stride s/2.  Uses the grid's iterate as scratch, so it runs
// once the grid's stage solution has been interpolated to the next grid.
static __device__ void resident_setup_correction(const RGrid<T>& g, const double* __restrict__ Kf, int n_fine,
                                                 int ns) {
    const int n = g.n, s = n_fine / n, h2 = s / 2;
    for (int c = rank(); c < n * n; c += size()) {
        const int i = c & (n - 1), j = c >> g.lg;
        const size_t r0 = (size_t)(s * j) * n_fine + (size_t)s * i, r1 = r0 + (size_t)h2 * n_fine;
        const double a = __ldg(Kf + r0), b = __ldg(Kf + r0 + h2), cc = __ldg(Kf + r1), d = __ldg(Kf + r1 + h2);
        if (sizeof(T) == 8)
            g.p[c] = (T)exp(0.25 * (log(a) + log(b) + log(cc) + log(d)));
        else   // FP32 correction coefficients of the mixed form
            g.p[c] = (T)expf(0.25f * (logf((float)a) + logf((float)b) + logf((float)cc) + logf((float)d)));
    }
    sync();
    for (int c = rank(); c < n * n; c += size()) {
        const int i = c & (n - 1), j = c >> g.lg;
        const T k = g.p[c];
        const T tb = ns ? T(2) * k : T(0);
        const T te = (i < n - 1) ? harm(k, g.p[c + 1]) : T(2) * k;
        const T tn = (j < n - 1) ? harm(k, g.p[c + n]) : tb;
        g.te[c] = te;
        g.tn[c] = tn;
        if (i == 0) g.tw[j] = T(2) * k;
        if (j == 0) g.ts[i] = tb;
    }
    sync();
    resident_setup_diag(g);
    sync();
}

// ------------------------------------------------------------------ V-cycle pieces
// The stage problem's Dirichlet data of cell (i, j) moved to the rhs (the
// south / north edge faces are 0 unless those edges are Dirichlet).
template <typename G, typename U>
static __device__ __forceinline__ U dirichlet_at(const G& g, int c, int i, int j, const Ghost<U>& d) {
    U v = U(0);
    if (i == 0) v += g.tw[j] * d.w;
    if (i == g.n - 1) v += g.te[c] * d.e;
    if (d.ns && j == 0) v += g.ts[i] * d.s;
    if (d.ns && j == g.n - 1) v += g.tn[c] * d.n;
    return v;
}

// Right-hand side of cell (i, j): stored, or the stage problem's Dirichlet data.
static __device__ __forceinline__ T rhs_at(const RGrid<T>& g, int c, int i, int j, const Ghost<T>& d) {
    if (g.b) return g.b[c];
    return dirichlet_at(g, c, i, j, d);
}

static __device__ __forceinline__ T diag_at(const RGrid<T>& g, int c, int i, int j) {
    const T tw = (i > 0) ? g.te[c - 1] : g.tw[j];
    const T ts = (j > 0) ? g.tn[c - g.n] : g.ts[i];
    return tw + g.te[c] + ts + g.tn[c];
}

static __device__ __forceinline__ T divide_by_diag(const RGrid<T>& g, T acc, int c, int i, int j) {
    if (g.dinv) return acc * g.dinv[c];
    return acc / diag_at(g, c, i, j);
}

// Gauss-Jordan inverse of the coarsest operator, all threads of the CTA.
// A is SPD, so no pivoting.
static __device__ void resident_coarse_inverse(const RGrid<T>& g, T* ainv, T* A) {
    const int n = g.n, m = n * n;
    for (int e = rank(); e < m * m; e += size()) {
        const int lm = 2 * g.lg;   // m = n^2 = 2^lm
        const int r = e >> lm, c = e & (m - 1);
        T v = T(0);
        if (r == c) {
            v = diag_at(g, r, r & (n - 1), r >> g.lg);
        } else {
            const int ri = r & (n - 1), rj = r >> g.lg, ci = c & (n - 1), cj = c >> g.lg;
            if (rj == cj && ci == ri + 1) v = -g.te[r];
            if (rj == cj && ci == ri - 1) v = -g.te[c];
            if (ri == ci && cj == rj + 1) v = -g.tn[r];
            if (ri == ci && cj == rj - 1) v = -g.tn[c];
        }
        A[e] = v;
        ainv[e] = (r == c) ? T(1) : T(0);
    }
    sync();
    for (int k = 0; k < m; ++k) {
        const T piv = A[k * m + k];
        sync();
        for (int c = rank(); c < m; c += size()) {
            A[k * m + c] /= piv;
            ainv[k * m + c] /= piv;
        }
        sync();
        for (int e = rank(); e < m * m; e += size()) {
            const int r = e >> (2 * g.lg), c = e & (m - 1);
            if (r == k) continue;
            const T f = A[r * m + k];   // column k is left alone until the next phase
            if (c != k) A[e] -= f * A[k * m + c];
            ainv[e] -= f * ainv[k * m + c];
        }
        sync();
        for (int r = rank(); r < m; r += size())
            if (r != k) A[r * m + k] = T(0);
        sync();
    }
}

static __device__ __forceinline__ void resident_coarse_solve(const RGrid<T>& g, const T* ainv, const Ghost<T>& d) {
    const int n = g.n, m = n * n;
    T acc = T(0);
    if (rank() < m)
        for (int c = 0; c < m; ++c) acc += ainv[rank() * m + c] * rhs_at(g, c, c & (n - 1), c >> g.lg, d);
    sync();
    if (rank() < m) g.p[rank()] = acc;
    sync();
}

static __device__ __forceinline__ void resident_rbgs(const RGrid<T>& g, const Ghost<T>& d) {
    const int n = g.n, half = n * n / 2, hn = n / 2;
    for (int color = 0; color < 2; ++color) {
        for (int h = rank(); h < half; h += size()) {
            const int j = h >> (g.lg - 1);
            const int i = 2 * (h & (hn - 1)) + ((j + color) & 1);
            const int c = j * n + i;
            T acc = rhs_at(g, c, i, j, d);
            if (i > 0) acc += g.te[c - 1] * g.p[c - 1];
            if (i < n - 1) acc += g.te[c] * g.p[c + 1];
            if (j > 0) acc += g.tn[c - n] * g.p[c - n];
            if (j < n - 1) acc += g.tn[c] * g.p[c + n];
            g.p[c] = divide_by_diag(g, acc, c, i, j);
        }
        sync();
    }
}

static __device__ __forceinline__ T resident_residual(const RGrid<T>& g, int c, int i, int j, const Ghost<T>& d) {
    const int n = g.n;
    T v = diag_at(g, c, i, j) * g.p[c];
    if (i > 0) v -= g.te[c - 1] * g.p[c - 1];
    if (i < n - 1) v -= g.te[c] * g.p[c + 1];
    if (j > 0) v -= g.tn[c - n] * g.p[c - n];
    if (j < n - 1) v -= g.tn[c] * g.p[c + n];
    return rhs_at(g, c, i, j, d) - v;
}

static __device__ __forceinline__ void resident_restrict(const RGrid<T>& f, const RGrid<T>& cg, const Ghost<T>& d) {
    const int nc = cg.n, nf = f.n;
    for (int C = rank(); C < nc * nc; C += size()) {
        const int I = C & (nc - 1), J = C >> cg.lg, i0 = 2 * I, j0 = 2 * J, c0 = j0 * nf + i0;
        const T r00 = resident_residual(f, c0, i0, j0, d);
        const T r10 = resident_residual(f, c0 + 1, i0 + 1, j0, d);
        const T r01 = resident_residual(f, c0 + nf, i0, j0 + 1, d);
        const T r11 = resident_residual(f, c0 + nf + 1, i0 + 1, j0 + 1, d);
        cg.b[C] = r00 + r10 + r01 + r11;
        cg.p[C] = T(0);
    }
    sync();
}

// Coarse value with ghosts: 2g - u across a Dirichlet edge, the edge value
// mirrored across a no-flow edge; a corner ghost takes the x rule on the y
// ghost.
template <typename U>
static __device__ __forceinline__ U ghost_x(const U* uc, int nc, int I, int J, const Ghost<U>& g) {
    if (I < 0) return U(2) * g.w - uc[J * nc];
    if (I > nc - 1) return U(2) * g.e - uc[J * nc + nc - 1];
    return uc[J * nc + I];
}
template <typename U>
static __device__ __forceinline__ U ghost(const U* uc, int nc, int I, int J, const Ghost<U>& g) {
    if (J < 0) {
        const U edge = ghost_x(uc, nc, I, 0, g);
        return g.ns ? U(2) * g.s - edge : edge;
    }
    if (J > nc - 1) {
        const U edge = ghost_x(uc, nc, I, nc - 1, g);
        return g.ns ? U(2) * g.n - edge : edge;
    }
    return ghost_x(uc, nc, I, J, g);
}

// out (+)= bilinear interpolation of uc (nc x nc) onto the 2nc x 2nc grid.
template <typename U>
static __device__ __forceinline__ void resident_prolong(const U* uc, int nc, U* out, const Ghost<U>& gd, bool add) {
    const int nf = 2 * nc, lgf = ilog2(nf);
    for (int c = rank(); c < nf * nf; c += size()) {
        const int i = c & (nf - 1), j = c >> lgf, I = i >> 1, J = j >> 1;
        const int Ix = (i & 1) ? I + 1 : I - 1;
        const int Jy = (j & 1) ? J + 1 : J - 1;
        const U v = (U(9) * ghost(uc, nc, I, J, gd) + U(3) * ghost(uc, nc, Ix, J, gd) +
                     U(3) * ghost(uc, nc, I, Jy, gd) + U(1) * ghost(uc, nc, Ix, Jy, gd)) /
                    U(16);
        out[c] = add ? out[c] + v : v;
    }
    sync();
}

// One V(nu1, nu2) cycle on grid k, iteratively: descend (smooth, restrict
// the residual), exact coarsest solve, ascend (prolong the correction,
// smooth).  The boundary data d only enter through a grid without a stored
// rhs; the corrections take zero ghost data on the same edges.
static __device__ void resident_vcycle(const RLayout<T>& L, int k, int nu1, int nu2, const Ghost<T>& d) {
    for (int l = k; l >= 1; --l) {
        for (int s = 0; s < nu1; ++s) resident_rbgs(L.g[l], d);
        resident_restrict(L.g[l], L.g[l - 1], d);
    }
    resident_coarse_solve(L.g[0], L.ainv, d);
    const Ghost<T> zero{T(0), T(0), T(0), T(0), d.ns};
    for (int l = 1; l <= k; ++l) {
        resident_prolong(L.g[l - 1].p, L.g[l - 1].n, L.g[l].p, zero, true);
        for (int s = 0; s < nu2; ++s) resident_rbgs(L.g[l], d);
    }
}

// Sum of a and b over the CTA; every thread gets the totals.
static __device__ __forceinline__ void block_sum2(double a, double b, double* red, double& A, double& B) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if (WARP) {
        A = __shfl_sync(0xffffffffu, a, 0);
        B = __shfl_sync(0xffffffffu, b, 0);
        return;
    }
    const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[warp] = a;
        red[32 + warp] = b;
    }
    sync();
    if (rank() == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < nw; ++w) {
            sa += red[w];
            sb += red[32 + w];
        }
        red[64] = sa;
        red[65] = sb;
    }
    sync();
    A = red[64];
    B = red[65];
    sync();
}

// Stage problem of grid k written into its rhs: the Dirichlet data.
static __device__ __forceinline__ void resident_stage_rhs(const RGrid<T>& g, const Ghost<T>& d) {
    for (int c = rank(); c < g.n * g.n; c += size()) {
        const int i = c & (g.n - 1), j = c >> g.lg;
        g.b[c] = dirichlet_at(g, c, i, j, d);
    }
    sync();
}

// ||r||^2 and ||rhs||^2 of the stage problem on grid k (V-cycle type).
static __device__ void stage_norms(const RGrid<T>& g, const Ghost<T>& d, double* red, double& rr, double& bb) {
    double a = 0.0, b = 0.0;
    for (int c = rank(); c < g.n * g.n; c += size()) {
        const int i = c & (g.n - 1), j = c >> g.lg;
        const double r = (double)resident_residual(g, c, i, j, d);
        const double f = (double)rhs_at(g, c, i, j, d);
        a += r * r;
        b += f * f;
    }
    block_sum2(a, b, red, rr, bb);
}

// FP64 residual of the stage problem on h into the FP32 grid's rhs (the
// correction equation), zero the correction; returns the norms.
static __device__ void ir_residual(const HGrid& h, const RGrid<T>& g, const Ghost<double>& d, double* red,
                            double& rr, double& bb) {
    const int n = h.n;
    double a = 0.0, b = 0.0;
    for (int c = rank(); c < n * n; c += size()) {
        const int i = c & (n - 1), j = c >> h.lg;
        const double tw = (i > 0) ? h.te[c - 1] : h.tw[j];
        const double ts = (j > 0) ? h.tn[c - n] : h.ts[i];
        const double f = dirichlet_at(h, c, i, j, d);
        double v = (tw + h.te[c] + ts + h.tn[c]) * h.p[c];
        if (i > 0) v -= h.te[c - 1] * h.p[c - 1];
        if (i < n - 1) v -= h.te[c] * h.p[c + 1];
        if (j > 0) v -= h.tn[c - n] * h.p[c - n];
        if (j < n - 1) v -= h.tn[c] * h.p[c + n];
        const double r = f - v;
        g.b[c] = (T)r;
        g.p[c] = T(0);
        a += r * r;
        b += f * f;
    }
    block_sum2(a, b, red, rr, bb);
}

// The QoI of Table 1 (valid in thread 0).  Case II: Q = sum_j te(n-1, j)
// (p(n-1, j) - pE), warp 0 reduces.  Case I (d.ns): u(0.5, 0.5), the mean of
// the four centre cells.
template <typename P, typename Q>
static __device__ __forceinline__ double outflux_of(const P* te, const Q* p, int n, const Ghost<double>& d) {
    const double pE = d.e;
    if (d.ns) {
        const int c = (n / 2 - 1) * n + n / 2 - 1;
        return 0.25 * (((double)p[c] + (double)p[c + 1]) + ((double)p[c + n] + (double)p[c + n + 1]));
    }
    double acc = 0.0;
    if (rank() < 32) {
        for (int j = rank(); j < n; j += 32) {
            const int c = j * n + n - 1;
            acc += (double)te[c] * ((double)p[c] - pE);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    }
    return acc;
}

// Outflux broadcast to every thread of the CTA.
template <typename P, typename Q>
static __device__ __forceinline__ double stage_outflux(const P* te, const Q* p, int n, const Ghost<double>& d,
                                                       double* red) {
    const double q = outflux_of(te, p, n, d);
    if (WARP) return __shfl_sync(0xffffffffu, q, 0);
    if (rank() == 0) red[70] = q;
    sync();
    const double out = red[70];
    sync();
    return out;
}

};

struct ResidentArgs {
    int n_fine, n0;
    size_t S;
    const double* K;
    Ghost<double> bd;   // boundary data (Table 1)
    int nu0, nu1, nu2;
    int ir;   // V-cycles between residual tests of a converged stage
    int converged, max_cycles;
    double tol, qtol;
    double *qf, *qc, *p_out;
    int32_t* status;
    double* flops;   // nullable (profiling): [0] solver flops, [1] their FP64 part, [2] model bytes
};

// Solver flops of one V(nu1, nu2) cycle from grid k down: per grid j >= 1,
// nu1 + nu2 sweeps of 10 flops a cell, residual + restriction 10, correction
// 8; the coarsest solve a dense 16 x 16 product.
__device__ __forceinline__ double vcycle_flops(int n0, int k, int nu1, int nu2) {
    double f = 2.0 * (n0 * n0) * (n0 * n0);
    for (int j = 1; j <= k; ++j) {
        const double c = (double)(n0 << j) * (n0 << j);
        f += c * (10.0 * (nu1 + nu2) + 18.0);
    }
    return f;
}

// Algorithmic bytes of the same cycle in the streaming byte model of the
// level-wise kernels (each sweep reads p, K, b and writes p: 16 B per cell in
// FP32; residual + restriction 13 B and prolongation + correction 9 B per
// fine cell; twice that in FP64), the yardstick the resident kernel's
// effective bandwidth is quoted against.
__device__ __forceinline__ double vcycle_bytes(int n0, int k, int nu1, int nu2, int ts) {
    double b = 0.0;
    for (int j = 1; j <= k; ++j) {
        const double c = (double)(n0 << j) * (n0 << j);
        b += c * (16.0 * (nu1 + nu2) + 22.0) * (ts / 4.0);
    }
    return b;
}

// Shared memory of one CTA: a layout table per group, then each group's data.
template <typename T>
__host__ __device__ inline size_t resident_slot_bytes() {
    return ((sizeof(RLayout<T>) + 15) / 16) * 16;
}

template <typename T, bool MIXED, bool WARP>
__global__ void __launch_bounds__(512, 1) k_fmg_resident(ResidentArgs a) {
    using R = Res<T, WARP>;
    extern __shared__ __align__(16) char smem[];
    const int groups = WARP ? (int)(blockDim.x >> 5) : 1;
    const int grp = WARP ? (int)(threadIdx.x >> 5) : 0;
    RLayout<T>* slot = reinterpret_cast<RLayout<T>*>(smem + grp * resident_slot_bytes<T>());
    const size_t data_bytes = resident_layout<T>(nullptr, a.n_fine, a.n0, MIXED, WARP).bytes;
    char* data = smem + groups * resident_slot_bytes<T>() + grp * data_bytes;
    if (R::rank() == 0) *slot = resident_layout<T>(data, a.n_fine, a.n0, MIXED, WARP);
    R::sync();
    const RLayout<T>& L = *slot;
    // the boundary data in the V-cycle arithmetic, and zero data on the same
    // edges for the mixed form's correction equation
    const Ghost<T> td{(T)a.bd.w, (T)a.bd.e, (T)a.bd.s, (T)a.bd.n, a.bd.ns};
    const Ghost<T> t0{T(0), T(0), T(0), T(0), a.bd.ns};
    const int m = L.m;
    const size_t stride = (size_t)gridDim.x * groups;
    for (size_t s = (size_t)blockIdx.x * groups + grp; s < a.S; s += stride) {
        const double* Kf = a.K + s * (size_t)a.n_fine * a.n_fine;
        for (int k = 0; k <= m; ++k) {
            const HGrid* h = (MIXED && k >= m - 1) ? &L.h[k - (m - 1)] : nullptr;
            R::resident_setup_grid(L.g[k], h, Kf, a.n_fine, a.bd.ns);
        }
        R::sync();
        for (int k = 0; k <= m; ++k) R::resident_setup_diag(L.g[k]);
        R::sync();
        R::resident_coarse_inverse(L.g[0], L.ainv, L.work);
        bool ok = true;
        double q_coarse = NAN, q_fine = NAN;
        double work = 0.0;   // solver flops of this sample (V-cycles and residual tests)
        double work64 = 0.0; // the FP64 part of them
        double model = 0.0;  // their algorithmic bytes (byte model of the level-wise kernels)
        constexpr int ts = (int)sizeof(T);

        // the stages giving Q^f and (where it is asked for) Q^c are refined
        // when converged; otherwise stage m - 1 only gives stage m its start
        const bool refine_c = a.converged && a.qc != nullptr;
        for (int k = 0; k <= m; ++k) {
            const RGrid<T>& g = L.g[k];
            const bool refined = a.converged && (k == m || (k == m - 1 && refine_c));
            if (k > 0) {
                if (MIXED && refined && k == m && m >= 1 && refine_c) {
                    // FP64 interpolation of the refined stage m-1 solution
                    R::resident_prolong(L.h[0].p, L.h[0].n, L.h[1].p, a.bd, false);
                } else {
                    R::resident_prolong(L.g[k - 1].p, L.g[k - 1].n, g.p, td, false);
                }
                // grid k-1 now only carries corrections of the V-cycles on grid k
                R::resident_setup_correction(L.g[k - 1], Kf, a.n_fine, a.bd.ns);
                if (k == 1) R::resident_coarse_inverse(L.g[0], L.ainv, L.work);
            }
            if (g.b) R::resident_stage_rhs(g, td);
            if (k == 0) R::resident_coarse_solve(g, L.ainv, td);
            if (!refined) {
                if (k > 0) {
                    for (int it = 0; it < a.nu0; ++it) R::resident_vcycle(L, k, a.nu1, a.nu2, td);
                    work += a.nu0 * vcycle_flops(a.n0, k, a.nu1, a.nu2);
                    model += a.nu0 * vcycle_bytes(a.n0, k, a.nu1, a.nu2, ts);
                }
            } else if (!MIXED) {
                // FP64: V-cycles on the stage problem until the residual or
                // outflux-change test passes
                double q_prev = NAN;
                for (int it = 0;; ++it) {
                    double rr, bb;
                    R::stage_norms(g, td, L.red, rr, bb);
                    work += 14.0 * g.n * g.n;
                    model += 20.0 * g.n * g.n;
                    const double q = R::stage_outflux(g.te, g.p, g.n, a.bd, L.red);
                    if (rr <= a.tol * a.tol * bb) break;
                    if (a.qtol > 0 && fabs(q - q_prev) <= a.qtol * fabs(q)) break;
                    q_prev = q;
                    if (it >= a.max_cycles) {
                        ok = false;
                        break;
                    }
                    for (int v = 0; v < a.ir; ++v) R::resident_vcycle(L, k, a.nu1, a.nu2, td);
                    work += a.ir * vcycle_flops(a.n0, k, a.nu1, a.nu2);
                    model += a.ir * vcycle_bytes(a.n0, k, a.nu1, a.nu2, ts);
                }
            } else {
                // mixed: FP64 residual -> FP32 V-cycle on the correction -> FP64 update
                const HGrid& h = L.h[k - (m - 1)];
                if (!(k == m && m >= 1 && refine_c)) {
                    for (int c = R::rank(); c < h.n * h.n; c += R::size()) h.p[c] = (double)g.p[c];
                    R::sync();
                }
                double q_prev = NAN;
                for (int it = 0;; ++it) {
                    double rr, bb;
                    R::ir_residual(h, g, a.bd, L.red, rr, bb);
                    work += 14.0 * h.n * h.n;
                    work64 += 14.0 * h.n * h.n;
                    model += 20.0 * h.n * h.n;
                    const double q = R::stage_outflux(h.te, h.p, h.n, a.bd, L.red);
                    if (rr <= a.tol * a.tol * bb) break;
                    if (a.qtol > 0 && fabs(q - q_prev) <= a.qtol * fabs(q)) break;
                    q_prev = q;
                    if (it >= a.max_cycles) {
                        ok = false;
                        break;
                    }
                    // ir FP32 V-cycles on the correction equation per FP64 residual
                    for (int v = 0; v < a.ir; ++v) R::resident_vcycle(L, k, a.nu1, a.nu2, t0);
                    work += a.ir * vcycle_flops(a.n0, k, a.nu1, a.nu2) + (double)h.n * h.n;
                    work64 += (double)h.n * h.n;
                    model += a.ir * vcycle_bytes(a.n0, k, a.nu1, a.nu2, ts);
                    for (int c = R::rank(); c < h.n * h.n; c += R::size()) h.p[c] += (double)g.p[c];
                    R::sync();
                }
            }
            // outflux of the stage (the FP64 iterate in mixed refined stages)
            if (k == m || (k == m - 1 && a.qc)) {
                double q;
                if (MIXED && refined) {
                    const HGrid& h = L.h[k - (m - 1)];
                    q = R::outflux_of(h.te, h.p, h.n, a.bd);
                } else {
                    q = R::outflux_of(g.te, g.p, g.n, a.bd);
                }
                if (k == m) q_fine = q;
                else q_coarse = q;
                R::sync();
            }
        }
        if (R::rank() == 0) {
            if (a.flops) {
                atomicAdd(a.flops, work);
                atomicAdd(a.flops + 1, MIXED ? work64 : work);
                atomicAdd(a.flops + 2, model);
            }
            a.qf[s] = q_fine;
            if (a.qc) a.qc[s] = q_coarse;
            if (a.status) a.status[s] = ok ? FM_OK : FM_ENOTCONV;
        }
        if (a.p_out) {
            const bool fine64 = MIXED && a.converged;
            double* po = a.p_out + s * (size_t)a.n_fine * a.n_fine;
            for (int c = R::rank(); c < a.n_fine * a.n_fine; c += R::size())
                po[c] = fine64 ? L.h[1].p[c] : (double)L.g[m].p[c];
        }
        R::sync();
    }
}

size_t resident_smem_bytes(int n_fine, int n0, bool mixed, bool warp) {
    return mixed ? resident_layout<float>(nullptr, n_fine, n0, true, warp).bytes
                 : resident_layout<double>(nullptr, n_fine, n0, false, warp).bytes;
}

constexpr size_t kResidentSmemMax = 227 * 1024;

// Grids up to 16 x 16 run one sample per warp (four per CTA, barriers are
// __syncwarp); larger grids one sample per CTA.
template <typename T, bool MIXED, bool WARP>
static bool launch_resident(fm_ctx* ctx, const ResidentArgs& a, cudaStream_t st) {
    const int groups = WARP ? 4 : 1;
    const size_t smem = groups * (resident_slot_bytes<T>() + resident_smem_bytes(a.n_fine, a.n0, MIXED, WARP));
    if (smem > kResidentSmemMax) return false;
    // a 32 x 32 sample on 128 threads: four CTAs per SM (shared memory
    // allows four, registers four at 128 threads); measured 1.45x the
    // samples per second of 256 threads (two CTAs per SM), the half-sweeps
    // being latency-bound
    const int threads = WARP ? 32 * groups : (a.n_fine >= 64 ? 512 : 128);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fmg_resident<T, MIXED, WARP>, threads, smem);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const size_t need = (a.S + groups - 1) / groups;
    const size_t grid = std::min<size_t>(need, (size_t)std::max(per_sm, 1) * sms);
    const double cells = (double)a.S * a.n_fine * a.n_fine;
    const int pi = prof_start(ctx, kFamResidentFmg, st);
    ResidentArgs b = a;
    b.flops = prof_counter(ctx, pi);
    k_fmg_resident<T, MIXED, WARP><<<(unsigned)grid, threads, smem, st>>>(b);
    prof_stop(ctx, pi, st, 8.0 * cells + 16.0 * a.S, 0.0);
    return true;
}

template <typename T, bool MIXED>
static bool launch_resident(fm_ctx* ctx, const ResidentArgs& a, cudaStream_t st) {
    if (a.n_fine <= 16) return launch_resident<T, MIXED, true>(ctx, a, st);
    return launch_resident<T, MIXED, false>(ctx, a, st);
}

void resident_init_attributes() {
    static std::once_flag once;
    std::call_once(once, [] {
        const int m = (int)kResidentSmemMax;
        cudaFuncSetAttribute(k_fmg_resident<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
        cudaFuncSetAttribute(k_fmg_resident<float, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
        cudaFuncSetAttribute(k_fmg_resident<double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
        cudaFuncSetAttribute(k_fmg_resident<double, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
    });
}

bool fmg_resident_launch(fm_ctx* ctx, int n_fine, int n0, size_t S, const double* d_K,
                         const fm_solve_params& prm, double* qf, double* qc, double* p_out,
                         int32_t* status, cudaStream_t st) {
    if (n0 & (n0 - 1)) return false;   // power-of-two hierarchies only (shift-and-mask indexing)
    ResidentArgs a;
    a.n_fine = n_fine;
    a.n0 = n0;
    a.S = S;
    a.K = d_K;
    const Bnd bd = bnd_of(prm);
    a.bd = Ghost<double>{bd.g[0], bd.g[1], bd.g[2], bd.g[3], bd.ns};
    a.nu0 = prm.nu0;
    a.nu1 = prm.nu1;
    a.nu2 = prm.nu2;
    a.ir = cycles_per_test(prm);
    a.converged = prm.converged;
    a.max_cycles = prm.max_cycles;
    a.tol = prm.tol;
    a.qtol = prm.qtol;
    a.qf = qf;
    a.qc = qc;
    a.p_out = p_out;
    a.status = status;
    a.flops = nullptr;
    if (prm.precision == FM_PREC_MIXED) return launch_resident<float, true>(ctx, a, st);
    return launch_resident<double, false>(ctx, a, st);
}

}  // namespace fm
