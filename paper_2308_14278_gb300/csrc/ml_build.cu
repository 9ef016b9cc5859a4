// Field set-up kernels: lens binning into the level-1 grid (§3.2 Level 1),
// the truncation bound that picks the Taylor order, the far-field Taylor
// coefficients at the level-2 nodes (§3.2 Level 2) and the per-node records
// of the mixed-precision path.
#include "ml_internal.cuh"

#include <math.h>

namespace ml {

// ---------------------------------------------------------------------------
// Lens binning: extended level-1 cell of each lens and a stable counting sort.
// ---------------------------------------------------------------------------

// Level-1 cell of lens k in the grid extended by one ring:
// ex = floor((x - rx0) / l1x) + 1 in [0, NEx), likewise ey; bucket NE for
// lenses outside the ring (far from every cell).
__global__ void k_lens_cells(Geo g, const double *__restrict__ x, const double *__restrict__ y,
                             int64_t n, int32_t *__restrict__ cell, int32_t *__restrict__ count)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double fx = floor((x[k] - g.rx0) / g.l1x) + 1.0;
    double fy = floor((y[k] - g.ry0) / g.l1y) + 1.0;
    int32_t NE = (int32_t)(g.NEx * g.NEy);
    int32_t c = NE;
    if (fx >= 0.0 && fx < (double)g.NEx && fy >= 0.0 && fy < (double)g.NEy)
        c = (int32_t)fy * (int32_t)g.NEx + (int32_t)fx;
    cell[k] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of nb bucket counts into start[0..nb] by one CTA.
__global__ void k_scan(const int32_t *__restrict__ count, int32_t *__restrict__ start, int64_t nb)
{
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int32_t v = i < nb ? count[i] : 0;
        int32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        int32_t off = carry + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (i < nb) start[i] = off + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = off + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[nb] = carry;
}

// Stable scatter by one warp: lenses are taken 32 at a time in index order;
// lanes with equal buckets get consecutive slots in lane order.
__global__ void k_scatter(const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ m, const int32_t *__restrict__ cell, int64_t n,
                          const int32_t *__restrict__ start, int64_t nb, int32_t *cursor_g,
                          double *__restrict__ sx, double *__restrict__ sy,
                          double *__restrict__ sm, int32_t *__restrict__ scell,
                          int32_t *__restrict__ perm, int use_smem)
{
    extern __shared__ int32_t cur_s[];
    int32_t *cur = use_smem ? cur_s : cursor_g;
    int lane = threadIdx.x;
    for (int64_t b = lane; b < nb; b += 32) cur[b] = start[b];
    __syncwarp();
    for (int64_t base = 0; base < n; base += 32) {
        int64_t k = base + lane;
        bool ok = k < n;
        int32_t c = ok ? cell[k] : -1;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        unsigned peers = __match_any_sync(0xffffffffu, c) & act;
        int rank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        int32_t basepos = 0;
        if (ok && lane == leader) {
            basepos = cur[c];
            cur[c] = basepos + __popc(peers);
        }
        basepos = __shfl_sync(0xffffffffu, basepos, leader < 0 ? 0 : leader);
        if (ok) {
            int32_t pos = basepos + rank;
            sx[pos] = x[k];
            sy[pos] = y[k];
            sm[pos] = m[k];
            scell[pos] = c;
            perm[pos] = (int32_t)k;
        }
        __syncwarp();
    }
}

cudaError_t launch_lens_cells(const Geo &g, const double *x, const double *y, int64_t n,
                              int32_t *cell, int32_t *count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_lens_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, x, y, n, cell, count);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *count, int32_t *start, int64_t nb, cudaStream_t s)
{
    k_scan<<<1, 1024, 0, s>>>(count, start, nb);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const double *x, const double *y, const double *m,
                           const int32_t *cell, int64_t n, const int32_t *start, int64_t nb,
                           int32_t *cursor, double *sx, double *sy, double *sm, int32_t *scell,
                           int32_t *perm, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    size_t smem = (size_t)nb * sizeof(int32_t);
    int use_smem = smem <= 96 * 1024;
    if (use_smem && smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_scatter<<<1, 32, use_smem ? smem : 0, s>>>(x, y, m, cell, n, start, nb, cursor, sx, sy, sm,
                                                 scell, perm, use_smem);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Truncation bound of the far series, per level-1 cell and Taylor order.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool is_near_cell(int32_t lc, int64_t NEx, int64_t NE, int64_t ex,
                                             int64_t ey)
{
    if (lc >= NE) return false;
    int64_t lx = lc % NEx, ly = lc / NEx;
    return (lx - ex <= 1 && ex - lx <= 1 && ly - ey <= 1 && ey - ly <= 1);
}

// bound[c * PMAX + (p - 1)] = sum_{k far} m_k rho^{p+1} / (D_k^{p+1} (D_k - rho))
// with rho the largest ray-node distance in a level-2 cell and D_k the
// distance from lens k to the box of the cell's node centres: an upper bound
// of the truncation error |sum_{n>p} c_n d^n| for every ray of the cell.
__global__ void k_p_bound(Geo g, LensTable L, double *__restrict__ bound)
{
    int64_t c = blockIdx.x;
    int64_t c1x = c % g.N1x, c1y = c / g.N1x;
    int64_t ex = c1x + 1, ey = c1y + 1, NE = g.NEx * g.NEy;
    int64_t a2x = c1x * g.l2sx, b2x = min((c1x + 1) * (int64_t)g.l2sx, g.N2x) - 1;
    int64_t a2y = c1y * g.l2sy, b2y = min((c1y + 1) * (int64_t)g.l2sy, g.N2y) - 1;
    double x0 = g.rx0 + (a2x + 0.5) * g.l2x, x1 = g.rx0 + (b2x + 0.5) * g.l2x;
    double y0 = g.ry0 + (a2y + 0.5) * g.l2y, y1 = g.ry0 + (b2y + 0.5) * g.l2y;
    double hx = 0.5 * (double)(g.n2x - 1) * g.l3x, hy = 0.5 * (double)(g.n2y - 1) * g.l3y;
    // the bound is an estimate used to pick p: FP32 is ample (the distances
    // are formed in FP64 first); rho is rounded up by 1e-6 relative
    const float rho = (float)(sqrt(hx * hx + hy * hy) * (1.0 + 1e-6));
    float acc[PMAX];
#pragma unroll
    for (int q = 0; q < PMAX; ++q) acc[q] = 0.f;
    for (int64_t k = threadIdx.x; k < L.n; k += blockDim.x) {
        if (is_near_cell(L.cell[k], g.NEx, NE, ex, ey)) continue;
        double px = L.x[k], py = L.y[k];
        float dx = (float)(px < x0 ? x0 - px : (px > x1 ? px - x1 : 0.0));
        float dy = (float)(py < y0 ? y0 - py : (py > y1 ? py - y1 : 0.0));
        float D = sqrtf(dx * dx + dy * dy) * (1.f - 1e-6f);
        if (D <= rho) {
#pragma unroll
            for (int q = 0; q < PMAX; ++q) acc[q] = INFINITY;
            continue;
        }
        float u = rho / D;
        float t = (float)L.m[k] * u / (D - rho);  // times u^{p} below, p >= 1
#pragma unroll
        for (int q = 0; q < PMAX; ++q) {
            t *= u;
            acc[q] += t;
        }
    }
    __shared__ float red[PMAX][32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
        float v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < PMAX) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += (double)red[threadIdx.x][w];
        bound[c * PMAX + threadIdx.x] = v * (1.0 + 1e-5);
    }
}

cudaError_t launch_p_bound(const Geo &g, const LensTable &L, double *bound, cudaStream_t s)
{
    int64_t ncell = g.N1x * g.N1y;
    k_p_bound<<<(unsigned)ncell, 256, 0, s>>>(g, L, bound);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Far-field Taylor coefficients at the level-2 nodes, by direct summation:
// c_n = - sum_{k far} m_k / (z_k - z_node)^{n+1},  n = 0..p.
// One thread per node; the lens loop runs in the same order for every thread,
// so lens loads are broadcast within a warp.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(128) k_coeffs_direct(Geo g, LensTable L, double *__restrict__ coef)
{
    int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nn = g.N2x * g.N2y;
    bool live = node < nn;
    int64_t nd = live ? node : 0;
    int64_t c2x = nd % g.N2x, c2y = nd / g.N2x;
    double zx = g.rx0 + ((double)c2x + 0.5) * g.l2x;
    double zy = g.ry0 + ((double)c2y + 0.5) * g.l2y;
    int64_t ex = c2x / g.l2sx + 1, ey = c2y / g.l2sy + 1, NE = g.NEx * g.NEy;
    const int p = g.p;
    double cr[PMAX + 1], ci[PMAX + 1];
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) { cr[q] = 0.0; ci[q] = 0.0; }
    for (int64_t k = 0; k < L.n; ++k) {
        if (is_near_cell(L.cell[k], g.NEx, NE, ex, ey)) continue;
        double dx = L.x[k] - zx, dy = L.y[k] - zy;
        double inv = 1.0 / (dx * dx + dy * dy);
        double wr = dx * inv, wi = -dy * inv;          // w = 1 / (z_k - z_node)
        double tr = L.m[k] * wr, ti = L.m[k] * wi;     // m w^{n+1}, n = 0
#pragma unroll
        for (int q = 0; q <= PMAX; ++q) {
            if (q > p) break;
            cr[q] -= tr;
            ci[q] -= ti;
            double nr = tr * wr - ti * wi;
            double ni = tr * wi + ti * wr;
            tr = nr;
            ti = ni;
        }
    }
    if (!live) return;
    double *out = coef + node * (int64_t)(p + 1) * 2;
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) {
        if (q > p) break;
        out[2 * q] = cr[q];
        out[2 * q + 1] = ci[q];
    }
}

cudaError_t launch_coeffs_direct(const Geo &g, const LensTable &L, double *coef64, cudaStream_t s)
{
    int64_t nn = g.N2x * g.N2y;
    k_coeffs_direct<<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(g, L, coef64);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Node records for the mixed path: the smooth part of beta at each node
// (macro term of Eq. 1, sheet term and far-field c_0, Eq. 9) in map pixel
// units, split into an integer base and an FP32 fraction, plus c_n l3x^n,
// n = 1..p, in FP32 (the far series per power of the lattice offset).
// ---------------------------------------------------------------------------

__global__ void k_node_finalize(Geo g, const double *__restrict__ coef, unsigned char *__restrict__ out)
{
    int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nn = g.N2x * g.N2y;
    if (node >= nn) return;
    int64_t c2x = node % g.N2x, c2y = node / g.N2x;
    double zx = g.rx0 + ((double)c2x + 0.5) * g.l2x;
    double zy = g.ry0 + ((double)c2y + 0.5) * g.l2y;
    const double *c = coef + node * (int64_t)(g.p + 1) * 2;
    // beta = macro(theta) + kappa_* (theta - c_sheet) - conj(F), F(z_node) = c_0
    double mx, my;
    macro64(g, zx, zy, mx, my);
    double bx = mx + sheet_kx(g) * (zx - g.sheet_cx) - c[0];
    double by = my + sheet_ky(g) * (zy - g.sheet_cy) + c[1];
    double Sx = (bx - g.mx0) / g.dpx;
    double Sy = (by - g.my0) / g.dpy;
    double fbx = floor(Sx);
    fbx = fmin(fmax(fbx, -16777216.0), 16777216.0);
    // slope of the macro and sheet terms in theta_x at the node, and the
    // per-row shift of beta_x (fold: d_x z_x + d_y z_y and d_y z_x l3y)
    const double ax = g.macro == ML_MACRO_FOLD ? g.dx * zx + g.dy * zy : 1.0 - g.kappa - g.gamma;
    const double bq = g.macro == ML_MACRO_FOLD ? g.dy * zx * g.l3y : 0.0;
    unsigned char *rec = out + node * node_stride(g.p);
    *reinterpret_cast<double *>(rec) = Sy;
    *reinterpret_cast<int *>(rec + 8) = (int)fbx;
    *reinterpret_cast<float *>(rec + 12) = (float)(Sx - fbx);
    *reinterpret_cast<float *>(rec + 16) = (float)((ax + sheet_kx(g)) * g.l3x / g.dpx);
    *reinterpret_cast<float *>(rec + 20) = (float)(bq / g.dpx);
    // c_n per power of the lattice offset u: c_n l3x^n
    float2 *cf = reinterpret_cast<float2 *>(rec + 24);
    double ln = 1.0;
    for (int q = 1; q <= g.p; ++q) {
        ln *= g.l3x;
        cf[q - 1] = make_float2((float)(c[2 * q] * ln), (float)(c[2 * q + 1] * ln));
    }
}

cudaError_t launch_node_finalize(const Geo &g, const double *coef64, unsigned char *nodes,
                                 cudaStream_t s)
{
    int64_t nn = g.N2x * g.N2y;
    k_node_finalize<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(g, coef64, nodes);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Hierarchical coefficient build.  The node coefficients c_n are the Taylor
// coefficients of f_C(z) = sum_{k far of C} m_k / (z - z_k) at the node; they
// are reached through two exact re-expansions instead of one sum per node:
//   1. boxes B of level-1 cells (about square): f_box(z) = sum_j A_j U^j,
//      U = (z - z_B)/h_B, from the lenses outside B's 3 x 3 box block;
//   2. sub-blocks s of each level-1 cell C (about square): a_j, the box
//      series shifted to z_s plus the lenses inside B's box block but outside
//      C's 3 x 3 block summed directly;
//   3. each node: c_n = h_s^-n sum_{j>=n} C(j, n) a_j e^{j-n}, e = (z_node - z_s)/h_s.
// The far set of C is exactly the lenses outside C's 3 x 3 block (a lens in
// that block is in B's box block too), so the result equals the direct sum up
// to the truncation of the two series (order HP = 32, convergence ratios
// below 0.6 by the choice of box and sub-block sizes) and FP64 rounding.
// ---------------------------------------------------------------------------

constexpr int HP = 32;               // order of the box and sub-block series
constexpr int HPARTS = 16;           // lens partitions per box (partial sums)

// Binomial coefficients C(n, k), n, k <= HP (exact in FP64), built once at
// compile time by Pascal's rule.
struct BinomTable {
    double v[(HP + 1) * (HP + 1)];
    constexpr BinomTable() : v()
    {
        for (int n = 0; n <= HP; ++n)
            for (int k = 0; k <= HP; ++k)
                v[n * (HP + 1) + k] = k > n ? 0.0 : (k == 0 || k == n ? 1.0
                                                    : v[(n - 1) * (HP + 1) + k - 1] + v[(n - 1) * (HP + 1) + k]);
    }
};
__constant__ BinomTable c_binom = BinomTable();

struct Hier {
    int64_t bxn, byn;                // level-1 cells per box side
    int64_t NBx, NBy;                // boxes across the level-1 grid
    int64_t nsx, nsy;                // sub-blocks per level-1 cell side
    double hB;                       // box scale (half-diagonal)
};

__host__ __device__ inline Hier hier_of(const Geo &g)
{
    Hier h;
    double s = fmax(fmax(g.l1x, g.l1y), sqrt((double)g.n3x * g.l3x * (double)g.n3y * g.l3y / 48.0));
    h.bxn = (int64_t)fmax(1.0, floor(s / g.l1x + 0.5));
    h.byn = (int64_t)fmax(1.0, floor(s / g.l1y + 0.5));
    h.NBx = (g.N1x + h.bxn - 1) / h.bxn;
    h.NBy = (g.N1y + h.byn - 1) / h.byn;
    double ar = g.l1x / g.l1y;
    h.nsx = ar >= 1.0 ? (int64_t)fmin((double)g.l2sx, floor(ar + 0.5)) : 1;
    h.nsy = ar < 1.0 ? (int64_t)fmin((double)g.l2sy, floor(1.0 / ar + 0.5)) : 1;
    if (h.nsx < 1) h.nsx = 1;
    if (h.nsy < 1) h.nsy = 1;
    h.hB = 0.5 * sqrt((double)(h.bxn * h.bxn) * g.l1x * g.l1x + (double)(h.byn * h.byn) * g.l1y * g.l1y);
    return h;
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Level-1 cell index of each sorted lens, unbounded (clamped to +-2^28).
__global__ void k_lens_l1(Geo g, LensTable L, int2 *__restrict__ lc)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= L.n) return;
    double fx = floor((L.x[k] - g.rx0) / g.l1x), fy = floor((L.y[k] - g.ry0) / g.l1y);
    fx = fmin(fmax(fx, -268435456.0), 268435456.0);
    fy = fmin(fmax(fy, -268435456.0), 268435456.0);
    lc[k] = make_int2((int)fx, (int)fy);
}

// Accumulate -(m/h) w^{j+1}, w = h / (z_k - z_c), j = 0..HP, into acc.
__device__ __forceinline__ void p2l_add(double m, double dx, double dy, double h,
                                        double *ar, double *ai)
{
    double inv = h / (dx * dx + dy * dy);
    double wr = dx * inv, wi = -dy * inv;
    double tr = (m / h) * wr, ti = (m / h) * wi;
#pragma unroll
    for (int j = 0; j <= HP; ++j) {
        ar[j] -= tr;
        ai[j] -= ti;
        double nr = tr * wr - ti * wi;
        double ni = tr * wi + ti * wr;
        tr = nr;
        ti = ni;
    }
}

// Sum the (HP+1) complex accumulators of a 128-thread block into out (global).
__device__ void block_sum_store(double *ar, double *ai, double *__restrict__ out, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j <= HP; ++j) {
        double vr = ar[j], vi = ai[j];
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_down_sync(0xffffffffu, vr, o);
            vi += __shfl_down_sync(0xffffffffu, vi, o);
        }
        if (lane == 0) {
            red[(wid * (HP + 1) + j) * 2] = vr;
            red[(wid * (HP + 1) + j) * 2 + 1] = vi;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= HP; j += blockDim.x) {
        double vr = 0.0, vi = 0.0;
        for (int w = 0; w < nw; ++w) {
            vr += red[(w * (HP + 1) + j) * 2];
            vi += red[(w * (HP + 1) + j) * 2 + 1];
        }
        out[2 * j] = vr;
        out[2 * j + 1] = vi;
    }
}

// 1. box series from the lenses outside the box's 3 x 3 box block; grid
// (NB, HPARTS), each block summing one partition of the lenses.
__global__ void __launch_bounds__(128) k_box_p2l(Geo g, LensTable L, const int2 *__restrict__ lc,
                                                 Hier h, double *__restrict__ part)
{
    __shared__ double red[4 * (HP + 1) * 2];
    const int64_t b = blockIdx.x, Bx = b % h.NBx, By = b / h.NBx;
    const double zx = g.rx0 + ((double)Bx + 0.5) * (double)h.bxn * g.l1x;
    const double zy = g.ry0 + ((double)By + 0.5) * (double)h.byn * g.l1y;
    double ar[HP + 1], ai[HP + 1];
#pragma unroll
    for (int j = 0; j <= HP; ++j) { ar[j] = 0.0; ai[j] = 0.0; }
    const int64_t k0 = L.n * blockIdx.y / HPARTS, k1 = L.n * (blockIdx.y + 1) / HPARTS;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        int2 c = lc[k];
        int64_t lbx = floor_div(c.x, h.bxn), lby = floor_div(c.y, h.byn);
        if (lbx - Bx <= 1 && Bx - lbx <= 1 && lby - By <= 1 && By - lby <= 1) continue;
        p2l_add(L.m[k], L.x[k] - zx, L.y[k] - zy, h.hB, ar, ai);
    }
    block_sum_store(ar, ai, part + (b * HPARTS + blockIdx.y) * (HP + 1) * 2, red);
}

// 2. sub-block series: box series shifted to z_s plus the direct sum of the
// lenses in the box block but outside the cell's 3 x 3 block.
__global__ void __launch_bounds__(128) k_sub_p2l(Geo g, LensTable L, const int2 *__restrict__ lc,
                                                 Hier h, const double *__restrict__ part,
                                                 double *__restrict__ sub)
{
    __shared__ double red[4 * (HP + 1) * 2];
    __shared__ double A[(HP + 1) * 2];
    __shared__ double binom[(HP + 1) * (HP + 1)];
    const int64_t s = blockIdx.x;
    const int64_t nsub = h.nsx * h.nsy;
    const int64_t cell = s / nsub, sb = s % nsub;
    const int64_t cx = cell % g.N1x, cy = cell / g.N1x;
    const int64_t sa = sb % h.nsx, sbb = sb / h.nsx;
    // node columns [ua, ub) and rows [va, vb) of the sub-block inside the cell
    const int64_t ua = (sa * g.l2sx + h.nsx - 1) / h.nsx, ub = ((sa + 1) * g.l2sx + h.nsx - 1) / h.nsx;
    const int64_t va = (sbb * g.l2sy + h.nsy - 1) / h.nsy, vb = ((sbb + 1) * g.l2sy + h.nsy - 1) / h.nsy;
    const double zx = g.rx0 + (double)cx * g.l1x + 0.5 * (double)(ua + ub) * g.l2x;
    const double zy = g.ry0 + (double)cy * g.l1y + 0.5 * (double)(va + vb) * g.l2y;
    const double hs = 0.5 * sqrt((double)((ub - ua) * (ub - ua)) * g.l2x * g.l2x +
                                 (double)((vb - va) * (vb - va)) * g.l2y * g.l2y);
    const int64_t Bx = cx / h.bxn, By = cy / h.byn;
    double ar[HP + 1], ai[HP + 1];
#pragma unroll
    for (int j = 0; j <= HP; ++j) { ar[j] = 0.0; ai[j] = 0.0; }
    // lenses of the box block (3 x 3 boxes) outside the cell's 3 x 3 block.
    // Cells of the binning grid (the lattice and its ring) are contiguous
    // runs of the sorted table, one per row; lenses beyond the ring (the last
    // bucket) are scanned only when the box block reaches past the ring.
    const int64_t xlo = (Bx - 1) * h.bxn, xhi = (Bx + 2) * h.bxn - 1;
    const int64_t ylo = (By - 1) * h.byn, yhi = (By + 2) * h.byn - 1;
    const int64_t NE = g.NEx * g.NEy;
    const int64_t rx0 = max(xlo, (int64_t)-1), rx1 = min(xhi, g.N1x);
    const int64_t ry0 = max(ylo, (int64_t)-1), ry1 = min(yhi, g.N1y);
    for (int64_t ry = ry0; ry <= ry1 && rx0 <= rx1; ++ry) {
        const int64_t b0 = (ry + 1) * g.NEx + (rx0 + 1), b1 = (ry + 1) * g.NEx + (rx1 + 1);
        const int64_t k0 = L.start[b0], k1 = L.start[b1 + 1];
        const bool near_row = ry - cy <= 1 && cy - ry <= 1;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            if (near_row) {
                const int64_t lx = lc[k].x;
                if (lx - cx <= 1 && cx - lx <= 1) continue;
            }
            p2l_add(L.m[k], L.x[k] - zx, L.y[k] - zy, hs, ar, ai);
        }
    }
    if (xlo < -1 || xhi > g.N1x || ylo < -1 || yhi > g.N1y) {
        for (int64_t k = L.start[NE] + threadIdx.x; k < L.start[NE + 1]; k += blockDim.x) {
            const int2 c = lc[k];
            const int64_t lbx = floor_div(c.x, h.bxn), lby = floor_div(c.y, h.byn);
            const bool in_box_block = lbx - Bx <= 1 && Bx - lbx <= 1 && lby - By <= 1 && By - lby <= 1;
            if (!in_box_block) continue;
            p2l_add(L.m[k], L.x[k] - zx, L.y[k] - zy, hs, ar, ai);
        }
    }
    // box series of this cell's box: sum of the partitions (fixed order)
    const int64_t b = By * h.NBx + Bx;
    for (int j = threadIdx.x; j <= HP; j += blockDim.x) {
        double vr = 0.0, vi = 0.0;
        for (int q = 0; q < HPARTS; ++q) {
            vr += part[((b * HPARTS + q) * (HP + 1) + j) * 2];
            vi += part[((b * HPARTS + q) * (HP + 1) + j) * 2 + 1];
        }
        A[2 * j] = vr;
        A[2 * j + 1] = vi;
    }
    for (int t = threadIdx.x; t < (HP + 1) * (HP + 1); t += blockDim.x) binom[t] = c_binom.v[t];
    __syncthreads();
    block_sum_store(ar, ai, sub + s * (HP + 1) * 2, red);
    __syncthreads();
    // shift the box series to z_s: coefficient of V^j, V = (z - z_s)/hs, is
    // rho^j sum_{i>=j} C(i, j) A_i d^{i-j},  d = (z_s - z_B)/h_B, rho = hs/h_B
    const double zBx = g.rx0 + ((double)Bx + 0.5) * (double)h.bxn * g.l1x;
    const double zBy = g.ry0 + ((double)By + 0.5) * (double)h.byn * g.l1y;
    const double dr = (zx - zBx) / h.hB, di = (zy - zBy) / h.hB, rho = hs / h.hB;
    for (int j = threadIdx.x; j <= HP; j += blockDim.x) {
        double vr = 0.0, vi = 0.0;
        for (int i = HP; i >= j; --i) {      // Horner in d
            double c = binom[i * (HP + 1) + j];
            double nr = vr * dr - vi * di + c * A[2 * i];
            double ni = vr * di + vi * dr + c * A[2 * i + 1];
            vr = nr;
            vi = ni;
        }
        double sc = pow(rho, (double)j);
        sub[(s * (HP + 1) + j) * 2] += vr * sc;
        sub[(s * (HP + 1) + j) * 2 + 1] += vi * sc;
    }
}

// 3. node coefficients from the sub-block series.
__global__ void __launch_bounds__(128) k_node_shift(Geo g, Hier h, const double *__restrict__ sub,
                                                   double *__restrict__ coef)
{
    // node-uniform loop indices: the binomials come from the constant cache
    const double *binom = c_binom.v;
    int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= g.N2x * g.N2y) return;
    int64_t c2x = node % g.N2x, c2y = node / g.N2x;
    int64_t cx = c2x / g.l2sx, cy = c2y / g.l2sy;
    int64_t u = c2x - cx * g.l2sx, v = c2y - cy * g.l2sy;
    int64_t sa = u * h.nsx / g.l2sx, sbb = v * h.nsy / g.l2sy;
    int64_t ua = (sa * g.l2sx + h.nsx - 1) / h.nsx, ub = ((sa + 1) * g.l2sx + h.nsx - 1) / h.nsx;
    int64_t va = (sbb * g.l2sy + h.nsy - 1) / h.nsy, vb = ((sbb + 1) * g.l2sy + h.nsy - 1) / h.nsy;
    double hs = 0.5 * sqrt((double)((ub - ua) * (ub - ua)) * g.l2x * g.l2x +
                           (double)((vb - va) * (vb - va)) * g.l2y * g.l2y);
    // e = (z_node - z_s)/hs
    double er = ((double)u + 0.5 - 0.5 * (double)(ua + ub)) * g.l2x / hs;
    double ei = ((double)v + 0.5 - 0.5 * (double)(va + vb)) * g.l2y / hs;
    const int64_t s = (cy * g.N1x + cx) * h.nsx * h.nsy + sbb * h.nsx + sa;
    const double *a = sub + s * (HP + 1) * 2;
    double *out = coef + node * (int64_t)(g.p + 1) * 2;
    // The mixed mode keeps c_1..c_p in FP32 (node records), so they are summed
    // in FP32 there: the shifted series decays (ratio < 0.6), no term cancels
    // far below the sum.  c_0, the node's far deflection, stays FP64; the FP64
    // near/far mode takes every order in FP64.
    const bool fp32_tail = g.precision == ML_PREC_MIXED;
    double hn = 1.0;
    for (int n = 0; n <= g.p; ++n) {
        if (n > 0 && fp32_tail) {
            const float erf = (float)er, eif = (float)ei;
            float vr = 0.f, vi = 0.f;
            for (int j = HP; j >= n; --j) {
                const float c = (float)binom[j * (HP + 1) + n];
                const float nr = __fmaf_rn(vr, erf, __fmaf_rn(-vi, eif, c * (float)a[2 * j]));
                const float ni = __fmaf_rn(vr, eif, __fmaf_rn(vi, erf, c * (float)a[2 * j + 1]));
                vr = nr;
                vi = ni;
            }
            out[2 * n] = (double)vr / hn;
            out[2 * n + 1] = (double)vi / hn;
        } else {
            double vr = 0.0, vi = 0.0;
            for (int j = HP; j >= n; --j) {
                double c = binom[j * (HP + 1) + n];
                double nr = vr * er - vi * ei + c * a[2 * j];
                double ni = vr * ei + vi * er + c * a[2 * j + 1];
                vr = nr;
                vi = ni;
            }
            out[2 * n] = vr / hn;
            out[2 * n + 1] = vi / hn;
        }
        hn *= hs;
    }
}

size_t hier_scratch_doubles(const Geo &g)
{
    Hier h = hier_of(g);
    size_t nb = (size_t)(h.NBx * h.NBy), ns = (size_t)(g.N1x * g.N1y * h.nsx * h.nsy);
    return (nb * HPARTS + ns) * (HP + 1) * 2;
}

cudaError_t launch_coeffs_hier(const Geo &g, const LensTable &L, double *coef64, double *scratch,
                               size_t scratch_doubles, cudaStream_t s)
{
    Hier h = hier_of(g);
    if (scratch_doubles < hier_scratch_doubles(g)) return cudaErrorInvalidValue;
    size_t nb = (size_t)(h.NBx * h.NBy), ns = (size_t)(g.N1x * g.N1y * h.nsx * h.nsy);
    double *part = scratch;
    double *sub = scratch + nb * HPARTS * (HP + 1) * 2;
    int2 *lc = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&lc, sizeof(int2) * (size_t)(L.n > 0 ? L.n : 1), s);
    if (e != cudaSuccess) return e;
    if (L.n > 0) k_lens_l1<<<(unsigned)((L.n + 255) / 256), 256, 0, s>>>(g, L, lc);
    dim3 gb((unsigned)nb, HPARTS);
    k_box_p2l<<<gb, 128, 0, s>>>(g, L, lc, h, part);
    k_sub_p2l<<<(unsigned)ns, 128, 0, s>>>(g, L, lc, h, part, sub);
    int64_t nn = g.N2x * g.N2y;
    k_node_shift<<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(g, h, sub, coef64);
    e = cudaGetLastError();
    cudaFreeAsync(lc, s);
    return e;
}

// Convergence ratios of the two series (for checks): largest |z - z_c| / min
// distance to a lens of the series' set, over boxes and sub-blocks.
void hier_ratios(const Geo &g, double *box_ratio, double *sub_ratio)
{
    Hier h = hier_of(g);
    double bw = (double)h.bxn * g.l1x, bh = (double)h.byn * g.l1y;
    double rb = h.hB + 0.5 * sqrt(g.l2x * g.l2x + g.l2y * g.l2y);
    *box_ratio = rb / (1.5 * fmin(bw, bh));
    double sw = ceil((double)g.l2sx / h.nsx) * g.l2x, sh = ceil((double)g.l2sy / h.nsy) * g.l2y;
    double rs = 0.5 * sqrt(sw * sw + sh * sh) + 0.5 * sqrt(g.l2x * g.l2x + g.l2y * g.l2y);
    double dmin = fmin(g.l1x + 0.5 * (g.l1x - sw), g.l1y + 0.5 * (g.l1y - sh));
    *sub_ratio = rs / dmin;
}

}  // namespace ml
