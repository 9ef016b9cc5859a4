// Field set-up kernels: lens binning into the level-1 grid (§3.2 Level 1),
// the truncation bound that picks the Taylor order, the far-field Taylor
// coefficients at the level-2 nodes (§3.2 Level 2) and the per-node records
// of the mixed-precision path.
#include "ml_internal.cuh"
#include "ml_alloc.h"

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

// Exclusive scan of nb bucket counts into start[0..nb] by the calling CTA
// (start[nb] = the total).  count and start may be the same array.
__device__ void cta_exclusive_scan(const int32_t *count, int32_t *start, int64_t nb)
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
    __syncthreads();
}

__global__ void k_scan(const int32_t *__restrict__ count, int32_t *__restrict__ start, int64_t nb)
{
    cta_exclusive_scan(count, start, nb);
}

// Stable counting-sort placement by one CTA: item k (of [0, n)) with bucket
// key(k) >= 0 goes to slot start[key] + (number of earlier items with that
// key); key < 0 items are skipped.  Warp w takes a contiguous chunk of the
// items; pass 1 counts each warp's items per bucket into its row of cnt
// (W x nb), pass 2 turns the rows into each warp's first slot per bucket (warp
// order), pass 3 walks the chunk again and places 32 items at a time, equal
// keys in lane order.  With start == nullptr the bucket starts are computed
// here into ostart[0..nb].
constexpr int SCAT_THREADS = 1024;

template <class Key, class Emit>
__device__ void cta_stable_scatter(const Key &key, int64_t n, int64_t nb, const int32_t *start,
                                   int32_t *ostart, int32_t *cnt, const Emit &emit)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int64_t chunk = (n + W - 1) / W;
    const int64_t kb = min(n, w * chunk), ke = min(n, kb + chunk);
    int32_t *my = cnt + w * nb;
    for (int64_t b = lane; b < nb; b += 32) my[b] = 0;
    __syncwarp();
    for (int64_t base = kb; base < ke; base += 32) {
        const int64_t k = base + lane;
        const int32_t c = k < ke ? key(k) : -1;
        const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
        const unsigned peers = __match_any_sync(0xffffffffu, c) & act;
        if (c >= 0 && lane == __ffs(peers) - 1) my[c] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (start == nullptr) {
        for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
            int32_t t = 0;
            for (int q = 0; q < W; ++q) t += cnt[q * nb + b];
            ostart[b] = t;
        }
        __syncthreads();
        cta_exclusive_scan(ostart, ostart, nb);
        start = ostart;
    }
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
        int32_t run = start[b];
        for (int q = 0; q < W; ++q) {
            const int32_t t = cnt[q * nb + b];
            cnt[q * nb + b] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int64_t base = kb; base < ke; base += 32) {
        const int64_t k = base + lane;
        const int32_t c = k < ke ? key(k) : -1;
        const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
        const unsigned peers = __match_any_sync(0xffffffffu, c) & act;
        const int leader = __ffs(peers) - 1;
        int32_t pos0 = 0;
        if (c >= 0 && lane == leader) {
            pos0 = my[c];
            my[c] = pos0 + __popc(peers);
        }
        pos0 = __shfl_sync(0xffffffffu, pos0, leader < 0 ? 0 : leader);
        if (c >= 0) emit(k, pos0 + __popc(peers & ((1u << lane) - 1u)));
        __syncwarp();
    }
}

__device__ __forceinline__ void split_f32(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

struct CellKey {
    const int32_t *cell;
    __device__ int32_t operator()(int64_t k) const { return cell[k]; }
};

// The sorted lens table: lenses by extended level-1 cell, stable in input order.
__global__ void __launch_bounds__(SCAT_THREADS) k_scatter(const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ m, const int32_t *__restrict__ cell, int64_t n,
                          const int32_t *__restrict__ start, int64_t nb, int32_t *cnt,
                          double *__restrict__ sx, double *__restrict__ sy,
                          double *__restrict__ sm, int32_t *__restrict__ scell,
                          int32_t *__restrict__ perm, float *__restrict__ f32)
{
    auto emit = [&](int64_t k, int32_t pos) {
        const double xv = x[k], yv = y[k], mv = m[k];
        sx[pos] = xv;
        sy[pos] = yv;
        sm[pos] = mv;
        scell[pos] = cell[k];
        perm[pos] = (int32_t)k;
        split_f32(xv, f32[pos], f32[n + pos]);
        split_f32(yv, f32[2 * n + pos], f32[3 * n + pos]);
        f32[4 * n + pos] = (float)mv;
    };
    cta_stable_scatter(CellKey{cell}, n, nb, start, nullptr, cnt, emit);
}

// FP32 copies of unsorted lenses (the autotuner's bound evaluations).
__global__ void k_split_f32(const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ m, int64_t n, float *__restrict__ f32)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    split_f32(x[k], f32[k], f32[n + k]);
    split_f32(y[k], f32[2 * n + k], f32[3 * n + k]);
    f32[4 * n + k] = (float)m[k];
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
                           double *sx, double *sy, double *sm, int32_t *scell, int32_t *perm,
                           float *f32, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int32_t *cnt = nullptr;
    cudaError_t e = ml_malloc_async((void **)&cnt, sizeof(int32_t) * (size_t)(SCAT_THREADS / 32) * (size_t)nb, s);
    if (e != cudaSuccess) return e;
    k_scatter<<<1, SCAT_THREADS, 0, s>>>(x, y, m, cell, n, start, nb, cnt, sx, sy, sm, scell, perm, f32);
    e = cudaGetLastError();
    cudaFreeAsync(cnt, s);
    return e;
}

cudaError_t launch_split_f32(const double *x, const double *y, const double *m, int64_t n,
                             float *f32, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_split_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, m, n, f32);
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

// Approximate square root and reciprocal (PTX sqrt.approx / rcp.approx,
// relative error below 2^-23 for the normal inputs met here).
__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Distance from a lens (hi + lo coordinates) to the interval [a, b] (hi + lo
// ends) along one axis, in FP32: each hi difference is rounded once (relative
// 2^-24), the lo terms are below 2^-24 of the coordinates.
__device__ __forceinline__ float gap_hilo(float ph, float pl, float ah, float al, float bh, float bl)
{
    const float below = __fadd_rn(__fsub_rn(ah, ph), __fsub_rn(al, pl));
    const float above = __fadd_rn(__fsub_rn(ph, bh), __fsub_rn(pl, bl));
    return fmaxf(0.f, fmaxf(below, above));
}

// bound[c * PMAX + (p - 1)] = sum_{k far} m_k rho^{p+1} / (D_k^{p+1} (D_k - rho))
// with rho the largest ray-node distance in a level-2 cell and D_k the
// distance from lens k to the box of the cell's node centres: an upper bound
// of the truncation error |sum_{n>p} c_n d^n| for every ray of the cell.
// It only picks p, so it runs in FP32 on hi + lo lens coordinates: D is
// rounded down by 1e-6 relative (its FP32 error is below 4e-7), rho up by
// 1e-6, and the sum up by 1e-5 (rounding of the powers and the sums).  The
// near lenses are the cell's 3 x 3 block: three runs of extended cell ids.
// PB_CELLS consecutive level-1 cells per block: each lens record is read once
// for all of them (one lens table pass per block).
#ifndef ML_PB_CELLS
#define ML_PB_CELLS 2
#endif
#ifndef ML_PB_THREADS
#define ML_PB_THREADS 128
#endif
constexpr int PB_CELLS = ML_PB_CELLS;

__global__ void __launch_bounds__(ML_PB_THREADS) k_p_bound(Geo g, LensTable L, double *__restrict__ bound)
{
    const int64_t ncell = g.N1x * g.N1y;
    const int64_t cbase = (int64_t)blockIdx.x * PB_CELLS;
    const double hx = 0.5 * (double)(g.n2x - 1) * g.l3x, hy = 0.5 * (double)(g.n2y - 1) * g.l3y;
    const float rho = (float)(sqrt(hx * hx + hy * hy) * (1.0 + 1e-6));
    float x0h[PB_CELLS], x0l[PB_CELLS], x1h[PB_CELLS], x1l[PB_CELLS];
    float y0h[PB_CELLS], y0l[PB_CELLS], y1h[PB_CELLS], y1l[PB_CELLS];
    int32_t n0[PB_CELLS];
    const int32_t nstep = (int32_t)g.NEx;
#pragma unroll
    for (int i = 0; i < PB_CELLS; ++i) {
        const int64_t c = min(cbase + i, ncell - 1);
        const int64_t c1x = c % g.N1x, c1y = c / g.N1x;
        const int64_t a2x = c1x * g.l2sx, b2x = min((c1x + 1) * (int64_t)g.l2sx, g.N2x) - 1;
        const int64_t a2y = c1y * g.l2sy, b2y = min((c1y + 1) * (int64_t)g.l2sy, g.N2y) - 1;
        const double x0 = g.rx0 + (a2x + 0.5) * g.l2x, x1 = g.rx0 + (b2x + 0.5) * g.l2x;
        const double y0 = g.ry0 + (a2y + 0.5) * g.l2y, y1 = g.ry0 + (b2y + 0.5) * g.l2y;
        x0h[i] = (float)x0; x0l[i] = (float)(x0 - (double)x0h[i]);
        x1h[i] = (float)x1; x1l[i] = (float)(x1 - (double)x1h[i]);
        y0h[i] = (float)y0; y0l[i] = (float)(y0 - (double)y0h[i]);
        y1h[i] = (float)y1; y1l[i] = (float)(y1 - (double)y1h[i]);
        // extended ids of the near block: rows c1y..c1y+2, columns c1x..c1x+2
        n0[i] = (int32_t)(c1y * g.NEx + c1x);
    }
    float acc[PB_CELLS][PMAX];
#pragma unroll
    for (int i = 0; i < PB_CELLS; ++i)
#pragma unroll
        for (int q = 0; q < PMAX; ++q) acc[i][q] = 0.f;
    for (int64_t k = threadIdx.x; k < L.n; k += blockDim.x) {
        const int32_t cell = L.cell[k];
        const float xh = L.xh[k], xl = L.xl[k], yh = L.yh[k], yl = L.yl[k], mf = L.mf[k];
#pragma unroll
        for (int i = 0; i < PB_CELLS; ++i) {
            const int32_t lc = cell - n0[i];
            if ((unsigned)lc < 3u || (unsigned)(lc - nstep) < 3u || (unsigned)(lc - 2 * nstep) < 3u) continue;
            const float dx = gap_hilo(xh, xl, x0h[i], x0l[i], x1h[i], x1l[i]);
            const float dy = gap_hilo(yh, yl, y0h[i], y0l[i], y1h[i], y1l[i]);
            const float D = __fmul_rn(sqrt_approx(__fmaf_rn(dx, dx, __fmul_rn(dy, dy))), 1.f - 1e-6f);
            if (D <= rho) {
#pragma unroll
                for (int q = 0; q < PMAX; ++q) acc[i][q] = INFINITY;
                continue;
            }
            const float u = __fmul_rn(rho, rcp_approx(D));
            float t = __fmul_rn(__fmul_rn(mf, u), rcp_approx(__fsub_rn(D, rho)));  // times u^{p} below
#pragma unroll
            for (int q = 0; q < PMAX; ++q) {
                t = __fmul_rn(t, u);
                acc[i][q] = __fadd_rn(acc[i][q], t);
            }
        }
    }
    __shared__ float red[PB_CELLS][PMAX][ML_PB_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < PB_CELLS; ++i)
#pragma unroll
        for (int q = 0; q < PMAX; ++q) {
            float v = acc[i][q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[i][q][wid] = v;
        }
    __syncthreads();
    if (threadIdx.x < PB_CELLS * PMAX) {
        const int i = threadIdx.x / PMAX, q = threadIdx.x % PMAX;
        if (cbase + i < ncell) {
            double v = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += (double)red[i][q][w];
            bound[(cbase + i) * PMAX + q] = v * (1.0 + 1e-5);
        }
    }
}

cudaError_t launch_p_bound(const Geo &g, const LensTable &L, double *bound, cudaStream_t s)
{
    int64_t ncell = g.N1x * g.N1y;
    k_p_bound<<<(unsigned)((ncell + PB_CELLS - 1) / PB_CELLS), ML_PB_THREADS, 0, s>>>(g, L, bound);
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
    double fbx = floor(Sx), fby = floor(Sy);
    fbx = fmin(fmax(fbx, -16777216.0), 16777216.0);
    fby = fmin(fmax(fby, -16777216.0), 16777216.0);
    // slope of the macro and sheet terms in theta_x at the node, and the
    // per-row shift of beta_x (fold: d_x z_x + d_y z_y and d_y z_x l3y)
    const double ax = g.macro == ML_MACRO_FOLD ? g.dx * zx + g.dy * zy : 1.0 - g.kappa - g.gamma;
    const double bq = g.macro == ML_MACRO_FOLD ? g.dy * zx * g.l3y : 0.0;
    unsigned char *rec = out + node * node_stride(g.p);
    *reinterpret_cast<int *>(rec) = (int)fby;
    *reinterpret_cast<float *>(rec + 4) = (float)(Sy - fby);
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
// The same in global memory, for loops whose lanes read different entries
// (consecutive lanes, consecutive addresses: coalesced, cached).
__device__ BinomTable g_binom = BinomTable();

// The same rounded to FP32, for the FP32 tail orders of the node shift.
struct BinomTableF {
    float v[(HP + 1) * (HP + 1)];
    constexpr BinomTableF() : v()
    {
        BinomTable b;
        for (int i = 0; i < (HP + 1) * (HP + 1); ++i) v[i] = (float)b.v[i];
    }
};
__constant__ BinomTableF c_binomf = BinomTableF();

struct Hier {
    int64_t bxn, byn;                // level-1 cells per box side
    int64_t NBx, NBy;                // boxes across the level-1 grid
    int64_t nsx, nsy;                // sub-blocks per level-1 cell side
    double hB;                       // box scale (half-diagonal)
};

// Box size: the box series costs (boxes) x (lenses) terms and the sub-block
// series (sub-blocks) x (lenses of a 3 x 3 box block) terms; for lenses
// spread over the lattice the sum is smallest near 3 sqrt(sub-blocks) boxes
// (at least 48), and a box is at least one level-1 cell each way.
__host__ __device__ inline Hier hier_of(const Geo &g)
{
    Hier h;
    double ar = g.l1x / g.l1y;
    h.nsx = ar >= 1.0 ? (int64_t)fmin((double)g.l2sx, floor(ar + 0.5)) : 1;
    h.nsy = ar < 1.0 ? (int64_t)fmin((double)g.l2sy, floor(1.0 / ar + 0.5)) : 1;
    if (h.nsx < 1) h.nsx = 1;
    if (h.nsy < 1) h.nsy = 1;
    const double nsub = (double)g.N1x * (double)g.N1y * (double)(h.nsx * h.nsy);
    const double nbox = fmax(48.0, 3.0 * sqrt(nsub));
    double s = fmax(fmax(g.l1x, g.l1y), sqrt((double)g.n3x * g.l3x * (double)g.n3y * g.l3y / nbox));
    h.bxn = (int64_t)fmax(1.0, floor(s / g.l1x + 0.5));
    h.byn = (int64_t)fmax(1.0, floor(s / g.l1y + 0.5));
    h.NBx = (g.N1x + h.bxn - 1) / h.bxn;
    h.NBy = (g.N1y + h.byn - 1) / h.byn;
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

// Accumulate -(m/h) w^{j+1}, w = h / (z_k - z_c), into acc for j = 0..J,
// where J ends the lens's series once |w|^{J+1} < 2^-52: the omitted terms
// add up to less than 2^-52 (m/h) |w| / (1 - |w|), the rounding level of the
// lens's own leading term (|w| < 0.6 for every lens of a series set).  With
// |w|^2 = h * inv the condition is J + 1 >= 72.09 / -ln|w|^2; 74 covers the
// FP32 logarithm.  ih = 1/h.
__device__ __forceinline__ void p2l_add(double m, double dx, double dy, double h, double ih,
                                        double *ar, double *ai)
{
    double inv = h / (dx * dx + dy * dy);
    double wr = dx * inv, wi = -dy * inv;
    const float lw = __logf((float)(h * inv));
    const int J = lw < -74.0f / (float)(HP + 1) ? (int)(-74.0f / lw) : HP;
    double tr = (m * ih) * wr, ti = (m * ih) * wi;
#pragma unroll
    for (int j = 0; j <= HP; ++j) {
        if (j > J) break;
        ar[j] -= tr;
        ai[j] -= ti;
        double nr = tr * wr - ti * wi;
        double ni = tr * wi + ti * wr;
        tr = nr;
        ti = ni;
    }
}

// Sum the (HP+1) complex accumulators over a warp's lanes.  Orders 0..31
// (64 values) go through a reduce-scatter: at each of five steps a lane keeps
// the half of its values that its lane bit selects, sends the other half to
// its partner and adds what it receives, so that lane l ends with the warp's
// sums of order l (about 64 additions per lane instead of 320 for a shuffle
// tree per value), returned in (sr, si); order HP takes a shuffle tree and
// every lane gets it in (xr, xi).
static_assert(HP == 32, "warp_sum_orders' reduce-scatter assumes 33 orders");
__device__ __forceinline__ void warp_sum_orders(const double *ar, const double *ai, double &sr, double &si,
                                                double &xr, double &xi)
{
    const int lane = threadIdx.x & 31;
    double v[64];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        v[2 * j] = ar[j];
        v[2 * j + 1] = ai[j];
    }
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int o = 16 >> st, half = 32 >> st;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double lo = v[i], hi = v[i + half];
            const double send = upper ? lo : hi;
            const double keep = upper ? hi : lo;
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    sr = v[0];
    si = v[1];
    xr = ar[HP];
    xi = ai[HP];
    for (int o = 16; o > 0; o >>= 1) {
        xr += __shfl_xor_sync(0xffffffffu, xr, o);
        xi += __shfl_xor_sync(0xffffffffu, xi, o);
    }
}

// Sum the (HP+1) complex accumulators of a 128-thread block into out
// (global) in a fixed order: each warp's sums (warp_sum_orders), then the
// warps' sums added in warp order.
__device__ void block_sum_store(double *ar, double *ai, double *__restrict__ out, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double sr, si, xr, xi;
    warp_sum_orders(ar, ai, sr, si, xr, xi);
    red[(wid * (HP + 1) + lane) * 2] = sr;
    red[(wid * (HP + 1) + lane) * 2 + 1] = si;
    if (lane == 0) {
        red[(wid * (HP + 1) + HP) * 2] = xr;
        red[(wid * (HP + 1) + HP) * 2 + 1] = xi;
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

// Lenses outside the binning ring (the last bucket of the sorted table)
// that lie in some box block: a CSR by box over the box grid extended by one
// box on each side, stable in table order, so that a sub-block reads just
// its box block's outer lenses (three runs of bins).
struct OuterKey {
    const int2 *lc;
    Hier h;
    int64_t k0;
    __device__ int32_t operator()(int64_t i) const
    {
        const int2 c = lc[k0 + i];
        const int64_t bx = floor_div(c.x, h.bxn), by = floor_div(c.y, h.byn);
        if (bx < -1 || bx > h.NBx || by < -1 || by > h.NBy) return -1;
        return (int32_t)((by + 1) * (h.NBx + 2) + (bx + 1));
    }
};

__global__ void __launch_bounds__(SCAT_THREADS) k_outer_csr(const int2 *__restrict__ lc, const int32_t *__restrict__ start,
                                                            int64_t NE, Hier h, int32_t *cnt, int32_t *ostart,
                                                            int32_t *oidx)
{
    const int64_t k0 = start[NE], n = start[NE + 1] - k0;
    const int64_t nb = (h.NBx + 2) * (h.NBy + 2);
    auto emit = [&](int64_t i, int32_t pos) { oidx[pos] = (int32_t)(k0 + i); };
    cta_stable_scatter(OuterKey{lc, h, k0}, n, nb, nullptr, ostart, cnt, emit);
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
    const double ihB = 1.0 / h.hB;
    double ar[HP + 1], ai[HP + 1];
#pragma unroll
    for (int j = 0; j <= HP; ++j) { ar[j] = 0.0; ai[j] = 0.0; }
    const int64_t k0 = L.n * blockIdx.y / HPARTS, k1 = L.n * (blockIdx.y + 1) / HPARTS;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        int2 c = lc[k];
        int64_t lbx = floor_div(c.x, h.bxn), lby = floor_div(c.y, h.byn);
        if (lbx - Bx <= 1 && Bx - lbx <= 1 && lby - By <= 1 && By - lby <= 1) continue;
        p2l_add(L.m[k], L.x[k] - zx, L.y[k] - zy, h.hB, ihB, ar, ai);
    }
    block_sum_store(ar, ai, part + (b * HPARTS + blockIdx.y) * (HP + 1) * 2, red);
}

// 2. sub-block series: box series shifted to z_s plus the direct sum of the
// lenses in the box block but outside the cell's 3 x 3 block.  One warp per
// sub-block (a sub-block sums a few hundred lenses at most, and its fixed
// work, the shift, is one order per lane), SUB_WARPS sub-blocks per block.
constexpr int SUB_WARPS = 4;

__global__ void __launch_bounds__(32 * SUB_WARPS, 3) k_sub_p2l(Geo g, LensTable L, const int2 *__restrict__ lc,
                                                             Hier h, const double *__restrict__ part,
                                                             const int32_t *__restrict__ ostart,
                                                             const int32_t *__restrict__ oidx,
                                                             double *__restrict__ sub, float *__restrict__ sub32,
                                                             int32_t *__restrict__ j64, int64_t ns)
{
    __shared__ double shA[SUB_WARPS][(HP + 1) * 2];
    __shared__ double shR[SUB_WARPS][HP + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * SUB_WARPS + wid;
    if (s >= ns) return;                     // warp-uniform; the kernel has no block barrier
    double *A = shA[wid], *red = shR[wid];
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
    const double ihs = 1.0 / hs;
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
    const int64_t rx0 = max(xlo, (int64_t)-1), rx1 = min(xhi, g.N1x);
    const int64_t ry0 = max(ylo, (int64_t)-1), ry1 = min(yhi, g.N1y);
    for (int64_t ry = ry0; ry <= ry1 && rx0 <= rx1; ++ry) {
        const int64_t b0 = (ry + 1) * g.NEx + (rx0 + 1), b1 = (ry + 1) * g.NEx + (rx1 + 1);
        const int64_t k0 = L.start[b0], k1 = L.start[b1 + 1];
        const bool near_row = ry - cy <= 1 && cy - ry <= 1;
        for (int64_t k = k0 + lane; k < k1; k += 32) {
            if (near_row) {
                const int64_t lx = lc[k].x;
                if (lx - cx <= 1 && cx - lx <= 1) continue;
            }
            p2l_add(L.m[k], L.x[k] - zx, L.y[k] - zy, hs, ihs, ar, ai);
        }
    }
    if (xlo < -1 || xhi > g.N1x || ylo < -1 || yhi > g.N1y) {
        const int64_t obx = h.NBx + 2;
        for (int64_t by = By - 1; by <= By + 1; ++by) {
            const int64_t b0 = (by + 1) * obx + Bx;          // bins of boxes Bx-1..Bx+1
            for (int64_t q = ostart[b0] + lane; q < ostart[b0 + 3]; q += 32) {
                const int32_t k = oidx[q];
                p2l_add(L.m[k], L.x[k] - zx, L.y[k] - zy, hs, ihs, ar, ai);
            }
        }
    }
    // box series of this cell's box: sum of the partitions (fixed order)
    const int64_t b = By * h.NBx + Bx;
    for (int j = lane; j <= HP; j += 32) {
        double vr = 0.0, vi = 0.0;
        for (int q = 0; q < HPARTS; ++q) {
            vr += part[((b * HPARTS + q) * (HP + 1) + j) * 2];
            vi += part[((b * HPARTS + q) * (HP + 1) + j) * 2 + 1];
        }
        A[2 * j] = vr;
        A[2 * j + 1] = vi;
    }
    // the direct sums: lane j holds order j, every lane order HP
    double sr, si, xr, xi;
    warp_sum_orders(ar, ai, sr, si, xr, xi);
    __syncwarp();
    // shift the box series to z_s: coefficient of V^j, V = (z - z_s)/hs, is
    // rho^j sum_{i>=j} C(i, j) A_i d^{i-j},  d = (z_s - z_B)/h_B, rho = hs/h_B
    const double zBx = g.rx0 + ((double)Bx + 0.5) * (double)h.bxn * g.l1x;
    const double zBy = g.ry0 + ((double)By + 0.5) * (double)h.byn * g.l1y;
    const double dr = (zx - zBx) / h.hB, di = (zy - zBy) / h.hB, rho = hs / h.hB;
    for (int j = lane; j <= HP; j += 32) {
        double vr = 0.0, vi = 0.0;
        for (int i = HP; i >= j; --i) {      // Horner in d
            const double c = g_binom.v[i * (HP + 1) + j];
            const double nr = vr * dr - vi * di + c * A[2 * i];
            const double ni = vr * di + vi * dr + c * A[2 * i + 1];
            vr = nr;
            vi = ni;
        }
        double sc = 1.0, rp = rho;           // rho^j by squaring
        for (int e = j; e > 0; e >>= 1, rp *= rp)
            if (e & 1) sc *= rp;
        const double fr = (j == HP ? xr : sr) + vr * sc;
        const double fi = (j == HP ? xi : si) + vi * sc;
        sub[(s * (HP + 1) + j) * 2] = fr;
        sub[(s * (HP + 1) + j) * 2 + 1] = fi;
        sub32[(s * (HP + 1) + j) * 2] = (float)fr;
        sub32[(s * (HP + 1) + j) * 2 + 1] = (float)fi;
        red[j] = fabs(fr) + fabs(fi);
    }
    __syncwarp();
    // FP64 length of the node's c_0 sum: the orders above j64 add up (in
    // |re| + |im|) to at most 2^-35 max(|re a_0|, |im a_0|), so their FP32 sum
    // (error below 2^-19 of that, |e| <= 1) stays under the FP64 rounding of c_0
    if (lane == 0) {
        const double lim = 2.9103830456733704e-11 * fmax(fabs(sub[s * (HP + 1) * 2]),
                                                         fabs(sub[s * (HP + 1) * 2 + 1]));
        double tail = 0.0;
        int J = HP;
        while (J > 0 && tail + red[J] <= lim) tail += red[J--];
        j64[s] = J;
    }
}

// 3. node coefficients from the sub-block series.  Index arithmetic in 32
// bits (level-2 cells per level-1 side and sub-block counts are small), the
// scales by reciprocals.
__global__ void __launch_bounds__(128) k_node_shift(Geo g, Hier h, const double *__restrict__ sub,
                                                   const float *__restrict__ sub32,
                                                   const int32_t *__restrict__ j64,
                                                   double *__restrict__ coef)
{
    // node-uniform loop indices: the binomials come from the constant cache
    const double *binom = c_binom.v;
    const float *binomf = c_binomf.v;
    int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= g.N2x * g.N2y) return;
    const int64_t c2y64 = node / g.N2x;
    const int c2x = (int)(node - c2y64 * g.N2x), c2y = (int)c2y64;
    const int l2sx = g.l2sx, l2sy = g.l2sy, nsx = (int)h.nsx, nsy = (int)h.nsy;
    const int cx = c2x / l2sx, cy = c2y / l2sy;
    const int u = c2x - cx * l2sx, v = c2y - cy * l2sy;
    const int sa = u * nsx / l2sx, sbb = v * nsy / l2sy;
    const int ua = (sa * l2sx + nsx - 1) / nsx, ub = ((sa + 1) * l2sx + nsx - 1) / nsx;
    const int va = (sbb * l2sy + nsy - 1) / nsy, vb = ((sbb + 1) * l2sy + nsy - 1) / nsy;
    const double hs = 0.5 * sqrt((double)((ub - ua) * (ub - ua)) * g.l2x * g.l2x +
                                 (double)((vb - va) * (vb - va)) * g.l2y * g.l2y);
    const double ihs = 1.0 / hs;
    // e = (z_node - z_s)/hs
    const double er = ((double)u + 0.5 - 0.5 * (double)(ua + ub)) * g.l2x * ihs;
    const double ei = ((double)v + 0.5 - 0.5 * (double)(va + vb)) * g.l2y * ihs;
    const int64_t s = ((int64_t)cy * g.N1x + cx) * (nsx * nsy) + sbb * nsx + sa;
    const double *a = sub + s * (HP + 1) * 2;
    const float *af = sub32 + s * (HP + 1) * 2;
    double *out = coef + node * (int64_t)(g.p + 1) * 2;
    // The mixed mode keeps c_1..c_p in FP32 (node records), so they are summed
    // in FP32 there: the shifted series decays (ratio < 0.6), no term cancels
    // far below the sum.  c_0, the node's far deflection, is FP64 up to order
    // j64[s] and FP32 above (the sub-block's bound); the FP64 near/far mode
    // takes c_1..c_p in FP64.
    const bool fp32_tail = g.precision == ML_PREC_MIXED;
    const float erf = (float)er, eif = (float)ei;
    {
        const int J = j64[s];
        float tr = 0.f, ti = 0.f;
        for (int j = HP; j > J; --j) {
            const float nr = __fmaf_rn(tr, erf, __fmaf_rn(-ti, eif, af[2 * j]));
            const float ni = __fmaf_rn(tr, eif, __fmaf_rn(ti, erf, af[2 * j + 1]));
            tr = nr;
            ti = ni;
        }
        double vr = tr, vi = ti;
        for (int j = J; j >= 0; --j) {
            const double nr = vr * er - vi * ei + a[2 * j];
            const double ni = vr * ei + vi * er + a[2 * j + 1];
            vr = nr;
            vi = ni;
        }
        out[0] = vr;
        out[1] = vi;
    }
    double ihn = 1.0;
    for (int n = 1; n <= g.p; ++n) {
        ihn *= ihs;
        if (fp32_tail) {
            float vr = 0.f, vi = 0.f;
            for (int j = HP; j >= n; --j) {
                const float c = binomf[j * (HP + 1) + n];
                const float nr = __fmaf_rn(vr, erf, __fmaf_rn(-vi, eif, c * af[2 * j]));
                const float ni = __fmaf_rn(vr, eif, __fmaf_rn(vi, erf, c * af[2 * j + 1]));
                vr = nr;
                vi = ni;
            }
            out[2 * n] = (double)vr * ihn;
            out[2 * n + 1] = (double)vi * ihn;
        } else {
            double vr = 0.0, vi = 0.0;
            for (int j = HP; j >= n; --j) {
                double c = binom[j * (HP + 1) + n];
                double nr = vr * er - vi * ei + c * a[2 * j];
                double ni = vr * ei + vi * er + c * a[2 * j + 1];
                vr = nr;
                vi = ni;
            }
            out[2 * n] = vr * ihn;
            out[2 * n + 1] = vi * ihn;
        }
    }
}

// FP64 box partials and sub-block series, then the FP32 copy of the latter
// (half a double per value, rounded up).
size_t hier_scratch_doubles(const Geo &g)
{
    Hier h = hier_of(g);
    size_t nb = (size_t)(h.NBx * h.NBy), ns = (size_t)(g.N1x * g.N1y * h.nsx * h.nsy);
    return (nb * HPARTS + ns) * (HP + 1) * 2 + (ns * (HP + 1) * 2 + 1) / 2 + (ns + 1) / 2 + 1;
}

cudaError_t launch_coeffs_hier(const Geo &g, const LensTable &L, double *coef64, double *scratch,
                               size_t scratch_doubles, cudaStream_t s)
{
    Hier h = hier_of(g);
    if (scratch_doubles < hier_scratch_doubles(g)) return cudaErrorInvalidValue;
    size_t nb = (size_t)(h.NBx * h.NBy), ns = (size_t)(g.N1x * g.N1y * h.nsx * h.nsy);
    double *part = scratch;
    double *sub = scratch + nb * HPARTS * (HP + 1) * 2;
    float *sub32 = reinterpret_cast<float *>(sub + ns * (HP + 1) * 2);
    int32_t *j64 = reinterpret_cast<int32_t *>(sub32 + ns * (HP + 1) * 2);
    // per-lens level-1 cells, then the outer lenses' CSR by box
    const size_t nl = (size_t)(L.n > 0 ? L.n : 1);
    const size_t nob = (size_t)((h.NBx + 2) * (h.NBy + 2));
    const size_t ints = 2 * nl + (nob + 1) + nl + (size_t)(SCAT_THREADS / 32) * nob;
    int32_t *iw = nullptr;
    cudaError_t e = ml_malloc_async((void **)&iw, sizeof(int32_t) * ints, s);
    if (e != cudaSuccess) return e;
    int2 *lc = reinterpret_cast<int2 *>(iw);
    int32_t *ostart = iw + 2 * nl, *oidx = ostart + nob + 1, *ocnt = oidx + nl;
    if (L.n > 0) k_lens_l1<<<(unsigned)((L.n + 255) / 256), 256, 0, s>>>(g, L, lc);
    k_outer_csr<<<1, SCAT_THREADS, 0, s>>>(lc, L.start, g.NEx * g.NEy, h, ocnt, ostart, oidx);
    dim3 gb((unsigned)nb, HPARTS);
    k_box_p2l<<<gb, 128, 0, s>>>(g, L, lc, h, part);
    k_sub_p2l<<<(unsigned)((ns + SUB_WARPS - 1) / SUB_WARPS), 32 * SUB_WARPS, 0, s>>>(g, L, lc, h, part, ostart,
                                                                                  oidx, sub, sub32, j64,
                                                                                  (int64_t)ns);
    int64_t nn = g.N2x * g.N2y;
    k_node_shift<<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(g, h, sub, sub32, j64, coef64);
    e = cudaGetLastError();
    cudaFreeAsync(iw, s);
    return e;
}


}  // namespace ml
