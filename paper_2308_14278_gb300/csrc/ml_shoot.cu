// Ray-shooting kernels (§3.2 Level 3: "each ray is assigned to a GPU
// thread"; here each warp takes a task of 32 lattice rows and each lane walks
// its row).
//
//  - k_shoot_mixed<P>: persistent kernel of the mixed-precision mode.  A task
//    is 32 consecutive ray rows inside one level-1 row band times a run of
//    level-2 columns inside one level-1 column.  The task's near lenses (the
//    3 x 3 block of level-1 cells, Fig. 1) are staged in shared memory as FP32
//    offsets; each lane evaluates the node's Taylor series as a polynomial in
//    its x offset, subtracts the near sum, bins the ray and merges runs of
//    rays that fall in the same pixel before one atomic add.
//  - k_shoot_direct64 / k_shoot_nearfar64: one thread per ray, FP64, the
//    reference-precision modes.
//  - k_trace_*: the same arithmetic for listed rays, returning beta.
#include "ml_internal.cuh"

#include <math.h>

namespace ml {

// ---- helpers shared by the FP64 modes ---------------------------------------

__device__ __forceinline__ void sheet64(const Geo &g, double tx, double ty, double &sx, double &sy)
{
    // deflection of the negative sheet (Eq. 6): -kappa_* u inside the disc,
    // -kappa_* R^2 u / |u|^2 outside
    double ux = tx - g.sheet_cx, uy = ty - g.sheet_cy;
    double s2 = ux * ux + uy * uy, R2 = g.sheet_r * g.sheet_r;
    double f = s2 <= R2 ? -g.kappa_star : -g.kappa_star * R2 / s2;
    sx = f * ux;
    sy = f * uy;
}

// beta of ray (i, j) in FP64 by the direct sum over all lenses (Eq. 6).
// Returns false for a ray that coincides with a lens.
__device__ bool beta_direct64(const ShootArgs &a, int64_t i, int64_t j, double &bx, double &by)
{
    const Geo &g = a.g;
    double tx = g.rx0 + ((double)i + 0.5) * g.l3x;
    double ty = g.ry0 + ((double)j + 0.5) * g.l3y;
    double ax = 0.0, ay = 0.0;
    bool hit = false;
    for (int64_t k = 0; k < a.L.n; ++k) {
        double dx = tx - a.L.x[k], dy = ty - a.L.y[k];
        double r2 = dx * dx + dy * dy;
        hit |= (r2 == 0.0);
        double s = a.L.m[k] / r2;
        ax += dx * s;
        ay += dy * s;
    }
    double sx, sy;
    sheet64(g, tx, ty, sx, sy);
    bx = (1.0 - g.kappa - g.gamma) * tx - ax - sx;
    by = (1.0 - g.kappa + g.gamma) * ty - ay - sy;
    return !hit;
}

// beta of ray (i, j) in FP64 by the near/far scheme (Eq. 9): near lenses of
// the 3 x 3 level-1 block summed directly, far field from the node series.
__device__ bool beta_nearfar64(const ShootArgs &a, int64_t i, int64_t j, double &bx, double &by)
{
    const Geo &g = a.g;
    double tx = g.rx0 + ((double)i + 0.5) * g.l3x;
    double ty = g.ry0 + ((double)j + 0.5) * g.l3y;
    int64_t c1x = i / g.n1x, c1y = j / g.n1y;
    int64_t c2x = i / g.n2x, c2y = j / g.n2y;
    double ax = 0.0, ay = 0.0;
    bool hit = false;
    for (int64_t ey = c1y; ey <= c1y + 2; ++ey) {
        int64_t b0 = ey * g.NEx + c1x;
        for (int32_t k = a.L.start[b0]; k < a.L.start[b0 + 3]; ++k) {
            double dx = tx - a.L.x[k], dy = ty - a.L.y[k];
            double r2 = dx * dx + dy * dy;
            hit |= (r2 == 0.0);
            double s = a.L.m[k] / r2;
            ax += dx * s;
            ay += dy * s;
        }
    }
    double zx = g.rx0 + ((double)c2x + 0.5) * g.l2x;
    double zy = g.ry0 + ((double)c2y + 0.5) * g.l2y;
    double dr = tx - zx, di = ty - zy;
    const double *c = a.coef64 + (c2y * g.N2x + c2x) * (int64_t)(g.p + 1) * 2;
    double Fr = 0.0, Fi = 0.0;
    for (int n = g.p; n >= 0; --n) {      // Horner: F = F d + c_n
        double nr = Fr * dr - Fi * di + c[2 * n];
        double ni = Fr * di + Fi * dr + c[2 * n + 1];
        Fr = nr;
        Fi = ni;
    }
    double sx, sy;
    sheet64(g, tx, ty, sx, sy);
    bx = (1.0 - g.kappa - g.gamma) * tx - ax - Fr - sx;   // alpha_far = conj(F)
    by = (1.0 - g.kappa + g.gamma) * ty - ay + Fi - sy;
    return !hit;
}

__device__ __forceinline__ void deposit_one(const ShootArgs &a, bool ok, double bx, double by,
                                            unsigned long long &in, unsigned long long &out,
                                            unsigned long long &drop, unsigned &ovf)
{
    const Geo &g = a.g;
    if (!ok) { ++drop; return; }
    if (g.deposit == ML_DEPOSIT_NGP) {
        double fx = floor((bx - g.mx0) / g.dpx), fy = floor((by - g.my0) / g.dpy);
        if (fx >= 0.0 && fx < (double)g.mnx && fy >= 0.0 && fy < (double)g.mny) {
            unsigned old = atomicAdd(a.map_u32 + (int64_t)fy * g.mnx + (int64_t)fx, 1u);
            ovf |= (old == 0xFFFFFFFFu);
            ++in;
        } else {
            ++out;
        }
    } else {
        // cloud in cell: bilinear weights to the four pixel centres around beta
        double fx = (bx - g.mx0) / g.dpx - 0.5, fy = (by - g.my0) / g.dpy - 0.5;
        double flx = floor(fx), fly = floor(fy);
        if (!(flx >= -1.0 && flx < (double)g.mnx && fly >= -1.0 && fly < (double)g.mny)) {
            ++out;
            return;
        }
        float wx = (float)(fx - flx), wy = (float)(fy - fly);
        int ix = (int)flx, iy = (int)fly;
        bool any = false;
        for (int q = 0; q < 4; ++q) {
            int px = ix + (q & 1), py = iy + (q >> 1);
            if (px < 0 || px >= g.mnx || py < 0 || py >= g.mny) continue;
            float w = ((q & 1) ? wx : 1.f - wx) * ((q >> 1) ? wy : 1.f - wy);
            atomicAdd(a.map_f32 + (int64_t)py * g.mnx + px, w);
            any = true;
        }
        if (any) ++in; else ++out;
    }
}

__device__ void flush_stats(const ShootArgs &a, unsigned long long in, unsigned long long out,
                            unsigned long long drop, unsigned long long pairs,
                            unsigned long long tasks, unsigned ovf)
{
    for (int o = 16; o > 0; o >>= 1) {
        in += __shfl_down_sync(0xffffffffu, in, o);
        out += __shfl_down_sync(0xffffffffu, out, o);
        drop += __shfl_down_sync(0xffffffffu, drop, o);
        pairs += __shfl_down_sync(0xffffffffu, pairs, o);
        ovf |= __shfl_down_sync(0xffffffffu, ovf, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (in) atomicAdd(a.stats + ML_STAT_RAYS_IN, in);
        if (out) atomicAdd(a.stats + ML_STAT_RAYS_OUT, out);
        if (drop) atomicAdd(a.stats + ML_STAT_RAYS_DROP, drop);
        if (pairs) atomicAdd(a.stats + ML_STAT_NEAR_PAIRS, pairs);
        if (tasks) atomicAdd(a.stats + ML_STAT_TASKS, tasks);
        if (ovf) atomicOr(a.status, 1u);
    }
}

// One thread per ray over [ray_begin, ray_end), FP64 (direct or near/far).
template <bool NEARFAR>
__global__ void __launch_bounds__(256) k_shoot_fp64(ShootArgs a)
{
    unsigned long long in = 0, out = 0, drop = 0, pairs = 0;
    unsigned ovf = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = a.ray_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < a.ray_end;
         r += stride) {
        int64_t i = r % a.g.n3x, j = r / a.g.n3x;
        double bx, by;
        bool ok = NEARFAR ? beta_nearfar64(a, i, j, bx, by) : beta_direct64(a, i, j, bx, by);
        deposit_one(a, ok, bx, by, in, out, drop, ovf);
    }
    flush_stats(a, in, out, drop, pairs, 0, ovf);
}

// ---- mixed precision: per-task staging and the walk --------------------------

struct TaskShape {
    int64_t row0, rows_end;         // ray rows of the task
    int64_t c1x, c1y, c2a, c2b;     // level-1 cell, level-2 column range
};

__device__ __forceinline__ bool decode_task(const ShootArgs &a, int64_t t, TaskShape &ts)
{
    const Geo &g = a.g;
    int64_t rg = a.rg_first + t / a.n_cc, cc = t % a.n_cc;
    int64_t c1y = rg / a.groups_per_band, grp = rg % a.groups_per_band;
    ts.c1y = c1y;
    ts.row0 = c1y * g.n1y + 32 * grp;
    ts.rows_end = min(min(ts.row0 + 32, (c1y + 1) * g.n1y), g.n3y);
    ts.c1x = cc / a.cc_per_l1;
    int64_t sub = cc % a.cc_per_l1;
    ts.c2a = ts.c1x * g.l2sub + sub * a.l2_per_cc;
    ts.c2b = min(min(ts.c2a + a.l2_per_cc, (ts.c1x + 1) * (int64_t)g.l2sub), g.N2x);
    return ts.row0 < ts.rows_end && ts.c2a < ts.c2b;
}

// Near-lens list of level-1 cell (c1x, c1y): three runs of the sorted table.
struct NearRuns {
    int32_t s0, n0, s1, n1, s2, n2;
    __device__ __forceinline__ int total() const { return n0 + n1 + n2; }
    __device__ __forceinline__ int32_t index(int k) const
    {
        return k < n0 ? s0 + k : (k < n0 + n1 ? s1 + (k - n0) : s2 + (k - n0 - n1));
    }
};

__device__ __forceinline__ NearRuns near_runs(const ShootArgs &a, int64_t c1x, int64_t c1y)
{
    NearRuns nr;
    const int32_t *st = a.L.start;
    int64_t b0 = c1y * a.g.NEx + c1x, b1 = b0 + a.g.NEx, b2 = b1 + a.g.NEx;
    nr.s0 = st[b0]; nr.n0 = st[b0 + 3] - nr.s0;
    nr.s1 = st[b1]; nr.n1 = st[b1 + 3] - nr.s1;
    nr.s2 = st[b2]; nr.n2 = st[b2 + 3] - nr.s2;
    return nr;
}

// Near records computed from the FP64 lens table, for tracing single rays.
struct GlobalNear {
    const LensTable *L;
    NearRuns nr;
    double xnode, yref;
    __device__ __forceinline__ float4 rec(int k) const
    {
        int32_t id = nr.index(k);
        return make_float4((float)(L->x[id] - xnode), (float)(L->y[id] - yref), (float)L->m[id], 0.f);
    }
    __device__ __forceinline__ float2 lo(int k) const
    {
        int32_t id = nr.index(k);
        double dx = L->x[id] - xnode, dy = L->y[id] - yref;
        return make_float2((float)(dx - (double)(float)dx), (float)(dy - (double)(float)dy));
    }
};

template <int P>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32) k_shoot_mixed(ShootArgs a)
{
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *near = smem + wid * a.near_cap;
    float2 *nlo = reinterpret_cast<float2 *>(smem + WARPS_PER_CTA * a.near_cap) + wid * a.near_cap;
    const Geo &g = a.g;
    const int64_t jb = a.ray_begin / g.n3x, ib = a.ray_begin % g.n3x;
    const int64_t je = (a.ray_end - 1) / g.n3x, ie = (a.ray_end - 1) % g.n3x + 1;

    unsigned long long in = 0, out = 0, drop = 0, pairs = 0, tasks = 0;
    unsigned ovf = 0;
    uint32_t cur = PIX_OUT;
    unsigned cnt = 0, pold = 0, pcnt = 0;

    for (;;) {
        int64_t t = 0;
        int stop = 0;
        if (lane == 0) {
            t = (int64_t)atomicAdd(a.work, 1ull);
            stop = *a.abort_flag;
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop) {
            if (lane == 0) atomicOr(a.status, 2u);
            break;
        }
        if (t >= a.n_tasks) break;
        TaskShape ts;
        if (!decode_task(a, t, ts)) continue;
        ++tasks;
        // stage the near lenses: y offset from the task's first row and mass
        const NearRuns nr = near_runs(a, ts.c1x, ts.c1y);
        const int nn = nr.total();
        const double yref = g.ry0 + ((double)ts.row0 + 0.5) * g.l3y;
        __syncwarp();
        for (int k = lane; k < nn; k += 32) {
            int32_t idx = nr.index(k);
            double dy = a.L.y[idx] - yref;
            float hi = (float)dy;
            near[k] = make_float4(0.f, hi, (float)a.L.m[idx], __int_as_float(idx));
            nlo[k].y = (float)(dy - (double)hi);
        }
        const int64_t j = ts.row0 + lane;
        const bool active = j < ts.rows_end && j >= jb && j <= je;
        const double dyl_d = (double)lane * g.l3y;
        const float dyl = (float)dyl_d;
        const float dyl_lo = (float)(dyl_d - (double)dyl);
        const int64_t c2y = j / g.n2y;
        const float q = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
        for (int64_t c2x = ts.c2a; c2x < ts.c2b; ++c2x) {
            const double xnode = g.rx0 + ((double)c2x + 0.5) * g.l2x;
            __syncwarp();
            for (int k = lane; k < nn; k += 32) {
                double dx = a.L.x[__float_as_int(near[k].w)] - xnode;
                float hi = (float)dx;
                near[k].x = hi;
                nlo[k].x = (float)(dx - (double)hi);
            }
            __syncwarp();
            if (!active) continue;
            const int64_t i0 = c2x * g.n2x;
            int64_t ia = i0, iend = min(i0 + g.n2x, g.n3x);
            if (j == jb) ia = max(ia, ib);
            if (j == je) iend = min(iend, ie);
            if (ia >= iend) continue;
            RowPoly<P> rp;
            row_setup<P>(a.nodes + (c2y * g.N2x + c2x) * node_stride(P), q, a, rp);
            pairs += (unsigned long long)nn * (unsigned long long)(iend - ia);
            float u = __fadd_rn((float)(ia - i0), a.c0_f);
            for (int64_t i = ia; i < iend; ++i, u += 1.f) {
                float tt = __fmul_rn(u, a.l3x_f);
                float X, Y, ax, ay;
                row_eval<P>(rp, tt, X, Y);
                near_sum_f32(SmemNear{near, nlo}, nn, u, tt, dyl, dyl_lo, a.l3x_f, a.l3x_lo, a.rc2, ax, ay);
                X = __fmaf_rn(-ax, a.ipx_f, X);
                Y = __fmaf_rn(-ay, a.ipy_f, Y);
                uint32_t pix = classify(X, Y, ax, rp.bx, rp.by, g.mnx, g.mny);
                if (pix != cur) {
                    if (cnt) {
                        if (cur < PIX_DROP) {
                            ovf |= (pold > 0xFFFFFFFFu - pcnt);
                            pold = atomicAdd(a.map_u32 + cur, cnt);
                            pcnt = cnt;
                            in += cnt;
                        } else if (cur == PIX_OUT) {
                            out += cnt;
                        } else {
                            drop += cnt;
                        }
                    }
                    cur = pix;
                    cnt = 0;
                }
                ++cnt;
            }
        }
    }
    if (cnt) {
        if (cur < PIX_DROP) {
            ovf |= (pold > 0xFFFFFFFFu - pcnt);
            pold = atomicAdd(a.map_u32 + cur, cnt);
            pcnt = cnt;
            in += cnt;
        } else if (cur == PIX_OUT) {
            out += cnt;
        } else {
            drop += cnt;
        }
    }
    ovf |= (pold > 0xFFFFFFFFu - pcnt);
    // near pairs are counted per lane; sum over lanes is the exact pair count
    flush_stats(a, in, out, drop, pairs, lane == 0 ? tasks : 0, ovf);
}

// Cloud-in-cell variant of the mixed kernel (float map, four atomics per ray).
template <int P>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32) k_shoot_mixed_cic(ShootArgs a)
{
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *near = smem + wid * a.near_cap;
    float2 *nlo = reinterpret_cast<float2 *>(smem + WARPS_PER_CTA * a.near_cap) + wid * a.near_cap;
    const Geo &g = a.g;
    const int64_t jb = a.ray_begin / g.n3x, ib = a.ray_begin % g.n3x;
    const int64_t je = (a.ray_end - 1) / g.n3x, ie = (a.ray_end - 1) % g.n3x + 1;
    unsigned long long in = 0, out = 0, drop = 0, pairs = 0, tasks = 0;
    for (;;) {
        int64_t t = 0;
        int stop = 0;
        if (lane == 0) {
            t = (int64_t)atomicAdd(a.work, 1ull);
            stop = *a.abort_flag;
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop) {
            if (lane == 0) atomicOr(a.status, 2u);
            break;
        }
        if (t >= a.n_tasks) break;
        TaskShape ts;
        if (!decode_task(a, t, ts)) continue;
        ++tasks;
        const NearRuns nr = near_runs(a, ts.c1x, ts.c1y);
        const int nn = nr.total();
        const double yref = g.ry0 + ((double)ts.row0 + 0.5) * g.l3y;
        __syncwarp();
        for (int k = lane; k < nn; k += 32) {
            int32_t idx = nr.index(k);
            double dy = a.L.y[idx] - yref;
            float hi = (float)dy;
            near[k] = make_float4(0.f, hi, (float)a.L.m[idx], __int_as_float(idx));
            nlo[k].y = (float)(dy - (double)hi);
        }
        const int64_t j = ts.row0 + lane;
        const bool active = j < ts.rows_end && j >= jb && j <= je;
        const double dyl_d = (double)lane * g.l3y;
        const float dyl = (float)dyl_d;
        const float dyl_lo = (float)(dyl_d - (double)dyl);
        const int64_t c2y = j / g.n2y;
        const float q = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
        for (int64_t c2x = ts.c2a; c2x < ts.c2b; ++c2x) {
            const double xnode = g.rx0 + ((double)c2x + 0.5) * g.l2x;
            __syncwarp();
            for (int k = lane; k < nn; k += 32) {
                double dx = a.L.x[__float_as_int(near[k].w)] - xnode;
                float hi = (float)dx;
                near[k].x = hi;
                nlo[k].x = (float)(dx - (double)hi);
            }
            __syncwarp();
            if (!active) continue;
            const int64_t i0 = c2x * g.n2x;
            int64_t ia = i0, iend = min(i0 + g.n2x, g.n3x);
            if (j == jb) ia = max(ia, ib);
            if (j == je) iend = min(iend, ie);
            if (ia >= iend) continue;
            RowPoly<P> rp;
            row_setup<P>(a.nodes + (c2y * g.N2x + c2x) * node_stride(P), q, a, rp);
            pairs += (unsigned long long)nn * (unsigned long long)(iend - ia);
            float u = __fadd_rn((float)(ia - i0), a.c0_f);
            for (int64_t i = ia; i < iend; ++i, u += 1.f) {
                float tt = __fmul_rn(u, a.l3x_f);
                float X, Y, ax, ay;
                row_eval<P>(rp, tt, X, Y);
                near_sum_f32(SmemNear{near, nlo}, nn, u, tt, dyl, dyl_lo, a.l3x_f, a.l3x_lo, a.rc2, ax, ay);
                X = __fmaf_rn(-ax, a.ipx_f, X);
                Y = __fmaf_rn(-ay, a.ipy_f, Y);
                if (ax != ax) { ++drop; continue; }
                float fx = __fsub_rn(X, 0.5f), fy = __fsub_rn(Y, 0.5f);
                float flx = floorf(fx), fly = floorf(fy);
                float wx = __fsub_rn(fx, flx), wy = __fsub_rn(fy, fly);
                unsigned ix = (unsigned)rp.bx + (unsigned)__float2int_rd(flx);
                unsigned iy = (unsigned)rp.by + (unsigned)__float2int_rd(fly);
                bool any = false;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    unsigned px = ix + (unsigned)(qq & 1), py = iy + (unsigned)(qq >> 1);
                    if (px >= (unsigned)g.mnx || py >= (unsigned)g.mny) continue;
                    float w = __fmul_rn((qq & 1) ? wx : 1.f - wx, (qq >> 1) ? wy : 1.f - wy);
                    atomicAdd(a.map_f32 + (int64_t)py * g.mnx + px, w);
                    any = true;
                }
                if (any) ++in; else ++out;
            }
        }
    }
    flush_stats(a, in, out, drop, pairs, lane == 0 ? tasks : 0, 0u);
}

// ---- tracing: the same per-ray arithmetic for listed rays -------------------

template <int P>
__global__ void k_trace_mixed(ShootArgs a, const int64_t *__restrict__ idx, int64_t n,
                              double *__restrict__ beta, int32_t *__restrict__ pix)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const Geo &g = a.g;
    int64_t r = idx[q];
    if (r < 0 || r >= g.n3x * g.n3y) {
        beta[2 * q] = beta[2 * q + 1] = __longlong_as_double(0x7ff8000000000000ll);
        pix[2 * q] = pix[2 * q + 1] = -3;
        return;
    }
    int64_t i = r % g.n3x, j = r / g.n3x;
    int64_t c1x = i / g.n1x, c1y = j / g.n1y;
    int64_t c2x = i / g.n2x, c2y = j / g.n2y;
    int64_t row0 = c1y * g.n1y + 32 * ((j - c1y * g.n1y) / 32);
    double yref = g.ry0 + ((double)row0 + 0.5) * g.l3y;
    double xnode = g.rx0 + ((double)c2x + 0.5) * g.l2x;
    float dyl = (float)((double)(j - row0) * g.l3y);
    float qf = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
    RowPoly<P> rp;
    row_setup<P>(a.nodes + (c2y * g.N2x + c2x) * node_stride(P), qf, a, rp);
    float u = __fadd_rn((float)(i - c2x * g.n2x), a.c0_f);
    float tt = __fmul_rn(u, a.l3x_f);
    float X, Y;
    row_eval<P>(rp, tt, X, Y);
    // near sum over the same lenses, in the same order, with records built
    // and summed exactly as in the walk
    const NearRuns nr = near_runs(a, c1x, c1y);
    const double dyl_d = (double)(j - row0) * g.l3y;
    const float dyl_lo = (float)(dyl_d - (double)dyl);
    float sx, sy;
    near_sum_f32(GlobalNear{&a.L, nr, xnode, yref}, nr.total(), u, tt, dyl, dyl_lo, a.l3x_f,
                 a.l3x_lo, a.rc2, sx, sy);
    X = __fmaf_rn(-sx, a.ipx_f, X);
    Y = __fmaf_rn(-sy, a.ipy_f, Y);
    uint32_t p = classify(X, Y, sx, rp.bx, rp.by, g.mnx, g.mny);
    beta[2 * q] = g.mx0 + ((double)rp.bx + (double)X) * g.dpx;
    beta[2 * q + 1] = g.my0 + ((double)rp.by + (double)Y) * g.dpy;
    if (p == PIX_DROP) { pix[2 * q] = -2; pix[2 * q + 1] = -2; }
    else if (p == PIX_OUT) { pix[2 * q] = -1; pix[2 * q + 1] = -1; }
    else { pix[2 * q] = (int32_t)(p % (uint32_t)g.mnx); pix[2 * q + 1] = (int32_t)(p / (uint32_t)g.mnx); }
}

template <bool NEARFAR>
__global__ void k_trace_fp64(ShootArgs a, const int64_t *__restrict__ idx, int64_t n,
                             double *__restrict__ beta, int32_t *__restrict__ pix)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const Geo &g = a.g;
    int64_t r = idx[q];
    if (r < 0 || r >= g.n3x * g.n3y) {
        beta[2 * q] = beta[2 * q + 1] = __longlong_as_double(0x7ff8000000000000ll);
        pix[2 * q] = pix[2 * q + 1] = -3;
        return;
    }
    int64_t i = r % g.n3x, j = r / g.n3x;
    double bx, by;
    bool ok = NEARFAR ? beta_nearfar64(a, i, j, bx, by) : beta_direct64(a, i, j, bx, by);
    beta[2 * q] = bx;
    beta[2 * q + 1] = by;
    if (!ok) { pix[2 * q] = -2; pix[2 * q + 1] = -2; return; }
    double fx = floor((bx - g.mx0) / g.dpx), fy = floor((by - g.my0) / g.dpy);
    if (fx >= 0.0 && fx < (double)g.mnx && fy >= 0.0 && fy < (double)g.mny) {
        pix[2 * q] = (int32_t)fx;
        pix[2 * q + 1] = (int32_t)fy;
    } else {
        pix[2 * q] = -1;
        pix[2 * q + 1] = -1;
    }
}

// ---- dispatch ----------------------------------------------------------------

// Taylor orders with a compiled mixed kernel; other orders round up.
int mixed_p_supported(int p)
{
    static const int avail[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
    for (int v : avail)
        if (v >= p) return v;
    return -1;
}

template <int P>
static cudaError_t launch_mixed_p(const ShootArgs &a, int num_sms, cudaStream_t s)
{
    size_t smem = (size_t)a.near_cap * WARPS_PER_CTA * (sizeof(float4) + sizeof(float2));
    auto kern = a.g.deposit == ML_DEPOSIT_NGP ? k_shoot_mixed<P> : k_shoot_mixed_cic<P>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                  WARPS_PER_CTA * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t warps_needed = a.n_tasks;
    int64_t blocks = (int64_t)num_sms * per_sm;
    int64_t need = (warps_needed + WARPS_PER_CTA - 1) / WARPS_PER_CTA;
    if (need < blocks) blocks = need > 0 ? need : 1;
    kern<<<(unsigned)blocks, WARPS_PER_CTA * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_shoot(const ShootArgs &a, int num_sms, cudaStream_t s)
{
    if (a.ray_end <= a.ray_begin) return cudaSuccess;
    if (a.g.precision == ML_PREC_MIXED) {
        switch (a.g.p) {
        case 1: return launch_mixed_p<1>(a, num_sms, s);
        case 2: return launch_mixed_p<2>(a, num_sms, s);
        case 3: return launch_mixed_p<3>(a, num_sms, s);
        case 4: return launch_mixed_p<4>(a, num_sms, s);
        case 5: return launch_mixed_p<5>(a, num_sms, s);
        case 6: return launch_mixed_p<6>(a, num_sms, s);
        case 8: return launch_mixed_p<8>(a, num_sms, s);
        case 10: return launch_mixed_p<10>(a, num_sms, s);
        case 12: return launch_mixed_p<12>(a, num_sms, s);
        case 16: return launch_mixed_p<16>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
        }
    }
    int64_t n = a.ray_end - a.ray_begin;
    int64_t blocks = (n + 255) / 256;
    int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (a.g.precision == ML_PREC_NEARFAR64)
        k_shoot_fp64<true><<<(unsigned)blocks, 256, 0, s>>>(a);
    else
        k_shoot_fp64<false><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_trace(const ShootArgs &a, const int64_t *idx, int64_t n, double *beta,
                         int32_t *pix, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((n + 127) / 128);
    if (a.g.precision == ML_PREC_MIXED) {
        switch (a.g.p) {
#define ML_TRACE_CASE(P) case P: k_trace_mixed<P><<<blocks, 128, 0, s>>>(a, idx, n, beta, pix); break;
        ML_TRACE_CASE(1) ML_TRACE_CASE(2) ML_TRACE_CASE(3) ML_TRACE_CASE(4) ML_TRACE_CASE(5)
        ML_TRACE_CASE(6) ML_TRACE_CASE(8) ML_TRACE_CASE(10) ML_TRACE_CASE(12) ML_TRACE_CASE(16)
#undef ML_TRACE_CASE
        default: return cudaErrorInvalidValue;
        }
    } else if (a.g.precision == ML_PREC_NEARFAR64) {
        k_trace_fp64<true><<<blocks, 128, 0, s>>>(a, idx, n, beta, pix);
    } else {
        k_trace_fp64<false><<<blocks, 128, 0, s>>>(a, idx, n, beta, pix);
    }
    return cudaGetLastError();
}

}  // namespace ml
