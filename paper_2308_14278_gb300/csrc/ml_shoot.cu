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
#include "ml_task.cuh"

#include <math.h>

#include <algorithm>

// CTAs per SM the mixed kernels are compiled for (register budget).
#ifndef ML_MIN_BLOCKS
#define ML_MIN_BLOCKS 3
#endif

namespace ml {

// ---- helpers shared by the FP64 modes ---------------------------------------

__device__ __forceinline__ void sheet64(const Geo &g, double tx, double ty, double &sx, double &sy)
{
    if (g.sheet_shape == ML_SHEET_STRIP) {
        // unbounded slab of half-width R: -2 kappa_* (theta_y - c_y) inside, constant outside
        const double v = fmin(fmax(ty - g.sheet_cy, -g.sheet_r), g.sheet_r);
        sx = 0.0;
        sy = -2.0 * g.kappa_star * v;
        return;
    }
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
    double mx, my;
    macro64(g, tx, ty, mx, my);
    bx = mx - ax - sx;
    by = my - ay - sy;
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
    double mx, my;
    macro64(g, tx, ty, mx, my);
    bx = mx - ax - Fr - sx;   // alpha_far = conj(F)
    by = my - ay + Fi - sy;
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

// Per-lane counts of the certified walk (walk_span): rays whose source
// position was evaluated one by one, and spans of rays certified to share a
// pixel without being evaluated.
struct SpanCount {
    unsigned long long evals = 0, spans = 0;
};

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

// Per-lane run-length state of the NGP deposit: consecutive rays of a lane's
// walk usually land in the same pixel (the macro map compresses x), so counts
// are merged and added with one atomic when the pixel changes.  The atomics
// return nothing (fire-and-forget reductions); a wrapped uint32 count is found
// afterwards by comparing the map's 64-bit sum with the in-map ray counter.
struct RunState {
    int cx, cy;
    unsigned cnt;
    unsigned in, out;
};

__device__ __forceinline__ void run_flush(RunState &rs, uint32_t *map, int mnx, int mny)
{
    if (rs.cnt == 0) return;
    if ((unsigned)rs.cx < (unsigned)mnx && (unsigned)rs.cy < (unsigned)mny) {
        atomicAdd(map + (size_t)rs.cy * (unsigned)mnx + (unsigned)rs.cx, rs.cnt);
        rs.in += rs.cnt;
    } else {
        rs.out += rs.cnt;
    }
}

__device__ __forceinline__ void run_add(RunState &rs, int gx, int gy, uint32_t *map, int mnx, int mny)
{
    if (gx != rs.cx || gy != rs.cy) {
        run_flush(rs, map, mnx, mny);
        rs.cx = gx;
        rs.cy = gy;
        rs.cnt = 0;
    }
    ++rs.cnt;
}

// Lane-valid ray of a warp-uniform walk position.
__device__ __forceinline__ bool in_range(int k, int k0, int k1) { return k >= k0 && k < k1; }

// Run-length step for one ray, with a warp vote so that the common case (no
// lane changes pixel) takes no divergent branch; the flush inside is
// predicated.  `valid` rays of other lanes' ranges do not count.
__device__ __forceinline__ void run_step(RunState &rs, bool valid, int gx, int gy, uint32_t *map,
                                         int mnx, int mny)
{
    const bool chg = valid && (gx != rs.cx || gy != rs.cy);
    if (__ballot_sync(0xffffffffu, chg)) {
        if (chg) {
            if (rs.cnt) {
                if ((unsigned)rs.cx < (unsigned)mnx && (unsigned)rs.cy < (unsigned)mny) {
                    atomicAdd(map + (size_t)rs.cy * (unsigned)mnx + (unsigned)rs.cx, rs.cnt);
                    rs.in += rs.cnt;
                } else {
                    rs.out += rs.cnt;
                }
            }
            rs.cx = gx;
            rs.cy = gy;
            rs.cnt = 0;
        }
    }
    rs.cnt += valid ? 1u : 0u;
}

// Flush a finished run of `cnt` rays in pixel (cx, cy) (predicated use).
__device__ __forceinline__ void flush_run(RunState &rs, int cx, int cy, unsigned cnt, uint32_t *map,
                                          int mnx, int mny)
{
    if (cnt == 0) return;
    if ((unsigned)cx < (unsigned)mnx && (unsigned)cy < (unsigned)mny) {
        atomicAdd(map + (size_t)cy * (unsigned)mnx + (unsigned)cx, cnt);
        rs.in += cnt;
    } else {
        rs.out += cnt;
    }
}

// One level-2 column of a warp's walk when every active lane covers the
// warp's whole range [kbeg, kend) ("on" lanes) and the near list has NN
// lenses (NN known at compile time: records and the lane's dy^2 and scaled
// dy in registers).  Rays go in pairs; a run's length is the distance between the
// indices where it starts and ends, so no per-ray counting is needed; one
// warp vote per pair decides whether any lane's pixel changed, and one flush
// serves a pair (a second one only when both rays change pixel).  There is
// one copy of the pair code and none for an odd tail, which keeps the nine
// specialisations small enough for the instruction cache.  Per ray the
// arithmetic is exactly near_sum_lat's and row_eval's; the row polynomial's
// (X, Y) pair and the floor's round-down add run on two-lane FP32
// instructions, whose lanes round as the scalar ones.
//
// Pixels are compared in their raw floor form: the bit pattern r of
// X + 1.5 * 2^23 rounded toward -inf, so that pixel = r - 0x4B400000 + base
// (wrapping 32-bit arithmetic, a bijection); the pixel itself is formed only
// when a run is flushed.  A ray that coincides with a lens (close-pass path
// fails) gets X = -1e30, which sends it far outside the map; it is
// counted as dropped there and as out by the run, and the kernel's epilogue
// subtracts the dropped rays from the out count.
//
// CLOSE = false when no ray of the warp's walk can come within the close-pass
// radius of a near lens (checked per row against the lens's distance to the
// row's ray segment, with a margin): the per-ray minimum distance and its
// vote are then skipped; the close-pass branch could not be taken anyway.
template <int P, int NN, bool CLOSE>
__device__ __forceinline__ void walk_fixed(const RowPoly<P> &rp, const ShootArgs &a, const SmemNear &nl,
                                           int kbeg, int kend, bool on, float dyl, float dyl_lo,
                                           RunState &rs, unsigned &drop)
{
    float lx[NN > 0 ? NN : 1], lm[NN > 0 ? NN : 1], dy2[NN > 0 ? NN : 1], dyy[NN > 0 ? NN : 1];
#pragma unroll
    for (int q = 0; q < NN; ++q) {
        float4 L = nl.near[q];
        lx[q] = L.x;
        lm[q] = L.z;
        const float dy = __fsub_rn(L.y, dyl);
        dy2[q] = __fmul_rn(dy, dy);
        dyy[q] = __fmul_rn(dy, a.yx_f);
    }
    const Geo &g = a.g;
    const unsigned offx = (unsigned)rp.bx - 0x4B400000u, offy = (unsigned)rp.by - 0x4B400000u;
    unsigned rcx = (unsigned)rs.cx - offx, rcy = (unsigned)rs.cy - offy;   // raw form of the run's pixel
    int kst = kbeg;                      // first ray of the current run in this walk
    // the row polynomial as (X, Y) coefficient pairs: a ray's two Horner
    // chains run as one chain of two-lane FMAs (row_eval's arithmetic)
    f32x2 C[P + 1];
#pragma unroll
    for (int m = 0; m <= P; ++m) C[m] = pack2(rp.X[m], rp.Y[m]);
    auto poly = [&](f32x2 U) {
        f32x2 v = C[P];
#pragma unroll
        for (int m = P - 1; m >= 0; --m) v = fma2(v, U, C[m]);
        return v;
    };
    const f32x2 MAGIC = pack2(12582912.0f, 12582912.0f), TWO = pack2(2.f, 2.f);
    const float ub = __fadd_rn((float)kbeg, a.c0_f);
    f32x2 U0 = pack2(ub, ub);
    const float ub1 = __fadd_rn(ub, 1.f);
    f32x2 U1 = pack2(ub1, ub1);

    // near sum of one ray added to its pixel position (exactly near_sum_lat's
    // arithmetic)
    auto near = [&](float uu, float &X, float &Y, float &mn) {
        mn = 3.0e38f;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            float dx = __fsub_rn(lx[q], uu);
            float r2 = __fmaf_rn(dx, dx, dy2[q]);
            if (CLOSE) mn = fminf(mn, r2);
            float sv = __fmul_rn(lm[q], rcp_approx(r2));
            X = __fmaf_rn(dx, sv, X);
            Y = __fmaf_rn(dyy[q], sv, Y);
        }
    };
    auto raw = [&](float X, float Y, unsigned &rx, unsigned &ry) {
        float fx, fy;
        unpack2(add2_rd(pack2(X, Y), MAGIC), fx, fy);
        rx = (unsigned)__float_as_int(fx);
        ry = (unsigned)__float_as_int(fy);
    };
    // a close pass redoes the ray from its row polynomial; a failed one (ray
    // on a lens) sends the ray far outside the map.  One copy of the code for
    // both rays of a pair (rare path).
    auto close_pair = [&](bool c0, bool c1, float u0, float &X0, float &Y0, float &X1, float &Y1) {
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
            const bool c = r ? c1 : c0;
            if (c) {
                const float uu = __fadd_rn(u0, (float)r);
                float X, Y;
                unpack2(poly(pack2(uu, uu)), X, Y);
                if (!near_sum_hilo_lat(nl, NN, uu, dyl, dyl_lo, a.yx_f, X, Y)) {
                    X = -1.0e30f;
                    ++drop;
                }
                if (r) { X1 = X; Y1 = Y; } else { X0 = X; Y0 = Y; }
            }
        }
    };

    // pairs of rays; after an odd last ray the pair's second ray is the
    // lattice's next one (index kend), evaluated but never counted: run
    // lengths are index differences bounded by kend, so a run it starts has
    // no rays; it takes no close pass
    for (int k = kbeg; k < kend; k += 2, U0 = add2(U0, TWO), U1 = add2(U1, TWO)) {
        float u, u1, uh;
        unpack2(U0, u, uh);
        unpack2(U1, u1, uh);
        float X0, Y0, X1, Y1, mn0, mn1;
        unpack2(poly(U0), X0, Y0);
        unpack2(poly(U1), X1, Y1);
        near(u, X0, Y0, mn0);
        near(u1, X1, Y1, mn1);
        if (NN > 0 && CLOSE) {
            const bool c0 = on && mn0 < a.rc2u, c1 = on && mn1 < a.rc2u;
            if (__ballot_sync(0xffffffffu, c0 || c1)) close_pair(c0, c1 && k + 1 < kend, u, X0, Y0, X1, Y1);
        }
        unsigned rx0, ry0, rx1, ry1;
        raw(X0, Y0, rx0, ry0);
        raw(X1, Y1, rx1, ry1);
        // after ray 0 the run's pixel is ray 0's whether or not it changed
        const bool ch0 = on && (rx0 != rcx || ry0 != rcy);
        const bool ch1 = on && (rx1 != rx0 || ry1 != ry0);
        if (__ballot_sync(0xffffffffu, ch0 || ch1)) {
            if (ch0 || ch1) {
                // the current run ends before ray 0 (ch0) or after it (ray 0
                // continues it); if both changed, ray 0 is a run of its own
                flush_run(rs, (int)(rcx + offx), (int)(rcy + offy),
                          rs.cnt + (unsigned)(k - kst) + (ch0 ? 0u : 1u), a.map_u32, g.mnx, g.mny);
                rs.cnt = 0;
                if (ch0 && ch1) flush_run(rs, (int)(rx0 + offx), (int)(ry0 + offy), 1u, a.map_u32, g.mnx, g.mny);
                kst = ch1 ? k + 1 : k;
                rcx = ch1 ? rx1 : rx0;
                rcy = ch1 ? ry1 : ry0;
            }
        }
    }
    if (on) rs.cnt += (unsigned)(kend - kst);
    rs.cx = (int)(rcx + offx);
    rs.cy = (int)(rcy + offy);
}

// The same for a near list of any length (read from shared memory).
template <int P>
__device__ __forceinline__ void walk_any(const RowPoly<P> &rp, const ShootArgs &a, const SmemNear &nl,
                                         int nn, int kbeg, int kend, int k0, int k1, float dyl,
                                         float dyl_lo, RunState &rs, unsigned &drop)
{
    const Geo &g = a.g;
    float u = __fadd_rn((float)kbeg, a.c0_f);
    for (int k = kbeg; k < kend; k += 2, u += 2.f) {
        const float u1 = __fadd_rn(u, 1.f);
        float X0, Y0, X1, Y1, mn0, mn1;
        row_eval<P>(rp, u, X0, Y0);
        row_eval<P>(rp, u1, X1, Y1);
        near_sum2_lat(nl, nn, u, u1, dyl, a.yx_f, X0, Y0, mn0, X1, Y1, mn1);
        const bool v0 = in_range(k, k0, k1), v1 = in_range(k + 1, k0, k1);
        const bool c0 = v0 && mn0 < a.rc2u, c1 = v1 && mn1 < a.rc2u;
        bool ok0 = true, ok1 = true;
        if (__ballot_sync(0xffffffffu, c0 || c1)) {
            if (c0) {
                row_eval<P>(rp, u, X0, Y0);
                ok0 = near_sum_hilo_lat(nl, nn, u, dyl, dyl_lo, a.yx_f, X0, Y0);
            }
            if (c1) {
                row_eval<P>(rp, u1, X1, Y1);
                ok1 = near_sum_hilo_lat(nl, nn, u1, dyl, dyl_lo, a.yx_f, X1, Y1);
            }
        }
        int gx0, gy0, gx1, gy1;
        pixel_xy(X0, Y0, rp.bx, rp.by, gx0, gy0);
        pixel_xy(X1, Y1, rp.bx, rp.by, gx1, gy1);
        if (!ok0) { gx0 = -1; gy0 = -1; ++drop; }
        if (!ok1) { gx1 = -1; gy1 = -1; ++drop; }
        run_step(rs, v0, gx0, gy0, a.map_u32, g.mnx, g.mny);
        run_step(rs, v1, gx1, gy1, a.map_u32, g.mnx, g.mny);
    }
}

// Approximate reciprocal square root (rsqrt.approx.ftz.f32); used only in
// the certification bounds below, which carry a safety factor.
__device__ __forceinline__ float rsqrt_approx(float y)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

constexpr int NN_DYN = 5;   // walk_span: near list of any length, read from shared memory

// Span-walk counts of a warp into the field's counters.
__device__ void flush_spans(const ShootArgs &a, const SpanCount &sc)
{
    unsigned long long ev = sc.evals, sp = sc.spans;
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_down_sync(0xffffffffu, ev, o);
        sp += __shfl_down_sync(0xffffffffu, sp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ev) atomicAdd(a.stats + ML_STAT_RAYS_EVAL, ev);
        if (sp) atomicAdd(a.stats + ML_STAT_SPANS, sp);
    }
}

// Certified walk of one level-2 column (NGP counts).  Each lane walks its own
// ray range [k0, k1) of its row in steps.  A step evaluates a window of W
// consecutive rays kb, kb+1, ... with exactly the per-ray arithmetic of
// walk_fixed / near_sum_lat / row_eval, after the lane's last evaluated ray
// ka.  When kb > ka + 1 the rays strictly between them are not evaluated:
// they join the current run only if ray kb lands in the run's pixel and a
// bound proves that every ray between lands there too; otherwise the lane
// takes nothing from this step and retries with a shorter gap.  Every ray
// therefore gets the pixel the per-ray walk gives it, and the counts are
// bit-identical.  The gap is chosen so that the window starts ML_SPAN_MARGIN
// rays short of where the lane's (X, Y) slope says the next pixel edge lies,
// so that one step usually crosses it.  The window's rays are evaluated
// together, in straight-line code: their Horner chains are independent and
// interleave, the near list is read once for all of them, and one warp vote
// serves the window's close-pass test.
//
// The bound.  Along the row the walk's value X(u) (and Y(u)) is the FP32
// evaluation of F(u) = P(u) + sum_q (lx_q - u) m_q / ((lx_q - u)^2 + dy2_q)
// (Y: the terms dyy_q m_q / (...)), with P the row polynomial and the FP32
// lens constants taken as exact reals.  For a ray between a and b:
//  - rounding: |X - F| <= E = c eps (S_P + sum_q m_q / rho_q), with
//    S_P = sum |C_m| U^m (U the lane's largest |u|), eps = 2^-24, rho_q the
//    lens's smallest distance to the span's rays and c = 2 (P + nn + 8), at
//    least twice the count of roundings on the path (Horner FMAs, per lens
//    the offset, r^2, reciprocal, mass product and accumulation);
//  - shape: F lies within K = (b - a)^2 / 8 max|F''| of the chord between
//    F(a) and F(b), with |F''| <= sum m(m-1) |C_m| U^(m-2) + sum_q 2 m_q / rho_q^3
//    (Y: 6 m_q |dyy_q| / rho_q^4): with r^2 = x^2 + dy2 and c = x / r, a
//    lens's term m x / r^2 has second derivative (2 m / r^3) c (4 c^2 - 3),
//    and |4 c^3 - 3 c| <= 1 on [-1, 1] (the Chebyshev polynomial T_3); its y
//    term m dyy / r^2 has (m dyy / r^4) (8 c^2 - 2), at most 6 in size;
//  - so X lies in [min(X_a, X_b) - 2E - K, max(X_a, X_b) + 2E + K] (margin
//    widened by 1 %, ends rounded outwards); if that interval has one floor,
//    and the same holds for Y, every ray between shares the anchor's pixel;
//  - when |X_b - X_a| - 2E > (b - a)^2 max|F''| (= 8K), F' has one sign on
//    the span (it is within (b - a) max|F''| of the chord's slope, by the
//    mean value theorem), so F is monotone, lies between F(a) and F(b), and
//    the interval needs no K: near a pixel edge, spans several times longer
//    pass.
// A span whose rays could come within the close-pass radius of a lens is never
// certified (those rays would take the hi/lo arithmetic), and anchors outside
// |X|, |Y| < 2^21 (rays dropped on a lens) are never certified from.
template <int P, int NN>
__device__ __forceinline__ void walk_span(const RowPoly<P> &rp, const ShootArgs &a, const SmemNear &nl,
                                          int nn_dyn, int k0, int k1, float dyl, float dyl_lo,
                                          RunState &rs, unsigned &drop, SpanCount &sc)
{
    constexpr int W = ML_SPAN_W;                // rays evaluated per step
    constexpr bool REG = NN < NN_DYN;
    constexpr int NR = (REG && NN > 0) ? NN : 1;
    float lx[NR], lm[NR], dy2[NR], dyy[NR];
    if constexpr (REG) {
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const float4 L = nl.near[q];
            lx[q] = L.x;
            lm[q] = L.z;
            const float dy = __fsub_rn(L.y, dyl);
            dy2[q] = __fmul_rn(dy, dy);
            dyy[q] = __fmul_rn(dy, a.yx_f);
        }
    }
    const int nlen = REG ? NN : nn_dyn;
    // record q of the near list: the registers, or shared memory with the
    // per-lane terms formed as near_sum_lat forms them
    auto rec = [&](int q, float &x, float &m, float &d2, float &dd) {
        if constexpr (REG) {
            x = lx[q]; m = lm[q]; d2 = dy2[q]; dd = dyy[q];
        } else {
            const float4 L = nl.near[q];
            const float dy = __fsub_rn(L.y, dyl);
            x = L.x; m = L.z; d2 = __fmul_rn(dy, dy); dd = __fmul_rn(dy, a.yx_f);
        }
    };
    f32x2 C[P + 1];
#pragma unroll
    for (int m = 0; m <= P; ++m) C[m] = pack2(rp.X[m], rp.Y[m]);
    const f32x2 MAGIC = pack2(12582912.0f, 12582912.0f);
    constexpr float LIM = 2097152.0f;           // 2^21

    // source positions of rays kb .. kb+W-1 by the per-ray arithmetic, in raw
    // floor form; dr[r] marks a ray on a lens (sent far outside the map, as
    // walk_fixed does).  Called by all lanes together (the close-pass branch
    // is taken by warp vote); av[r] says which rays the lane will use.
    float X[W], Y[W];
    unsigned rx[W], ry[W];
    bool dr[W];
    auto eval_window = [&](int kb, const bool (&av)[W]) {
        float u[W];
        f32x2 v[W];
#pragma unroll
        for (int r = 0; r < W; ++r) {
            u[r] = __fadd_rn((float)(kb + r), a.c0_f);
            v[r] = C[P];
        }
#pragma unroll
        for (int m = P - 1; m >= 0; --m) {
#pragma unroll
            for (int r = 0; r < W; ++r) v[r] = fma2(v[r], pack2(u[r], u[r]), C[m]);
        }
#pragma unroll
        for (int r = 0; r < W; ++r) {
            unpack2(v[r], X[r], Y[r]);
            dr[r] = false;
        }
        // (nlen is warp-uniform: an empty near list skips the lens loop and its vote)
        if (!(REG && NN == 0) && nlen > 0) {
            float mn[W];
#pragma unroll
            for (int r = 0; r < W; ++r) mn[r] = 3.0e38f;
            auto lens = [&](int q) {
                float x, m, d2, dd;
                rec(q, x, m, d2, dd);
#pragma unroll
                for (int r = 0; r < W; ++r) {
                    const float dx = __fsub_rn(x, u[r]);
                    const float r2 = __fmaf_rn(dx, dx, d2);
                    mn[r] = fminf(mn[r], r2);
                    const float sv = __fmul_rn(m, rcp_approx(r2));
                    X[r] = __fmaf_rn(dx, sv, X[r]);
                    Y[r] = __fmaf_rn(dd, sv, Y[r]);
                }
            };
            if constexpr (REG) {
#pragma unroll
                for (int q = 0; q < NR; ++q) lens(q);
            } else {
                for (int q = 0; q < nlen; ++q) lens(q);
            }
            bool cl[W], any = false;
#pragma unroll
            for (int r = 0; r < W; ++r) {
                cl[r] = av[r] && mn[r] < a.rc2u;
                any |= cl[r];
            }
            if (__any_sync(0xffffffffu, any)) {
                // rare: one copy of the hi/lo path, the window rotated through slot 0
#pragma unroll 1
                for (int i = 0; i < W; ++i) {
                    if (cl[0]) {
                        unpack2(v[0], X[0], Y[0]);
                        if (!near_sum_hilo_lat(nl, nlen, u[0], dyl, dyl_lo, a.yx_f, X[0], Y[0])) {
                            X[0] = -1.0e30f;
                            dr[0] = true;
                        }
                    }
                    const float u0 = u[0], X0 = X[0], Y0 = Y[0];
                    const f32x2 v0 = v[0];
                    const bool c0 = cl[0], d0 = dr[0];
#pragma unroll
                    for (int r = 0; r + 1 < W; ++r) {
                        u[r] = u[r + 1]; X[r] = X[r + 1]; Y[r] = Y[r + 1];
                        v[r] = v[r + 1]; cl[r] = cl[r + 1]; dr[r] = dr[r + 1];
                    }
                    u[W - 1] = u0; X[W - 1] = X0; Y[W - 1] = Y0;
                    v[W - 1] = v0; cl[W - 1] = c0; dr[W - 1] = d0;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < W; ++r) {
            float fx, fy;
            unpack2(add2_rd(pack2(X[r], Y[r]), MAGIC), fx, fy);
            rx[r] = (unsigned)__float_as_int(fx);
            ry[r] = (unsigned)__float_as_int(fy);
        }
    };

    // bounds of the row polynomial over the lane's range: S = sum |C_m| U^m,
    // Q = sum_{m>=2} m (m-1) |C_m| U^(m-2), rounded upwards
    const bool on = k1 > k0;
    const float ulo = __fadd_rn((float)k0, a.c0_f);
    const float uhi = __fadd_rn((float)(on ? k1 - 1 : k0), a.c0_f);
    const float Um = fmaxf(fabsf(ulo), fabsf(uhi));
    float SX = fabsf(rp.X[P]), SY = fabsf(rp.Y[P]);
#pragma unroll
    for (int m = P - 1; m >= 0; --m) {
        SX = __fmaf_ru(SX, Um, fabsf(rp.X[m]));
        SY = __fmaf_ru(SY, Um, fabsf(rp.Y[m]));
    }
    float QX = 0.f, QY = 0.f;
    if constexpr (P >= 2) {
        QX = (float)(P * (P - 1)) * fabsf(rp.X[P]);
        QY = (float)(P * (P - 1)) * fabsf(rp.Y[P]);
#pragma unroll
        for (int m = P - 1; m >= 2; --m) {
            QX = __fmaf_ru(QX, Um, (float)(m * (m - 1)) * fabsf(rp.X[m]));
            QY = __fmaf_ru(QY, Um, (float)(m * (m - 1)) * fabsf(rp.Y[m]));
        }
    }
    const float rcut = __fmaf_ru(1.01f, a.rc2u, 1e-30f);
    // 2 c eps: twice the rounding bound's factor (see above)
    const float c2e = (float)(4 * (P + 8 + nlen)) * 5.9604645e-8f;

    auto certify = [&](int ka, int kb, float Xa, float Ya, float Xb, float Yb) {
        if (!(fabsf(Xa) < LIM && fabsf(Xb) < LIM && fabsf(Ya) < LIM && fabsf(Yb) < LIM)) return false;
        const float ua = __fadd_rn((float)ka, a.c0_f), ub = __fadd_rn((float)kb, a.c0_f);
        float tX = 0.f, tY = 0.f, cX = QX, cY = QY;
        bool clear = true;
        if (!(REG && NN == 0) && nlen > 0) {
            auto lens = [&](int q) {
                float x, m, d2, dd;
                rec(q, x, m, d2, dd);
                const float dist = fmaxf(0.f, fmaxf(__fsub_rd(ua, x), __fsub_rd(x, ub)));
                const float rho2 = __fmaf_rd(dist, dist, d2);
                clear &= rho2 > rcut;
                const float ir2 = rcp_approx(rho2), ir = rsqrt_approx(rho2);
                const float mr = m * ir, md = m * fabsf(dd);
                tX += mr;
                tY = fmaf(md, ir2, tY);
                cX = fmaf(2.f * mr, ir2, cX);
                cY = fmaf(6.f * md, ir2 * ir2, cY);
            };
            if constexpr (REG) {
#pragma unroll
                for (int q = 0; q < NR; ++q) lens(q);
            } else {
                for (int q = 0; q < nlen; ++q) lens(q);
            }
        }
        const float w = __fsub_rn(ub, ua);
        const float kk = 0.125f * w * w;
        // 2E and K of each component; where the chord's rise exceeds what the
        // curvature can undo over the span, |F(b) - F(a)| - 2E > (b - a)^2
        // max|F''| = 8K, F' keeps one sign (mean value theorem), F lies
        // between F(a) and F(b), and K is not needed
        const float eX = c2e * (SX + tX), eY = c2e * (SY + tY);
        const float kX = kk * cX, kY = kk * cY;
        const bool monoX = __fsub_rd(__fmul_rd(fabsf(__fsub_rn(Xb, Xa)), 0.9999998f), eX) > 8.1f * kX;
        const bool monoY = __fsub_rd(__fmul_rd(fabsf(__fsub_rn(Yb, Ya)), 0.9999998f), eY) > 8.1f * kY;
        const float MX = 1.01f * (monoX ? eX : eX + kX);
        const float MY = 1.01f * (monoY ? eY : eY + kY);
        const bool okx = floor_to_int(__fsub_rd(fminf(Xa, Xb), MX)) == floor_to_int(__fadd_ru(fmaxf(Xa, Xb), MX));
        const bool oky = floor_to_int(__fsub_rd(fminf(Ya, Yb), MY)) == floor_to_int(__fadd_ru(fmaxf(Ya, Yb), MY));
        return clear && okx && oky;
    };

    const Geo &g = a.g;
    const unsigned offx = (unsigned)rp.bx - 0x4B400000u, offy = (unsigned)rp.by - 0x4B400000u;
    unsigned rcx = (unsigned)rs.cx - offx, rcy = (unsigned)rs.cy - offy;   // run pixel, raw form
    int kst = k0;                 // first ray of the current run in this walk
    int ka = k0 - 1;              // last evaluated ray (none yet)
    float Xa = 0.f, Ya = 0.f;
    int gap = 1;                  // next window at ka + gap
    unsigned ev = 0, spn = 0;     // this column's evaluations and certified spans
    for (;;) {
        const bool act = on && ka + 1 < k1;
        if (!__any_sync(0xffffffffu, act)) break;
        const int kb = act ? min(ka + gap, k1 - 1) : ka + 1;
        const bool span = act && kb > ka + 1;
        bool av[W];
#pragma unroll
        for (int r = 0; r < W; ++r) av[r] = act && kb + r < k1;
        eval_window(kb, av);
        bool ok = act;
        if (span) {
            const bool same = rx[0] == rcx && ry[0] == rcy;
            ok = same && certify(ka, kb, Xa, Ya, X[0], Y[0]);
            spn += ok ? 1u : 0u;
            if (!ok) {
                ++ev;
                // ray kb is past a pixel edge: the next window starts where the
                // chord from ka crosses it; otherwise the bound failed, and the
                // gap halves
                int g2 = (kb - ka) >> 1;
                if (!same && fabsf(Xa) < LIM && fabsf(X[0]) < LIM && fabsf(Ya) < LIM && fabsf(Y[0]) < LIM) {
                    float t = 1.f;
                    const float fa = __fsub_rn(__int_as_float((int)rcx), 12582912.0f);
                    const float ga = __fsub_rn(__int_as_float((int)rcy), 12582912.0f);
                    if (rx[0] != rcx) {
                        const float e = X[0] > Xa ? __fadd_rn(fa, 1.f) : fa;
                        t = fminf(t, __fsub_rn(e, Xa) * rcp_approx(__fsub_rn(X[0], Xa)));
                    }
                    if (ry[0] != rcy) {
                        const float e = Y[0] > Ya ? __fadd_rn(ga, 1.f) : ga;
                        t = fminf(t, __fsub_rn(e, Ya) * rcp_approx(__fsub_rn(Y[0], Ya)));
                    }
                    g2 = floor_to_int(fmaxf(t, 0.f) * (float)(kb - ka) - ML_SPAN_MARGIN);
                }
                gap = max(1, min(g2, kb - ka - 1));
            }
        }
        if (ok) {
            // slope baseline: the last evaluated ray, or at the column's start
            // the window's first ray
            const int kp = ka < k0 ? kb : ka;
            const float Xp = ka < k0 ? X[0] : Xa, Yp = ka < k0 ? Y[0] : Ya;
#pragma unroll
            for (int r = 0; r < W; ++r) {
                if (av[r]) {
                    ++ev;
                    if (dr[r]) ++drop;
                    if (rx[r] != rcx || ry[r] != rcy) {
                        flush_run(rs, (int)(rcx + offx), (int)(rcy + offy), rs.cnt + (unsigned)(kb + r - kst),
                                  a.map_u32, g.mnx, g.mny);
                        rs.cnt = 0;
                        kst = kb + r;
                        rcx = rx[r];
                        rcy = ry[r];
                    }
                    ka = kb + r;
                    Xa = X[r];
                    Ya = Y[r];
                }
            }
            // rays to the next pixel edge along the slope since the baseline;
            // the next window starts ML_SPAN_MARGIN rays before it
            gap = 1;
            if (ka > kp && fabsf(Xa) < LIM && fabsf(Ya) < LIM && fabsf(Xp) < LIM && fabsf(Yp) < LIM) {
                // (one reciprocal per component on the step's critical path)
                const float fk = (float)(ka - kp);
                const float dX = __fsub_rn(Xa, Xp), dY = __fsub_rn(Ya, Yp);
                const float fX = __fsub_rn(Xa, __fsub_rn(__int_as_float((int)rcx), 12582912.0f));
                const float fY = __fsub_rn(Ya, __fsub_rn(__int_as_float((int)rcy), 12582912.0f));
                const float gX = (dX > 0.f ? __fsub_rn(1.f, fX) : fX) * fk;
                const float gY = (dY > 0.f ? __fsub_rn(1.f, fY) : fY) * fk;
                const float n = fminf(fminf(gX * rcp_approx(fabsf(dX)), gY * rcp_approx(fabsf(dY))), 1048576.f);
                gap = max(1, floor_to_int(n - ML_SPAN_MARGIN));
            }
        }
    }
    if (on) rs.cnt += (unsigned)(k1 - kst);
    rs.cx = (int)(rcx + offx);
    rs.cy = (int)(rcy + offy);
    sc.evals += ev;
    sc.spans += spn;
}

// Keeps a value in a register: the compiler may not recompute it (it would
// otherwise rebuild FP64-derived constants inside the walk, and FP64
// arithmetic is slow on this GPU).
__device__ __forceinline__ float pin(float v)
{
    asm volatile("" : "+f"(v));
    return v;
}

// One warp task of the mixed kernel (NGP deposit): stage the near list, then
// walk each level-2 column of the task.  Shared by the single-map and the
// batched persistent kernels.
// SPAN: 0 the per-ray walk only; 1 the certified walk in one copy for every
// near-list length; 2 the same with a second copy for empty near lists.
template <int P, int SPAN>
__device__ __forceinline__ void shoot_task(const ShootArgs &a, int64_t t, float4 *near, float2 *nlo,
                                           int lane, float dyl, float dyl_lo, RunState &rs,
                                           unsigned &drop, unsigned long long &pairs,
                                           unsigned long long &tasks, SpanCount &sc)
{
    const Geo &g = a.g;
    TaskShape ts;
    if (!decode_task(a, t, ts)) return;
    ++tasks;
    const SmemNear nl{near, nlo};
    const int64_t jb = a.ray_begin / g.n3x, ib = a.ray_begin % g.n3x;
    const int64_t je = (a.ray_end - 1) / g.n3x, ie = (a.ray_end - 1) % g.n3x + 1;
    const NearRuns nr = near_runs(a, ts.c1x, ts.c1y);
    const double yref = g.ry0 + ((double)ts.row0 + 0.5) * g.l3y;
    const int nn = stage_near_y<true>(a, nr, yref, near, nlo, lane);
    const int64_t j = ts.row0 + lane;
    const bool active = j < ts.rows_end && j >= jb && j <= je;
    const int64_t c2y = j / g.n2y;
    const float q = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
    const RowY ry = row_y(q, a);
    for (int64_t c2x = ts.c2a; c2x < ts.c2b; ++c2x) {
        stage_near_x<true>(a, nn, g.rx0 + ((double)c2x + 0.5) * g.l2x, near, nlo, lane);
        const int64_t i0 = c2x * g.n2x;
        int k0 = 0, k1 = (int)(min(i0 + g.n2x, g.n3x) - i0);
        if (j == jb) k0 = max(k0, (int)max((int64_t)0, ib - i0));
        if (j == je) k1 = min(k1, (int)max((int64_t)0, ie - i0));
        if (!active || k0 >= k1) { k0 = 0; k1 = 0; }
        // warp-uniform walk range: the union of the lanes' ranges
        const int kbeg = __reduce_min_sync(0xffffffffu, k1 > k0 ? k0 : 0x7fffffff);
        const int kend = __reduce_max_sync(0xffffffffu, k1);
        if (kbeg >= kend) continue;
        RowPoly<P> rp;
        row_setup<P>(a.nodes + (min(c2y, g.N2y - 1) * g.N2x + c2x) * node_stride(P), q, ry, a, rp);
        pairs += (unsigned long long)nn * (unsigned long long)(k1 - k0);
        if constexpr (SPAN) {
            // the certified walk where runs are long: no near lens, or every
            // near lens farther than a.span_far lattice units from every ray
            // of the warp's walk; elsewhere the per-ray walk
            bool far = true;
            if (nn > 0) {
                bool close = false;
                if (k1 > k0) {
                    const float ulo = __fadd_rn((float)k0, a.c0_f), uhi = __fadd_rn((float)(k1 - 1), a.c0_f);
                    for (int q = 0; q < nn; ++q) {
                        const float4 L = near[q];
                        const float dy = __fsub_rn(L.y, dyl);
                        const float dx = fmaxf(0.f, fmaxf(ulo - L.x, L.x - uhi));
                        close |= __fmaf_rn(dx, dx, dy * dy) < a.span_far * a.span_far;
                    }
                }
                far = !__any_sync(0xffffffffu, close);
            }
            if (far) {
                // one copy of the walk for every near-list length (its lens loops
                // run from shared memory) in the single-map kernel, where a second
                // copy for empty lists measured slower, its code competing for the
                // instruction cache; the batch kernel, whose lens-dense maps walk
                // most lens columns ray by ray, measured faster with it
                if (SPAN == 2 && nn == 0)
                    walk_span<P, 0>(rp, a, nl, nn, k0, k1, dyl, dyl_lo, rs, drop, sc);
                else
                    walk_span<P, NN_DYN>(rp, a, nl, nn, k0, k1, dyl, dyl_lo, rs, drop, sc);
                continue;
            }
        }
        {
        sc.evals += (unsigned long long)(k1 - k0);
        const bool on = k1 > k0;
        const bool uniform = !__any_sync(0xffffffffu, on && (k0 != kbeg || k1 != kend));
        if (uniform && nn <= 4) {
            // can a ray of this walk pass within the close-pass radius of a lens?
            // (distance from each lens to the row's ray segment, 1 % margin
            // against the FP32 rounding of the per-ray r^2)
            bool close = false;
            if (on) {
                const float ulo = __fadd_rn((float)kbeg, a.c0_f);
                const float uhi = __fadd_rn((float)(kend - 1), a.c0_f);
                for (int q = 0; q < nn; ++q) {
                    const float4 L = near[q];
                    const float dy = __fsub_rn(L.y, dyl);
                    const float dx = fmaxf(0.f, fmaxf(ulo - L.x, L.x - uhi));
                    close |= __fmaf_rn(dx, dx, dy * dy) <= 1.01f * a.rc2u + 1e-30f;
                }
            }
            if (__any_sync(0xffffffffu, close)) {
                switch (nn) {
                case 0: walk_fixed<P, 0, false>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                case 1: walk_fixed<P, 1, true>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                case 2: walk_fixed<P, 2, true>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                case 3: walk_fixed<P, 3, true>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                default: walk_fixed<P, 4, true>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                }
            } else {
                switch (nn) {
                case 0: walk_fixed<P, 0, false>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                case 1: walk_fixed<P, 1, false>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                case 2: walk_fixed<P, 2, false>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                case 3: walk_fixed<P, 3, false>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                default: walk_fixed<P, 4, false>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, rs, drop); break;
                }
            }
        } else {
            walk_any<P>(rp, a, nl, nn, kbeg, kend, k0, k1, dyl, dyl_lo, rs, drop);
        }
        }
    }
}

// Lane offset from a task's first row in lattice units, lane * l3y / l3x
// rounded once from FP64, and its remainder.
__device__ __forceinline__ void lane_dy(double l3yx, int lane, float &dyl, float &dyl_lo)
{
    const double d = (double)lane * l3yx;
    dyl = pin((float)d);
    dyl_lo = pin((float)(d - (double)(float)d));
}

template <int P, bool SPAN>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, ML_MIN_BLOCKS) k_shoot_mixed(ShootArgs a)
{
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *near = smem + wid * a.near_cap;
    float2 *nlo = reinterpret_cast<float2 *>(smem + WARPS_PER_CTA * a.near_cap) + wid * a.near_cap;
    RunState rs{-1, -1, 0u, 0u, 0u};
    unsigned drop = 0;
    unsigned long long pairs = 0, tasks = 0;
    SpanCount sc;
    float dyl, dyl_lo;
    lane_dy(a.l3yx, lane, dyl, dyl_lo);
    for (;;) {
        bool stop;
        const int64_t t = fetch_task(a, lane, stop);
        if (stop || t >= a.n_tasks) break;
        shoot_task<P, SPAN ? 1 : 0>(a, t, near, nlo, lane, dyl, dyl_lo, rs, drop, pairs, tasks, sc);
    }
    run_flush(rs, a.map_u32, a.g.mnx, a.g.mny);
    // dropped rays were sent far outside the map and counted as out above
    flush_stats(a, rs.in, rs.out - drop, drop, pairs, lane == 0 ? tasks : 0, 0u);
    flush_spans(a, sc);
}

// Batched persistent kernel: one launch over the tasks of many maps (all
// built with the same Taylor order P).  Global task t belongs to the map m
// with task_base[m] <= t < task_base[m+1]; a warp flushes its runs and
// counters into a map's buffers when it moves on to another map.
template <int P, bool SPAN>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, ML_MIN_BLOCKS) k_shoot_batch(BatchArgs b)
{
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *near = smem + wid * b.near_cap;
    float2 *nlo = reinterpret_cast<float2 *>(smem + WARPS_PER_CTA * b.near_cap) + wid * b.near_cap;
    RunState rs{-1, -1, 0u, 0u, 0u};
    unsigned drop = 0;
    unsigned long long pairs = 0, tasks = 0;
    SpanCount sc;
    float dyl = 0.f, dyl_lo = 0.f;
    int cur = -1;
    const int64_t total = b.task_base[b.n_maps];
    for (;;) {
        long long t = 0;
        int ab = 0;
        if (lane == 0) {
            t = (long long)atomicAdd(b.work, 1ull);
            ab = *b.abort_flag;
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        ab = __shfl_sync(0xffffffffu, ab, 0);
        if (ab) {
            if (lane == 0) atomicOr(b.status, 2u);
            break;
        }
        if (t >= total) break;
        int lo = 0, hi = b.n_maps;            // last m with task_base[m] <= t
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (b.task_base[mid] <= t) lo = mid; else hi = mid;
        }
        if (lo != cur) {
            if (cur >= 0) {
                const ShootArgs &ac = b.args[cur];
                run_flush(rs, ac.map_u32, ac.g.mnx, ac.g.mny);
                flush_stats(ac, rs.in, rs.out - drop, drop, pairs, lane == 0 ? tasks : 0, 0u);
                flush_spans(ac, sc);
                rs = RunState{-1, -1, 0u, 0u, 0u};
                drop = 0;
                pairs = 0;
                tasks = 0;
                sc = SpanCount{};
            }
            cur = lo;
            lane_dy(b.args[cur].l3yx, lane, dyl, dyl_lo);
        }
        shoot_task<P, SPAN ? 2 : 0>(b.args[cur], t - b.task_base[cur], near, nlo, lane, dyl, dyl_lo, rs,
                                    drop, pairs, tasks, sc);
    }
    if (cur >= 0) {
        const ShootArgs &ac = b.args[cur];
        run_flush(rs, ac.map_u32, ac.g.mnx, ac.g.mny);
        flush_stats(ac, rs.in, rs.out - drop, drop, pairs, lane == 0 ? tasks : 0, 0u);
        flush_spans(ac, sc);
    }
}

// Cloud-in-cell variant: a float map.  A ray's bilinear weights go to the
// four pixel centres around it; consecutive rays of a lane that share those
// four pixels (the macro map compresses x) have their weights summed in
// registers, and the run is added with four atomics when the quad changes.
struct CicRun {
    unsigned qx = 0xFFFFFFFFu, qy = 0xFFFFFFFFu;   // lower-left pixel of the quad
    unsigned rc = 0;                               // rays of the run
    float W0 = 0.f, W1 = 0.f, W2 = 0.f, W3 = 0.f;  // summed weights
    unsigned in = 0, out = 0;
};

__device__ __forceinline__ void cic_flush(CicRun &r, float *map, unsigned mnx, unsigned mny)
{
    if (r.rc == 0) return;
    bool any = false;
    // the quad's second column and row, in wrapping 32-bit arithmetic
    // (qx = 0xFFFFFFFF is the column left of the map, whose neighbour is 0)
    const unsigned px1 = r.qx + 1u, py1 = r.qy + 1u;
    const bool x0 = r.qx < mnx, x1 = px1 < mnx, y0 = r.qy < mny, y1 = py1 < mny;
    if (x0 && y0) { atomicAdd(map + ((size_t)r.qy * mnx + r.qx), r.W0); any = true; }
    if (x1 && y0) { atomicAdd(map + ((size_t)r.qy * mnx + px1), r.W1); any = true; }
    if (x0 && y1) { atomicAdd(map + ((size_t)py1 * mnx + r.qx), r.W2); any = true; }
    if (x1 && y1) { atomicAdd(map + ((size_t)py1 * mnx + px1), r.W3); any = true; }
    if (any) r.in += r.rc; else r.out += r.rc;
}

__device__ __forceinline__ void cic_start(CicRun &r, unsigned ix, unsigned iy)
{
    r.qx = ix;
    r.qy = iy;
    r.W0 = r.W1 = r.W2 = r.W3 = 0.f;
    r.rc = 0;
}

__device__ __forceinline__ void cic_add(CicRun &r, float wx, float wy)
{
    const float ox = 1.f - wx, oy = 1.f - wy;
    r.W0 = __fmaf_rn(ox, oy, r.W0);
    r.W1 = __fmaf_rn(wx, oy, r.W1);
    r.W2 = __fmaf_rn(ox, wy, r.W2);
    r.W3 = __fmaf_rn(wx, wy, r.W3);
    ++r.rc;
}

// One level-2 column of the CIC walk when every active lane covers the
// warp's whole range and the near list has NN <= 4 lenses (in registers).
// Pairs of rays (the second masked off after an odd last ray), one warp vote
// per pair before any flush.  Per ray the arithmetic is exactly
// near_sum_f32's, near_sum_hilo's and row_eval's, as the adjoint recomputes.
template <int P, int NN>
__device__ __forceinline__ void cic_walk(const RowPoly<P> &rp, const ShootArgs &a, const SmemNear &nl,
                                         int kbeg, int kend, bool on, float dyl, float dyl_lo,
                                         CicRun &cr, unsigned &drop)
{
    float lx[NN > 0 ? NN : 1], lm[NN > 0 ? NN : 1], dy[NN > 0 ? NN : 1], dy2[NN > 0 ? NN : 1];
#pragma unroll
    for (int q = 0; q < NN; ++q) {
        const float4 L = nl.near[q];
        lx[q] = L.x;
        lm[q] = L.z;
        dy[q] = __fsub_rn(dyl, L.y);
        dy2[q] = __fmul_rn(dy[q], dy[q]);
    }
    const unsigned mnx = (unsigned)a.g.mnx, mny = (unsigned)a.g.mny;
    // row polynomial as (X, Y) pairs for two-lane FMAs (row_eval's arithmetic)
    f32x2 C[P + 1];
#pragma unroll
    for (int m = 0; m <= P; ++m) C[m] = pack2(rp.X[m], rp.Y[m]);
    auto poly = [&](f32x2 U) {
        f32x2 v = C[P];
#pragma unroll
        for (int m = P - 1; m >= 0; --m) v = fma2(v, U, C[m]);
        return v;
    };
    const f32x2 TWO = pack2(2.f, 2.f);
    auto near = [&](float t, float &sx, float &sy, float &mn) {
        sx = 0.f; sy = 0.f; mn = 3.0e38f;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const float dx = __fsub_rn(t, lx[q]);
            const float r2 = __fmaf_rn(dx, dx, dy2[q]);
            mn = fminf(mn, r2);
            const float sv = __fmul_rn(lm[q], rcp_approx(r2));
            sx = __fmaf_rn(dx, sv, sx);
            sy = __fmaf_rn(dy[q], sv, sy);
        }
    };
    const float ub = __fadd_rn((float)kbeg, a.c0_f), ub1 = __fadd_rn(ub, 1.f);
    f32x2 U0 = pack2(ub, ub), U1 = pack2(ub1, ub1);
    for (int k = kbeg; k < kend; k += 2, U0 = add2(U0, TWO), U1 = add2(U1, TWO)) {
        float u, u1, uh;
        unpack2(U0, u, uh);
        unpack2(U1, u1, uh);
        bool v0 = on, v1 = on && k + 1 < kend;
        const float t0 = __fmul_rn(u, a.l3x_f), t1 = __fmul_rn(u1, a.l3x_f);
        float X0, Y0, X1, Y1, sx0, sy0, mn0, sx1, sy1, mn1;
        unpack2(poly(U0), X0, Y0);
        unpack2(poly(U1), X1, Y1);
        near(t0, sx0, sy0, mn0);
        near(t1, sx1, sy1, mn1);
        if (NN > 0) {
            const bool c0 = v0 && mn0 < a.rc2, c1 = v1 && mn1 < a.rc2;
            if (__ballot_sync(0xffffffffu, c0 || c1)) {
                if (c0 && !near_sum_hilo(nl, NN, u, t0, dyl, dyl_lo, a.l3x_f, a.l3x_lo, sx0, sy0)) {
                    v0 = false;
                    ++drop;
                }
                if (c1 && !near_sum_hilo(nl, NN, u1, t1, dyl, dyl_lo, a.l3x_f, a.l3x_lo, sx1, sy1)) {
                    v1 = false;
                    ++drop;
                }
            }
        }
        X0 = __fmaf_rn(-sx0, a.ipx_f, X0);
        Y0 = __fmaf_rn(-sy0, a.ipy_f, Y0);
        X1 = __fmaf_rn(-sx1, a.ipx_f, X1);
        Y1 = __fmaf_rn(-sy1, a.ipy_f, Y1);
        unsigned ix0, iy0, ix1, iy1;
        float wx0, wy0, wx1, wy1;
        cic_quad(rp.bx, rp.by, X0, Y0, ix0, iy0, wx0, wy0);
        cic_quad(rp.bx, rp.by, X1, Y1, ix1, iy1, wx1, wy1);
        // ray 1 compares with the quad after ray 0
        const bool ch0 = v0 && (ix0 != cr.qx || iy0 != cr.qy);
        const bool ch1 = v1 && (ix1 != (v0 ? ix0 : cr.qx) || iy1 != (v0 ? iy0 : cr.qy));
        const bool any = __ballot_sync(0xffffffffu, ch0 || ch1) != 0u;
        if (any && ch0) {
            cic_flush(cr, a.map_f32, mnx, mny);
            cic_start(cr, ix0, iy0);
        }
        if (v0) cic_add(cr, wx0, wy0);
        if (any && ch1) {
            cic_flush(cr, a.map_f32, mnx, mny);
            cic_start(cr, ix1, iy1);
        }
        if (v1) cic_add(cr, wx1, wy1);
    }
}

template <int P>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, ML_MIN_BLOCKS) k_shoot_mixed_cic(ShootArgs a)
{
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *near = smem + wid * a.near_cap;
    float2 *nlo = reinterpret_cast<float2 *>(smem + WARPS_PER_CTA * a.near_cap) + wid * a.near_cap;
    const SmemNear nl{near, nlo};
    const Geo &g = a.g;
    const int64_t jb = a.ray_begin / g.n3x, ib = a.ray_begin % g.n3x;
    const int64_t je = (a.ray_end - 1) / g.n3x, ie = (a.ray_end - 1) % g.n3x + 1;
    unsigned drop = 0;
    unsigned long long pairs = 0, tasks = 0;
    CicRun cr;
    const unsigned mnx = (unsigned)g.mnx, mny = (unsigned)g.mny;
    const double dyl_d = (double)lane * g.l3y;
    const float dyl = pin((float)dyl_d);
    const float dyl_lo = pin((float)(dyl_d - (double)(float)dyl_d));
    for (;;) {
        bool stop;
        const int64_t t = fetch_task(a, lane, stop);
        if (stop || t >= a.n_tasks) break;
        TaskShape ts;
        if (!decode_task(a, t, ts)) continue;
        ++tasks;
        const NearRuns nr = near_runs(a, ts.c1x, ts.c1y);
        const double yref = g.ry0 + ((double)ts.row0 + 0.5) * g.l3y;
        const int nn = stage_near_y<false>(a, nr, yref, near, nlo, lane);
        const int64_t j = ts.row0 + lane;
        const bool active = j < ts.rows_end && j >= jb && j <= je;
        const int64_t c2y = j / g.n2y;
        const float q = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
        const RowY ry = row_y(q, a);
        for (int64_t c2x = ts.c2a; c2x < ts.c2b; ++c2x) {
            stage_near_x<false>(a, nn, g.rx0 + ((double)c2x + 0.5) * g.l2x, near, nlo, lane);
            const int64_t i0 = c2x * g.n2x;
            int k0 = 0, k1 = (int)(min(i0 + g.n2x, g.n3x) - i0);
            if (j == jb) k0 = max(k0, (int)max((int64_t)0, ib - i0));
            if (j == je) k1 = min(k1, (int)max((int64_t)0, ie - i0));
            if (!active || k0 >= k1) { k0 = 0; k1 = 0; }
            const int kbeg = __reduce_min_sync(0xffffffffu, k1 > k0 ? k0 : 0x7fffffff);
            const int kend = __reduce_max_sync(0xffffffffu, k1);
            if (kbeg >= kend) continue;
            RowPoly<P> rp;
            row_setup<P>(a.nodes + (min(c2y, g.N2y - 1) * g.N2x + c2x) * node_stride(P), q, ry, a, rp);
            pairs += (unsigned long long)nn * (unsigned long long)(k1 - k0);
            const bool on = k1 > k0;
            const bool uniform = !__any_sync(0xffffffffu, on && (k0 != kbeg || k1 != kend));
            if (uniform && nn <= 4) {
                switch (nn) {
                case 0: cic_walk<P, 0>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, cr, drop); break;
                case 1: cic_walk<P, 1>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, cr, drop); break;
                case 2: cic_walk<P, 2>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, cr, drop); break;
                case 3: cic_walk<P, 3>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, cr, drop); break;
                default: cic_walk<P, 4>(rp, a, nl, kbeg, kend, on, dyl, dyl_lo, cr, drop); break;
                }
                continue;
            }
            if (!on) continue;
            // any near-list length, ragged ranges: one ray at a time
            float u = __fadd_rn((float)k0, a.c0_f);
            for (int k = k0; k < k1; ++k, u += 1.f) {
                const float t0 = __fmul_rn(u, a.l3x_f);
                float X, Y, ax, ay, mn;
                row_eval<P>(rp, u, X, Y);
                near_sum_f32(nl, nn, t0, dyl, ax, ay, mn);
                bool ok = true;
                if (mn < a.rc2) ok = near_sum_hilo(nl, nn, u, t0, dyl, dyl_lo, a.l3x_f, a.l3x_lo, ax, ay);
                if (!ok) { ++drop; continue; }
                X = __fmaf_rn(-ax, a.ipx_f, X);
                Y = __fmaf_rn(-ay, a.ipy_f, Y);
                unsigned ix, iy;
                float wx, wy;
                cic_quad(rp.bx, rp.by, X, Y, ix, iy, wx, wy);
                if (ix != cr.qx || iy != cr.qy) {
                    cic_flush(cr, a.map_f32, mnx, mny);
                    cic_start(cr, ix, iy);
                }
                cic_add(cr, wx, wy);
            }
        }
    }
    cic_flush(cr, a.map_f32, mnx, mny);
    flush_stats(a, cr.in, cr.out, drop, pairs, lane == 0 ? tasks : 0, 0u);
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
    const double dyl_d = (double)(j - row0) * a.l3yx;
    const float dyl = (float)dyl_d;
    const float dyl_lo = (float)(dyl_d - (double)dyl);
    float qf = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
    RowPoly<P> rp;
    row_setup<P>(a.nodes + (c2y * g.N2x + c2x) * node_stride(P), qf, row_y(qf, a), a, rp);
    float u = __fadd_rn((float)(i - c2x * g.n2x), a.c0_f);
    float X, Y, mn;
    row_eval<P>(rp, u, X, Y);
    const NearRuns nr = near_runs(a, c1x, c1y);
    const GlobalNear nl{&a.L, nr, xnode, yref, a.il3x, a.mpx};
    const int nn = nr.total();
    near_sum_lat(nl, nn, u, dyl, a.yx_f, X, Y, mn);
    bool ok = true;
    if (mn < a.rc2u) {
        row_eval<P>(rp, u, X, Y);
        ok = near_sum_hilo_lat(nl, nn, u, dyl, dyl_lo, a.yx_f, X, Y);
    }
    int gx, gy;
    pixel_xy(X, Y, rp.bx, rp.by, gx, gy);
    // beta in theta_E from the kernel's own pixel-unit value
    beta[2 * q] = g.mx0 + ((double)rp.bx + (double)X) * g.dpx;
    beta[2 * q + 1] = g.my0 + ((double)rp.by + (double)Y) * g.dpy;
    if (!ok) { pix[2 * q] = -2; pix[2 * q + 1] = -2; }
    else if ((unsigned)gx >= (unsigned)g.mnx || (unsigned)gy >= (unsigned)g.mny) {
        pix[2 * q] = -1; pix[2 * q + 1] = -1;
    } else { pix[2 * q] = gx; pix[2 * q + 1] = gy; }
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
    auto kern = a.g.deposit != ML_DEPOSIT_NGP ? k_shoot_mixed_cic<P>
                : a.walk == ML_WALK_CERTIFIED ? k_shoot_mixed<P, true> : k_shoot_mixed<P, false>;
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

template <int P>
static cudaError_t launch_batch_p(const BatchArgs &b, int num_sms, cudaStream_t s)
{
    size_t smem = (size_t)b.near_cap * WARPS_PER_CTA * (sizeof(float4) + sizeof(float2));
    auto kern = b.walk == ML_WALK_CERTIFIED ? k_shoot_batch<P, true> : k_shoot_batch<P, false>;
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
    int64_t blocks = (int64_t)num_sms * per_sm;
    int64_t need = (b.total_tasks + WARPS_PER_CTA - 1) / WARPS_PER_CTA;
    if (need < blocks) blocks = need > 0 ? need : 1;
    kern<<<(unsigned)blocks, WARPS_PER_CTA * 32, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &b, int p, int num_sms, cudaStream_t s)
{
    switch (p) {
    case 1: return launch_batch_p<1>(b, num_sms, s);
    case 2: return launch_batch_p<2>(b, num_sms, s);
    case 3: return launch_batch_p<3>(b, num_sms, s);
    case 4: return launch_batch_p<4>(b, num_sms, s);
    case 5: return launch_batch_p<5>(b, num_sms, s);
    case 6: return launch_batch_p<6>(b, num_sms, s);
    case 8: return launch_batch_p<8>(b, num_sms, s);
    case 10: return launch_batch_p<10>(b, num_sms, s);
    case 12: return launch_batch_p<12>(b, num_sms, s);
    case 16: return launch_batch_p<16>(b, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
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
