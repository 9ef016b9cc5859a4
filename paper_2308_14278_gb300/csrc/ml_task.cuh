// Task decomposition and near-lens staging of the mixed-precision kernels
// (shooting, tracing and the adjoint): a task is 32 consecutive ray rows of
// one level-1 row band times a run of level-2 columns of one level-1 column;
// its near lenses (the 3 x 3 block of level-1 cells, §3.2) are staged per
// warp as FP32 offsets with their rounding remainders.
#pragma once

#include "ml_internal.cuh"

namespace ml {

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
    ts.c2a = ts.c1x * g.l2sx + sub * a.l2_per_cc;
    ts.c2b = min(min(ts.c2a + a.l2_per_cc, (ts.c1x + 1) * (int64_t)g.l2sx), g.N2x);
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

// Task staging common to the mixed kernels: near lens list of the task's
// level-1 cell as FP32 offsets from the first row (y) and, per level-2
// column, from the node (x), with their rounding remainders.  LAT: offsets in
// lattice units (divided by l3x) and masses in pixel units (m / (l3x dpx)),
// for the counting kernels; else theta_E units and plain masses.
template <bool LAT>
__device__ __forceinline__ int stage_near_y(const ShootArgs &a, const NearRuns &nr, double yref,
                                            float4 *near, float2 *nlo, int lane)
{
    const int nn = nr.total();
    __syncwarp();
    for (int k = lane; k < nn; k += 32) {
        int32_t idx = nr.index(k);
        double dy = a.L.y[idx] - yref;
        if (LAT) dy *= a.il3x;
        float hi = (float)dy;
        const double m = LAT ? a.L.m[idx] * a.mpx : a.L.m[idx];
        near[k] = make_float4(0.f, hi, (float)m, __int_as_float(idx));
        nlo[k].y = (float)(dy - (double)hi);
    }
    return nn;
}

template <bool LAT>
__device__ __forceinline__ void stage_near_x(const ShootArgs &a, int nn, double xnode,
                                             float4 *near, float2 *nlo, int lane)
{
    __syncwarp();
    for (int k = lane; k < nn; k += 32) {
        double dx = a.L.x[__float_as_int(near[k].w)] - xnode;
        if (LAT) dx *= a.il3x;
        float hi = (float)dx;
        near[k].x = hi;
        nlo[k].x = (float)(dx - (double)hi);
    }
    __syncwarp();
}

__device__ __forceinline__ int64_t fetch_task(const ShootArgs &a, int lane, bool &stop)
{
    long long t = 0;
    int ab = 0;
    if (lane == 0) {
        t = (long long)atomicAdd(a.work, 1ull);
        ab = *a.abort_flag;
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    ab = __shfl_sync(0xffffffffu, ab, 0);
    stop = ab != 0;
    if (stop && lane == 0) atomicOr(a.status, 2u);
    return t;
}

// Near records computed from the FP64 lens table, for single rays: theta_E
// units (sc = msc = 1) or lattice units (sc = 1/l3x, msc = 1/(l3x dpx)), the
// values stage_near_y/x produce.
struct GlobalNear {
    const LensTable *L;
    NearRuns nr;
    double xnode, yref, sc, msc;
    __device__ __forceinline__ float4 rec(int k) const
    {
        int32_t id = nr.index(k);
        return make_float4((float)((L->x[id] - xnode) * sc), (float)((L->y[id] - yref) * sc),
                           (float)(L->m[id] * msc), 0.f);
    }
    __device__ __forceinline__ float2 lo(int k) const
    {
        int32_t id = nr.index(k);
        double dx = (L->x[id] - xnode) * sc, dy = (L->y[id] - yref) * sc;
        return make_float2((float)(dx - (double)(float)dx), (float)(dy - (double)(float)dy));
    }
};

}  // namespace ml
