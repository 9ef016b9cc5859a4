// Adjoint of the cloud-in-cell magnification map (the differentiable form
// of the deposition, Eq. 12 with bilinear weights).
//
// With M = (S_I / S_S) * CIC(rays) and G = dLoss/dM, each ray's dLoss/dbeta
// follows from its four bilinear weights, and the chain rule through the
// lens equation (Eq. 6, sheet included) gives, with d = theta -
// theta_k and r^2 = |d|^2:
//   dbeta/dkappa = (-theta_x, -theta_y),  dbeta/dgamma = (-theta_x, +theta_y),
//   dbeta/dkappa_* = theta - c            (inside the sheet's disc),
//   dbeta/dm_k = -d / r^2,  dbeta/dtheta_k = m_k (I r^2 - 2 d d^T) / r^4.
//
// Two kernels compute it:
//  - k_adj_rays + k_adj_far (the default): the transpose of the forward's
//    near/far split (Eq. 9).  Each ray is recomputed by the forward's own
//    arithmetic; its near lenses take the exact pair terms above, and its
//    far lenses act only through the node coefficients c_n, so the ray adds
//    G (theta - z_node)^n to the moments M_n of its level-2 node.  A far lens
//    then receives, per node,
//      dL/dm_k = Re sum_n M_n w^{n+1},
//      dL/dz_k = -m_k sum_n (n+1) M_n w^{n+2}  (dL/dx_k = Re, dL/dy_k = -Im),
//    with w = 1 / (z_k - z_node) and G = dL/dbeta_x + i dL/dbeta_y: the exact
//    gradient of the forward as computed, truncation included.
//  - k_cic_adjoint_direct: every ray against every lens with the exact
//    point-mass derivatives (a cross-check; cost rays x lenses).
#include "ml_internal.cuh"
#include "ml_task.cuh"

#include <math.h>

#include <algorithm>
#include <type_traits>

namespace ml {

// ---- direct form ------------------------------------------------------------

// With M = (S_I / S_S) * CIC(rays) and G = dLoss/dM, each ray's dLoss/dbeta
// follows from its four bilinear weights, and the chain rule through Eq. 6
// gives (d = theta - theta_k, r^2 = |d|^2):
//   dbeta/dkappa = (-theta_x, -theta_y),  dbeta/dgamma = (-theta_x, +theta_y),
//   dbeta/dkappa_* = theta - c            (inside the sheet's disc),
//   dbeta/dm_k = -d / r^2,  dbeta/dtheta_k = m_k (I r^2 - 2 d d^T) / r^4.
// The lens terms use the exact point-mass derivative for every lens; the
// forward's far series differs from the direct sum only by its truncation
// (far_bound).  Rays are recomputed with the forward's own arithmetic.

constexpr int ADJ_THREADS = 256;
constexpr int ADJ_LPT = 4;                          // lenses per thread per pass

// dLoss/dbeta of one ray from its cloud-in-cell weights: with the ray at
// pixel coordinates (bx + X, by + Y), weights (1-wx)(1-wy), wx(1-wy),
// (1-wx)wy, wx wy to the four nearest pixel centres, and
//   dL/dbeta_x = ipx [(G10 - G00)(1 - wy) + (G11 - G01) wy],
//   dL/dbeta_y = ipy [(G01 - G00)(1 - wx) + (G11 - G10) wx],
// ipx = (S_I / S_S) / dpx.  Pixels outside the map contribute nothing.
// The quad's four dL/dM differences (G1 - G0, G3 - G2, G2 - G0, G3 - G1),
// pixels outside the map counting 0.
struct QuadG {
    float e10, e32, e20, e31;
};

__device__ __forceinline__ QuadG quad_g(const Geo &g, const float *__restrict__ G, unsigned ix, unsigned iy)
{
    float Gv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned px = ix + (unsigned)(q & 1), py = iy + (unsigned)(q >> 1);
        Gv[q] = (px < (unsigned)g.mnx && py < (unsigned)g.mny) ? __ldg(G + (size_t)py * (unsigned)g.mnx + px)
                                                               : 0.f;
    }
    return QuadG{__fsub_rn(Gv[1], Gv[0]), __fsub_rn(Gv[3], Gv[2]), __fsub_rn(Gv[2], Gv[0]),
                 __fsub_rn(Gv[3], Gv[1])};
}

// The two formulas above with a fixed operation order, shared by every
// adjoint path so that they agree ray by ray.
__device__ __forceinline__ void quad_dbeta(const QuadG &q, float wx, float wy, float ipx, float ipy,
                                           float &gbx, float &gby)
{
    gbx = __fmul_rn(ipx, __fmaf_rn(q.e32, wy, __fmul_rn(q.e10, __fsub_rn(1.f, wy))));
    gby = __fmul_rn(ipy, __fmaf_rn(q.e31, wx, __fmul_rn(q.e20, __fsub_rn(1.f, wx))));
}

__device__ __forceinline__ void cic_dbeta(const Geo &g, const float *__restrict__ G, int bx, int by,
                                          float X, float Y, float ipx, float ipy, float &gbx,
                                          float &gby)
{
    unsigned ix, iy;
    float wx, wy;
    cic_quad(bx, by, X, Y, ix, iy, wx, wy);
    quad_dbeta(quad_g(g, G, ix, iy), wx, wy, ipx, ipy, gbx, gby);
}

// Position (pixel units) of ray r by exactly the mixed forward's arithmetic.
template <int P>
__device__ __forceinline__ bool forward_ray(const ShootArgs &a, int64_t r, float &X, float &Y, int &bx,
                                            int &by)
{
    const Geo &g = a.g;
    int64_t i = r % g.n3x, j = r / g.n3x;
    int64_t c1x = i / g.n1x, c1y = j / g.n1y;
    int64_t c2x = i / g.n2x, c2y = j / g.n2y;
    int64_t row0 = c1y * g.n1y + 32 * ((j - c1y * g.n1y) / 32);
    double yref = g.ry0 + ((double)row0 + 0.5) * g.l3y;
    double xnode = g.rx0 + ((double)c2x + 0.5) * g.l2x;
    const double dyl_d = (double)(j - row0) * g.l3y;
    const float dyl = (float)dyl_d;
    const float dyl_lo = (float)(dyl_d - (double)dyl);
    float qf = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
    RowPoly<P> rp;
    row_setup<P>(a.nodes + (c2y * g.N2x + c2x) * node_stride(P), qf, row_y(qf, a), a, rp);
    float u = __fadd_rn((float)(i - c2x * g.n2x), a.c0_f);
    float tt = __fmul_rn(u, a.l3x_f);
    float ax, ay, mn;
    row_eval<P>(rp, u, X, Y);
    const NearRuns nr = near_runs(a, c1x, c1y);
    const GlobalNear nl{&a.L, nr, xnode, yref, 1.0, 1.0};
    const int nn = nr.total();
    near_sum_f32(nl, nn, tt, dyl, ax, ay, mn);
    bool ok = true;
    if (mn < a.rc2) ok = near_sum_hilo(nl, nn, u, tt, dyl, dyl_lo, a.l3x_f, a.l3x_lo, ax, ay);
    X = __fmaf_rn(-ax, a.ipx_f, X);
    Y = __fmaf_rn(-ay, a.ipy_f, Y);
    bx = rp.bx;
    by = rp.by;
    return ok;
}

// Grid (ray tiles, lens passes).  Pass y handles lenses [y * T * LPT, ...).
template <int P>
__global__ void __launch_bounds__(ADJ_THREADS) k_cic_adjoint_direct(ShootArgs a, const float *__restrict__ G,
                                                            const double *__restrict__ lx,
                                                            const double *__restrict__ ly,
                                                            const double *__restrict__ lm,
                                                            int64_t n_lens, double *__restrict__ glens,
                                                            double *__restrict__ gpar, double scale)
{
    __shared__ float4 rays[ADJ_THREADS];    // (theta - ref, dL/dbeta)
    __shared__ int cnt;
    __shared__ double red[3][ADJ_THREADS / 32];
    const Geo &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t lens0 = (int64_t)blockIdx.y * ADJ_THREADS * ADJ_LPT;
    double sx[ADJ_LPT], sy[ADJ_LPT], sm[ADJ_LPT];
#pragma unroll
    for (int q = 0; q < ADJ_LPT; ++q) { sx[q] = 0.0; sy[q] = 0.0; sm[q] = 0.0; }
    double pk = 0.0, pg = 0.0, ps = 0.0;
    // A tile is a segment of one lattice row, so ray offsets from its centre
    // stay below 128 l3 and the FP32 differences theta - theta_k keep their
    // relative precision down to the closest rays.
    const int64_t nseg = (g.n3x + ADJ_THREADS - 1) / ADJ_THREADS;
    const int64_t j_lo = a.ray_begin / g.n3x, j_hi = (a.ray_end - 1) / g.n3x;
    const int64_t n_tiles = (j_hi - j_lo + 1) * nseg;
    const float ipx = (float)(scale / g.dpx), ipy = (float)(scale / g.dpy);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t jt = j_lo + tile / nseg, i0 = (tile % nseg) * ADJ_THREADS;
        const double refx = g.rx0 + ((double)i0 + (0.5 * ADJ_THREADS + 0.5)) * g.l3x;
        const double refy = g.ry0 + ((double)jt + 0.5) * g.l3y;
        if (tid == 0) cnt = 0;
        __syncthreads();
        // phase A: this thread's ray, its dLoss/dbeta, the parameter terms
        const int64_t it = i0 + tid, r = jt * g.n3x + it;
        float gbx = 0.f, gby = 0.f;
        double tx = 0.0, ty = 0.0;
        if (it < g.n3x && r >= a.ray_begin && r < a.ray_end) {
            float X, Y;
            int bxi, byi;
            if (forward_ray<P>(a, r, X, Y, bxi, byi)) cic_dbeta(g, G, bxi, byi, X, Y, ipx, ipy, gbx, gby);
            tx = g.rx0 + ((double)it + 0.5) * g.l3x;
            ty = refy;
        }
        const bool live = gbx != 0.f || gby != 0.f;
        if (live && blockIdx.y == 0) {
            pk += -(double)gbx * tx - (double)gby * ty;
            pg += -(double)gbx * tx + (double)gby * ty;
            ps += (double)gbx * (tx - g.sheet_cx) + (double)gby * (ty - g.sheet_cy);
        }
        // compact the live rays of the tile
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        int wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(&cnt, __popc(bal));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (live) {
            int slot = wbase + __popc(bal & ((1u << lane) - 1u));
            rays[slot] = make_float4((float)(tx - refx), (float)(ty - refy), gbx, gby);
        }
        __syncthreads();
        // phase B: this thread's lenses against the tile's live rays
        const int nlive = cnt;
        if (nlive > 0) {
            float ox[ADJ_LPT], oy[ADJ_LPT], ax[ADJ_LPT], ay[ADJ_LPT], am[ADJ_LPT];
#pragma unroll
            for (int q = 0; q < ADJ_LPT; ++q) {
                int64_t k = lens0 + tid + (int64_t)q * ADJ_THREADS;
                bool have = k < n_lens;
                ox[q] = have ? (float)(lx[k] - refx) : 1.0e18f;
                oy[q] = have ? (float)(ly[k] - refy) : 1.0e18f;
                ax[q] = 0.f; ay[q] = 0.f; am[q] = 0.f;
            }
            for (int jr = 0; jr < nlive; ++jr) {
                const float4 R = rays[jr];
#pragma unroll
                for (int q = 0; q < ADJ_LPT; ++q) {
                    float dx = R.x - ox[q], dy = R.y - oy[q];
                    float r2 = fmaf(dx, dx, dy * dy);
                    float inv = rcp_approx(r2);
                    float t = fmaf(R.z, dx, R.w * dy) * inv;       // (dL/dbeta . d) / r^2
                    float u2 = 2.f * t * inv;
                    am[q] += t;
                    ax[q] += fmaf(R.z, inv, -dx * u2);
                    ay[q] += fmaf(R.w, inv, -dy * u2);
                }
            }
#pragma unroll
            for (int q = 0; q < ADJ_LPT; ++q) { sx[q] += ax[q]; sy[q] += ay[q]; sm[q] += am[q]; }
        }
        __syncthreads();
    }
    // lens gradients: dL/dx_k = m_k * sum(...), dL/dm_k = -sum(t)
#pragma unroll
    for (int q = 0; q < ADJ_LPT; ++q) {
        int64_t k = lens0 + tid + (int64_t)q * ADJ_THREADS;
        if (k >= n_lens) continue;
        atomicAdd(glens + 3 * k + 0, lm[k] * sx[q]);
        atomicAdd(glens + 3 * k + 1, lm[k] * sy[q]);
        atomicAdd(glens + 3 * k + 2, -sm[q]);
    }
    if (blockIdx.y == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            pk += __shfl_down_sync(0xffffffffu, pk, o);
            pg += __shfl_down_sync(0xffffffffu, pg, o);
            ps += __shfl_down_sync(0xffffffffu, ps, o);
        }
        if (lane == 0) { red[0][wid] = pk; red[1][wid] = pg; red[2][wid] = ps; }
        __syncthreads();
        if (tid < 3) {
            double v = 0.0;
            for (int w = 0; w < ADJ_THREADS / 32; ++w) v += red[tid][w];
            atomicAdd(gpar + tid, v);
        }
    }
}

cudaError_t launch_cic_adjoint_direct(const ShootArgs &a, const float *G, const double *lx, const double *ly,
                               const double *lm, int64_t n_lens, double *glens, double *gpar,
                               double scale, int num_sms, cudaStream_t s)
{
    if (a.ray_end <= a.ray_begin) return cudaSuccess;
    const int64_t tiles = ((a.ray_end - 1) / a.g.n3x - a.ray_begin / a.g.n3x + 1) *
                          ((a.g.n3x + ADJ_THREADS - 1) / ADJ_THREADS);
    int64_t bx = std::min<int64_t>(tiles, (int64_t)num_sms * 8);
    int64_t by = std::max<int64_t>(1, (n_lens + ADJ_THREADS * ADJ_LPT - 1) / (ADJ_THREADS * ADJ_LPT));
    if (by > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)bx, (unsigned)by);
    switch (a.g.p) {
#define ML_ADJ_CASE(PP) case PP: k_cic_adjoint_direct<PP><<<grid, ADJ_THREADS, 0, s>>>(a, G, lx, ly, lm, n_lens, glens, gpar, scale); break;
    ML_ADJ_CASE(1) ML_ADJ_CASE(2) ML_ADJ_CASE(3) ML_ADJ_CASE(4) ML_ADJ_CASE(5)
    ML_ADJ_CASE(6) ML_ADJ_CASE(8) ML_ADJ_CASE(10) ML_ADJ_CASE(12) ML_ADJ_CASE(16)
#undef ML_ADJ_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}


// ---- near/far form ------------------------------------------------------------

constexpr int ADJ_BUF = 128;          // buffered rays per warp for the near pass
constexpr int FAR_THREADS = 256;      // lenses per block of k_adj_far
constexpr int FAR_NODES = 32;         // nodes per shared-memory tile of k_adj_far

// Near pass: the buffered rays (x offset from the node, y offset from the
// task's first row, dL/dbeta) against the task's near lenses.  Lane = (lens
// slot, ray group): with a chunk of c <= 32 lenses, floor(32 / c) groups of c
// lanes take every group-th ray, two rays per step with separate sums, and
// the groups are summed at the end, so short lists keep the lanes busy.  Per
// pair, t = (g . d) / r^2 and
//   ax += (g_x - 2 d_x t) / r^2,  ay += (g_y - 2 d_y t) / r^2,  am += t,
// later scaled to dL/dx_k = m_k ax, dL/dy_k = m_k ay, dL/dm_k = -am.
__device__ __forceinline__ void near_pair(const float4 &R, const float4 &L, const float2 &lo, float &ax,
                                          float &ay, float &am)
{
    const float dx = __fsub_rn(__fsub_rn(R.x, L.x), lo.x);
    const float dy = __fsub_rn(__fsub_rn(R.y, L.y), lo.y);
    const float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    const float inv = rcp_approx(r2);
    const float tq = __fmul_rn(__fmaf_rn(R.z, dx, __fmul_rn(R.w, dy)), inv);
    const float v = -2.f * tq;
    am += tq;
    ax = __fmaf_rn(inv, __fmaf_rn(dx, v, R.z), ax);
    ay = __fmaf_rn(inv, __fmaf_rn(dy, v, R.w), ay);
}

__device__ __forceinline__ void near_pass(const float4 *near, const float2 *nlo, double *acc,
                                          const float4 *buf, int nn, int nb, int lane)
{
    __syncwarp();
    for (int c0 = 0; c0 < nn; c0 += 32) {
        const int cn = min(32, nn - c0);            // lenses in this chunk
        const int ngrp = 32 / cn, used = ngrp * cn;
        const int sl = lane % cn, grp = lane / cn;
        const bool have = lane < used;
        const int slot = c0 + sl;
        const float4 L = have ? near[slot] : make_float4(1.0e18f, 1.0e18f, 0.f, 0.f);
        const float2 lo = have ? nlo[slot] : make_float2(0.f, 0.f);
        float ax = 0.f, ay = 0.f, am = 0.f, bx = 0.f, by = 0.f, bm = 0.f;
        int r = have ? grp : nb;
        for (; r + ngrp < nb; r += 2 * ngrp) {
            const float4 R0 = buf[r], R1 = buf[r + ngrp];
            near_pair(R0, L, lo, ax, ay, am);
            near_pair(R1, L, lo, bx, by, bm);
        }
        if (r < nb) near_pair(buf[r], L, lo, ax, ay, am);
        ax += bx;
        ay += by;
        am += bm;
        // sum the groups of each slot into group 0
        for (int off = cn; off < used; off <<= 1) {
            const float ox = __shfl_down_sync(0xffffffffu, ax, off);
            const float oy = __shfl_down_sync(0xffffffffu, ay, off);
            const float om = __shfl_down_sync(0xffffffffu, am, off);
            if (lane + off < used) {
                ax += ox;
                ay += oy;
                am += om;
            }
        }
        if (grp == 0 && have) {
            acc[3 * slot] += (double)ax;
            acc[3 * slot + 1] += (double)ay;
            acc[3 * slot + 2] += (double)am;
        }
    }
    __syncwarp();
}

// t-power sums T_j = sum G t^j of one lane's rays to moments
// M_n = sum G (t + i s)^n = sum_j C(n, j) (i s)^{n-j} T_j, in place.  This is
// the transpose of the Taylor shift of row_setup: the same synthetic-division
// steps taken in reverse order with each step transposed.
template <int P>
__device__ __forceinline__ void moments_from_tpowers(float (&T)[2 * (P + 1)], float s)
{
#pragma unroll
    for (int k = P - 1; k >= 0; --k) {
#pragma unroll
        for (int n = k; n < P; ++n) {
            // T_{n+1} += (i s) T_n
            T[2 * (n + 1)] = __fmaf_rn(-s, T[2 * n + 1], T[2 * (n + 1)]);
            T[2 * (n + 1) + 1] = __fmaf_rn(s, T[2 * n], T[2 * (n + 1) + 1]);
        }
    }
}

struct AdjArgs {
    const float *G;         // dLoss/dM, mny x mnx
    double *gs;             // per sorted lens: dL/dx, dL/dy, dL/dm
    double *gpar;           // dL/dkappa, dL/dgamma, dL/dkappa_*
    double2 *mom;           // (P+1) per node: scaled moments sum G ((theta - z_node)/h)^n
    float ipx, ipy;         // (S_I / S_S) / dpx, / dpy
    float hinv;             // 1 / h, h = half-diagonal of a level-2 cell
    float l3y_f;
};

// Shared memory of k_adj_rays, in float4 units: near records, their
// remainders (float2), the FP64 near-lens sums (3 doubles per slot), the ray
// buffers.
__host__ __device__ inline size_t adj_smem_f4(int cap)
{
    const size_t w = WARPS_PER_CTA;
    return w * cap + (w * cap + 1) / 2 + (w * cap * 3 + 1) / 2 + w * ADJ_BUF;
}

// Per task (the forward's decomposition): recompute every ray exactly as the
// CIC shooting kernel does, take its dLoss/dbeta, and accumulate
//  - kappa, gamma, kappa_* terms (FP32 per lane and level-2 column, FP64 across),
//  - the moments of its level-2 node (FP32 t-power sums per lane, converted
//    and reduced over the lanes of one node, FP64 atomics),
//  - the near-lens pair terms (near_pass, FP64 per warp, FP64 atomics per task).
#ifndef ML_ADJ_LOWP_BLOCKS
#define ML_ADJ_LOWP_BLOCKS 2
#endif

template <int P>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, (P <= 4 ? ML_ADJ_LOWP_BLOCKS : 2))
    k_adj_rays(ShootArgs a, AdjArgs d)
{
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int cap = a.near_cap;
    const int W = WARPS_PER_CTA;
    float4 *near = smem + wid * cap;
    float2 *nlo = reinterpret_cast<float2 *>(smem + W * cap) + wid * cap;
    double *acc = reinterpret_cast<double *>(smem + W * cap + (W * cap + 1) / 2) + 3 * wid * cap;
    float4 *buf = smem + W * cap + (W * cap + 1) / 2 + (W * cap * 3 + 1) / 2 + wid * ADJ_BUF;
    const SmemNear nl{near, nlo};
    const Geo &g = a.g;
    double pk = 0.0, pg = 0.0, ps = 0.0;
    for (;;) {
        bool stop;
        const int64_t t = fetch_task(a, lane, stop);
        if (stop || t >= a.n_tasks) break;
        TaskShape ts;
        if (!decode_task(a, t, ts)) continue;
        const NearRuns nr = near_runs(a, ts.c1x, ts.c1y);
        const double yref = g.ry0 + ((double)ts.row0 + 0.5) * g.l3y;
        const int nn = stage_near_y<false>(a, nr, yref, near, nlo, lane);
        for (int k = lane; k < 3 * nn; k += 32) acc[k] = 0.0;
        const int64_t j = ts.row0 + lane;
        const bool active = j < ts.rows_end;
        const double dyl_d = (double)lane * g.l3y;
        const float dyl = (float)dyl_d;
        const float dyl_lo = (float)(dyl_d - (double)dyl);
        const int64_t c2y = j / g.n2y;
        const float q = (float)((double)(j - c2y * g.n2y) + 0.5 - 0.5 * (double)g.n2y);
        const RowY ry = row_y(q, a);
        const double yrow = yref + dyl_d;
        const float s_h = __fmul_rn(__fmul_rn(q, d.l3y_f), d.hinv);
        // lanes of one node row band: [first, seg_last]; the first one adds
        const int seg_last = (int)min((int64_t)31, (c2y + 1) * g.n2y - 1 - ts.row0);
        const bool head = active && (lane == 0 || j == c2y * g.n2y);
        for (int64_t c2x = ts.c2a; c2x < ts.c2b; ++c2x) {
            const double xnode = g.rx0 + ((double)c2x + 0.5) * g.l2x;
            stage_near_x<false>(a, nn, xnode, near, nlo, lane);
            const int64_t i0 = c2x * g.n2x;
            const int kend = (int)(min(i0 + g.n2x, g.n3x) - i0);
            RowPoly<P> rp;
            row_setup<P>(a.nodes + (min(c2y, g.N2y - 1) * g.N2x + c2x) * node_stride(P), q, ry, a, rp);
            float T[2 * (P + 1)];
#pragma unroll
            for (int n = 0; n < 2 * (P + 1); ++n) T[n] = 0.f;
            float sgx = 0.f, sgy = 0.f, stx = 0.f;
            int nb = 0;
            float u = a.c0_f;
            // Tasks with at most one near lens (nearly all on fine level-1
            // cells): rays in pairs with the forward's arithmetic, and the
            // dL/dM differences of the lane's current pixel quad, reloaded
            // after a warp vote when a ray leaves it (quad_dbeta as
            // cic_dbeta).  A near lens is held in registers; its forward terms
            // are near_sum_f32's and its gradient terms near_pair's, summed
            // per lane over the column and then over the warp.
            auto walk = [&](auto nn_c) {
                constexpr int NN = decltype(nn_c)::value;
                float lx = 0.f, lm = 0.f, fdy = 0.f, fdy2 = 0.f, lxl = 0.f, gdy = 0.f, gdy2 = 0.f;
                if (NN == 1) {
                    const float4 L = near[0];
                    const float2 lo = nlo[0];
                    lx = L.x;
                    lm = L.z;
                    fdy = __fsub_rn(dyl, L.y);
                    fdy2 = __fmul_rn(fdy, fdy);
                    lxl = lo.x;
                    gdy = __fsub_rn(__fsub_rn(dyl, L.y), lo.y);
                    gdy2 = __fmul_rn(gdy, gdy);
                }
                float nax = 0.f, nay = 0.f, nam = 0.f;
                unsigned cqx = 0xFFFFFFFFu, cqy = 0xFFFFFFFFu;
                auto load_quad = [&](unsigned ix, unsigned iy) {
                    cqx = ix;
                    cqy = iy;
                    return quad_g(g, d.G, ix, iy);
                };
                // the cache starts as a real quad (the one whose only pixel
                // in the map is (0, 0)), with its own values
                QuadG cq = load_quad(cqx, cqy);
                auto add_ray = [&](float gbx, float gby, float tt) {
                    sgx += gbx;
                    sgy += gby;
                    stx = __fmaf_rn(gbx, tt, stx);
                    const float th = __fmul_rn(tt, d.hinv);
                    float pw = 1.f;
#pragma unroll
                    for (int n = 0; n <= P; ++n) {
                        T[2 * n] = __fmaf_rn(gbx, pw, T[2 * n]);
                        T[2 * n + 1] = __fmaf_rn(gby, pw, T[2 * n + 1]);
                        pw = __fmul_rn(pw, th);
                    }
                };
                auto near_fwd = [&](float tt, float &X, float &Y, float &r2) {
                    const float dx = __fsub_rn(tt, lx);
                    r2 = __fmaf_rn(dx, dx, fdy2);
                    const float sv = __fmul_rn(lm, rcp_approx(r2));
                    const float sx = __fmaf_rn(dx, sv, 0.f), sy = __fmaf_rn(fdy, sv, 0.f);
                    X = __fmaf_rn(-sx, a.ipx_f, X);
                    Y = __fmaf_rn(-sy, a.ipy_f, Y);
                };
                auto near_grad = [&](bool ok, float tt, float gbx, float gby) {
                    const float dx = __fsub_rn(__fsub_rn(tt, lx), lxl);
                    const float r2 = __fmaf_rn(dx, dx, gdy2);
                    const float inv = rcp_approx(r2);
                    const float tq = __fmul_rn(__fmaf_rn(gbx, dx, __fmul_rn(gby, gdy)), inv);
                    const float v = -2.f * tq;
                    if (ok) {
                        nam += tq;
                        nax = __fmaf_rn(inv, __fmaf_rn(dx, v, gbx), nax);
                        nay = __fmaf_rn(inv, __fmaf_rn(gdy, v, gby), nay);
                    }
                };
                for (int k = 0; k < kend; k += 2, u += 2.f) {
                    const bool on1 = active && k + 1 < kend;
                    const float u1 = __fadd_rn(u, 1.f);
                    const float t0 = __fmul_rn(u, a.l3x_f), t1 = __fmul_rn(u1, a.l3x_f);
                    float X0, Y0, X1, Y1;
                    row_eval<P>(rp, u, X0, Y0);
                    row_eval<P>(rp, u1, X1, Y1);
                    bool ok0 = active, ok1 = on1;
                    if (NN == 1) {
                        const float Xp0 = X0, Yp0 = Y0, Xp1 = X1, Yp1 = Y1;
                        float r20, r21;
                        near_fwd(t0, X0, Y0, r20);
                        near_fwd(t1, X1, Y1, r21);
                        const bool c0 = ok0 && r20 < a.rc2, c1 = ok1 && r21 < a.rc2;
                        if (__ballot_sync(0xffffffffu, c0 || c1)) {
                            if (c0) {
                                float ax, ay;
                                ok0 = near_sum_hilo(nl, 1, u, t0, dyl, dyl_lo, a.l3x_f, a.l3x_lo, ax, ay);
                                X0 = __fmaf_rn(-ax, a.ipx_f, Xp0);
                                Y0 = __fmaf_rn(-ay, a.ipy_f, Yp0);
                            }
                            if (c1) {
                                float ax, ay;
                                ok1 = near_sum_hilo(nl, 1, u1, t1, dyl, dyl_lo, a.l3x_f, a.l3x_lo, ax, ay);
                                X1 = __fmaf_rn(-ax, a.ipx_f, Xp1);
                                Y1 = __fmaf_rn(-ay, a.ipy_f, Yp1);
                            }
                        }
                    }
                    unsigned ix0, iy0, ix1, iy1;
                    float wx0, wy0, wx1, wy1;
                    cic_quad(rp.bx, rp.by, X0, Y0, ix0, iy0, wx0, wy0);
                    cic_quad(rp.bx, rp.by, X1, Y1, ix1, iy1, wx1, wy1);
                    // ray 1 compares with the quad after ray 0 (unchanged
                    // when ray 0 is dropped)
                    const bool ch0 = ok0 && (ix0 != cqx || iy0 != cqy);
                    const bool ch1 = ok1 && (ix1 != (ok0 ? ix0 : cqx) || iy1 != (ok0 ? iy0 : cqy));
                    const bool any = __ballot_sync(0xffffffffu, ch0 || ch1) != 0u;
                    float gx0, gy0, gx1, gy1;
                    if (any && ch0) cq = load_quad(ix0, iy0);
                    quad_dbeta(cq, wx0, wy0, d.ipx, d.ipy, gx0, gy0);
                    if (any && ch1) cq = load_quad(ix1, iy1);
                    quad_dbeta(cq, wx1, wy1, d.ipx, d.ipy, gx1, gy1);
                    gx0 = ok0 ? gx0 : 0.f;
                    gy0 = ok0 ? gy0 : 0.f;
                    gx1 = ok1 ? gx1 : 0.f;
                    gy1 = ok1 ? gy1 : 0.f;
                    add_ray(gx0, gy0, t0);
                    add_ray(gx1, gy1, t1);
                    if (NN == 1) {
                        near_grad(ok0, t0, gx0, gy0);
                        near_grad(ok1, t1, gx1, gy1);
                    }
                }
                if (NN == 1) {
                    for (int off = 16; off > 0; off >>= 1) {
                        nax += __shfl_down_sync(0xffffffffu, nax, off);
                        nay += __shfl_down_sync(0xffffffffu, nay, off);
                        nam += __shfl_down_sync(0xffffffffu, nam, off);
                    }
                    if (lane == 0) {
                        acc[0] += (double)nax;
                        acc[1] += (double)nay;
                        acc[2] += (double)nam;
                    }
                    __syncwarp();
                }
            };
            if (nn == 0) {
                walk(std::integral_constant<int, 0>{});
            } else if (nn == 1) {
                walk(std::integral_constant<int, 1>{});
            } else
            for (int k = 0; k < kend; ++k, u += 1.f) {
                const float t0 = __fmul_rn(u, a.l3x_f);
                float gbx = 0.f, gby = 0.f;
                if (active) {
                    float X, Y, ax, ay, mn;
                    row_eval<P>(rp, u, X, Y);
                    near_sum_f32(nl, nn, t0, dyl, ax, ay, mn);
                    bool ok = true;
                    if (mn < a.rc2)
                        ok = near_sum_hilo(nl, nn, u, t0, dyl, dyl_lo, a.l3x_f, a.l3x_lo, ax, ay);
                    if (ok) {
                        X = __fmaf_rn(-ax, a.ipx_f, X);
                        Y = __fmaf_rn(-ay, a.ipy_f, Y);
                        cic_dbeta(g, d.G, rp.bx, rp.by, X, Y, d.ipx, d.ipy, gbx, gby);
                    }
                }
                const bool live = gbx != 0.f || gby != 0.f;
                if (live) {
                    sgx += gbx;
                    sgy += gby;
                    stx = __fmaf_rn(gbx, t0, stx);
                    const float th = __fmul_rn(t0, d.hinv);
                    float pw = 1.f;
#pragma unroll
                    for (int n = 0; n <= P; ++n) {
                        T[2 * n] = __fmaf_rn(gbx, pw, T[2 * n]);
                        T[2 * n + 1] = __fmaf_rn(gby, pw, T[2 * n + 1]);
                        pw = __fmul_rn(pw, th);
                    }
                }
                if (nn > 0) {
                    const unsigned bal = __ballot_sync(0xffffffffu, live);
                    if (bal) {
                        const int cnt = __popc(bal);
                        if (nb + cnt > ADJ_BUF) {
                            near_pass(near, nlo, acc, buf, nn, nb, lane);
                            nb = 0;
                        }
                        if (live) buf[nb + __popc(bal & ((1u << lane) - 1u))] = make_float4(t0, dyl, gbx, gby);
                        nb += cnt;
                    }
                }
            }
            if (nb > 0) near_pass(near, nlo, acc, buf, nn, nb, lane);
            // macro terms: sum g_x theta_x = x_node sum g_x + sum g_x t
            if (active) {
                const double xs = xnode * (double)sgx + (double)stx, ys = yrow * (double)sgy;
                pk -= xs + ys;
                pg += ys - xs;
                ps += xs - g.sheet_cx * (double)sgx + ys - g.sheet_cy * (double)sgy;
            }
            // the node's moments from this column's rays
            moments_from_tpowers<P>(T, s_h);
#pragma unroll
            for (int n = 0; n < 2 * (P + 1); ++n) {
                float v = T[n];
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float o = __shfl_down_sync(0xffffffffu, v, off);
                    if (lane + off <= seg_last) v += o;
                }
                T[n] = v;
            }
            if (head) {
                double *m = reinterpret_cast<double *>(d.mom + (c2y * g.N2x + c2x) * (P + 1));
#pragma unroll
                for (int n = 0; n < 2 * (P + 1); ++n)
                    if (T[n] != 0.f) atomicAdd(m + n, (double)T[n]);
            }
        }
        // near-lens gradients of the task, in sorted lens order
        __syncwarp();
        for (int k = lane; k < nn; k += 32) {
            const int32_t idx = __float_as_int(near[k].w);
            const double mk = a.L.m[idx];
            atomicAdd(d.gs + 3 * (int64_t)idx, mk * acc[3 * k]);
            atomicAdd(d.gs + 3 * (int64_t)idx + 1, mk * acc[3 * k + 1]);
            atomicAdd(d.gs + 3 * (int64_t)idx + 2, -acc[3 * k + 2]);
        }
        __syncwarp();
    }
    for (int off = 16; off > 0; off >>= 1) {
        pk += __shfl_down_sync(0xffffffffu, pk, off);
        pg += __shfl_down_sync(0xffffffffu, pg, off);
        ps += __shfl_down_sync(0xffffffffu, ps, off);
    }
    if (lane == 0) {
        atomicAdd(d.gpar, pk);
        atomicAdd(d.gpar + 1, pg);
        atomicAdd(d.gpar + 2, ps);
    }
}

// Far lenses: thread = sorted lens, a block walks node tiles.  A lens in the
// node's 3 x 3 level-1 block is skipped (its terms came from the near pass).
// With w = 1 / (z_k - z_node), v = h w and the scaled moments Mh_n:
//   A = sum Mh_n v^n, B = sum (n+1) Mh_n v^n,
//   dL/dm_k += Re(w A),  dL/dx_k += -m_k Re(w^2 B),  dL/dy_k += m_k Im(w^2 B).
// Lens offsets from the node grid are carried as an integer (exact in FP32)
// plus a fraction, so z_k - z_node keeps FP32 relative precision.
template <int P>
__global__ void __launch_bounds__(FAR_THREADS) k_adj_far(Geo g, LensTable L, const double2 *__restrict__ mom,
                                                         float h, double *__restrict__ gs)
{
    __shared__ float2 sm[FAR_NODES * (P + 1)];
    __shared__ int4 sn[FAR_NODES];
    const int tid = threadIdx.x;
    const int64_t k = blockIdx.x * (int64_t)FAR_THREADS + tid;
    const bool have = k < L.n;
    const int64_t NE = g.NEx * g.NEy;
    float uxi = 0.f, uxf = 0.f, uyi = 0.f, uyf = 0.f;
    int lcx = -1000, lcy = -1000;
    if (have) {
        double ux = (L.x[k] - g.rx0) / g.l2x - 0.5, uy = (L.y[k] - g.ry0) / g.l2y - 0.5;
        double fx = fmin(fmax(floor(ux), -8388608.0), 8388608.0);
        double fy = fmin(fmax(floor(uy), -8388608.0), 8388608.0);
        uxi = (float)fx;
        uxf = (float)(ux - fx);
        uyi = (float)fy;
        uyf = (float)(uy - fy);
        const int32_t c = L.cell[k];
        if (c < NE) {
            lcx = (int)(c % g.NEx);
            lcy = (int)(c / g.NEx);
        }
    }
    const float l2x = (float)g.l2x, l2y = (float)g.l2y;
    const int64_t nn = g.N2x * g.N2y, ntile = (nn + FAR_NODES - 1) / FAR_NODES;
    double gx = 0.0, gy = 0.0, gm = 0.0;
    for (int64_t tile = blockIdx.y; tile < ntile; tile += gridDim.y) {
        __syncthreads();
        const int64_t n0 = tile * FAR_NODES;
        for (int qq = tid; qq < FAR_NODES * (P + 1); qq += FAR_THREADS) {
            const int64_t node = n0 + qq / (P + 1);
            const double2 v = node < nn ? mom[node * (P + 1) + qq % (P + 1)] : make_double2(0.0, 0.0);
            sm[qq] = make_float2((float)v.x, (float)v.y);
        }
        __syncthreads();
        if (tid < FAR_NODES) {
            const int64_t node = n0 + tid;
            int4 v = make_int4(-1, 0, 0, 0);
            bool any = false;
            for (int n = 0; n <= P; ++n) {
                const float2 c = sm[tid * (P + 1) + n];
                any |= (c.x != 0.f) | (c.y != 0.f);
            }
            if (node < nn && any) {
                const int c2x = (int)(node % g.N2x), c2y = (int)(node / g.N2x);
                v = make_int4(c2x, c2y, c2x / g.l2sx + 1, c2y / g.l2sy + 1);
            }
            sn[tid] = v;
        }
        __syncthreads();
        if (!have) continue;
        float ax = 0.f, ay = 0.f, am = 0.f;
        for (int qn = 0; qn < FAR_NODES; ++qn) {
            const int4 nd = sn[qn];
            if (nd.x < 0) continue;
            if (abs(lcx - nd.z) <= 1 && abs(lcy - nd.w) <= 1) continue;
            const float dx = __fmul_rn(__fadd_rn(__fsub_rn(uxi, (float)nd.x), uxf), l2x);
            const float dy = __fmul_rn(__fadd_rn(__fsub_rn(uyi, (float)nd.y), uyf), l2y);
            const float inv = rcp_approx(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
            const float wr = dx * inv, wi = -dy * inv;
            const float vr = h * wr, vi = h * wi;
            const float2 *M = sm + qn * (P + 1);
            float Ar = M[P].x, Ai = M[P].y;
            float Br = (float)(P + 1) * Ar, Bi = (float)(P + 1) * Ai;
#pragma unroll
            for (int n = P - 1; n >= 0; --n) {
                const float2 c = M[n];
                const float tr = __fmaf_rn(Ar, vr, __fmaf_rn(-Ai, vi, c.x));
                const float ti = __fmaf_rn(Ar, vi, __fmaf_rn(Ai, vr, c.y));
                Ar = tr;
                Ai = ti;
                const float ur = __fmaf_rn(Br, vr, __fmaf_rn(-Bi, vi, (float)(n + 1) * c.x));
                const float ui = __fmaf_rn(Br, vi, __fmaf_rn(Bi, vr, (float)(n + 1) * c.y));
                Br = ur;
                Bi = ui;
            }
            am += wr * Ar - wi * Ai;
            const float w2r = wr * wr - wi * wi, w2i = 2.f * wr * wi;
            ax -= w2r * Br - w2i * Bi;
            ay += w2r * Bi + w2i * Br;
        }
        gx += (double)ax;
        gy += (double)ay;
        gm += (double)am;
    }
    if (have) {
        const double mk = L.m[k];
        atomicAdd(gs + 3 * k, mk * gx);
        atomicAdd(gs + 3 * k + 1, mk * gy);
        atomicAdd(gs + 3 * k + 2, gm);
    }
}

// Sorted order to the caller's order.
__global__ void k_adj_unsort(const double *__restrict__ gs, const int32_t *__restrict__ perm, int64_t n,
                             double *__restrict__ out)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = perm[k];
    out[3 * o] = gs[3 * k];
    out[3 * o + 1] = gs[3 * k + 1];
    out[3 * o + 2] = gs[3 * k + 2];
}

template <int P>
cudaError_t launch_adj_p(const ShootArgs &a, const AdjArgs &d, int num_sms, cudaStream_t s)
{
    const size_t smem = adj_smem_f4(a.near_cap) * sizeof(float4);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_rays<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_rays<P>,
                                                                  WARPS_PER_CTA * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)num_sms * per_sm;
    const int64_t need = (a.n_tasks + WARPS_PER_CTA - 1) / WARPS_PER_CTA;
    if (need < blocks) blocks = need > 0 ? need : 1;
    k_adj_rays<P><<<(unsigned)blocks, WARPS_PER_CTA * 32, smem, s>>>(a, d);
    e = cudaGetLastError();
    if (e != cudaSuccess || a.L.n == 0) return e;
    const int64_t lens_blocks = (a.L.n + FAR_THREADS - 1) / FAR_THREADS;
    const int64_t ntile = (a.g.N2x * a.g.N2y + FAR_NODES - 1) / FAR_NODES;
    if (lens_blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    // about eight blocks per SM in all
    const int64_t want = ((int64_t)num_sms * 8 + lens_blocks - 1) / lens_blocks;
    const int64_t by = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, ntile), 65535));
    const float h = (float)(0.5 * sqrt(a.g.l2x * a.g.l2x + a.g.l2y * a.g.l2y));
    k_adj_far<P><<<dim3((unsigned)lens_blocks, (unsigned)by), FAR_THREADS, 0, s>>>(a.g, a.L, d.mom, h, d.gs);
    return cudaGetLastError();
}

cudaError_t launch_cic_adjoint_nearfar(const ShootArgs &a, const float *G, double *gs, double *gpar,
                                       double2 *mom, const int32_t *perm, double *glens, double scale,
                                       int num_sms, cudaStream_t s)
{
    AdjArgs d;
    d.G = G;
    d.gs = gs;
    d.gpar = gpar;
    d.mom = mom;
    d.ipx = (float)(scale / a.g.dpx);
    d.ipy = (float)(scale / a.g.dpy);
    d.hinv = (float)(1.0 / (0.5 * sqrt(a.g.l2x * a.g.l2x + a.g.l2y * a.g.l2y)));
    d.l3y_f = (float)a.g.l3y;
    cudaError_t e;
    switch (a.g.p) {
    case 1: e = launch_adj_p<1>(a, d, num_sms, s); break;
    case 2: e = launch_adj_p<2>(a, d, num_sms, s); break;
    case 3: e = launch_adj_p<3>(a, d, num_sms, s); break;
    case 4: e = launch_adj_p<4>(a, d, num_sms, s); break;
    case 5: e = launch_adj_p<5>(a, d, num_sms, s); break;
    case 6: e = launch_adj_p<6>(a, d, num_sms, s); break;
    case 8: e = launch_adj_p<8>(a, d, num_sms, s); break;
    case 10: e = launch_adj_p<10>(a, d, num_sms, s); break;
    case 12: e = launch_adj_p<12>(a, d, num_sms, s); break;
    case 16: e = launch_adj_p<16>(a, d, num_sms, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || a.L.n == 0) return e;
    k_adj_unsort<<<(unsigned)((a.L.n + 255) / 256), 256, 0, s>>>(gs, perm, a.L.n, glens);
    return cudaGetLastError();
}

}  // namespace ml
