// Internal declarations of the GB300 microlensing library: derived geometry,
// device-buffer bundles, launch wrappers and the per-ray arithmetic that the
// shooting and tracing kernels share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ml.h"

namespace ml {

constexpr int PMAX = 16;                  // highest Taylor order supported
constexpr uint32_t PIX_OUT = 0xFFFFFFFFu;   // run-length code: outside the map
constexpr uint32_t PIX_DROP = 0xFFFFFFFEu;  // run-length code: ray hit a lens
constexpr int WARPS_PER_CTA = 8;

// The certified walk (ML_WALK_CERTIFIED): rays it evaluates per step (its
// window), rays short of the predicted pixel edge at which a window starts,
// and the distance in lattice units within which a near lens makes it hand a
// warp's level-2 column to the per-ray walk (runs shorten and certified spans
// stay short near a lens).
#ifndef ML_SPAN_W
#define ML_SPAN_W 2
#endif
#ifndef ML_SPAN_MARGIN
#define ML_SPAN_MARGIN 1.0f
#endif
#ifndef ML_SPAN_FAR
#define ML_SPAN_FAR 3000.0f
#endif

// Parameters derived from an ml_field_desc (§3.1 and §3.2).
struct Geo {
    double kappa, gamma, kappa_star;
    int32_t macro;                  // ML_MACRO_LINEAR or ML_MACRO_FOLD
    double kappa0, dx, dy;          // fold parameters (Eq. 5)
    double sheet_cx, sheet_cy, sheet_r;
    int32_t sheet_shape;            // ML_SHEET_DISC or ML_SHEET_STRIP
    double rx0, ry0, rx1, ry1;      // ray rectangle
    double l3x, l3y;                // level-3 pixel (ray spacing)
    int64_t n3x, n3y;               // lattice size
    double mx0, my0, dpx, dpy;      // map origin and pixel size
    int32_t mnx, mny;
    int64_t n_star_in;
    double l0;
    int32_t l2sx, l2sy, p;      // level-2 cells per level-1 side; Taylor order
    int64_t n1x, n1y, n2x, n2y;     // rays per level-1 / level-2 cell side
    int64_t N1x, N1y, N2x, N2y;     // cells across the lattice
    double l1x, l1y, l2x, l2y;      // = n1 * l3, n2 * l3
    int64_t NEx, NEy;               // level-1 grid with one ring around it
    int32_t precision, deposit;
};

// Lenses sorted by extended level-1 cell (a ring of cells around the lattice
// included); lenses outside the ring follow in one last bucket.
struct LensTable {
    const double *x, *y, *m;        // sorted, FP64
    const int32_t *cell;            // extended cell id of each sorted lens, NE for outside
    const int32_t *start;           // NE + 2 offsets: bucket b holds [start[b], start[b+1])
    int64_t n;
    // FP32 copies for the truncation bound: x = xh + xl and y = yh + yl to
    // about 2^-48 relative, mf = m rounded
    const float *xh, *xl, *yh, *yl, *mf;
};

// Per-node record of the mixed-precision path, stride 24 + 8p bytes:
//   int32 by;  float fy;  int32 bx;  float fx;  float ax;  float bq;  float2 c[p]
// (by + fy, bx + fx) is the smooth part of beta at the node in map pixel units
// (macro model, sheet and far-field c_0; fx, fy in [0, 1)); ax is d(beta_x)/d(theta_x) of the
// macro and sheet terms at the node in pixels per ray column (l3x); bq is the
// change of beta_x per ray row (pixels; the fold's d_y theta_x term, else 0);
// c[n-1] = c_n l3x^n in FP32, n = 1..p: the far-field Taylor coefficient of
// Eq. 9 per power of the lattice offset u (theta_x - x_node = u l3x).
__host__ __device__ inline size_t node_stride(int p) { return 24 + 8 * (size_t)p; }

// Everything a shooting or tracing kernel needs.
struct ShootArgs {
    Geo g;
    LensTable L;
    const double *coef64;           // (p+1) complex FP64 per node (near/far FP64 mode)
    const unsigned char *nodes;     // node records (mixed mode)
    uint32_t *map_u32;
    float *map_f32;
    unsigned long long *stats;      // ML_STAT_* counters on the device
    unsigned int *status;           // bit 0 overflow, bit 1 aborted
    unsigned long long *work;       // persistent-kernel task counter
    const volatile int *abort_flag; // mapped host flag
    // ray range of this launch
    int64_t ray_begin, ray_end;
    // task decomposition of the mixed kernel
    int64_t rg_first, n_rg, groups_per_band, n_cc, cc_per_l1, l2_per_cc;
    int64_t n_tasks;
    int near_cap;                   // float4 slots of shared memory per warp
    int walk;                       // ML_WALK_CERTIFIED or ML_WALK_PER_RAY (mixed NGP)
    float span_far;                 // certified walk: lens columns spanned only if every near
                                    // lens lies farther than this (lattice units)
    // float constants of the mixed kernel
    float l3x_f, l3x_lo, c0_f, ipx_f, ipy_f;
    float cxy_f;                    // change of the u slope of beta_x per ray row (fold: d_y l3y l3x / dpx)
    float q2_f;                     // beta_x curvature in u (fold: d_x l3x^2 / (2 dpx)), else 0
    float rc2;                      // close-pass radius^2 of near_sum_f32 (theta_E^2)
    float rc2u;                     // the same in lattice units (near_sum_lat)
    float l3yx_f;                   // l3y / l3x: a ray row in lattice units
    float yx_f;                     // dpx / dpy: y deflection per x deflection unit (pixels)
    double rho_y;                   // (d(macro_y)/d(theta_y) + kappa_*) * l3y / dpy
    double l3yx;                    // l3y / l3x (FP64)
    double il3x;                    // 1 / l3x
    double mpx;                     // 1 / (l3x dpx): lens mass to lattice-unit pixel deflection
};

// Many maps in one persistent launch: per-map arguments (device array) and
// the prefix sums of their task counts.
struct BatchArgs {
    const ShootArgs *args;
    const int64_t *task_base;       // n_maps + 1 entries
    int n_maps;
    int near_cap;                   // largest near_cap of the maps
    int walk;                       // ML_WALK_* of every map of the batch
    int64_t total_tasks;
    unsigned long long *work;
    const volatile int *abort_flag;
    unsigned int *status;           // bit 1: aborted
};

// ---- launch wrappers (defined in the .cu files) ----
cudaError_t launch_lens_cells(const Geo &g, const double *x, const double *y, int64_t n,
                              int32_t *cell, int32_t *count, cudaStream_t s);
cudaError_t launch_scan(const int32_t *count, int32_t *start, int64_t nb, cudaStream_t s);
cudaError_t launch_scatter(const double *x, const double *y, const double *m,
                           const int32_t *cell, int64_t n, const int32_t *start, int64_t nb,
                           double *sx, double *sy, double *sm, int32_t *scell, int32_t *perm,
                           float *f32, cudaStream_t s);
cudaError_t launch_split_f32(const double *x, const double *y, const double *m, int64_t n,
                             float *f32, cudaStream_t s);
// FP32 copies of n lenses in one buffer of 5 n floats: xh, xl, yh, yl, mf
inline void set_f32(LensTable &L, const float *f32, int64_t n)
{
    L.xh = f32; L.xl = f32 + n; L.yh = f32 + 2 * n; L.yl = f32 + 3 * n; L.mf = f32 + 4 * n;
}
cudaError_t launch_p_bound(const Geo &g, const LensTable &L, double *bound, cudaStream_t s);
cudaError_t launch_coeffs_direct(const Geo &g, const LensTable &L, double *coef64, cudaStream_t s);
cudaError_t launch_coeffs_hier(const Geo &g, const LensTable &L, double *coef64, double *scratch,
                               size_t scratch_doubles, cudaStream_t s);
size_t hier_scratch_doubles(const Geo &g);
cudaError_t launch_node_finalize(const Geo &g, const double *coef64, unsigned char *nodes,
                                 cudaStream_t s);
cudaError_t launch_shoot(const ShootArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_trace(const ShootArgs &a, const int64_t *idx, int64_t n, double *beta,
                         int32_t *pix, cudaStream_t s);
cudaError_t launch_batch(const BatchArgs &b, int p, int num_sms, cudaStream_t s);
cudaError_t launch_cic_adjoint_direct(const ShootArgs &a, const float *G, const double *lx,
                                      const double *ly, const double *lm, int64_t n_lens,
                                      double *glens, double *gpar, double scale, int num_sms,
                                      cudaStream_t s);
cudaError_t launch_cic_adjoint_nearfar(const ShootArgs &a, const float *G, double *gs, double *gpar,
                                       double2 *mom, const int32_t *perm, double *glens, double scale,
                                       int num_sms, cudaStream_t s);
cudaError_t launch_mu(const Geo &g, const uint32_t *cu, const float *cf, int want, void *out,
                      double scale, cudaStream_t s);
cudaError_t launch_light_curves(const Geo &g, const uint32_t *cu, const float *cf, double scale,
                                const double *tracks, int n_tracks, int n_samples,
                                double sigma_px, float *out, cudaStream_t s);
cudaError_t launch_light_curves_noalloc(const Geo &g, const uint32_t *cu, const float *cf,
                                        double scale, const double *tracks_host, int n_tracks,
                                        int n_samples, double sigma_px, float *out, cudaStream_t s);
int light_curve_taps(double sigma_px, float taps[129]);
cudaError_t launch_peaks(const uint32_t *N, int nx, int ny, int along, double nsigma, uint8_t *mask,
                         int32_t *peaks, int64_t capacity, unsigned long long *found, cudaStream_t s);
cudaError_t launch_map_sum(const uint32_t *map, size_t n, unsigned long long *sum, int num_sms,
                           cudaStream_t s);
cudaError_t launch_light_curves_adj(int mnx, int mny, const double *d_tracks, int n_tracks,
                                    int n_samples, double sigma_px, const float *dl, float *gmap,
                                    cudaStream_t s);
cudaError_t launch_light_curves_dev(const Geo &g, const uint32_t *cu, const float *cf, double scale,
                                    const double *d_tracks, int n_tracks, int n_samples, int h,
                                    const float *d_taps, float *out, cudaStream_t s);
int mixed_p_supported(int p);     // the Taylor order the mixed kernel will use for p
// FP32 FMA throughput probe: blocks x 256 threads, eight chains of `iters`
// FMAs each (scalar, or two-lane fma.rn.f32x2); fma_peak_flop is its flop count.
cudaError_t launch_fma_peak(bool two_lane, unsigned blocks, int64_t iters, float *sink,
                            cudaStream_t s);
double fma_peak_flop(bool two_lane, unsigned blocks, int64_t iters);

// ---- shared device arithmetic ---------------------------------------------

#if defined(__CUDACC__)

// Inside the sheet, beta gains kappa_* (theta - c) (disc) or
// 2 kappa_* (theta_y - c_y) y-hat (strip): the linear coefficients.
__host__ __device__ inline double sheet_kx(const Geo &g) { return g.sheet_shape == ML_SHEET_STRIP ? 0.0 : g.kappa_star; }
__host__ __device__ inline double sheet_ky(const Geo &g) { return g.sheet_shape == ML_SHEET_STRIP ? 2.0 * g.kappa_star : g.kappa_star; }

// The smooth (macro) part of beta in FP64: the constant-(kappa, gamma) form
// of Eq. 1, or the fold of Eq. 5 as printed in Eq. 6.
__host__ __device__ inline void macro64(const Geo &g, double tx, double ty, double &mx, double &my)
{
    if (g.macro == ML_MACRO_FOLD) {
        mx = 0.5 * g.dx * tx * tx + g.dy * tx * ty;
        my = 2.0 * (1.0 - g.kappa0) * ty;
    } else {
        mx = (1.0 - g.kappa - g.gamma) * tx;
        my = (1.0 - g.kappa + g.gamma) * ty;
    }
}

// Near-lens records in theta units (CIC forward and adjoint): rec(k) =
// (x_k - x_node, y_k - y_ref, m_k, -) rounded to FP32, lo(k) = the rounding
// remainders of the two offsets.  Deflection of the near lenses (the directly
// summed part of Eq. 9) in FP32 on these node-relative coordinates:
//   dx = t - lx,  dy = dyl - ly,  t = u * l3x (u a half-integer lattice offset).
// The FP32 rounding of the offsets costs a relative error of about
// 2^-23 (|t| + |dyl|) / r for a ray at distance r from a lens.  Rays that pass
// closer than r_c (sqrt(rc2), where that error could exceed 5e-7) redo the
// sum with the offsets carried as hi + lo float pairs (near_sum_hilo).
//
// The counting kernels (NGP) and the tracer take the same sum in lattice
// units: offsets divided by l3x, so that the ray's x offset is u itself
// (exact in FP32), and masses scaled to pixel units, m' = m / (l3x dpx).  The
// near deflection then adds to the row polynomial's pixel value directly:
//   X += (lx - u) m' / r^2,  Y += (ly - dyl) (dpx/dpy) m' / r^2.
// The same error argument holds with r_c / l3x (rc2u).
// Approximate reciprocal (the PTX rcp.approx.ftz.f32 instruction, relative
// error below 2^-23).  The near sums use m * rcp(r^2); r^2 never comes near
// the float range limits for lenses and rays inside a field.
__device__ __forceinline__ float rcp_approx(float y)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

template <class Near>
__device__ __forceinline__ void near_sum_f32(const Near &nl, int nn, float t, float dyl,
                                             float &ax, float &ay, float &rmin)
{
    float sx = 0.f, sy = 0.f, mn = 3.0e38f;
    for (int k = 0; k < nn; ++k) {
        float4 L = nl.rec(k);
        float dy = __fsub_rn(dyl, L.y);
        float dy2 = __fmul_rn(dy, dy);
        float dx = __fsub_rn(t, L.x);
        float r2 = __fmaf_rn(dx, dx, dy2);
        mn = fminf(mn, r2);
        float s = __fmul_rn(L.z, rcp_approx(r2));
        sx = __fmaf_rn(dx, s, sx);
        sy = __fmaf_rn(dy, s, sy);
    }
    ax = sx;
    ay = sy;
    rmin = mn;
}

// Lattice-unit near sum of one ray at offset u, added to the ray's pixel
// position (X, Y); rmin = the smallest r^2 (lattice units).
template <class Near>
__device__ __forceinline__ void near_sum_lat(const Near &nl, int nn, float u, float dyl, float yx,
                                             float &X, float &Y, float &rmin)
{
    float mn = 3.0e38f;
    for (int k = 0; k < nn; ++k) {
        float4 L = nl.rec(k);
        float dy = __fsub_rn(L.y, dyl);
        float dy2 = __fmul_rn(dy, dy);
        float dyy = __fmul_rn(dy, yx);
        float dx = __fsub_rn(L.x, u);
        float r2 = __fmaf_rn(dx, dx, dy2);
        mn = fminf(mn, r2);
        float s = __fmul_rn(L.z, rcp_approx(r2));
        X = __fmaf_rn(dx, s, X);
        Y = __fmaf_rn(dyy, s, Y);
    }
    rmin = mn;
}

// The same for two rays of one row (u0, u1), sharing each lens record and
// dy; per ray the operations are exactly those of near_sum_lat.
template <class Near>
__device__ __forceinline__ void near_sum2_lat(const Near &nl, int nn, float u0, float u1, float dyl,
                                              float yx, float &X0, float &Y0, float &rmin0,
                                              float &X1, float &Y1, float &rmin1)
{
    float mn0 = 3.0e38f, mn1 = 3.0e38f;
    for (int k = 0; k < nn; ++k) {
        float4 L = nl.rec(k);
        float dy = __fsub_rn(L.y, dyl);
        float dy2 = __fmul_rn(dy, dy);
        float dyy = __fmul_rn(dy, yx);
        float dx0 = __fsub_rn(L.x, u0);
        float dx1 = __fsub_rn(L.x, u1);
        float r20 = __fmaf_rn(dx0, dx0, dy2);
        float r21 = __fmaf_rn(dx1, dx1, dy2);
        mn0 = fminf(mn0, r20);
        mn1 = fminf(mn1, r21);
        float s0 = __fmul_rn(L.z, rcp_approx(r20));
        float s1 = __fmul_rn(L.z, rcp_approx(r21));
        X0 = __fmaf_rn(dx0, s0, X0);
        Y0 = __fmaf_rn(dyy, s0, Y0);
        X1 = __fmaf_rn(dx1, s1, X1);
        Y1 = __fmaf_rn(dyy, s1, Y1);
    }
    rmin0 = mn0;
    rmin1 = mn1;
}

// Close-pass path in lattice units: u is exact, so only the records' and the
// row's rounding remainders are carried.  Adds to (X, Y), which the caller
// resets to the row polynomial's value.  Returns false when the ray
// coincides with a lens even at this precision.
template <class Near>
__device__ __forceinline__ bool near_sum_hilo_lat(const Near &nl, int nn, float u, float dyl,
                                                  float dyl_lo, float yx, float &X, float &Y)
{
    bool hit = false;
    for (int k = 0; k < nn; ++k) {
        float4 L = nl.rec(k);
        float2 R = nl.lo(k);
        float dx = __fadd_rn(__fsub_rn(L.x, u), R.x);
        float dy = __fadd_rn(__fsub_rn(L.y, dyl), __fsub_rn(R.y, dyl_lo));
        float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        hit |= (r2 == 0.f);
        float s = __fmul_rn(L.z, rcp_approx(r2));
        X = __fmaf_rn(dx, s, X);
        Y = __fmaf_rn(__fmul_rn(dy, yx), s, Y);
    }
    return !hit;
}

// Close-pass path: the near sum with the offsets carried as hi + lo float
// pairs (t = u * (l3x_hi + l3x_lo) split by an exact FMA remainder).  Returns
// false when the ray coincides with a lens even at this precision.
template <class Near>
__device__ __forceinline__ bool near_sum_hilo(const Near &nl, int nn, float u, float t, float dyl,
                                           float dyl_lo, float l3x_hi, float l3x_lo,
                                           float &ax, float &ay)
{
    float t_lo = __fmaf_rn(u, l3x_lo, __fmaf_rn(u, l3x_hi, -t));
    float sx = 0.f, sy = 0.f;
    bool hit = false;
    for (int k = 0; k < nn; ++k) {
        float4 L = nl.rec(k);
        float2 R = nl.lo(k);
        float dx = __fadd_rn(__fsub_rn(t, L.x), __fsub_rn(t_lo, R.x));
        float dy = __fadd_rn(__fsub_rn(dyl, L.y), __fsub_rn(dyl_lo, R.y));
        float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        hit |= (r2 == 0.f);
        float s = __fmul_rn(L.z, rcp_approx(r2));
        sx = __fmaf_rn(dx, s, sx);
        sy = __fmaf_rn(dy, s, sy);
    }
    ax = sx;
    ay = sy;
    return !hit;
}

// Near records staged in shared memory by the shooting kernels.
struct SmemNear {
    const float4 *near;
    const float2 *lo_;
    __device__ __forceinline__ float4 rec(int k) const { return near[k]; }
    __device__ __forceinline__ float2 lo(int k) const { return lo_[k]; }
};

// Per-ray-row polynomial of the smooth part of beta (map pixel units) in the
// node-relative lattice offset u (theta_x - x_node = u l3x):
// X(u) = sum X[m] u^m,  Y(u) = sum Y[m] u^m, with integer bases bx, by
// (pixel = base + floor(value)).
template <int P>
struct RowPoly {
    float X[P + 1], Y[P + 1];
    int bx, by;
};

// The smooth y shift of a ray row at node-relative offset q * l3y (q a
// half-integer): q * rho_y pixels, taken once per row in FP64 and split into
// an integer and an FP32 fraction, so that the per-node row setup needs no
// FP64 arithmetic (this GPU's FP64 rate is 1/64 of FP32's).
struct RowY {
    int iq;
    float fq;
};

__device__ __forceinline__ RowY row_y(float q, const ShootArgs &a)
{
    const double y = (double)q * a.rho_y;
    const double k = floor(y);
    return RowY{(int)k, (float)(y - k)};
}

// Build the row polynomial of one node for the ray row at node-relative y
// offset q * l3y (q a half-integer), in lattice units s = q l3y / l3x: the
// far series F = sum_{n=1..P} c_n l3x^n (u + i s)^n is re-expanded in u by a
// Taylor shift (repeated synthetic division), then beta_x = Sx + Ax u -
// Re F / dpx and beta_y = Sy + Ay q + Im F / dpy.
template <int P>
__device__ __forceinline__ void row_setup(const unsigned char *rec, float q, RowY ry, const ShootArgs &a,
                                          RowPoly<P> &rp)
{
    const int by0 = *reinterpret_cast<const int *>(rec);
    const float fy = *reinterpret_cast<const float *>(rec + 4);
    const int bx0 = *reinterpret_cast<const int *>(rec + 8);
    const float fx = *reinterpret_cast<const float *>(rec + 12);
    const float axn = *reinterpret_cast<const float *>(rec + 16);
    const float bqn = *reinterpret_cast<const float *>(rec + 20);
    const float2 *c = reinterpret_cast<const float2 *>(rec + 24);
    const float s = __fmul_rn(q, a.l3yx_f);
    float br[P + 1], bi[P + 1];
    br[0] = 0.f;
    bi[0] = 0.f;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        float2 cn = c[n - 1];
        br[n] = cn.x;
        bi[n] = cn.y;
    }
    // b_n += (i s) b_{n+1}:  (i s)(u + i v) = -s v + i s u
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int n = P - 1; n >= k; --n) {
            float nr = __fmaf_rn(-s, bi[n + 1], br[n]);
            float ni = __fmaf_rn(s, br[n + 1], bi[n]);
            br[n] = nr;
            bi[n] = ni;
        }
    }
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        rp.X[m] = __fmul_rn(-br[m], a.ipx_f);
        rp.Y[m] = __fmul_rn(bi[m], a.ipy_f);
    }
    // macro and sheet terms: slope at the node plus its change per row, the
    // fold's curvature, and the fold's per-row shift of beta_x
    rp.X[1] = __fadd_rn(rp.X[1], __fmaf_rn(a.cxy_f, q, axn));
    if constexpr (P >= 2) rp.X[2] = __fadd_rn(rp.X[2], a.q2_f);
    // x base: fx in [0, 1) plus the far-field offset of this row
    float x0 = __fadd_rn(__fmaf_rn(bqn, q, fx), rp.X[0]);
    float kx = floorf(x0);
    rp.X[0] = __fsub_rn(x0, kx);
    rp.bx = bx0 + (int)kx;
    // y base: the node's and the row's integer parts, their fractions and
    // the far-field offset of this row in FP32
    float y0f = __fadd_rn(__fadd_rn(fy, ry.fq), rp.Y[0]);
    float ky = floorf(y0f);
    rp.Y[0] = __fsub_rn(y0f, ky);
    rp.by = by0 + ry.iq + (int)ky;
}

template <int P>
__device__ __forceinline__ void row_eval(const RowPoly<P> &rp, float u, float &X, float &Y)
{
    float x = rp.X[P], y = rp.Y[P];
#pragma unroll
    for (int m = P - 1; m >= 0; --m) {
        x = __fmaf_rn(x, u, rp.X[m]);
        y = __fmaf_rn(y, u, rp.Y[m]);
    }
    X = x;
    Y = y;
}

// Pairs of FP32 values in one 64-bit register for Blackwell's two-lane FP32
// instructions (add/fma .f32x2): each lane is rounded exactly as the scalar
// instruction, so a pair computes the same bits as two scalar operations in
// one issue slot.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Both lanes rounded toward -inf (the floor trick below, on a pair).
__device__ __forceinline__ f32x2 add2_rd(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// floor(X) as an int using FP32 adds only.  On this GPU float-to-int
// conversions issue to the narrow FP64 pipe, which a per-ray conversion
// saturates.  For |X| < 2^22 the sum X + 1.5 * 2^23 rounded toward -inf is
// exactly 1.5 * 2^23 + floor(X) (its ulp is 1), and its bit pattern minus
// that of 1.5 * 2^23 is floor(X).  Larger |X| (and +-inf, NaN) give results
// of magnitude >= 2^22 with the sign of X: pixels far outside any map.
__device__ __forceinline__ int floor_to_int(float X)
{
    return __float_as_int(__fadd_rd(X, 12582912.0f)) - 0x4B400000;
}

// floor(X) both as an int and as a float (exact for |X| < 2^22).
__device__ __forceinline__ int floor_both(float X, float &fl)
{
    float s = __fadd_rd(X, 12582912.0f);
    fl = __fsub_rn(s, 12582912.0f);
    return __float_as_int(s) - 0x4B400000;
}

// Quad (lower-left pixel) and bilinear weights of a ray at pixel-unit (X, Y)
// off the row bases.
__device__ __forceinline__ void cic_quad(const int bx, const int by, float X, float Y, unsigned &ix,
                                         unsigned &iy, float &wx, float &wy)
{
    const float fx = __fsub_rn(X, 0.5f), fy = __fsub_rn(Y, 0.5f);
    float flx, fly;
    const int kx = floor_both(fx, flx), ky = floor_both(fy, fly);
    wx = __fsub_rn(fx, flx);
    wy = __fsub_rn(fy, fly);
    ix = (unsigned)bx + (unsigned)kx;
    iy = (unsigned)by + (unsigned)ky;
}

// Nearest-grid-point pixel coordinates of the ray (Eq. 12 binning), before
// the bounds check; wrapping 32-bit arithmetic keeps far values out of
// [0, mnx) x [0, mny).
__device__ __forceinline__ void pixel_xy(float X, float Y, int bx, int by, int &gx, int &gy)
{
    gx = (int)((unsigned)bx + (unsigned)floor_to_int(X));
    gy = (int)((unsigned)by + (unsigned)floor_to_int(Y));
}

#endif  // __CUDACC__

}  // namespace ml
