// C ABI of the microlensing library: descriptor validation, the parameter
// derivation of §3.1-§3.2, device buffers, and stream-ordered launches.
#include "ml_internal.cuh"
#include "ml_alloc.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

using namespace ml;

namespace {

thread_local std::string g_err;

ml_status fail(ml_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

ml_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ML_ERR_OOM : ML_ERR_CUDA;
}

#define ML_CK(call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);           \
    } while (0)

// Abort flags live in mapped pinned host memory.  Pinning memory is an
// operating-system call that costs far more than a field's other set-up, so
// the flags come from a process-wide pool of pinned pages (one int per field
// or batch), reused after release.
struct FlagPool {
    std::mutex mu;
    std::vector<int *> free_slots;
};
FlagPool g_flags;
constexpr int kFlagsPerPage = 1024;

cudaError_t flag_get(int **h, int **d)
{
    std::lock_guard<std::mutex> lock(g_flags.mu);
    if (g_flags.free_slots.empty()) {
        int *page = nullptr;
        cudaError_t e = cudaHostAlloc((void **)&page, kFlagsPerPage * sizeof(int),
                                      cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return e;
        for (int i = kFlagsPerPage - 1; i >= 0; --i) g_flags.free_slots.push_back(page + i);
    }
    int *slot = g_flags.free_slots.back();
    cudaError_t e = cudaHostGetDevicePointer((void **)d, slot, 0);
    if (e != cudaSuccess) return e;
    g_flags.free_slots.pop_back();
    *slot = 0;
    *h = slot;
    return cudaSuccess;
}

void flag_put(int *h)
{
    if (!h) return;
    std::lock_guard<std::mutex> lock(g_flags.mu);
    g_flags.free_slots.push_back(h);
}

}  // namespace

struct ml_field {
    Geo g{};
    int device = 0;
    int num_sms = 0;
    int build_used = 0;
    double far_bound = 0.0;
    int32_t max_near = 0;
    uint64_t max_launch_rays = 0;
    uint64_t rays_asked = 0, launches = 0;
    int64_t n_lens = 0;
    int32_t tuned = 0;
    // certified walk: a warp's level-2 column with near lenses is spanned only
    // if they all lie farther than this from its rays (lattice units; +inf:
    // such columns always take the per-ray walk); the autotuner measures both
    float span_far = ML_SPAN_FAR;
    // certified walk at all: false runs the per-ray kernel (the autotuner
    // measures it beside the two thresholds; fields with near lenses nearly
    // everywhere gain nothing from spans)
    bool use_span = true;
    ml_field_desc desc{};            // parameters (lens pointers cleared)
    std::vector<double> worst;       // truncation bound per Taylor order (worst level-1 cell)
    // device buffers
    double *d_x = nullptr, *d_y = nullptr, *d_m = nullptr;
    int32_t *d_cell = nullptr, *d_count = nullptr, *d_start = nullptr;
    double *d_sx = nullptr, *d_sy = nullptr, *d_sm = nullptr;
    float *d_f32 = nullptr;          // FP32 copies of the sorted lenses (LensTable xh..mf)
    int32_t *d_scell = nullptr;
    int32_t *d_perm = nullptr;       // sorted position -> index in the caller's lens arrays
    double *d_coef64 = nullptr;
    unsigned char *d_nodes = nullptr;
    uint32_t *d_map_u32 = nullptr;
    float *d_map_f32 = nullptr;
    unsigned long long *d_stats = nullptr, *d_work = nullptr, *d_sum = nullptr;
    // map sum bookkeeping for the wrap-around check: the map's 64-bit sum
    // must equal map_base + (rays_in - in_at_set)
    uint64_t map_base = 0, in_at_set = 0;
    unsigned int *d_status = nullptr;
    int *h_abort = nullptr, *d_abort = nullptr;
    std::vector<void *> owned;       // device allocations to free

    template <class T>
    cudaError_t alloc(T **p, size_t count, cudaStream_t s)
    {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = ml_malloc_async((void **)p, count * sizeof(T), s);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    }
    void release()
    {
        if (!owned.empty() || h_abort) cudaDeviceSynchronize();
        for (void *p : owned) cudaFree(p);
        owned.clear();
        flag_put(h_abort);
        h_abort = nullptr;
    }
    LensTable table() const
    {
        LensTable L;
        L.x = d_sx; L.y = d_sy; L.m = d_sm; L.cell = d_scell; L.start = d_start; L.n = n_lens;
        set_f32(L, d_f32, n_lens);
        return L;
    }
};

namespace {

bool is_fin(double v) { return isfinite(v) != 0; }

int64_t round_half_up(double v) { return (int64_t)floor(v + 0.5); }

// §3.1-§3.2: ray rectangle, lattice, N_*, level grids.
ml_status derive_geometry(const ml_field_desc &d, const std::vector<double> &hx,
                          const std::vector<double> &hy, Geo &g)
{
    g.kappa = d.kappa;
    g.gamma = d.gamma;
    g.kappa_star = d.kappa_star;
    g.macro = d.macro_mode;
    g.kappa0 = d.kappa0;
    g.dx = d.d_x;
    g.dy = d.d_y;
    g.sheet_cx = d.sheet_cx;
    g.sheet_cy = d.sheet_cy;
    g.sheet_r = d.sheet_radius;
    g.sheet_shape = d.sheet_shape;
    g.precision = d.precision;
    g.deposit = d.deposit;
    g.mnx = d.map_nx;
    g.mny = d.map_ny;
    g.mx0 = d.map_x0;
    g.my0 = d.map_y0;
    g.dpx = (d.map_x1 - d.map_x0) / d.map_nx;
    g.dpy = (d.map_y1 - d.map_y0) / d.map_ny;
    double rx0, rx1, ry0, ry1;
    if (d.ray_x0 == 0.0 && d.ray_y0 == 0.0 && d.ray_x1 == 0.0 && d.ray_y1 == 0.0 &&
        d.macro_mode == ML_MACRO_FOLD) {
        // bounding box of the pre-image of s' under the fold map (Eq. 5):
        // theta_y = beta_y / (2 (1 - kappa0)); for fixed theta_y and d_x > 0 the
        // images of beta_x <= b1 lie within t* +- s1, t* = -d_y theta_y / d_x,
        // s1 = sqrt(2 b1 / d_x + (d_y theta_y / d_x)^2); t* + s1 is convex and
        // t* - s1 concave in theta_y, so the extremes sit at the ends of its range
        const double w = 0.5 * (20.0 * sqrt(d.kappa_star));
        const double a = 2.0 * (1.0 - d.kappa0);
        double b0 = d.map_x0 - w, b1 = d.map_x1 + w, dx = d.d_x, dy = d.d_y;
        if (dx < 0.0) {              // mirror beta_x
            const double t = b0;
            b0 = -b1;
            b1 = -t;
            dx = -dx;
            dy = -dy;
        }
        (void)b0;
        if (!(b1 > 0.0))
            return fail(ML_ERR_INVALID_ARG, "the protected map has no images under the fold map "
                                            "(it lies beyond the caustic)");
        const double ty[2] = {(d.map_y0 - w) / a, (d.map_y1 + w) / a};
        rx0 = INFINITY;
        rx1 = -INFINITY;
        for (double t : ty) {
            const double c = -dy * t / dx;
            const double s1 = sqrt(2.0 * b1 / dx + (dy * t / dx) * (dy * t / dx));
            rx0 = std::min(rx0, c - s1);
            rx1 = std::max(rx1, c + s1);
        }
        ry0 = std::min(ty[0], ty[1]);
        ry1 = std::max(ty[0], ty[1]);
    } else if (d.ray_x0 == 0.0 && d.ray_y0 == 0.0 && d.ray_x1 == 0.0 && d.ray_y1 == 0.0) {
        // pre-image of s' = s widened by 10 sqrt(kappa_*) per side (§3.1)
        double w = 0.5 * (20.0 * sqrt(d.kappa_star));
        double a = 1.0 - d.kappa - d.gamma, b = 1.0 - d.kappa + d.gamma;
        if (a == 0.0 || b == 0.0)
            return fail(ML_ERR_INVALID_ARG, "macro map is singular (1-kappa-gamma or 1-kappa+gamma "
                                            "is 0): give the ray rectangle explicitly");
        double xa = (d.map_x0 - w) / a, xb = (d.map_x1 + w) / a;
        double ya = (d.map_y0 - w) / b, yb = (d.map_y1 + w) / b;
        rx0 = std::min(xa, xb); rx1 = std::max(xa, xb);
        ry0 = std::min(ya, yb); ry1 = std::max(ya, yb);
    } else {
        rx0 = d.ray_x0; rx1 = d.ray_x1; ry0 = d.ray_y0; ry1 = d.ray_y1;
    }
    if (!(rx1 > rx0) || !(ry1 > ry0) || !is_fin(rx0) || !is_fin(rx1) || !is_fin(ry0) ||
        !is_fin(ry1))
        return fail(ML_ERR_INVALID_ARG, "empty or non-finite ray rectangle");
    g.rx0 = rx0; g.rx1 = rx1; g.ry0 = ry0; g.ry1 = ry1;
    double lix = rx1 - rx0, liy = ry1 - ry0;
    if (d.n_rays_x == 0 && d.n_rays_y == 0) {
        if (!(d.n_av > 0.0) || !is_fin(d.n_av))
            return fail(ML_ERR_INVALID_ARG, "need n_av > 0 or explicit n_rays_x, n_rays_y");
        double n_rays = d.n_av * d.map_nx * d.map_ny;          // Eq. 8
        double l3 = sqrt(lix * liy / n_rays);                  // Eq. 11
        g.n3x = std::max<int64_t>(1, round_half_up(lix / l3));
        g.n3y = std::max<int64_t>(1, round_half_up(liy / l3));
    } else {
        if (d.n_rays_x <= 0 || d.n_rays_y <= 0)
            return fail(ML_ERR_INVALID_ARG, "n_rays_x and n_rays_y must both be positive");
        g.n3x = d.n_rays_x;
        g.n3y = d.n_rays_y;
    }
    if ((double)g.n3x * (double)g.n3y > 9.0e18)
        return fail(ML_ERR_INVALID_ARG, "ray lattice too large for 64-bit indices");
    g.l3x = lix / g.n3x;
    g.l3y = liy / g.n3y;
    int64_t n_in = 0;
    for (size_t k = 0; k < hx.size(); ++k)
        if (hx[k] >= rx0 && hx[k] < rx1 && hy[k] >= ry0 && hy[k] < ry1) ++n_in;
    g.n_star_in = n_in;
    g.l0 = n_in > 0 ? sqrt(lix * liy / (double)n_in) : INFINITY;
    double l1x = d.l1_x > 0.0 ? d.l1_x : std::min(g.l0, lix / 10.0);   // Eq. 10
    double l1y = d.l1_y > 0.0 ? d.l1_y : std::min(g.l0, liy / 10.0);
    g.l2sx = d.l2_sub_x > 0 ? d.l2_sub_x : 20;
    g.l2sy = d.l2_sub_y > 0 ? d.l2_sub_y : 20;
    double l2x = l1x / g.l2sx, l2y = l1y / g.l2sy;
    g.n2x = std::max<int64_t>(1, round_half_up(l2x / g.l3x));
    g.n2y = std::max<int64_t>(1, round_half_up(l2y / g.l3y));
    g.n1x = g.l2sx * g.n2x;
    g.n1y = g.l2sy * g.n2y;
    g.N1x = (g.n3x + g.n1x - 1) / g.n1x;
    g.N1y = (g.n3y + g.n1y - 1) / g.n1y;
    g.N2x = (g.n3x + g.n2x - 1) / g.n2x;
    g.N2y = (g.n3y + g.n2y - 1) / g.n2y;
    g.l1x = (double)g.n1x * g.l3x;
    g.l1y = (double)g.n1y * g.l3y;
    g.l2x = (double)g.n2x * g.l3x;
    g.l2y = (double)g.n2y * g.l3y;
    g.NEx = g.N1x + 2;
    g.NEy = g.N1y + 2;
    return ML_OK;
}

ml_status validate(const ml_field_desc *d)
{
    if (!d) return fail(ML_ERR_INVALID_ARG, "desc is NULL");
    if (d->abi_version != ML_ABI_VERSION)
        return fail(ML_ERR_INVALID_ARG, "abi_version mismatch (expected " +
                                            std::to_string(ML_ABI_VERSION) + ")");
    if (d->precision < ML_PREC_DIRECT64 || d->precision > ML_PREC_MIXED)
        return fail(ML_ERR_INVALID_ARG, "unknown precision mode");
    if (d->deposit != ML_DEPOSIT_NGP && d->deposit != ML_DEPOSIT_CIC)
        return fail(ML_ERR_INVALID_ARG, "unknown deposit mode");
    if (d->build < ML_BUILD_AUTO || d->build > ML_BUILD_HIERARCHICAL)
        return fail(ML_ERR_INVALID_ARG, "unknown build mode");
    if (d->n_lens < 0) return fail(ML_ERR_INVALID_ARG, "n_lens < 0");
    if (d->n_lens > 0 && (!d->lens_x || !d->lens_y || !d->lens_m))
        return fail(ML_ERR_INVALID_ARG, "lens arrays are NULL");
    if (d->n_lens > (1 << 30)) return fail(ML_ERR_INVALID_ARG, "too many lenses (max 2^30)");
    if (d->map_nx <= 0 || d->map_ny <= 0) return fail(ML_ERR_INVALID_ARG, "empty map");
    if ((uint64_t)d->map_nx * (uint64_t)d->map_ny >= 0xFFFFFFF0ull)
        return fail(ML_ERR_INVALID_ARG, "map has 2^32 pixels or more");
    if (!(d->map_x1 > d->map_x0) || !(d->map_y1 > d->map_y0) || !is_fin(d->map_x0) ||
        !is_fin(d->map_x1) || !is_fin(d->map_y0) || !is_fin(d->map_y1))
        return fail(ML_ERR_INVALID_ARG, "map rectangle is empty or not finite");
    if (!is_fin(d->kappa) || !is_fin(d->gamma) || !is_fin(d->kappa_star) || d->kappa_star < 0.0)
        return fail(ML_ERR_INVALID_ARG, "kappa, gamma must be finite and kappa_* >= 0");
    if (!is_fin(d->sheet_cx) || !is_fin(d->sheet_cy) || !is_fin(d->sheet_radius) ||
        d->sheet_radius < 0.0)
        return fail(ML_ERR_INVALID_ARG, "sheet disc must be finite with radius >= 0");
    if (d->taylor_p < 0 || d->taylor_p > PMAX)
        return fail(ML_ERR_INVALID_ARG, "taylor_p must be in [0, 16]");
    if (d->l2_sub_x < 0 || d->l2_sub_x > 4096 || d->l2_sub_y < 0 || d->l2_sub_y > 4096)
        return fail(ML_ERR_INVALID_ARG, "bad l2_sub_x / l2_sub_y");
    if (d->l1_x < 0.0 || d->l1_y < 0.0) return fail(ML_ERR_INVALID_ARG, "negative l1 size");
    if (d->far_tol < 0.0) return fail(ML_ERR_INVALID_ARG, "negative far_tol");
    if (d->macro_mode != ML_MACRO_LINEAR && d->macro_mode != ML_MACRO_FOLD)
        return fail(ML_ERR_INVALID_ARG, "unknown macro_mode");
    if (d->sheet_shape != ML_SHEET_DISC && d->sheet_shape != ML_SHEET_STRIP)
        return fail(ML_ERR_INVALID_ARG, "unknown sheet_shape");
    if (d->walk != ML_WALK_CERTIFIED && d->walk != ML_WALK_PER_RAY)
        return fail(ML_ERR_INVALID_ARG, "unknown walk");
    if (!(d->span_far >= 0.0)) return fail(ML_ERR_INVALID_ARG, "span_far must be >= 0");
    if (d->macro_mode == ML_MACRO_FOLD &&
        (!is_fin(d->kappa0) || !is_fin(d->d_x) || !is_fin(d->d_y) || d->kappa0 == 1.0 || d->d_x == 0.0))
        return fail(ML_ERR_INVALID_ARG, "fold macro needs finite kappa0 != 1 and d_x != 0");
    return ML_OK;
}

bool rays_inside_sheet(const Geo &g)
{
    if (g.sheet_shape == ML_SHEET_STRIP)
        return g.ry0 - g.sheet_cy >= -g.sheet_r && g.ry1 - g.sheet_cy <= g.sheet_r;
    double R2 = g.sheet_r * g.sheet_r;
    double xs[2] = {g.rx0 - g.sheet_cx, g.rx1 - g.sheet_cx};
    double ys[2] = {g.ry0 - g.sheet_cy, g.ry1 - g.sheet_cy};
    for (double x : xs)
        for (double y : ys)
            if (x * x + y * y > R2) return false;
    return true;
}

// ---- level-1/level-2 grid autotuner ---------------------------------------------
//
// The paper fixes L1 by Eq. 10 and L2 = L1 / 20.  A finer level-2 grid along
// the long side of the level-1 cells shrinks the expansion radius, so a lower
// Taylor order meets the same truncation bound, at the price of more nodes to
// build; smaller level-1 cells shorten the near lists, at the price of more
// cells and nodes.  The tuner evaluates level-1 scales (1, 1/sqrt 2, 1/2 of
// Eq. 10's size, unless the caller fixed L1) times (l2_sub_x, l2_sub_y)
// candidates with their rigorous bound (one p_bound launch each) and their
// mean near-list length, and ranks them by a cost model of GB300 measurements:
//   time = rays * ray_cost(P, near) + nodes * (P + 1) * node_cost,
// the field's build plus one shot of all its rays.

// Shooting time per ray of the mixed kernel on the whole GB300, in
// picoseconds, against the Taylor order P, measured at a fixed level-2 grid
// on three fields: the paper-scale field (1.36 near lenses per ray) and two
// of the batched maps (2.36 and 3.29), which also have shorter pixel runs.
// Below 1.36 the paper-scale field's curve is scaled by what its smaller
// level-1 cells measured (0.19, 0.37 and 0.73 near lenses per ray: 0.81,
// 0.83 and 0.875 of it at P = 4, 6 and 8 alike).  Fields in between are
// interpolated linearly in the mean near count; above the last curve each
// further near lens adds kCostPairPs.
constexpr int kCostOrders[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
constexpr int kCostRows = 6;
constexpr double kCostNear[kCostRows] = {0.19, 0.37, 0.73, 1.36, 2.36, 3.29};
constexpr double kCost136[10] = {0.837, 0.917, 0.969, 1.04, 1.128, 1.186, 1.335, 1.491, 1.732, 1.978};
constexpr double kCostLow[3] = {0.81, 0.83, 0.875};
constexpr double kCostPs[2][10] = {
    {1.52, 1.604, 1.662, 1.746, 1.824, 1.964, 2.14, 2.331, 2.572, 2.805},
    {1.757, 1.833, 1.894, 1.966, 2.061, 2.235, 2.423, 2.621, 2.832, 3.087},
};
constexpr double kCostPairPs = 0.24;

double cost_row(int r, int q)
{
    if (r < 3) return kCost136[q] * kCostLow[r];
    if (r == 3) return kCost136[q];
    return kCostPs[r - 4][q];
}

double ray_cost_ps(int P, double near_per_ray)
{
    int q = 9;
    for (int i = 0; i < 10; ++i)
        if (kCostOrders[i] >= P) { q = i; break; }
    if (near_per_ray <= kCostNear[0]) return cost_row(0, q);
    if (near_per_ray >= kCostNear[kCostRows - 1])
        return cost_row(kCostRows - 1, q) + (near_per_ray - kCostNear[kCostRows - 1]) * kCostPairPs;
    int r = 0;
    while (near_per_ray >= kCostNear[r + 1]) ++r;
    const double f = (near_per_ray - kCostNear[r]) / (kCostNear[r + 1] - kCostNear[r]);
    return (1.0 - f) * cost_row(r, q) + f * cost_row(r + 1, q);
}
// Field build, nanoseconds: per level-2 node and coefficient, and per
// level-1 cell (truncation bound, box and sub-block series); measured as the
// create time's growth with the node count at a fixed order and with the
// level-1 cell count (paper-scale map and the Table-1 fold field alike).
constexpr double kNodeCostNs = 0.12;
constexpr double kCellCostNs = 400.0;

struct GridChoice {
    int sx = 20, sy = 20, p = 0;
    double l1x = 0.0, l1y = 0.0;    // level-1 size; 0 = Eq. 10's
    double cost = 0.0;
    float span_far = ML_SPAN_FAR;   // certified walk's lens-column threshold (see ml_field)
    bool use_span = true;           // certified walk at all (see ml_field)
};

// One candidate level-2 grid of a field: its subdivisions, the compiled
// Taylor order its truncation bound needs, and its size.
struct TuneCand {
    int sx, sy, P;
    double nodes, rays, cells;
    double near_per_ray;            // mean near-list length over the level-1 cells
    double l1x, l1y;                // level-1 size; 0 = Eq. 10's
    double n2x;                     // rays per level-2 cell along a lattice row
    int walk;                       // ML_WALK_* of the field
    double span_frac;               // expected share of rays the certified walk may span
};

// Shooting time per ray of the certified walk, picoseconds: a least-squares
// fit to 13 grids of the paper-scale field (level-1 cells of 1/2, 1/sqrt 2 and
// 1 times Eq. 10's, level-2 cells of 88 to 1400 rays along a row, p = 4 to 8;
// largest error 8 %).  Per-ray work is small and near lenses, the per-column
// set-up (one per level-2 cell and row) and the order P carry the cost.
double span_cost_ps(int P, double near_per_ray, double n2x)
{
    return 0.145 + 0.238 * near_per_ray + 30.6 / std::max(1.0, n2x) + 0.0159 * P;
}

// The certified walk spans a warp's level-2 column only when every near lens
// lies farther than ML_SPAN_FAR lattice units from its rays; elsewhere it
// runs the per-ray walk.  For lenses spread evenly over the 3 x 3 block of
// level-1 cells, the share of columns without such a lens is
// exp(-near * pi (ML_SPAN_FAR l3)^2 / (9 l1x l1y)).
double span_share(double near_per_ray, double l3, double l1x, double l1y)
{
    const double r = (double)ML_SPAN_FAR * l3;
    return exp(-near_per_ray * 3.14159265358979 * r * r / (9.0 * l1x * l1y));
}

double cand_cost(const TuneCand &c, int P)
{
    const double f = c.walk == ML_WALK_CERTIFIED ? c.span_frac : 0.0;
    const double ps = f * span_cost_ps(P, c.near_per_ray, c.n2x) + (1.0 - f) * ray_cost_ps(P, c.near_per_ray);
    return c.rays * ps * 1e-3 + c.nodes * (P + 1) * kNodeCostNs + c.cells * kCellCostNs;   // ns
}

uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h;
}

uint64_t tune_key(const ml_field_desc &d, const std::vector<double> &hx, const std::vector<double> &hy,
                  const std::vector<double> &hm)
{
    uint64_t h = 1469598103934665603ull;
    auto mixd = [&](double v) { uint64_t u; memcpy(&u, &v, 8); h = mix64(h, u); };
    mixd(d.kappa); mixd(d.gamma); mixd(d.kappa_star); mixd(d.sheet_cx); mixd(d.sheet_cy);
    mixd(d.sheet_radius); mixd(d.ray_x0); mixd(d.ray_y0); mixd(d.ray_x1); mixd(d.ray_y1);
    mixd(d.n_av); mixd(d.map_x0); mixd(d.map_y0); mixd(d.map_x1); mixd(d.map_y1);
    mixd(d.l1_x); mixd(d.l1_y); mixd(d.far_tol);
    h = mix64(h, (uint64_t)d.n_rays_x); h = mix64(h, (uint64_t)d.n_rays_y);
    h = mix64(h, (uint64_t)d.map_nx); h = mix64(h, (uint64_t)d.map_ny);
    h = mix64(h, (uint64_t)d.taylor_p); h = mix64(h, (uint64_t)hx.size());
    h = mix64(h, (uint64_t)d.walk); h = mix64(h, (uint64_t)d.macro_mode);
    h = mix64(h, (uint64_t)d.sheet_shape); mixd(d.kappa0); mixd(d.d_x); mixd(d.d_y);
    // the lens arrays in four independent lanes (no serial dependency per word),
    // then the lanes into the parameter hash
    uint64_t l[4] = {0x243F6A8885A308D3ull, 0x13198A2E03707344ull, 0xA4093822299F31D0ull,
                     0x082EFA98EC4E6C89ull};
    const std::vector<double> *arr[3] = {&hx, &hy, &hm};
    for (const std::vector<double> *a : arr) {
        const size_t n = a->size();
        size_t k = 0;
        for (; k + 4 <= n; k += 4)
            for (int q = 0; q < 4; ++q) {
                uint64_t u;
                memcpy(&u, &(*a)[k + q], 8);
                l[q] = mix64(l[q], u);
            }
        for (; k < n; ++k) {
            uint64_t u;
            memcpy(&u, &(*a)[k], 8);
            l[0] = mix64(l[0], u);
        }
    }
    for (int q = 0; q < 4; ++q) h = mix64(h, l[q]);
    return h;
}

std::mutex g_tune_mu;
std::unordered_map<uint64_t, std::vector<TuneCand>> g_tune_cache;

// Feasible candidate grids of a field (cached per process by a hash of the
// descriptor's parameters and the lens arrays).
ml_status tune_candidates(uint64_t key, const ml_field_desc &d, const std::vector<double> &hx,
                          const std::vector<double> &hy, const std::vector<double> &hm,
                          const double *dx, const double *dy, const double *dm, cudaStream_t s,
                          std::vector<TuneCand> &out)
{
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { out = it->second; return ML_OK; }
    }
    const int64_t n = (int64_t)hx.size();
    Geo g0;
    ml_status st = derive_geometry(d, hx, hy, g0);
    if (st != ML_OK) return st;
    const bool xlong = g0.l1x >= g0.l1y;
    static const int fine[] = {20, 40, 60, 80, 120, 160};
    static const int coarse[] = {10, 20};
    // level-1 scales: Eq. 10's size unless the caller fixed it
    std::vector<double> scales{1.0};
    if (d.l1_x == 0.0 && d.l1_y == 0.0)
        for (double sc : {0.70710678118654752, 0.5, 0.35355339059327373}) scales.push_back(sc);
    struct Cand { int sx, sy; double l1x, l1y; Geo g; int32_t *cells; int32_t *counts; double *bound; };
    std::vector<Cand> cands;
    float *f32 = nullptr;            // FP32 copies of the (unsorted) lenses for the bounds
    cudaError_t e = ml_malloc_async((void **)&f32, sizeof(float) * 5 * (size_t)std::max<int64_t>(n, 1), s);
    if (e == cudaSuccess) e = launch_split_f32(dx, dy, dm, n, f32, s);
    for (double sc : scales)
    for (int a : fine)
        for (int b : coarse) {
            if (e != cudaSuccess) break;
            Cand c{};
            c.sx = xlong ? a : b;
            c.sy = xlong ? b : a;
            c.l1x = sc == 1.0 ? d.l1_x : sc * g0.l1x;
            c.l1y = sc == 1.0 ? d.l1_y : sc * g0.l1y;
            ml_field_desc dc = d;
            dc.l2_sub_x = c.sx;
            dc.l2_sub_y = c.sy;
            dc.l1_x = c.l1x;
            dc.l1_y = c.l1y;
            if (derive_geometry(dc, hx, hy, c.g) != ML_OK) continue;
            if (c.g.n2x < 2 || c.g.n2y < 1 || c.g.N2x * c.g.N2y > ((int64_t)1 << 26)) continue;
            if (c.g.NEx * c.g.NEy >= ((int64_t)1 << 30)) continue;
            const int64_t NE = c.g.NEx * c.g.NEy;
            e = ml_malloc_async((void **)&c.cells, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), s);
            if (e == cudaSuccess) e = ml_malloc_async((void **)&c.counts, sizeof(int32_t) * (size_t)(NE + 1), s);
            if (e == cudaSuccess)
                e = ml_malloc_async((void **)&c.bound, sizeof(double) * (size_t)(c.g.N1x * c.g.N1y * PMAX), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(c.counts, 0, sizeof(int32_t) * (size_t)(NE + 1), s);
            if (e == cudaSuccess) e = launch_lens_cells(c.g, dx, dy, n, c.cells, c.counts, s);
            if (e == cudaSuccess) {
                LensTable L;
                L.x = dx; L.y = dy; L.m = dm; L.cell = c.cells; L.start = nullptr; L.n = n;
                set_f32(L, f32, n);
                c.g.p = 1;
                e = launch_p_bound(c.g, L, c.bound, s);
            }
            cands.push_back(c);
            if (e != cudaSuccess) break;
        }
    const double tol = d.far_tol > 0.0 ? d.far_tol : 1e-7;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<TuneCand> res;
    for (Cand &c : cands) {
        if (e != cudaSuccess) break;
        std::vector<double> bound((size_t)(c.g.N1x * c.g.N1y * PMAX));
        e = cudaMemcpy(bound.data(), c.bound, bound.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        // mean near-list length over the level-1 cells (3 x 3 block counts of
        // the binned lenses; cells of the lattice weigh alike)
        std::vector<int32_t> cnt((size_t)(c.g.NEx * c.g.NEy + 1));
        e = cudaMemcpy(cnt.data(), c.counts, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        double tot = 0.0;
        for (int64_t cy = 0; cy < c.g.N1y; ++cy)
            for (int64_t cx = 0; cx < c.g.N1x; ++cx)
                for (int64_t dy = 0; dy < 3; ++dy)
                    for (int64_t dxx = 0; dxx < 3; ++dxx)
                        tot += cnt[(size_t)((cy + dy) * c.g.NEx + cx + dxx)];
        const double near_per_ray = tot / (double)std::max<int64_t>(1, c.g.N1x * c.g.N1y);
        int p = d.taylor_p;
        if (p == 0) {
            p = PMAX;
            for (int q = 1; q <= PMAX; ++q) {
                double w = 0.0;
                for (size_t k = 0; k < bound.size() / PMAX; ++k) w = std::max(w, bound[k * PMAX + q - 1]);
                if (w <= tol) { p = q; break; }
            }
        }
        if (d.macro_mode == ML_MACRO_FOLD) p = std::max(p, 2);
        res.push_back(TuneCand{c.sx, c.sy, mixed_p_supported(p), (double)c.g.N2x * (double)c.g.N2y,
                               (double)c.g.n3x * (double)c.g.n3y, (double)c.g.N1x * (double)c.g.N1y,
                               near_per_ray, c.l1x, c.l1y, (double)c.g.n2x, d.walk,
                               span_share(near_per_ray, c.g.l3x, c.g.l1x, c.g.l1y)});
    }
    for (Cand &c : cands) {
        if (c.cells) cudaFreeAsync(c.cells, s);
        if (c.counts) cudaFreeAsync(c.counts, s);
        if (c.bound) cudaFreeAsync(c.bound, s);
    }
    if (f32) cudaFreeAsync(f32, s);
    if (e != cudaSuccess) return cuda_fail(e, "grid autotuner");
    out = res;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = res;
    return ML_OK;
}

// Cheapest candidate of a single field (its own order).
GridChoice best_single(const std::vector<TuneCand> &cands)
{
    GridChoice best;
    bool found = false;
    for (const TuneCand &c : cands) {
        double cost = cand_cost(c, c.P);
        if (!found || cost < best.cost) {
            best.sx = c.sx; best.sy = c.sy; best.p = c.P; best.cost = cost;
            best.l1x = c.l1x; best.l1y = c.l1y;
            found = true;
        }
    }
    return best;
}

ml_status measure_grid(const ml_field_desc &d, const std::vector<double> &hx, const std::vector<double> &hy,
                       const std::vector<double> &hm, const TuneCand &c, cudaStream_t s, double &est_ms,
                       float &span_far, bool &use_span);

std::unordered_map<uint64_t, GridChoice> g_measured;   // guarded by g_tune_mu

// The model ranks the candidates; with `measure` its best grid at each of
// the three best level-1 scales is built and timed (measure_grid) and the
// fastest by measurement is taken.  The
// model's error is largest between fields of different kinds (walk lengths,
// pixel runs), which the measurement settles; its cost, about the build and
// a fiftieth of one shot per candidate, is paid once per process and field.
ml_status tune_grid(const ml_field_desc &d, const std::vector<double> &hx, const std::vector<double> &hy,
                    const std::vector<double> &hm, const double *dx, const double *dy, const double *dm,
                    cudaStream_t s, bool measure, GridChoice &best)
{
    std::vector<TuneCand> cands;
    const uint64_t key = tune_key(d, hx, hy, hm);
    ml_status st = tune_candidates(key, d, hx, hy, hm, dx, dy, dm, s, cands);
    if (st != ML_OK) return st;
    best = cands.empty() ? GridChoice() : best_single(cands);
    if (!measure || cands.size() < 2) return ML_OK;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_measured.find(key);
        if (it != g_measured.end()) { best = it->second; return ML_OK; }
    }
    // the model's best grid at each level-1 scale, best scales first: the
    // level-1 size moves the near-lens count, where the model is least sure
    std::vector<size_t> order;
    for (size_t i = 0; i < cands.size(); ++i) {
        bool placed = false;
        for (size_t &j : order)
            if (cands[j].l1x == cands[i].l1x && cands[j].l1y == cands[i].l1y) {
                if (cand_cost(cands[i], cands[i].P) < cand_cost(cands[j], cands[j].P)) j = i;
                placed = true;
                break;
            }
        if (!placed) order.push_back(i);
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return cand_cost(cands[a], cands[a].P) < cand_cost(cands[b], cands[b].P);
    });
    double best_est = 0.0;
    bool found = false;
    for (size_t i = 0; i < std::min<size_t>(3, order.size()); ++i) {
        const TuneCand &c = cands[order[i]];
        double est = 0.0;
        float far = ML_SPAN_FAR;
        bool span = true;
        // a candidate that cannot be built (near lists too long for the
        // mixed kernel's shared memory, memory) is passed over
        if (measure_grid(d, hx, hy, hm, c, s, est, far, span) != ML_OK) {
            cudaGetLastError();
            continue;
        }
        if (getenv("ML_TUNE_LOG"))
            fprintf(stderr, "ml tune: l1 %.4g x %.4g  l2 (%d, %d)  p %d  model %.2f ms  measured %.2f ms\n",
                    c.l1x, c.l1y, c.sx, c.sy, c.P, cand_cost(c, c.P) * 1e-6, est);
        if (!found || est < best_est) {
            found = true;
            best_est = est;
            best.sx = c.sx; best.sy = c.sy; best.p = c.P; best.cost = cand_cost(c, c.P);
            best.l1x = c.l1x; best.l1y = c.l1y;
            best.span_far = far;
            best.use_span = span;
        }
    }
    g_err.clear();
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_measured[key] = best;
    return ML_OK;
}

// Lens arrays of a descriptor on the host.
ml_status load_lenses(const ml_field_desc &d, std::vector<double> &hx, std::vector<double> &hy,
                      std::vector<double> &hm)
{
    const int64_t n = d.n_lens;
    hx.resize(n); hy.resize(n); hm.resize(n);
    if (n == 0) return ML_OK;
    if (d.lens_mem_is_device) {
        ML_CK(cudaMemcpy(hx.data(), d.lens_x, n * sizeof(double), cudaMemcpyDeviceToHost));
        ML_CK(cudaMemcpy(hy.data(), d.lens_y, n * sizeof(double), cudaMemcpyDeviceToHost));
        ML_CK(cudaMemcpy(hm.data(), d.lens_m, n * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        memcpy(hx.data(), d.lens_x, n * sizeof(double));
        memcpy(hy.data(), d.lens_y, n * sizeof(double));
        memcpy(hm.data(), d.lens_m, n * sizeof(double));
    }
    return ML_OK;
}

// Plan: device check, lenses, (tuned) geometry, binning, near-list size and
// the truncation bound of every Taylor order; f->worst holds the bound.
ml_status create_plan(const ml_field_desc *d_in, cudaStream_t s, ml_field *f)
{
    ML_CK(cudaGetDevice(&f->device));
    // three attributes, not cudaGetDeviceProperties (which queries them all)
    int cc_major = 0, cc_minor = 0;
    ML_CK(cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, f->device));
    ML_CK(cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, f->device));
    ML_CK(cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, f->device));
    if (cc_major != 10 || cc_minor != 3)
        return fail(ML_ERR_CUDA, "this library is built for sm_103a (GB300); device is sm_" +
                                     std::to_string(cc_major) + std::to_string(cc_minor));
    f->desc = *d_in;
    ml_field_desc *d = &f->desc;

    const int64_t n = d->n_lens;
    f->n_lens = n;
    std::vector<double> hx(n), hy(n), hm(n);
    if (n > 0) {
        if (d->lens_mem_is_device) {
            ML_CK(cudaMemcpy(hx.data(), d->lens_x, n * sizeof(double), cudaMemcpyDeviceToHost));
            ML_CK(cudaMemcpy(hy.data(), d->lens_y, n * sizeof(double), cudaMemcpyDeviceToHost));
            ML_CK(cudaMemcpy(hm.data(), d->lens_m, n * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
            memcpy(hx.data(), d->lens_x, n * sizeof(double));
            memcpy(hy.data(), d->lens_y, n * sizeof(double));
            memcpy(hm.data(), d->lens_m, n * sizeof(double));
        }
        for (int64_t k = 0; k < n; ++k)
            if (!is_fin(hx[k]) || !is_fin(hy[k]) || !is_fin(hm[k]))
                return fail(ML_ERR_INVALID_ARG, "lens " + std::to_string(k) + " is not finite");
    }
    d->lens_x = d->lens_y = d->lens_m = nullptr;   // copied; the desc keeps only parameters
    ML_CK(f->alloc(&f->d_x, n, s));
    ML_CK(f->alloc(&f->d_y, n, s));
    ML_CK(f->alloc(&f->d_m, n, s));
    if (n > 0) {
        ML_CK(cudaMemcpyAsync(f->d_x, hx.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        ML_CK(cudaMemcpyAsync(f->d_y, hy.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        ML_CK(cudaMemcpyAsync(f->d_m, hm.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    if (d->tune && d->precision == ML_PREC_MIXED && d->l2_sub_x == 0 && d->l2_sub_y == 0) {
        GridChoice gc;
        ml_status st = tune_grid(*d, hx, hy, hm, f->d_x, f->d_y, f->d_m, s, true, gc);
        if (st != ML_OK) return st;
        d->l2_sub_x = gc.sx;
        d->l2_sub_y = gc.sy;
        d->l1_x = gc.l1x;
        d->l1_y = gc.l1y;
        if (d->span_far == 0.0) {
            f->span_far = gc.span_far;
            f->use_span = gc.use_span;
        }
        f->tuned = 1;
    }
    if (d->span_far > 0.0) f->span_far = (float)std::min(d->span_far, 3.0e38);
    ml_status st = derive_geometry(*d, hx, hy, f->g);
    if (st != ML_OK) return st;
    Geo &g = f->g;
    const bool nearfar = d->precision != ML_PREC_DIRECT64;
    if (nearfar && !rays_inside_sheet(g))
        return fail(ML_ERR_UNSUPPORTED, "near/far modes need the whole ray rectangle inside the "
                                        "sheet's disc; use ML_PREC_DIRECT64");
    if (d->precision == ML_PREC_MIXED &&
        (g.n2x >= (1 << 23) || g.n2y >= (1 << 22) || g.n1y > (int64_t)1 << 40))
        return fail(ML_ERR_UNSUPPORTED, "level-2 cells too large for FP32 offsets");
    if (g.NEx * g.NEy >= (int64_t)1 << 30)
        return fail(ML_ERR_UNSUPPORTED, "level-1 grid too large");
    f->max_launch_rays = d->max_launch_rays ? d->max_launch_rays : (1ull << 36);

    // lenses, binning (§3.2 Level 1)
    const int64_t NE = g.NEx * g.NEy;
    ML_CK(f->alloc(&f->d_cell, n, s));
    ML_CK(f->alloc(&f->d_count, NE + 1, s));
    ML_CK(f->alloc(&f->d_start, NE + 2, s));
    ML_CK(f->alloc(&f->d_sx, n, s));
    ML_CK(f->alloc(&f->d_sy, n, s));
    ML_CK(f->alloc(&f->d_sm, n, s));
    ML_CK(f->alloc(&f->d_scell, n, s));
    ML_CK(f->alloc(&f->d_perm, n, s));
    ML_CK(f->alloc(&f->d_f32, 5 * n, s));
    ML_CK(f->alloc(&f->d_stats, ML_STAT_COUNT, s));
    ML_CK(f->alloc(&f->d_sum, 1, s));
    ML_CK(f->alloc(&f->d_work, 1, s));
    ML_CK(f->alloc(&f->d_status, 1, s));
    ML_CK(flag_get(&f->h_abort, &f->d_abort));
    ML_CK(cudaMemsetAsync(f->d_count, 0, (NE + 1) * sizeof(int32_t), s));
    ML_CK(cudaMemsetAsync(f->d_stats, 0, ML_STAT_COUNT * sizeof(unsigned long long), s));
    ML_CK(cudaMemsetAsync(f->d_status, 0, sizeof(unsigned), s));
    ML_CK(launch_lens_cells(g, f->d_x, f->d_y, n, f->d_cell, f->d_count, s));
    ML_CK(launch_scan(f->d_count, f->d_start, NE + 1, s));
    ML_CK(launch_scatter(f->d_x, f->d_y, f->d_m, f->d_cell, n, f->d_start, NE + 1, f->d_sx,
                         f->d_sy, f->d_sm, f->d_scell, f->d_perm, f->d_f32, s));
    if (!nearfar) return ML_OK;

    // largest near list: the 3 x 3 block of each level-1 cell
    std::vector<int32_t> start(NE + 2);
    ML_CK(cudaMemcpyAsync(start.data(), f->d_start, (NE + 2) * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, s));
    ML_CK(cudaStreamSynchronize(s));
    int32_t mx = 0;
    for (int64_t cy = 0; cy < g.N1y; ++cy)
        for (int64_t cx = 0; cx < g.N1x; ++cx) {
            int32_t t = 0;
            for (int64_t ey = cy; ey <= cy + 2; ++ey) {
                int64_t b = ey * g.NEx + cx;
                t += start[b + 3] - start[b];
            }
            mx = std::max(mx, t);
        }
    f->max_near = mx;
    if (d->precision == ML_PREC_MIXED && (int64_t)mx * WARPS_PER_CTA * 24 > 200 * 1024)
        return fail(ML_ERR_UNSUPPORTED, "a level-1 cell has " + std::to_string(mx) +
                                            " near lenses; use a finer level-1 grid (l1_x, l1_y)");

    // truncation bound of every Taylor order, worst level-1 cell
    std::vector<double> bound((size_t)(g.N1x * g.N1y) * PMAX);
    double *d_bound = nullptr;
    ML_CK(ml_malloc_async((void **)&d_bound, bound.size() * sizeof(double), s));
    g.p = 1;
    cudaError_t e = launch_p_bound(g, f->table(), d_bound, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bound.data(), d_bound, bound.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_bound, s);
    if (e != cudaSuccess) return cuda_fail(e, "truncation bound");
    ML_CK(cudaStreamSynchronize(s));
    f->worst.assign(PMAX, 0.0);
    for (size_t c = 0; c < bound.size() / PMAX; ++c)
        for (int q = 0; q < PMAX; ++q) f->worst[q] = std::max(f->worst[q], bound[c * PMAX + q]);
    return ML_OK;
}

// The Taylor order the plan's bound asks for (far_tol), rounded up to a
// compiled order in the mixed mode.
int planned_order(const ml_field *f)
{
    const ml_field_desc *d = &f->desc;
    int p = d->taylor_p;
    if (p == 0) {
        double tol = d->far_tol > 0.0 ? d->far_tol : 1e-7;
        p = PMAX;
        for (int q = 1; q <= PMAX; ++q)
            if (f->worst[q - 1] <= tol) { p = q; break; }
    }
    // the fold's macro term is quadratic in theta_x: the row polynomials need degree 2
    if (d->macro_mode == ML_MACRO_FOLD && d->precision != ML_PREC_DIRECT64) p = std::max(p, 2);
    if (d->precision == ML_PREC_MIXED) p = mixed_p_supported(p);
    return p;
}

// Finish: far-field coefficients of order p at every level-2 node (§3.2
// Level 2), node records, zeroed map.
ml_status create_finish(ml_field *f, int p, cudaStream_t s, bool sync = true)
{
    const ml_field_desc *d = &f->desc;
    Geo &g = f->g;
    if (d->precision != ML_PREC_DIRECT64) {
        g.p = p;
        f->far_bound = f->worst[p - 1];
        const LensTable L = f->table();
        const int64_t nodes = g.N2x * g.N2y;
        ML_CK(f->alloc(&f->d_coef64, (size_t)nodes * (p + 1) * 2, s));
        f->build_used = ML_BUILD_DIRECT;
        bool done = false;
        if (d->build != ML_BUILD_DIRECT) {
            size_t ns = hier_scratch_doubles(g);
            if (ns > 0) {
                double *scratch = nullptr;
                ML_CK(ml_malloc_async((void **)&scratch, ns * sizeof(double), s));
                cudaError_t e = launch_coeffs_hier(g, L, f->d_coef64, scratch, ns, s);
                cudaFreeAsync(scratch, s);
                if (e != cudaSuccess) return cuda_fail(e, "hierarchical coefficient build");
                f->build_used = ML_BUILD_HIERARCHICAL;
                done = true;
            } else if (d->build == ML_BUILD_HIERARCHICAL) {
                return fail(ML_ERR_UNSUPPORTED, "hierarchical build not available");
            }
        }
        if (!done) ML_CK(launch_coeffs_direct(g, L, f->d_coef64, s));
        if (d->precision == ML_PREC_MIXED) {
            ML_CK(f->alloc(&f->d_nodes, (size_t)nodes * node_stride(p), s));
            ML_CK(launch_node_finalize(g, f->d_coef64, f->d_nodes, s));
        }
    } else {
        g.p = 0;
    }
    const size_t npix = (size_t)g.mnx * g.mny;
    if (d->deposit == ML_DEPOSIT_NGP) {
        ML_CK(f->alloc(&f->d_map_u32, npix, s));
        ML_CK(cudaMemsetAsync(f->d_map_u32, 0, npix * sizeof(uint32_t), s));
    } else {
        ML_CK(f->alloc(&f->d_map_f32, npix, s));
        ML_CK(cudaMemsetAsync(f->d_map_f32, 0, npix * sizeof(float), s));
    }
    if (sync) ML_CK(cudaStreamSynchronize(s));
    ML_CK(cudaGetLastError());
    return ML_OK;
}

ml_status create_impl(const ml_field_desc *d, cudaStream_t s, ml_field *f)
{
    ml_status st = create_plan(d, s, f);
    if (st != ML_OK) return st;
    return create_finish(f, d->precision == ML_PREC_DIRECT64 ? 0 : planned_order(f), s);
}

// Build a candidate grid's field and time it: the build (host clock, the
// stream synchronised on both sides) plus a centred slice of rays (CUDA
// events, after a short untimed range that loads the kernel), scaled to the
// whole lattice.  The lenses come from the tuner's host copies (the
// descriptor being built has handed its own pointers over already).
ml_status measure_grid(const ml_field_desc &d, const std::vector<double> &hx, const std::vector<double> &hy,
                       const std::vector<double> &hm, const TuneCand &c, cudaStream_t s, double &est_ms,
                       float &span_far, bool &use_span)
{
    ml_field_desc dc = d;
    dc.lens_x = hx.data();
    dc.lens_y = hy.data();
    dc.lens_m = hm.data();
    dc.n_lens = (int64_t)hx.size();
    dc.lens_mem_is_device = 0;
    dc.tune = 0;
    dc.l2_sub_x = c.sx;
    dc.l2_sub_y = c.sy;
    dc.l1_x = c.l1x;
    dc.l1_y = c.l1y;
    ml_field *f = new (std::nothrow) ml_field();
    if (!f) return fail(ML_ERR_OOM, "host allocation failed");
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    ml_status st = ML_OK;
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e2);
    if (ce != cudaSuccess) st = cuda_fail(ce, "grid autotuner");
    const auto t0 = std::chrono::steady_clock::now();
    if (st == ML_OK) st = create_impl(&dc, s, f);
    const double create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st == ML_OK) {
        // the time per ray is the slope between slices of n and 2n rays, which
        // cancels a launch's fixed start and tail
        const Geo &g = f->g;
        const uint64_t total = (uint64_t)g.n3x * (uint64_t)g.n3y;
        const uint64_t n = std::min<uint64_t>(total / 2, std::max<uint64_t>(500000000ull, total / 100));
        const uint64_t r0 = (total - 2 * n) / 2;
        const uint64_t warm = std::min<uint64_t>(n, 64ull * (uint64_t)g.n3x);
        // the certified walk is timed with lens columns spanned beyond five
        // distances about a factor two apart (lattice spacings: where spanning
        // pays depends on the lenses' pull in pixels per spacing, which differs
        // between fields), with them always walked ray by ray, and without
        // spans (the per-ray kernel); the fastest counts
        const bool certified = f->desc.walk == ML_WALK_CERTIFIED && f->g.deposit == ML_DEPOSIT_NGP;
        constexpr int NV = 7;
        const float fars[NV] = {ML_SPAN_FAR, 1500.f, 700.f, 300.f, 100.f, 3.0e38f, 3.0e38f};
        static const char *const names[NV] = {" (lens columns spanned beyond 3000)",
                                              " (lens columns spanned beyond 1500)",
                                              " (lens columns spanned beyond 700)",
                                              " (lens columns spanned beyond 300)",
                                              " (lens columns spanned beyond 100)",
                                              " (lens columns per ray)", " (no spans)"};
        double best_ray = -1.0;
        for (int v = 0; v < (certified ? NV : 1) && st == ML_OK; ++v) {
            f->span_far = fars[v];
            f->use_span = v < NV - 1;
            float ms[2] = {0.f, 0.f};
            st = ml_shoot_rays(f, r0, r0 + warm, s);
            for (int q = 0; q < 2 && st == ML_OK && n > 0; ++q) {
                ce = cudaEventRecord(e1, s);
                if (ce == cudaSuccess) st = ml_shoot_rays(f, r0, r0 + (q + 1) * n, s);
                if (st == ML_OK && ce == cudaSuccess) ce = cudaEventRecord(e2, s);
                if (st == ML_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e2);
                if (st == ML_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms[q], e1, e2);
                if (st == ML_OK && ce != cudaSuccess) st = cuda_fail(ce, "grid autotuner");
            }
            const double per_ray = n > 0 ? std::max(0.0, (double)(ms[1] - ms[0])) / (double)n : 0.0;
            if (st == ML_OK && (best_ray < 0.0 || per_ray < best_ray)) {
                best_ray = per_ray;
                span_far = fars[v];
                use_span = v < NV - 1;
            }
            if (st == ML_OK && getenv("ML_TUNE_LOG"))
                fprintf(stderr, "ml tune:   create %.2f ms, %.3g and %.3g of %.3g rays in %.3f and %.3f ms%s\n",
                        create_ms, (double)n, (double)(2 * n), (double)total, ms[0], ms[1],
                        certified ? names[v] : "");
        }
        if (st == ML_OK) est_ms = create_ms + best_ray * (double)total;
    }
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    f->release();
    delete f;
    return st;
}

ShootArgs make_args(const ml_field *f)
{
    ShootArgs a;
    memset(&a, 0, sizeof(a));
    a.g = f->g;
    a.L = f->table();
    a.coef64 = f->d_coef64;
    a.nodes = f->d_nodes;
    a.map_u32 = f->d_map_u32;
    a.map_f32 = f->d_map_f32;
    a.stats = f->d_stats;
    a.status = f->d_status;
    a.work = f->d_work;
    a.abort_flag = f->d_abort;
    const Geo &g = f->g;
    a.near_cap = std::max(1, f->max_near);
    a.walk = f->desc.walk == ML_WALK_CERTIFIED && f->use_span ? ML_WALK_CERTIFIED : ML_WALK_PER_RAY;
    a.span_far = f->span_far;
    a.l3x_f = (float)g.l3x;
    a.l3x_lo = (float)(g.l3x - (double)a.l3x_f);
    a.c0_f = (float)(0.5 - 0.5 * (double)g.n2x);
    // close-pass radius: FP32 offsets of size up to |t| + |dyl| give a relative
    // near-term error of 2 * 2^-24 (|t| + |dyl|) / r; below r_c it could pass
    // 5e-7, so those rays take the hi/lo path
    // (the same radius in lattice units for the counting kernels' sums)
    {
        double rc = 4.0 * 5.9604644775390625e-8 * (0.5 * g.l2x + 32.0 * g.l3y) / 5e-7;
        a.rc2 = (float)(rc * rc);
        a.rc2u = (float)((rc / g.l3x) * (rc / g.l3x));
    }
    a.ipx_f = (float)(1.0 / g.dpx);
    a.ipy_f = (float)(1.0 / g.dpy);
    a.l3yx = g.l3y / g.l3x;
    a.l3yx_f = (float)a.l3yx;
    a.il3x = 1.0 / g.l3x;
    a.mpx = 1.0 / (g.l3x * g.dpx);
    a.yx_f = (float)(g.dpx / g.dpy);
    const bool fold = g.macro == ML_MACRO_FOLD;
    // macro terms of the row polynomial per power of u (theta_x offset u l3x)
    a.cxy_f = fold ? (float)(g.dy * g.l3y * g.l3x / g.dpx) : 0.f;
    a.q2_f = fold ? (float)(0.5 * g.dx * g.l3x * g.l3x / g.dpx) : 0.f;
    a.rho_y = ((fold ? 2.0 * (1.0 - g.kappa0) : 1.0 - g.kappa + g.gamma) + sheet_ky(g)) * g.l3y / g.dpy;
    return a;
}

// Task decomposition of rays [b, e) for the mixed kernel.
void set_tasks(ShootArgs &a, const Geo &g, int64_t b, int64_t e)
{
    a.ray_begin = b;
    a.ray_end = e;
    const int64_t gpb = (g.n1y + 31) / 32;
    const int64_t l2_per_cc = std::max<int64_t>(1, std::min<int64_t>(g.l2sx, (2048 + g.n2x - 1) / g.n2x));
    const int64_t cc_per_l1 = (g.l2sx + l2_per_cc - 1) / l2_per_cc;
    const int64_t jb = b / g.n3x, je = (e - 1) / g.n3x;
    auto rg = [&](int64_t j) { return (j / g.n1y) * gpb + (j % g.n1y) / 32; };
    a.groups_per_band = gpb;
    a.rg_first = rg(jb);
    a.n_rg = rg(je) - a.rg_first + 1;
    a.l2_per_cc = l2_per_cc;
    a.cc_per_l1 = cc_per_l1;
    a.n_cc = g.N1x * cc_per_l1;
    a.n_tasks = a.n_rg * a.n_cc;
}

}  // namespace

// Many maps run as one: fields, their kernel arguments on the device, the
// task prefix sums, and the buffers of the step's outputs.
struct ml_batch {
    // maps that share a Taylor order run in one persistent launch
    struct Group {
        int p = 0, near_cap = 1;
        std::vector<int> maps;
        ShootArgs *d_args = nullptr;
        int64_t *d_base = nullptr;
        unsigned long long *d_work = nullptr;
        int64_t total_tasks = 0;
    };
    int device = 0, num_sms = 0;
    std::vector<Group> groups;
    std::vector<ml_field *> fields;
    std::vector<size_t> mu_off;
    unsigned int *d_status = nullptr;
    int *h_abort = nullptr, *d_abort = nullptr;
    float *d_mu = nullptr;
    int tpm = 0, n_samples = 0, taps_h = 0;
    double *d_tracks = nullptr;
    float *d_taps = nullptr, *d_curves = nullptr;
    cudaStream_t s_int = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // one branch per Taylor order: the groups' persistent launches run on
    // streams of their own (parallel branches of the graph), so that one
    // group's blocks fill the SMs another group's tail leaves idle
    std::vector<cudaStream_t> s_grp;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> owned;

    template <class T>
    cudaError_t alloc(T **ptr, size_t count, cudaStream_t s)
    {
        *ptr = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = ml_malloc_async((void **)ptr, count * sizeof(T), s);
        if (e == cudaSuccess) owned.push_back(*ptr);
        return e;
    }
    void release()
    {
        cudaDeviceSynchronize();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (s_int) cudaStreamDestroy(s_int);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (cudaEvent_t ev : ev_join) cudaEventDestroy(ev);
        for (cudaStream_t st : s_grp) cudaStreamDestroy(st);
        ev_join.clear();
        s_grp.clear();
        exec = nullptr; graph = nullptr; ev_in = ev_out = ev_fork = nullptr; s_int = nullptr;
        for (void *q : owned) cudaFree(q);
        owned.clear();
        flag_put(h_abort);
        h_abort = nullptr;
        for (ml_field *f : fields) {
            if (!f) continue;
            f->release();
            delete f;
        }
        fields.clear();
    }
};

namespace {

// The whole batch step on stream s (recorded into a graph when capturing).
cudaError_t batch_enqueue(ml_batch *b, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (ml_field *f : b->fields) {
        const size_t npix = (size_t)f->g.mnx * f->g.mny;
        if ((e = cudaMemsetAsync(f->d_map_u32, 0, npix * sizeof(uint32_t), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(f->d_stats, 0, ML_STAT_COUNT * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(f->d_status, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    for (const ml_batch::Group &gr : b->groups)
        if ((e = cudaMemsetAsync(gr.d_work, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->ev_fork, s)) != cudaSuccess) return e;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const ml_batch::Group &gr = b->groups[gi];
        cudaStream_t sg = b->s_grp[gi];
        if ((e = cudaStreamWaitEvent(sg, b->ev_fork, 0)) != cudaSuccess) return e;
        BatchArgs ba;
        ba.args = gr.d_args;
        ba.task_base = gr.d_base;
        ba.n_maps = (int)gr.maps.size();
        ba.near_cap = gr.near_cap;
        ba.walk = b->fields.empty() ? ML_WALK_CERTIFIED : b->fields[0]->desc.walk;
        ba.total_tasks = gr.total_tasks;
        ba.work = gr.d_work;
        ba.abort_flag = b->d_abort;
        ba.status = b->d_status;
        if ((e = launch_batch(ba, gr.p, b->num_sms, sg)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(b->ev_join[gi], sg)) != cudaSuccess) return e;
    }
    for (cudaEvent_t ev : b->ev_join)
        if ((e = cudaStreamWaitEvent(s, ev, 0)) != cudaSuccess) return e;
    for (size_t i = 0; i < b->fields.size(); ++i) {
        const ml_field *f = b->fields[i];
        const Geo &g = f->g;
        const double scale = (g.l3x * g.l3y) / (g.dpx * g.dpy);
        if ((e = launch_mu(g, f->d_map_u32, nullptr, ML_MAP_MU_F32, b->d_mu + b->mu_off[i], scale, s)) !=
            cudaSuccess)
            return e;
        if (b->tpm > 0) {
            e = launch_light_curves_dev(g, f->d_map_u32, nullptr, scale, b->d_tracks + 4 * i * b->tpm,
                                        b->tpm, b->n_samples, b->taps_h, b->d_taps,
                                        b->d_curves + i * (size_t)b->tpm * b->n_samples, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

ml_status batch_create_impl(const ml_field_desc *descs, int32_t n, int32_t tpm, const double *tracks,
                            int32_t n_samples, double sigma_px, cudaStream_t s, ml_batch *b)
{
    ML_CK(cudaGetDevice(&b->device));
    for (int32_t i = 0; i < n; ++i) {
        ml_status st = validate(&descs[i]);
        if (st != ML_OK) return fail(st, "map " + std::to_string(i) + ": " + g_err);
        if (descs[i].precision != ML_PREC_MIXED || descs[i].deposit != ML_DEPOSIT_NGP)
            return fail(ML_ERR_UNSUPPORTED, "batches take ML_PREC_MIXED with ML_DEPOSIT_NGP");
        if (descs[i].walk != descs[0].walk)
            return fail(ML_ERR_INVALID_ARG, "every map of a batch takes the same walk");
    }
    // Tuned maps take the grid the cost model ranks first for them, each
    // with its own Taylor order; maps of one order share a persistent launch.
    std::vector<ml_field_desc> plan(descs, descs + n);
    std::vector<char> tuned(n, 0);
    for (int32_t i = 0; i < n; ++i) {
        if (!(plan[i].tune && plan[i].l2_sub_x == 0 && plan[i].l2_sub_y == 0)) continue;
        std::vector<double> hx, hy, hm;
        ml_status st = load_lenses(plan[i], hx, hy, hm);
        if (st != ML_OK) return st;
        const size_t nl = std::max<size_t>(hx.size(), 1);
        double *dx = nullptr, *dy = nullptr, *dm = nullptr;
        ML_CK(ml_malloc_async((void **)&dx, nl * sizeof(double), s));
        ML_CK(ml_malloc_async((void **)&dy, nl * sizeof(double), s));
        ML_CK(ml_malloc_async((void **)&dm, nl * sizeof(double), s));
        cudaError_t e = cudaSuccess;
        if (!hx.empty()) {
            e = cudaMemcpyAsync(dx, hx.data(), hx.size() * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dy, hy.data(), hy.size() * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dm, hm.data(), hm.size() * sizeof(double), cudaMemcpyHostToDevice, s);
        }
        GridChoice best;
        // the batch's grids come from the cost model alone (timing every map
        // would cost more than it saves); the per-ray model ranks them: on
        // the lens-dense maps of a batch the certified walk runs mostly per
        // ray, and the certified model (fitted on a sparse field) misranks
        ml_field_desc model = plan[i];
        model.walk = ML_WALK_PER_RAY;
        if (e == cudaSuccess) st = tune_grid(model, hx, hy, hm, dx, dy, dm, s, false, best);
        cudaFreeAsync(dx, s);
        cudaFreeAsync(dy, s);
        cudaFreeAsync(dm, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch tuner");
        if (st != ML_OK) return st;
        if (best.p > 0) {
            plan[i].l2_sub_x = best.sx;
            plan[i].l2_sub_y = best.sy;
            plan[i].l1_x = best.l1x;
            plan[i].l1_y = best.l1y;
            tuned[i] = 1;
        }
    }
    b->fields.assign(n, nullptr);
    for (int32_t i = 0; i < n; ++i) {
        b->fields[i] = new (std::nothrow) ml_field();
        if (!b->fields[i]) return fail(ML_ERR_OOM, "host allocation failed");
        ml_status st = create_plan(&plan[i], s, b->fields[i]);
        if (st != ML_OK) return fail(st, "map " + std::to_string(i) + ": " + g_err);
        b->fields[i]->tuned = tuned[i];
        // not timed per map: the batches measured (lens-dense fields) run
        // faster with lens columns walked ray by ray
        if (plan[i].span_far == 0.0) b->fields[i]->span_far = 3.0e38f;
    }
    // coefficient builds of different maps overlap on a few streams
    {
        constexpr int kBuildStreams = 8;
        cudaStream_t bs[kBuildStreams] = {};
        cudaEvent_t ready = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, s);
        for (int q = 0; q < kBuildStreams && e == cudaSuccess; ++q) {
            e = cudaStreamCreateWithFlags(&bs[q], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(bs[q], ready, 0);
        }
        ml_status st = ML_OK;
        for (int32_t i = 0; i < n && e == cudaSuccess && st == ML_OK; ++i) {
            st = create_finish(b->fields[i], planned_order(b->fields[i]), bs[i % kBuildStreams], false);
            if (st != ML_OK) st = fail(st, "map " + std::to_string(i) + ": " + g_err);
        }
        for (int q = 0; q < kBuildStreams; ++q) {
            if (!bs[q]) continue;
            cudaError_t e2 = cudaStreamSynchronize(bs[q]);
            if (e == cudaSuccess) e = e2;
            cudaStreamDestroy(bs[q]);
        }
        if (ready) cudaEventDestroy(ready);
        if (st != ML_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "batch build");
    }
    b->num_sms = b->fields[0]->num_sms;
    size_t mu_total = 0;
    for (int32_t i = 0; i < n; ++i) {
        b->mu_off.push_back(mu_total);
        mu_total += (size_t)b->fields[i]->g.mnx * b->fields[i]->g.mny;
    }
    for (int32_t i = 0; i < n; ++i) {
        const int P = b->fields[i]->g.p;
        auto it = std::find_if(b->groups.begin(), b->groups.end(),
                               [P](const ml_batch::Group &gr) { return gr.p == P; });
        if (it == b->groups.end()) {
            b->groups.emplace_back();
            b->groups.back().p = P;
            it = b->groups.end() - 1;
        }
        it->maps.push_back(i);
    }
    for (ml_batch::Group &gr : b->groups) {
        const size_t m = gr.maps.size();
        std::vector<ShootArgs> args(m);
        std::vector<int64_t> base(m + 1, 0);
        for (size_t q = 0; q < m; ++q) {
            ml_field *f = b->fields[gr.maps[q]];
            args[q] = make_args(f);
            set_tasks(args[q], f->g, 0, f->g.n3x * f->g.n3y);
            gr.near_cap = std::max(gr.near_cap, args[q].near_cap);
            base[q + 1] = base[q] + args[q].n_tasks;
        }
        gr.total_tasks = base[m];
        ML_CK(b->alloc(&gr.d_args, m, s));
        ML_CK(b->alloc(&gr.d_base, m + 1, s));
        ML_CK(b->alloc(&gr.d_work, 1, s));
        ML_CK(cudaMemcpyAsync(gr.d_args, args.data(), sizeof(ShootArgs) * m, cudaMemcpyHostToDevice, s));
        ML_CK(cudaMemcpyAsync(gr.d_base, base.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, s));
        // the host copies must outlive the asynchronous transfers
        ML_CK(cudaStreamSynchronize(s));
    }
    ML_CK(b->alloc(&b->d_status, 1, s));
    ML_CK(b->alloc(&b->d_mu, mu_total, s));
    ML_CK(flag_get(&b->h_abort, &b->d_abort));
    if (tpm > 0) {
        float taps[129];
        b->taps_h = light_curve_taps(sigma_px, taps);
        b->tpm = tpm;
        b->n_samples = n_samples;
        ML_CK(b->alloc(&b->d_taps, 2 * b->taps_h + 1, s));
        ML_CK(b->alloc(&b->d_tracks, (size_t)4 * n * tpm, s));
        ML_CK(b->alloc(&b->d_curves, (size_t)n * tpm * n_samples, s));
        ML_CK(cudaMemcpyAsync(b->d_taps, taps, sizeof(float) * (2 * b->taps_h + 1),
                              cudaMemcpyHostToDevice, s));
        ML_CK(cudaMemcpyAsync(b->d_tracks, tracks, sizeof(double) * 4 * (size_t)n * tpm,
                              cudaMemcpyHostToDevice, s));
    }
    ML_CK(cudaStreamCreateWithFlags(&b->s_int, cudaStreamNonBlocking));
    ML_CK(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    ML_CK(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    ML_CK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        cudaStream_t sg = nullptr;
        cudaEvent_t ev = nullptr;
        ML_CK(cudaStreamCreateWithFlags(&sg, cudaStreamNonBlocking));
        b->s_grp.push_back(sg);
        ML_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->ev_join.push_back(ev);
    }
    ML_CK(cudaStreamSynchronize(s));
    return ML_OK;
}

}  // namespace

namespace ml {
cudaError_t ml_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[MAXDEV] = {};
    if (dev < 0 || dev >= MAXDEV) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            e = cudaMemPoolCreate(&np, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;   // never trim at synchronisation
            e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(np);
                return e;
            }
            pools[dev] = np;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// peak statistics kernels (ml_maps.cu): out holds n_peaks, sum_counts and
// n_positions, nbins 64-bit counters each
cudaError_t launch_peak_stats(const uint32_t *N, int nx, int ny, int along, const uint8_t *mask,
                              double origin, double step, double caustic, const double *edges,
                              int nbins, int32_t *bin_of, unsigned long long *out, int num_sms,
                              cudaStream_t s);
}  // namespace ml

extern "C" {

ml_status ml_batch_create(const ml_field_desc *descs, int32_t n, int32_t tracks_per_map,
                          const double *tracks, int32_t n_samples, double sigma_px, void *stream,
                          ml_batch **out)
{
    if (!out) return fail(ML_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1) return fail(ML_ERR_INVALID_ARG, "need n >= 1 descriptors");
    if (tracks_per_map < 0 || (tracks_per_map > 0 && (!tracks || n_samples < 1 ||
                                                      !(sigma_px > 0.0) || sigma_px > 16.0)))
        return fail(ML_ERR_INVALID_ARG, "bad light-curve arguments");
    ml_batch *b = new (std::nothrow) ml_batch();
    if (!b) return fail(ML_ERR_OOM, "host allocation failed");
    ml_status st = batch_create_impl(descs, n, tracks_per_map, tracks, n_samples, sigma_px,
                                     (cudaStream_t)stream, b);
    if (st != ML_OK) {
        std::string keep = g_err;
        b->release();
        delete b;
        cudaGetLastError();
        g_err = keep;
        return st;
    }
    *out = b;
    return ML_OK;
}

ml_status ml_batch_run(ml_batch *b, int32_t use_graph, void *stream)
{
    if (!b) return fail(ML_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    ML_CK(cudaEventRecord(b->ev_in, s));
    ML_CK(cudaStreamWaitEvent(b->s_int, b->ev_in, 0));
    if (use_graph) {
        if (!b->exec) {
            ML_CK(cudaStreamBeginCapture(b->s_int, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = batch_enqueue(b, b->s_int);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->s_int, &graph);
            if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "batch capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "batch capture");
            b->graph = graph;
            ML_CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
        ML_CK(cudaGraphLaunch(b->exec, b->s_int));
    } else {
        ML_CK(batch_enqueue(b, b->s_int));
    }
    ML_CK(cudaEventRecord(b->ev_out, b->s_int));
    ML_CK(cudaStreamWaitEvent(s, b->ev_out, 0));
    for (ml_field *f : b->fields) {
        f->launches = 1;
        f->rays_asked = (uint64_t)f->g.n3x * (uint64_t)f->g.n3y;
        f->map_base = 0;
        f->in_at_set = 0;
    }
    return ML_OK;
}

ml_status ml_batch_field(ml_batch *b, int32_t i, ml_field **out)
{
    if (!b || !out || i < 0 || i >= (int32_t)b->fields.size())
        return fail(ML_ERR_INVALID_ARG, "bad batch index");
    *out = b->fields[i];
    return ML_OK;
}

ml_status ml_batch_mu(ml_batch *b, int32_t i, float *out, int32_t out_is_device, void *stream)
{
    if (!b || !out || i < 0 || i >= (int32_t)b->fields.size())
        return fail(ML_ERR_INVALID_ARG, "bad batch index");
    cudaStream_t s = (cudaStream_t)stream;
    const ml_field *f = b->fields[i];
    const size_t npix = (size_t)f->g.mnx * f->g.mny;
    ML_CK(cudaMemcpyAsync(out, b->d_mu + b->mu_off[i], npix * sizeof(float),
                          out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_is_device) ML_CK(cudaStreamSynchronize(s));
    return ML_OK;
}

ml_status ml_batch_curves(ml_batch *b, float *out, int32_t out_is_device, void *stream)
{
    if (!b || !out) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (b->tpm == 0) return fail(ML_ERR_STATE, "the batch has no tracks");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cnt = b->fields.size() * (size_t)b->tpm * b->n_samples;
    ML_CK(cudaMemcpyAsync(out, b->d_curves, cnt * sizeof(float),
                          out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_is_device) ML_CK(cudaStreamSynchronize(s));
    return ML_OK;
}

ml_status ml_batch_abort(ml_batch *b, int32_t on)
{
    if (!b) return fail(ML_ERR_INVALID_ARG, "batch is NULL");
    *(volatile int *)b->h_abort = on ? 1 : 0;
    return ML_OK;
}

ml_status ml_batch_destroy(ml_batch *b)
{
    if (!b) return ML_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    b->release();
    cudaSetDevice(cur);
    delete b;
    return ML_OK;
}

int32_t ml_abi_version(void) { return ML_ABI_VERSION; }

const char *ml_last_error(void) { return g_err.c_str(); }

ml_status ml_field_create(const ml_field_desc *desc, void *stream, ml_field **out)
{
    if (!out) return fail(ML_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ml_status st = validate(desc);
    if (st != ML_OK) return st;
    ml_field *f = new (std::nothrow) ml_field();
    if (!f) return fail(ML_ERR_OOM, "host allocation failed");
    st = create_impl(desc, (cudaStream_t)stream, f);
    if (st != ML_OK) {
        std::string keep = g_err;
        f->release();
        delete f;
        cudaGetLastError();
        g_err = keep;
        return st;
    }
    g_err.clear();
    *out = f;
    return ML_OK;
}

ml_status ml_shoot_rays(ml_field *f, uint64_t ray_begin, uint64_t ray_end, void *stream)
{
    if (!f) return fail(ML_ERR_INVALID_ARG, "field is NULL");
    const Geo &g = f->g;
    const uint64_t total = (uint64_t)g.n3x * (uint64_t)g.n3y;
    if (ray_begin > ray_end || ray_end > total)
        return fail(ML_ERR_INVALID_ARG, "ray range outside the lattice [0, " +
                                            std::to_string(total) + ")");
    cudaStream_t s = (cudaStream_t)stream;
    ShootArgs a = make_args(f);
    for (uint64_t b = ray_begin; b < ray_end;) {
        uint64_t e = std::min<uint64_t>(ray_end, b + f->max_launch_rays);
        a.ray_begin = (int64_t)b;
        a.ray_end = (int64_t)e;
        if (g.precision == ML_PREC_MIXED) {
            set_tasks(a, g, (int64_t)b, (int64_t)e);
            ML_CK(cudaMemsetAsync(f->d_work, 0, sizeof(unsigned long long), s));
        }
        ML_CK(launch_shoot(a, f->num_sms, s));
        ++f->launches;
        b = e;
    }
    f->rays_asked += ray_end - ray_begin;
    return ML_OK;
}

ml_status ml_trace_rays(ml_field *f, const int64_t *ray_idx, int64_t n, double *beta, int32_t *pix,
                        void *stream)
{
    if (!f) return fail(ML_ERR_INVALID_ARG, "field is NULL");
    if (n < 0 || (n > 0 && (!ray_idx || !beta || !pix)))
        return fail(ML_ERR_INVALID_ARG, "bad trace arguments");
    ShootArgs a = make_args(f);
    ML_CK(launch_trace(a, ray_idx, n, beta, pix, (cudaStream_t)stream));
    return ML_OK;
}

ml_status ml_magnification_map(ml_field *f, int32_t want, void *out, int32_t out_is_device,
                               void *stream)
{
    if (!f || !out) return fail(ML_ERR_INVALID_ARG, "field or out is NULL");
    if (want < ML_MAP_COUNTS_U32 || want > ML_MAP_MU_F64)
        return fail(ML_ERR_INVALID_ARG, "unknown map kind");
    const Geo &g = f->g;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)g.mnx * g.mny;
    const double scale = (g.l3x * g.l3y) / (g.dpx * g.dpy);   // S_I / S_S, Eq. 12
    if (want == ML_MAP_COUNTS_U32) {
        if (!f->d_map_u32) return fail(ML_ERR_STATE, "a CIC field has no integer counts");
        ML_CK(cudaMemcpyAsync(out, f->d_map_u32, npix * sizeof(uint32_t),
                              out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        if (!out_is_device) ML_CK(cudaStreamSynchronize(s));
        return ML_OK;
    }
    const size_t esz = want == ML_MAP_MU_F32 ? 4 : 8;
    void *dst = out;
    bool staged = false;             // through a device buffer and a copy
    if (!out_is_device) {
        // page-locked host memory the GPU addresses (pinned and mapped, as
        // cudaHostAlloc gives under unified addressing): the kernel writes the
        // map straight into it over the host link, with no device buffer and
        // no separate transfer; other host memory goes through a copy
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer != nullptr && (uintptr_t)pa.devicePointer % 16 == 0) {
            dst = pa.devicePointer;
        } else {
            cudaGetLastError();
            ML_CK(ml_malloc_async(&dst, npix * esz, s));
            staged = true;
        }
    } else if ((uintptr_t)out % 16 != 0) {
        return fail(ML_ERR_INVALID_ARG, "device output must be 16-byte aligned");
    }
    cudaError_t e = launch_mu(g, f->d_map_u32, f->d_map_f32, want, dst, scale, s);
    if (e == cudaSuccess && staged)
        e = cudaMemcpyAsync(out, dst, npix * esz, cudaMemcpyDeviceToHost, s);
    if (staged) cudaFreeAsync(dst, s);
    if (!out_is_device && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "magnification map");
    return ML_OK;
}

ml_status ml_light_curves(ml_field *f, const double *tracks, int32_t n_tracks, int32_t n_samples,
                          double sigma_px, float *out, int32_t out_is_device, void *stream)
{
    if (!f || !tracks || !out) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (n_tracks < 1 || n_samples < 1) return fail(ML_ERR_INVALID_ARG, "need >= 1 track and sample");
    if (!(sigma_px > 0.0) || sigma_px > 16.0) return fail(ML_ERR_INVALID_ARG, "sigma_px must be in (0, 16]");
    for (int q = 0; q < 4 * n_tracks; ++q)
        if (!is_fin(tracks[q])) return fail(ML_ERR_INVALID_ARG, "track coordinates must be finite");
    const Geo &g = f->g;
    cudaStream_t s = (cudaStream_t)stream;
    const double scale = (g.l3x * g.l3y) / (g.dpx * g.dpy);
    const size_t nout = (size_t)n_tracks * n_samples;
    double *d_tr = nullptr;
    float *dst = out;
    ML_CK(ml_malloc_async((void **)&d_tr, sizeof(double) * 4 * n_tracks, s));
    cudaError_t e = cudaMemcpyAsync(d_tr, tracks, sizeof(double) * 4 * n_tracks,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !out_is_device) e = ml_malloc_async((void **)&dst, nout * sizeof(float), s);
    if (e == cudaSuccess)
        e = launch_light_curves(g, f->d_map_u32, f->d_map_f32, scale, d_tr, n_tracks, n_samples,
                                sigma_px, dst, s);
    if (e == cudaSuccess && !out_is_device)
        e = cudaMemcpyAsync(out, dst, nout * sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_tr, s);
    if (!out_is_device && dst != out) cudaFreeAsync(dst, s);
    if (e == cudaSuccess && !out_is_device) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "light curves");
    return ML_OK;
}

namespace {

ml_status map_lc_args(const void *a, const void *b, const double *tracks, int32_t nx, int32_t ny,
                      int32_t n_tracks, int32_t n_samples, double sigma_px)
{
    if (!a || !b || !tracks) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (nx < 1 || ny < 1) return fail(ML_ERR_INVALID_ARG, "map size must be positive");
    if (n_tracks < 1 || n_samples < 1) return fail(ML_ERR_INVALID_ARG, "need >= 1 track and sample");
    if (!(sigma_px > 0.0) || sigma_px > 16.0) return fail(ML_ERR_INVALID_ARG, "sigma_px must be in (0, 16]");
    for (int q = 0; q < 4 * n_tracks; ++q)
        if (!is_fin(tracks[q])) return fail(ML_ERR_INVALID_ARG, "track coordinates must be finite");
    return ML_OK;
}

}  // namespace

ml_status ml_map_light_curves(const float *mu, int32_t nx, int32_t ny, const double *tracks,
                              int32_t n_tracks, int32_t n_samples, double sigma_px, float *out,
                              void *stream)
{
    ml_status st = map_lc_args(mu, out, tracks, nx, ny, n_tracks, n_samples, sigma_px);
    if (st != ML_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Geo g{};
    g.mnx = nx;
    g.mny = ny;
    double *d_tr = nullptr;
    ML_CK(ml_malloc_async((void **)&d_tr, sizeof(double) * 4 * n_tracks, s));
    cudaError_t e = cudaMemcpyAsync(d_tr, tracks, sizeof(double) * 4 * n_tracks, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_light_curves(g, nullptr, mu, 1.0, d_tr, n_tracks, n_samples, sigma_px, out, s);
    cudaFreeAsync(d_tr, s);
    if (e != cudaSuccess) return cuda_fail(e, "map light curves");
    return ML_OK;
}

ml_status ml_map_light_curves_backward(int32_t nx, int32_t ny, const double *tracks, int32_t n_tracks,
                                       int32_t n_samples, double sigma_px, const float *dL_dcurves,
                                       float *dL_dmu, void *stream)
{
    ml_status st = map_lc_args(dL_dcurves, dL_dmu, tracks, nx, ny, n_tracks, n_samples, sigma_px);
    if (st != ML_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *d_tr = nullptr;
    ML_CK(cudaMemsetAsync(dL_dmu, 0, sizeof(float) * (size_t)nx * (size_t)ny, s));
    ML_CK(ml_malloc_async((void **)&d_tr, sizeof(double) * 4 * n_tracks, s));
    cudaError_t e = cudaMemcpyAsync(d_tr, tracks, sizeof(double) * 4 * n_tracks, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_light_curves_adj(nx, ny, d_tr, n_tracks, n_samples, sigma_px, dL_dcurves, dL_dmu, s);
    cudaFreeAsync(d_tr, s);
    if (e != cudaSuccess) return cuda_fail(e, "light-curve adjoint");
    return ML_OK;
}

ml_status ml_light_curves_noalloc(ml_field *f, const double *tracks, int32_t n_tracks,
                                  int32_t n_samples, double sigma_px, float *out, void *stream)
{
    if (!f || !tracks || !out) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (n_tracks < 1 || n_samples < 1) return fail(ML_ERR_INVALID_ARG, "need >= 1 track and sample");
    if (n_tracks > ML_NOALLOC_MAX_TRACKS)
        return fail(ML_ERR_INVALID_ARG, "n_tracks " + std::to_string(n_tracks) +
                                            " exceeds ML_NOALLOC_MAX_TRACKS (" +
                                            std::to_string(ML_NOALLOC_MAX_TRACKS) + ")");
    if (!(sigma_px > 0.0) || sigma_px > 16.0) return fail(ML_ERR_INVALID_ARG, "sigma_px must be in (0, 16]");
    for (int q = 0; q < 4 * n_tracks; ++q)
        if (!is_fin(tracks[q])) return fail(ML_ERR_INVALID_ARG, "track coordinates must be finite");
    const Geo &g = f->g;
    const double scale = (g.l3x * g.l3y) / (g.dpx * g.dpy);
    ML_CK(launch_light_curves_noalloc(g, f->d_map_u32, f->d_map_f32, scale, tracks, n_tracks,
                                      n_samples, sigma_px, out, (cudaStream_t)stream));
    return ML_OK;
}

ml_status ml_cic_forward(ml_field *f, float *mu, void *stream)
{
    if (!f || !mu) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (f->g.deposit != ML_DEPOSIT_CIC || f->g.precision != ML_PREC_MIXED)
        return fail(ML_ERR_STATE, "the differentiable map needs ML_DEPOSIT_CIC and ML_PREC_MIXED");
    ml_status st = ml_field_clear(f, stream);
    if (st != ML_OK) return st;
    st = ml_shoot_rays(f, 0, (uint64_t)f->g.n3x * (uint64_t)f->g.n3y, stream);
    if (st != ML_OK) return st;
    return ml_magnification_map(f, ML_MAP_MU_F32, mu, 1, stream);
}

ml_status ml_cic_backward_ex(ml_field *f, const float *dL_dM, double *grad_lens, double *grad_params,
                             int32_t method, void *stream)
{
    if (!f || !dL_dM || !grad_lens || !grad_params) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (method != ML_ADJOINT_NEARFAR && method != ML_ADJOINT_DIRECT)
        return fail(ML_ERR_INVALID_ARG, "unknown adjoint method");
    if (f->g.deposit != ML_DEPOSIT_CIC || f->g.precision != ML_PREC_MIXED)
        return fail(ML_ERR_STATE, "the adjoint needs a field with ML_DEPOSIT_CIC and ML_PREC_MIXED");
    if (f->g.macro != ML_MACRO_LINEAR || f->g.sheet_shape != ML_SHEET_DISC)
        return fail(ML_ERR_UNSUPPORTED, "the adjoint's parameter terms are those of the "
                                        "constant-(kappa, gamma) macro model with a disc sheet");
    cudaStream_t s = (cudaStream_t)stream;
    const Geo &g = f->g;
    const int64_t n = std::max<int64_t>(f->n_lens, 0);
    ShootArgs a = make_args(f);
    const double scale = (g.l3x * g.l3y) / (g.dpx * g.dpy);
    ML_CK(cudaMemsetAsync(grad_lens, 0, sizeof(double) * 3 * (size_t)n, s));
    ML_CK(cudaMemsetAsync(grad_params, 0, sizeof(double) * 3, s));
    if (method == ML_ADJOINT_DIRECT) {
        a.ray_begin = 0;
        a.ray_end = g.n3x * g.n3y;
        ML_CK(launch_cic_adjoint_direct(a, dL_dM, f->d_x, f->d_y, f->d_m, f->n_lens, grad_lens,
                                        grad_params, scale, f->num_sms, s));
        return ML_OK;
    }
    set_tasks(a, g, 0, g.n3x * g.n3y);
    const size_t n_mom = (size_t)(g.N2x * g.N2y) * (size_t)(g.p + 1);
    double *gs = nullptr;
    double2 *mom = nullptr;
    cudaError_t e = ml_malloc_async((void **)&gs, sizeof(double) * 3 * (size_t)std::max<int64_t>(n, 1), s);
    if (e == cudaSuccess) e = ml_malloc_async((void **)&mom, sizeof(double2) * n_mom, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gs, 0, sizeof(double) * 3 * (size_t)n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mom, 0, sizeof(double2) * n_mom, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_work, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_cic_adjoint_nearfar(a, dL_dM, gs, grad_params, mom, f->d_perm, grad_lens, scale,
                                       f->num_sms, s);
    if (gs) cudaFreeAsync(gs, s);
    if (mom) cudaFreeAsync(mom, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint");
    return ML_OK;
}

ml_status ml_cic_backward(ml_field *f, const float *dL_dM, double *grad_lens, double *grad_params,
                          void *stream)
{
    return ml_cic_backward_ex(f, dL_dM, grad_lens, grad_params, ML_ADJOINT_NEARFAR, stream);
}

ml_status ml_field_set_counts(ml_field *f, const uint32_t *counts, int32_t in_is_device, void *stream)
{
    if (!f || !counts) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (!f->d_map_u32) return fail(ML_ERR_STATE, "a CIC field has no integer counts");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)f->g.mnx * f->g.mny;
    unsigned long long sum = 0, st[ML_STAT_COUNT];
    ML_CK(cudaMemcpyAsync(f->d_map_u32, counts, npix * sizeof(uint32_t),
                          in_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    ML_CK(launch_map_sum(f->d_map_u32, npix, f->d_sum, f->num_sms, s));
    ML_CK(cudaMemcpyAsync(&sum, f->d_sum, sizeof(sum), cudaMemcpyDeviceToHost, s));
    ML_CK(cudaMemcpyAsync(st, f->d_stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    ML_CK(cudaStreamSynchronize(s));
    f->map_base = sum;
    f->in_at_set = st[ML_STAT_RAYS_IN];
    return ML_OK;
}

ml_status ml_find_peaks(ml_field *f, int32_t along, double nsigma, uint8_t *mask, int32_t *peaks,
                        int64_t capacity, int64_t *n_found, void *stream)
{
    if (!f || !n_found) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (!f->d_map_u32) return fail(ML_ERR_STATE, "peak identification needs an NGP count map");
    if (along != ML_ALONG_X && along != ML_ALONG_Y) return fail(ML_ERR_INVALID_ARG, "unknown curve direction");
    if (!(nsigma > 0.0) || !is_fin(nsigma)) return fail(ML_ERR_INVALID_ARG, "nsigma must be positive");
    if (capacity < 0 || (capacity > 0 && !peaks)) return fail(ML_ERR_INVALID_ARG, "bad peak list");
    if (mask && (uintptr_t)mask % 4 != 0) return fail(ML_ERR_INVALID_ARG, "mask must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)f->g.mnx * f->g.mny;
    uint8_t *m = mask;
    unsigned long long *found = nullptr, h_found = 0;
    cudaError_t e = cudaSuccess;
    if (!m) e = ml_malloc_async((void **)&m, npix + 4, s);
    if (e == cudaSuccess) e = ml_malloc_async((void **)&found, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_peaks(f->d_map_u32, f->g.mnx, f->g.mny, along, nsigma, m, peaks, capacity, found, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_found, found, sizeof(h_found), cudaMemcpyDeviceToHost, s);
    if (found) cudaFreeAsync(found, s);
    if (!mask && m) cudaFreeAsync(m, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "peak identification");
    *n_found = (int64_t)h_found;
    return ML_OK;
}

ml_status ml_peak_statistics(ml_field *f, int32_t along, double nsigma, const uint8_t *mask,
                             double caustic, const double *edges, int32_t nbins, uint64_t *n_peaks,
                             uint64_t *sum_counts, uint64_t *n_positions, void *stream)
{
    if (!f || !edges || !n_peaks || !sum_counts || !n_positions)
        return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (!f->d_map_u32) return fail(ML_ERR_STATE, "peak statistics need an NGP count map");
    if (along != ML_ALONG_X && along != ML_ALONG_Y) return fail(ML_ERR_INVALID_ARG, "unknown curve direction");
    if (nbins < 1 || nbins > ML_PEAK_STATS_MAX_BINS) return fail(ML_ERR_INVALID_ARG, "nbins out of range");
    if (!is_fin(caustic)) return fail(ML_ERR_INVALID_ARG, "caustic must be finite");
    for (int b = 0; b <= nbins; ++b)
        if (!is_fin(edges[b]) || (b > 0 && !(edges[b] > edges[b - 1])))
            return fail(ML_ERR_INVALID_ARG, "edges must be finite and strictly ascending");
    if (!mask && (!(nsigma > 0.0) || !is_fin(nsigma))) return fail(ML_ERR_INVALID_ARG, "nsigma must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    const int nx = f->g.mnx, ny = f->g.mny;
    const size_t npix = (size_t)nx * ny;
    const int len = along == ML_ALONG_X ? nx : ny;
    const double origin = along == ML_ALONG_X ? f->g.mx0 : f->g.my0;
    const double step = along == ML_ALONG_X ? f->g.dpx : f->g.dpy;
    // one scratch block: counters, edges, bin of each position, then (when the
    // caller gives no mask) the mask and the found counter of the peak step
    const size_t o_edges = 3 * (size_t)nbins * sizeof(unsigned long long);
    const size_t o_bins = o_edges + ((size_t)(nbins + 1) * sizeof(double) + 15) / 16 * 16;
    const size_t o_mask = o_bins + ((size_t)len * sizeof(int32_t) + 15) / 16 * 16;
    const size_t o_found = o_mask + (npix + 4 + 15) / 16 * 16;
    const size_t bytes = mask ? o_mask : o_found + 16;
    char *scratch = nullptr;
    std::vector<unsigned long long> h(3 * (size_t)nbins);
    cudaError_t e = ml_malloc_async((void **)&scratch, bytes, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + o_edges, edges, (size_t)(nbins + 1) * sizeof(double),
                            cudaMemcpyHostToDevice, s);
    const uint8_t *m = mask;
    if (e == cudaSuccess && !mask) {
        uint8_t *mm = reinterpret_cast<uint8_t *>(scratch + o_mask);
        e = launch_peaks(f->d_map_u32, nx, ny, along, nsigma, mm, nullptr, 0,
                         reinterpret_cast<unsigned long long *>(scratch + o_found), s);
        m = mm;
    }
    if (e == cudaSuccess)
        e = launch_peak_stats(f->d_map_u32, nx, ny, along, m, origin, step, caustic,
                              reinterpret_cast<const double *>(scratch + o_edges), nbins,
                              reinterpret_cast<int32_t *>(scratch + o_bins),
                              reinterpret_cast<unsigned long long *>(scratch), f->num_sms, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), scratch, h.size() * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "peak statistics");
    for (int b = 0; b < nbins; ++b) {
        n_peaks[b] = h[b];
        sum_counts[b] = h[(size_t)nbins + b];
        n_positions[b] = h[2 * (size_t)nbins + b];
    }
    return ML_OK;
}

ml_status ml_field_clear(ml_field *f, void *stream)
{
    if (!f) return fail(ML_ERR_INVALID_ARG, "field is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)f->g.mnx * f->g.mny;
    if (f->d_map_u32) ML_CK(cudaMemsetAsync(f->d_map_u32, 0, npix * sizeof(uint32_t), s));
    if (f->d_map_f32) ML_CK(cudaMemsetAsync(f->d_map_f32, 0, npix * sizeof(float), s));
    ML_CK(cudaMemsetAsync(f->d_stats, 0, ML_STAT_COUNT * sizeof(unsigned long long), s));
    ML_CK(cudaMemsetAsync(f->d_status, 0, sizeof(unsigned), s));
    f->rays_asked = 0;
    f->launches = 0;
    f->map_base = 0;
    f->in_at_set = 0;
    return ML_OK;
}

ml_status ml_field_stats(ml_field *f, uint64_t out[ML_STAT_COUNT], void *stream)
{
    if (!f || !out) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long st[ML_STAT_COUNT], sum = 0;
    unsigned flags = 0;
    if (f->d_map_u32)
        ML_CK(launch_map_sum(f->d_map_u32, (size_t)f->g.mnx * f->g.mny, f->d_sum, f->num_sms, s));
    ML_CK(cudaMemcpyAsync(st, f->d_stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    ML_CK(cudaMemcpyAsync(&flags, f->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    if (f->d_map_u32) ML_CK(cudaMemcpyAsync(&sum, f->d_sum, sizeof(sum), cudaMemcpyDeviceToHost, s));
    ML_CK(cudaStreamSynchronize(s));
    // a wrapped pixel loses 2^32 from the map's sum
    if (f->d_map_u32 && sum != f->map_base + (st[ML_STAT_RAYS_IN] - f->in_at_set)) flags |= 1u;
    for (int q = 0; q < ML_STAT_COUNT; ++q) out[q] = st[q];
    out[ML_STAT_LAUNCHES] = f->launches;
    out[ML_STAT_FLAGS] = flags;
    out[ML_STAT_RAYS_ASKED] = f->rays_asked;
    if (flags & 1u) return fail(ML_ERR_OVERFLOW, "a uint32 pixel count wrapped");
    if (flags & 2u) return fail(ML_ERR_ABORTED, "shooting was aborted");
    return ML_OK;
}

ml_status ml_field_info(const ml_field *f, ml_field_params *out)
{
    if (!f || !out) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    const Geo &g = f->g;
    memset(out, 0, sizeof(*out));
    out->ray_x0 = g.rx0; out->ray_y0 = g.ry0; out->ray_x1 = g.rx1; out->ray_y1 = g.ry1;
    out->l3x = g.l3x; out->l3y = g.l3y;
    out->n_rays_x = g.n3x; out->n_rays_y = g.n3y;
    out->map_x0 = g.mx0; out->map_y0 = g.my0; out->dpx = g.dpx; out->dpy = g.dpy;
    out->map_nx = g.mnx; out->map_ny = g.mny;
    out->n_star_in = g.n_star_in; out->l0 = g.l0;
    out->n1x = g.n1x; out->n1y = g.n1y; out->n2x = g.n2x; out->n2y = g.n2y;
    out->N1x = g.N1x; out->N1y = g.N1y; out->N2x = g.N2x; out->N2y = g.N2y;
    out->taylor_p = g.p; out->l2_sub_x = g.l2sx; out->l2_sub_y = g.l2sy;
    out->tuned = f->tuned;
    out->precision = g.precision; out->deposit = g.deposit;
    out->max_near = f->max_near;
    out->build = f->build_used;
    out->far_bound = f->far_bound;
    out->mu_per_count = (g.l3x * g.l3y) / (g.dpx * g.dpy);
    out->span_far = f->span_far;
    out->spans = f->desc.walk == ML_WALK_CERTIFIED && f->use_span ? 1 : 0;
    return ML_OK;
}

ml_status ml_fp32_fma_peak(int32_t two_lane, int32_t blocks_per_sm, int64_t iters, float *sink,
                           double *flop, void *stream)
{
    if (!sink || !flop) return fail(ML_ERR_INVALID_ARG, "NULL argument");
    if (blocks_per_sm < 1 || blocks_per_sm > 8) return fail(ML_ERR_INVALID_ARG, "blocks_per_sm must be in [1, 8]");
    if (iters < 1 || iters > (int64_t(1) << 32)) return fail(ML_ERR_INVALID_ARG, "iters must be in [1, 2^32]");
    int dev = 0, sms = 0;
    ML_CK(cudaGetDevice(&dev));
    ML_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)sms * (unsigned)blocks_per_sm;
    ML_CK(launch_fma_peak(two_lane != 0, blocks, iters, sink, (cudaStream_t)stream));
    *flop = fma_peak_flop(two_lane != 0, blocks, iters);
    return ML_OK;
}

ml_status ml_field_abort(ml_field *f, int32_t on)
{
    if (!f) return fail(ML_ERR_INVALID_ARG, "field is NULL");
    *(volatile int *)f->h_abort = on ? 1 : 0;
    return ML_OK;
}

ml_status ml_field_destroy(ml_field *f)
{
    if (!f) return ML_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(f->device);
    f->release();
    cudaSetDevice(cur);
    delete f;
    return ML_OK;
}

}  // extern "C"
