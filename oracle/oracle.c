/*
 * FP64 oracle for inverse ray-shooting through point-mass microlenses in a
 * locally linearised macro lens (Yang, Chen, Zheng & Luo, "Simulation of the
 * microlensing effect near the critical curve of the galaxy cluster").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct CPU code that the
 * tests, the smoke check and the benchmark's CPU-baseline leg use to check
 * the CUDA library.  Nothing in the product path may call it.  It shares no
 * code with the CUDA library.
 *
 * Units: angles in Einstein radii theta_E (Eq. 7), masses in units of M.
 * All arithmetic is IEEE binary64; build with -ffp-contract=off so that x86
 * and Arm hosts give the same bits.
 *
 * Lens equation: a macro term plus the microlens and negative-sheet terms of
 * Eq. 6:
 *   beta = macro(theta)
 *          - sum_k m_k (theta - theta_k) / |theta - theta_k|^2
 *          - alpha_{-kappa*}(theta)
 * with macro(theta) either the constant-(kappa, gamma) form of Eq. 1,
 * diag(1-kappa-gamma, 1-kappa+gamma) theta, or the fold form of Eq. 5 as
 * printed in Eq. 6, (d_x theta_x^2 / 2 + d_y theta_x theta_y,
 * 2 (1 - kappa_0) theta_y), whose Jacobian determinant is the
 * 2 (1 - kappa_0) (theta . d) of Eq. 4
 * with alpha_{-kappa*} the field of a uniform sheet of surface density
 * -kappa_* laid where the lenses are: a disc (centre c, radius R),
 * -kappa_* (theta - c) inside and -kappa_* R^2 (theta - c)/|theta - c|^2
 * outside; or a strip unbounded in x and bounded in y (centre line c_y,
 * half-width R), -2 kappa_* (theta_y - c_y) y-hat inside and
 * -2 kappa_* R sign(theta_y - c_y) y-hat outside.
 *
 * Ray lattice (§3.2, Level 3, Eq. 11): ray (i, j) sits at the centre of
 * level-3 pixel (i, j): theta = (rx0 + (i + 1/2) l3x, ry0 + (j + 1/2) l3y);
 * linear ray index r = j * n3x + i.
 *
 * Source-plane binning (§3.2, Eq. 12): pixel ix = floor((beta_x - mx0)/dpx),
 * kept iff 0 <= ix < mnx (likewise y).  A ray that lands exactly on a lens
 * (|theta - theta_k| = 0) is "dropped" and counted apart.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double kappa, gamma, kappa_star;
    double sheet_cx, sheet_cy, sheet_r;
    double rx0, ry0, l3x, l3y;
    int64_t n3x, n3y;
    double mx0, my0, dpx, dpy;
    int64_t mnx, mny;
    int64_t macro_mode;        /* 0: constant (kappa, gamma), Eq. 1; 1: fold, Eq. 5 */
    double kappa0, d_x, d_y;   /* fold parameters (d in 1/theta_E) */
    int64_t sheet_shape;       /* 0: disc, 1: strip along x */
} orc_geom;

/* Three-level grid of §3.2 as laid on the ray lattice: a level-2 cell holds
 * n2x x n2y rays, a level-1 cell n1x x n1y rays, n1 = l2sub * n2. */
typedef struct {
    int64_t n1x, n1y, n2x, n2y;
    int64_t N1x, N1y;          /* level-1 cells covering the lattice */
    int32_t p;                 /* highest Taylor order kept */
} orc_grid;

typedef struct {
    const double *x, *y, *m;
    int64_t n;
} orc_lenses;

/* ---- Eq. 6: the terms of the lens equation ------------------------------ */

/* Microlens deflection by direct summation over a lens list (§3.2: the
 * deflection of all microlenses summed for each ray).  Returns 1 if the ray
 * coincides with a lens. */
static int deflect_direct(const orc_lenses *L, const int64_t *sel, int64_t nsel,
                          double tx, double ty, double *ax, double *ay)
{
    double sx = 0.0, sy = 0.0;
    int64_t count = sel ? nsel : L->n;
    for (int64_t q = 0; q < count; ++q) {
        int64_t k = sel ? sel[q] : q;
        double dx = tx - L->x[k];
        double dy = ty - L->y[k];
        double r2 = dx * dx + dy * dy;
        if (r2 == 0.0) return 1;
        sx += L->m[k] * dx / r2;
        sy += L->m[k] * dy / r2;
    }
    *ax = sx;
    *ay = sy;
    return 0;
}

/* Deflection of the compensating negative sheet, alpha_{-kappa*} of Eq. 6:
 * minus the field of a uniform sheet of density kappa_*, whose divergence is
 * 2 kappa_* inside. */
static void sheet_deflection(const orc_geom *g, double tx, double ty,
                             double *ax, double *ay)
{
    double ux = tx - g->sheet_cx, uy = ty - g->sheet_cy;
    if (g->sheet_shape == 1) {
        /* an unbounded slab: by symmetry the field is along y, 2 kappa_* uy inside */
        double h = g->sheet_r;
        double v = uy > h ? h : (uy < -h ? -h : uy);
        *ax = 0.0;
        *ay = -2.0 * g->kappa_star * v;
        return;
    }
    double s2 = ux * ux + uy * uy;
    double R2 = g->sheet_r * g->sheet_r;
    if (s2 <= R2) {
        *ax = -g->kappa_star * ux;
        *ay = -g->kappa_star * uy;
    } else {
        *ax = -g->kappa_star * R2 * ux / s2;
        *ay = -g->kappa_star * R2 * uy / s2;
    }
}

/* The smooth (macro) part of beta: the constant-kappa, gamma lens of Eq. 1,
 * diag(1 - kappa - gamma, 1 - kappa + gamma) theta, or the fold of Eq. 5 near
 * the critical curve (the quadratic in theta_x, and 2 (1 - kappa_0) theta_y). */
static void macro_term(const orc_geom *g, double tx, double ty, double *mx, double *my)
{
    if (g->macro_mode == 1) {
        *mx = 0.5 * g->d_x * tx * tx + g->d_y * tx * ty;
        *my = 2.0 * (1.0 - g->kappa0) * ty;
    } else {
        *mx = (1.0 - g->kappa - g->gamma) * tx;
        *my = (1.0 - g->kappa + g->gamma) * ty;
    }
}

/* Ray r of the lattice: the centre of level-3 pixel (i, j), r = j n3x + i
 * (§3.2 Level 3). */
static void ray_position(const orc_geom *g, int64_t r, double *tx, double *ty)
{
    int64_t i = r % g->n3x, j = r / g->n3x;
    *tx = g->rx0 + ((double)i + 0.5) * g->l3x;
    *ty = g->ry0 + ((double)j + 0.5) * g->l3y;
}

/* Full lens equation (Eq. 6), direct sum. */
static int beta_direct(const orc_geom *g, const orc_lenses *L, double tx, double ty,
                       double *bx, double *by)
{
    double ax, ay, sx, sy, mx, my;
    if (deflect_direct(L, NULL, 0, tx, ty, &ax, &ay)) return 1;
    sheet_deflection(g, tx, ty, &sx, &sy);
    macro_term(g, tx, ty, &mx, &my);
    *bx = mx - ax - sx;
    *by = my - ay - sy;
    return 0;
}

/* Nearest-grid-point bin of Eq. 12; returns -1 outside the map. */
static int64_t bin_of(const orc_geom *g, double bx, double by)
{
    double fx = floor((bx - g->mx0) / g->dpx);
    double fy = floor((by - g->my0) / g->dpy);
    if (!(fx >= 0.0 && fx < (double)g->mnx && fy >= 0.0 && fy < (double)g->mny))
        return -1;
    return (int64_t)fy * g->mnx + (int64_t)fx;
}

/* ---- threading: a plain parallel-for over ray ranges --------------------- */

typedef void (*range_fn)(void *ctx, int64_t b, int64_t e, int tid);
typedef struct { range_fn fn; void *ctx; int64_t b, e; int tid; } job_t;

static void *job_main(void *a)
{
    job_t *j = (job_t *)a;
    j->fn(j->ctx, j->b, j->e, j->tid);
    return NULL;
}

static void parallel_for(range_fn fn, void *ctx, int64_t b, int64_t e, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (e - b < nthreads) nthreads = (int)((e - b) > 0 ? (e - b) : 1);
    pthread_t th[256];
    job_t jobs[256];
    if (nthreads > 256) nthreads = 256;
    int64_t n = e - b;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].tid = t;
        jobs[t].b = b + n * t / nthreads;
        jobs[t].e = b + n * (t + 1) / nthreads;
        if (nthreads == 1) { job_main(&jobs[t]); return; }
        pthread_create(&th[t], NULL, job_main, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ---- direct-sum shooting: the plain definition of the map --------------- */

typedef struct {
    const orc_geom *g; orc_lenses L;
    uint64_t *counts; uint64_t stats[256][3];
} shoot_ctx;

static void shoot_range(void *c, int64_t b, int64_t e, int tid)
{
    shoot_ctx *s = (shoot_ctx *)c;
    uint64_t in = 0, out = 0, dropped = 0;
    for (int64_t r = b; r < e; ++r) {
        double tx, ty, bx, by;
        ray_position(s->g, r, &tx, &ty);
        if (beta_direct(s->g, &s->L, tx, ty, &bx, &by)) { ++dropped; continue; }
        int64_t p = bin_of(s->g, bx, by);
        if (p < 0) { ++out; continue; }
        __atomic_fetch_add(&s->counts[p], 1, __ATOMIC_RELAXED);
        ++in;
    }
    s->stats[tid][0] = in; s->stats[tid][1] = out; s->stats[tid][2] = dropped;
}

/* Shoot rays [ray_begin, ray_end) and add their counts N_ij (Eq. 12) to
 * `counts` (uint64, mny x mnx row-major).  stats = {in map, out, dropped}. */
int orc_shoot_direct(const orc_geom *g, const double *x, const double *y, const double *m,
                     int64_t n, int64_t ray_begin, int64_t ray_end,
                     uint64_t *counts, uint64_t *stats, int nthreads)
{
    shoot_ctx *s = (shoot_ctx *)calloc(1, sizeof(shoot_ctx));
    if (!s) return 1;
    s->g = g; s->L.x = x; s->L.y = y; s->L.m = m; s->L.n = n; s->counts = counts;
    parallel_for(shoot_range, s, ray_begin, ray_end, nthreads);
    stats[0] = stats[1] = stats[2] = 0;
    for (int t = 0; t < 256; ++t) {
        stats[0] += s->stats[t][0]; stats[1] += s->stats[t][1]; stats[2] += s->stats[t][2];
    }
    free(s);
    return 0;
}

/* ---- per-ray source positions ------------------------------------------ */

typedef struct {
    const orc_geom *g; orc_lenses L; const orc_grid *grid;
    const int64_t *idx; double *beta; int32_t *flag; int mode;
} beta_ctx;

static int beta_interp(const orc_geom *g, const orc_grid *grid, const orc_lenses *L,
                       int64_t r, double *bx, double *by);

static void beta_range(void *c, int64_t b, int64_t e, int tid)
{
    (void)tid;
    beta_ctx *s = (beta_ctx *)c;
    for (int64_t q = b; q < e; ++q) {
        double tx, ty, bx = 0.0, by = 0.0;
        int64_t r = s->idx[q];
        ray_position(s->g, r, &tx, &ty);
        int drop = s->mode == 0 ? beta_direct(s->g, &s->L, tx, ty, &bx, &by)
                                : beta_interp(s->g, s->grid, &s->L, r, &bx, &by);
        s->beta[2 * q] = bx; s->beta[2 * q + 1] = by; s->flag[q] = drop;
    }
}

/* Source position beta (Eq. 6, direct sum over all lenses) of the rays with
 * linear indices idx[0..nidx).  flag[q] = 1 marks a dropped ray. */
int orc_beta_direct(const orc_geom *g, const double *x, const double *y, const double *m,
                    int64_t n, const int64_t *idx, int64_t nidx,
                    double *beta, int32_t *flag, int nthreads)
{
    beta_ctx s = { g, { x, y, m, n }, NULL, idx, beta, flag, 0 };
    parallel_for(beta_range, &s, 0, nidx, nthreads);
    return 0;
}

/* ---- the near/far scheme of §3.2 (Eq. 9), brute force -------------------- */

/* Level-1 cell of a lens (§3.2, Level 1), clamped to one ring outside the
 * lattice; anything further away is far for every cell. */
static void lens_cell(const orc_geom *g, const orc_grid *grid, double x, double y,
                      int64_t *cx, int64_t *cy)
{
    double l1x = (double)grid->n1x * g->l3x, l1y = (double)grid->n1y * g->l3y;
    double fx = floor((x - g->rx0) / l1x), fy = floor((y - g->ry0) / l1y);
    if (fx < -2.0) fx = -2.0;
    if (fx > (double)grid->N1x + 1.0) fx = (double)grid->N1x + 1.0;
    if (fy < -2.0) fy = -2.0;
    if (fy > (double)grid->N1y + 1.0) fy = (double)grid->N1y + 1.0;
    *cx = (int64_t)fx;
    *cy = (int64_t)fy;
}

/* Is lens k near to level-1 cell (c1x, c1y)?  Near = inside the 3 x 3 block
 * of level-1 cells centred on it (the dotted box of Fig. 1). */
static int is_near(const orc_geom *g, const orc_grid *grid, const orc_lenses *L,
                   int64_t k, int64_t c1x, int64_t c1y)
{
    int64_t cx, cy;
    lens_cell(g, grid, L->x[k], L->y[k], &cx, &cy);
    return llabs(cx - c1x) <= 1 && llabs(cy - c1y) <= 1;
}

static void node_of(const orc_geom *g, const orc_grid *grid, int64_t c2x, int64_t c2y,
                    double *zx, double *zy)
{
    double l2x = (double)grid->n2x * g->l3x, l2y = (double)grid->n2y * g->l3y;
    *zx = g->rx0 + ((double)c2x + 0.5) * l2x;
    *zy = g->ry0 + ((double)c2y + 0.5) * l2y;
}

/* Taylor coefficients of the far field at a level-2 node (§3.2, Level 2):
 * conj(alpha_far)(z) = sum_n c_n (z - z_node)^n with
 * c_n = - sum_{k far} m_k / (z_k - z_node)^{n+1},  n = 0..p,
 * the far set being every lens outside the node's 3 x 3 level-1 block. */
static void node_coeffs(const orc_geom *g, const orc_grid *grid, const orc_lenses *L,
                        int64_t c2x, int64_t c2y, double complex *c)
{
    double zx, zy;
    node_of(g, grid, c2x, c2y, &zx, &zy);
    int64_t c1x = c2x * grid->n2x / grid->n1x, c1y = c2y * grid->n2y / grid->n1y;
    for (int n = 0; n <= grid->p; ++n) c[n] = 0.0;
    for (int64_t k = 0; k < L->n; ++k) {
        if (is_near(g, grid, L, k, c1x, c1y)) continue;
        double complex w = 1.0 / ((L->x[k] - zx) + I * (L->y[k] - zy));
        double complex t = L->m[k] * w;
        for (int n = 0; n <= grid->p; ++n) {
            c[n] -= t;
            t *= w;
        }
    }
}

/* Eq. 9 with the near part summed directly and the far part taken from the
 * node's Taylor series. */
static int beta_interp(const orc_geom *g, const orc_grid *grid, const orc_lenses *L,
                       int64_t r, double *bx, double *by)
{
    int64_t i = r % g->n3x, j = r / g->n3x;
    double tx, ty;
    ray_position(g, r, &tx, &ty);
    int64_t c1x = i / grid->n1x, c1y = j / grid->n1y;
    int64_t c2x = i / grid->n2x, c2y = j / grid->n2y;

    int64_t *near = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L->n > 0 ? L->n : 1));
    int64_t nn = 0;
    for (int64_t k = 0; k < L->n; ++k)
        if (is_near(g, grid, L, k, c1x, c1y)) near[nn++] = k;
    double ax = 0.0, ay = 0.0;
    int drop = deflect_direct(L, near, nn, tx, ty, &ax, &ay);
    free(near);
    if (drop) return 1;

    double complex c[64];
    node_coeffs(g, grid, L, c2x, c2y, c);
    double zx, zy;
    node_of(g, grid, c2x, c2y, &zx, &zy);
    double complex d = (tx - zx) + I * (ty - zy);
    double complex F = 0.0;
    for (int n = grid->p; n >= 0; --n) F = F * d + c[n];
    /* alpha_far = conj(F) */
    double sx, sy, mx, my;
    sheet_deflection(g, tx, ty, &sx, &sy);
    macro_term(g, tx, ty, &mx, &my);
    *bx = mx - ax - creal(F) - sx;
    *by = my - ay + cimag(F) - sy;
    return 0;
}

/* Source positions by the near/far scheme, computed brute force. */
int orc_beta_interp(const orc_geom *g, const orc_grid *grid, const double *x, const double *y,
                    const double *m, int64_t n, const int64_t *idx, int64_t nidx,
                    double *beta, int32_t *flag, int nthreads)
{
    if (grid->p < 0 || grid->p > 62) return 1;
    beta_ctx s = { g, { x, y, m, n }, grid, idx, beta, flag, 1 };
    parallel_for(beta_range, &s, 0, nidx, nthreads);
    return 0;
}

/* Far-field Taylor coefficients c_0..c_p of the listed level-2 nodes,
 * out[(q * (p+1) + n) * 2 + {0,1}] = (Re, Im) of c_n at node q. */
int orc_node_coeffs(const orc_geom *g, const orc_grid *grid, const double *x, const double *y,
                    const double *m, int64_t n, const int64_t *c2x, const int64_t *c2y,
                    int64_t nnodes, double *out)
{
    if (grid->p < 0 || grid->p > 62) return 1;
    orc_lenses L = { x, y, m, n };
    double complex c[64];
    for (int64_t q = 0; q < nnodes; ++q) {
        node_coeffs(g, grid, &L, c2x[q], c2y[q], c);
        for (int k = 0; k <= grid->p; ++k) {
            out[(q * (grid->p + 1) + k) * 2] = creal(c[k]);
            out[(q * (grid->p + 1) + k) * 2 + 1] = cimag(c[k]);
        }
    }
    return 0;
}

/* Truncation bound of the far series at ray r:
 * |sum_{n>p} c_n d^n| <= sum_{k far} m_k rho^{p+1} / (r_k^{p+1} (r_k - rho)),
 * rho = |z - z_node|, r_k = |z_k - z_node| (geometric tail of 1/(z_k - z)).
 * Returns +inf if some far lens is not farther from the node than the ray. */
int orc_remainder_bound(const orc_geom *g, const orc_grid *grid, const double *x,
                        const double *y, const double *m, int64_t n,
                        const int64_t *idx, int64_t nidx, double *out)
{
    orc_lenses L = { x, y, m, n };
    for (int64_t q = 0; q < nidx; ++q) {
        int64_t r = idx[q];
        int64_t i = r % g->n3x, j = r / g->n3x;
        double tx, ty, zx, zy;
        ray_position(g, r, &tx, &ty);
        int64_t c2x = i / grid->n2x, c2y = j / grid->n2y;
        int64_t c1x = i / grid->n1x, c1y = j / grid->n1y;
        node_of(g, grid, c2x, c2y, &zx, &zy);
        double rho = hypot(tx - zx, ty - zy), b = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            if (is_near(g, grid, &L, k, c1x, c1y)) continue;
            double rk = hypot(x[k] - zx, y[k] - zy);
            if (rk <= rho) { b = INFINITY; break; }
            b += m[k] * pow(rho / rk, (double)(grid->p + 1)) / (rk - rho);
        }
        out[q] = b;
    }
    return 0;
}

/* ---- cloud-in-cell deposition and its adjoint --------------------------- */

/* Cloud-in-cell weights of a ray at source position (bx, by): the ray is
 * shared between the four pixel centres around it, pixel (i, j) having its
 * centre at (mx0 + (i + 1/2) dpx, my0 + (j + 1/2) dpy). */
static void cic_cell(const orc_geom *g, double bx, double by, int64_t *ix, int64_t *iy,
                     double *wx, double *wy)
{
    double fx = (bx - g->mx0) / g->dpx - 0.5;
    double fy = (by - g->my0) / g->dpy - 0.5;
    double flx = floor(fx), fly = floor(fy);
    *wx = fx - flx;
    *wy = fy - fly;
    /* clamp far-away rays to a sentinel cell outside the map */
    if (flx < -2.0 || flx > (double)g->mnx + 1.0) flx = -2.0;
    if (fly < -2.0 || fly > (double)g->mny + 1.0) fly = -2.0;
    *ix = (int64_t)flx;
    *iy = (int64_t)fly;
}

typedef struct {
    const orc_geom *g; orc_lenses L; double **part; int nthreads;
} cic_ctx;

static void cic_range(void *c, int64_t b, int64_t e, int tid)
{
    cic_ctx *s = (cic_ctx *)c;
    const orc_geom *g = s->g;
    double *map = s->part[tid];
    for (int64_t r = b; r < e; ++r) {
        double tx, ty, bx, by, wx, wy;
        int64_t ix, iy;
        ray_position(g, r, &tx, &ty);
        if (beta_direct(g, &s->L, tx, ty, &bx, &by)) continue;
        cic_cell(g, bx, by, &ix, &iy, &wx, &wy);
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb) {
                int64_t px = ix + a, py = iy + bb;
                if (px < 0 || px >= g->mnx || py < 0 || py >= g->mny) continue;
                double w = (a ? wx : 1.0 - wx) * (bb ? wy : 1.0 - wy);
                map[py * g->mnx + px] += w;
            }
    }
}

/* Cloud-in-cell ray map of rays [ray_begin, ray_end): map (mny x mnx, FP64)
 * receives the sum of each ray's bilinear weights (units: rays). */
int orc_cic_forward(const orc_geom *g, const double *x, const double *y, const double *m,
                    int64_t n, int64_t ray_begin, int64_t ray_end, double *map, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int64_t npix = g->mnx * g->mny;
    double **part = (double **)calloc((size_t)nthreads, sizeof(double *));
    for (int t = 0; t < nthreads; ++t) part[t] = (double *)calloc((size_t)npix, sizeof(double));
    cic_ctx s = { g, { x, y, m, n }, part, nthreads };
    parallel_for(cic_range, &s, ray_begin, ray_end, nthreads);
    for (int t = 0; t < nthreads; ++t) {
        for (int64_t p = 0; p < npix; ++p) map[p] += part[t][p];
        free(part[t]);
    }
    free(part);
    return 0;
}

typedef struct {
    const orc_geom *g; orc_lenses L; const double *G; double scale;
    double **glens; double (*gpar)[3];
} grad_ctx;

/* Adjoint of the cloud-in-cell map.  With M = scale * (CIC map) and a given
 * G = dLoss/dM, each ray's dLoss/dbeta follows from the bilinear weights, and
 * the chain rule through Eq. 6 gives
 *   dbeta/dkappa   = (-theta_x, -theta_y)
 *   dbeta/dgamma   = (-theta_x, +theta_y)
 *   dbeta/dkappa_* = (theta - c)            inside the sheet's disc,
 *                    R^2 (theta - c)/|theta - c|^2 outside,
 *   dbeta/dm_k     = -(theta - theta_k)/|theta - theta_k|^2,
 *   dbeta/dtheta_k = m_k (I r^2 - 2 d d^T) / r^4,  d = theta - theta_k. */
static void grad_range(void *c, int64_t b, int64_t e, int tid)
{
    grad_ctx *s = (grad_ctx *)c;
    const orc_geom *g = s->g;
    const orc_lenses *L = &s->L;
    double *gl = s->glens[tid];
    double *gp = s->gpar[tid];
    for (int64_t r = b; r < e; ++r) {
        double tx, ty, bx, by, wx, wy;
        int64_t ix, iy;
        ray_position(g, r, &tx, &ty);
        if (beta_direct(g, L, tx, ty, &bx, &by)) continue;
        cic_cell(g, bx, by, &ix, &iy, &wx, &wy);
        double Gv[2][2];
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb) {
                int64_t px = ix + a, py = iy + bb;
                Gv[a][bb] = (px < 0 || px >= g->mnx || py < 0 || py >= g->mny)
                                ? 0.0 : s->G[py * g->mnx + px];
            }
        double gbx = s->scale / g->dpx *
                     ((Gv[1][0] - Gv[0][0]) * (1.0 - wy) + (Gv[1][1] - Gv[0][1]) * wy);
        double gby = s->scale / g->dpy *
                     ((Gv[0][1] - Gv[0][0]) * (1.0 - wx) + (Gv[1][1] - Gv[1][0]) * wx);
        if (gbx == 0.0 && gby == 0.0) continue;
        gp[0] += gbx * (-tx) + gby * (-ty);
        gp[1] += gbx * (-tx) + gby * (ty);
        double ux = tx - g->sheet_cx, uy = ty - g->sheet_cy, s2 = ux * ux + uy * uy;
        double R2 = g->sheet_r * g->sheet_r;
        if (s2 <= R2) gp[2] += gbx * ux + gby * uy;
        else gp[2] += (gbx * ux + gby * uy) * R2 / s2;
        for (int64_t k = 0; k < L->n; ++k) {
            double dx = tx - L->x[k], dy = ty - L->y[k];
            double r2 = dx * dx + dy * dy;
            double r4 = r2 * r2;
            gl[3 * k + 2] += -(gbx * dx + gby * dy) / r2;
            double jxx = L->m[k] * (r2 - 2.0 * dx * dx) / r4;
            double jxy = L->m[k] * (-2.0 * dx * dy) / r4;
            double jyy = L->m[k] * (r2 - 2.0 * dy * dy) / r4;
            gl[3 * k + 0] += gbx * jxx + gby * jxy;
            gl[3 * k + 1] += gbx * jxy + gby * jyy;
        }
    }
}

/* Gradient of a loss of M = scale * CIC(rays [b, e)) given G = dLoss/dM:
 * glens[3k + {0,1,2}] = dLoss/d(x_k, y_k, m_k); gpar = dLoss/d(kappa, gamma, kappa_*). */
int orc_cic_grad(const orc_geom *g, const double *x, const double *y, const double *m,
                 int64_t n, int64_t ray_begin, int64_t ray_end, const double *G,
                 double scale, double *glens, double *gpar, int nthreads)
{
    if (g->macro_mode != 0) return -2;     /* kappa, gamma terms are those of Eq. 1 */
    if (g->sheet_shape != 0) return -3;    /* dbeta/dkappa_* above is the disc sheet's */
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    double **gl = (double **)calloc((size_t)nthreads, sizeof(double *));
    double (*gp)[3] = calloc((size_t)nthreads, sizeof(double[3]));
    for (int t = 0; t < nthreads; ++t) gl[t] = (double *)calloc((size_t)(3 * n), sizeof(double));
    grad_ctx s = { g, { x, y, m, n }, G, scale, gl, gp };
    parallel_for(grad_range, &s, ray_begin, ray_end, nthreads);
    memset(glens, 0, sizeof(double) * (size_t)(3 * n));
    gpar[0] = gpar[1] = gpar[2] = 0.0;
    for (int t = 0; t < nthreads; ++t) {
        for (int64_t k = 0; k < 3 * n; ++k) glens[k] += gl[t][k];
        for (int q = 0; q < 3; ++q) gpar[q] += gp[t][q];
        free(gl[t]);
    }
    free(gl);
    free(gp);
    return 0;
}
