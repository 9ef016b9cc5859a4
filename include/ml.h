/*
 * ml.h - C ABI of the GB300 microlensing ray-shooting library.
 *
 * Computes source-plane magnification maps by inverse ray-shooting through a
 * field of point-mass microlenses embedded in a locally linearised macro lens,
 * following Yang, Chen, Zheng & Luo, "Simulation of the microlensing effect
 * near the critical curve of the galaxy cluster" (§2-§3).
 *
 * Conventions (every entry point):
 *  - Angles are in Einstein radii theta_E of the unit mass (Eq. 7); masses in
 *    units of that mass.
 *  - Every call returns an ml_status; nothing throws across the ABI.  On an
 *    error, ml_last_error() returns a message for the calling thread.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are ordered on that stream; a call that must read device
 *    results on the host (ml_field_create, ml_field_stats) synchronises it.
 *  - The library owns ml_field objects and every device buffer inside them
 *    (stream-ordered allocations on the device current at create time).  The
 *    caller owns every pointer it passes in and every output buffer.
 *  - Pointers documented as "device" must point to memory of the field's
 *    device; "host" pointers to ordinary (pageable or pinned) host memory.
 *  - The library is built for sm_103a only and fails with ML_ERR_CUDA on any
 *    other device.  There is no CPU fallback.
 */
#ifndef ML_H
#define ML_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ML_ABI_VERSION 4

typedef enum {
    ML_OK = 0,
    ML_ERR_INVALID_ARG = 1,  /* a null pointer, a bad size or an inconsistent descriptor */
    ML_ERR_OOM = 2,          /* a device or host allocation failed */
    ML_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    ML_ERR_ABORTED = 4,      /* ml_field_abort() stopped a shooting run; the map holds a prefix */
    ML_ERR_OVERFLOW = 5,     /* a uint32 pixel count wrapped; the map is invalid */
    ML_ERR_STATE = 6,        /* the call does not fit the field's mode (e.g. counts of a CIC map) */
    ML_ERR_UNSUPPORTED = 7   /* the inputs need a feature this build does not have */
} ml_status;

/* precision modes (ml_field_desc.precision) */
#define ML_PREC_DIRECT64   0  /* FP64 direct sum over all lenses for every ray (§3.2, first formula) */
#define ML_PREC_NEARFAR64  1  /* FP64 near/far scheme (Eq. 9), node coefficients in FP64 */
#define ML_PREC_MIXED      2  /* near sum and Taylor evaluation in FP32 on node-relative
                                 coordinates; node coefficients, node positions and the
                                 integer pixel base in FP64 */

/* deposition modes (ml_field_desc.deposit) */
#define ML_DEPOSIT_NGP 0      /* nearest grid point: uint32 ray counts N_ij (§3.2) */
#define ML_DEPOSIT_CIC 1      /* cloud in cell: float32 bilinear ray weights */

/* coefficient builds (ml_field_desc.build) */
#define ML_BUILD_AUTO         0  /* hierarchical when it is available, else direct */
#define ML_BUILD_DIRECT       1  /* far-field sum evaluated at every level-2 node */
#define ML_BUILD_HIERARCHICAL 2  /* high-order expansions shifted to the nodes */

/* ml_magnification_map(want) */
#define ML_MAP_COUNTS_U32 0   /* N_ij as uint32 (NGP only) */
#define ML_MAP_MU_F32     1   /* mu_ij = N_ij S_I / S_S (Eq. 12) as float32 */
#define ML_MAP_MU_F64     2   /* the same as float64 */

/* indices into the array filled by ml_field_stats */
#define ML_STAT_RAYS_IN     0  /* rays binned inside the map */
#define ML_STAT_RAYS_OUT    1  /* rays landing outside the map */
#define ML_STAT_RAYS_DROP   2  /* rays that hit a lens exactly (|theta - theta_k| = 0) */
#define ML_STAT_NEAR_PAIRS  3  /* ray-lens pairs summed directly */
#define ML_STAT_TASKS       4  /* warp tasks processed */
#define ML_STAT_LAUNCHES    5  /* shooting kernel launches */
#define ML_STAT_FLAGS       6  /* bit 0: count overflow, bit 1: aborted */
#define ML_STAT_RAYS_ASKED  7  /* rays requested by ml_shoot_rays so far */
#define ML_STAT_RAYS_EVAL   8  /* mixed NGP mode: rays whose source position was evaluated
                                  one by one (the rest were certified, see ML_WALK_CERTIFIED) */
#define ML_STAT_SPANS       9  /* mixed NGP mode: spans of rays certified to share a pixel */
#define ML_STAT_COUNT      10  /* length of the ml_field_stats array */

/* Ray walks of the mixed mode's NGP counts (ml_field_desc.walk).  Both give
 * every ray the pixel of the same per-ray FP32 arithmetic (Eq. 9), so their
 * count maps are bit-identical.
 *  ML_WALK_CERTIFIED (0, default): along a lattice row a lane evaluates a
 *    probe ray ahead of its last evaluated ray; when both land in one pixel
 *    and a rigorous bound (FP32 rounding of the evaluation, plus the
 *    curvature of the row's deflection between them) shows that every ray
 *    between them lands there too, those rays are counted without being
 *    evaluated.  Otherwise the probe moves closer, down to the next ray.
 *  ML_WALK_PER_RAY (1): every ray is evaluated. */
#define ML_WALK_CERTIFIED 0
#define ML_WALK_PER_RAY   1

typedef struct ml_field ml_field;  /* opaque, owned by the library */

/*
 * Description of one magnification map.  Zero-initialise, set abi_version =
 * ML_ABI_VERSION, then fill in what is needed; zero fields take the defaults
 * stated beside them.
 */
typedef struct {
    int32_t abi_version;
    int32_t precision;          /* ML_PREC_*; default ML_PREC_DIRECT64 (= 0) */
    int32_t deposit;            /* ML_DEPOSIT_*; default NGP */
    int32_t build;              /* ML_BUILD_*; default AUTO */

    /* Macro model, Eq. 1 with constant convergence and shear: total kappa,
     * shear gamma, and the stellar convergence kappa_* removed by the
     * negative sheet of Eq. 6. */
    double kappa, gamma, kappa_star;

    /* Microlenses (Eq. 6): positions and masses, n_lens entries, FP64,
     * copied at create time.  Host or device memory per lens_mem_is_device. */
    const double *lens_x, *lens_y, *lens_m;
    int64_t n_lens;
    int32_t lens_mem_is_device;
    int32_t taylor_p;           /* highest Taylor order of the far field; 0 = the
                                   smallest order whose truncation bound meets far_tol */

    /* Support of the negative mass sheet: a uniform disc of density
     * -kappa_* with this centre and radius (reading of Eq. 6). */
    double sheet_cx, sheet_cy, sheet_radius;

    /* Ray rectangle (image plane).  All four zero: the pre-image of the map
     * widened by the protection band 10 sqrt(kappa_*) per side (§3.1). */
    double ray_x0, ray_y0, ray_x1, ray_y1;
    /* Rays per side.  Both zero: N_rays = n_av * map_nx * map_ny (Eq. 8) on a
     * square lattice of spacing L_3 (Eq. 11). */
    int64_t n_rays_x, n_rays_y;
    double n_av;

    /* Source-plane map: [map_x0, map_x1) x [map_y0, map_y1), map_nx x map_ny
     * pixels, row-major with x fastest. */
    double map_x0, map_y0, map_x1, map_y1;
    int32_t map_nx, map_ny;

    /* Level grids (§3.2).  l1_x, l1_y zero: Eq. 10 on each side (or the
     * autotuner's size when tune is set).  l2_sub_x, l2_sub_y: level-2 cells
     * per level-1 cell along x and y; both zero: the paper's 20 x 20, or the
     * autotuner's choice when tune is set. */
    double l1_x, l1_y;
    int32_t l2_sub_x, l2_sub_y;
    double far_tol;             /* target truncation bound for taylor_p = 0; 0 = 1e-7 */
    uint64_t max_launch_rays;   /* rays per shooting launch; 0 = 2^36 */
    int32_t tune;               /* 1, with l2_sub_x = l2_sub_y = 0: the autotuner picks
                                   the level-2 grid (and with it p) and, unless l1_x or
                                   l1_y is set, the level-1 size (1, 1/sqrt2, 1/2 or
                                   1/(2 sqrt2) of Eq. 10's): a cost model ranks 48 grids,
                                   then the best grid of each of the three best level-1
                                   sizes is built and timed on slices of rays and the
                                   fastest is taken.  The far-field bound stays within
                                   far_tol.  The choice is cached per process for the same
                                   descriptor and lenses; ML_TUNE_LOG=1 in the environment
                                   prints the timed candidates. */
    int32_t walk;               /* ML_WALK_*; default ML_WALK_CERTIFIED */

    /* Macro model.  ML_MACRO_LINEAR (0): the constant-(kappa, gamma) form of
     * Eq. 1 above.  ML_MACRO_FOLD (1): the fold near the critical curve, Eq. 5
     * as printed in Eq. 6:
     *   macro(theta) = (d_x theta_x^2 / 2 + d_y theta_x theta_y, 2 (1 - kappa0) theta_y),
     * with d = -(grad kappa)_0 - (grad gamma)_0 in units of 1/theta_E
     * (kappa and gamma are then unused).  The default ray rectangle is the
     * bounding box of the pre-image of the protected map, which must reach
     * beyond the caustic (images exist).  The gradients of ml_cic_backward are
     * defined for ML_MACRO_LINEAR only. */
    int32_t macro_mode;
    /* Shape of the negative sheet of Eq. 6 (a uniform sheet laid where the
     * lenses are).  ML_SHEET_DISC (0): the disc (sheet_cx, sheet_cy,
     * sheet_radius) above.  ML_SHEET_STRIP (1): a strip unbounded in x with
     * centre line sheet_cy and half-width sheet_radius in y, for lenses in a
     * long rectangle; its field is -2 kappa_* (theta_y - sheet_cy) y-hat
     * inside.  The near/far modes need every ray inside the sheet. */
    int32_t sheet_shape;
    double kappa0, d_x, d_y;
    /* Certified walk (ML_WALK_CERTIFIED): a warp's level-2 column that has
     * near lenses is walked in certified spans only if every near lens lies
     * farther than span_far lattice spacings (l3x) from its rays, else ray by
     * ray.  0: the library's choice (3000; with tune, whichever of 3000, 1500,
     * 700, 300, 100, +inf and no certified spans at all measured fastest; in a
     * batch, +inf).  Any choice gives the same counts. */
    double span_far;
} ml_field_desc;

/* Macro models of ml_field_desc.macro_mode. */
enum { ML_MACRO_LINEAR = 0, ML_MACRO_FOLD = 1 };
/* Sheet shapes of ml_field_desc.sheet_shape. */
enum { ML_SHEET_DISC = 0, ML_SHEET_STRIP = 1 };

/* Derived parameters of a field (what §3.1-§3.2 compute from the desc). */
typedef struct {
    double ray_x0, ray_y0, ray_x1, ray_y1;  /* ray rectangle */
    double l3x, l3y;                        /* level-3 pixel (ray spacing) */
    int64_t n_rays_x, n_rays_y;             /* lattice size; ray r = j * n_rays_x + i */
    double map_x0, map_y0, dpx, dpy;        /* map origin and pixel size */
    int32_t map_nx, map_ny;
    int64_t n_star_in;                      /* lenses inside the ray rectangle (N_* of §3.1) */
    double l0;                              /* mean spacing per lens (Eq. 10); +inf if none */
    int64_t n1x, n1y, n2x, n2y;             /* rays per level-1 and level-2 cell side */
    int64_t N1x, N1y, N2x, N2y;             /* cells across the lattice */
    int32_t taylor_p;
    int32_t l2_sub_x, l2_sub_y;             /* level-2 cells per level-1 cell side */
    int32_t precision, deposit;
    int32_t max_near;                       /* largest near-lens list of a level-1 cell */
    int32_t build;                          /* coefficient build that ran (ML_BUILD_*) */
    int32_t tuned;                          /* 1 if the autotuner chose the level-2 grid */
    double far_bound;                       /* truncation bound at taylor_p (theta_E) */
    double mu_per_count;                    /* S_I / S_S of Eq. 12 */
    double span_far;                        /* certified walk's lens-column threshold in use */
    int32_t spans;                          /* 1 if the counting kernel walks certified spans (the
                                               autotuner may find the per-ray kernel faster) */
    int32_t reserved;
} ml_field_params;

/*
 * ml_field_create - set up one map (§3.1 parameters, §3.2 level grids, the
 * far-field Taylor coefficients at every level-2 node, a zeroed map).
 *  desc:   host pointer, read only; lens arrays are copied.
 *  stream: stream for the device work; synchronised before return.
 *  out:    receives the new field (host pointer to a handle).
 * Errors: ML_ERR_INVALID_ARG for a bad descriptor (null lens arrays with
 * n_lens > 0, empty map, singular macro map with no explicit ray rectangle,
 * non-positive sizes, abi_version mismatch); ML_ERR_UNSUPPORTED when the
 * near/far modes meet rays outside the sheet's disc, or a level-1 cell has
 * more near lenses than shared memory holds; ML_ERR_OOM; ML_ERR_CUDA.
 * On error *out is NULL and nothing is leaked.
 */
ml_status ml_field_create(const ml_field_desc *desc, void *stream, ml_field **out);

/*
 * ml_shoot_rays - shoot rays with linear lattice indices [ray_begin, ray_end)
 * (ray r = (i, j), i = r mod n_rays_x, j = r div n_rays_x, at the centre of
 * level-3 pixel (i, j); §3.2 Level 3) and add them to the map: NGP counts
 * N_ij, or CIC weights.  Accumulates across calls, so disjoint ranges can be
 * shot in any order (bit-identical NGP result).  Asynchronous on `stream`;
 * long ranges are split into launches of at most max_launch_rays rays.
 * Errors: ML_ERR_INVALID_ARG if ray_begin > ray_end or ray_end exceeds the
 * lattice; ML_ERR_CUDA.  Errors found inside kernels (overflow, abort) are
 * reported by ml_field_stats / ml_field_check.
 */
ml_status ml_shoot_rays(ml_field *f, uint64_t ray_begin, uint64_t ray_end, void *stream);

/*
 * ml_magnification_map - write the map: want = ML_MAP_COUNTS_U32 (NGP counts,
 * map_ny x map_nx uint32), ML_MAP_MU_F32 or ML_MAP_MU_F64 (mu_ij = N_ij S_I /
 * S_S, Eq. 12; for CIC maps the weights take the place of N_ij).
 *  out: caller-owned buffer of map_nx * map_ny elements, device memory if
 *       out_is_device else host memory (then the call synchronises stream).
 *       Host memory that is page-locked and mapped (cudaHostAlloc, pinned
 *       tensors) receives mu straight from the kernel over the host link;
 *       other host memory receives it through a device buffer and a copy.
 * Errors: ML_ERR_STATE for counts of a CIC map; ML_ERR_INVALID_ARG; ML_ERR_CUDA.
 */
ml_status ml_magnification_map(ml_field *f, int32_t want, void *out, int32_t out_is_device,
                               void *stream);

/*
 * ml_light_curves - light curves of a Gaussian source (§4.1, Fig. 3): the
 * magnification map convolved with a normalised Gaussian of sigma_px pixels
 * (taps at integer offsets up to 4 sigma, zero outside the map), sampled
 * bilinearly between pixel centres at n_samples equally spaced points of each
 * straight track, endpoints included.
 *  tracks: host, n_tracks x (x0, y0, x1, y1) in map pixel coordinates (pixel
 *          i spans [i, i+1)).
 *  out:    n_tracks x n_samples float32, device if out_is_device else host.
 * Errors: ML_ERR_INVALID_ARG (sigma_px <= 0 or > 64, counts < 1); ML_ERR_CUDA.
 */
ml_status ml_light_curves(ml_field *f, const double *tracks, int32_t n_tracks, int32_t n_samples,
                          double sigma_px, float *out, int32_t out_is_device, void *stream);

/*
 * ml_light_curves_noalloc - the light curves of ml_light_curves, computed
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory once they are
 * running, for example a process that reserved its whole memory budget at
 * start-up and runs close to it, or a timing-critical loop in which an
 * allocation's implicit device synchronisation or a possible out-of-memory
 * failure is unacceptable.  It calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch (the Gaussian taps and a device copy of the
 * tracks) lives in a fixed array inside the library, ML_NOALLOC_MAX_TRACKS
 * tracks (about 513 KB), which every device that loads the library holds
 * until the process exits.
 *  tracks:  host, n_tracks x (x0, y0, x1, y1) in map pixel coordinates.
 *  out:     DEVICE buffer of n_tracks x n_samples float32 (caller-owned).
 * The first call on each device looks up the array's device address.  All
 * calls share the one array: calls that overlap on the GPU (different
 * streams without ordering) race, so order them on one stream.  Nothing in
 * the array needs clearing: each call overwrites the part it uses.
 * Errors: ML_ERR_INVALID_ARG for n_tracks > ML_NOALLOC_MAX_TRACKS, counts < 1,
 * sigma_px outside (0, 16] or NULL pointers; ML_ERR_CUDA.
 */
#define ML_NOALLOC_MAX_TRACKS 16384
ml_status ml_light_curves_noalloc(ml_field *f, const double *tracks, int32_t n_tracks,
                                  int32_t n_samples, double sigma_px, float *out, void *stream);

/*
 * ml_trace_rays - source positions of single rays by exactly the arithmetic
 * the shooting kernel of the field's precision mode uses (for checking):
 * Eq. 9 in the near/far modes, Eq. 6 summed over all lenses in
 * ML_PREC_DIRECT64, and the pixel of Eq. 12's binning.
 *  ray_idx: device, n linear ray indices (each < n_rays_x * n_rays_y).
 *  beta:    device, n x 2 float64, source position in theta_E.
 *  pix:     device, n x 2 int32, the pixel the shooting kernel bins the ray
 *           into, (-1, -1) outside the map, (-2, -2) for a dropped ray,
 *           (-3, -3) with NaN beta for an index outside the lattice.
 * Errors: ML_ERR_INVALID_ARG; ML_ERR_CUDA.
 */
ml_status ml_trace_rays(ml_field *f, const int64_t *ray_idx, int64_t n, double *beta,
                        int32_t *pix, void *stream);

/*
 * ml_map_light_curves - the light curves of ml_light_curves (§4.1: Gaussian
 * source, taps at integer offsets |t| <= floor(4 sigma) normalised to 1,
 * bilinear sampling between pixel centres, n_samples equally spaced points
 * from (x0, y0) to (x1, y1) inclusive) evaluated on a caller's map.
 *  mu:     device, ny x nx float32 (any map: mu, or a dLoss-weighted map).
 *  tracks: host, n_tracks x (x0, y0, x1, y1) in map pixel coordinates.
 *  out:    device, n_tracks x n_samples float32.
 * Stream-ordered.  Errors: ML_ERR_INVALID_ARG (NULL, sizes, sigma outside
 * (0, 16], non-finite tracks); ML_ERR_CUDA.
 */
ml_status ml_map_light_curves(const float *mu, int32_t nx, int32_t ny, const double *tracks,
                              int32_t n_tracks, int32_t n_samples, double sigma_px, float *out,
                              void *stream);

/*
 * ml_map_light_curves_backward - the transpose of ml_map_light_curves: given
 * dL_dcurves (device, n_tracks x n_samples float32), writes dL_dmu (device,
 * ny x nx float32, overwritten) = sum over samples of the sample's gradient
 * times its bilinear and Gaussian weights (§4.1's light curves transposed; the
 * paper has no gradient).  With ml_cic_backward it gives the gradient of a
 * light-curve loss with respect to the lens field.
 * Stream-ordered; errors as ml_map_light_curves.
 */
ml_status ml_map_light_curves_backward(int32_t nx, int32_t ny, const double *tracks, int32_t n_tracks,
                                       int32_t n_samples, double sigma_px, const float *dL_dcurves,
                                       float *dL_dmu, void *stream);

/*
 * ml_cic_forward - the differentiable map: clears the field, shoots all its
 * rays and writes M = (S_I / S_S) * cloud-in-cell weights (Eq. 12 with
 * bilinear weights to the four nearest pixel centres) as float32.
 *  mu: device, map_ny x map_nx float32, 16-byte aligned; caller-owned.
 * Stream-ordered.  Errors: ML_ERR_STATE unless the field is ML_DEPOSIT_CIC
 * and ML_PREC_MIXED; ML_ERR_INVALID_ARG; ML_ERR_CUDA.
 */
ml_status ml_cic_forward(ml_field *f, float *mu, void *stream);

/*
 * ml_cic_backward - gradient of a loss of the cloud-in-cell magnification
 * map M = (S_I / S_S) * CIC weights (Eq. 12 with bilinear weights), given
 * G = dLoss/dM, with respect to every lens position and mass and to kappa,
 * gamma and kappa_* (the terms of Eq. 6).  Deflections are recomputed by the
 * forward's own arithmetic, not stored.  Near lenses take the exact
 * point-mass derivatives; far lenses act through the node series of Eq. 9,
 * so the result is the gradient of the forward as computed (it differs from
 * the derivative of the direct sum by the series truncation, far_bound).
 * The field must be ML_DEPOSIT_CIC and ML_PREC_MIXED.  Uses the field's task
 * counter: do not run it concurrently with ml_shoot_rays on the same field.
 *  dL_dM:       device, map_ny x map_nx float32.
 *  grad_lens:   device, n_lens x 3 float64 (d/dx_k, d/dy_k, d/dm_k) in the
 *               order the lenses were given; overwritten.
 *  grad_params: device, 3 float64 (d/dkappa, d/dgamma, d/dkappa_*); overwritten.
 * Errors: ML_ERR_STATE for other field modes; ML_ERR_INVALID_ARG; ML_ERR_CUDA.
 */
ml_status ml_cic_backward(ml_field *f, const float *dL_dM, double *grad_lens, double *grad_params,
                          void *stream);

/* Adjoint methods of ml_cic_backward_ex. */
enum {
    ML_ADJOINT_NEARFAR = 0, /* transpose of the near/far scheme (Eq. 9): near lenses pair by pair,
                               far lenses through moments of each level-2 node; the exact gradient
                               of the forward as computed.  Cost ~ rays (near + p) + nodes x lenses. */
    ML_ADJOINT_DIRECT = 1   /* every ray against every lens with the exact point-mass derivatives;
                               cost rays x lenses (a cross-check) */
};

/*
 * ml_cic_backward_ex - ml_cic_backward with a choice of method (above): Eq. 9
 * transposed, or Eq. 6 differentiated lens by lens.
 * ml_cic_backward is ml_cic_backward_ex(..., ML_ADJOINT_NEARFAR, ...).
 * The near/far method allocates its scratch (3 doubles per lens and
 * 2 (p + 1) doubles per level-2 node) stream-ordered and frees it before
 * returning.  Errors as ml_cic_backward, and ML_ERR_INVALID_ARG for an
 * unknown method.
 */
ml_status ml_cic_backward_ex(ml_field *f, const float *dL_dM, double *grad_lens, double *grad_params,
                             int32_t method, void *stream);

/*
 * ml_field_set_counts - replace the field's integer count map (NGP fields)
 * with `counts` (map_ny x map_nx uint32, device or host), stream-ordered.
 * Rays are independent (§3.2 Level 3), so a map's counts are the sum of the
 * counts of any partition of its rays.
 * For a map shot in shards on several GPUs: each GPU shoots its ray range,
 * the count maps are summed (integer addition, exact), and the sum is set
 * back before ml_magnification_map and ml_light_curves.  The counters
 * (ml_field_stats) are left as they are; the new map's sum becomes the base
 * of the wrap-around check.  Synchronises `stream`.  Errors: ML_ERR_STATE for
 * a CIC field; ML_ERR_INVALID_ARG; ML_ERR_CUDA.
 */
ml_status ml_field_set_counts(ml_field *f, const uint32_t *counts, int32_t in_is_device, void *stream);

/* Light-curve directions of ml_find_peaks. */
enum { ML_ALONG_X = 0, ML_ALONG_Y = 1 };

/*
 * ml_find_peaks - peak identification of §4.2 on the field's count map.
 * Light curves run along x (each map row is a curve; the neighbouring curves
 * are the rows above and below) or along y.  Step 1: position j of curve i
 * is a candidate when N_ij > N_i,j-1 and N_ij > N_i,j+1 and
 * h = N_ij - <N> > nsigma sqrt(<N>), <N> the mean of the three, tested as
 * (2N - a - b)^2 > 3 nsigma^2 (a + N + b) in FP64 (exact for counts below
 * 2^26); curve ends are never candidates.  Step 2: a candidate is a true peak
 * when a candidate lies among positions j-1, j, j+1 of both neighbouring
 * curves; the first and last curves have none.  The paper uses nsigma = 5.
 *  mask:     device, 4-byte aligned, map_ny x map_nx bytes + 4 bytes of
 *            padding; bit 0 candidate, bit 1 true peak; NULL to use internal
 *            scratch.
 *  peaks:    device, capacity x (ix, iy) int32 pairs of true peaks, in no
 *            particular order; may be NULL when capacity is 0.
 *  n_found:  host; the number of true peaks (may exceed capacity).
 * Synchronises `stream`.  Errors: ML_ERR_STATE for a CIC field;
 * ML_ERR_INVALID_ARG; ML_ERR_CUDA.
 */
ml_status ml_find_peaks(ml_field *f, int32_t along, double nsigma, uint8_t *mask, int32_t *peaks,
                        int64_t capacity, int64_t *n_found, void *stream);

/* Largest number of distance bins of ml_peak_statistics. */
#define ML_PEAK_STATS_MAX_BINS 2048

/*
 * ml_peak_statistics - the statistics of §4.2 (Figs. 4 and 5): the true peaks
 * of the field's count map, binned by the distance of the source from the
 * macro caustic, taken as a straight line across the curves (a local region
 * of the critical curve, §2).  Position j along a curve has the distance
 * d = |origin + (j + 1/2) step - caustic| of its pixel centre (origin, step:
 * map_x0, dpx for ML_ALONG_X; map_y0, dpy for ML_ALONG_Y), each operation
 * rounded separately in FP64; bin b holds edges[b] <= d < edges[b+1].  For
 * the fold model (Eq. 5) the caustic is beta_x = 0 to within
 * (d_y theta_y)^2 / (2 d_x).
 *  along:       the curve direction, as in ml_find_peaks.
 *  nsigma:      the peak threshold, used only when mask is NULL.
 *  mask:        device, the mask of ml_find_peaks for the same direction on
 *               the current map (read only); NULL to identify the peaks here
 *               first, in scratch memory.
 *  caustic:     the caustic's coordinate along the curves.
 *  edges:       host, nbins + 1 finite, strictly ascending distances.
 *  nbins:       1 .. ML_PEAK_STATS_MAX_BINS.
 *  n_peaks:     host, nbins: true peaks per bin.
 *  sum_counts:  host, nbins: the sum of N_ij over those peaks; the mean peak
 *               magnification is sum_counts S_I/S_S / n_peaks (Eq. 12).
 *  n_positions: host, nbins: the positions per bin where a true peak can
 *               occur (curves other than the first and last, positions other
 *               than the two ends); crossings per unit length of curve are
 *               n_peaks / (n_positions step).
 * Integer sums, so the result does not depend on the order of the work.
 * Synchronises `stream`.  Errors: ML_ERR_STATE for a CIC field;
 * ML_ERR_INVALID_ARG (NULL pointers, nbins out of range, edges not finite
 * and strictly ascending, a caustic not finite, nsigma <= 0 without a mask);
 * ML_ERR_CUDA.
 */
ml_status ml_peak_statistics(ml_field *f, int32_t along, double nsigma, const uint8_t *mask,
                             double caustic, const double *edges, int32_t nbins, uint64_t *n_peaks,
                             uint64_t *sum_counts, uint64_t *n_positions, void *stream);

/*
 * ml_field_clear - zero the map and the counters (stream-ordered).
 * Bookkeeping; no counterpart in the paper.
 */
ml_status ml_field_clear(ml_field *f, void *stream);

/*
 * ml_field_stats - synchronise `stream` and copy the field's counters
 * (ML_STAT_* indices) into out[ML_STAT_COUNT] (host).  For a uint32 count map it also
 * sums the map in 64 bits (one pass over the map): a pixel that wrapped
 * makes that sum fall short of the in-map ray count, which sets flag bit 0.
 * Returns ML_ERR_OVERFLOW or ML_ERR_ABORTED when the corresponding flag is
 * set, after filling out.  The counts check ray conservation (every lattice
 * ray of §3.2 Level 3 is in the map, out of it or dropped).
 */
ml_status ml_field_stats(ml_field *f, uint64_t out[ML_STAT_COUNT], void *stream);

/* ml_field_info - copy the derived parameters (§3.1-§3.2: ray rectangle,
 * lattice, level grids, Taylor order, S_I/S_S of Eq. 12) into *out (host). */
ml_status ml_field_info(const ml_field *f, ml_field_params *out);

/*
 * ml_field_abort - raise (on != 0) or lower the field's abort flag.  It lives
 * in mapped host memory; running shooting kernels read it between warp tasks
 * and stop early, leaving a valid partial map and setting the aborted flag.
 * Bookkeeping; no counterpart in the paper.
 */
ml_status ml_field_abort(ml_field *f, int32_t on);

/* ml_field_destroy - free the field and its device memory.  NULL is a no-op.
 * The library takes device memory from a stream-ordered pool of its own per
 * device, which keeps freed memory for the next fields (creating a field
 * then reuses its predecessor's buffers instead of mapping new ones); the
 * pool's memory is returned when the process exits.
 * Bookkeeping; no counterpart in the paper. */
ml_status ml_field_destroy(ml_field *f);

/*
 * Batched maps (many heterogeneous magnification maps in one CUDA graph of
 * persistent launches; the paper's statistics use 80 maps and 800 light
 * curves, §4.2).
 *
 * ml_batch_create - create n fields from descs[0..n) (ML_PREC_MIXED and
 * ML_DEPOSIT_NGP only).  Each field's Taylor order is planned from its own
 * truncation bound; a field with tune != 0 (and no level-2 subdivision given)
 * first takes the grid the autotuner's cost model ranks first for it (the
 * model alone: timing every map's candidates would cost more than it saves).
 * Maps of one compiled order share one persistent launch.  With
 * tracks_per_map > 0, `tracks` (host, n x tracks_per_map x 4, map pixel
 * coordinates) are kept on the device for the light curves of each run.
 * Synchronises `stream`.  Errors as ml_field_create, plus ML_ERR_UNSUPPORTED
 * for other modes.
 */
typedef struct ml_batch ml_batch;
ml_status ml_batch_create(const ml_field_desc *descs, int32_t n, int32_t tracks_per_map,
                          const double *tracks, int32_t n_samples, double sigma_px, void *stream,
                          ml_batch **out);

/*
 * ml_batch_run - one step of the whole batch, ordered on `stream`: zero all
 * maps and counters, shoot every ray of every map with one persistent kernel
 * launch per Taylor order present (its warps take tasks of all its maps from
 * one queue), convert every map to
 * mu (Eq. 12) into the batch's buffers and compute the light curves.  With
 * use_graph != 0 the step is captured once into a CUDA graph on the batch's
 * internal stream and replayed by every later call.
 */
ml_status ml_batch_run(ml_batch *b, int32_t use_graph, void *stream);

/* ml_batch_field - borrowed handle of map i (owned by the batch: do not
 * destroy it); usable with ml_field_stats, ml_field_info, ml_trace_rays,
 * ml_magnification_map, ml_light_curves.  Bookkeeping; no counterpart in the
 * paper. */
ml_status ml_batch_field(ml_batch *b, int32_t i, ml_field **out);

/* ml_batch_mu - copy map i's mu (Eq. 12, float32, from the last run) into
 * out (device or host memory; host output synchronises `stream`). */
ml_status ml_batch_mu(ml_batch *b, int32_t i, float *out, int32_t out_is_device, void *stream);

/* ml_batch_curves - copy all light curves (§4.1) of the last run, n x
 * tracks_per_map x n_samples float32, into out (device or host). */
ml_status ml_batch_curves(ml_batch *b, float *out, int32_t out_is_device, void *stream);

/* ml_batch_abort - raise or lower the batch's abort flag (see ml_field_abort).
 * Bookkeeping; no counterpart in the paper. */
ml_status ml_batch_abort(ml_batch *b, int32_t on);

/* ml_batch_destroy - free the batch and its fields.  NULL is a no-op.
 * Bookkeeping; no counterpart in the paper. */
ml_status ml_batch_destroy(ml_batch *b);

/* Message of the last failed call on this thread ("" if none).  Bookkeeping;
 * no counterpart in the paper. */
const char *ml_last_error(void);

/*
 * ml_fp32_fma_peak - one launch of an FP32 fused multiply-add throughput
 * probe, the measured denominator of the shooting kernels' roofline.  The
 * paper has no counterpart: it is a measurement helper.  SMs x blocks_per_sm
 * blocks of 256 threads each run eight independent chains of `iters` FMAs
 * (a <- a b + c), as scalar FFMA (two_lane = 0) or as the two-lane
 * fma.rn.f32x2 instruction (two_lane = 1, two FMAs per instruction).
 *  sink:  device, >= 8 x SMs floats; written only if a chain reached an
 *         impossible value (keeps the chains from being optimised away).
 *  flop:  host, receives the launch's flop count (2 per FMA).
 * The caller times the launch on `stream` (CUDA events) and divides.
 * Errors: ML_ERR_INVALID_ARG (NULL, blocks_per_sm outside [1, 8], iters
 * outside [1, 2^32]); ML_ERR_CUDA.
 */
ml_status ml_fp32_fma_peak(int32_t two_lane, int32_t blocks_per_sm, int64_t iters, float *sink,
                           double *flop, void *stream);

/* ABI version the library was built with (ML_ABI_VERSION).  Bookkeeping; no
 * counterpart in the paper. */
int32_t ml_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ML_H */
