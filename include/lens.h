/*
 * lens.h -- C ABI of liblens.so: GB300 (sm_103a) FMM-IPM microlensing hot path.
 *
 * Method: Jimenez-Vicente & Mediavilla (2022), "Fast Multipole Method for
 * Gravitational Lensing. Application to High Magnification Quasar
 * Microlensing".  The library evaluates the lens equation (Eq. 1)
 *
 *     y = diag(1 - kappa_s - gamma, 1 - kappa_s + gamma) x
 *         - sum_i m_i (x - x_i) / |x - x_i|^2
 *
 * (point lenses in Einstein units; smooth convergence kappa_s and shear
 * gamma as allowed by the footnote to Eq. 1, shear along x1) at many rays
 * with a Fast Multipole Method (Sec. 2.1 and Appendix A: quadtree, P2M, M2M,
 * M2L, L2L, L2P, P2P), and turns a grid of deflected cells into a
 * magnification map by first-order Inverse Polygon Mapping (Sec. 2.3 and the
 * five-step FMM-IPM algorithm of Sec. 2.4, including its ray chunking).
 *
 * Conventions shared by every call
 *   - Every pointer marked "dev" is CUDA device memory on the current device;
 *     "host" pointers are ordinary host memory.  All floating-point arrays are
 *     float64, C-contiguous.  Positions are interleaved pairs (x1, x2).
 *   - The caller owns every buffer it passes.  A plan owns its internal
 *     arrays, which it obtains from the caller's lens_allocator (or, when the
 *     allocator pointer is NULL, from a stream-ordered memory pool the library
 *     keeps per device, which retains up to 16 GiB of freed blocks for reuse)
 *     and frees in lens_plan_destroy.
 *   - Every call returns a lens_status; on error the outputs are undefined
 *     and lens_last_error() gives a message (thread-local).  No call aborts
 *     or throws across the ABI.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it unless noted.
 *   - A star exactly at a ray contributes nothing to that ray.
 *   - Environment LENS_FAULT=alloc@K or launch@K makes the K-th internal
 *     allocation or kernel launch of the process fail with
 *     LENS_EFAULT_INJECTED (host-side fault injection for tests).
 */
#ifndef LENS_H
#define LENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lens_plan lens_plan; /* opaque: star tree + expansions */

typedef enum {
  LENS_OK = 0,
  LENS_EINVAL = 1,          /* bad argument (size, order, non-finite input) */
  LENS_ENOMEM = 2,          /* an allocation failed */
  LENS_ECUDA = 3,           /* a CUDA runtime call or launch failed */
  LENS_EDEPTH = 4,          /* tree needs more levels than max_depth allows */
  LENS_EDOMAIN = 5,         /* a ray lies outside the plan's target region */
  LENS_ETIMEOUT = 6,        /* a bounded device wait expired */
  LENS_EFAULT_INJECTED = 7  /* LENS_FAULT fault injection fired */
} lens_status;

/* Device-memory provider for plan internals.  alloc returns a device pointer
 * (NULL on failure) usable on `stream`; free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} lens_allocator;

typedef enum {
  LENS_FP64 = 0,      /* every step in float64 */
  LENS_FP32_BULK = 1  /* P2P / L2P / M2P in float32 with compensated sums,
                         near-field offsets as float-float (pairs of float32)
                         from each leaf's centre; P2M accumulated in float32
                         (each star's scaled offset formed in float64);
                         M2M, M2L, L2L and P2L in float64.  The lens
                         equation is the float64 value at the leaf centre
                         (a c1 - Re b0, b c2 + Im b0) plus the ray's part
                         a dx - Re f - near formed in float-float (~48-bit
                         significand): within a few float32 ulps of the
                         deflection, not float64 */
} lens_precision;

typedef struct {
  int p;               /* expansion order (Appendix A: error ~ (ratio)^p), 1..64 */
  int leaf_size;       /* a box is split while it holds more stars, 1..1024 */
  int prec;            /* lens_precision */
  int max_depth;       /* quadtree depth cap, 0 = default (28), at most 28 */
  int has_target_box;  /* 1: target_box below is valid */
  double target_box[4];/* [x1_min, x1_max, x2_min, x2_max]: region of the rays
                          (local expansions are formed only for boxes that meet
                          it); 0 = the whole root box */
} lens_build_opts;

/* Image-plane cell grid (Sec. 2.4, step 2): cell (i, j) is
 * [x0 + i h, x0 + (i+1) h) x [y0 + j h, y0 + (j+1) h), i < nx, j < ny.
 * Its corner rays are x = x0 + i h, y = y0 + j h for i <= nx, j <= ny. */
typedef struct {
  double x0, y0, h;
  int64_t nx, ny;
} lens_grid;

/* Source-plane map window: [u0, u1) x [v0, v1) covered by npx x npy pixels;
 * pixel (px, py) is map[py * npx + px]. */
typedef struct {
  double u0, u1, v0, v1;
} lens_box;

/* Flux ledger of one map (areas in image-plane units, Einstein radius^2):
 * area_in_map + area_outside + area_dropped + area_degenerate = area_total. */
typedef struct {
  double cells, area_total, area_in_map, area_outside, area_dropped,
      area_degenerate, cells_dropped, cells_degenerate;
  int64_t chunks;      /* grid chunks processed (Sec. 2.4, step 2) */
  double ms_deflect;   /* stream time of the deflection phase (all chunks) */
  double ms_ipm;       /* stream time of the IPM phase (all chunks) */
  /* algorithmic work and kernel-only device time (CUDA events around the
   * launches of the fused L2P+P2P+M2P kernel and of the IPM kernels) */
  double rays;         /* corner rays deflected (chunk seams counted twice) */
  double p2p_pairs;    /* ray-star pairs summed directly (U lists) */
  double m2p_evals;    /* ray-box multipole evaluations (W lists) */
  double ipm_updates;  /* (cell, pixel) map increments */
  double cells_queued; /* cells sent to the warp-per-cell path */
  double cells_ext;    /* of those, ill-conditioned cells redone in float-float (~48 bits) */
  double ms_eval_kernel;
  double ms_ipm_kernel;
  int64_t launches;    /* kernels this call launched */
  double cells_refined; /* (sub)cells over the cap split 2 x 2 (lens_ipm_map_refined) */
  int64_t fused;        /* 1: the fused deflection + IPM kernel ran (lens_ipm_map_ex) */
  double ms_fused_kernel; /* device time of the fused kernel (all chunks) */
  double rays_evaluated;  /* corner evaluations, including the corners that the
                             fused kernel's overlapping work items share */
} lens_ipm_stats;

typedef struct {
  int64_t n_stars, n_boxes, n_leaves, n_active_boxes, n_active_leaves;
  int64_t n_v, n_x, n_u, n_w;  /* interaction-list entries (active boxes) */
  int64_t u_stars;             /* sum over active leaves of stars in U lists */
  int levels, p, leaf_size, prec;
  double root_lo[2], root_size;
  int64_t device_bytes;        /* plan-owned device memory */
  double ms_build;             /* device time of the build, tree to expansions */
  int64_t build_launches;      /* kernels the build launched */
  double ms_tree;              /* of ms_build: boxes and interaction lists */
  double ms_far_local;         /* device time of the far-field launch (M2L over the
                                  V lists and P2L over the X lists, all levels) */
} lens_plan_info;

/* ---- FMM plan ------------------------------------------------------------
 * Builds the quadtree over the stars (Appendix A, step 1: Morton keys, radix
 * sort, adaptive split of boxes holding more than leaf_size stars; empty
 * quadrants stay as leaves so leaves tile the root), the upward pass (P2M,
 * M2M: Appendix A steps 2-3) and the downward pass (M2L over interaction
 * lists, L2L, plus the adaptive P2L lists: Appendix A steps 4-5) for every
 * box that meets the target region.
 *   stars_xy: dev, n x 2; masses: dev, n (any real values); n >= 1.
 *   kappa_s, gamma: smooth field (footnote to Eq. 1).
 *   opts: host; allocator: host or NULL (the library's stream-ordered pool on
 *   `stream`, one per device, which keeps up to 16 GiB of freed blocks for
 *   reuse).
 *   *out receives the plan.  Synchronises `stream` a few times (tree and
 *   list sizes).  The tree and lists are formed on `stream`; the expansions
 *   then run on a high-priority stream owned by the plan, and the call
 *   returns without waiting for them: every later call with this plan, on
 *   any stream, waits for the part it reads (evaluations for the
 *   expansions, the adjoint for the tree alone), and lens_plan_info_get and
 *   lens_plan_destroy wait for all of it.
 * Errors: EINVAL (n < 1, p outside 1..64, leaf_size outside 1..1024,
 * non-finite star or mass, bad target box), ENOMEM, ECUDA, EDEPTH. */
lens_status lens_fmm_build(const double* stars_xy, const double* masses,
                           int64_t n, double kappa_s, double gamma,
                           const lens_build_opts* opts,
                           const lens_allocator* allocator, void* stream,
                           lens_plan** out);

/* Eq. 1 at m arbitrary rays (Sec. 2.1, item 3: targets need not lie on a
 * grid): L2P + P2P (+ M2P for the adaptive W lists), then y.
 *   rays_xy: dev m x 2; y_out: dev m x 2; jac_out: dev m x 4 (row-major
 *   dy/dx) or NULL.  Rays must lie in the plan's target region (EDOMAIN
 *   otherwise; reported after a stream synchronisation).  m = 0 is a no-op. */
lens_status lens_deflect(lens_plan* plan, const double* rays_xy, int64_t m,
                         double* y_out, double* jac_out, void* stream);

/* Lensing potential psi(x) = sum_i m_i ln|x - x_i| + kappa_s |x|^2 / 2 +
 * gamma (x1^2 - x2^2) / 2 at m rays (dev m x 2, inside the plan's target
 * region), whose gradient is x - y of Eq. 1 (the potential of the
 * cosmological-lens example, Sec. 2.5).  Through the plan's expansions: the
 * field's multipole and local coefficients integrated once (Appendix A's
 * expansions of the complex logarithm) plus one real constant per box,
 * float64 throughout whatever the plan's precision (a float32-bulk plan's
 * multipoles carry float32 P2M sums).  A star exactly at a ray contributes
 * nothing.  psi_out: dev m.  Synchronises `stream`.  LENS_EDOMAIN for a
 * ray outside the target region or not finite. */
lens_status lens_potential(lens_plan* plan, const double* rays_xy, int64_t m,
                           double* psi_out, void* stream);

/* Eq. 1 at the corner rays of grid rows row0 .. row0+nrows-1 (corner rows,
 * 0 <= row0, row0 + nrows <= ny + 1), all columns 0..nx.
 *   y_out: dev nrows x (nx+1) x 2 (row-major); jac_out: dev
 *   nrows x (nx+1) x 4 or NULL.  No ray array is materialised. */
lens_status lens_deflect_grid(lens_plan* plan, const lens_grid* grid,
                              int64_t row0, int64_t nrows, double* y_out,
                              double* jac_out, void* stream);

/* FMM-IPM magnification map (Sec. 2.4 steps 2-4): the grid is split into row
 * chunks of at most max_cells_per_chunk cells (0 = sized from free device
 * memory; never more than 64 cells per map pixel or 2^30 cells, after which
 * the float32 accumulators are flushed into a running float-float sum); each
 * chunk's corner rays
 * are deflected and each cell's mapped
 * quadrilateral is apportioned over the pixels it overlaps (signed-area
 * fraction, Sec. 2.3), accumulating
 *     map[pix] = sum_cells h^2 * a_pix / A_P / S*     (S* = pixel area).
 * Cells whose pixel bounding box spans more than bbox_cap_px pixels on a side
 * are dropped and booked in the ledger (bbox_cap_px = 0: no cap).
 *   map_out: dev npy x npx (overwritten; between chunks it holds the running
 *   sum as float pairs, so its contents are the map only once the call has
 *   returned LENS_OK); stats: host or NULL.
 * Synchronises `stream` at the end. */
lens_status lens_ipm_map(lens_plan* plan, const lens_grid* grid,
                         const lens_box* box, int npx, int npy,
                         int64_t max_cells_per_chunk, int bbox_cap_px,
                         double* map_out, lens_ipm_stats* stats, void* stream);

/* lens_ipm_map with critical-cell refinement instead of the drop rule: a cell
 * whose pixel box spans more than bbox_cap_px pixels on a side (or has a
 * corner beyond 2^30 pixels) is split into 2 x 2 sub-cells of half the side,
 * the new corner rays deflected through the plan like lens_deflect, each
 * sub-cell carrying a quarter of the area; up to refine_levels times, after
 * which a sub-cell still over the cap is dropped and booked as before.
 * (Sec. 2.3 leaves such cells to the higher-order IPM; this is the adaptive
 * step toward it.)  refine_levels 0..16 (0: lens_ipm_map); needs
 * bbox_cap_px > 0.  stats->cells_refined counts the cells split.  The ledger
 * keeps its areas in image-plane units (a sub-cell of level l counts 4^-l
 * cells), the cell counts count sub-cells as cells.
 * Errors: as lens_ipm_map; EDOMAIN if the grid leaves the target region. */
lens_status lens_ipm_map_refined(lens_plan* plan, const lens_grid* grid,
                                 const lens_box* box, int npx, int npy,
                                 int64_t max_cells_per_chunk, int bbox_cap_px,
                                 int refine_levels, double* map_out,
                                 lens_ipm_stats* stats, void* stream);

/* ---- several lens planes (Sec. 1: ray tracing through several lens planes
 * repeats the mapping plane by plane; footnote to the thin-lens
 * approximation: a 3D lens as a collection of thin planes) ---------------
 * Plane i (in order of distance from the observer) holds n point lenses and
 * a smooth field, each deflection scaled to the source plane as in Eq. 1:
 *     alpha_i(x) = sum_k m_ik (x - x_ik) / |x - x_ik|^2
 *                  + diag(kappa_s + gamma, kappa_s - gamma) x.
 * A ray entering at x_1 reaches plane j at
 *     x_j = x_1 - sum_{i<j} beta[i K + j] alpha_i(x_i)
 * and the source plane at y = x_1 - sum_i alpha_i(x_i); beta[i K + j]
 * (i < j) is the distance ratio D_ij D_s / (D_j D_is) of the pair (other
 * entries are not read).  With one plane this is Eq. 1. */
typedef struct {
  const double* stars_xy;  /* dev n x 2 (may be NULL when n = 0) */
  const double* masses;    /* dev n */
  int64_t n;               /* >= 0 */
  double kappa_s, gamma;   /* the plane's smooth field */
} lens_plane;

/* y at m rays (dev m x 2) through nplanes planes (1..64, host array of
 * lens_plane; beta: host nplanes x nplanes, row-major).  Per plane an FMM
 * plan is built over its stars (opts: p, leaf_size, prec, max_depth; the
 * target region is the bounding box of the rays' positions on that plane),
 * the rays are deflected through it as by lens_deflect, and one kernel moves
 * them on to the next plane.  y_out: dev m x 2; x_planes_out: dev
 * nplanes x m x 2 (the positions x_i at each plane) or NULL.  Scratch and
 * plans from allocator (may be NULL: the library's pool).  Synchronises
 * `stream` once per plane.  Errors: EINVAL (bad sizes, NULL buffers,
 * non-finite kappa_s, gamma or beta), EDOMAIN (a position that is not
 * finite), and those of lens_fmm_build. */
lens_status lens_multiplane_deflect(const lens_plane* planes, int nplanes,
                                    const double* beta,
                                    const lens_build_opts* opts,
                                    const double* rays_xy, int64_t m,
                                    double* y_out, double* x_planes_out,
                                    const lens_allocator* allocator,
                                    void* stream);

/* FMM-IPM magnification map through several planes: the chunk loop of
 * lens_ipm_map (Sec. 2.4 steps 2-4) with each chunk's corner rays traced
 * through every plane as by lens_multiplane_deflect (plans built per chunk
 * and plane), then apportioned to the map by the same first-order IPM.
 * Arguments as lens_ipm_map (map_out overwritten; stats: host or NULL, its
 * rays counting corner rays deflected by planes with stars) plus the planes,
 * beta, opts and allocator of lens_multiplane_deflect.  Synchronises
 * `stream`. */
lens_status lens_multiplane_ipm_map(const lens_plane* planes, int nplanes,
                                    const double* beta,
                                    const lens_build_opts* opts,
                                    const lens_grid* grid, const lens_box* box,
                                    int npx, int npy,
                                    int64_t max_cells_per_chunk,
                                    int bbox_cap_px, double* map_out,
                                    lens_ipm_stats* stats,
                                    const lens_allocator* allocator,
                                    void* stream);

/* lens_ipm_map_refined with a choice of kernels (flags):
 *   LENS_MAP_SEPARATE -- the deflection kernel writes every corner of a chunk
 *     to device memory as pixel coordinates, then the IPM kernels read them;
 *   LENS_MAP_FUSED -- float32-bulk plans only: one kernel deflects the
 *     corners of a rectangle of one leaf's grid rays (the leaf's expansions
 *     and near stars staged once) into shared memory and apportions every
 *     cell whose four corners lie in the rectangle (Sec. 2.4 steps 3 and 4
 *     with no corner round trip); rectangles of one leaf overlap by one row or
 *     column of corners, which both evaluate from the same leaf data to the
 *     same bits, so each cell's polygon is the one the separate path forms;
 *     only corners on leaf boundaries are written out, for the cells that
 *     straddle two leaves, mapped afterwards;
 *   0 -- the library's default for the plan.
 * The two paths give the same map up to the order of the float32 additions.
 * stats->fused tells which ran. */
#define LENS_MAP_FUSED 1u
#define LENS_MAP_SEPARATE 2u
lens_status lens_ipm_map_ex(lens_plan* plan, const lens_grid* grid,
                            const lens_box* box, int npx, int npy,
                            int64_t max_cells_per_chunk, int bbox_cap_px,
                            int refine_levels, unsigned flags, double* map_out,
                            lens_ipm_stats* stats, void* stream);

/* Adjoint of lens_deflect (not in the paper): given grad_y = dL/dy at the m
 * rays, the transposed FMM (L2P^T, L2L^T, M2L^T, M2M^T, P2M^T, P2P^T, M2P^T,
 * P2L^T on the same tree) gives
 *   grad_xy: dev n x 2 = dL/dx_i (caller's star order),
 *   grad_m:  dev n     = dL/dm_i,
 *   grad_kg: dev 2     = dL/dkappa_s, dL/dgamma.
 * Any output pointer may be NULL. */
lens_status lens_deflect_adjoint(lens_plan* plan, const double* rays_xy,
                                 int64_t m, const double* grad_y,
                                 double* grad_xy, double* grad_m,
                                 double* grad_kg, void* stream);

/* Tree and list statistics of a plan (host struct). */
lens_status lens_plan_info_get(const lens_plan* plan, lens_plan_info* info);

void lens_plan_destroy(lens_plan* plan);

/* ---- Direct sum ----------------------------------------------------------
 * Eq. 1 by O(N* x N_x) direct summation on the GPU (Sec. 2.1): the baseline
 * the FMM is measured against.  prec = LENS_FP64 or LENS_FP32_BULK
 * (float32 pair terms on split hi/lo coordinates with compensated partial
 * sums).  Buffers as in lens_deflect; scratch from allocator (may be NULL). */
lens_status lens_direct_deflect(const double* stars_xy, const double* masses,
                                int64_t n, double kappa_s, double gamma,
                                const double* rays_xy, int64_t m, int prec,
                                double* y_out, double* jac_out,
                                const lens_allocator* allocator, void* stream);

/* ---- Direct sum without allocation ----------------------------------------
 * The paper has no counterpart: this is a service for callers that may not
 * allocate device memory (a host application that owns the whole device
 * memory budget and passes the library only its inputs and outputs, a
 * memory-capped service whose pool must not grow, a loop that cannot let an
 * allocation stall or fail mid-step).  Same result as lens_direct_deflect
 * with prec = LENS_FP32_BULK; its scratch (n split stars) lives in one fixed
 * static device array of 262144 stars (5 MiB) that every GPU loading the
 * library holds until exit.  Rules:
 *   - n <= 262144, else LENS_EINVAL before any launch;
 *   - the first call on a device looks up the array's address (with that
 *     device current) and caches it; make that first call before any stream
 *     capture;
 *   - calls share the one array: two calls that overlap on the GPU (other
 *     streams, other host threads) race, so the caller must order them; each
 *     call rewrites all scratch it reads, nothing has to start at zero;
 *   - no cudaMalloc, cudaFree or allocating library call is made.
 * Buffers as in lens_direct_deflect (dev pointers; jac_out may be NULL). */
lens_status lens_direct_deflect_noalloc(const double* stars_xy,
                                        const double* masses, int64_t n,
                                        double kappa_s, double gamma,
                                        const double* rays_xy, int64_t m,
                                        double* y_out, double* jac_out,
                                        void* stream);

/* ---- Gaussian-source light curve (differentiable loss) --------------------
 * F_k = sum_r w_ray exp(-|y_r - s_k|^2 / (2 sigma^2)) / (2 pi sigma^2) for
 * |y_r - s_k| <= trunc sigma: the magnification of a Gaussian source (Sec.
 * 2.5) at the ns samples of a track (light curves: Sec. 3.3).
 *   y: dev m x 2 mapped rays; samples: dev ns x 2; F_out: dev ns. */
lens_status lens_light_curve(const double* y, int64_t m, double w_ray,
                             const double* samples, int64_t ns, double sigma,
                             double trunc, double* F_out, void* stream);

/* dL/dy for L = sum_k (F_k - T_k)^2: F, T dev ns; grad_y_out dev m x 2. */
lens_status lens_light_curve_grad(const double* y, int64_t m, double w_ray,
                                  const double* samples, int64_t ns,
                                  double sigma, double trunc, const double* F,
                                  const double* T, double* grad_y_out,
                                  void* stream);

/* ---- consumers of a magnification map (Sec. 3: magnification histograms of
 * finite sources, light curves along source tracks).  map: dev npy x npx,
 * row-major as lens_ipm_map writes it. */

/* The map seen by a circular Gaussian source of sigma_px pixels (Sec. 3:
 * magnification of sources of a given size): the map convolved with
 * exp(-|d|^2 / 2 sigma^2) over the pixel offsets d with |d| <= trunc sigma_px
 * (the profile cut at an isophote; floor(trunc sigma_px) <= 1024), each output
 * pixel renormalised to the part of that disk inside the map.  out: dev
 * npy x npx (may not alias map).  Scratch from allocator (may be NULL: the
 * library's pool).  Synchronises `stream`. */
lens_status lens_map_source(const double* map, int npx, int npy, double sigma_px,
                            double trunc, double* out,
                            const lens_allocator* allocator, void* stream);

/* Histogram of n values (dev) into nbins equal bins of [lo, hi), of
 * log10(value) when log_bins != 0 (values <= 0 then count as below).
 * counts: dev int64[nbins + 2]: [0] below lo, [1..nbins] the bins,
 * [nbins + 1] at or above hi.  nbins 1..8192. */
lens_status lens_map_histogram(const double* values, int64_t n, double lo,
                               double hi, int nbins, int log_bins,
                               int64_t* counts, void* stream);

/* The map at ns source positions (dev ns x 2, source-plane coordinates of
 * the map window box): bilinear between pixel centres, clamped to the
 * outermost centres.  out: dev ns. */
lens_status lens_map_track(const double* map, int npx, int npy,
                           const lens_box* box, const double* positions,
                           int64_t ns, double* out, void* stream);

/* ---- images on a deflected ray grid (Sec. 2.5: the images of a background
 * Gaussian source behind a simulated halo, from a regular grid of deflected
 * rays).  y: dev (ny+1) x (nx+1) x 2, the corner positions in the source
 * plane as lens_deflect_grid writes them for `grid`. */

/* Images of the point source (beta1, beta2).  Cell (i, j) is an image cell
 * when beta lies in the bounding box of its deflected corners and their
 * closed polygon (i,j) -> (i+1,j) -> (i+1,j+1) -> (i,j+1) winds around it:
 * an edge a -> b adds +1 when a_2 <= beta_2 < b_2 and beta is left of it, -1
 * when b_2 <= beta_2 < a_2 and beta is right of it, the orientation
 * (b - a) x (beta - a) taken in rounded float64 without contraction (a
 * source on an edge shared by two cells is claimed by one of them, the same
 * one on any machine).  In an image cell the bilinear interpolation of the
 * corners is inverted by 20 Newton steps from the cell centre (cell
 * coordinates kept within [-1, 2]): the image is that point, its signed
 * magnification h^2 / det J of the bilinear map there (INFINITY if det J
 * is 0).  A cell holding a point mass reports that mass's infinitely
 * demagnified image (|mu| ~ 0).
 * out: dev max_out x 3 (x1, x2, mu); cells: dev int64 max_out (j * nx + i);
 * both in no particular order and may be NULL when max_out is 0.
 * n_found: host, the number of image cells; entries past max_out are not
 * written (call again with a larger buffer).  Scratch from the library's
 * pool.  Synchronises `stream`. */
lens_status lens_find_images(const double* y, const lens_grid* grid,
                             double beta1, double beta2, int64_t max_out,
                             double* out, int64_t* cells, int64_t* n_found,
                             void* stream);

/* The lensed image of a Gaussian source: out[r] = exp(-|y_r - beta|^2 /
 * (2 sigma^2)), the source's peak-normalised surface brightness at each of m
 * rays (dev m x 2); out: dev m. */
lens_status lens_source_image(const double* y, int64_t m, double beta1,
                              double beta2, double sigma, double* out,
                              void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* lens_last_error(void);

/* Library version string. */
const char* lens_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LENS_H */
