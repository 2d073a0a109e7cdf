/*
 * amrmg.h -- C ABI of the GB300 AMR multigrid Poisson solve for
 * electrostatic particle-in-cell (Frey, Adelmann & Locans, arXiv 1812.03689).
 *
 * The library solves, on the unit cube with homogeneous Dirichlet faces or
 * the Robin faces that approximate an open boundary (Eq. robin_bc),
 *     L^comp phi = -rho / eps0      on the composite domain  (Sec. 5.3)
 * over a block-structured, cell-centred, ratio-2 refinement hierarchy
 * (Sec. 3, Eq. mesh_spacing: h_l = 1 / (n0 * 2^l)), by residual-correction
 * AMR V-cycles (Alg. 1-3) with red-black Gauss-Seidel smoothing,
 * flux matching at coarse-fine faces (Eq. flux_differencing) and two-step
 * quadratic Lagrange ghost interpolation (Eq. 2d_lagrange, Tab. bit_pattern,
 * Tab. Lagrange_2d_linear).  A step of the particle-in-cell loop is
 * amr_deposit -> amr_solve -> amr_gather (Fig. sc_workflow).
 *
 * Conventions (all entry points):
 *  - Every call returns an amr_status; on failure amr_last_error() gives a
 *    thread-local message.  Invalid arguments return AMR_EINVAL before any
 *    device work.  A hierarchy stays destroyable after any failure.
 *  - All device work runs on the CUDA stream given to amr_create_hierarchy,
 *    in stream order.  Calls return when their work is enqueued, except
 *    amr_solve (waits once per convergence check to read the residual
 *    norms), amr_step and the amr_get_* / amr_set_* copies, which return
 *    when their results are in host memory.
 *  - Pointers are DEVICE pointers unless the argument name ends in _host.
 *    Particle arrays are structure-of-arrays float64 of length n, owned by
 *    the caller; the hierarchy owns all grid memory.
 *  - Units are the caller's: the solve uses rho/eps0 with eps0 from the
 *    descriptor (default 1).
 *  - Dense level layout (amr_get_level / amr_set_level / amr_get_mask): the
 *    bounding box [lo, hi] (inclusive, level index space) of the level's
 *    valid cells, i fastest then j then k, i.e. element
 *    ((k - lo[2]) * ny + (j - lo[1])) * nx + (i - lo[0]) with
 *    nx = hi[0] - lo[0] + 1 etc.  Cells of the box outside the level read
 *    as 0 and are ignored on write.
 */
#ifndef AMRMG_H
#define AMRMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amr_hierarchy amr_hierarchy; /* opaque, library-owned */

typedef enum {
    AMR_OK = 0,
    AMR_EINVAL = 1,    /* invalid argument; nothing was done */
    AMR_ENOMEM = 2,    /* device or host allocation failed */
    AMR_ENOCONV = 3,   /* max_iter V-cycles without reaching eps; phi valid */
    AMR_ECUDA = 4,     /* a CUDA call failed (message has the CUDA error) */
    AMR_ETIMEOUT = 5,  /* a bounded device wait ran out */
    AMR_ENESTING = 6,  /* boxes not aligned to coarse cells or not properly nested */
    AMR_EOUTSIDE = 7   /* a particle lies outside [h0, 1 - h0]^3 */
} amr_status;

enum {
    AMR_TAG_REL_RHO = 0, /* refine where rho > lambda * max rho (per level) */
    AMR_TAG_ABS_RHO = 1, /* refine where |rho| >= lambda (Eq. tag_charge) */
    AMR_TAG_BOXES = 2,   /* explicit boxes */
    /* regrid policies only (amr_regrid_boxes; they need solved fields): */
    AMR_TAG_PHI = 3,     /* refine where |phi| >= lambda * max |phi| (per level) */
    AMR_TAG_EFIELD = 4   /* refine where |E_w| >= lambda * max |E_w| for some w */
};

enum { AMR_FP64 = 0, AMR_MIXED = 1 };

/* Domain-face conditions (Sec. 5.2).  AMR_BC_ROBIN is the paper's open-
 * boundary approximation d phi/dn + phi/d = 0 (Eq. robin_bc) by central
 * difference across the face: ghost = alpha phi_0, alpha = (2d - h)/(2d + h)
 * on a grid of spacing h. */
enum { AMR_BC_DIRICHLET = 0, AMR_BC_ROBIN = 1, AMR_BC_PERIODIC = 2 };

enum { AMR_RHO = 0, AMR_PHI = 1, AMR_RES = 2, AMR_EX = 3, AMR_EY = 4, AMR_EZ = 5 };

enum { AMR_NORM_INF = 0, AMR_NORM_1 = 1, AMR_NORM_2 = 2 };

#define AMR_MAX_LEVELS 6

/*
 * Hierarchy descriptor (Sec. 3 and Sec. 4.2).
 *  n0          base cells per axis (level 0 covers the unit cube); n0 must be
 *              a multiple of brick/2 and at least 8.
 *  max_level   requested finest level l_max (0 .. AMR_MAX_LEVELS-1); tagging
 *              may stop earlier when nothing is tagged.
 *  brick       fine brick edge in cells (even, default 8): tagging marks
 *              aligned blocks of brick/2 cells of level l, each refined into
 *              one brick of level l+1.
 *  tag_mode    AMR_TAG_REL_RHO, AMR_TAG_ABS_RHO or AMR_TAG_BOXES.
 *  tag_lambda  threshold of the tagging modes.
 *  buffer_cells tags are grown by this many cells (Chebyshev) before the
 *              block marking (default 1).
 *  n_boxes, boxes  for AMR_TAG_BOXES: host array [n_boxes][7] =
 *              (level, lo_i, lo_j, lo_k, hi_i, hi_j, hi_k), inclusive, in
 *              that level's index space; lo even and hi odd on every axis.
 *  precision   AMR_FP64 (all arithmetic FP64) or AMR_MIXED (FP32 smoothing
 *              and transfers, FP64 residual, interface flux and bottom).
 *  eps0        permittivity (default 1).
 *  bc          AMR_BC_DIRICHLET (phi = 0 on the faces, default),
 *              AMR_BC_ROBIN or AMR_BC_PERIODIC (Sec. 5.2).  Only level 0
 *              touches the faces (proper nesting keeps refined levels two
 *              cells inside).  With Robin or periodic faces the level-0
 *              bottom solve is always geometric multigrid (the exact
 *              sine-transform bottom diagonalises Dirichlet only).  Periodic
 *              faces make the operator singular (constants): amr_solve then
 *              replaces rho by rho - <rho> (<.> the volume mean over the
 *              composite domain: a uniform neutralising background, written
 *              back into the hierarchy's rho) and returns the mean-free
 *              potential; such hierarchies are not accepted by
 *              amr_batch_create, and amr_solve runs them through the
 *              captured graph even when the persistent option is set.
 *  robin_d     artificial distance d > 0 of AMR_BC_ROBIN, in unit-cube
 *              lengths (ignored for Dirichlet).  AMR_EINVAL if bc is unknown
 *              or d is not a positive finite number.
 * Proper nesting (Fig. amr): the footprint of level l+1, grown by two cells of
 * level l, must lie inside the domain and inside level l's valid region;
 * tagging keeps only blocks that satisfy it and explicit boxes that violate
 * it fail with AMR_ENESTING.
 */
typedef struct {
    int n0;
    int max_level;
    int brick;
    int tag_mode;
    double tag_lambda;
    int buffer_cells;
    int n_boxes;
    const int *boxes_host;
    int precision;
    double eps0;
    int bc;
    double robin_d;
    /* 0: no limit; > 0: creation fails with AMR_ENOMEM (and allocates
     * nothing that stays) rather than hold more than this many device bytes
     * (the budget cap of the served form; amr_device_bytes counts them) */
    int64_t max_device_bytes;
} amr_desc;

/* Fill *d with the defaults (n0 = 64, max_level = 0, brick = 8,
 * AMR_TAG_REL_RHO, lambda = 0.1, buffer 1, no boxes, AMR_FP64, eps0 = 1,
 * AMR_BC_DIRICHLET). */
int amr_desc_default(amr_desc *d);

/*
 * Create a hierarchy.  With a tagging mode the particles (device arrays,
 * n may be 0 only with AMR_TAG_BOXES) are deposited level by level to tag
 * the next level.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  On success *out owns all device memory of the hierarchy.
 * Errors: AMR_EINVAL (descriptor), AMR_ENESTING (boxes), AMR_EOUTSIDE,
 * AMR_ENOMEM, AMR_ECUDA.
 */
int amr_create_hierarchy(const amr_desc *desc, const double *x, const double *y, const double *z,
                         const double *q, int64_t n, void *cuda_stream, amr_hierarchy **out);

/* Release everything the hierarchy owns (NULL is a no-op). */
void amr_destroy(amr_hierarchy *h);

/*
 * Cloud-in-cell charge deposit of n particles onto every level (each level
 * receives all particles on its own grid; values are kept on its valid
 * cells): rho^l at cell centre (i + 1/2) h_l gets q w_x w_y w_z / h_l^3 with
 * the linear weights of the two nearest centres per axis.  Replaces the
 * previous rho.  FP64 atomics: the summation order is not fixed, so rho is
 * reproducible to rounding (~1e-16 relative), not bitwise.
 */
int amr_deposit(amr_hierarchy *h, const double *x, const double *y, const double *z, const double *q,
                int64_t n);

/* Solve options (Alg. 2).  Defaults: eps 1e-10, AMR_NORM_2, max_iter 100,
 * nu_pre = nu_post = 2, bottom_cycles 2, warm_start 0, use_graph 1.  The
 * graph of a hierarchy is captured on the first solve with a given
 * (nu_pre, nu_post, bottom_cycles, warm_start) and reused afterwards; while
 * the per-launch timers (amr_profile) are on, solves run host-driven. */
typedef struct {
    double eps;        /* stop when ||r^l||_p <= eps ||rho^l||_p on every level */
    int norm;          /* AMR_NORM_INF, AMR_NORM_1, AMR_NORM_2 */
    int max_iter;      /* maximum number of V-cycles */
    int nu_pre, nu_post; /* red-black Gauss-Seidel sweeps (red + black each) */
    int bottom_cycles; /* geometric-multigrid V-cycles of the level-0 solve
                          (ignored when that solve is exact, see
                          amr_bottom_solver) */
    int warm_start;    /* 1: start from the current phi, 0: from phi = 0 */
    int use_graph;     /* 1: the whole solve is one captured CUDA graph with a
                          device-side convergence loop (no host round trip per
                          V-cycle); 0: host-driven loop, one launch per kernel */
    int persistent;    /* 1: the whole solve is one persistent cooperative
                          kernel executing the recorded operations in rounds
                          separated by a bounded grid barrier (overrides
                          use_graph) */
} amr_solve_opts;

int amr_solve_opts_default(amr_solve_opts *o);

/* Per-solve statistics. */
typedef struct {
    int iters;                      /* V-cycles performed */
    int status;                     /* AMR_OK or AMR_ENOCONV */
    int n_levels;
    double rel_res[AMR_MAX_LEVELS]; /* final ||r^l|| / ||rho^l|| per level */
    double ms_total;                /* wall time of the call */
} amr_solve_stats;

/*
 * Alg. 2: initial composite residuals, V-cycles (Alg. 3; the level-0
 * correction solved exactly or by geometric multigrid, see
 * amr_bottom_solver) until every level meets the
 * stopping test or max_iter, then average down (phi^l <- U phi^l +
 * R phi^{l+1}) and E^l = -G^l phi^l on every level.  Returns AMR_ENOCONV
 * (stats filled, phi and E valid) if max_iter is reached.  stats may be NULL.
 */
int amr_solve(amr_hierarchy *h, const amr_solve_opts *opts, amr_solve_stats *stats);

/*
 * Particle binning (the step before the deposit; cf. Sec. 4, where the
 * particles are redistributed to the boxes of the level they live on):
 * keys[p] = the brick (8^3 cells counted from the lower corner of the level's
 * valid bounding box) that holds particle p's cell, on the finest level whose
 * valid cells hold all 8 of its cloud-in-cell nodes, with the bricks of all
 * levels numbered level after level, coarse first; 0xFFFFFFFF for a particle
 * with no such level (outside level 0's interior, non-finite).  perm lists
 * the particle indices sorted by key (a counting sort; the order of equal
 * keys is unspecified).  keys (n) and perm (n) are caller-owned device
 * arrays; *nkeys_out (host) receives the number of bricks.  Stream-ordered:
 * the outputs are ready when the hierarchy's stream reaches this point.
 * The first call allocates the bucket array.  Errors: AMR_EINVAL (null or
 * n outside 0 .. 2^31-1), AMR_ENOMEM.
 */
int amr_bin(amr_hierarchy *h, const double *x, const double *y, const double *z, int64_t n, uint32_t *keys,
            int64_t *perm, int64_t *nkeys_out);

/*
 * Solve n independent hierarchies to the same options at once (Alg. 2 for
 * each): every hierarchy's captured solve graph (the one amr_solve uses) is
 * launched on one of n_streams library-owned streams, round robin, after
 * the work already queued on the hierarchy's own stream and before the work
 * queued there later.  Small hierarchies leave most of the GPU idle one at
 * a time; side by side their graphs fill it.  Results are the same bits as
 * amr_solve of each.  Hierarchies with periodic faces are solved one after
 * another after the others.  stats (may be NULL): n entries.  Returns when
 * every solve has finished.  This is the batched work of amr_batch_* run as
 * concurrent graphs instead of one persistent launch (no counterpart in the
 * paper, which solves one hierarchy at a time).  Errors: AMR_EINVAL (null or
 * repeated hierarchy, n < 1, n_streams < 1, bad options), AMR_ENOCONV (some
 * hierarchy did not converge; all results valid), AMR_ECUDA.
 */
int amr_solve_many(amr_hierarchy *const *hs, int n, const amr_solve_opts *opts, int n_streams,
                   amr_solve_stats *stats);

/*
 * Cloud-in-cell interpolation of E (and phi if phi != NULL) to n particles
 * from the finest level whose valid cells hold all 8 nodes of the particle
 * (interpolate step of Fig. sc_workflow).  Outputs are device arrays.
 */
int amr_gather(amr_hierarchy *h, const double *x, const double *y, const double *z, int64_t n, double *ex,
               double *ey, double *ez, double *phi);

/*
 * One whole particle-in-cell field step through host memory: copies the
 * particles from host arrays to library-owned device buffers, deposits,
 * solves and gathers, and copies E back to host arrays.  The copies run in
 * up to eight chunks of the particles on a library-owned copy stream, each
 * chunk's deposit (gather) waiting only for its own copy, so that copies
 * overlap the deposit and the gather; from page-locked host arrays the
 * copies are asynchronous.  Returns when the results are in host memory.
 * Host arrays: n doubles each, caller-owned.  stats may be NULL.  Errors:
 * AMR_EINVAL (null pointer, n < 1), AMR_ENOMEM (staging buffers),
 * AMR_ENOCONV (results valid), AMR_EOUTSIDE (particles whose nodes leave
 * level 0's interior; results valid for the others), AMR_ECUDA.
 */
int amr_step(amr_hierarchy *h, const double *x_host, const double *y_host, const double *z_host,
             const double *q_host, int64_t n, const amr_solve_opts *opts, double *ex_host, double *ey_host,
             double *ez_host, amr_solve_stats *stats);

/* Alg. 1 on every level with the current phi; rel_out[l] = ||r^l||_p /
 * ||rho^l||_p (a level with ||rho^l|| = 0 uses the largest ||rho^l||). */
int amr_residual(amr_hierarchy *h, int norm, double *rel_out_host);

/* Average down then E = -G phi on every level, from the current phi. */
int amr_field_from_phi(amr_hierarchy *h);

int amr_num_levels(const amr_hierarchy *h, int *n_levels);

/* Valid bounding box of a level and its number of valid cells. */
int amr_level_box(const amr_hierarchy *h, int level, int lo[3], int hi[3], int64_t *n_valid);

/* Copy a field of a level to / from a host array in the dense level layout.
 * field: AMR_RHO (stored as rho/eps0), AMR_PHI, AMR_RES, AMR_EX..AMR_EZ. */
int amr_get_level(amr_hierarchy *h, int level, int field, double *out_host);
int amr_set_level(amr_hierarchy *h, int level, int field, const double *in_host);

/* Cell kinds in the dense level layout: 0 outside the level, 1 valid and
 * uncovered, 2 valid and covered by level+1. */
int amr_get_mask(amr_hierarchy *h, int level, int8_t *out_host);

/* How many coarse-fine ghosts use the quadratic, linear and constant
 * stencils (Sec. 5.1 pattern selection). */
int amr_ghost_stats(const amr_hierarchy *h, int64_t out_host[3]);

/*
 * Regrid (Sec. 4.2, AMR policies): the boxes of a new hierarchy's refined
 * levels from h's CURRENT fields.  For l = 0, 1, ... (l < levels of h,
 * l + 1 <= max_level) the valid cells of h's level l are tagged by `policy`
 * with threshold lambda:
 *   AMR_TAG_REL_RHO  rho > lambda * max rho     AMR_TAG_ABS_RHO  |rho eps0| >= lambda (Eq. tag_charge)
 *   AMR_TAG_PHI      |phi| >= lambda * max |phi|
 *   AMR_TAG_EFIELD   |E_w| >= lambda * max |E_w| for some w in {x, y, z}
 * (maxima over the level's valid cells; a zero maximum tags nothing; the
 * potential and field are those of the last amr_solve or
 * amr_field_from_phi).  Tags are grown by buffer_cells (Chebyshev distance)
 * and mark aligned blocks of brick/2 cells of level l, each a brick of the
 * new level l+1, kept only if the block grown by two cells lies inside the
 * domain and inside the NEW level l (proper nesting).  Tagging and marking
 * run on h's stream; the call returns when the boxes are on the host.
 * boxes_host: caller array of cap boxes of 7 ints (level, lo[3], hi[3],
 * inclusive, in (k, j, i) block order per level), the AMR_TAG_BOXES layout
 * of amr_desc; *n_boxes_out gets the number made.  Errors: AMR_EINVAL for a
 * bad argument or when cap is smaller than the number made (then
 * *n_boxes_out holds the number needed), AMR_ENOMEM, AMR_ECUDA.
 */
int amr_regrid_boxes(amr_hierarchy *h, int policy, double lambda, int buffer_cells, int max_level, int *boxes_host,
                     int cap, int *n_boxes_out);

/*
 * Warm start after a regrid: phi of every level of dst is set from src's
 * level of the same index where src holds the cell, else from the parent
 * cell of dst's next coarser level (piecewise constant, the prolongation
 * of the V-cycle).  A following amr_solve with warm_start = 1 starts from
 * it.  Both hierarchies need the same n0.  Enqueued on dst's stream (src's
 * stream is synchronised first when they differ).  Errors: AMR_EINVAL,
 * AMR_ECUDA.
 */
int amr_transfer_phi(const amr_hierarchy *src, amr_hierarchy *dst);

/*
 * Buffer cells against the spurious self-force of particles near a
 * coarse-fine face (Sec. 4, corrected with buffer cells as in the work the
 * paper cites): from this call on, amr_gather (and amr_step) interpolates a
 * particle from a refined level only if every cell within Chebyshev
 * distance buffer_cells of its 8 cloud-in-cell nodes is valid on that
 * level, else from the next coarser level.  0 (the default) is the plain
 * rule: the finest level holding the 8 nodes.  Builds one byte per cell of
 * every refined level (stream-ordered).  Errors: AMR_EINVAL (buffer_cells
 * outside 0..8), AMR_ENOMEM, AMR_ECUDA.
 */
int amr_set_gather_buffer(amr_hierarchy *h, int buffer_cells);

/*
 * Domain transform (Sec. 4.1, Fig. sc_workflow): particles at x (particle
 * space) are mapped into the unit cube the hierarchy covers,
 *     u = 1/2 + (x - centre) / S,   S = 2 s,   s = (1 + delta) max_i Gamma_i,
 * Gamma_i = max_d |x_i,d - centre_d| (Gamma of the paper with l = (1, 1, 1):
 * the computation space is a cube), so the particles fill the central
 * 1/(1 + delta) of the cube (delta: the box increment, 0.2 in the paper's
 * runs).  x, y, z, u, v, w: device arrays of n float64 (u may alias x for
 * an in-place map); centre_host: 3 doubles.  *scale_out_host gets S, the
 * particle-space length of the cube's edge.  Element-wise arithmetic with
 * rounded operations only (no FMA), so u is the same bits as the formula
 * in FP64.  Returns when S is on the host.  Errors: AMR_EINVAL (bad
 * arguments, delta < 0, no particle away from the centre, non-finite
 * coordinates), AMR_ENOMEM, AMR_ECUDA.
 */
int amr_domain_transform(const double *x, const double *y, const double *z, int64_t n, const double centre_host[3],
                         double delta, double *u, double *v, double *w, double *scale_out_host, void *cuda_stream);

/*
 * Back to particle space on the grid (Fig. sc_workflow; Eqs.
 * potential_transform and efield_transform with S of amr_domain_transform):
 * phi <- phi / S and E <- E / S^2 on every level, so that amr_gather then
 * interpolates particle-space fields at the cube coordinates u.  Call after
 * amr_solve and before amr_gather; the next amr_solve recomputes phi and E
 * (use warm_start = 0, the rescaled phi is not the cube's solution).
 * Errors: AMR_EINVAL (S not positive and finite), AMR_ECUDA.
 */
int amr_rescale_fields(amr_hierarchy *h, double S);

/*
 * Kick-drift particle push with the gathered field (the integration step
 * around the space-charge solve): p <- p + (q/m) dt E, then x <- x + dt p,
 * per particle, in place (device arrays of n float64; p is the velocity in
 * the caller's units; non-relativistic).  Rounded operations only (same bits
 * as the formula in FP64).  Errors: AMR_EINVAL, AMR_ECUDA.
 */
int amr_push(double *x, double *y, double *z, double *px, double *py, double *pz, const double *ex, const double *ey,
             const double *ez, int64_t n, double q_over_m, double dt, void *cuda_stream);

/*
 * Beam moments (Eqs. rms_sigma and halo) of n >= 1 particles, about the
 * centroid: out_host[0..2] = <w>, out_host[3..5] = sigma_w = sqrt(<(w -
 * <w>)^2>), out_host[6..8] = xi_w = <(w - <w>)^4> / <(w - <w>)^2>^2 (0 when
 * the spread is 0), w = x, y, z.  FP64 sums (atomic, so reproducible to
 * rounding).  Returns when the values are on the host.  Errors: AMR_EINVAL,
 * AMR_ENOMEM, AMR_ECUDA.
 */
int amr_moments(const double *x, const double *y, const double *z, int64_t n, double out_host[9], void *cuda_stream);

/* Upper bound of the device bytes a hierarchy of this descriptor would hold
 * when its finest level is no larger than a fraction `fill` (0 < fill <= 1)
 * of its index space (used for admission by memory budget). */
int amr_hierarchy_bytes(const amr_desc *desc, double fill, int64_t *bytes_out);

/* Device bytes the hierarchy holds. */
int amr_device_bytes(const amr_hierarchy *h, int64_t *bytes_out);

/* Number of kernels this library launched on the hierarchy's stream since
 * it was created (a counter kept by the host launch wrappers). */
int amr_kernel_launches(const amr_hierarchy *h, int64_t *count_out);

/* How the V-cycle solves the level-0 correction equation A_nf^0 e^0 = r^0
 * (Alg. 3, the bottom of the recursion; the paper leaves the method open):
 * AMR_BOTTOM_EXACT = sine transforms along x and y and tridiagonal solves
 * along z (exact up to rounding; chosen for n0 <= 64 with n0 a multiple
 * of 4 unless the environment sets AMR_BOTTOM=mg), AMR_BOTTOM_GMG =
 * bottom_cycles geometric-multigrid V-cycles with a dense coarsest solve. */
enum { AMR_BOTTOM_GMG = 0, AMR_BOTTOM_EXACT = 1 };
int amr_bottom_solver(const amr_hierarchy *h, int *kind_out);

/*
 * Per-launch kernel timers.  amr_profile(h, 1) resets the totals and from
 * then on brackets every kernel the library launches with a pair of CUDA
 * events on the hierarchy's stream, solves running host-driven (one launch
 * per operation); amr_profile(h, 2) does the same but runs each graph solve
 * as its captured graph unrolled to the V-cycle count of the solve before
 * the call -- the same kernels and grouped launches as the solve graph --
 * with an event-record node before and after every kernel node (an
 * operation of a grouped launch is charged its share of the group's
 * algorithmic bytes); amr_profile(h, 0) stops.  Kinds are
 * 0 .. amr_profile_num_kinds()-1 (deposit, gather, residual, rbgs, restrict,
 * prolong, finish, cf_correct, flux, grad, average_down, norms,
 * mg_restrict, mg_prolong, coarse_solve, elementwise, coarse_part, check,
 * mg_bottom, bin, sine_transform, tridiagonal; amr_profile_kind_name).
 * amr_profile_read
 * waits for the pending events and returns, for one kind, the summed
 * device time of its launches (ms), their number and their summed
 * algorithmic bytes (the bytes the method must move per launch).
 */
int amr_profile(amr_hierarchy *h, int mode);
int amr_profile_num_kinds(void);
const char *amr_profile_kind_name(int kind);
int amr_profile_read(amr_hierarchy *h, int kind, double *ms_total, int64_t *launches, double *alg_bytes);
/* Summed algorithmic floating-point operations (an FMA counts 2) of the
 * timed launches of one kind, in the precision the kind computes in; 0 for
 * kinds without a flop count (the smoother, kind "rbgs", has one: 8 per
 * updated cell, 3 per red cell of a sweep that starts from zero; the
 * exact bottom's sine transforms count their adds and multiplies). */
int amr_profile_read_flops(amr_hierarchy *h, int kind, double *alg_flops);
/* The same kinds' algorithmic arithmetic instructions in the precision they
 * compute in (an FMA counts 1): the work an FP64-bound kernel issues to the
 * FP64 pipe, whose rate amr_probe_fp64_fma measures.  Counted for the
 * kinds with a flop count. */
int amr_profile_read_ops(amr_hierarchy *h, int kind, double *alg_ops);

/*
 * Batched solve: n independent hierarchies (any mix of sizes and depths)
 * solved together by ONE persistent kernel launch, replayed from a CUDA
 * graph.  Each hierarchy's init / V-cycle / tail operations are recorded
 * once at amr_batch_create, and the whole launch (parameter uploads, the
 * kernel, the state read-backs) is captured there as a graph that every
 * amr_batch_solve replays.  The kernel runs on thread-block clusters: each
 * cluster takes the next hierarchy from a queue (largest first) and runs
 * its solve alone -- the V-cycles while that hierarchy is above its
 * tolerance -- with the cluster's hardware barrier between operations, so
 * hierarchies of all sizes progress side by side without a grid-wide
 * barrier.  Setting AMR_BATCH=rounds at creation selects the earlier form
 * instead: one cooperative launch that interleaves the hierarchies in rounds
 * (round r holds operation r of every hierarchy) separated by a grid barrier
 * whose waits are bounded (AMR_ETIMEOUT).  Either way the results are those
 * of solving each hierarchy alone with the same options, bit for bit.  The
 * batch launches on the first hierarchy's stream after the others' streams
 * are synchronised.  stats receives n entries (may be NULL); returns
 * AMR_ENOCONV if any hierarchy stopped at max_iter.  The hierarchies must
 * outlive the batch.
 */
typedef struct amr_batch amr_batch;
int amr_batch_create(amr_hierarchy *const *hs, int n, const amr_solve_opts *opts, amr_batch **out);
int amr_batch_solve(amr_batch *b, amr_solve_stats *stats);
void amr_batch_destroy(amr_batch *b);

/*
 * Self-test of the failure path of the persistent kernel's grid barrier:
 * runs the hierarchy's solve program with a barrier that can never complete
 * (it expects more blocks than are launched), so every wait runs out after
 * limit_ms (1..10000) and the kernel returns.  Returns AMR_ETIMEOUT when the
 * bounded wait worked; the hierarchy stays usable (phi must be re-solved).
 */
int amr_selftest_barrier_timeout(amr_hierarchy *h, int limit_ms);

/*
 * Served form: continuous batching of independent solve requests.
 * Each request describes a hierarchy (base n0, max_level, precision) and a
 * seeded isotropic Gaussian bunch (n_particles, sigma, centre, seed) that is
 * generated on the device (Philox-4x32-10 counter-based generator with the
 * Box-Muller transform, equal charges 1/n) -- or the caller's particles --
 * and an arrival time.  amr_serve
 * runs the request loop: requests are admitted in arrival order as soon as
 * one of max_slots slots is free and the request's estimated device bytes
 * (amr_request_bytes) fit in budget_bytes next to the admitted ones; each
 * slot runs deposit -> tagged hierarchy -> solve (opts) -> gather on its own
 * CUDA stream from its own host thread, so admitted requests overlap on the
 * device; a request's hierarchy and multigrid state stay on the device
 * until it completes.  realtime = 1 releases requests at their arrival_s
 * (wall clock from the start of the call), 0 releases all at once.
 * A request's hierarchy is created with its charge (the estimate) as a hard
 * cap on its device bytes; one whose tagged boxes need more gives the charge
 * back, waits until twice the charge is free (at most the whole budget)
 * while nothing new is admitted, and is created again under the larger cap,
 * so the admitted requests never hold more than budget_bytes.
 * results[i] gets the times (seconds from the start), status (AMR_ENOMEM if
 * the request alone exceeds the budget), iterations, largest relative
 * residual, device bytes and checksums of the gathered field
 * (sum Ex, sum Ey, sum Ez, sum |E| over the particles, fixed-order sums).
 * Returns when every request has completed.
 */
typedef struct {
    int n0, max_level, precision;
    int64_t n_particles;
    double sigma, centre[3];
    uint64_t seed;
    double arrival_s;
    /* Optional caller-owned device arrays of n_particles doubles each: when
     * x is non-NULL the request solves these particles (y, z, q must be
     * non-NULL too, AMR_EINVAL otherwise) instead of the seeded bunch; they
     * must stay valid and unchanged until amr_serve returns. */
    const double *x, *y, *z, *q;
    /* Optional caller-owned device buffer of 4 n_particles doubles: the
     * gathered Ex, Ey, Ez and phi at the particles, one block of
     * n_particles each (NULL: only the checksums are kept). */
    double *field_out;
} amr_request;

typedef struct {
    double arrival_s, admit_s, done_s;
    int status, iters, n_levels;
    int retried; /* 1: outgrew its charge and was created again under a larger one */
    double rel_res_max;
    int64_t device_bytes;
    double checksum[4];
} amr_request_result;

typedef struct {
    int64_t budget_bytes;
    int max_slots;
    int realtime;
    /* Fraction of each request's estimate charged at admission and used as
     * its hierarchy's cap (0 or >= 1: the whole estimate).  Below 1 more
     * requests run side by side; one that needs more than its charge is
     * created again under a larger one, as above, so the budget still holds. */
    double admit_fraction;
} amr_serve_config;

int amr_serve(const amr_serve_config *cfg, const amr_request *reqs, int n, const amr_solve_opts *opts,
              amr_request_result *results);

/* Device bytes the server reserves for a request at admission. */
int amr_request_bytes(const amr_request *r, int64_t *bytes_out);

/*
 * Allocation-free masked norms (the paper has no counterpart: this is a
 * library service).  For callers that cannot call cudaMalloc -- code that
 * runs while a CUDA graph is being captured on its thread, callers that own
 * the device memory pool and forbid other allocations, real-time loops
 * where an allocation may synchronise the device -- this computes, on the
 * given stream, out3[0] = sum v^2, out3[1] = sum |v|, out3[2] = max |v|
 * over the elements t < n with mask[t] == 1, or mask[t] == 1 or 2 when
 * covered_too (mask == NULL: all elements; the mask convention of
 * amr_get_mask: 1 valid uncovered, 2 valid covered), i.e. the norms that
 * amr_residual's stopping test uses.  A NaN element makes every one of the
 * three NaN (the max is taken on the bits of |v|, where NaN sorts above
 * +inf, as in the library's own norms).
 * v, mask and out3 are device pointers owned by the caller.  It allocates
 * nothing: its scratch is a fixed 24 KiB device array in the library
 * (up to 1024 per-block partials) that every GPU loading the library keeps
 * until the process exits.  n may be at most 67,108,864 (AMR_EINVAL
 * beyond).  The first call on a device looks up the array's device address
 * with that device current (make that first call before any stream
 * capture); later calls do no setup.  All calls share the one array, so
 * calls whose kernels overlap on the GPU race: serialise them (one stream,
 * or events).  The result is a fixed-order sum, reproducible for a given n.
 */
int amr_masked_norms_noalloc(const double *v, const uint8_t *mask, int64_t n, int covered_too, double *out3,
                             void *cuda_stream);

/*
 * FP64 arithmetic throughput probe (the paper has no counterpart: it
 * measures the denominator of the roofline of the FP64-bound kernels).  One
 * launch of as many 256-thread blocks as are resident on the device, each
 * thread running 8 independent chains of `iters` dependent FP64 FMAs, timed
 * with CUDA events on the given stream after a shorter warm-up launch.
 * *gfma_per_s receives the FMA rate (1e9 FMA/s; one FMA = 2 flops), *ms_out
 * (may be NULL) the timed launch's duration.  iters in 1 .. 2^30 (AMR_EINVAL
 * otherwise).  Allocates a small output array from the stream-ordered pool.
 */
int amr_probe_fp64_fma(int64_t iters, double *gfma_per_s, double *ms_out, void *cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char *amr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMRMG_H */
