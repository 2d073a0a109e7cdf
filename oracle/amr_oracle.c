/*
 * amr_oracle.c -- plain, slow, FP64 CPU oracle of the AMR multigrid Poisson
 * solve of Frey, Adelmann & Locans, "On Architecture and Performance of
 * Adaptive Mesh Refinement in an Electrostatics Particle-In-Cell Code"
 * (arXiv 1812.03689).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing of the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes, in the paper's order and notation:
 *   - a block-structured, ratio-2, cell-centred hierarchy (Sec. 3, Eq.
 *     mesh_spacing; proper nesting, Fig. amr), built from explicit boxes or by
 *     charge-density tagging (Eq. tag_charge) with a fixed brick rule;
 *   - cloud-in-cell deposition of every particle onto every level;
 *   - the per-level matrices of Sec. 5.3 (A_nf, A_comp, B_crse, B_fine, R, I,
 *     G, U) assembled EXPLICITLY as CSR matrices from the flux-differencing
 *     formulas (Eqs. lap_flux_differencing, coarse_fluxes, flux_differencing)
 *     and the two-step Lagrange ghost interpolation (Eq. 2d_lagrange, with the
 *     pattern selection of Tab. bit_pattern and Tab. Lagrange_2d_linear);
 *   - Alg. 1 (RESIDUAL), Alg. 2 (SOLVE) and Alg. 3 (RELAX) literally, with
 *     red-black Gauss-Seidel smoothing and a conjugate-gradient bottom solve;
 *   - average-down, E = -G phi (Alg. 2) and cloud-in-cell gather.
 *
 * Threads (OpenMP, when the compiler has it; orc_set_threads): only loops
 * whose iterations are independent run in parallel -- matrix rows, the cells
 * of one colour of a red-black sweep, vector updates and the particles of
 * the gather -- so each result is the one the serial loop gives.  The inner
 * products of the conjugate-gradient bottom solve are summed in fixed blocks
 * of rows (partial sums in block order), so they do not depend on the
 * thread count either.  The deposit stays serial, in particle order.
 *
 * Sign convention: A = -L (positive definite), right-hand side b = rho/eps0,
 * residual r = b - A phi, which is Alg. 1's "r = rho - A phi" with eps0
 * absorbed into rho.
 *
 * Readings of silent or garbled passages (each also listed in the design
 * notes of the repository):
 *   - Alg. 3 prolongation step: e^l <- e^l + I e^{l-1} (the printed
 *     "e^l <- I e^{l-1}" would discard the pre-smoothed correction).
 *   - Alg. 3 uncovered-residual step: on uncovered cells of level l-1 the
 *     residual is rho^{l-1} - A_comp phi^{l-1} - B_crse phi^{l-2}
 *     - B_fine phi^l; covered cells keep the restricted value.
 *   - Pre- and post-smoothing start from a zero error.
 *   - R is the 8-cell average, I is piecewise constant.
 *   - Homogeneous Dirichlet at the domain faces, linear ghost -phi_0.
 *   - Robin faces (Eq. robin_bc, d phi/dn + phi/d = 0, "central difference"):
 *     the face lies midway between the boundary cell centre phi_0 and its
 *     ghost phi_g, the normal derivative there is (phi_g - phi_0)/h and the
 *     face value the mean (phi_g + phi_0)/2, so phi_g = alpha phi_0 with
 *     alpha = (2d - h)/(2d + h); alpha = -1 is the Dirichlet ghost (d -> 0).
 *   - Periodic faces (Sec. 5.2 lists them beside Dirichlet and Robin): the
 *     neighbour across a face of level 0 is the cell on the opposite face
 *     (refined levels never reach the faces).  The operator is then singular
 *     (constants), so the solve takes the neutralised density rho - <rho>
 *     (<.> the volume mean over the composite domain, a uniform background
 *     of opposite charge), the level-0 bottom problem its mean-free part,
 *     and the result is the mean-free potential.
 *   - Ghost availability bit = 1 iff the coarse cell is in the domain, valid
 *     on level l-1 and not covered by level l; no match of any quadratic or
 *     linear pattern falls back to the coarse cell value itself.
 *   - Proper nesting (Fig. amr) with a margin of two cells of the coarser
 *     level around the finer level's footprint.
 *   - Stopping test: ||r^l||_p <= eps ||rho^l||_p on every level, norms over
 *     the level's valid cells (r is zero on covered cells); a level with
 *     ||rho^l|| = 0 uses the largest ||rho^l|| of all levels.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXLEV 6
#define PAD 2

/* Loops shorter than this stay serial. */
#define PAR_MIN 8192
/* Rows per block of the blocked inner products. */
#define DOT_BLOCK 4096

/* ------------------------------------------------------------------ CSR -- */

typedef struct {
    int nrows, ncols;
    int *ptr;      /* nrows+1 */
    int *col;
    double *val;
    int nnz, cap;
} csr;

static void csr_init(csr *m, int nrows, int ncols)
{
    m->nrows = nrows;
    m->ncols = ncols;
    m->ptr = (int *)calloc((size_t)nrows + 1, sizeof(int));
    m->cap = 16;
    m->nnz = 0;
    m->col = (int *)malloc(sizeof(int) * (size_t)m->cap);
    m->val = (double *)malloc(sizeof(double) * (size_t)m->cap);
}

static void csr_free(csr *m)
{
    free(m->ptr);
    free(m->col);
    free(m->val);
    memset(m, 0, sizeof(*m));
}

/* Row accumulator: entries of one row, duplicates merged. */
typedef struct {
    int n;
    int col[256];
    double val[256];
} rowacc;

static void row_add(rowacc *r, int col, double v)
{
    for (int i = 0; i < r->n; ++i)
        if (r->col[i] == col) {
            r->val[i] += v;
            return;
        }
    if (r->n >= 256) {
        fprintf(stderr, "oracle: row accumulator overflow\n");
        abort();
    }
    r->col[r->n] = col;
    r->val[r->n] = v;
    r->n++;
}

/* Append row `row` (rows must be appended in increasing order). */
static void csr_put_row(csr *m, int row, const rowacc *r)
{
    if (m->nnz + r->n > m->cap) {
        while (m->nnz + r->n > m->cap) m->cap *= 2;
        m->col = (int *)realloc(m->col, sizeof(int) * (size_t)m->cap);
        m->val = (double *)realloc(m->val, sizeof(double) * (size_t)m->cap);
    }
    /* insertion sort by column, for a canonical layout */
    int start = m->nnz;
    for (int i = 0; i < r->n; ++i) {
        int c = r->col[i];
        double v = r->val[i];
        int p = m->nnz;
        while (p > start && m->col[p - 1] > c) {
            m->col[p] = m->col[p - 1];
            m->val[p] = m->val[p - 1];
            --p;
        }
        m->col[p] = c;
        m->val[p] = v;
        m->nnz++;
    }
    m->ptr[row + 1] = m->nnz;
}

/* Rows that were never put are empty: make ptr monotone. */
static void csr_finish(csr *m)
{
    for (int i = 0; i < m->nrows; ++i)
        if (m->ptr[i + 1] < m->ptr[i]) m->ptr[i + 1] = m->ptr[i];
}

/* y = y + alpha * M x (rows independent) */
static void csr_axpy(const csr *m, double alpha, const double *x, double *y)
{
#pragma omp parallel for schedule(static) if (m->nrows > PAR_MIN)
    for (int i = 0; i < m->nrows; ++i) {
        double s = 0.0;
        for (int p = m->ptr[i]; p < m->ptr[i + 1]; ++p) s += m->val[p] * x[m->col[p]];
        y[i] += alpha * s;
    }
}

/* ---------------------------------------------------------- hierarchy -- */

typedef struct {
    int lo[3], hi[3];   /* bounding box of the valid cells (level index space) */
    int dim[3];         /* padded box extent: hi - lo + 1 + 2*PAD */
    int8_t *valid;      /* padded box: 1 if the cell belongs to this level */
    int8_t *covered;    /* padded box: 1 if the cell is covered by level l+1 */
    int *row;           /* padded box -> vector index or -1 */
    int n;              /* number of valid cells */
    int *cell;          /* vector index -> global (i,j,k), 3 ints */
    double h;
    double *rho_pad;    /* padded box deposit accumulator */
    double *rho, *phi, *res, *err, *phisave, *de, *ef[3];
    /* matrices of Sec. 5.3 */
    csr Anf, Acomp, Bcrse, Bfine, R, I, G[3], Gc[3];
} olevel;

typedef struct {
    int n0;
    int nlev;           /* l_max + 1 */
    int lmax_req;
    double eps0;
    double robin_d;     /* artificial distance d of Eq. robin_bc; 0 = Dirichlet */
    int brick;          /* fine brick edge of tagged levels */
    int periodic;       /* 1: periodic domain faces */
    int gather_buffer;  /* refined level used by the gather only b cells inside */
    olevel L[MAXLEV];
    long ghost_order_count[3]; /* quadratic, linear, constant fall-back */
    char err[256];
} ohier;

static int nlevcells(const ohier *H, int l) { return H->n0 << l; }

static int64_t pidx(const olevel *lv, int i, int j, int k)
{
    int a = i - lv->lo[0] + PAD, b = j - lv->lo[1] + PAD, c = k - lv->lo[2] + PAD;
    if (a < 0 || b < 0 || c < 0 || a >= lv->dim[0] || b >= lv->dim[1] || c >= lv->dim[2]) return -1;
    return ((int64_t)c * lv->dim[1] + b) * lv->dim[0] + a;
}

static int is_valid(const olevel *lv, int i, int j, int k)
{
    int64_t p = pidx(lv, i, j, k);
    return p >= 0 && lv->valid[p];
}

static int is_covered(const olevel *lv, int i, int j, int k)
{
    int64_t p = pidx(lv, i, j, k);
    return p >= 0 && lv->covered[p];
}

static int row_of(const olevel *lv, int i, int j, int k)
{
    int64_t p = pidx(lv, i, j, k);
    return p >= 0 ? lv->row[p] : -1;
}

static int in_domain(const ohier *H, int l, const int c[3])
{
    int n = nlevcells(H, l);
    return c[0] >= 0 && c[1] >= 0 && c[2] >= 0 && c[0] < n && c[1] < n && c[2] < n;
}

/* Ghost factor alpha at a domain face of level l: phi_ghost = alpha phi_0.
 * Dirichlet phi = 0 at the face: alpha = -1.  Robin d phi/dn + phi/d = 0 by
 * central difference across the face (Eq. robin_bc):
 * (phi_g - phi_0)/h + (phi_g + phi_0)/(2d) = 0. */
/* The periodic image of cell c of level l inside the domain. */
static void wrap_cell(const ohier *H, int l, const int c[3], int out[3])
{
    int n = nlevcells(H, l);
    for (int d = 0; d < 3; ++d) out[d] = ((c[d] % n) + n) % n;
}

static double phys_ghost(const ohier *H, int l)
{
    if (H->robin_d <= 0.0) return -1.0;
    double h = H->L[l].h, d = H->robin_d;
    return (2.0 * d - h) / (2.0 * d + h);
}

/* Allocate level l's padded box over [lo,hi] with all cells invalid. */
static void level_alloc_box(ohier *H, int l, const int lo[3], const int hi[3])
{
    olevel *lv = &H->L[l];
    int64_t tot = 1;
    for (int d = 0; d < 3; ++d) {
        lv->lo[d] = lo[d];
        lv->hi[d] = hi[d];
        lv->dim[d] = hi[d] - lo[d] + 1 + 2 * PAD;
        tot *= lv->dim[d];
    }
    lv->valid = (int8_t *)calloc((size_t)tot, 1);
    lv->covered = (int8_t *)calloc((size_t)tot, 1);
    lv->row = (int *)malloc(sizeof(int) * (size_t)tot);
    for (int64_t p = 0; p < tot; ++p) lv->row[p] = -1;
    lv->rho_pad = (double *)calloc((size_t)tot, sizeof(double));
    lv->h = 1.0 / (double)nlevcells(H, l);
}

static int64_t level_box_cells(const olevel *lv)
{
    return (int64_t)lv->dim[0] * lv->dim[1] * lv->dim[2];
}

/* Number the valid cells in (k, j, i) lexicographic order. */
static void level_number(ohier *H, int l)
{
    olevel *lv = &H->L[l];
    int n = 0;
    for (int k = lv->lo[2]; k <= lv->hi[2]; ++k)
        for (int j = lv->lo[1]; j <= lv->hi[1]; ++j)
            for (int i = lv->lo[0]; i <= lv->hi[0]; ++i)
                if (is_valid(lv, i, j, k)) lv->row[pidx(lv, i, j, k)] = n++;
    lv->n = n;
    lv->cell = (int *)malloc(sizeof(int) * 3 * (size_t)(n > 0 ? n : 1));
    for (int k = lv->lo[2]; k <= lv->hi[2]; ++k)
        for (int j = lv->lo[1]; j <= lv->hi[1]; ++j)
            for (int i = lv->lo[0]; i <= lv->hi[0]; ++i) {
                int r = row_of(lv, i, j, k);
                if (r >= 0) {
                    lv->cell[3 * r] = i;
                    lv->cell[3 * r + 1] = j;
                    lv->cell[3 * r + 2] = k;
                }
            }
    size_t nn = (size_t)(n > 0 ? n : 1);
    lv->rho = (double *)calloc(nn, sizeof(double));
    lv->phi = (double *)calloc(nn, sizeof(double));
    lv->res = (double *)calloc(nn, sizeof(double));
    lv->err = (double *)calloc(nn, sizeof(double));
    lv->phisave = (double *)calloc(nn, sizeof(double));
    lv->de = (double *)calloc(nn, sizeof(double));
    for (int d = 0; d < 3; ++d) lv->ef[d] = (double *)calloc(nn, sizeof(double));
}

/* ------------------------------------------------------------ deposit -- */

/* Cloud-in-cell deposit of all particles onto level l's padded box: node
 * (cell centre) i at (i + 1/2) h, weight 1 - |x/h - 1/2 - i| on the two
 * nearest centres per axis; density = q * w / h^3. Particle order. */
static void deposit_level(ohier *H, int l, const double *x, const double *y, const double *z,
                          const double *q, long np)
{
    olevel *lv = &H->L[l];
    int64_t tot = level_box_cells(lv);
    memset(lv->rho_pad, 0, sizeof(double) * (size_t)tot);
    double h = lv->h, inv_vol = 1.0 / (h * h * h);
    for (long p = 0; p < np; ++p) {
        double s[3] = {x[p] / h - 0.5, y[p] / h - 0.5, z[p] / h - 0.5};
        int i0[3];
        double w[3][2];
        for (int d = 0; d < 3; ++d) {
            double f = floor(s[d]);
            i0[d] = (int)f;
            w[d][1] = s[d] - f;
            w[d][0] = 1.0 - w[d][1];
        }
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int64_t pi = pidx(lv, i0[0] + a, i0[1] + b, i0[2] + c);
                    if (pi < 0) continue;
                    lv->rho_pad[pi] += q[p] * w[0][a] * w[1][b] * w[2][c] * inv_vol;
                }
    }
    for (int r = 0; r < lv->n; ++r) {
        const int *c = &lv->cell[3 * r];
        lv->rho[r] = lv->rho_pad[pidx(lv, c[0], c[1], c[2])] / H->eps0;
    }
}

/* ------------------------------------------------------------ tagging -- */

/* Proper-nesting margin, in cells of the coarser level: the footprint of
 * level l+1 grown by NEST cells must lie inside the domain and inside the
 * valid region of level l.  Two cells guarantee that no uncovered cell of
 * level l lies between a face leaving level l and a covered cell (so no
 * level-l ghost reads a covered value) and that every 5x5 ghost surface of
 * level l+1 lies inside level l. */
#define NEST 2

/* Tag cells of level l of hierarchy Ht (Sec. 4.2, AMR policies) by charge
 * density (Eq. tag_charge: |rho| >= lambda, mode 1; relative to the level
 * maximum, rho > lambda * max rho, mode 0), by potential (|phi| >= lambda
 * max |phi|, mode 3) or by electric field (|E_w| >= lambda max |E_w| for
 * some w in {x, y, z}, mode 4), maxima over the level's valid cells (a zero
 * maximum tags nothing); grow the tags by `buffer` cells (Chebyshev
 * distance), mark every aligned block of bc^3 cells of level l that holds a
 * grown tag, keep a block only if the block grown by NEST cells lies inside
 * the domain and inside the valid region of level l of hierarchy H (proper
 * nesting; H = Ht when a hierarchy is built, the new hierarchy when one is
 * regridded), and return the kept blocks refined by 2 as boxes of level l+1.
 * Boxes are listed in (k, j, i) block order. */
static int tag_level_from(ohier *H, const ohier *Ht, int l, int mode, double lambda, int buffer, int bc,
                          int **boxes_out)
{
    const olevel *tl = &Ht->L[l];
    olevel *lv = &H->L[l];
    double mx = -INFINITY, mphi = 0.0, me[3] = {0.0, 0.0, 0.0};
    for (int r = 0; r < tl->n; ++r) {
        if (tl->rho[r] > mx) mx = tl->rho[r];
        if (fabs(tl->phi[r]) > mphi) mphi = fabs(tl->phi[r]);
        for (int d = 0; d < 3; ++d)
            if (fabs(tl->ef[d][r]) > me[d]) me[d] = fabs(tl->ef[d][r]);
    }
    int64_t tot = level_box_cells(tl);
    int8_t *tag = (int8_t *)calloc((size_t)tot, 1);
    int ntag = 0;
    for (int r = 0; r < tl->n; ++r) {
        double v = tl->rho[r] * Ht->eps0;
        int t;
        if (mode == 1)
            t = fabs(v) >= lambda;
        else if (mode == 3)
            t = mphi > 0.0 && fabs(tl->phi[r]) >= lambda * mphi;
        else if (mode == 4) {
            t = 0;
            for (int d = 0; d < 3; ++d)
                if (me[d] > 0.0 && fabs(tl->ef[d][r]) >= lambda * me[d]) t = 1;
        } else
            t = mx > 0.0 && tl->rho[r] > lambda * mx;
        if (t) {
            const int *c = &tl->cell[3 * r];
            tag[pidx(tl, c[0], c[1], c[2])] = 1;
            ntag++;
        }
    }
    int nl = nlevcells(H, l);
    int nb = nl / bc;
    int blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) {
        int a = tl->lo[d] - buffer, b = tl->hi[d] + buffer;
        if (a < 0) a = 0;
        if (b > nl - 1) b = nl - 1;
        blo[d] = a / bc;
        bhi[d] = b / bc;
        if (bhi[d] > nb - 1) bhi[d] = nb - 1;
    }
    int cap = 64, cnt = 0;
    int *boxes = (int *)malloc(sizeof(int) * 6 * (size_t)cap);
    for (int bk = blo[2]; bk <= bhi[2]; ++bk)
        for (int bj = blo[1]; bj <= bhi[1]; ++bj)
            for (int bi = blo[0]; bi <= bhi[0]; ++bi) {
                int b3[3] = {bi, bj, bk};
                /* any grown tag inside the block? */
                int marked = 0;
                for (int k = bk * bc - buffer; k < bk * bc + bc + buffer && !marked; ++k)
                    for (int j = bj * bc - buffer; j < bj * bc + bc + buffer && !marked; ++j)
                        for (int i = bi * bc - buffer; i < bi * bc + bc + buffer && !marked; ++i) {
                            int64_t p = pidx(tl, i, j, k);
                            if (p >= 0 && tag[p]) marked = 1;
                        }
                if (!marked) continue;
                /* proper nesting: block grown by NEST cells inside the valid region */
                int ok = 1;
                for (int k = bk * bc - NEST; k < bk * bc + bc + NEST && ok; ++k)
                    for (int j = bj * bc - NEST; j < bj * bc + bc + NEST && ok; ++j)
                        for (int i = bi * bc - NEST; i < bi * bc + bc + NEST && ok; ++i) {
                            int c[3] = {i, j, k};
                            if (!in_domain(H, l, c) || !is_valid(lv, i, j, k)) ok = 0;
                        }
                if (!ok) continue;
                if (cnt == cap) {
                    cap *= 2;
                    boxes = (int *)realloc(boxes, sizeof(int) * 6 * (size_t)cap);
                }
                for (int d = 0; d < 3; ++d) {
                    boxes[6 * cnt + d] = 2 * bc * b3[d];
                    boxes[6 * cnt + 3 + d] = 2 * bc * b3[d] + 2 * bc - 1;
                }
                cnt++;
            }
    free(tag);
    (void)ntag;
    *boxes_out = boxes;
    return cnt;
}

static int tag_level(ohier *H, int l, int mode, double lambda, int buffer, int bc, int **boxes_out)
{
    return tag_level_from(H, H, l, mode, lambda, buffer, bc, boxes_out);
}

/* Build level l (l >= 1) as the union of boxes (level-l index space,
 * inclusive). Returns 0, or -1 on a nesting/alignment violation. */
static int build_level_from_boxes(ohier *H, int l, int nbox, const int *boxes)
{
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
    int n = nlevcells(H, l);
    for (int b = 0; b < nbox; ++b)
        for (int d = 0; d < 3; ++d) {
            int a = boxes[6 * b + d], e = boxes[6 * b + 3 + d];
            if (a < 0 || e >= n || a > e || (a & 1) || !(e & 1)) {
                snprintf(H->err, sizeof(H->err), "level %d box %d not aligned to coarse cells or outside", l, b);
                return -1;
            }
            if (a < lo[d]) lo[d] = a;
            if (e > hi[d]) hi[d] = e;
        }
    level_alloc_box(H, l, lo, hi);
    olevel *lv = &H->L[l];
    for (int b = 0; b < nbox; ++b)
        for (int k = boxes[6 * b + 2]; k <= boxes[6 * b + 5]; ++k)
            for (int j = boxes[6 * b + 1]; j <= boxes[6 * b + 4]; ++j)
                for (int i = boxes[6 * b + 0]; i <= boxes[6 * b + 3]; ++i)
                    lv->valid[pidx(lv, i, j, k)] = 1;
    /* proper nesting in level l-1: parent grown by NEST cells valid on l-1 */
    olevel *cv = &H->L[l - 1];
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                if (!is_valid(lv, i, j, k)) continue;
                int P[3] = {i >> 1, j >> 1, k >> 1};
                for (int c = -NEST; c <= NEST; ++c)
                    for (int b = -NEST; b <= NEST; ++b)
                        for (int a = -NEST; a <= NEST; ++a) {
                            int Q[3] = {P[0] + a, P[1] + b, P[2] + c};
                            if (!in_domain(H, l - 1, Q) || !is_valid(cv, Q[0], Q[1], Q[2])) {
                                snprintf(H->err, sizeof(H->err), "level %d not properly nested in level %d", l, l - 1);
                                return -1;
                            }
                        }
                cv->covered[pidx(cv, P[0], P[1], P[2])] = 1;
            }
    return 0;
}

/* ------------------------------------------------ ghost interpolation -- */

/* Bit patterns printed in Tab. bit_pattern (5x5 surface, label i + 5 j) and
 * Tab. Lagrange_2d_linear (3x3 surface, label i + 3 j), in table order. */
static const unsigned long QUAD_PATTERN[9] = {473536UL, 14798UL, 236768UL, 15153152UL, 947072UL,
                                              29596UL, 7399UL, 7576576UL, 30306304UL};
static const unsigned long LIN_PATTERN[4] = {27UL, 216UL, 432UL, 54UL};

/* Lagrange basis weights at t for nodes u[0..m-1]. */
static void lagrange_weights(int m, const double *u, double t, double *w)
{
    for (int i = 0; i < m; ++i) {
        double num = 1.0, den = 1.0;
        for (int k = 0; k < m; ++k)
            if (k != i) {
                num *= (t - u[k]);
                den *= (u[i] - u[k]);
            }
        w[i] = num / den;
    }
}

/* First column / row used by a pattern on a w x w surface. */
static void pattern_origin(unsigned long pat, int w, int *i0, int *j0)
{
    int imin = w, jmin = w;
    for (int j = 0; j < w; ++j)
        for (int i = 0; i < w; ++i)
            if (pat & (1UL << (i + w * j))) {
                if (i < imin) imin = i;
                if (j < jmin) jmin = j;
            }
    *i0 = imin;
    *j0 = jmin;
}

/* Coarse stencil of the intermediate value phi_int for the ghost of fine
 * cell f (level l >= 1) across its face (d, s), s = +-1 (step 1 of the
 * two-step interpolation of Eq. 2d_lagrange).  Writes up to 9 (coarse row,
 * weight) pairs, returns the count, and reports the order used
 * (2 quadratic, 1 linear, 0 constant). */
static int ghost_stencil(ohier *H, int l, const int f[3], int d, int s, int *cols, double *w, int *order)
{
    olevel *cv = &H->L[l - 1];
    int C[3] = {f[0] >> 1, f[1] >> 1, f[2] >> 1};
    C[d] += s;
    int ax[2], na = 0;
    for (int e = 0; e < 3; ++e)
        if (e != d) ax[na++] = e;
    double t[2];
    for (int e = 0; e < 2; ++e) t[e] = (f[ax[e]] & 1) ? 0.25 : -0.25;
    /* availability of the 5x5 surface through C perpendicular to d */
    unsigned long m25 = 0;
    for (int jj = 0; jj < 5; ++jj)
        for (int ii = 0; ii < 5; ++ii) {
            int Q[3] = {C[0], C[1], C[2]};
            Q[ax[0]] += ii - 2;
            Q[ax[1]] += jj - 2;
            if (in_domain(H, l - 1, Q) && is_valid(cv, Q[0], Q[1], Q[2]) && !is_covered(cv, Q[0], Q[1], Q[2]))
                m25 |= 1UL << (ii + 5 * jj);
        }
    for (int cs = 0; cs < 9; ++cs) {
        unsigned long pat = QUAD_PATTERN[cs];
        if ((m25 & pat) != pat) continue;
        int i0, j0;
        pattern_origin(pat, 5, &i0, &j0);
        double ua[3], ub[3], wa[3], wb[3];
        for (int m = 0; m < 3; ++m) {
            ua[m] = (double)(i0 + m - 2);
            ub[m] = (double)(j0 + m - 2);
        }
        lagrange_weights(3, ua, t[0], wa);
        lagrange_weights(3, ub, t[1], wb);
        int n = 0;
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                int Q[3] = {C[0], C[1], C[2]};
                Q[ax[0]] += (int)ua[a];
                Q[ax[1]] += (int)ub[b];
                cols[n] = row_of(cv, Q[0], Q[1], Q[2]);
                w[n] = wa[a] * wb[b];
                n++;
            }
        *order = 2;
        return n;
    }
    unsigned long m9 = 0;
    for (int jj = 0; jj < 3; ++jj)
        for (int ii = 0; ii < 3; ++ii)
            if (m25 & (1UL << ((ii + 1) + 5 * (jj + 1)))) m9 |= 1UL << (ii + 3 * jj);
    for (int cs = 0; cs < 4; ++cs) {
        unsigned long pat = LIN_PATTERN[cs];
        if ((m9 & pat) != pat) continue;
        int i0, j0;
        pattern_origin(pat, 3, &i0, &j0);
        double ua[2], ub[2], wa[2], wb[2];
        for (int m = 0; m < 2; ++m) {
            ua[m] = (double)(i0 + m - 1);
            ub[m] = (double)(j0 + m - 1);
        }
        lagrange_weights(2, ua, t[0], wa);
        lagrange_weights(2, ub, t[1], wb);
        int n = 0;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                int Q[3] = {C[0], C[1], C[2]};
                Q[ax[0]] += (int)ua[a];
                Q[ax[1]] += (int)ub[b];
                cols[n] = row_of(cv, Q[0], Q[1], Q[2]);
                w[n] = wa[a] * wb[b];
                n++;
            }
        *order = 1;
        return n;
    }
    cols[0] = row_of(cv, C[0], C[1], C[2]);
    w[0] = 1.0;
    *order = 0;
    return 1;
}

/* Normal-direction weights of step 2: quadratic through phi_1 (-3/2 h_f),
 * phi_0 (-1/2 h_f) and phi_int (+h_f, the coarse centre), at +1/2 h_f. */
static void normal_weights(double *w_int, double *w0, double *w1)
{
    double u[3] = {1.0, -0.5, -1.5}, w[3];
    lagrange_weights(3, u, 0.5, w);
    *w_int = w[0];
    *w0 = w[1];
    *w1 = w[2];
}

/* --------------------------------------------------- matrix assembly -- */

/* A fine cell f on level l with a face (d, s) leaving the level: its ghost
 * is w_int*I(phi^{l-1}) + w0*phi_f + w1*phi_f1, with f1 = f - s e_d.
 * Adds coef * (ghost) to row accumulators: fine part into `fine`, coarse
 * part into `crse`. */
static void add_ghost(ohier *H, int l, const int f[3], int d, int s, double coef, rowacc *fine, rowacc *crse,
                      int count_stats)
{
    double wi, w0, w1;
    normal_weights(&wi, &w0, &w1);
    olevel *lv = &H->L[l];
    int f1[3] = {f[0], f[1], f[2]};
    f1[d] -= s;
    int rf = row_of(lv, f[0], f[1], f[2]);
    int rf1 = row_of(lv, f1[0], f1[1], f1[2]);
    if (rf < 0 || rf1 < 0) {
        fprintf(stderr, "oracle: fine cell without inward neighbour\n");
        abort();
    }
    row_add(fine, rf, coef * w0);
    row_add(fine, rf1, coef * w1);
    int cols[9], order;
    double w[9];
    int n = ghost_stencil(H, l, f, d, s, cols, w, &order);
    if (count_stats) H->ghost_order_count[2 - order]++;
    for (int k = 0; k < n; ++k) {
        if (cols[k] < 0) {
            fprintf(stderr, "oracle: ghost stencil uses an invalid coarse cell\n");
            abort();
        }
        row_add(crse, cols[k], coef * wi * w[k]);
    }
}

static void assemble_level(ohier *H, int l)
{
    olevel *lv = &H->L[l];
    int lmax = H->nlev - 1;
    int n = lv->n;
    int nc = (l > 0) ? H->L[l - 1].n : 0;
    int nf = (l < lmax) ? H->L[l + 1].n : 0;
    double h = lv->h, ih2 = 1.0 / (h * h);
    csr_init(&lv->Anf, n, n);
    csr_init(&lv->Acomp, n, n);
    csr_init(&lv->Bcrse, n, nc);
    csr_init(&lv->Bfine, n, nf);
    csr_init(&lv->R, n, nf);
    csr_init(&lv->I, n, nc);
    for (int d = 0; d < 3; ++d) {
        csr_init(&lv->G[d], n, n);
        csr_init(&lv->Gc[d], n, nc);
    }
    rowacc anf, bcr, acp, bfi, bcr2, rr, ii, g, gc;
    for (int r = 0; r < n; ++r) {
        const int *x = &lv->cell[3 * r];
        int cov = is_covered(lv, x[0], x[1], x[2]);
        anf.n = bcr.n = acp.n = bfi.n = bcr2.n = 0;
        /* A_nf and B_crse: 7-point Laplacian, ghost alpha phi_0 at the
         * domain faces, Lagrange ghost at faces leaving the level. */
        for (int d = 0; d < 3; ++d)
            for (int s = -1; s <= 1; s += 2) {
                int nb[3] = {x[0], x[1], x[2]};
                nb[d] += s;
                if (!in_domain(H, l, nb) && H->periodic) {
                    int wb[3];
                    wrap_cell(H, l, nb, wb);
                    row_add(&anf, r, ih2);
                    row_add(&anf, row_of(lv, wb[0], wb[1], wb[2]), -ih2);
                } else if (!in_domain(H, l, nb)) {
                    /* A = -L; L gets (alpha phi_0 - phi_0)/h^2 */
                    row_add(&anf, r, (1.0 - phys_ghost(H, l)) * ih2);
                } else if (is_valid(lv, nb[0], nb[1], nb[2])) {
                    row_add(&anf, r, ih2);
                    row_add(&anf, row_of(lv, nb[0], nb[1], nb[2]), -ih2);
                } else {
                    /* A = -L; L gets (ghost - phi_0)/h^2 */
                    row_add(&anf, r, ih2);
                    add_ghost(H, l, x, d, s, -ih2, &anf, &bcr, 1);
                }
            }
        csr_put_row(&lv->Anf, r, &anf);
        csr_put_row(&lv->Bcrse, r, &bcr);
        /* A_comp and B_fine on uncovered cells of a non-finest level: faces to
         * covered cells use the fine-averaged flux of Eq. flux_differencing. */
        if (l == lmax) {
            csr_put_row(&lv->Acomp, r, &anf);
        } else if (!cov) {
            for (int d = 0; d < 3; ++d)
                for (int s = -1; s <= 1; s += 2) {
                    int nb[3] = {x[0], x[1], x[2]};
                    nb[d] += s;
                    if (!in_domain(H, l, nb) && H->periodic) {
                        int wb[3];
                        wrap_cell(H, l, nb, wb);
                        if (is_covered(lv, wb[0], wb[1], wb[2])) {
                            fprintf(stderr, "oracle: covered periodic image\n");
                            abort();
                        }
                        row_add(&acp, r, ih2);
                        row_add(&acp, row_of(lv, wb[0], wb[1], wb[2]), -ih2);
                    } else if (!in_domain(H, l, nb)) {
                        row_add(&acp, r, (1.0 - phys_ghost(H, l)) * ih2);
                    } else if (is_valid(lv, nb[0], nb[1], nb[2]) && !is_covered(lv, nb[0], nb[1], nb[2])) {
                        row_add(&acp, r, ih2);
                        row_add(&acp, row_of(lv, nb[0], nb[1], nb[2]), -ih2);
                    } else if (is_valid(lv, nb[0], nb[1], nb[2])) {
                        /* covered neighbour: L gets (1/h_c) * (1/4) sum_k
                         * (phi_fk - ghost_k)/h_f = 1/(2 h_c^2) sum_k (...) */
                        double c = 0.5 * ih2;
                        for (int tb = 0; tb < 2; ++tb)
                            for (int ta = 0; ta < 2; ++ta) {
                                int fk[3];
                                int ax[2], na = 0;
                                for (int e = 0; e < 3; ++e)
                                    if (e != d) ax[na++] = e;
                                fk[d] = 2 * nb[d] + (s > 0 ? 0 : 1);
                                fk[ax[0]] = 2 * x[ax[0]] + ta;
                                fk[ax[1]] = 2 * x[ax[1]] + tb;
                                int rfk = row_of(&H->L[l + 1], fk[0], fk[1], fk[2]);
                                /* A = -L: -c * phi_fk + c * ghost_k, the ghost of fk
                                 * across its face (d, -s) towards this cell */
                                row_add(&bfi, rfk, -c);
                                add_ghost(H, l + 1, fk, d, -s, c, &bfi, &acp, 0);
                            }
                    } else {
                        row_add(&acp, r, ih2);
                        add_ghost(H, l, x, d, s, -ih2, &acp, &bcr2, 0);
                    }
                }
            csr_put_row(&lv->Acomp, r, &acp);
            csr_put_row(&lv->Bfine, r, &bfi);
        }
        /* R: 8-cell average onto covered cells */
        if (l < lmax && cov) {
            rr.n = 0;
            for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a)
                        row_add(&rr, row_of(&H->L[l + 1], 2 * x[0] + a, 2 * x[1] + b, 2 * x[2] + c), 0.125);
            csr_put_row(&lv->R, r, &rr);
        }
        /* I: piecewise-constant prolongation from the parent */
        if (l > 0) {
            ii.n = 0;
            row_add(&ii, row_of(&H->L[l - 1], x[0] >> 1, x[1] >> 1, x[2] >> 1), 1.0);
            csr_put_row(&lv->I, r, &ii);
        }
        /* G_d: central difference (phi_{+d} - phi_{-d}) / (2h), ghosts as in A_nf */
        for (int d = 0; d < 3; ++d) {
            g.n = gc.n = 0;
            for (int s = -1; s <= 1; s += 2) {
                double c = 0.5 * s / h;
                int nb[3] = {x[0], x[1], x[2]};
                nb[d] += s;
                if (!in_domain(H, l, nb) && H->periodic) {
                    int wb[3];
                    wrap_cell(H, l, nb, wb);
                    row_add(&g, row_of(lv, wb[0], wb[1], wb[2]), c);
                } else if (!in_domain(H, l, nb)) {
                    row_add(&g, r, c * phys_ghost(H, l));
                } else if (is_valid(lv, nb[0], nb[1], nb[2])) {
                    row_add(&g, row_of(lv, nb[0], nb[1], nb[2]), c);
                } else {
                    add_ghost(H, l, x, d, s, c, &g, &gc, 0);
                }
            }
            csr_put_row(&lv->G[d], r, &g);
            csr_put_row(&lv->Gc[d], r, &gc);
        }
    }
    csr_finish(&lv->Anf);
    csr_finish(&lv->Acomp);
    csr_finish(&lv->Bcrse);
    csr_finish(&lv->Bfine);
    csr_finish(&lv->R);
    csr_finish(&lv->I);
    for (int d = 0; d < 3; ++d) {
        csr_finish(&lv->G[d]);
        csr_finish(&lv->Gc[d]);
    }
}

/* --------------------------------------------------------- algorithms -- */

static void vzero(double *v, int n) { memset(v, 0, sizeof(double) * (size_t)(n > 0 ? n : 1)); }
static void vcopy(double *dst, const double *src, int n) { memcpy(dst, src, sizeof(double) * (size_t)(n > 0 ? n : 1)); }

/* Alg. 1 RESIDUAL(l) into out (length n_l). */
static void residual_into(ohier *H, int l, double *out)
{
    olevel *lv = &H->L[l];
    int lmax = H->nlev - 1;
    vcopy(out, lv->rho, lv->n);
    if (l == lmax) {
        csr_axpy(&lv->Anf, -1.0, lv->phi, out);
        if (l > 0) csr_axpy(&lv->Bcrse, -1.0, H->L[l - 1].phi, out);
    } else {
        csr_axpy(&lv->Acomp, -1.0, lv->phi, out);
        if (l > 0) csr_axpy(&lv->Bcrse, -1.0, H->L[l - 1].phi, out);
        csr_axpy(&lv->Bfine, -1.0, H->L[l + 1].phi, out);
        for (int r = 0; r < lv->n; ++r) {
            const int *c = &lv->cell[3 * r];
            if (is_covered(lv, c[0], c[1], c[2])) out[r] = 0.0;
        }
    }
}

/* Red-black Gauss-Seidel on A_nf^l x = b: colour = parity of i+j+k, red
 * (even) first; nu sweeps of (red, black). */
static void smooth(ohier *H, int l, double *x, const double *b, int nu)
{
    olevel *lv = &H->L[l];
    const csr *A = &lv->Anf;
    /* the cells of one colour couple only to the other colour (A_nf has no
     * same-colour entries), so they are updated independently */
    for (int it = 0; it < nu; ++it)
        for (int colour = 0; colour < 2; ++colour)
#pragma omp parallel for schedule(static) if (lv->n > PAR_MIN)
            for (int r = 0; r < lv->n; ++r) {
                const int *c = &lv->cell[3 * r];
                if (((c[0] + c[1] + c[2]) & 1) != colour) continue;
                double diag = 0.0, s = b[r];
                for (int p = A->ptr[r]; p < A->ptr[r + 1]; ++p) {
                    if (A->col[p] == r)
                        diag += A->val[p];
                    else
                        s -= A->val[p] * x[A->col[p]];
                }
                x[r] = s / diag;
            }
}

/* sum_i u_i v_i, summed in blocks of DOT_BLOCK rows: partial sums in
 * parallel, then added in block order. */
static double dot(const double *u, const double *v, int n)
{
    int nb = (n + DOT_BLOCK - 1) / DOT_BLOCK;
    double *part = (double *)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static) if (nb > 2)
    for (int b = 0; b < nb; ++b) {
        int i1 = (b + 1) * DOT_BLOCK < n ? (b + 1) * DOT_BLOCK : n;
        double s = 0.0;
        for (int i = b * DOT_BLOCK; i < i1; ++i) s += u[i] * v[i];
        part[b] = s;
    }
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    free(part);
    return s;
}

/* Conjugate gradients on A_nf^0 x = b (level 0 is symmetric positive
 * definite with the Dirichlet or Robin ghosts, |alpha| < 1), from x = 0,
 * until
 * ||b - A x||_2 <= rtol ||b||_2. */
static int bottom_cg(ohier *H, double *x, const double *b, double rtol, int maxit)
{
    olevel *lv = &H->L[0];
    int n = lv->n;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *Ap = (double *)malloc(sizeof(double) * (size_t)n);
    vzero(x, n);
    vcopy(r, b, n);
    if (H->periodic) {
        /* singular level 0: solve for the mean-free part of b */
        double m = 0.0;
        for (int i = 0; i < n; ++i) m += r[i];
        m /= n;
        for (int i = 0; i < n; ++i) r[i] -= m;
    }
    vcopy(p, r, n);
    double rr = dot(r, r, n), bb;
    bb = rr;
    int it = 0;
    if (bb > 0.0) {
        for (it = 0; it < maxit && rr > rtol * rtol * bb; ++it) {
            vzero(Ap, n);
            csr_axpy(&lv->Anf, 1.0, p, Ap);
            double pAp = dot(p, Ap, n);
            double alpha = rr / pAp;
#pragma omp parallel for schedule(static) if (n > PAR_MIN)
            for (int i = 0; i < n; ++i) {
                x[i] += alpha * p[i];
                r[i] -= alpha * Ap[i];
            }
            double rr2 = dot(r, r, n);
            double beta = rr2 / rr;
            rr = rr2;
#pragma omp parallel for schedule(static) if (n > PAR_MIN)
            for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        }
    }
    free(r);
    free(p);
    free(Ap);
    return it;
}

typedef struct {
    int nu1, nu2;
    double bottom_rtol;
    int bottom_maxit;
} relax_opts;

/* Alg. 3 RELAX(l). */
static void relax(ohier *H, int l, const relax_opts *o)
{
    olevel *lv = &H->L[l];
    int lmax = H->nlev - 1;
    int n = lv->n;
    if (l == lmax) {
        vcopy(lv->res, lv->rho, n);
        csr_axpy(&lv->Anf, -1.0, lv->phi, lv->res);
        if (l > 0) csr_axpy(&lv->Bcrse, -1.0, H->L[l - 1].phi, lv->res);
    }
    if (l > 0) {
        olevel *cv = &H->L[l - 1];
        double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        vcopy(lv->phisave, lv->phi, n);
        vzero(cv->err, cv->n);
        vzero(lv->err, n);
        smooth(H, l, lv->err, lv->res, o->nu1);
        for (int i = 0; i < n; ++i) lv->phi[i] += lv->err[i];
        /* restrict on the covered domain: R (r - A_nf e - B_crse e^{l-1}) */
        vcopy(tmp, lv->res, n);
        csr_axpy(&lv->Anf, -1.0, lv->err, tmp);
        csr_axpy(&lv->Bcrse, -1.0, cv->err, tmp);
        double *rc = (double *)calloc((size_t)(cv->n > 0 ? cv->n : 1), sizeof(double));
        csr_axpy(&cv->R, 1.0, tmp, rc);
        /* residual on the uncovered domain of level l-1 */
        double *ru = (double *)malloc(sizeof(double) * (size_t)(cv->n > 0 ? cv->n : 1));
        vcopy(ru, cv->rho, cv->n);
        csr_axpy(&cv->Acomp, -1.0, cv->phi, ru);
        if (l - 1 > 0) csr_axpy(&cv->Bcrse, -1.0, H->L[l - 2].phi, ru);
        csr_axpy(&cv->Bfine, -1.0, lv->phi, ru);
        for (int r = 0; r < cv->n; ++r) {
            const int *c = &cv->cell[3 * r];
            cv->res[r] = is_covered(cv, c[0], c[1], c[2]) ? rc[r] : ru[r];
        }
        free(rc);
        free(ru);
        relax(H, l - 1, o);
        /* e^l <- e^l + I e^{l-1} */
        csr_axpy(&lv->I, 1.0, cv->err, lv->err);
        /* r^l <- r^l - A_nf e^l - B_crse e^{l-1} */
        csr_axpy(&lv->Anf, -1.0, lv->err, lv->res);
        csr_axpy(&lv->Bcrse, -1.0, cv->err, lv->res);
        vzero(lv->de, n);
        smooth(H, l, lv->de, lv->res, o->nu2);
        for (int i = 0; i < n; ++i) {
            lv->err[i] += lv->de[i];
            lv->phi[i] = lv->phisave[i] + lv->err[i];
        }
        free(tmp);
    } else {
        bottom_cg(H, lv->err, lv->res, o->bottom_rtol, o->bottom_maxit);
        for (int i = 0; i < n; ++i) lv->phi[i] += lv->err[i];
    }
}

static double pnorm(const double *v, int n, int p)
{
    double s = 0.0;
    if (p == 0) {
        for (int i = 0; i < n; ++i)
            if (fabs(v[i]) > s) s = fabs(v[i]);
        return s;
    }
    if (p == 1) {
        for (int i = 0; i < n; ++i) s += fabs(v[i]);
        return s;
    }
    for (int i = 0; i < n; ++i) s += v[i] * v[i];
    return sqrt(s);
}

static void residual_all(ohier *H)
{
    for (int l = 0; l < H->nlev; ++l) residual_into(H, l, H->L[l].res);
}

/* ||r^l|| / ||rho^l|| per level (a zero ||rho^l|| uses the largest one). */
static double rel_residuals(ohier *H, int p, double *rel)
{
    double rn[MAXLEV], bn[MAXLEV], bmax = 0.0, worst = 0.0;
    for (int l = 0; l < H->nlev; ++l) {
        rn[l] = pnorm(H->L[l].res, H->L[l].n, p);
        bn[l] = pnorm(H->L[l].rho, H->L[l].n, p);
        if (bn[l] > bmax) bmax = bn[l];
    }
    for (int l = 0; l < H->nlev; ++l) {
        double b = bn[l] > 0.0 ? bn[l] : bmax;
        rel[l] = b > 0.0 ? rn[l] / b : rn[l];
        if (rel[l] > worst) worst = rel[l];
    }
    return worst;
}

static void average_down(ohier *H)
{
    for (int l = H->nlev - 2; l >= 0; --l) {
        olevel *lv = &H->L[l];
        double *rc = (double *)calloc((size_t)(lv->n > 0 ? lv->n : 1), sizeof(double));
        csr_axpy(&lv->R, 1.0, H->L[l + 1].phi, rc);
        for (int r = 0; r < lv->n; ++r) {
            const int *c = &lv->cell[3 * r];
            if (is_covered(lv, c[0], c[1], c[2])) lv->phi[r] = rc[r];
        }
        free(rc);
    }
}

static void efield(ohier *H)
{
    for (int l = 0; l < H->nlev; ++l) {
        olevel *lv = &H->L[l];
        for (int d = 0; d < 3; ++d) {
            vzero(lv->ef[d], lv->n);
            csr_axpy(&lv->G[d], -1.0, lv->phi, lv->ef[d]);
            if (l > 0) csr_axpy(&lv->Gc[d], -1.0, H->L[l - 1].phi, lv->ef[d]);
        }
    }
}

/* ------------------------------------------------------------ C entry -- */

static void hier_free(ohier *H)
{
    for (int l = 0; l < MAXLEV; ++l) {
        olevel *lv = &H->L[l];
        free(lv->valid);
        free(lv->covered);
        free(lv->row);
        free(lv->cell);
        free(lv->rho_pad);
        free(lv->rho);
        free(lv->phi);
        free(lv->res);
        free(lv->err);
        free(lv->phisave);
        free(lv->de);
        for (int d = 0; d < 3; ++d) free(lv->ef[d]);
        if (lv->Anf.ptr) {
            csr_free(&lv->Anf);
            csr_free(&lv->Acomp);
            csr_free(&lv->Bcrse);
            csr_free(&lv->Bfine);
            csr_free(&lv->R);
            csr_free(&lv->I);
            for (int d = 0; d < 3; ++d) {
                csr_free(&lv->G[d]);
                csr_free(&lv->Gc[d]);
            }
        }
    }
    free(H);
}

static char g_err[256];

const char *orc_last_error(void) { return g_err; }

/*
 * Create a hierarchy on the unit cube with n0^3 base cells.
 *   tag_mode 0: rho > lambda * max rho;  1: |rho| >= lambda (Eq. tag_charge);
 *   2: explicit boxes: boxes[nbox][7] = (level, lo[3], hi[3]) in that level's
 *      index space, inclusive.
 * Particles (may be np = 0) are deposited on every level as it is built.
 */
void *orc_create_bc(int n0, int lmax, int brick, int tag_mode, double lambda, int buffer, int nbox,
                    const int *boxes, const double *x, const double *y, const double *z, const double *q, long np,
                    double eps0, double robin_d)
{
    /* robin_d < 0 selects periodic faces */
    g_err[0] = 0;
    if (n0 < 4 || lmax < 0 || lmax >= MAXLEV || brick < 2 || (brick & 1) || (n0 % (brick / 2)) ||
        tag_mode < 0 || tag_mode > 2) {
        snprintf(g_err, sizeof(g_err), "invalid arguments");
        return NULL;
    }
    ohier *H = (ohier *)calloc(1, sizeof(ohier));
    H->n0 = n0;
    H->brick = brick;
    H->lmax_req = lmax;
    H->eps0 = eps0 > 0.0 ? eps0 : 1.0;
    H->robin_d = robin_d > 0.0 ? robin_d : 0.0;
    H->periodic = robin_d < 0.0;
    int lo[3] = {0, 0, 0}, hi[3] = {n0 - 1, n0 - 1, n0 - 1};
    level_alloc_box(H, 0, lo, hi);
    olevel *l0 = &H->L[0];
    for (int k = 0; k < n0; ++k)
        for (int j = 0; j < n0; ++j)
            for (int i = 0; i < n0; ++i) l0->valid[pidx(l0, i, j, k)] = 1;
    H->nlev = 1;
    /* levels are numbered only once their covered flags are final */
    int built = 0;
    for (int l = 1; l <= lmax; ++l) {
        int nb = 0, *bx = NULL, own = 0;
        if (tag_mode == 2) {
            bx = (int *)malloc(sizeof(int) * 6 * (size_t)(nbox > 0 ? nbox : 1));
            for (int b = 0; b < nbox; ++b)
                if (boxes[7 * b] == l) {
                    for (int e = 0; e < 6; ++e) bx[6 * nb + e] = boxes[7 * b + 1 + e];
                    nb++;
                }
            own = 1;
        } else {
            /* tagging needs rho on level l-1 */
            if (built < l) {
                level_number(H, l - 1);
                deposit_level(H, l - 1, x, y, z, q, np);
                built = l;
            }
            nb = tag_level(H, l - 1, tag_mode, lambda, buffer, brick / 2, &bx);
            own = 1;
        }
        if (nb == 0) {
            if (own) free(bx);
            break;
        }
        if (built >= l) {
            /* level l-1 was numbered for tagging; its covered flags change
             * now, which does not alter its numbering (valid cells only). */
        }
        if (build_level_from_boxes(H, l, nb, bx) != 0) {
            snprintf(g_err, sizeof(g_err), "%s", H->err);
            free(bx);
            hier_free(H);
            return NULL;
        }
        free(bx);
        H->nlev = l + 1;
    }
    for (int l = 0; l < H->nlev; ++l) {
        if (l >= built) level_number(H, l);
        deposit_level(H, l, x, y, z, q, np);
    }
    for (int l = 0; l < H->nlev; ++l) assemble_level(H, l);
    return H;
}

/* Regrid (Sec. 4.2): a new hierarchy with the old one's base grid, brick,
 * eps0 and faces whose level l+1 (l+1 <= lmax) is made of the blocks tagged
 * on the OLD level l by policy `mode` (0: rho > lambda max rho, 1: |rho| >=
 * lambda, 3: |phi| >= lambda max |phi|, 4: |E_w| >= lambda max |E_w|), from
 * the old level's current fields, kept under proper nesting in the NEW
 * level l; then the particles are deposited on every new level. */
void *orc_regrid(void *old, int mode, double lambda, int buffer, int lmax, const double *x, const double *y,
                 const double *z, const double *q, long np)
{
    g_err[0] = 0;
    const ohier *O = (const ohier *)old;
    if (!O || lmax < 0 || lmax >= MAXLEV || mode < 0 || mode > 4 || mode == 2 || buffer < 0) {
        snprintf(g_err, sizeof(g_err), "invalid arguments");
        return NULL;
    }
    ohier *H = (ohier *)calloc(1, sizeof(ohier));
    H->n0 = O->n0;
    H->brick = O->brick;
    H->lmax_req = lmax;
    H->eps0 = O->eps0;
    H->robin_d = O->robin_d;
    H->periodic = O->periodic;
    int n0 = O->n0;
    int lo[3] = {0, 0, 0}, hi[3] = {n0 - 1, n0 - 1, n0 - 1};
    level_alloc_box(H, 0, lo, hi);
    olevel *l0 = &H->L[0];
    for (int k = 0; k < n0; ++k)
        for (int j = 0; j < n0; ++j)
            for (int i = 0; i < n0; ++i) l0->valid[pidx(l0, i, j, k)] = 1;
    H->nlev = 1;
    for (int l = 1; l <= lmax && l - 1 < O->nlev; ++l) {
        int *bx = NULL;
        int nb = tag_level_from(H, O, l - 1, mode, lambda, buffer, H->brick / 2, &bx);
        if (nb == 0) {
            free(bx);
            break;
        }
        if (build_level_from_boxes(H, l, nb, bx) != 0) {
            snprintf(g_err, sizeof(g_err), "%s", H->err);
            free(bx);
            hier_free(H);
            return NULL;
        }
        free(bx);
        H->nlev = l + 1;
    }
    for (int l = 0; l < H->nlev; ++l) {
        level_number(H, l);
        deposit_level(H, l, x, y, z, q, np);
    }
    for (int l = 0; l < H->nlev; ++l) assemble_level(H, l);
    return H;
}

/* orc_create_bc with homogeneous Dirichlet faces. */
void *orc_create(int n0, int lmax, int brick, int tag_mode, double lambda, int buffer, int nbox,
                 const int *boxes, const double *x, const double *y, const double *z, const double *q, long np,
                 double eps0)
{
    return orc_create_bc(n0, lmax, brick, tag_mode, lambda, buffer, nbox, boxes, x, y, z, q, np, eps0, 0.0);
}

/* Threads of the parallel loops (ignored without OpenMP); returns the
 * number in use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void orc_destroy(void *h)
{
    if (h) hier_free((ohier *)h);
}

int orc_nlevels(void *h) { return ((ohier *)h)->nlev; }

/* Valid bounding box and cell count of level l. */
void orc_level_box(void *h, int l, int *lo, int *hi, int *n)
{
    olevel *lv = &((ohier *)h)->L[l];
    for (int d = 0; d < 3; ++d) {
        lo[d] = lv->lo[d];
        hi[d] = lv->hi[d];
    }
    *n = lv->n;
}

static double *field_ptr(olevel *lv, int f)
{
    switch (f) {
    case 0: return lv->rho;
    case 1: return lv->phi;
    case 2: return lv->res;
    case 3: return lv->ef[0];
    case 4: return lv->ef[1];
    case 5: return lv->ef[2];
    case 6: return lv->err;
    default: return NULL;
    }
}

/* Fields: 0 rho, 1 phi, 2 residual, 3-5 E, 6 error.  Dense layout over the
 * valid bounding box, i fastest; invalid cells read as 0 and are ignored on
 * write.  rho is stored as rho/eps0. */
int orc_get_field(void *h, int l, int f, double *out)
{
    ohier *H = (ohier *)h;
    olevel *lv = &H->L[l];
    double *v = field_ptr(lv, f);
    if (!v) return -1;
    int nx = lv->hi[0] - lv->lo[0] + 1, ny = lv->hi[1] - lv->lo[1] + 1, nz = lv->hi[2] - lv->lo[2] + 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int r = row_of(lv, lv->lo[0] + i, lv->lo[1] + j, lv->lo[2] + k);
                out[((int64_t)k * ny + j) * nx + i] = r >= 0 ? v[r] : 0.0;
            }
    return 0;
}

int orc_set_field(void *h, int l, int f, const double *in)
{
    ohier *H = (ohier *)h;
    olevel *lv = &H->L[l];
    double *v = field_ptr(lv, f);
    if (!v) return -1;
    int nx = lv->hi[0] - lv->lo[0] + 1, ny = lv->hi[1] - lv->lo[1] + 1, nz = lv->hi[2] - lv->lo[2] + 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int r = row_of(lv, lv->lo[0] + i, lv->lo[1] + j, lv->lo[2] + k);
                if (r >= 0) v[r] = in[((int64_t)k * ny + j) * nx + i];
            }
    return 0;
}

/* 0 outside the level, 1 valid and uncovered, 2 valid and covered. */
void orc_get_mask(void *h, int l, int8_t *out)
{
    olevel *lv = &((ohier *)h)->L[l];
    int nx = lv->hi[0] - lv->lo[0] + 1, ny = lv->hi[1] - lv->lo[1] + 1, nz = lv->hi[2] - lv->lo[2] + 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int gi = lv->lo[0] + i, gj = lv->lo[1] + j, gk = lv->lo[2] + k;
                int8_t m = 0;
                if (is_valid(lv, gi, gj, gk)) m = is_covered(lv, gi, gj, gk) ? 2 : 1;
                out[((int64_t)k * ny + j) * nx + i] = m;
            }
}

void orc_deposit(void *h, const double *x, const double *y, const double *z, const double *q, long np)
{
    ohier *H = (ohier *)h;
    for (int l = 0; l < H->nlev; ++l) deposit_level(H, l, x, y, z, q, np);
}

/* Alg. 2 SOLVE: returns the number of V-cycles; rel[] gets the final
 * per-level relative residuals.  If warm == 0 phi starts from zero.
 * Average-down and E are applied at the end. */
/* Volume mean of a per-level field over the composite domain (uncovered
 * valid cells of every level, all valid cells of the finest; the unit cube
 * has volume 1). */
static double composite_mean(ohier *H, int which)
{
    double s = 0.0;
    for (int l = 0; l < H->nlev; ++l) {
        olevel *lv = &H->L[l];
        double v = lv->h * lv->h * lv->h;
        const double *a = which ? lv->phi : lv->rho;
        for (int r = 0; r < lv->n; ++r) {
            const int *c = &lv->cell[3 * r];
            if (l < H->nlev - 1 && is_covered(lv, c[0], c[1], c[2])) continue;
            s += a[r] * v;
        }
    }
    return s;
}

static void subtract_all(ohier *H, int which, double m)
{
    for (int l = 0; l < H->nlev; ++l) {
        double *a = which ? H->L[l].phi : H->L[l].rho;
        for (int r = 0; r < H->L[l].n; ++r) a[r] -= m;
    }
}

int orc_solve(void *h, double eps, int p, int imax, int nu1, int nu2, double bottom_rtol, int warm, double *rel)
{
    ohier *H = (ohier *)h;
    if (H->periodic) subtract_all(H, 0, composite_mean(H, 0)); /* neutralising background */
    if (!warm)
        for (int l = 0; l < H->nlev; ++l) vzero(H->L[l].phi, H->L[l].n);
    relax_opts o = {nu1, nu2, bottom_rtol, 100000};
    residual_all(H);
    int i = 0;
    double worst = rel_residuals(H, p, rel);
    while (i < imax && worst > eps) {
        relax(H, H->nlev - 1, &o);
        residual_all(H);
        worst = rel_residuals(H, p, rel);
        ++i;
    }
    average_down(H);
    if (H->periodic) subtract_all(H, 1, composite_mean(H, 1)); /* mean-free potential */
    efield(H);
    return i;
}

/* Alg. 1 on every level with the current phi; rel[] as in orc_solve. */
void orc_residual(void *h, int p, double *rel)
{
    ohier *H = (ohier *)h;
    residual_all(H);
    rel_residuals(H, p, rel);
}

void orc_average_down(void *h) { average_down((ohier *)h); }
void orc_efield(void *h) { efield((ohier *)h); }

/* Cloud-in-cell gather of E (and phi if phi_out != NULL) from the finest
 * level whose valid cells hold all 8 nodes of the particle. */
/* Buffer cells against the spurious self-force near coarse-fine faces (the
 * paper corrects it with buffer cells, citing Vay et al.): a particle is
 * interpolated from a refined level only if every cell within Chebyshev
 * distance b of its 8 cloud-in-cell nodes is valid there, else from the
 * next coarser level; b = 0 is the plain rule. */
void orc_set_gather_buffer(void *h, int b) { ((ohier *)h)->gather_buffer = b > 0 ? b : 0; }

void orc_gather(void *h, const double *x, const double *y, const double *z, long np, double *ex, double *ey,
                double *ez, double *phi_out)
{
    ohier *H = (ohier *)h;
    /* particles independent */
#pragma omp parallel for schedule(static) if (np > PAR_MIN)
    for (long p = 0; p < np; ++p) {
        double e[3] = {0, 0, 0}, ph = 0.0;
        for (int l = H->nlev - 1; l >= 0; --l) {
            olevel *lv = &H->L[l];
            double hh = lv->h;
            double s[3] = {x[p] / hh - 0.5, y[p] / hh - 0.5, z[p] / hh - 0.5};
            int i0[3];
            double w[3][2];
            for (int d = 0; d < 3; ++d) {
                double f = floor(s[d]);
                i0[d] = (int)f;
                w[d][1] = s[d] - f;
                w[d][0] = 1.0 - w[d][1];
            }
            /* the 8 nodes, and on a refined level every cell within
             * Chebyshev distance gather_buffer of them, must be valid */
            int ok = 1, bb = l > 0 ? H->gather_buffer : 0;
            for (int c = -bb; c < 2 + bb && ok; ++c)
                for (int b = -bb; b < 2 + bb && ok; ++b)
                    for (int a = -bb; a < 2 + bb && ok; ++a)
                        if (!is_valid(lv, i0[0] + a, i0[1] + b, i0[2] + c)) ok = 0;
            if (!ok && l > 0) continue;
            if (!ok) break; /* outside level 0's interior: E = 0 */
            for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        int r = row_of(lv, i0[0] + a, i0[1] + b, i0[2] + c);
                        double ww = w[0][a] * w[1][b] * w[2][c];
                        for (int d = 0; d < 3; ++d) e[d] += ww * lv->ef[d][r];
                        ph += ww * lv->phi[r];
                    }
            break;
        }
        ex[p] = e[0];
        ey[p] = e[1];
        ez[p] = e[2];
        if (phi_out) phi_out[p] = ph;
    }
}

/* Particle binning (the bin step of the field solve, before the deposit):
 * key of particle p = the brick (8^3 cells, counted from the lower corner of
 * the level's valid bounding box) holding the particle's cell, on the finest
 * level whose valid cells hold all 8 of its cloud-in-cell nodes, numbered
 * level after level (coarse first); 0xFFFFFFFF for a particle with no such
 * level.  perm lists the particles sorted by key, equal keys in particle
 * order (counting sort).  Returns the number of keys (bricks). */
#define ORC_BRICK 8
#define ORC_NOKEY 0xFFFFFFFFu
long orc_bin(void *h, const double *x, const double *y, const double *z, long np, unsigned *keys, long *perm)
{
    ohier *H = (ohier *)h;
    long off[MAXLEV + 1];
    int nb[MAXLEV][3];
    off[0] = 0;
    for (int l = 0; l < H->nlev; ++l) {
        for (int d = 0; d < 3; ++d) nb[l][d] = (H->L[l].hi[d] - H->L[l].lo[d] + 1 + ORC_BRICK - 1) / ORC_BRICK;
        off[l + 1] = off[l] + (long)nb[l][0] * nb[l][1] * nb[l][2];
    }
    const long nkeys = off[H->nlev];
    for (long p = 0; p < np; ++p) {
        const double pos[3] = {x[p], y[p], z[p]};
        unsigned key = ORC_NOKEY;
        for (int l = H->nlev - 1; l >= 0; --l) {
            olevel *lv = &H->L[l];
            int i0[3], cell[3];
            int finite = 1;
            for (int d = 0; d < 3; ++d) {
                if (!(fabs(pos[d]) < 1e6)) finite = 0; /* non-finite or far away: no key */
                double s = pos[d] / lv->h - 0.5;
                i0[d] = finite ? (int)floor(s) : 0;
                cell[d] = finite ? (int)floor(pos[d] / lv->h) : 0;
            }
            if (!finite) break;
            int ok = 1;
            for (int c = 0; c < 2 && ok; ++c)
                for (int b = 0; b < 2 && ok; ++b)
                    for (int a = 0; a < 2 && ok; ++a)
                        if (!is_valid(lv, i0[0] + a, i0[1] + b, i0[2] + c)) ok = 0;
            if (!ok) continue;
            int br[3];
            for (int d = 0; d < 3; ++d) br[d] = (cell[d] - lv->lo[d]) / ORC_BRICK;
            key = (unsigned)(off[l] + br[0] + (long)nb[l][0] * (br[1] + (long)nb[l][1] * br[2]));
            break;
        }
        keys[p] = key;
    }
    /* counting sort, stable: bucket nkeys collects the particles without a key */
    long *cnt = (long *)calloc((size_t)nkeys + 2, sizeof(long));
    for (long p = 0; p < np; ++p) cnt[(keys[p] == ORC_NOKEY ? nkeys : (long)keys[p]) + 1]++;
    for (long k = 0; k <= nkeys; ++k) cnt[k + 1] += cnt[k];
    for (long p = 0; p < np; ++p) perm[cnt[keys[p] == ORC_NOKEY ? nkeys : (long)keys[p]]++] = p;
    free(cnt);
    return nkeys;
}

/* Matrix export: which = 0 A_nf, 1 A_comp, 2 B_crse, 3 B_fine, 4 R, 5 I,
 * 6-8 G_d, 9-11 the coarse part of G_d.  With ptr == NULL only the sizes
 * are returned. */
int orc_matrix(void *h, int l, int which, int *nrows, int *ncols, int *nnz, int *ptr, int *col, double *val)
{
    olevel *lv = &((ohier *)h)->L[l];
    csr *m;
    switch (which) {
    case 0: m = &lv->Anf; break;
    case 1: m = &lv->Acomp; break;
    case 2: m = &lv->Bcrse; break;
    case 3: m = &lv->Bfine; break;
    case 4: m = &lv->R; break;
    case 5: m = &lv->I; break;
    case 6: case 7: case 8: m = &lv->G[which - 6]; break;
    case 9: case 10: case 11: m = &lv->Gc[which - 9]; break;
    default: return -1;
    }
    *nrows = m->nrows;
    *ncols = m->ncols;
    *nnz = m->nnz;
    if (ptr) {
        memcpy(ptr, m->ptr, sizeof(int) * (size_t)(m->nrows + 1));
        memcpy(col, m->col, sizeof(int) * (size_t)m->nnz);
        memcpy(val, m->val, sizeof(double) * (size_t)m->nnz);
    }
    return 0;
}

/* Cell coordinates of the vector rows of level l (3 ints per row). */
void orc_cells(void *h, int l, int *out)
{
    olevel *lv = &((ohier *)h)->L[l];
    memcpy(out, lv->cell, sizeof(int) * 3 * (size_t)lv->n);
}

/* How many fine ghosts used the quadratic, linear and constant stencils. */
void orc_ghost_stats(void *h, long *out)
{
    ohier *H = (ohier *)h;
    for (int i = 0; i < 3; ++i) out[i] = H->ghost_order_count[i];
}

/* Pattern decoding helpers exposed for the table pins. */
unsigned long orc_quad_pattern(int c) { return (c >= 0 && c < 9) ? QUAD_PATTERN[c] : 0; }
unsigned long orc_lin_pattern(int c) { return (c >= 0 && c < 4) ? LIN_PATTERN[c] : 0; }

/* Ghost stencil query for one fine cell/face of level l (tests). */
int orc_ghost_stencil(void *h, int l, int fi, int fj, int fk, int d, int s, int *cols, double *w, int *order)
{
    int f[3] = {fi, fj, fk};
    return ghost_stencil((ohier *)h, l, f, d, s, cols, w, order);
}
