// Device kernels of the AMR multigrid solve (sm_103a).
//
// Every stencil operation works on the dense padded level boxes described
// in amr_internal.h, x fastest (coalesced rows per warp).  Operator
// conventions: A = -L, residual r = b - A u, and for a cell p the 7-point
// flux-differenced stencil (Eq. lap_flux_differencing with the coarse fluxes
// of Eq. coarse_fluxes) is split as
//     (L u)_p = (S - D u_p) / h^2,   D = k / 3,
// where each face contributes
//     neighbour valid on the level          S += u_n,            k += 3
//     physical boundary (Dirichlet 0)       ghost -u_p:           k += 6
//     coarse-fine face (level l >= 1)       ghost (2/3) u_p - (1/5) u_o + C:
//                                           S -= u_o / 5,        k += 1
// (u_o the inward neighbour opposite the face; C the coarse part, the
// (8/15)-weighted step-1 interpolation of Eq. 2d_lagrange, added by the
// surface operation).  In composite mode a face towards a covered cell
// contributes nothing here: the surface operation adds the fine-averaged
// flux of Eq. flux_differencing.
//
// FP64 on this part runs about two lanes per SM and is charged per warp
// instruction, so the operations keep every lane of a warp on useful cells
// (one thread per cell of the colour being relaxed) and take a warp-uniform
// fast path (six plain neighbours: D = 6, 7 FP64 instructions per update);
// the general path reads D and 1/D from tables instead of converting and
// dividing.
//
// Each operation is a device function of one 128-thread block of a virtual
// grid.  It runs either as its own kernel (one launch per operation, chained
// by programmatic dependent launch, captured in CUDA graphs by the driver)
// or as a phase of the persistent program kernel k_program, which executes
// a recorded sequence of rounds of phases (from one or many hierarchies)
// separated by a bounded grid barrier, with the convergence loop on the
// device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "amr_internal.h"
#include "stencil.cuh"

namespace amr {

namespace {

constexpr int BX = 32, BY = 4, NT = BX * BY;
constexpr double kThird = 1.0 / 3.0;

// Programmatic dependent launch: wait until the preceding kernel in the
// stream has completed and its memory is visible, then let the next kernel
// be launched while this one runs (a no-op without the launch attribute).
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Row of the thread within its 32 x 4 virtual block.  Kernels whose blocks
// hold several virtual blocks (blockDim.y a multiple of 4) run one virtual
// block per group of four rows.
__device__ __forceinline__ int ty() { return threadIdx.y & (BY - 1); }
__device__ __forceinline__ int tid() { return ty() * BX + threadIdx.x; }

__host__ __device__ inline int64_t pad_index(const Grid &g, int i, int j, int k)
{
    return (int64_t)(k - g.lo[2] + 1) * g.sz + (int64_t)(j - g.lo[1] + 1) * g.sy + (i - g.lo[0] + 1);
}

// One thread per interior cell, numbered row by row within a z-plane, NT
// to a virtual block (plane_cell decodes it): short rows still fill whole
// warps, as in colour_grid below.
__host__ __device__ inline dim3 cell_grid(const Grid &g)
{
    const int64_t cells = (int64_t)(g.n[0] - 2) * (g.n[1] - 2);
    return dim3((unsigned)((cells + NT - 1) / NT), 1u, (unsigned)(g.n[2] - 2));
}

// Cell (a, b) of virtual block bx of cell_grid(g) in its plane; false past
// the plane's last cell (then a = b = 1, a valid index to read harmlessly).
__device__ __forceinline__ bool plane_cell(const Grid &g, int bx, int &a, int &b)
{
    const int nx = g.n[0] - 2, t = bx * NT + tid(), r = t / nx;
    const bool ok = r < g.n[1] - 2;
    a = 1 + (ok ? t - r * nx : 0);
    b = 1 + (ok ? r : 0);
    return ok;
}

// One thread per cell of one colour, numbered row by row within a z-plane
// (half the row extent per row), NT of them to a virtual block: short rows
// (a refined box is often only 30-50 cells wide) still fill whole warps,
// which matters because an FP64 instruction costs the same pipe time
// whatever the number of lanes it has work for.
__host__ __device__ inline int colour_half(const Grid &g) { return (g.n[0] - 2 + 1) / 2; }

__host__ __device__ inline dim3 colour_grid(const Grid &g)
{
    const int64_t cells = (int64_t)colour_half(g) * (g.n[1] - 2);
    return dim3((unsigned)((cells + NT - 1) / NT), 1u, (unsigned)(g.n[2] - 2));
}

unsigned elem_blocks(int64_t n)
{
    int64_t b = (n + NT - 1) / NT;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Offset to the periodic image across face f (0..5 = -x, +x, -y, +y, -z,
// +z) of a cell on that face of a domain-filling grid.
__device__ __forceinline__ int64_t wrap_off(const Grid &g, int f)
{
    const int d = f >> 1;
    const int64_t st = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
    const int64_t span = (int64_t)(g.n[d] - 3) * st;
    return (f & 1) ? -span : span;
}

// The general (not all-plain) stencil of a cell of a grid with periodic
// faces: a neighbour outside the grid is the cell on the opposite face.
// A separate branch, so that the other grids keep their own code path.
template <bool COMP, typename T>
__device__ __forceinline__ void stencil_S_periodic(const Grid &g, const T *u, int64_t p, bool act, T &S, int &k)
{
    const int64_t off[6] = {-1, 1, -g.sy, g.sy, -g.sz, g.sz};
    T c[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    int kk = 0;
    if (act) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            int64_t o = off[f];
            uint8_t m = g.mask[p + o];
            if (m == 0) {
                o = wrap_off(g, f);
                m = g.mask[p + o];
            }
            if constexpr (!COMP) m = m != 0; // A_nf: every valid neighbour takes part
            const bool valid = m == 1;
            c[f] = face_c(valid, m, g.dirichlet, valid ? u[p + o] : T(0), T(0), kk);
        }
    }
    S = sum6(c[0], c[1], c[2], c[3], c[4], c[5]);
    k = kk;
}

// S and the face code k of the split above, for an active cell p.  All 32
// lanes of the warp must call it (inactive lanes with act = false): the
// fast path (six plain neighbours, no mask tests) is taken when every active
// lane has them; it sums in the same tree as the general path.  PER: the
// grid has periodic faces (its own operations, so that the other grids'
// kernels carry no periodic code).
template <bool COMP, typename T, bool PER = false>
__device__ __forceinline__ void stencil_S(const Grid &g, const T *u, int64_t p, bool act, T &S, int &k)
{
    const int64_t off[6] = {-1, 1, -g.sy, g.sy, -g.sz, g.sz};
    if constexpr (!COMP) {
        // one neighbour-code byte instead of six mask reads
        unsigned cd = act ? g.code[p] : 0x7fu;
        if (__all_sync(0xffffffffu, (cd & 63u) == 63u)) {
            k = 18;
            S = act ? sum6(u[p - 1], u[p + 1], u[p - g.sy], u[p + g.sy], u[p - g.sz], u[p + g.sz]) : T(0);
            return;
        }
        if constexpr (PER) {
            stencil_S_periodic<false>(g, u, p, act, S, k);
            return;
        }
        T c[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        int kk = 0;
        if (act) {
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                bool valid = (cd >> f) & 1u;
                T un = valid ? u[p + off[f]] : T(0);
                T uo = (!valid && !g.dirichlet) ? u[p - off[f]] : T(0);
                c[f] = face_c(valid, (uint8_t)valid, g.dirichlet, un, uo, kk);
            }
        }
        S = sum6(c[0], c[1], c[2], c[3], c[4], c[5]);
        k = kk;
        return;
    }
    uint8_t m[6] = {1, 1, 1, 1, 1, 1};
    bool fast = true;
    if (act) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            m[f] = g.mask[p + off[f]];
            fast &= (m[f] == 1);
        }
    }
    if (__all_sync(0xffffffffu, fast)) {
        k = 18;
        S = act ? sum6(u[p - 1], u[p + 1], u[p - g.sy], u[p + g.sy], u[p - g.sz], u[p + g.sz]) : T(0);
        return;
    }
    if constexpr (PER) {
        stencil_S_periodic<true>(g, u, p, act, S, k);
        return;
    }
    T c[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    int kk = 0;
    if (act) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            bool valid = m[f] == 1;
            // the opposite cell is read only for a coarse-fine face
            T un = valid ? u[p + off[f]] : T(0);
            T uo = (!valid && m[f] == 0 && !g.dirichlet) ? u[p - off[f]] : T(0);
            c[f] = face_c(valid, m[f], g.dirichlet, un, uo, kk);
        }
    }
    S = sum6(c[0], c[1], c[2], c[3], c[4], c[5]);
    k = kk;
}

// Face code k of cell p from its neighbour code (for the first sweep from a
// zero iterate, which needs no neighbour values).
__device__ __forceinline__ int face_code(const Grid &g, int64_t p)
{
    int nv = __popc(g.code[p] & 63u);
    return 3 * nv + (6 - nv) * (g.dirichlet ? g.dirichlet : 1);
}

// ------------------------------------------------------- operation args

template <typename T>
struct ResidualA {
    Grid g;
    const T *rho, *u;
    T *r;
    int comp, zero_covered;
    int listed; // 1: one thread per entry of g.clist (both colours)
};

template <typename T>
struct RbgsA {
    Grid g;
    T *x;
    const T *rhs;
    int colour, mode; // mode 1: e += x, phi += x; mode 2: phi += x (updated cells)
    T *e, *phi;
    int listed; // 1: one thread per entry of g.clist (the launch grid covers the list)
};

template <typename T>
struct RestrictA {
    Grid gf, gc;
    int clo[3], cn[3];
    T *rf;
    const T *ef;
    T *phif, *rc;
    const int *cov; // non-null: one thread per entry (the covered cells of gc, padded indices)
    int ncov;
};

template <typename T>
struct ProlongA {
    Grid gf, gc;
    T *ef, *rf, *phif;
    const T *ec;
    int listed; // 1: one thread per entry of gf.clist (both colours)
};

// Grid-stride element-wise operations (stride = virtual blocks x 128).
template <typename T>
struct ElemA {
    int64_t n, stride;
    int kind; // 0 fill a = v; 1 a += v * b; 2 a += b and c += b
    T v;
    T *a;
    const T *b;
    T *c;
};

struct ConvA {
    int64_t n, stride;
    int kind; // 0: rho32 = res32 = r64, phi32 = 0;  1: phi64 += phi32
    const uint8_t *mask; // cells outside the level (mask 0) are skipped
    const double *r64;
    double *phi64;
    float *rho32, *res32, *phi32;
};

template <typename T>
struct CpA {
    int nface;
    const int8_t *cnt;
    const int *cidx;
    const double *cw;
    const T *uc;
    double *cp;
};

template <typename T>
struct SurfaceA {
    // fine side: r_f += scale_f * sum of the cell's cp
    int ncell;
    const int *cell_f, *cell_ptr;
    const double *cp_f;
    T *rf;
    double scale_f;
    // coarse side: r_C += scale_c * sum over C's fine faces of
    // (u_f - ghost_f) = (1/3) u_f + (1/5) u_f1 - cp
    int ncrse;
    const int *crse_c, *crse_ptr, *crse_face, *ff, *ff1;
    const double *cp_c;
    const T *uf;
    T *rc;
    double scale_c;
};

struct GradA {
    Grid g;
    const double *u;
    double *e0, *e1, *e2;
};

struct CfGradA {
    int ncell;
    const int *cell_f, *cell_ptr;
    const int8_t *dir;
    const double *cp;
    double *e0, *e1, *e2;
    double inv2h;
};

struct AvgDownA {
    Grid gf, gc;
    int clo[3], cn[3];
    const double *uf;
    double *uc;
};

struct NormA {
    int nslots, nblocks; // partial blocks used per slot (<= kPartialBlocks)
    int vec;             // every v[] 16-byte and every mask[] 4-byte aligned
    int64_t n[2 * kMaxLevels];
    const uint8_t *mask[2 * kMaxLevels];
    const double *v[2 * kMaxLevels];
    int covered_too[2 * kMaxLevels];
    const SolveParams *prm; // the norm p selects which partial is formed
    double *part;
};

struct CheckA {
    const double *part;
    int nlev, with_rho, is_body, use_cond, nblocks;
    const SolveParams *prm;
    SolveState *st;
    cudaGraphConditionalHandle cond;
};

template <typename T>
struct MgRestrictA {
    Grid gf, gc;
    const T *ef, *rf;
    T *rc, *ec;
    int first_red; // also the first red pass on grid gc from a zero iterate
};

template <typename T>
struct MgProlongA {
    Grid gf, gc;
    T *ef;
    const T *ec;
};

template <typename T>
struct CoarseA {
    Grid g;
    int m;
    const double *M;
    const T *r;
    T *e;
};

// Separable solve of the coarsest multigrid grid (n^3 cells, n > 11): one
// pass applies an n x n matrix along one axis, out_c = sum_q M[c n + q]
// in_q for every line; the pass with lam != null also divides by the
// eigenvalue sum of the mode, (lam_i + lam_j + lam_k) / h^2 (plus zero_add
// at mode (0, 0, 0), the regularisation of periodic faces).
template <typename TI, typename TO>
struct AxisA {
    int n, axis;
    int64_t sy, sz; // padded strides of the grid
    const TI *in;
    TO *out;
    const double *M;
    const double *lam; // n eigenvalues of the 1-D operator, or null
    double h2, zero_add;
};

struct DepositA {
    int nlev;
    Grid g[kMaxLevels];
    double ih[kMaxLevels], ih3[kMaxLevels]; // 1/h and 1/h^3 per level
    int lg[kMaxLevels];                     // log2 of 1/h per level, -1 unless a power of two
    double *rho[kMaxLevels];
    int *outside;
    double inv_eps0;
    const double *x, *y, *z, *q;
    int64_t n;
};

// Level-0 exact bottom solve (see op_dst / op_triz): a sine transform of
// lines of the n^3 interior (along x or y) by the n x n matrix MT
// (out_m = sum_i MT[i n + m] in_i), and per (kx, ky) mode a tridiagonal
// solve along z.
template <typename TI, typename TO>
struct DstA {
    int n, axis;      // interior extent of the cube; 0: lines along x, 1: along y
    int inv;          // 0: forward (MT[i n + m] = S[m][i]), 1: inverse (MT[m n + i] = S[m][i])
    int64_t sy, sz;   // padded strides
    const TI *in;
    TO *out;
    const double *MT;
    TO *phi;          // non-null: also phi += out
};

// Fast sine transform of the level-0 lines (n a power of two, 32 <= n <= 256;
// see op_fdst): L lines of the interior per virtual block.
template <typename TI, typename TO>
struct FdstA {
    int n, lg;        // interior extent and log2(n)
    int L;            // lines per virtual block (L n = kFdstElems)
    int axis;         // 0: lines along x, 1: along y
    int inv;          // 0: forward, 1: inverse
    int64_t sy, sz;   // padded strides
    const TI *in;
    TO *out;
    const double *tab; // [n - 1] stage factors 1 / (2 cos(pi (2i+1) / (2M))) by block size M
    TO *phi;          // non-null: also phi += out (inverse only)
};

struct TrizA {
    int n;
    int64_t sy, sz;
    double *u;        // rhs in, solution out (in place)
    const double *iw; // [part][k][mode] reciprocal pivots of the two half systems
    double h2;
    const double *fm; // non-null: per-mode factor replacing h2 (h^2 times the
                      // transforms' basis scales, which the fast transforms leave out)
};

struct GatherA {
    int nlev;
    Grid g[kMaxLevels];
    double ih[kMaxLevels]; // 1/h per level
    int lg[kMaxLevels];    // log2 of 1/h per level, -1 unless a power of two
    const double *e[kMaxLevels][3];
    const double *phi[kMaxLevels];
    const double *x, *y, *z;
    int64_t n;
    double *ex, *ey, *ez, *phio;
};

// ------------------------------------------------------------ operations

template <typename T, bool PER = false>
__device__ __forceinline__ void op_residual(const ResidualA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &g = A.g;
    bool in;
    int64_t p;
    if (A.listed) {
        const int t = bx * NT + tid();
        in = t < g.ccnt[0] + g.ccnt[1];
        if (!__any_sync(0xffffffffu, in)) return;
        p = in ? g.clist[t] : g.sz + g.sy + 1;
    } else {
        int a, b;
        in = plane_cell(g, bx, a, b); // lanes past the plane stay (warp votes below)
        p = (int64_t)(1 + bz) * g.sz + (int64_t)b * g.sy + a;
    }
    uint8_t m = in ? g.mask[p] : 0;
    if (A.comp && m == 2 && A.zero_covered) A.r[p] = T(0);
    bool act = m == 1 || (!A.comp && m == 2);
    T S;
    int k;
    if (A.comp)
        stencil_S<true, T, PER>(g, A.u, p, act, S, k);
    else
        stencil_S<false, T, PER>(g, A.u, p, act, S, k);
    if (act) A.r[p] = A.rho[p] + gih2<T>(g) * (S - diagD<T>(g, k) * A.u[p]);
}

template <typename T>
__device__ __forceinline__ void rbgs_store(const RbgsA<T> &A, int64_t p, T v)
{
    A.x[p] = v;
    if (A.mode == 1) {
        A.e[p] += v;
        A.phi[p] += v;
    } else if (A.mode == 2) {
        A.phi[p] += v;
    }
}

template <typename T, bool PER = false>
__device__ __forceinline__ void op_rbgs(const RbgsA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &g = A.g;
    if (A.listed) {
        // entry t of this colour's list: every lane of a warp but those
        // past the list's end has a valid cell
        const int t = bx * NT + tid(), n = g.ccnt[A.colour];
        const bool act = t < n;
        if (!__any_sync(0xffffffffu, act)) return;
        const int64_t p = act ? g.clist[(A.colour ? g.ccnt[0] : 0) + t] : g.sz + g.sy + 1;
        T S;
        int k;
        stencil_S<false, T, PER>(g, A.x, p, act, S, k);
        if (act) rbgs_store(A, p, gs_update(g, S, gh2<T>(g), A.rhs[p], k));
        return;
    }
    // colour cell t of plane c (see colour_grid); lanes past the plane's
    // last cell stay in the warp with act = false
    const int half = colour_half(g), t = bx * NT + tid(), r = t / half;
    const bool row_ok = r < g.n[1] - 2;
    int b = 1 + (row_ok ? r : 0);
    int c = 1 + bz;
    int base = g.lo[0] + g.lo[1] + g.lo[2] + b + c - 3;
    int a = 1 + 2 * (t - r * half) + ((A.colour + 1 + base) & 1);
    bool in = row_ok && a < g.n[0] - 1;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + (in ? a : 1);
    bool act = in && g.mask[p] != 0;
    T S;
    int k;
    stencil_S<false, T, PER>(g, A.x, p, act, S, k);
    if (act) rbgs_store(A, p, gs_update(g, S, gh2<T>(g), A.rhs[p], k));
}

// Red pass from a zero iterate: red cells get h^2 b / D (their neighbours
// are black, i.e. zero), black cells are set to zero.  One thread per cell.
template <typename T>
__device__ __forceinline__ void op_rbgs_first(const RbgsA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &g = A.g;
    if (A.listed) {
        // both colours' lists in one launch: red entries get h^2 b / D,
        // black ones zero
        const int t = bx * NT + tid();
        if (t >= g.ccnt[0] + g.ccnt[1]) return;
        const int64_t p = g.clist[t];
        if (t >= g.ccnt[0])
            A.x[p] = T(0);
        else
            rbgs_store(A, p, gs_update(g, T(0), gh2<T>(g), A.rhs[p], face_code(g, p)));
        return;
    }
    int a, b;
    if (!plane_cell(g, bx, a, b)) return;
    int c = 1 + bz;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
    if (g.mask[p] == 0) return;
    if (((g.lo[0] + g.lo[1] + g.lo[2] + a + b + c - 3) & 1) != 0) {
        A.x[p] = T(0);
        return;
    }
    rbgs_store(A, p, gs_update(g, T(0), gh2<T>(g), A.rhs[p], face_code(g, p)));
}

// Alg. 3 after the pre-smooth, one thread per covered coarse cell P of
// level l-1: for the 8 children f, t_f = r_f - (A_nf e)_f (homogeneous
// coarse-fine ghosts, e^{l-1} = 0), stored back into r_f; phi_f += e_f;
// r^{l-1}_P = mean of t_f (the 8-cell average R).
template <typename T>
__device__ __forceinline__ void op_restrict_amr(const RestrictA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &gf = A.gf, &gc = A.gc;
    int ci, cj, ck;
    int64_t P;
    bool act;
    if (A.cov) {
        // entry t of the covered-cell list: full warps of covered cells
        const int t = bx * NT + tid();
        act = t < A.ncov;
        if (!__any_sync(0xffffffffu, act)) return;
        P = act ? A.cov[t] : A.cov[0];
        const int c = (int)(P / gc.sz);
        const int64_t rem = P - (int64_t)c * gc.sz;
        const int b = (int)(rem / gc.sy);
        ci = gc.lo[0] + (int)(rem - (int64_t)b * gc.sy) - 1;
        cj = gc.lo[1] + b - 1;
        ck = gc.lo[2] + c - 1;
    } else {
        // footprint cells numbered row by row per plane (see cell_grid);
        // lanes past the plane stay in the warp (warp votes below) with
        // act = false
        const int n = bx * NT + tid(), r = n / A.cn[0];
        const bool in = r < A.cn[1];
        ci = A.clo[0] + (in ? n - r * A.cn[0] : 0);
        cj = A.clo[1] + (in ? r : 0);
        ck = A.clo[2] + bz;
        P = pad_index(gc, ci, cj, ck);
        act = in && gc.mask[P] == 2;
    }
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int64_t f = act ? pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2)) : 0;
        T S;
        int k;
        stencil_S<false>(gf, A.ef, f, act, S, k);
        if (act) {
            T ev = A.ef[f];
            T t = A.rf[f] + gih2<T>(gf) * (S - diagD<T>(gf, k) * ev);
            A.rf[f] = t;
            A.phif[f] += ev;
            acc += t;
        }
    }
    if (act) A.rc[P] = T(0.125) * acc;
}

// Alg. 3 prolongation and residual update, one thread per valid fine cell:
// v = I e^{l-1} (piecewise constant); e_f += v_f; phi_f += v_f (so that phi
// ends as phi_save + e without a saved copy); r_f -= (A_nf v)_f.
template <typename T>
__device__ __forceinline__ void op_prolong_amr(const ProlongA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &gf = A.gf, &gc = A.gc;
    int a, b, c;
    bool in;
    int64_t p;
    if (A.listed) {
        const int t = bx * NT + tid();
        in = t < gf.ccnt[0] + gf.ccnt[1];
        if (!__any_sync(0xffffffffu, in)) return;
        p = in ? gf.clist[t] : gf.sz + gf.sy + 1;
        c = (int)(p / gf.sz);
        const int64_t rem = p - (int64_t)c * gf.sz;
        b = (int)(rem / gf.sy);
        a = (int)(rem - (int64_t)b * gf.sy);
    } else {
        in = plane_cell(gf, bx, a, b); // lanes past the plane stay (warp vote below)
        c = 1 + bz;
        p = (int64_t)c * gf.sz + (int64_t)b * gf.sy + a;
    }
    bool act = in && gf.mask[p] != 0;
    int i = gf.lo[0] + a - 1, j = gf.lo[1] + b - 1, k = gf.lo[2] + c - 1;
    const int64_t off[6] = {-1, 1, -gf.sy, gf.sy, -gf.sz, gf.sz};
    bool fast = true;
    uint8_t m[6] = {1, 1, 1, 1, 1, 1};
    if (act) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            m[f] = gf.mask[p + off[f]];
            fast &= m[f] != 0;
        }
    }
    int64_t P = act ? pad_index(gc, i >> 1, j >> 1, k >> 1) : 0;
    // coarse offsets of the neighbour outside the parent, per axis
    const int64_t cst[3] = {1, gc.sy, gc.sz};
    int64_t out[3] = {(i & 1) ? cst[0] : -cst[0], (j & 1) ? cst[1] : -cst[1], (k & 1) ? cst[2] : -cst[2]};
    const T *ec = A.ec;
    T vp = act ? ec[P] : T(0), res;
    if (__all_sync(0xffffffffu, fast)) {
        // three neighbours share the parent; the other three see the
        // adjacent parents: sum_n v_n - 6 v_p = v_x + v_y + v_z - 3 v_p
        res = act ? ((ec[P + out[0]] + ec[P + out[1]]) + ec[P + out[2]]) - T(3) * vp : T(0);
    } else {
        T s = T(0);
        int kk = 0;
        if (act) {
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                int d = f >> 1;
                bool up = f & 1;
                // does the neighbour across face f leave the parent?
                bool leaves_n = up == ((((d == 0 ? i : (d == 1 ? j : k))) & 1) != 0);
                if (m[f] != 0) {
                    s += leaves_n ? ec[P + (up ? cst[d] : -cst[d])] : vp;
                    kk += 3;
                } else {
                    // the opposite neighbour then stays in the parent
                    T vo = leaves_n ? vp : ec[P + (up ? -cst[d] : cst[d])];
                    s -= T(kFifth) * vo;
                    kk += 1;
                }
            }
        }
        res = s - diagD<T>(gf, kk) * vp;
    }
    if (act) {
        A.ef[p] += vp;
        A.phif[p] += vp;
        A.rf[p] += gih2<T>(gf) * res;
    }
}

template <typename T>
__device__ __forceinline__ void op_elem(const ElemA<T> &A, int bx)
{
    for (int64_t t = (int64_t)bx * NT + tid(); t < A.n; t += A.stride) {
        if (A.kind == 0) {
            A.a[t] = A.v;
        } else if (A.kind == 1) {
            A.a[t] += A.v * A.b[t];
        } else {
            T v = A.b[t];
            A.a[t] += v;
            A.c[t] += v;
        }
    }
}

// Mixed precision: the FP32 right-hand side of the correction equation is
// the FP64 composite residual and the FP32 correction starts at zero
// (kind 0); afterwards phi (FP64) += the FP32 correction (kind 1).
// Only cells of the level are converted: outside cells keep the zeros that
// every array of the mixed form holds there (no kernel writes them), and
// their FP64 conversions would cost FP64-pipe time for nothing.
__device__ __forceinline__ void op_conv(const ConvA &A, int bx)
{
    for (int64_t t = (int64_t)bx * NT + tid(); t < A.n; t += A.stride) {
        if (A.mask[t] == 0) continue;
        if (A.kind == 0) {
            float v = (float)A.r64[t];
            A.rho32[t] = v;
            A.res32[t] = v;
            A.phi32[t] = 0.0f;
        } else {
            A.phi64[t] += (double)A.phi32[t];
        }
    }
}

// Coarse part of every coarse-fine ghost of a level: cp = sum of the
// (8/15)-weighted step-1 stencil over uc, one thread per face, accumulated
// in FP64 whatever the field's precision.
template <typename T>
__device__ __forceinline__ void op_cp(const CpA<T> &A, int bx)
{
    int q = bx * NT + tid();
    if (q >= A.nface) return;
    int n = A.cnt[q];
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += A.cw[q * kMaxStencil + k] * (double)A.uc[A.cidx[q * kMaxStencil + k]];
    A.cp[q] = acc;
}

// Interface corrections, accumulated in FP64 whatever the field precision.
template <typename T>
__device__ __forceinline__ void op_surface(const SurfaceA<T> &A, int bx)
{
    // the sums run in face order; the loads of four faces are issued
    // before their adds (a coarse cell has up to 24 fine faces, each a chain
    // of three dependent loads)
    int t = bx * NT + tid();
    if (t < A.ncell) {
        double acc = 0.0;
        int q = A.cell_ptr[t];
        const int q1 = A.cell_ptr[t + 1];
        for (; q + 4 <= q1; q += 4) {
            const double a0 = A.cp_f[q], a1 = A.cp_f[q + 1], a2 = A.cp_f[q + 2], a3 = A.cp_f[q + 3];
            acc += a0;
            acc += a1;
            acc += a2;
            acc += a3;
        }
        for (; q < q1; ++q) acc += A.cp_f[q];
        int f = A.cell_f[t];
        A.rf[f] = (T)((double)A.rf[f] + A.scale_f * acc);
        return;
    }
    t -= A.ncell;
    if (t < A.ncrse) {
        auto term = [&](double u, double u1, double cp) { return (kThird * u + kFifth * u1) - cp; };
        double acc = 0.0;
        int q = A.crse_ptr[t];
        const int q1 = A.crse_ptr[t + 1];
        for (; q + 4 <= q1; q += 4) {
            int fc[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) fc[r] = A.crse_face[q + r];
            int i0[4], i1[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                i0[r] = A.ff[fc[r]];
                i1[r] = A.ff1[fc[r]];
            }
            double u[4], u1[4], cp[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                u[r] = (double)A.uf[i0[r]];
                u1[r] = (double)A.uf[i1[r]];
                cp[r] = A.cp_c[fc[r]];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) acc += term(u[r], u1[r], cp[r]);
        }
        for (; q < q1; ++q) {
            const int face = A.crse_face[q];
            acc += term((double)A.uf[A.ff[face]], (double)A.uf[A.ff1[face]], A.cp_c[face]);
        }
        int C = A.crse_c[t];
        A.rc[C] = (T)((double)A.rc[C] + A.scale_c * acc);
    }
}

// E_d = -(u_{+d} - u_{-d}) / (2h) on valid cells; coarse-fine ghosts get
// their fine part here and their coarse part from op_cf_grad.
__device__ __forceinline__ void op_grad(const GradA &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &g = A.g;
    int a, b;
    if (!plane_cell(g, bx, a, b)) return;
    int c = 1 + bz;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
    if (g.mask[p] == 0) return;
    const int64_t st[3] = {1, g.sy, g.sz};
    const double *u = A.u;
    double up = u[p];
    double out[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double side[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int64_t o = s ? st[d] : -st[d];
            if (g.mask[p + o] != 0)
                side[s] = u[p + o];
            else if (g.periodic)
                side[s] = u[p + wrap_off(g, 2 * d + s)];
            else if (g.dirichlet)
                side[s] = g.robin ? g.robin->alpha * up : -up;
            else
                side[s] = (2.0 * kThird) * up - kFifth * u[p - o];
        }
        out[d] = -(side[1] - side[0]) * (0.5 / g.h);
    }
    A.e0[p] = out[0];
    A.e1[p] = out[1];
    A.e2[p] = out[2];
}

__device__ __forceinline__ void op_cf_grad(const CfGradA &A, int bx)
{
    int i = bx * NT + tid();
    if (i >= A.ncell) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = A.cell_ptr[i]; q < A.cell_ptr[i + 1]; ++q) {
        int d = A.dir[q] >> 1;
        double s = (A.dir[q] & 1) ? 1.0 : -1.0;
        acc[d] -= s * A.cp[q] * A.inv2h;
    }
    int f = A.cell_f[i];
    A.e0[f] += acc[0];
    A.e1[f] += acc[1];
    A.e2[f] += acc[2];
}

// Average down: covered coarse cells <- mean of their 8 children.
__device__ __forceinline__ void op_avgdown(const AvgDownA &A, int bx, int by, int bz)
{
    int ci = A.clo[0] + bx * BX + threadIdx.x;
    int cj = A.clo[1] + by * BY + ty();
    int ck = A.clo[2] + bz;
    if (ci >= A.clo[0] + A.cn[0] || cj >= A.clo[1] + A.cn[1] || ck >= A.clo[2] + A.cn[2]) return;
    int64_t P = pad_index(A.gc, ci, cj, ck);
    if (A.gc.mask[P] != 2) return;
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o)
        acc += A.uf[pad_index(A.gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2))];
    A.uc[P] = 0.125 * acc;
}

// max that keeps a NaN operand (fmax drops it)
__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// Fixed-order block reduction of (sum, sum, max) over the 128 threads; every
// thread returns the totals.
__device__ __forceinline__ void block_reduce3(double &s2, double &s1, double &mx)
{
    __shared__ double sh[3][NT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    int w = tid() >> 5, lane = tid() & 31;
    __syncthreads();
    if (lane == 0) {
        sh[0][w] = s2;
        sh[1][w] = s1;
        sh[2][w] = mx;
    }
    __syncthreads();
    s2 = s1 = mx = 0.0;
    for (int q = 0; q < NT / 32; ++q) {
        s2 += sh[0][q];
        s1 += sh[1][q];
        mx = nan_max(mx, sh[2][q]);
    }
}

// Accumulates cell value x (with mask byte m) into the partial of norm P:
// sum x^2 (P = 2, one FP64 FMA), sum |x| (P = 1, one FP64 add) or max |x|
// (P = inf) taken on the bit pattern of |x|, whose unsigned order is the
// numeric order of non-negative doubles (NaN sorts above +inf), so the max
// costs no FP64 instruction.
template <int P>
__device__ __forceinline__ void norm_acc(int cov, uint32_t m, double x, double &s, unsigned long long &mb)
{
    bool ok = m == 1u || (cov && m == 2u);
    // cells outside the norm become +0 by clearing their bits (integer
    // operations: the FP64 pipe is this loop's bound, one FMA or add a cell)
    if constexpr (P == AMR_NORM_2) {
        x = __longlong_as_double(__double_as_longlong(x) & (ok ? -1ll : 0ll));
        s = fma(x, x, s);
    } else if constexpr (P == AMR_NORM_1) {
        x = __longlong_as_double(__double_as_longlong(x) & (ok ? 0x7fffffffffffffffll : 0ll));
        s += x;
    } else {
        unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
        mb = max(mb, ok ? b : 0ull);
    }
}

// One norm's partial over cells [t0, n) with stride (aligned slots four
// cells at a time: one 32-bit mask word, two 16-byte value loads).
template <int P>
__device__ __forceinline__ void norm_loop(const uint8_t *mask, const double *v, int64_t n, int cov, int vec,
                                          int64_t t0, int64_t stride, double &s, unsigned long long &mb)
{
    int64_t done = 0;
    if (vec) {
        const int64_t ng = n >> 2;
        const uint32_t *m4 = reinterpret_cast<const uint32_t *>(mask);
        const double2 *v2 = reinterpret_cast<const double2 *>(v);
#pragma unroll 4
        for (int64_t g = t0; g < ng; g += stride) {
            uint32_t mm = m4[g];
            double2 a = v2[2 * g], b = v2[2 * g + 1];
            norm_acc<P>(cov, mm & 0xffu, a.x, s, mb);
            norm_acc<P>(cov, (mm >> 8) & 0xffu, a.y, s, mb);
            norm_acc<P>(cov, (mm >> 16) & 0xffu, b.x, s, mb);
            norm_acc<P>(cov, mm >> 24, b.y, s, mb);
        }
        done = ng << 2;
    }
    for (int64_t t = done + t0; t < n; t += stride) norm_acc<P>(cov, mask[t], v[t], s, mb);
}

// Per-block partial of ||v||_p over the cells with mask == 1 (or >= 1 when
// covered_too), one slot per virtual-grid row by.  The thread-to-cell
// assignment and the reduction tree are fixed, so the result is bitwise
// reproducible.  Partial layout per slot: [0, nb) the sum (p = 1, 2),
// [2 kPartialBlocks, +nb) the max (p = inf).
__device__ __forceinline__ void op_norms(const NormA &A, int bx, int by)
{
    int slot = by;
    const uint8_t *mask = A.mask[slot];
    const double *v = A.v[slot];
    int64_t n = A.n[slot];
    int cov = A.covered_too[slot];
    int pn = A.prm->norm;
    double s = 0.0;
    unsigned long long mb = 0ull;
    const int64_t t0 = (int64_t)bx * NT + tid(), stride = (int64_t)A.nblocks * NT;
    if (pn == AMR_NORM_2)
        norm_loop<AMR_NORM_2>(mask, v, n, cov, A.vec, t0, stride, s, mb);
    else if (pn == AMR_NORM_1)
        norm_loop<AMR_NORM_1>(mask, v, n, cov, A.vec, t0, stride, s, mb);
    else
        norm_loop<AMR_NORM_INF>(mask, v, n, cov, A.vec, t0, stride, s, mb);
    double s1 = 0.0, mx = __longlong_as_double((long long)mb);
    block_reduce3(s, s1, mx);
    if (tid() == 0) {
        double *p = A.part + (int64_t)slot * 3 * kPartialBlocks;
        p[bx] = s;
        p[2 * kPartialBlocks + bx] = mx;
    }
}

// Convergence test of Alg. 2 on the device: fixed-order sums of the
// partials, rel^l = ||r^l||_p / ||rho^l||_p (a zero ||rho^l|| uses the
// largest one), iteration count, and "another V-cycle" (also the graph
// condition when use_cond).
__device__ __forceinline__ void op_check(const CheckA &A)
{
    __shared__ double tot[2 * kMaxLevels][3];
    int nslots = A.with_rho ? 2 * A.nlev : A.nlev;
    for (int slot = 0; slot < nslots; ++slot) {
        const double *p = A.part + (int64_t)slot * 3 * kPartialBlocks;
        double s2 = 0.0, s1 = 0.0, mx = 0.0;
        for (int t = tid(); t < A.nblocks; t += NT) {
            s2 += __ldcg(p + t);
            double m = __ldcg(p + 2 * kPartialBlocks + t);
            mx = nan_max(mx, m);
        }
        block_reduce3(s2, s1, mx);
        if (tid() == 0) {
            tot[slot][0] = s2;
            tot[slot][1] = s1;
            tot[slot][2] = mx;
        }
    }
    __syncthreads();
    if (tid() != 0) return;
    SolveState *st = A.st;
    int pn = A.prm->norm;
    auto pick = [pn](const double *v) { return pn == AMR_NORM_2 ? sqrt(v[0]) : (pn == AMR_NORM_1 ? v[0] : v[2]); };
    if (A.with_rho)
        for (int l = 0; l < A.nlev; ++l) st->rhon[l] = pick(tot[A.nlev + l]);
    double bmax = 0.0;
    for (int l = 0; l < A.nlev; ++l) bmax = fmax(bmax, st->rhon[l]);
    double worst = 0.0;
    for (int l = 0; l < A.nlev; ++l) {
        double b = st->rhon[l] > 0.0 ? st->rhon[l] : bmax;
        double r = pick(tot[l]);
        double rel = b > 0.0 ? r / b : r;
        st->rel[l] = rel;
        worst = nan_max(worst, rel);
    }
    st->worst = worst;
    int it = A.is_body ? st->iters + 1 : 0;
    st->iters = it;
    // a NaN residual never counts as converged
    int go = !(worst <= A.prm->eps) && (it < A.prm->max_iter);
    st->go = go;
    if (A.use_cond) cudaGraphSetConditional(A.cond, go ? 1u : 0u);
}

// Level-0 multigrid restriction, one thread per coarse cell:
// r_c = mean over the children of (r_f - A e_f); e_c = 0.
template <typename T, bool PER = false>
__device__ __forceinline__ void op_mg_restrict(const MgRestrictA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &gf = A.gf, &gc = A.gc;
    int a, b;
    const bool act = plane_cell(gc, bx, a, b); // lanes past the plane stay (warp votes below)
    int c = 1 + bz;
    int ci = gc.lo[0] + a - 1, cj = gc.lo[1] + b - 1, ck = gc.lo[2] + c - 1;
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int64_t f = act ? pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2)) : 0;
        T S;
        int k;
        stencil_S<false, T, PER>(gf, A.ef, f, act, S, k);
        if (act) acc += A.rf[f] + gih2<T>(gf) * (S - diagD<T>(gf, k) * A.ef[f]);
    }
    if (act) {
        int64_t P = (int64_t)c * gc.sz + (int64_t)b * gc.sy + a;
        T r = T(0.125) * acc;
        A.rc[P] = r;
        // e_c = 0, or the red pass from zero (the arithmetic of op_rbgs_first
        // on the value just stored): red cells h^2 r / D, black cells 0
        T ev = T(0);
        if (A.first_red && ((ci + cj + ck) & 1) == 0 && (gc.code[P] & 64u))
            ev = gs_update(gc, T(0), gh2<T>(gc), r, face_code(gc, P));
        A.ec[P] = ev;
    }
}

// Level-0 multigrid trilinear prolongation of the correction, one thread
// per fine cell: weights 3/4 and 1/4 per axis on the two nearest coarse
// centres; outside the domain the coarse ghost is the domain-face ghost of
// the coarse grid per face crossed (-v for Dirichlet, alpha v for Robin).
template <typename T>
__device__ __forceinline__ void op_mg_prolong(const MgProlongA<T> &A, int bx, int by, int bz)
{
    (void)by;
    const Grid &gf = A.gf, &gc = A.gc;
    const T ralpha = gc.robin ? (T)gc.robin->alpha : T(-1);
    int a, b;
    if (!plane_cell(gf, bx, a, b)) return;
    int c = 1 + bz;
    int64_t p = (int64_t)c * gf.sz + (int64_t)b * gf.sy + a;
    int i = gf.lo[0] + a - 1, j = gf.lo[1] + b - 1, k = gf.lo[2] + c - 1;
    int I[3] = {i >> 1, j >> 1, k >> 1};
    int O[3] = {(i & 1) ? 1 : -1, (j & 1) ? 1 : -1, (k & 1) ? 1 : -1};
    int nc[3] = {gc.n[0] - 2, gc.n[1] - 2, gc.n[2] - 2};
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int sel[3] = {o & 1, (o >> 1) & 1, o >> 2};
        T w = T(1);
        int nref = 0;
        int Q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            w *= sel[d] ? T(0.25) : T(0.75);
            int q = I[d] + (sel[d] ? O[d] : 0);
            if (gc.periodic && (q < 0 || q >= nc[d])) {
                q = q < 0 ? q + nc[d] : q - nc[d]; // periodic image
            } else if (q < 0 || q >= nc[d]) {
                ++nref;
                q = I[d];
            }
            Q[d] = q;
        }
        T v = A.ec[pad_index(gc, Q[0], Q[1], Q[2])];
        if (gc.robin) {
            for (int r = 0; r < nref; ++r) v *= ralpha;
        } else if (nref & 1) {
            v = -v;
        }
        acc += w * v;
    }
    A.ef[p] += acc;
}

// Coarsest grid of the level-0 multigrid: e = M r with the dense FP64
// inverse M (order m), accumulated in FP64; one warp per row, r staged in
// shared memory (rs: m doubles of dynamic shared memory).
template <typename T>
__device__ __forceinline__ void op_coarse(const CoarseA<T> &A, int bx, double *rs)
{
    const Grid &g = A.g;
    int nx = g.n[0] - 2, ny = g.n[1] - 2;
    int m = A.m;
    __syncthreads();
    for (int t = tid(); t < m; t += NT) {
        int i = t % nx, j = (t / nx) % ny, k = t / (nx * ny);
        rs[t] = (double)A.r[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)];
    }
    __syncthreads();
    int row = bx * (NT / 32) + (tid() >> 5);
    int lane = tid() & 31;
    if (row >= m) return;
    double acc = 0.0;
    for (int c = lane; c < m; c += 32) acc = fma(A.M[(int64_t)row * m + c], rs[c], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        int i = row % nx, j = (row / nx) % ny, k = row / (nx * ny);
        A.e[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)] = (T)acc;
    }
}

template <typename TI, typename TO>
__device__ __forceinline__ void op_axis(const AxisA<TI, TO> &A, int bx)
{
    const int n = A.n;
    const int t = bx * NT + tid();
    if (t >= n * n * n) return;
    const int i = t % n, j = (t / n) % n, k = t / (n * n);
    const int c3[3] = {i, j, k};
    const int c = c3[A.axis];
    const int64_t st = A.axis == 0 ? 1 : (A.axis == 1 ? A.sy : A.sz);
    // the line through (i, j, k) along the axis, from coordinate 0
    const int64_t p0 = (int64_t)(k + 1) * A.sz + (int64_t)(j + 1) * A.sy + (i + 1) - (int64_t)c * st;
    const double *m = A.M + (int64_t)c * n;
    double acc = 0.0;
    for (int q = 0; q < n; ++q) acc = fma(m[q], (double)A.in[p0 + q * st], acc);
    if (A.lam) {
        double l = A.lam[i] + A.lam[j] + A.lam[k];
        if (t == 0) l += A.zero_add;
        acc = acc * A.h2 / l;
    }
    A.out[p0 + c * st] = (TO)acc;
}

// Cloud-in-cell deposit, one thread per particle, every level: node (cell
// centre) i at (i + 1/2) h, linear weights per axis, density q w / h^3.
// Exponent field not all ones (neither inf nor NaN), on the bits alone.
__device__ __forceinline__ bool finite_bits(double v)
{
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

// Cloud-in-cell coordinates of position p on a level of spacing 1/ih with
// padded-box origin lo: lower node (padded index) and the weight of the
// upper node per axis.  s = p/h - 1/2 is formed as fma(p, 1/h, -1/2), which
// is exactly p/h - 1/2 rounded once when h is a power of two; the lower node
// is floor(s) (clamped, so far-away positions stay in int range and land
// outside every box) and w1 = s - floor(s) is exact.
__device__ __forceinline__ void cic_axis(double p, double ih, int lo, int &loc, double &w1)
{
    double s = fma(p, ih, -0.5);
    int i = __double2int_rd(s);
    i = min(max(i, -8), 1 << 28);
    w1 = s - (double)i;
    loc = i - lo + 1;
}

// The same coordinates without FP64 instructions, for a level with 2^a
// cells per unit length (n0 a power of two).  A position p in [2^-8, 1) is
// exactly P = p 2^60 (its lowest mantissa bit is at least 2^-60), and
// s = p 2^a - 1/2 is S = P 2^a - 2^59 in 60-bit fixed point: the lower node
// is floor(s) = (P - 2^(59-a)) >> (60 - a) and the fraction's bits are the
// low 60 bits of S (computed modulo 2^64: the discarded high bits do not
// reach them).  w1 = frac(s) is the same double as in cic_axis (s is exact
// in FP64, so both are exact); it has at most 53 significant bits and is
// assembled from the integer by integer operations.
// Also requires p 2^a0 >= 1 (a0 the coarsest level's a): then s + 1/2 >= 1
// on every level, its unit in the last place is at most 1/2 and s is exact.
__device__ __forceinline__ bool fixed60(double p, int a0, unsigned long long &P)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(p);
    const int e = (int)(b >> 52); // biased exponent (sign bit 0 for p >= 0)
    if (e < 1015 || e > 1022) return false; // p not in [2^-8, 1) (or negative, non-finite)
    P = ((b & 0xfffffffffffffull) | (1ull << 52)) << (e - 1015);
    return (P >> (60 - a0)) != 0ull;
}

__device__ __forceinline__ double frac60_to_double(unsigned long long f)
{
    if (f == 0ull) return 0.0;
    const int lz = __clzll((long long)f);
    // leading one to bit 52 (f has at most 53 significant bits, so a right
    // shift drops only zeros)
    const unsigned long long m = lz >= 11 ? f << (lz - 11) : f >> (11 - lz);
    const unsigned long long bits = ((unsigned long long)(1026 - lz) << 52) | (m & 0xfffffffffffffull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void cic_axis_fixed(unsigned long long P, int a, int lo, int &loc, double &w1)
{
    const long long i = ((long long)P - (1ll << (59 - a))) >> (60 - a);
    const unsigned long long f = ((P << a) - (1ull << 59)) & ((1ull << 60) - 1ull);
    w1 = frac60_to_double(f);
    loc = (int)i - lo + 1;
}

// Fire-and-forget FP64 addition in global memory (a reduction: no value
// comes back, so the thread does not wait for the L2 round trip).
__device__ __forceinline__ void red_add(double *p, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// CIC deposit of every particle onto every level: rho^l += q w_a w_b w_c /
// (eps0 h_l^3) at the 8 nodes around the particle (FP64 atomics).  15 FP64
// instructions per particle and level for the weights on power-of-two grids,
// whose coordinates come from integer arithmetic (no divisions: 1/h and
// 1/h^3 come precomputed).  Non-finite positions deposit nothing and, like
// positions whose nodes are not all valid level-0 cells, count as outside.
__device__ __forceinline__ void deposit_one(const DepositA &A, double px, double py, double pz, double pq)
{
    if (!(finite_bits(px) && finite_bits(py) && finite_bits(pz))) {
        if (A.outside) atomicAdd(A.outside, 1);
        return;
    }
    // power-of-two levels: the coordinates by integer arithmetic
    unsigned long long P[3];
    const bool fx = A.lg[0] >= 0 && fixed60(px, A.lg[0], P[0]) && fixed60(py, A.lg[0], P[1]) &&
                   fixed60(pz, A.lg[0], P[2]);
    // the level loop unrolled (compile-time indices into the parameter
    // block: a runtime index would make the compiler copy it to local memory)
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l) {
        if (l >= A.nlev) break;
        const Grid &g = A.g[l];
        int loc[3];
        double w1[3];
        if (fx) {
            cic_axis_fixed(P[0], A.lg[l], g.lo[0], loc[0], w1[0]);
            cic_axis_fixed(P[1], A.lg[l], g.lo[1], loc[1], w1[1]);
            cic_axis_fixed(P[2], A.lg[l], g.lo[2], loc[2], w1[2]);
        } else {
            const double ih = A.ih[l];
            cic_axis(px, ih, g.lo[0], loc[0], w1[0]);
            cic_axis(py, ih, g.lo[1], loc[1], w1[1]);
            cic_axis(pz, ih, g.lo[2], loc[2], w1[2]);
        }
        bool inside = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) inside &= (loc[d] >= 0 && loc[d] + 1 < g.n[d]);
        if (l == 0 && A.outside) {
            // all nodes must be valid cells of level 0 (not the ring)
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) ok &= (loc[d] >= 1 && loc[d] + 1 <= g.n[d] - 2);
            if (!ok) atomicAdd(A.outside, 1);
        }
        // the 8 node weights q w_a w_b w_c / h^3, axis by axis: a weight t
        // splits into t w1 and t - t w1 = t w0 (15 FP64 operations per level
        // instead of 18 with w0 = 1 - w1 formed first)
        const double wq = pq * A.ih3[l];
        const double z1 = wq * w1[2], z0 = wq - z1;
        double yz[4]; // index db + 2 dc
        yz[1] = z0 * w1[1];
        yz[0] = z0 - yz[1];
        yz[3] = z1 * w1[1];
        yz[2] = z1 - yz[3];
        double wn[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            wn[2 * k + 1] = yz[k] * w1[0];
            wn[2 * k] = yz[k] - wn[2 * k + 1];
        }
        int64_t base = (int64_t)loc[2] * g.sz + (int64_t)loc[1] * g.sy + loc[0];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            int da = o & 1, db = (o >> 1) & 1, dc = o >> 2;
            int a = loc[0] + da, b = loc[1] + db, c = loc[2] + dc;
            if (!inside && (a < 0 || b < 0 || c < 0 || a >= g.n[0] || b >= g.n[1] || c >= g.n[2])) continue;
            red_add(A.rho[l] + base + (dc ? g.sz : 0) + (db ? g.sy : 0) + da, wn[o]);
        }
    }
}

// Two particles per thread (kDepositPer NT to a virtual block, consecutive
// threads on consecutive particles in each half): both particles' loads are
// issued before the first is deposited, so the second's are in flight
// during the first's arithmetic and atomics (one particle per thread left
// the kernel waiting on its loads: long-scoreboard stalls dominated once the
// integer coordinates had taken the FP64 pipe off the critical path).
constexpr int kDepositPer = 2;

__device__ __forceinline__ void op_deposit(const DepositA &A, int bx)
{
    const int64_t t0 = (int64_t)bx * (kDepositPer * NT) + tid();
    double px[kDepositPer], py[kDepositPer], pz[kDepositPer], pq[kDepositPer];
#pragma unroll
    for (int u = 0; u < kDepositPer; ++u) {
        const int64_t t = t0 + (int64_t)u * NT;
        const bool in = t < A.n;
        px[u] = in ? A.x[t] : 0.0;
        py[u] = in ? A.y[t] : 0.0;
        pz[u] = in ? A.z[t] : 0.0;
        pq[u] = in ? A.q[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kDepositPer; ++u)
        if (t0 + (int64_t)u * NT < A.n) deposit_one(A, px[u], py[u], pz[u], pq[u] * A.inv_eps0);
}

// Gather of E (and phi) by CIC from the finest level whose valid cells hold
// all 8 nodes of the particle.
// The level search (integer work: coordinates, bounds, masks) runs first
// for every lane; the FP64 interpolation runs after it, once for the whole
// warp whatever the levels its lanes found (inside the search loop the warp
// issued it once per distinct level of its lanes, and an FP64 instruction
// costs the pipe the same time however few lanes it has work for).
__device__ __forceinline__ void op_gather(const GatherA &A, int bx)
{
    // lanes past the last particle stay until the interpolation (the warp
    // reconverges there)
    const int64_t t = (int64_t)bx * NT + tid();
    const bool live = t < A.n;
    const double px = live ? A.x[t] : 0.5, py = live ? A.y[t] : 0.5, pz = live ? A.z[t] : 0.5;
    double E[3] = {0.0, 0.0, 0.0}, ph = 0.0;
    bool fin = live && finite_bits(px) && finite_bits(py) && finite_bits(pz);
    unsigned long long P[3];
    const bool fx = fin && A.lg[0] >= 0 && fixed60(px, A.lg[0], P[0]) && fixed60(py, A.lg[0], P[1]) &&
                   fixed60(pz, A.lg[0], P[2]);
    int lf = -1;
    int64_t base = 0, sy = 0, sz = 0;
    const double *e0 = nullptr, *e1 = nullptr, *e2 = nullptr, *pf = nullptr;
    double w1[3] = {0.0, 0.0, 0.0};
    // finest level first; compile-time level indices (see deposit_one)
#pragma unroll
    for (int l = kMaxLevels - 1; l >= 0; --l) {
        if (l >= A.nlev || !fin || lf >= 0) continue;
        const Grid &g = A.g[l];
        int loc[3];
        double v1[3];
        if (fx) {
            cic_axis_fixed(P[0], A.lg[l], g.lo[0], loc[0], v1[0]);
            cic_axis_fixed(P[1], A.lg[l], g.lo[1], loc[1], v1[1]);
            cic_axis_fixed(P[2], A.lg[l], g.lo[2], loc[2], v1[2]);
        } else {
            const double ih = A.ih[l];
            cic_axis(px, ih, g.lo[0], loc[0], v1[0]);
            cic_axis(py, ih, g.lo[1], loc[1], v1[1]);
            cic_axis(pz, ih, g.lo[2], loc[2], v1[2]);
        }
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) ok &= (loc[d] >= 0 && loc[d] + 1 < g.n[d]);
        if (!ok) continue;
        const int64_t b0 = (int64_t)loc[2] * g.sz + (int64_t)loc[1] * g.sy + loc[0];
        const int64_t co[8] = {0, 1, g.sy, g.sy + 1, g.sz, g.sz + 1, g.sz + g.sy, g.sz + g.sy + 1};
#pragma unroll
        for (int o = 0; o < 8; ++o) ok &= (g.mask[b0 + co[o]] != 0);
        if (!ok) continue;
        lf = l;
        base = b0;
        sy = g.sy;
        sz = g.sz;
        e0 = A.e[l][0];
        e1 = A.e[l][1];
        e2 = A.e[l][2];
        pf = A.phi[l];
        w1[0] = v1[0];
        w1[1] = v1[1];
        w1[2] = v1[2];
    }
    // every lane past its level search: one interpolation for the warp
    __syncwarp();
    if (lf >= 0) {
        const int64_t co[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
        const double w0[3] = {1.0 - w1[0], 1.0 - w1[1], 1.0 - w1[2]};
        const double wxy[4] = {w0[0] * w0[1], w1[0] * w0[1], w0[0] * w1[1], w1[0] * w1[1]};
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            double w = wxy[o & 3] * (o >> 2 ? w1[2] : w0[2]);
            int64_t p = base + co[o];
            E[0] = fma(w, e0[p], E[0]);
            E[1] = fma(w, e1[p], E[1]);
            E[2] = fma(w, e2[p], E[2]);
            if (A.phio) ph = fma(w, pf[p], ph);
        }
    }
    if (!live) return;
    A.ex[t] = E[0];
    A.ey[t] = E[1];
    A.ez[t] = E[2];
    if (A.phio) A.phio[t] = ph;
}

// --------------------------------------------- level-0 exact bottom solve

// The level-0 operator A_nf^0 (7-point, homogeneous Dirichlet through the
// ghost -u on every face of the n^3 box) is separable:
//   A = (1/h^2) (T (x) I (x) I + I (x) T (x) I + I (x) I (x) T),
// T = tridiag(-1, 2, -1) with 3 in both corners, whose orthonormal
// eigenvectors are the cell-centred sines S[m][i] = c_m sin(pi (m+1) (i+1/2)
// / n) (eigenvalues 4 sin^2(pi (m+1) / (2n))).  The solve e = A^{-1} r is
// a sine transform along x and along y, one tridiagonal solve along z per
// (kx, ky) mode, and the inverse transforms: exact up to rounding, in FP64.
constexpr int kDstLines = 2; // lines per virtual block

// The sine basis is mirror-symmetric twice over.  S[m][n-1-i] = (-1)^m S[m][i]
// splits a line u into sums s_i = u_i + u_{n-1-i} (even m) and differences
// d_i = u_i - u_{n-1-i} (odd m), i < h = n/2.  For odd m, with kappa = (m+1)/2,
// S[m][h-1-i] = (-1)^(kappa+1) S[m][i], so the differences split again into
// ds_i = d_i + d_{h-1-i} (m = 1 mod 4) and dd_i = d_i - d_{h-1-i} (m = 3 mod 4),
// i < q = n/4.  A forward transform is then h^2 + h q = 3 n^2 / 8 FMAs per line
// instead of n^2, and the inverse the same count in reverse: even-mode sums
// E_i (i < h), and the two quarter sums A_i, B_i (i < q) that give the
// odd-mode sums O_i = A_i + B_i, O_{h-1-i} = A_i - B_i.  One output per
// thread (when h is a multiple of 32, each warp holds outputs of one kind,
// so its lanes share one trip count).  Needs n a multiple of 4.

// Forward output j of a line (m = 2j for j < h, else m = 2(j-h)+1), from the
// folded line F (sums at 0..h-1, ds_i at n-1-i, dd_i at h+i) and the table
// MP[i n + j] = S[m(j)][i].
__device__ __forceinline__ double dst_fwd_one(const double *MP, const double *F, int n, int h, int j)
{
    double acc = 0.0;
    if (j < h) {
        for (int i = 0; i < h; ++i) acc = fma(MP[i * n + j], F[i], acc);
    } else {
        const int q = h / 2, k = j - h;
        const double *D = (k & 1) ? F + h : F + n - 1; // m = 3 mod 4: dd_i at h+i; m = 1 mod 4: ds_i at n-1-i
        const int sgn = (k & 1) ? 1 : -1;
        for (int i = 0; i < q; ++i) acc = fma(MP[i * n + j], D[sgn * i], acc);
    }
    return acc;
}

// Inverse partial sum j of a line L of coefficients, MI[m n + i] = S[m][i]:
// j < h: E_j; h <= j < h+q: A_{j-h} (modes 4k+1); else B_{j-h-q} (modes 4k+3).
__device__ __forceinline__ double dst_inv_one(const double *MI, const double *L, int n, int h, int j)
{
    double acc = 0.0;
    if (j < h) {
        for (int k = 0; k < h; ++k) acc = fma(MI[2 * k * n + j], L[2 * k], acc);
    } else {
        const int q = h / 2, r = (j - h) / q, i = j - h - r * q, m0 = 1 + 2 * r;
        for (int k = 0; k < q; ++k) acc = fma(MI[(4 * k + m0) * n + i], L[4 * k + m0], acc);
    }
    return acc;
}

template <typename TI, typename TO>
__device__ __forceinline__ void op_dst(const DstA<TI, TO> &A, int bx, double *sm)
{
    const int n = A.n, h = n / 2, LN = kDstLines * n;
    double *L = sm, *R = sm + LN;
    const int g0 = bx * kDstLines; // first line of the block
    // element e of the block's lines: axis 0 line-major (x contiguous),
    // axis 1 y-major so that consecutive threads read consecutive x
    auto index = [&](int e, int &l, int &j) -> int64_t {
        if (A.axis == 0) {
            l = e / n;
            j = e - l * n;
            int G = g0 + l;
            return (int64_t)(G / n + 1) * A.sz + (int64_t)(G % n + 1) * A.sy + (j + 1);
        }
        l = e % kDstLines;
        j = e / kDstLines;
        int G = g0 + l;
        return (int64_t)(G / n + 1) * A.sz + (int64_t)(j + 1) * A.sy + (G % n + 1);
    };
    __syncthreads();
    // loads batched four at a time in registers before the shared-memory
    // stores: each store would otherwise hold back the next load
    for (int e0 = tid(); e0 < LN; e0 += NT * 4) {
        double v[4];
        int li[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = e0 + NT * t;
            int l = 0, j = 0;
            int64_t p = e < LN ? index(e, l, j) : 0;
            v[t] = (e < LN && g0 + l < n * n) ? (double)A.in[p] : 0.0;
            li[t] = l * n + j;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (e0 + NT * t < LN) L[li[t]] = v[t];
    }
    __syncthreads();
    const int q = h / 2;
    if (!A.inv) {
        // both folds in place, one thread per (line, i < q): positions i,
        // h-1-i get the sums, n-1-i gets ds_i, h+i gets dd_i
        for (int e = tid(); e < kDstLines * q; e += NT) {
            const int l = e / q, i = e - l * q;
            double *u = L + l * n;
            const double a = u[i], b = u[n - 1 - i], c = u[h - 1 - i], d = u[h + i];
            const double d0 = a - b, d1 = c - d;
            u[i] = a + b;
            u[h - 1 - i] = c + d;
            u[n - 1 - i] = d0 + d1;
            u[h + i] = d0 - d1;
        }
        __syncthreads();
        for (int e = tid(); e < LN; e += NT) {
            const int l = e / n, j = e - l * n;
            const int m = j < h ? 2 * j : 2 * (j - h) + 1;
            R[l * n + m] = dst_fwd_one(A.MT, L + l * n, n, h, j);
        }
    } else {
        for (int e = tid(); e < LN; e += NT) {
            const int l = e / n, j = e - l * n;
            R[l * n + j] = dst_inv_one(A.MT, L + l * n, n, h, j);
        }
        __syncthreads();
        // out_i = E_i + O_i, out_{n-1-i} = E_i - O_i (i < h), O from A, B
        for (int e = tid(); e < kDstLines * q; e += NT) {
            const int l = e / q, i = e - l * q;
            const double *r = R + l * n;
            double *o = L + l * n;
            const double e0 = r[i], e1 = r[h - 1 - i], a = r[h + i], b = r[h + q + i];
            const double o0 = a + b, o1 = a - b;
            o[i] = e0 + o0;
            o[n - 1 - i] = e0 - o0;
            o[h - 1 - i] = e1 + o1;
            o[h + i] = e1 - o1;
        }
    }
    __syncthreads();
    const double *Y = A.inv ? L : R;
    for (int e = tid(); e < LN; e += NT) {
        int l, j;
        int64_t p = index(e, l, j);
        if (g0 + l >= n * n) continue;
        TO v = (TO)Y[l * n + j];
        A.out[p] = v;
        if (A.phi) A.phi[p] += v;
    }
}

// Tridiagonal solves along z, (1/h^2) tridiag(-1, mu + 2, -1) with corners
// mu + 3, in place.  The matrix is persymmetric, so the symmetric and the
// antisymmetric parts of the right-hand side solve two independent systems
// of n/2 unknowns (the middle coupling becomes -1 / +1 on the last
// diagonal): two lanes per (kx, ky) mode, each a chain of half the length,
// each step one dependent FP64 operation forward and two back (dependent
// FP64 operations take long on this part, so the chains need many warps
// beside them).
constexpr int kTrizModes = 16; // modes per warp (at most 16: two lanes each)

// One warp takes kTrizModes modes (two lanes each) and a block of four warps
// 4 kTrizModes, without shared memory.  The chains read their right-hand
// sides and pivots straight from global memory (consecutive modes are
// consecutive x: a warp's loads are contiguous) and keep the forward sweep's
// y in place of the values they consumed: at step k the two lanes of a mode
// have both read u_k and u_{n-1-k} before the symmetric lane writes y at k
// and the antisymmetric lane at n-1-k (__syncwarp between).  The back
// substitution, z_k = w_k (z_{k+1} + y_k), forms the outputs as it goes:
// each lane takes its partner's z by a shuffle, x_k = (zs + za) f and
// x_{n-1-k} = (zs - za) f (f = the per-mode factor, with the 1/2 of the half
// systems' right-hand sides folded in), written over the y it has just read.
// Without shared memory per chain every chain of the solve is resident at
// once (n^2 / kTrizModes warps; staging the lines in shared memory had
// allowed four blocks of one working warp per SM).
__device__ __forceinline__ void op_triz(const TrizA &A, int bx)
{
    const int n = A.n, nm = n * n, h = n / 2;
    const int lane = threadIdx.x & 31, warp = tid() >> 5;
    const int q0 = (bx * 4 + warp) * kTrizModes;
    const int s = lane & 1, m = lane >> 1;
    const int q = q0 + m;
    const bool on = m < kTrizModes && q < nm;
    const int qq = on ? q : 0;
    double *line = A.u + (int64_t)(qq % n + 1) + (int64_t)(qq / n + 1) * A.sy + A.sz; // k = 0
    const int64_t sz = A.sz;
    const double *w = A.iw + (int64_t)s * h * nm + qq; // w_k at w[k nm]
    const double sg = s ? -1.0 : 1.0;
    // forward: y_k = c_k + y_{k-1} w_{k-1}, c_k = u_k +- u_{n-1-k}; the
    // loads of a group of kG steps are issued together (they do not depend
    // on the chain, and the group's stores come after them)
    constexpr int kG = 8;
    double y = 0.0, wp = 0.0;
    int k = 0;
    for (; k + kG <= h; k += kG) {
        double ua[kG], ub[kG], wv[kG];
#pragma unroll
        for (int j = 0; j < kG; ++j) {
            ua[j] = line[(int64_t)(k + j) * sz];
            ub[j] = line[(int64_t)(n - 1 - k - j) * sz];
            wv[j] = w[(int64_t)(k + j) * nm];
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kG; ++j) {
            const double c = fma(sg, ub[j], ua[j]);
            y = (k + j) == 0 ? c : fma(y, wp, c);
            wp = wv[j];
            if (on) line[(int64_t)(s ? n - 1 - k - j : k + j) * sz] = y;
        }
    }
    for (; k < h; ++k) {
        const double a = line[(int64_t)k * sz], b = line[(int64_t)(n - 1 - k) * sz];
        const double c = fma(sg, b, a);
        y = k == 0 ? c : fma(y, wp, c);
        wp = w[(int64_t)k * nm];
        __syncwarp();
        if (on) line[(int64_t)(s ? n - 1 - k : k) * sz] = y;
    }
    __syncwarp();
    // back: z_{h-1} = y_{h-1} w_{h-1}, z_k = w_k (z_{k+1} + y_k); outputs on the
    // way (each lane reads and writes only its own chain's positions)
    const double f = 0.5 * (A.fm ? A.fm[qq] : A.h2);
    double z = 0.0;
    k = h - 1;
    for (; k + 1 >= kG; k -= kG) {
        double yv[kG], wv[kG];
#pragma unroll
        for (int j = 0; j < kG; ++j) {
            yv[j] = line[(int64_t)(s ? n - 1 - (k - j) : k - j) * sz];
            wv[j] = w[(int64_t)(k - j) * nm];
        }
#pragma unroll
        for (int j = 0; j < kG; ++j) {
            z = (k - j) == h - 1 ? yv[j] * wv[j] : (z + yv[j]) * wv[j];
            const double t = __shfl_xor_sync(0xffffffffu, z, 1);
            const double x = s ? (t - z) * f : (z + t) * f;
            if (on) line[(int64_t)(s ? n - 1 - (k - j) : k - j) * sz] = x;
        }
    }
    for (; k >= 0; --k) {
        const int64_t pos = (int64_t)(s ? n - 1 - k : k) * sz;
        const double yk = line[pos], wk = w[(int64_t)k * nm];
        z = k == h - 1 ? yk * wk : (z + yk) * wk;
        const double t = __shfl_xor_sync(0xffffffffu, z, 1);
        const double x = s ? (t - z) * f : (z + t) * f;
        if (on) line[pos] = x;
    }
}

// Fast sine transforms (n a power of two).  The orthonormal transform
// X_m = c_m sum_i u_i sin(pi (m+1) (2i+1) / (2n)) is a cosine transform in
// disguise: with y_i = (-1)^i u_i, sin(pi (m+1) (2i+1) / (2n)) (-1)^i =
// cos(pi (n-1-m) (2i+1) / (2n)), so X_m = c_m C_{n-1-m}(y) with C the
// (unnormalised) DCT-II, C_k(y) = sum_i y_i cos(pi k (2i+1) / (2n)).  C is
// computed by B. G. Lee's recursive split (IEEE Trans. ASSP 32, 1984): for a
// block of size M, g_i = y_i + y_{M-1-i} and h_i = (y_i - y_{M-1-i}) s_i with
// s_i = 1 / (2 cos(pi (2i+1) / (2M))), i < M/2, give C_{2k} = C'_k(g) and
// C_{2k+1} = C'_k(h) + C'_{k+1}(h) with C' the DCT-II of size M/2 and
// C'_{M/2} = 0 (from 2 cos a cos b = cos(a-b) + cos(a+b)).  The recursion is
// run as log2 n splitting stages (blocks of size n, n/2, ..., 2, each block's
// g in its first half and h in its second) and log2 n combining stages
// (blocks of size 2, 4, ..., n), ping-ponging between two shared-memory
// buffers: 3 FP64 operations per pair in a split and one in a combine, about
// 2 log2 n per value instead of the 3n/8 FMAs of the folded matrix
// transform.  The inverse, u = S^T X, is the transposed flow graph run
// backwards: scale by c, reverse, the transposed combines (G_k = X_{2k},
// H_k = X_{2k+1} + X_{2k-1}) for sizes n .. 2, the transposed splits
// (y_i = g_i + s_i h_i, y_{M-1-i} = g_i - s_i h_i) for sizes 2 .. n, then
// the sign (-1)^i.  The scales c_m of the four transforms of a solve (two
// forward, two inverse: c_mx^2 c_my^2 per mode) are applied once, by the
// tridiagonal solve's final multiply, not per transform.
constexpr int kFdstElems = 1024; // values per virtual block (L lines of n; 8 KB per buffer)

// Flip the sign of v when odd (an integer operation on the sign bit).
__device__ __forceinline__ double sign_flip(double v, int odd)
{
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(odd & 1) << 63));
}

template <typename TI, typename TO>
__device__ __forceinline__ void op_fdst(const FdstA<TI, TO> &A, int bx, double *sm)
{
    const int n = A.n, L = A.L, half = n >> 1;
    const int G0 = bx * L;
    // shared-memory layout: line l, position q at l sl + q sp; consecutive
    // threads take consecutive positions (x lines) or lines (y lines), so
    // both the global accesses and the butterflies stay unit-stride
    const int sl = A.axis == 0 ? n : 1, sp = A.axis == 0 ? 1 : L;
    double *a = sm, *b = sm + kFdstElems;
    auto decode = [&](int e, int &l, int &q) {
        if (A.axis == 0) {
            l = e >> A.lg;
            q = e & (n - 1);
        } else {
            l = e % L;
            q = e / L;
        }
    };
    auto gindex = [&](int l, int q) -> int64_t {
        const int G = G0 + l, c = G & (n - 1), k = G >> A.lg;
        return A.axis == 0 ? (int64_t)(k + 1) * A.sz + (int64_t)(c + 1) * A.sy + (q + 1)
                           : (int64_t)(k + 1) * A.sz + (int64_t)(q + 1) * A.sy + (c + 1);
    };
    __syncthreads();
    // loads batched four at a time in registers before the shared-memory
    // stores (as in op_dst)
    for (int e0 = tid(); e0 < kFdstElems; e0 += NT * 4) {
        double v[4];
        int sidx[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int l, q;
            decode(e0 + NT * t, l, q);
            const double u = (double)A.in[gindex(l, q)];
            if (!A.inv) {
                v[t] = sign_flip(u, q); // y_q = (-1)^q u_q
                sidx[t] = l * sl + q * sp;
            } else {
                v[t] = u; // X_m (its scale c_m applied by the tridiagonal solve), reversed
                sidx[t] = l * sl + (n - 1 - q) * sp;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) a[sidx[t]] = v[t];
    }
    __syncthreads();
    const int nb = L * half; // butterflies (pairs) per stage
    auto pair = [&](int t, int &l, int &i) {
        if (A.axis == 0) {
            l = t >> (A.lg - 1);
            i = t & (half - 1);
        } else {
            l = t % L;
            i = t / L;
        }
    };
    if (!A.inv) {
        // splits: block size M = n, n/2, ..., 2
        for (int lm = A.lg; lm >= 1; --lm) {
            const int M = 1 << lm, hm = M >> 1;
            const double *s = A.tab + (n - M);
            for (int t = tid(); t < nb; t += NT) {
                int l, i;
                pair(t, l, i);
                const int o = (i >> (lm - 1)) << lm, ii = i & (hm - 1);
                const double x = a[l * sl + (o + ii) * sp], y = a[l * sl + (o + M - 1 - ii) * sp];
                b[l * sl + (o + ii) * sp] = x + y;
                b[l * sl + (o + hm + ii) * sp] = (x - y) * s[ii];
            }
            __syncthreads();
            double *tmp = a;
            a = b;
            b = tmp;
        }
        // combines: block size M = 2, 4, ..., n
        for (int lm = 1; lm <= A.lg; ++lm) {
            const int M = 1 << lm, hm = M >> 1;
            for (int t = tid(); t < nb; t += NT) {
                int l, i;
                pair(t, l, i);
                const int o = (i >> (lm - 1)) << lm, k = i & (hm - 1);
                const double G = a[l * sl + (o + k) * sp], H = a[l * sl + (o + hm + k) * sp];
                const double H1 = k + 1 < hm ? a[l * sl + (o + hm + k + 1) * sp] : 0.0;
                b[l * sl + (o + 2 * k) * sp] = G;
                b[l * sl + (o + 2 * k + 1) * sp] = k + 1 < hm ? H + H1 : H;
            }
            __syncthreads();
            double *tmp = a;
            a = b;
            b = tmp;
        }
    } else {
        // transposed combines: block size M = n, n/2, ..., 2
        for (int lm = A.lg; lm >= 1; --lm) {
            const int M = 1 << lm, hm = M >> 1;
            for (int t = tid(); t < nb; t += NT) {
                int l, i;
                pair(t, l, i);
                const int o = (i >> (lm - 1)) << lm, k = i & (hm - 1);
                const double X0 = a[l * sl + (o + 2 * k) * sp], X1 = a[l * sl + (o + 2 * k + 1) * sp];
                const double Xm = k > 0 ? a[l * sl + (o + 2 * k - 1) * sp] : 0.0;
                b[l * sl + (o + k) * sp] = X0;
                b[l * sl + (o + hm + k) * sp] = k > 0 ? X1 + Xm : X1;
            }
            __syncthreads();
            double *tmp = a;
            a = b;
            b = tmp;
        }
        // transposed splits: block size M = 2, 4, ..., n
        for (int lm = 1; lm <= A.lg; ++lm) {
            const int M = 1 << lm, hm = M >> 1;
            const double *s = A.tab + (n - M);
            for (int t = tid(); t < nb; t += NT) {
                int l, i;
                pair(t, l, i);
                const int o = (i >> (lm - 1)) << lm, ii = i & (hm - 1);
                const double g = a[l * sl + (o + ii) * sp], hs = a[l * sl + (o + hm + ii) * sp] * s[ii];
                b[l * sl + (o + ii) * sp] = g + hs;
                b[l * sl + (o + M - 1 - ii) * sp] = g - hs;
            }
            __syncthreads();
            double *tmp = a;
            a = b;
            b = tmp;
        }
    }
    // forward: X_m = c_m C_{n-1-m}; inverse: u_q = (-1)^q y_q
    for (int e = tid(); e < kFdstElems; e += NT) {
        int l, q;
        decode(e, l, q);
        const int64_t p = gindex(l, q);
        if (!A.inv) {
            A.out[p] = (TO)a[l * sl + (n - 1 - q) * sp]; // C_{n-1-m}; c_m left to the solve
        } else {
            const TO v = (TO)sign_flip(a[l * sl + q * sp], q);
            A.out[p] = v;
            if (A.phi) A.phi[p] += v;
        }
    }
}

// ------------------------------------------ multigrid bottom (one cluster)

// The recursive part of the level-0 multigrid V-cycle below grid gb (every
// grid there small: at most 32^3 cells) as ONE launch of one thread-block
// cluster: the same operations in the same order as the per-launch path
// (pre-smooth passes from zero, restriction, the dense coarsest solve,
// prolongation, post-smooth passes), each spread over the cluster's CTAs in
// virtual 32 x 4 blocks and followed by a cluster barrier with
// release/acquire semantics, which is what makes one phase's global-memory
// results visible to the next.  Every cell computes the same expression as
// in the per-launch path, so the results are bitwise the same.
constexpr int kBottomMaxGrids = 16;
constexpr int kBottomCells = 32 * 32 * 32;

template <typename T>
struct BottomA {
    int gb, nmg, nu1, nu2;
    Grid g[kBottomMaxGrids];
    T *e[kBottomMaxGrids];
    T *r[kBottomMaxGrids];
    const double *M; // dense inverse of the coarsest operator (order m)
    int m;
};

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_ctas()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Hardware barrier of all threads of the cluster (all CTAs of a cluster are
// co-resident, so it always completes).
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One phase: virtual blocks of grid vg spread over the cluster (blockDim.y
// / 4 virtual blocks per CTA), then the cluster barrier.
template <typename F>
__device__ __forceinline__ void cluster_phase(dim3 vg, F &&f)
{
    const int per = (int)blockDim.y / BY;
    const int sub = (int)threadIdx.y / BY;
    const int nvb = (int)(vg.x * vg.y * vg.z);
    const int step = (int)cluster_ctas() * per;
    for (int v = (int)cluster_rank() * per + sub; v < nvb; v += step) {
        int bx = v % (int)vg.x, by = (v / (int)vg.x) % (int)vg.y, bz = v / (int)(vg.x * vg.y);
        f(bx, by, bz);
    }
    cluster_barrier();
}

template <typename T>
__device__ __forceinline__ void bottom_smooth(const Grid &G, T *e, const T *r, int nu, bool from_zero)
{
    for (int it = 0; it < nu; ++it) {
        RbgsA<T> R{G, e, r, 0, 0, nullptr, nullptr, 0};
        if (from_zero && it == 0)
            cluster_phase(cell_grid(G), [&](int bx, int by, int bz) { op_rbgs_first(R, bx, by, bz); });
        else
            cluster_phase(colour_grid(G), [&](int bx, int by, int bz) { op_rbgs(R, bx, by, bz); });
        R.colour = 1;
        cluster_phase(colour_grid(G), [&](int bx, int by, int bz) { op_rbgs(R, bx, by, bz); });
    }
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_mg_bottom(const __grid_constant__ BottomA<T> A)
{
    extern __shared__ double rs[];
    for (int g = A.gb; g < A.nmg - 1; ++g) {
        bottom_smooth<T>(A.g[g], A.e[g], A.r[g], A.nu1, true);
        MgRestrictA<T> R{A.g[g], A.g[g + 1], A.e[g], A.r[g], A.r[g + 1], A.e[g + 1]};
        cluster_phase(cell_grid(A.g[g + 1]), [&](int bx, int by, int bz) { op_mg_restrict(R, bx, by, bz); });
    }
    {
        // coarsest grid: e = M r, one warp per row (the arithmetic of op_coarse)
        const Grid &g = A.g[A.nmg - 1];
        const T *r = A.r[A.nmg - 1];
        T *e = A.e[A.nmg - 1];
        const int nx = g.n[0] - 2, ny = g.n[1] - 2, m = A.m;
        const int nthr = (int)(blockDim.x * blockDim.y), t0 = (int)(threadIdx.y * blockDim.x + threadIdx.x);
        for (int t = t0; t < m; t += nthr) {
            int i = t % nx, j = (t / nx) % ny, k = t / (nx * ny);
            rs[t] = (double)r[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)];
        }
        __syncthreads();
        const int lane = t0 & 31, nw = nthr >> 5;
        for (int row = (int)cluster_rank() * nw + (t0 >> 5); row < m; row += (int)cluster_ctas() * nw) {
            double acc = 0.0;
            for (int c = lane; c < m; c += 32) acc = fma(A.M[(int64_t)row * m + c], rs[c], acc);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                int i = row % nx, j = (row / nx) % ny, k = row / (nx * ny);
                e[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)] = (T)acc;
            }
        }
        cluster_barrier();
    }
    for (int g = A.nmg - 2; g >= A.gb; --g) {
        MgProlongA<T> P{A.g[g], A.g[g + 1], A.e[g], A.e[g + 1]};
        cluster_phase(cell_grid(A.g[g]), [&](int bx, int by, int bz) { op_mg_prolong(P, bx, by, bz); });
        bottom_smooth<T>(A.g[g], A.e[g], A.r[g], A.nu2, false);
    }
}

// ------------------------------------------------- operation dispatch

enum Op : int {
    OP_RESIDUAL_D, OP_RESIDUAL_F, OP_RBGS_D, OP_RBGS_F, OP_RBGS_FIRST_D, OP_RBGS_FIRST_F, OP_RESTRICT_D,
    OP_RESTRICT_F, OP_PROLONG_D, OP_PROLONG_F, OP_ELEM_D, OP_ELEM_F, OP_CONV, OP_CP_D, OP_CP_F, OP_SURFACE_D,
    OP_SURFACE_F, OP_GRAD, OP_CF_GRAD, OP_AVGDOWN, OP_NORMS, OP_CHECK, OP_MG_RESTRICT_D, OP_MG_RESTRICT_F,
    OP_MG_PROLONG_D, OP_MG_PROLONG_F, OP_COARSE_D, OP_COARSE_F, OP_DEPOSIT, OP_GATHER, OP_DST_DD, OP_DST_FD,
    OP_DST_DF, OP_TRIZ,
    // the residual and colour pass of grids with periodic faces
    OP_RESIDUAL_PD, OP_RESIDUAL_PF, OP_RBGS_PD, OP_RBGS_PF, OP_MG_RESTRICT_PD, OP_MG_RESTRICT_PF,
    // fast sine transforms of the exact level-0 bottom
    OP_FDST_DD, OP_FDST_FD, OP_FDST_DF,
    // separable solve of a large coarsest multigrid grid
    OP_AXIS_DD, OP_AXIS_FD, OP_AXIS_DF
};

union OpArgs {
    ResidualA<double> res_d;
    ResidualA<float> res_f;
    RbgsA<double> rb_d;
    RbgsA<float> rb_f;
    RestrictA<double> rs_d;
    RestrictA<float> rs_f;
    ProlongA<double> pr_d;
    ProlongA<float> pr_f;
    ElemA<double> el_d;
    ElemA<float> el_f;
    ConvA conv;
    CpA<double> cp_d;
    CpA<float> cp_f;
    SurfaceA<double> sf_d;
    SurfaceA<float> sf_f;
    GradA grad;
    CfGradA cfg;
    AvgDownA avg;
    NormA norm;
    CheckA chk;
    MgRestrictA<double> mr_d;
    MgRestrictA<float> mr_f;
    MgProlongA<double> mp_d;
    MgProlongA<float> mp_f;
    CoarseA<double> co_d;
    CoarseA<float> co_f;
    DepositA dep;
    GatherA gat;
    DstA<double, double> dst_dd;
    DstA<float, double> dst_fd;
    DstA<double, float> dst_df;
    TrizA triz;
    FdstA<double, double> fdst_dd;
    FdstA<float, double> fdst_fd;
    FdstA<double, float> fdst_df;
    AxisA<double, double> ax_dd;
    AxisA<float, double> ax_fd;
    AxisA<double, float> ax_df;
};

} // namespace

// One recorded operation of a program (device layout).
struct __align__(16) Phase {
    int op;
    int gx, gy, gz; // virtual grid
    int hier;       // hierarchy index within the program
    int vbase;      // first virtual block within its round
    size_t smem;    // dynamic shared memory the operation needs
    OpArgs a;
};

namespace {

// Operation OP on virtual block (bx, by, bz); OP is a compile-time
// constant in the single-operation kernels and a case of the switch in the
// program kernel.
template <int OP>
__device__ __forceinline__ void run_op(const Phase &P, int bx, int by, int bz, double *dyn)
{
    if constexpr (OP == OP_RESIDUAL_D) op_residual(P.a.res_d, bx, by, bz);
    else if constexpr (OP == OP_RESIDUAL_F) op_residual(P.a.res_f, bx, by, bz);
    else if constexpr (OP == OP_RBGS_D) op_rbgs(P.a.rb_d, bx, by, bz);
    else if constexpr (OP == OP_RBGS_F) op_rbgs(P.a.rb_f, bx, by, bz);
    else if constexpr (OP == OP_RBGS_FIRST_D) op_rbgs_first(P.a.rb_d, bx, by, bz);
    else if constexpr (OP == OP_RBGS_FIRST_F) op_rbgs_first(P.a.rb_f, bx, by, bz);
    else if constexpr (OP == OP_RESTRICT_D) op_restrict_amr(P.a.rs_d, bx, by, bz);
    else if constexpr (OP == OP_RESTRICT_F) op_restrict_amr(P.a.rs_f, bx, by, bz);
    else if constexpr (OP == OP_PROLONG_D) op_prolong_amr(P.a.pr_d, bx, by, bz);
    else if constexpr (OP == OP_PROLONG_F) op_prolong_amr(P.a.pr_f, bx, by, bz);
    else if constexpr (OP == OP_ELEM_D) op_elem(P.a.el_d, bx);
    else if constexpr (OP == OP_ELEM_F) op_elem(P.a.el_f, bx);
    else if constexpr (OP == OP_CONV) op_conv(P.a.conv, bx);
    else if constexpr (OP == OP_CP_D) op_cp(P.a.cp_d, bx);
    else if constexpr (OP == OP_CP_F) op_cp(P.a.cp_f, bx);
    else if constexpr (OP == OP_SURFACE_D) op_surface(P.a.sf_d, bx);
    else if constexpr (OP == OP_SURFACE_F) op_surface(P.a.sf_f, bx);
    else if constexpr (OP == OP_GRAD) op_grad(P.a.grad, bx, by, bz);
    else if constexpr (OP == OP_CF_GRAD) op_cf_grad(P.a.cfg, bx);
    else if constexpr (OP == OP_AVGDOWN) op_avgdown(P.a.avg, bx, by, bz);
    else if constexpr (OP == OP_NORMS) op_norms(P.a.norm, bx, by);
    else if constexpr (OP == OP_CHECK) op_check(P.a.chk);
    else if constexpr (OP == OP_MG_RESTRICT_D) op_mg_restrict(P.a.mr_d, bx, by, bz);
    else if constexpr (OP == OP_MG_RESTRICT_F) op_mg_restrict(P.a.mr_f, bx, by, bz);
    else if constexpr (OP == OP_MG_PROLONG_D) op_mg_prolong(P.a.mp_d, bx, by, bz);
    else if constexpr (OP == OP_MG_PROLONG_F) op_mg_prolong(P.a.mp_f, bx, by, bz);
    else if constexpr (OP == OP_COARSE_D) op_coarse(P.a.co_d, bx, dyn);
    else if constexpr (OP == OP_COARSE_F) op_coarse(P.a.co_f, bx, dyn);
    else if constexpr (OP == OP_DEPOSIT) op_deposit(P.a.dep, bx);
    else if constexpr (OP == OP_GATHER) op_gather(P.a.gat, bx);
    else if constexpr (OP == OP_DST_DD) op_dst(P.a.dst_dd, bx, dyn);
    else if constexpr (OP == OP_DST_FD) op_dst(P.a.dst_fd, bx, dyn);
    else if constexpr (OP == OP_DST_DF) op_dst(P.a.dst_df, bx, dyn);
    else if constexpr (OP == OP_TRIZ) op_triz(P.a.triz, bx);
    else if constexpr (OP == OP_RESIDUAL_PD) op_residual<double, true>(P.a.res_d, bx, by, bz);
    else if constexpr (OP == OP_RESIDUAL_PF) op_residual<float, true>(P.a.res_f, bx, by, bz);
    else if constexpr (OP == OP_RBGS_PD) op_rbgs<double, true>(P.a.rb_d, bx, by, bz);
    else if constexpr (OP == OP_RBGS_PF) op_rbgs<float, true>(P.a.rb_f, bx, by, bz);
    else if constexpr (OP == OP_MG_RESTRICT_PD) op_mg_restrict<double, true>(P.a.mr_d, bx, by, bz);
    else if constexpr (OP == OP_MG_RESTRICT_PF) op_mg_restrict<float, true>(P.a.mr_f, bx, by, bz);
    else if constexpr (OP == OP_FDST_DD) op_fdst(P.a.fdst_dd, bx, dyn);
    else if constexpr (OP == OP_FDST_FD) op_fdst(P.a.fdst_fd, bx, dyn);
    else if constexpr (OP == OP_FDST_DF) op_fdst(P.a.fdst_df, bx, dyn);
    else if constexpr (OP == OP_AXIS_DD) op_axis(P.a.ax_dd, bx);
    else if constexpr (OP == OP_AXIS_FD) op_axis(P.a.ax_fd, bx);
    else if constexpr (OP == OP_AXIS_DF) op_axis(P.a.ax_df, bx);
}

__device__ __forceinline__ void dispatch(const Phase &P, int bx, int by, int bz, double *dyn)
{
    switch (P.op) {
#define AMR_CASE(OP)                                                                                        \
    case OP: run_op<OP>(P, bx, by, bz, dyn); break;
    AMR_CASE(OP_RESIDUAL_D) AMR_CASE(OP_RESIDUAL_F) AMR_CASE(OP_RBGS_D) AMR_CASE(OP_RBGS_F)
    AMR_CASE(OP_RBGS_FIRST_D) AMR_CASE(OP_RBGS_FIRST_F) AMR_CASE(OP_RESTRICT_D) AMR_CASE(OP_RESTRICT_F)
    AMR_CASE(OP_PROLONG_D) AMR_CASE(OP_PROLONG_F) AMR_CASE(OP_ELEM_D) AMR_CASE(OP_ELEM_F) AMR_CASE(OP_CONV)
    AMR_CASE(OP_CP_D) AMR_CASE(OP_CP_F) AMR_CASE(OP_SURFACE_D) AMR_CASE(OP_SURFACE_F) AMR_CASE(OP_GRAD)
    AMR_CASE(OP_CF_GRAD) AMR_CASE(OP_AVGDOWN) AMR_CASE(OP_NORMS) AMR_CASE(OP_CHECK) AMR_CASE(OP_MG_RESTRICT_D)
    AMR_CASE(OP_MG_RESTRICT_F) AMR_CASE(OP_MG_PROLONG_D) AMR_CASE(OP_MG_PROLONG_F) AMR_CASE(OP_COARSE_D)
    AMR_CASE(OP_COARSE_F) AMR_CASE(OP_DEPOSIT) AMR_CASE(OP_GATHER) AMR_CASE(OP_DST_DD) AMR_CASE(OP_DST_FD)
    AMR_CASE(OP_DST_DF) AMR_CASE(OP_TRIZ) AMR_CASE(OP_FDST_DD) AMR_CASE(OP_FDST_FD) AMR_CASE(OP_FDST_DF)
    AMR_CASE(OP_AXIS_DD) AMR_CASE(OP_AXIS_FD) AMR_CASE(OP_AXIS_DF)
    // (no periodic operations: hierarchies with periodic faces are not run
    // by the program kernel, which keeps its registers for the others)
#undef AMR_CASE
    default: break;
    }
}

// One operation as its own kernel (128 threads as 32 x 4).
template <int OP>
__global__ void __launch_bounds__(NT) k_op(const __grid_constant__ Phase P)
{
    pdl_begin();
    extern __shared__ double dyn[];
    run_op<OP>(P, blockIdx.x, blockIdx.y, blockIdx.z, dyn);
}

// Several independent operations as ONE kernel: block v runs virtual block
// v - vstart[q] of phase q.  OPA and OPB are the (at most two) operations
// the phases use.
constexpr int kMaxGroup = 8;
struct GroupDesc {
    int n;
    int vstart[kMaxGroup + 1];
    Phase ph[kMaxGroup];
};

template <int OPA, int OPB>
__global__ void __launch_bounds__(NT) k_group(const __grid_constant__ GroupDesc G)
{
    pdl_begin();
    extern __shared__ double dyn[];
    const int v = blockIdx.x;
    int q = 0;
    while (q + 1 < G.n && v >= G.vstart[q + 1]) ++q;
    const Phase &P = G.ph[q];
    const int lv = v - G.vstart[q];
    const int bx = lv % P.gx, by = (lv / P.gx) % P.gy, bz = lv / (P.gx * P.gy);
    if (P.op == OPA) {
        run_op<OPA>(P, bx, by, bz, dyn);
        return;
    }
    if constexpr (OPB != OPA) {
        if (P.op == OPB) run_op<OPB>(P, bx, by, bz, dyn);
    }
}

// The residual norms and the convergence test in one kernel: every block
// writes its partials, and the last block to arrive (arrival counter,
// reset by that block) runs the test, reading the partials past L1.
__global__ void __launch_bounds__(NT) k_norms_check(const __grid_constant__ NormA A, const __grid_constant__ CheckA C,
                                                    int *counter)
{
    pdl_begin();
    op_norms(A, blockIdx.x, blockIdx.y);
    __shared__ int last;
    __syncthreads();
    if (tid() == 0) {
        __threadfence();
        last = atomicAdd(counter, 1) == (int)(gridDim.x * gridDim.y) - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    op_check(C);
    if (tid() == 0) *counter = 0;
}

// ------------------------------------------------- persistent programs

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned atom_add_release(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of the persistent program.  Counters only grow: at its e-th
// barrier a block adds one to its group's counter (release); the block
// completing its group (counter = e * group size) adds one to the top
// counter; everyone waits (acquire) until the top counter reaches
// e * groups.  A wait that outlasts limit_ns records a timeout (err = 1)
// and returns false, as does any wait once an error is recorded.  Blocks
// are co-resident (cooperative launch), so a healthy barrier completes.
__device__ bool grid_sync(ProgramCtl *ctl, unsigned nblocks, unsigned long long limit_ns, unsigned &epoch)
{
    __syncthreads();
    ++epoch;
    if (tid() == 0) {
        unsigned g = blockIdx.x % kBarGroups;
        unsigned gsize = nblocks / kBarGroups + (g < nblocks % kBarGroups ? 1u : 0u);
        unsigned ngroups = nblocks < (unsigned)kBarGroups ? nblocks : (unsigned)kBarGroups;
        if (atom_add_release(&ctl->grp[g][0], 1u) + 1u == epoch * gsize) atom_add_release(&ctl->top[0], 1u);
        unsigned target = epoch * ngroups;
        volatile int *verr = &ctl->err[0];
        if (ld_acquire(&ctl->top[0]) < target) {
            unsigned long long t0 = globaltimer();
            unsigned spins = 0;
            while (ld_acquire(&ctl->top[0]) < target) {
                if (*verr) break;
                if ((++spins & 63u) == 0 && globaltimer() - t0 > limit_ns) {
                    atomicExch(&ctl->err[0], 1);
                    break;
                }
            }
        }
    }
    __syncthreads();
    return *(volatile int *)&ctl->err[0] == 0;
}

// Copy phase q into shared memory (uniform across the block).
__device__ __forceinline__ void load_phase(const Phase *phases, int q, Phase &sp)
{
    static_assert(sizeof(Phase) % 16 == 0, "phase size");
    const int4 *src = (const int4 *)&phases[q];
    int4 *dst = (int4 *)&sp;
    __syncthreads();
    for (int w = tid(); w < (int)(sizeof(Phase) / 16); w += NT) dst[w] = src[w];
    __syncthreads();
}

// Runs rounds [r0, r1).  Each block takes a contiguous chunk of the
// round's virtual blocks, finds the phase of the chunk's first block once
// and walks forward; body rounds skip the phases of hierarchies that have
// stopped iterating (their flag is read once per phase).
constexpr int kGoCache = 1024; // hierarchies whose flags a block caches in shared memory

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// A body round with the converged hierarchies left out: the round's
// still-active virtual blocks (hierarchies whose cached flag sgo is set),
// in phase order, are split evenly over the blocks.  Warp 0 finds the
// block's first active virtual block by a warp-parallel prefix scan over the
// phases' virtual-block counts.
__device__ void run_body_round(const ProgramDesc &D, int p0, int p1, const unsigned char *sgo, Phase &sp, int &cur,
                               double *dyn)
{
    const Phase *phases = (const Phase *)D.phases;
    __shared__ int s_cnt, s_q, s_off;
    if (tid() < 32) {
        const int lane = tid();
        int tot = 0;
        for (int q = p0 + lane; q < p1; q += 32) tot += sgo[D.ph_hier[q]] ? D.ph_nvb[q] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        const int chunk = (tot + (int)gridDim.x - 1) / (int)gridDim.x;
        const int a0 = (int)blockIdx.x * chunk;
        const int cnt = max(0, min(chunk, tot - a0));
        int fq = p1, foff = 0, run = 0;
        if (cnt > 0)
            for (int base = p0; base < p1; base += 32) {
                const int q = base + lane;
                const int a = (q < p1 && sgo[D.ph_hier[q]]) ? D.ph_nvb[q] : 0;
                const int incl = warp_incl_scan(a, lane);
                const int excl = run + incl - a;
                const unsigned hit = __ballot_sync(0xffffffffu, a > 0 && a0 >= excl && a0 < excl + a);
                if (hit) {
                    const int L = __ffs(hit) - 1;
                    fq = __shfl_sync(0xffffffffu, q, L);
                    foff = a0 - __shfl_sync(0xffffffffu, excl, L);
                    break;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        if (lane == 0) {
            s_cnt = cnt;
            s_q = fq;
            s_off = foff;
        }
    }
    __syncthreads();
    int left = s_cnt, q = s_q, off = s_off;
    while (left > 0 && q < p1) {
        if (!sgo[D.ph_hier[q]]) {
            ++q;
            off = 0;
            continue;
        }
        // the phase is copied to shared memory once per change (operations
        // read their arguments many times; reading them in place from global
        // memory measured slower)
        if (q != cur) {
            load_phase(phases, q, sp);
            cur = q;
        }
        const int take = min(D.ph_nvb[q] - off, left);
        for (int lv = off; lv < off + take; ++lv) {
            int bx = lv % sp.gx, by = (lv / sp.gx) % sp.gy, bz = lv / (sp.gx * sp.gy);
            dispatch(sp, bx, by, bz, dyn);
        }
        left -= take;
        ++q;
        off = 0;
    }
}

__device__ bool run_rounds(const ProgramDesc &D, int r0, int r1, bool body, Phase &sp, int &cur, double *dyn,
                           unsigned &epoch, const unsigned char *sgo = nullptr)
{
    const Phase *phases = (const Phase *)D.phases;
    for (int r = r0; r < r1; ++r) {
        if (body && sgo) {
            run_body_round(D, D.round_ptr[r], D.round_ptr[r + 1], sgo, sp, cur, dyn);
            if (!grid_sync(D.ctl, D.nblocks_expected, D.limit_ns, epoch)) return false;
            continue;
        }
        int p0 = D.round_ptr[r], p1 = D.round_ptr[r + 1];
        int total = D.round_nvb[r];
        int chunk = (total + (int)gridDim.x - 1) / (int)gridDim.x;
        int vb0 = (int)blockIdx.x * chunk, vb1 = min(total, vb0 + chunk);
        if (vb0 < vb1) {
            int q = p0, hi = p1 - 1;
            while (q < hi) {
                int mid = (q + hi + 1) >> 1;
                if (phases[mid].vbase <= vb0)
                    q = mid;
                else
                    hi = mid - 1;
            }
            int next = q + 1 < p1 ? phases[q + 1].vbase : 0x7fffffff;
            if (q != cur) {
                load_phase(phases, q, sp);
                cur = q;
            }
            bool skip = body && *(volatile int *)&D.states[sp.hier]->go == 0;
            for (int v = vb0; v < vb1; ++v) {
                while (v >= next) {
                    ++q;
                    next = q + 1 < p1 ? phases[q + 1].vbase : 0x7fffffff;
                    load_phase(phases, q, sp);
                    cur = q;
                    skip = body && *(volatile int *)&D.states[sp.hier]->go == 0;
                }
                if (skip) continue;
                int lv = v - sp.vbase;
                int bx = lv % sp.gx, by = (lv / sp.gx) % sp.gy, bz = lv / (sp.gx * sp.gy);
                dispatch(sp, bx, by, bz, dyn);
            }
        }
        if (!grid_sync(D.ctl, D.nblocks_expected, D.limit_ns, epoch)) return false;
    }
    return true;
}

// A recorded program: init rounds, then the body rounds while any
// hierarchy still iterates (its check op sets go), then the tail rounds.
// MINB blocks per SM: 4 for a single hierarchy (127 registers, no spills),
// 8 for batches (their many small phases want more resident blocks).
template <int MINB>
__global__ void __launch_bounds__(NT, MINB) k_program(const __grid_constant__ ProgramDesc D)
{
    extern __shared__ double dyn[];
    __shared__ __align__(16) unsigned char spbuf[sizeof(Phase)];
    Phase &sp = *reinterpret_cast<Phase *>(spbuf);
    int cur = -1;        // phase held in sp (uniform across the block)
    unsigned epoch = 0;  // barriers passed
    // batches: the hierarchies' flags cached once per iteration (they change
    // only in each hierarchy's last body phase, after which that hierarchy
    // has no phase left in the iteration)
    __shared__ unsigned char sgo[kGoCache];
    const bool cache = D.nhier > 1 && D.nhier <= kGoCache;
    if (!run_rounds(D, D.init_r0, D.init_r1, false, sp, cur, dyn, epoch)) return;
    for (int it = 0; it <= D.max_loops; ++it) {
        int any = 0;
        for (int h = 0; h < D.nhier; ++h) any |= *(volatile int *)&D.states[h]->go;
        if (!any) break;
        if (cache) {
            __syncthreads();
            for (int h = tid(); h < D.nhier; h += NT) sgo[h] = *(volatile int *)&D.states[h]->go != 0;
            __syncthreads();
        }
        if (!run_rounds(D, D.body_r0, D.body_r1, true, sp, cur, dyn, epoch, cache ? sgo : nullptr)) return;
    }
    run_rounds(D, D.tail_r0, D.tail_r1, false, sp, cur, dyn, epoch);
}

// Batched programs on thread-block clusters.  Every cluster (csize blocks,
// co-resident by construction, with a hardware barrier) takes the next
// hierarchy from a queue (largest first, so that the long solves start
// early) and runs that hierarchy's recorded solve alone: its init phases,
// its V-cycle body while its own convergence flag asks for one, its tail,
// each phase's virtual blocks spread over the cluster's blocks and the
// phases separated by the cluster barrier (release/acquire at cluster
// scope: the phases of a hierarchy are executed by this cluster only).  No
// grid-wide barrier: a cluster never waits for another, and hierarchies of
// all sizes progress side by side over the whole GPU.  The operations and
// their order per hierarchy are those of the solo solve, so the results are
// the same bits.
__global__ void __launch_bounds__(NT) k_cluster_program(const __grid_constant__ ClusterDesc D)
{
    extern __shared__ double dyn[];
    __shared__ __align__(16) unsigned char spbuf[sizeof(Phase)];
    Phase &sp = *reinterpret_cast<Phase *>(spbuf);
    const Phase *phases = (const Phase *)D.phases;
    const int rank = (int)cluster_rank(), C = (int)cluster_ctas();
    unsigned *slot = D.queue + 1 + blockIdx.x / (unsigned)C;
    auto run = [&](int q0, int q1) {
        for (int q = q0; q < q1; ++q) {
            load_phase(phases, q, sp);
            const int nvb = sp.gx * sp.gy * sp.gz;
            for (int v = rank; v < nvb; v += C) {
                const int bx = v % sp.gx, by = (v / sp.gx) % sp.gy, bz = v / (sp.gx * sp.gy);
                dispatch(sp, bx, by, bz, dyn);
            }
            cluster_barrier();
        }
    };
    for (;;) {
        if (rank == 0 && tid() == 0) *slot = atomicAdd(D.queue, 1u);
        cluster_barrier();
        const unsigned k = *(volatile unsigned *)slot;
        cluster_barrier(); // the slot is read before rank 0 writes it again
        if (k >= (unsigned)D.nhier) break;
        const int *sg = D.hseg + 6 * D.order[k];
        SolveState *st = D.states[D.order[k]];
        run(sg[0], sg[1]);
        for (int it = 0; it < D.max_loops; ++it) {
            if (*(volatile int *)&st->go == 0) break;
            run(sg[2], sg[3]);
        }
        run(sg[4], sg[5]);
    }
}

// Coarse footprint box of fine level l in level l-1 index space.
void footprint(const Hierarchy &H, int l, int lo[3], int n[3])
{
    for (int d = 0; d < 3; ++d) {
        lo[d] = H.L[l].vlo[d] >> 1;
        n[d] = (H.L[l].vhi[d] >> 1) - lo[d] + 1;
    }
}

// Launch configuration of the operation kernels (32 x 4 threads,
// programmatic dependent launch unless disabled) handed to f.
template <typename F>
void launch_config(Hierarchy &H, dim3 grid, size_t smem, F &&f)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(BX, BY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = H.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = H.pdl ? 1 : 0;
    f(cfg);
}

// Launch one operation (programmatic dependent launch on) or, while a
// program is being recorded, append it to the program.
template <int OP, typename A>
void issue(Hierarchy &H, dim3 grid, const A &args, A OpArgs::*member, size_t smem = 0)
{
    Phase P;
    memset(&P, 0, sizeof(P));
    P.op = OP;
    P.gx = (int)grid.x;
    P.gy = (int)grid.y;
    P.gz = (int)grid.z;
    P.hier = H.rec_hier;
    P.smem = smem;
    P.a.*member = args;
    if (H.rec) {
        H.rec->push_back(P);
        return;
    }
    if (H.grouping) {
        H.group->push_back(P);
        return;
    }
    launch_config(H, grid, smem, [&](cudaLaunchConfig_t &cfg) { cudaLaunchKernelEx(&cfg, k_op<OP>, P); });
}

} // namespace

// ------------------------------------------------- grouped launches

namespace {

void launch_single(Hierarchy &H, const Phase &P)
{
    dim3 grid((unsigned)P.gx, (unsigned)P.gy, (unsigned)P.gz);
    switch (P.op) {
#define AMR_L(OPX)                                                                                           \
    case OPX: launch_config(H, grid, P.smem, [&](cudaLaunchConfig_t &cfg) { cudaLaunchKernelEx(&cfg, k_op<OPX>, P); }); break;
        AMR_L(OP_RESIDUAL_D) AMR_L(OP_RESIDUAL_F) AMR_L(OP_RBGS_D) AMR_L(OP_RBGS_F) AMR_L(OP_RBGS_FIRST_D)
        AMR_L(OP_RBGS_FIRST_F) AMR_L(OP_RESTRICT_D) AMR_L(OP_RESTRICT_F) AMR_L(OP_PROLONG_D) AMR_L(OP_PROLONG_F)
        AMR_L(OP_ELEM_D) AMR_L(OP_ELEM_F) AMR_L(OP_CONV) AMR_L(OP_CP_D) AMR_L(OP_CP_F) AMR_L(OP_SURFACE_D)
        AMR_L(OP_SURFACE_F) AMR_L(OP_GRAD) AMR_L(OP_CF_GRAD) AMR_L(OP_AVGDOWN) AMR_L(OP_NORMS) AMR_L(OP_CHECK)
        AMR_L(OP_MG_RESTRICT_D) AMR_L(OP_MG_RESTRICT_F) AMR_L(OP_MG_PROLONG_D) AMR_L(OP_MG_PROLONG_F)
        AMR_L(OP_COARSE_D) AMR_L(OP_COARSE_F) AMR_L(OP_DEPOSIT) AMR_L(OP_GATHER) AMR_L(OP_DST_DD)
        AMR_L(OP_DST_FD) AMR_L(OP_DST_DF) AMR_L(OP_TRIZ) AMR_L(OP_RESIDUAL_PD) AMR_L(OP_RESIDUAL_PF)
        AMR_L(OP_RBGS_PD) AMR_L(OP_RBGS_PF) AMR_L(OP_MG_RESTRICT_PD) AMR_L(OP_MG_RESTRICT_PF)
        AMR_L(OP_FDST_DD) AMR_L(OP_FDST_FD) AMR_L(OP_FDST_DF) AMR_L(OP_AXIS_DD) AMR_L(OP_AXIS_FD)
        AMR_L(OP_AXIS_DF)
#undef AMR_L
    default: break;
    }
}

using GroupFn = void (*)(Hierarchy &, const GroupDesc &, int, size_t);

template <int A, int B>
void launch_group_k(Hierarchy &H, const GroupDesc &G, int nblocks, size_t smem)
{
    launch_config(H, dim3((unsigned)nblocks), smem,
                  [&](cudaLaunchConfig_t &cfg) { cudaLaunchKernelEx(&cfg, k_group<A, B>, G); });
}

// The fused kernels of the combinations the V-cycle driver groups.
GroupFn group_kernel(int a, int b)
{
    struct E {
        int a, b;
        GroupFn f;
    };
    static const E table[] = {
        {OP_RESIDUAL_D, OP_CP_D, &launch_group_k<OP_RESIDUAL_D, OP_CP_D>},
        {OP_RESIDUAL_D, OP_RESIDUAL_D, &launch_group_k<OP_RESIDUAL_D, OP_RESIDUAL_D>},
        {OP_SURFACE_D, OP_SURFACE_D, &launch_group_k<OP_SURFACE_D, OP_SURFACE_D>},
        {OP_RESTRICT_D, OP_RESIDUAL_D, &launch_group_k<OP_RESTRICT_D, OP_RESIDUAL_D>},
        {OP_RESTRICT_F, OP_RESIDUAL_F, &launch_group_k<OP_RESTRICT_F, OP_RESIDUAL_F>},
        {OP_PROLONG_D, OP_CP_D, &launch_group_k<OP_PROLONG_D, OP_CP_D>},
        {OP_PROLONG_F, OP_CP_F, &launch_group_k<OP_PROLONG_F, OP_CP_F>},
    };
    for (const E &e : table)
        if ((e.a == a && e.b == b) || (e.a == b && e.b == a)) return e.f;
    return nullptr;
}

} // namespace

void group_begin(Hierarchy &H)
{
    // (recorded programs keep one round per phase: packing a group into one
    // round measured slower, its extra phase changes per block costing more
    // than the grid barriers it saves; host-driven profiling times every
    // operation alone, the profiled graph times the groups as launched)
    if (H.rec || (H.prof && !H.capturing)) return;
    if (!H.group) H.group = new std::vector<Phase>();
    H.group->clear();
    H.group_prof.clear();
    H.grouping = true;
}

namespace {

// Profiled graph: event-record nodes around the launch of operations
// [i0, i1) of the closed group; each operation is charged its share of the
// group's algorithmic bytes (equal shares when the group has none).
struct GroupTimer {
    Hierarchy &H;
    int ev = -1;
    size_t i0, i1;
    GroupTimer(Hierarchy &h, size_t a, size_t b) : H(h), i0(a), i1(b)
    {
        if (!H.prof_capture || i0 >= H.group_prof.size()) return;
        ev = Launch::prof_event_pair(H);
        Launch::prof_record(H, ev);
    }
    ~GroupTimer()
    {
        if (ev < 0) return;
        Launch::prof_record(H, ev + 1);
        const size_t hi = std::min(i1, H.group_prof.size());
        double tot = 0.0;
        for (size_t i = i0; i < hi; ++i) tot += H.group_prof[i].bytes;
        for (size_t i = i0; i < hi; ++i) {
            ProfRecord r = H.group_prof[i];
            r.ev = ev;
            r.share = tot > 0.0 ? r.bytes / tot : 1.0 / (double)(hi - i0);
            H.pending.push_back(r);
        }
    }
};

} // namespace

void group_end(Hierarchy &H)
{
    if (!H.grouping) return;
    H.grouping = false;
    std::vector<Phase> &ph = *H.group;
    if (ph.empty()) return;
    int a = ph[0].op, b = a;
    bool two = true;
    for (const Phase &p : ph)
        if (p.op != a) {
            if (b == a)
                b = p.op;
            else if (p.op != b)
                two = false;
        }
    GroupFn f = (ph.size() >= 2 && ph.size() <= (size_t)kMaxGroup && two) ? group_kernel(a, b) : nullptr;
    if (!f) {
        for (size_t i = 0; i < ph.size(); ++i) {
            GroupTimer gt(H, i, i + 1);
            launch_single(H, ph[i]);
            H.launches++;
        }
        ph.clear();
        return;
    }
    GroupDesc G;
    memset(&G, 0, sizeof(G));
    G.n = (int)ph.size();
    int v = 0;
    size_t smem = 0;
    for (int i = 0; i < G.n; ++i) {
        G.vstart[i] = v;
        G.ph[i] = ph[i];
        v += ph[i].gx * ph[i].gy * ph[i].gz;
        smem = std::max(smem, ph[i].smem);
    }
    G.vstart[G.n] = v;
    ph.clear();
    if (v == 0) return;
    GroupTimer gt(H, 0, (size_t)G.n);
    f(H, G, v, smem);
    H.launches++;
}

void group_free(Hierarchy &H)
{
    delete H.group;
    H.group = nullptr;
}

double valid_cells(const Hierarchy &H, const Grid &g)
{
    for (int l = 0; l < H.nlev; ++l)
        if (H.L[l].g.mask == g.mask) return (double)H.L[l].nvalid;
    return (double)(g.n[0] - 2) * (g.n[1] - 2) * (g.n[2] - 2);
}

int prof_resolve(Hierarchy &H)
{
    if (H.pending.empty()) return AMR_OK;
    cudaError_t e = cudaStreamSynchronize(H.stream);
    if (e != cudaSuccess) return cuda_fail(e, "profile");
    for (const ProfRecord &r : H.pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, H.evpool[r.ev], H.evpool[r.ev + 1]);
        H.kind_ms[r.kind] += ms * r.share;
        H.kind_bytes[r.kind] += r.bytes;
        H.kind_flops[r.kind] += r.flops;
        H.kind_ops[r.kind] += r.ops;
        H.kind_launches[r.kind]++;
    }
    H.pending.clear();
    H.evnext = 0;
    return AMR_OK;
}

const char *kind_name(int kind)
{
    static const char *names[K_NUM] = {"deposit",     "gather",      "residual",    "rbgs",         "restrict",
                                       "prolong",     "finish",      "cf_correct",  "flux",         "grad",
                                       "average_down", "norms",      "mg_restrict", "mg_prolong",   "coarse_solve",
                                       "elementwise", "coarse_part", "check", "mg_bottom", "bin",
                                       "sine_transform", "tridiagonal"};
    return (kind >= 0 && kind < K_NUM) ? names[kind] : "";
}

// ------------------------------------------------------------- launchers

template <typename T>
void launch_residual(Hierarchy &H, const Grid &g, const T *rho, const T *phi, T *res, int comp, int zero_covered)
{
    Launch L(H, K_RESIDUAL, 3.0 * sizeof(T) * valid_cells(H, g));
    ResidualA<T> A{g, rho, phi, res, comp, zero_covered, 0};
    if (g.clist && !g.periodic) {
        const int64_t m = (int64_t)g.ccnt[0] + g.ccnt[1];
        const dim3 lg((unsigned)std::max<int64_t>(1, (m + NT - 1) / NT), 1u, 1u);
        A.listed = 1;
        if constexpr (sizeof(T) == 8)
            issue<OP_RESIDUAL_D>(H, lg, A, &OpArgs::res_d);
        else
            issue<OP_RESIDUAL_F>(H, lg, A, &OpArgs::res_f);
        return;
    }
    if constexpr (sizeof(T) == 8) {
        if (g.periodic)
            issue<OP_RESIDUAL_PD>(H, cell_grid(g), A, &OpArgs::res_d);
        else
            issue<OP_RESIDUAL_D>(H, cell_grid(g), A, &OpArgs::res_d);
    } else {
        if (g.periodic)
            issue<OP_RESIDUAL_PF>(H, cell_grid(g), A, &OpArgs::res_f);
        else
            issue<OP_RESIDUAL_F>(H, cell_grid(g), A, &OpArgs::res_f);
    }
}

template <typename T>
void launch_rbgs(Hierarchy &H, const Grid &g, T *x, const T *b, int colour, int first, int mode, T *e, T *phi)
{
    // algorithmic bytes of one colour: the other colour's values, this
    // colour's right-hand side and new values, every cell's mask; flops:
    // 8 per updated cell (five adds, one FMA, one multiply)
    double cells = valid_cells(H, g);
    double bytes = (1.5 * sizeof(T) + 1.0) * cells;
    if (mode == 1) bytes += 2.0 * sizeof(T) * cells;
    if (mode == 2) bytes += 1.0 * sizeof(T) * cells;
    // per updated cell 8 flops in 7 instructions (5 adds, an FMA, a multiply);
    // from zero 3 flops, 2 multiplies
    Launch L(H, K_RBGS, bytes, (first ? 3.0 : 8.0) * 0.5 * cells, (first ? 2.0 : 7.0) * 0.5 * cells);
    RbgsA<T> A{g, x, b, colour, mode, e, phi, 0};
    if (g.clist && !g.periodic) {
        // one thread per listed cell of the colour (of both colours from zero)
        const int64_t m = first ? (int64_t)g.ccnt[0] + g.ccnt[1] : (int64_t)g.ccnt[colour];
        const dim3 lg((unsigned)std::max<int64_t>(1, (m + NT - 1) / NT), 1u, 1u);
        A.listed = 1;
        if constexpr (sizeof(T) == 8) {
            if (first)
                issue<OP_RBGS_FIRST_D>(H, lg, A, &OpArgs::rb_d);
            else
                issue<OP_RBGS_D>(H, lg, A, &OpArgs::rb_d);
        } else {
            if (first)
                issue<OP_RBGS_FIRST_F>(H, lg, A, &OpArgs::rb_f);
            else
                issue<OP_RBGS_F>(H, lg, A, &OpArgs::rb_f);
        }
        return;
    }
    if constexpr (sizeof(T) == 8)
    {
        if (first)
            issue<OP_RBGS_FIRST_D>(H, cell_grid(g), A, &OpArgs::rb_d);
        else if (g.periodic)
            issue<OP_RBGS_PD>(H, colour_grid(g), A, &OpArgs::rb_d);
        else
            issue<OP_RBGS_D>(H, colour_grid(g), A, &OpArgs::rb_d);
    } else {
        if (first)
            issue<OP_RBGS_FIRST_F>(H, cell_grid(g), A, &OpArgs::rb_f);
        else if (g.periodic)
            issue<OP_RBGS_PF>(H, colour_grid(g), A, &OpArgs::rb_f);
        else
            issue<OP_RBGS_F>(H, colour_grid(g), A, &OpArgs::rb_f);
    }
}

template <typename T>
void launch_restrict_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l], &C = H.L[l - 1];
    Fields<T> ff = fields<T>(F), fc = fields<T>(C);
    RestrictA<T> A{};
    A.gf = F.g;
    A.gc = C.g;
    footprint(H, l, A.clo, A.cn);
    A.rf = ff.res;
    A.ef = ff.err;
    A.phif = ff.phi;
    A.rc = fc.res;
    dim3 grid((unsigned)(((int64_t)A.cn[0] * A.cn[1] + NT - 1) / NT), 1u, (unsigned)A.cn[2]);
    if (C.cov && C.ncov > 0) {
        A.cov = C.cov;
        A.ncov = C.ncov;
        grid = dim3((unsigned)((C.ncov + NT - 1) / NT), 1u, 1u);
    }
    Launch L(H, K_RESTRICT, (5.0 + 1.0 / 8) * sizeof(T) * (double)F.nvalid);
    if constexpr (sizeof(T) == 8)
        issue<OP_RESTRICT_D>(H, grid, A, &OpArgs::rs_d);
    else
        issue<OP_RESTRICT_F>(H, grid, A, &OpArgs::rs_f);
}

template <typename T>
void launch_prolong_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l], &C = H.L[l - 1];
    Fields<T> ff = fields<T>(F), fc = fields<T>(C);
    ProlongA<T> A{F.g, C.g, ff.err, ff.res, ff.phi, fc.err, 0};
    Launch L(H, K_PROLONG, (6.0 + 1.0 / 8) * sizeof(T) * (double)F.nvalid);
    dim3 grid = cell_grid(F.g);
    if (F.g.clist && !F.g.periodic) {
        const int64_t m = (int64_t)F.g.ccnt[0] + F.g.ccnt[1];
        grid = dim3((unsigned)std::max<int64_t>(1, (m + NT - 1) / NT), 1u, 1u);
        A.listed = 1;
    }
    if constexpr (sizeof(T) == 8)
        issue<OP_PROLONG_D>(H, grid, A, &OpArgs::pr_d);
    else
        issue<OP_PROLONG_F>(H, grid, A, &OpArgs::pr_f);
}

template <typename T>
void launch_elem(Hierarchy &H, int kind, T *a, const T *b, T *c, T v, int64_t n, int prof_kind, double bytes)
{
    unsigned nb = elem_blocks(n);
    ElemA<T> A{n, (int64_t)nb * NT, kind, v, a, b, c};
    Launch L(H, prof_kind, bytes);
    if constexpr (sizeof(T) == 8)
        issue<OP_ELEM_D>(H, dim3(nb), A, &OpArgs::el_d);
    else
        issue<OP_ELEM_F>(H, dim3(nb), A, &OpArgs::el_f);
}

template <typename T>
void launch_finish_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l];
    Fields<T> ff = fields<T>(F);
    launch_elem<T>(H, 2, ff.err, ff.de, ff.phi, T(0), F.g.ncell, K_FINISH, 5.0 * sizeof(T) * (double)F.nvalid);
}

template <typename T>
void launch_fill(Hierarchy &H, T *p, T v, int64_t n)
{
    launch_elem<T>(H, 0, p, nullptr, nullptr, v, n, K_ELEMENTWISE, sizeof(T) * (double)n);
}

template <typename T>
void launch_axpy(Hierarchy &H, T *y, const T *x, T a, int64_t n)
{
    launch_elem<T>(H, 1, y, x, nullptr, a, n, K_ELEMENTWISE, 3.0 * sizeof(T) * (double)n);
}

void launch_to32(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    unsigned nb = elem_blocks(L.g.ncell);
    ConvA A{L.g.ncell, (int64_t)nb * NT, 0, L.mask, L.res, nullptr, L.rho32, L.res32, L.phi32};
    Launch Lc(H, K_ELEMENTWISE, 20.0 * (double)L.g.ncell);
    issue<OP_CONV>(H, dim3(nb), A, &OpArgs::conv);
}

void launch_add32(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    unsigned nb = elem_blocks(L.g.ncell);
    ConvA A{L.g.ncell, (int64_t)nb * NT, 1, L.mask, nullptr, L.phi, nullptr, nullptr, L.phi32};
    Launch Lc(H, K_ELEMENTWISE, 20.0 * (double)L.g.ncell);
    issue<OP_CONV>(H, dim3(nb), A, &OpArgs::conv);
}

template <typename T>
void launch_cp(Hierarchy &H, int l, const T *uc)
{
    CfTable &Tb = H.L[l].cf;
    if (Tb.nface == 0) return;
    CpA<T> A{Tb.nface, Tb.cnt, Tb.cidx, Tb.cw, uc, Tb.cp};
    Launch L(H, K_CP, Tb.nface * (8.0 + 9 * (12.0 + sizeof(T))));
    dim3 grid((unsigned)((Tb.nface + NT - 1) / NT));
    if constexpr (sizeof(T) == 8)
        issue<OP_CP_D>(H, grid, A, &OpArgs::cp_d);
    else
        issue<OP_CP_F>(H, grid, A, &OpArgs::cp_f);
}

void launch_cp_zero(Hierarchy &H, int l)
{
    CfTable &Tb = H.L[l].cf;
    if (Tb.nface == 0) return;
    launch_fill<double>(H, Tb.cp, 0.0, Tb.nface);
}

template <typename T>
void launch_surface(Hierarchy &H, int lf, T *rf, int lc, const T *uf, T *rc)
{
    SurfaceA<T> A{};
    double bytes = 0.0;
    if (lf > 0 && H.L[lf].cf.ncell) {
        CfTable &Tb = H.L[lf].cf;
        A.ncell = Tb.ncell;
        A.cell_f = Tb.cell_f;
        A.cell_ptr = Tb.cell_ptr;
        A.cp_f = Tb.cp;
        A.rf = rf;
        A.scale_f = H.L[lf].g.ih2;
        bytes += (8.0 + 2.0 * sizeof(T)) * Tb.ncell + 8.0 * Tb.nface;
    }
    if (lc > 0 && H.L[lc].cf.ncrse) {
        CfTable &Tb = H.L[lc].cf;
        A.ncrse = Tb.ncrse;
        A.crse_c = Tb.crse_c;
        A.crse_ptr = Tb.crse_ptr;
        A.crse_face = Tb.crse_face;
        A.ff = Tb.f;
        A.ff1 = Tb.f1;
        A.cp_c = Tb.cp;
        A.uf = uf;
        A.rc = rc;
        A.scale_c = 0.5 * H.L[lc - 1].g.ih2;
        bytes += (8.0 + 2.0 * sizeof(T)) * Tb.ncrse + (16.0 + 2.0 * sizeof(T)) * Tb.nface;
    }
    int n = A.ncell + A.ncrse;
    if (n == 0) return;
    Launch L(H, K_FLUX, bytes);
    dim3 grid((unsigned)((n + NT - 1) / NT));
    if constexpr (sizeof(T) == 8)
        issue<OP_SURFACE_D>(H, grid, A, &OpArgs::sf_d);
    else
        issue<OP_SURFACE_F>(H, grid, A, &OpArgs::sf_f);
}

void launch_grad(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    GradA A{L.g, L.phi, L.ef[0], L.ef[1], L.ef[2]};
    Launch Lc(H, K_GRAD, 32.0 * (double)L.nvalid);
    issue<OP_GRAD>(H, cell_grid(L.g), A, &OpArgs::grad);
}

void launch_cf_grad(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    CfTable &Tb = L.cf;
    if (Tb.ncell == 0) return;
    CfGradA A{Tb.ncell, Tb.cell_f, Tb.cell_ptr, Tb.dir, Tb.cp, L.ef[0], L.ef[1], L.ef[2], 0.5 / L.g.h};
    Launch Lc(H, K_CF, 48.0 * Tb.ncell + 8.0 * Tb.nface);
    issue<OP_CF_GRAD>(H, dim3((unsigned)((Tb.ncell + NT - 1) / NT)), A, &OpArgs::cfg);
}

void launch_average_down(Hierarchy &H, int l)
{
    Level &F = H.L[l + 1], &C = H.L[l];
    AvgDownA A{};
    A.gf = F.g;
    A.gc = C.g;
    footprint(H, l + 1, A.clo, A.cn);
    A.uf = F.phi;
    A.uc = C.phi;
    dim3 grid((unsigned)((A.cn[0] + BX - 1) / BX), (unsigned)((A.cn[1] + BY - 1) / BY), (unsigned)A.cn[2]);
    Launch Lc(H, K_AVGDOWN, 9.0 * (double)F.nvalid);
    issue<OP_AVGDOWN>(H, grid, A, &OpArgs::avg);
}

void launch_norms_check(Hierarchy &H, int with_rho, int is_body, unsigned long long cond, int use_cond)
{
    NormA A{};
    double bytes = 0.0;
    int ns = 0;
    for (int l = 0; l < H.nlev; ++l, ++ns) {
        A.n[ns] = H.L[l].g.ncell;
        A.mask[ns] = H.L[l].mask;
        A.v[ns] = H.L[l].res;
        A.covered_too[ns] = 0;
        bytes += 9.0 * (double)H.L[l].g.ncell;
    }
    if (with_rho)
        for (int l = 0; l < H.nlev; ++l, ++ns) {
            A.n[ns] = H.L[l].g.ncell;
            A.mask[ns] = H.L[l].mask;
            A.v[ns] = H.L[l].rho;
            A.covered_too[ns] = 1;
            bytes += 9.0 * (double)H.L[l].g.ncell;
        }
    A.nslots = ns;
    A.part = H.partials;
    A.prm = H.params;
    A.vec = 1;
    for (int q = 0; q < ns; ++q)
        if ((reinterpret_cast<uintptr_t>(A.v[q]) & 15) || (reinterpret_cast<uintptr_t>(A.mask[q]) & 3)) A.vec = 0;
    // partial blocks sized to the largest slot (16 cells per thread), at
    // most kPartialBlocks
    int64_t nmax = 0;
    for (int q = 0; q < ns; ++q) nmax = std::max(nmax, A.n[q]);
    int nb = (int)std::min<int64_t>(kPartialBlocks, std::max<int64_t>(1, (nmax + NT * 16 - 1) / (NT * 16)));
    A.nblocks = nb;
    CheckA C{H.partials, H.nlev, with_rho, is_body, use_cond, nb, H.params, H.state,
             (cudaGraphConditionalHandle)cond};
    if (!H.rec && (!H.prof || H.capturing) && H.nc_counter) {
        // one launch: norms, then the test in the last block to finish
        Launch Lc(H, K_NORMS, bytes + 24.0 * nb * ns);
        launch_config(H, dim3(nb, ns), 0, [&](cudaLaunchConfig_t &cfg) {
            cudaLaunchKernelEx(&cfg, k_norms_check, A, C, H.nc_counter);
        });
        return;
    }
    {
        Launch Lc(H, K_NORMS, bytes);
        issue<OP_NORMS>(H, dim3(nb, ns), A, &OpArgs::norm);
    }
    Launch Lc(H, K_CHECK, 24.0 * nb * ns);
    issue<OP_CHECK>(H, dim3(1), C, &OpArgs::chk);
}

template <typename T>
void launch_mg_restrict(Hierarchy &H, int g, int first_red)
{
    MgGrid &F = H.mg[g], &C = H.mg[g + 1];
    MgRestrictA<T> A{F.g, C.g, mg_e<T>(F), mg_r<T>(F), mg_r<T>(C), mg_e<T>(C), first_red};
    Launch Lc(H, K_MG_RESTRICT, 2.0 * sizeof(T) * (valid_cells(H, F.g) + valid_cells(H, C.g)));
    if constexpr (sizeof(T) == 8) {
        if (F.g.periodic)
            issue<OP_MG_RESTRICT_PD>(H, cell_grid(C.g), A, &OpArgs::mr_d);
        else
            issue<OP_MG_RESTRICT_D>(H, cell_grid(C.g), A, &OpArgs::mr_d);
    } else {
        if (F.g.periodic)
            issue<OP_MG_RESTRICT_PF>(H, cell_grid(C.g), A, &OpArgs::mr_f);
        else
            issue<OP_MG_RESTRICT_F>(H, cell_grid(C.g), A, &OpArgs::mr_f);
    }
}

template <typename T>
void launch_mg_prolong(Hierarchy &H, int g)
{
    MgGrid &F = H.mg[g], &C = H.mg[g + 1];
    MgProlongA<T> A{F.g, C.g, mg_e<T>(F), mg_e<T>(C)};
    Launch Lc(H, K_MG_PROLONG, 2.0 * sizeof(T) * valid_cells(H, F.g) + sizeof(T) * valid_cells(H, C.g));
    if constexpr (sizeof(T) == 8)
        issue<OP_MG_PROLONG_D>(H, cell_grid(F.g), A, &OpArgs::mp_d);
    else
        issue<OP_MG_PROLONG_F>(H, cell_grid(F.g), A, &OpArgs::mp_f);
}

template <typename T>
void launch_mg_coarse_solve(Hierarchy &H)
{
    MgGrid &G = H.mg[H.nmg - 1];
    if (H.csep_n > 0) {
        // separable: V^T along x, y, z (the last divides by the eigenvalue
        // sums), then V along z, y, x; FP64 between the passes
        const int n = H.csep_n;
        const double n3 = (double)n * n * n;
        const dim3 grid((unsigned)((n * n * n + NT - 1) / NT));
        double *t1 = H.csep_tmp[0], *t2 = H.csep_tmp[1];
        const Grid &g = G.g;
        auto pass = [&](auto in, auto out, int axis, const double *M, const double *lam) {
            using TI = std::remove_const_t<std::remove_pointer_t<decltype(in)>>;
            using TO = std::remove_pointer_t<decltype(out)>;
            AxisA<TI, TO> A{n, axis, g.sy, g.sz, in, out, M, lam, g.h2, H.csep_zero_add};
            Launch Lc(H, K_COARSE, (2.0 * 8.0 + 8.0) * n3, 2.0 * n * n3, n * n3);
            if constexpr (sizeof(TI) == 8 && sizeof(TO) == 8)
                issue<OP_AXIS_DD>(H, grid, A, &OpArgs::ax_dd);
            else if constexpr (sizeof(TI) == 4)
                issue<OP_AXIS_FD>(H, grid, A, &OpArgs::ax_fd);
            else
                issue<OP_AXIS_DF>(H, grid, A, &OpArgs::ax_df);
        };
        pass((const T *)mg_r<T>(G), t1, 0, H.csep_vt, nullptr);
        pass((const double *)t1, t2, 1, H.csep_vt, nullptr);
        pass((const double *)t2, t1, 2, H.csep_vt, H.csep_lam);
        pass((const double *)t1, t2, 2, H.csep_v, nullptr);
        pass((const double *)t2, t1, 1, H.csep_v, nullptr);
        pass((const double *)t1, mg_e<T>(G), 0, H.csep_v, nullptr);
        return;
    }
    int m = H.ncoarse;
    CoarseA<T> A{G.g, m, H.coarse_inv, mg_r<T>(G), mg_e<T>(G)};
    dim3 grid((unsigned)((m + NT / 32 - 1) / (NT / 32)));
    Launch Lc(H, K_COARSE, 8.0 * (double)m * m + 2.0 * sizeof(T) * m);
    if constexpr (sizeof(T) == 8)
        issue<OP_COARSE_D>(H, grid, A, &OpArgs::co_d, sizeof(double) * (size_t)m);
    else
        issue<OP_COARSE_F>(H, grid, A, &OpArgs::co_f, sizeof(double) * (size_t)m);
}

namespace {
__global__ void k_make_code(const Grid g, uint8_t *code)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.ncell) return;
    int a = (int)(p % g.sy), b = (int)((p / g.sy) % g.n[1]), c = (int)(p / g.sz);
    const int pos[3] = {a, b, c};
    const int64_t st[3] = {1, g.sy, g.sz};
    unsigned v = g.mask[p] != 0 ? 64u : 0u;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        int d = f >> 1, s = (f & 1) ? 1 : -1;
        int q = pos[d] + s;
        if (q >= 0 && q < g.n[d] && g.mask[p + s * st[d]] != 0) v |= 1u << f;
    }
    code[p] = (uint8_t)v;
}
} // namespace

void launch_make_code(Hierarchy &H, const Grid &g, uint8_t *code)
{
    unsigned nb = (unsigned)((g.ncell + 255) / 256);
    k_make_code<<<nb, 256, 0, H.stream>>>(g, code);
}

// The same solve with the fast transforms (op_fdst): n^2 lines per
// transform, kFdstElems / n to a virtual block.
template <typename T>
void launch_fdst_bottom(Hierarchy &H)
{
    Level &L0 = H.L[0];
    Fields<T> f = fields<T>(L0);
    const Grid &g = L0.g;
    const int n = H.n0;
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    const int L = kFdstElems / n;
    const double n3 = (double)n * n * n;
    const dim3 blocks((unsigned)(n * n / L));
    const size_t smem = 2 * sizeof(double) * (size_t)kFdstElems;
    // each transform: n^3 values in and out; per value log2(n) splits and
    // combines (3 + 1 flops per pair)
    const double tb = 16.0 * n3, tf = 2.0 * lg * n3;
    {
        Launch Lc(H, K_DST, tb, tf, tf);
        FdstA<T, double> A{n, lg, L, 0, 0, g.sy, g.sz, f.res, H.dst_a, H.dst_tab, nullptr};
        if constexpr (sizeof(T) == 8)
            issue<OP_FDST_DD>(H, blocks, A, &OpArgs::fdst_dd, smem);
        else
            issue<OP_FDST_FD>(H, blocks, A, &OpArgs::fdst_fd, smem);
    }
    {
        Launch Lc(H, K_DST, tb, tf, tf);
        FdstA<double, double> A{n, lg, L, 1, 0, g.sy, g.sz, H.dst_a, H.dst_b, H.dst_tab, nullptr};
        issue<OP_FDST_DD>(H, blocks, A, &OpArgs::fdst_dd, smem);
    }
    {
        Launch Lc(H, K_TRIZ, 24.0 * n3, 10.0 * n3, 7.0 * n3);
        TrizA A{n, g.sy, g.sz, H.dst_b, H.dst_iw, g.h2, H.dst_fm};
        issue<OP_TRIZ>(H, dim3((unsigned)((n * n + 4 * kTrizModes - 1) / (4 * kTrizModes))), A, &OpArgs::triz);
    }
    {
        Launch Lc(H, K_DST, tb, tf, tf);
        FdstA<double, double> A{n, lg, L, 1, 1, g.sy, g.sz, H.dst_b, H.dst_a, H.dst_tab, nullptr};
        issue<OP_FDST_DD>(H, blocks, A, &OpArgs::fdst_dd, smem);
    }
    {
        Launch Lc(H, K_DST, tb + 2.0 * sizeof(T) * n3, tf, tf + n3);
        FdstA<double, T> A{n, lg, L, 0, 1, g.sy, g.sz, H.dst_a, f.err, H.dst_tab, f.phi};
        if constexpr (sizeof(T) == 8)
            issue<OP_FDST_DD>(H, blocks, A, &OpArgs::fdst_dd, smem);
        else
            issue<OP_FDST_DF>(H, blocks, A, &OpArgs::fdst_df, smem);
    }
}

template <typename T>
void launch_dst_bottom(Hierarchy &H)
{
    if (H.dst_fast) {
        launch_fdst_bottom<T>(H);
        return;
    }
    Level &L0 = H.L[0];
    Fields<T> f = fields<T>(L0);
    const Grid &g = L0.g;
    const int n = H.n0;
    const double n3 = (double)n * n * n;
    const dim3 lines((unsigned)((n * n + kDstLines - 1) / kDstLines));
    const size_t smem = 2 * sizeof(double) * (size_t)kDstLines * n;
    // each transform: n^3 values in and out, 3 n^4 / 4 flops (3n/8 FMAs per
    // value after the two folds)
    const double tb = 16.0 * n3, tf = 0.75 * n3 * n;
    {
        Launch Lc(H, K_DST, tb, tf, 0.5 * tf);
        DstA<T, double> A{n, 0, 0, g.sy, g.sz, f.res, H.dst_a, H.dst_mf, nullptr};
        if constexpr (sizeof(T) == 8)
            issue<OP_DST_DD>(H, lines, A, &OpArgs::dst_dd, smem);
        else
            issue<OP_DST_FD>(H, lines, A, &OpArgs::dst_fd, smem);
    }
    {
        Launch Lc(H, K_DST, tb, tf, 0.5 * tf);
        DstA<double, double> A{n, 1, 0, g.sy, g.sz, H.dst_a, H.dst_b, H.dst_mf, nullptr};
        issue<OP_DST_DD>(H, lines, A, &OpArgs::dst_dd, smem);
    }
    {
        Launch Lc(H, K_TRIZ, 24.0 * n3, 10.0 * n3, 7.0 * n3);
        TrizA A{n, g.sy, g.sz, H.dst_b, H.dst_iw, g.h2, nullptr};
        issue<OP_TRIZ>(H, dim3((unsigned)((n * n + 4 * kTrizModes - 1) / (4 * kTrizModes))), A, &OpArgs::triz);
    }
    {
        Launch Lc(H, K_DST, tb, tf, 0.5 * tf);
        DstA<double, double> A{n, 1, 1, g.sy, g.sz, H.dst_b, H.dst_a, H.dst_mi, nullptr};
        issue<OP_DST_DD>(H, lines, A, &OpArgs::dst_dd, smem);
    }
    {
        Launch Lc(H, K_DST, tb + 2.0 * sizeof(T) * n3, tf, 0.5 * tf + n3);
        DstA<double, T> A{n, 0, 1, g.sy, g.sz, H.dst_a, f.err, H.dst_mi, f.phi};
        if constexpr (sizeof(T) == 8)
            issue<OP_DST_DD>(H, lines, A, &OpArgs::dst_dd, smem);
        else
            issue<OP_DST_DF>(H, lines, A, &OpArgs::dst_df, smem);
    }
}

template void launch_dst_bottom<double>(Hierarchy &);
template void launch_dst_bottom<float>(Hierarchy &);

// ------------------------------------------------- particle binning

namespace {

constexpr int kBinBrick = 8;
constexpr uint32_t kNoKey = 0xFFFFFFFFu;

struct BinA {
    int nlev, nkeys;
    Grid g[kMaxLevels];
    double ih[kMaxLevels];
    int nb[kMaxLevels][3];
    int off[kMaxLevels];
    const double *x, *y, *z;
    int64_t n;
    uint32_t *keys;
    unsigned *cnt; // nkeys + 1 buckets (the last one: particles without a key)
};

// Key of each particle (the brick of its cell on the finest level whose
// valid cells hold all 8 of its CIC nodes; kNoKey if none) and the bucket
// counts.
__global__ void k_bin_keys(const __grid_constant__ BinA A)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.n) return;
    const double px = A.x[t], py = A.y[t], pz = A.z[t];
    uint32_t key = kNoKey;
    if (finite_bits(px) && finite_bits(py) && finite_bits(pz)) {
        const double pos[3] = {px, py, pz};
        for (int l = A.nlev - 1; l >= 0; --l) {
            const Grid &g = A.g[l];
            const double ih = A.ih[l];
            int loc[3];
            double w1;
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                cic_axis(pos[d], ih, g.lo[d], loc[d], w1);
                ok &= (loc[d] >= 0 && loc[d] + 1 < g.n[d]);
            }
            if (!ok) continue;
            const int64_t base = (int64_t)loc[2] * g.sz + (int64_t)loc[1] * g.sy + loc[0];
            const int64_t co[8] = {0, 1, g.sy, g.sy + 1, g.sz, g.sz + 1, g.sz + g.sy, g.sz + g.sy + 1};
#pragma unroll
            for (int o = 0; o < 8; ++o) ok &= (g.mask[base + co[o]] != 0);
            if (!ok) continue;
            // the particle's cell is one of its nodes, so it lies in the box
            int br[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) br[d] = (__double2int_rd(pos[d] * ih) - g.lo[d]) / kBinBrick;
            key = (uint32_t)(A.off[l] + br[0] + A.nb[l][0] * (br[1] + A.nb[l][1] * br[2]));
            break;
        }
    }
    A.keys[t] = key;
    atomicAdd(&A.cnt[key == kNoKey ? A.nkeys : (int)key], 1u);
}

// Exclusive prefix sum of the m bucket counts, in place, by one block.
__global__ void __launch_bounds__(1024) k_bin_scan(unsigned *cnt, int m)
{
    __shared__ unsigned part[1024];
    const int t = threadIdx.x, chunk = (m + 1023) / 1024;
    const int a0 = min(m, t * chunk), a1 = min(m, a0 + chunk);
    unsigned s = 0;
    for (int i = a0; i < a1; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - s; // exclusive
    for (int i = a0; i < a1; ++i) {
        unsigned c = cnt[i];
        cnt[i] = run;
        run += c;
    }
}

// perm[offset of the particle's bucket + arrival order] = particle.
__global__ void k_bin_scatter(const uint32_t *keys, int64_t n, int nkeys, unsigned *pos, int64_t *perm)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t key = keys[t];
    const unsigned p = atomicAdd(&pos[key == kNoKey ? nkeys : (int)key], 1u);
    perm[p] = t;
}

} // namespace

int64_t bin_num_keys(const Hierarchy &H)
{
    int64_t tot = 0;
    for (int l = 0; l < H.nlev; ++l) {
        int64_t c = 1;
        for (int d = 0; d < 3; ++d) c *= (H.L[l].vhi[d] - H.L[l].vlo[d] + 1 + kBinBrick - 1) / kBinBrick;
        tot += c;
    }
    return tot;
}

int launch_bin(Hierarchy &H, const double *x, const double *y, const double *z, int64_t n, uint32_t *keys,
               int64_t *perm)
{
    BinA A{};
    A.nlev = H.nlev;
    int64_t off = 0;
    for (int l = 0; l < H.nlev; ++l) {
        A.g[l] = H.L[l].g;
        A.ih[l] = 1.0 / H.L[l].g.h;
        int64_t c = 1;
        for (int d = 0; d < 3; ++d) {
            A.nb[l][d] = (H.L[l].vhi[d] - H.L[l].vlo[d] + 1 + kBinBrick - 1) / kBinBrick;
            c *= A.nb[l][d];
        }
        A.off[l] = (int)off;
        off += c;
    }
    A.nkeys = (int)off;
    if (!H.bin_cnt) {
        if (cudaMallocAsync((void **)&H.bin_cnt, sizeof(unsigned) * (size_t)(off + 1), H.stream) != cudaSuccess) {
            cudaGetLastError();
            H.bin_cnt = nullptr;
            set_error("out of memory (binning)");
            return AMR_ENOMEM;
        }
        H.allocs.push_back(H.bin_cnt);
        H.device_bytes += (int64_t)sizeof(unsigned) * (off + 1);
    }
    if (n == 0) return AMR_OK;
    A.x = x;
    A.y = y;
    A.z = z;
    A.n = n;
    A.keys = keys;
    A.cnt = H.bin_cnt;
    cudaMemsetAsync(H.bin_cnt, 0, sizeof(unsigned) * (size_t)(off + 1), H.stream);
    const unsigned nb = (unsigned)((n + 255) / 256);
    {
        Launch L(H, K_BIN, 32.0 * (double)n);
        k_bin_keys<<<nb, 256, 0, H.stream>>>(A);
    }
    {
        Launch L(H, K_BIN, 8.0 * (double)(off + 1));
        k_bin_scan<<<1, 1024, 0, H.stream>>>(H.bin_cnt, (int)off + 1);
    }
    {
        Launch L(H, K_BIN, 12.0 * (double)n);
        k_bin_scatter<<<nb, 256, 0, H.stream>>>(keys, n, (int)off, H.bin_cnt, perm);
    }
    return AMR_OK;
}

int mg_bottom_grid(const Hierarchy &H)
{
    if (H.csep_n > 0) return -1; // the one-cluster bottom needs the dense coarsest inverse
    // opt-in: on GB300 the FP64 work of the bottom grids is ALU-bound on the
    // cluster's 16 SMs (about two FP64 lanes each), which makes one cluster
    // launch slower than the ~20 graph-launched kernels it replaces
    const char *s = getenv("AMR_MG_BOTTOM");
    if (!s || s[0] != '1' || H.periodic) return -1; // (its smoother has no periodic images)
    for (int g = 1; g + 1 < H.nmg && g < kBottomMaxGrids; ++g) {
        const Grid &G = H.mg[g].g;
        if ((int64_t)(G.n[0] - 2) * (G.n[1] - 2) * (G.n[2] - 2) <= kBottomCells) return g;
    }
    return -1;
}

template <typename T>
void launch_mg_bottom(Hierarchy &H, int gb, int nu1, int nu2)
{
    BottomA<T> A{};
    A.gb = gb;
    A.nmg = H.nmg;
    A.nu1 = nu1;
    A.nu2 = nu2;
    double bytes = 0.0;
    for (int g = 0; g < H.nmg; ++g) {
        A.g[g] = H.mg[g].g;
        A.e[g] = mg_e<T>(H.mg[g]);
        A.r[g] = mg_r<T>(H.mg[g]);
        if (g >= gb) {
            double cells = valid_cells(H, A.g[g]);
            if (g + 1 < H.nmg) bytes += (2.0 * (nu1 + nu2) * (1.5 * sizeof(T) + 1.0) + 4.0 * sizeof(T)) * cells;
        }
    }
    A.M = H.coarse_inv;
    A.m = H.ncoarse;
    bytes += 8.0 * (double)A.m * A.m;
    // the largest cluster the device runs: 16 CTAs (non-portable) or 8
    static std::atomic<int> csize{0};
    auto fn = k_mg_bottom<T>;
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3(BX, 32);
    cfg.dynamicSmemBytes = sizeof(double) * (size_t)A.m;
    cfg.stream = H.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    if (csize.load() == 0) {
        int c = 8;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cfg.gridDim = dim3(16);
            at[0].val.clusterDim.x = 16;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) c = 16;
        }
        cudaGetLastError();
        csize.store(c);
    }
    int c = csize.load();
    cfg.gridDim = dim3((unsigned)c);
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    Launch Lc(H, K_MG_BOTTOM, bytes);
    cudaError_t e = cudaLaunchKernelEx(&cfg, fn, A);
    if (e != cudaSuccess) cuda_fail(e, "multigrid bottom launch");
}

template void launch_mg_bottom<double>(Hierarchy &, int, int, int);
template void launch_mg_bottom<float>(Hierarchy &, int, int, int);

// log2 of level l's cells per unit length (n0 2^l), or -1 unless n0 is a
// power of two (then the particle kernels take integer coordinates; a up to
// 30 keeps the node index in int range and every shift of cic_axis_fixed in
// range).
int pow2_log(const Hierarchy &H, int l)
{
    if (H.n0 <= 0 || (H.n0 & (H.n0 - 1))) return -1;
    int a = 0;
    while ((1 << a) < H.n0) ++a;
    a += l;
    return a <= 30 ? a : -1;
}

void launch_deposit(Hierarchy &H, const double *x, const double *y, const double *z, const double *q, int64_t n,
                    int level_only)
{
    if (n <= 0) return;
    DepositA A{};
    int l0 = level_only >= 0 ? level_only : 0, l1 = level_only >= 0 ? level_only + 1 : H.nlev;
    A.nlev = l1 - l0;
    for (int l = l0; l < l1; ++l) {
        A.g[l - l0] = H.L[l].g;
        A.ih[l - l0] = 1.0 / H.L[l].g.h;
        A.ih3[l - l0] = A.ih[l - l0] * A.ih[l - l0] * A.ih[l - l0];
        A.rho[l - l0] = H.L[l].rho;
        A.lg[l - l0] = pow2_log(H, l);
    }
    A.outside = (l0 == 0) ? H.outside : nullptr;
    A.inv_eps0 = 1.0 / H.eps0;
    A.x = x;
    A.y = y;
    A.z = z;
    A.q = q;
    A.n = n;
    double cells = 0.0;
    for (int l = l0; l < l1; ++l) cells += (double)H.L[l].nvalid;
    Launch Lc(H, K_DEPOSIT, 32.0 * (double)n + 8.0 * cells);
    issue<OP_DEPOSIT>(H, dim3((unsigned)((n + kDepositPer * NT - 1) / (kDepositPer * NT))), A, &OpArgs::dep);
}

void launch_gather(Hierarchy &H, const double *x, const double *y, const double *z, int64_t n, double *ex,
                   double *ey, double *ez, double *phi)
{
    if (n <= 0) return;
    GatherA A{};
    A.nlev = H.nlev;
    for (int l = 0; l < H.nlev; ++l) {
        A.g[l] = H.L[l].g;
        // gather buffer: a refined level is used only where its eroded
        // mask holds all 8 nodes
        if (l > 0 && H.gather_buffer > 0 && H.L[l].gmask) A.g[l].mask = H.L[l].gmask;
        A.ih[l] = 1.0 / H.L[l].g.h;
        A.lg[l] = pow2_log(H, l);
        for (int d = 0; d < 3; ++d) A.e[l][d] = H.L[l].ef[d];
        A.phi[l] = H.L[l].phi;
    }
    A.x = x;
    A.y = y;
    A.z = z;
    A.n = n;
    A.ex = ex;
    A.ey = ey;
    A.ez = ez;
    A.phio = phi;
    Launch Lc(H, K_GATHER, (phi ? 64.0 : 48.0) * (double)n);
    issue<OP_GATHER>(H, dim3((unsigned)((n + NT - 1) / NT)), A, &OpArgs::gat);
}

// ------------------------------------------------------- program launch

// Per-hierarchy recorded segments (init, body, tail) of a program.
struct ProgramRecorder {
    std::vector<std::vector<Phase>> seg[3];
};

ProgramRecorder *recorder_new(int nhier)
{
    ProgramRecorder *R = new ProgramRecorder();
    for (auto &s : R->seg) s.resize(nhier);
    return R;
}

void recorder_delete(ProgramRecorder *R) { delete R; }

void record_begin(Hierarchy &H, ProgramRecorder *R, int hier, int segment)
{
    H.rec = &R->seg[segment][hier];
    H.rec_hier = hier;
}

void record_end(Hierarchy &H)
{
    H.rec = nullptr;
    H.rec_hier = 0;
}

void program_free(Program &P)
{
    if (P.dev) cudaFree(P.dev);
    if (P.states) cudaFree(P.states);
    if (P.ctl) cudaFree(P.ctl);
    P = Program();
}

// Zip the hierarchies' segments into rounds (round r of a segment holds
// phase r of every hierarchy that has one), lay out the rounds with their
// virtual-block bases, and upload the program.
int program_compile(ProgramRecorder *R, SolveState *const *states_host, int nhier, cudaStream_t stream, Program &P)
{
    program_free(P);
    std::vector<Phase> flat;
    std::vector<int> ptr{0}, nvb;
    int rbeg[4] = {0, 0, 0, 0};
    size_t smem = 0;
    for (int sg = 0; sg < 3; ++sg) {
        size_t len = 0;
        for (auto &v : R->seg[sg]) len = std::max(len, v.size());
        rbeg[sg] = (int)nvb.size();
        for (size_t r = 0; r < len; ++r) {
            int base = 0;
            for (int h = 0; h < nhier; ++h) {
                const auto &v = R->seg[sg][h];
                if (r >= v.size()) continue;
                Phase p = v[r];
                p.vbase = base;
                base += p.gx * p.gy * p.gz;
                smem = std::max(smem, p.smem);
                flat.push_back(p);
            }
            ptr.push_back((int)flat.size());
            nvb.push_back(base);
        }
        P.n_phases[sg] = 0;
        for (auto &v : R->seg[sg]) P.n_phases[sg] += (int64_t)v.size();
    }
    rbeg[3] = (int)nvb.size();
    std::vector<int> phier(flat.size()), pnvb(flat.size());
    for (size_t q = 0; q < flat.size(); ++q) {
        phier[q] = flat[q].hier;
        pnvb[q] = flat[q].gx * flat[q].gy * flat[q].gz;
    }
    const size_t nf = std::max<size_t>(flat.size(), 1);
    size_t off_ptr = sizeof(Phase) * nf;
    size_t off_nvb = off_ptr + sizeof(int) * ptr.size();
    size_t off_ph = off_nvb + sizeof(int) * std::max<size_t>(nvb.size(), 1);
    size_t off_pn = off_ph + sizeof(int) * nf;
    size_t bytes = off_pn + sizeof(int) * nf;
    std::vector<char> img(bytes, 0);
    if (!flat.empty()) memcpy(img.data(), flat.data(), sizeof(Phase) * flat.size());
    memcpy(img.data() + off_ptr, ptr.data(), sizeof(int) * ptr.size());
    if (!nvb.empty()) memcpy(img.data() + off_nvb, nvb.data(), sizeof(int) * nvb.size());
    if (!flat.empty()) {
        memcpy(img.data() + off_ph, phier.data(), sizeof(int) * flat.size());
        memcpy(img.data() + off_pn, pnvb.data(), sizeof(int) * flat.size());
    }
    if (cudaMalloc(&P.dev, bytes) != cudaSuccess || cudaMalloc((void **)&P.states, sizeof(void *) * nhier) != cudaSuccess ||
        cudaMalloc((void **)&P.ctl, sizeof(ProgramCtl)) != cudaSuccess) {
        cudaGetLastError();
        program_free(P);
        set_error("out of memory (program)");
        return AMR_ENOMEM;
    }
    P.bytes = bytes;
    cudaError_t e = cudaMemcpyAsync(P.dev, img.data(), bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.states, states_host, sizeof(void *) * nhier, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        program_free(P);
        return cuda_fail(e, "program upload");
    }
    ProgramDesc &D = P.D;
    D.phases = P.dev;
    D.round_ptr = (const int *)((const char *)P.dev + off_ptr);
    D.round_nvb = (const int *)((const char *)P.dev + off_nvb);
    D.ph_hier = (const int *)((const char *)P.dev + off_ph);
    D.ph_nvb = (const int *)((const char *)P.dev + off_pn);
    D.init_r0 = rbeg[0];
    D.init_r1 = rbeg[1];
    D.body_r0 = rbeg[1];
    D.body_r1 = rbeg[2];
    D.tail_r0 = rbeg[2];
    D.tail_r1 = rbeg[3];
    D.nhier = nhier;
    D.max_loops = 1 << 20;
    D.states = P.states;
    D.ctl = P.ctl;
    D.limit_ns = 2000000000ull;
    P.smem = smem;
    return AMR_OK;
}

void cluster_free(ClusterProgram &P)
{
    if (P.dev) cudaFree(P.dev);
    if (P.states) cudaFree(P.states);
    if (P.queue) cudaFree(P.queue);
    P = ClusterProgram{};
}

int cluster_compile(ProgramRecorder *R, SolveState *const *states_host, const double *work, int nhier,
                    cudaStream_t stream, ClusterProgram &P)
{
    cluster_free(P);
    std::vector<Phase> flat;
    std::vector<int> hseg(6 * (size_t)nhier);
    size_t smem = 0;
    for (int h = 0; h < nhier; ++h)
        for (int sg = 0; sg < 3; ++sg) {
            hseg[6 * h + 2 * sg] = (int)flat.size();
            for (const Phase &p : R->seg[sg][h]) {
                flat.push_back(p);
                smem = std::max(smem, p.smem);
            }
            hseg[6 * h + 2 * sg + 1] = (int)flat.size();
        }
    std::vector<int> order(nhier);
    for (int h = 0; h < nhier; ++h) order[h] = h;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    // cluster size and co-resident clusters for this shared memory
    static int csize = 0;
    if (csize == 0) {
        cudaFuncSetAttribute(k_cluster_program, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
        csize = 8;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(BX, BY);
    cfg.gridDim = dim3((unsigned)csize);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_cluster_program, &cfg);
    if (e != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        set_error("no co-resident thread-block clusters for the batched program");
        return AMR_ECUDA;
    }
    const size_t nf = std::max<size_t>(flat.size(), 1);
    const size_t off_seg = sizeof(Phase) * nf;
    const size_t off_ord = off_seg + sizeof(int) * hseg.size();
    const size_t bytes = off_ord + sizeof(int) * order.size();
    std::vector<char> img(bytes, 0);
    if (!flat.empty()) memcpy(img.data(), flat.data(), sizeof(Phase) * flat.size());
    memcpy(img.data() + off_seg, hseg.data(), sizeof(int) * hseg.size());
    memcpy(img.data() + off_ord, order.data(), sizeof(int) * order.size());
    if (cudaMalloc(&P.dev, bytes) != cudaSuccess || cudaMalloc((void **)&P.states, sizeof(void *) * nhier) != cudaSuccess ||
        cudaMalloc((void **)&P.queue, sizeof(unsigned) * (1 + (size_t)nclusters)) != cudaSuccess) {
        cudaGetLastError();
        cluster_free(P);
        set_error("out of memory (batched program)");
        return AMR_ENOMEM;
    }
    P.bytes = bytes;
    e = cudaMemcpyAsync(P.dev, img.data(), bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.states, states_host, sizeof(void *) * nhier, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cluster_free(P);
        return cuda_fail(e, "batched program upload");
    }
    P.D.phases = P.dev;
    P.D.hseg = (const int *)((const char *)P.dev + off_seg);
    P.D.order = (const int *)((const char *)P.dev + off_ord);
    P.D.nhier = nhier;
    P.D.max_loops = 1 << 20;
    P.D.states = P.states;
    P.D.queue = P.queue;
    P.smem = smem;
    P.clusters = nclusters;
    P.csize = csize;
    P.n_phases = (int64_t)flat.size();
    return AMR_OK;
}

int cluster_run(ClusterProgram &P, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(P.queue, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return cuda_fail(e, "batched program reset");
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P.csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(BX, BY);
    cfg.gridDim = dim3((unsigned)(P.csize * P.clusters));
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_cluster_program, P.D);
    if (e != cudaSuccess) return cuda_fail(e, "batched program launch");
    return AMR_OK;
}

// Launch a compiled program as one cooperative kernel: a few blocks per SM,
// all co-resident.  expected_blocks > 0 overrides the barrier's block count
// (used only by the timeout self-test, where it makes every wait run out).
int program_run(Hierarchy &H, Program &P, cudaStream_t stream, unsigned long long limit_ns, int expected_blocks)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_program<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
        cudaFuncSetAttribute(k_program<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
    }
    const bool batch = P.D.nhier > 1;
    auto kern = batch ? k_program<8> : k_program<4>;
    // co-resident blocks per SM for this program's shared memory
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, P.smem);
    int want = batch ? 8 : 4;
    if (const char *s = getenv("AMR_PROGRAM_BLOCKS_PER_SM")) want = atoi(s);
    const int per_sm = std::max(1, std::min(nb, want));
    int blocks = per_sm * sms;
    ProgramDesc D = P.D;
    D.limit_ns = limit_ns;
    D.nblocks_expected = expected_blocks > 0 ? (unsigned)expected_blocks : (unsigned)blocks;
    cudaError_t e = cudaMemsetAsync(P.ctl, 0, sizeof(ProgramCtl), stream);
    if (e != cudaSuccess) return cuda_fail(e, "program reset");
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(BX, BY);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, D);
    if (e != cudaSuccess) return cuda_fail(e, "program launch");
    H.launches++;
    P.blocks = blocks;
    return AMR_OK;
}

#define AMR_INSTANTIATE(T)                                                                                  \
    template void launch_residual<T>(Hierarchy &, const Grid &, const T *, const T *, T *, int, int);       \
    template void launch_rbgs<T>(Hierarchy &, const Grid &, T *, const T *, int, int, int, T *, T *);       \
    template void launch_restrict_amr<T>(Hierarchy &, int);                                                 \
    template void launch_prolong_amr<T>(Hierarchy &, int);                                                  \
    template void launch_finish_amr<T>(Hierarchy &, int);                                                   \
    template void launch_cp<T>(Hierarchy &, int, const T *);                                                \
    template void launch_surface<T>(Hierarchy &, int, T *, int, const T *, T *);                            \
    template void launch_mg_restrict<T>(Hierarchy &, int, int);                                             \
    template void launch_mg_prolong<T>(Hierarchy &, int);                                                   \
    template void launch_mg_coarse_solve<T>(Hierarchy &);                                                   \
    template void launch_fill<T>(Hierarchy &, T *, T, int64_t);                                             \
    template void launch_axpy<T>(Hierarchy &, T *, const T *, T, int64_t);
AMR_INSTANTIATE(double)
AMR_INSTANTIATE(float)
#undef AMR_INSTANTIATE

} // namespace amr
