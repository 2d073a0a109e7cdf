// Device kernels of the AMR multigrid solve (sm_103a, FP64).
//
// Every stencil kernel works on the dense padded level boxes described in
// amr_internal.h, x fastest (coalesced rows per warp).  Operator
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
// surface kernels).  In composite mode a face towards a covered cell
// contributes nothing here: the surface kernel adds the fine-averaged flux
// of Eq. flux_differencing.
//
// FP64 on this part runs about two lanes per SM and is charged per warp
// instruction, so the kernels keep every lane of a warp on useful cells
// (one thread per cell of the colour being relaxed) and take a warp-uniform
// fast path (six plain neighbours: D = 6, 7 FP64 instructions per update);
// the general path reads D and 1/D from tables instead of converting and
// dividing.
#include <cuda_runtime.h>

#include "amr_internal.h"

namespace amr {

namespace {

constexpr int BX = 32, BY = 4;
constexpr double kThird = 1.0 / 3.0;
constexpr double kFifth = 0.2;

// Programmatic dependent launch: wait until the preceding kernel in the
// stream has completed and its memory is visible, then let the next kernel
// be launched while this one runs (hides the launch latency of the chain
// of small dependent kernels; a no-op when launched without the attribute).
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// D = k/3 and 1/D = 3/k for the face codes k = 0..36 of the split above.
#define AMR_K(k) ((double)(k) / 3.0)
#define AMR_IK(k) ((k) ? 3.0 / (double)(k) : 0.0)
#define AMR_ROW(M, b) M(b), M(b + 1), M(b + 2), M(b + 3), M(b + 4), M(b + 5)
__constant__ double c_D[37] = {AMR_ROW(AMR_K, 0), AMR_ROW(AMR_K, 6), AMR_ROW(AMR_K, 12), AMR_ROW(AMR_K, 18),
                               AMR_ROW(AMR_K, 24), AMR_ROW(AMR_K, 30), AMR_K(36)};
__constant__ double c_invD[37] = {AMR_ROW(AMR_IK, 0), AMR_ROW(AMR_IK, 6), AMR_ROW(AMR_IK, 12),
                                  AMR_ROW(AMR_IK, 18), AMR_ROW(AMR_IK, 24), AMR_ROW(AMR_IK, 30), AMR_IK(36)};
#define AMR_KF(k) ((float)(k) / 3.0f)
#define AMR_IKF(k) ((k) ? 3.0f / (float)(k) : 0.0f)
__constant__ float c_Df[37] = {AMR_ROW(AMR_KF, 0), AMR_ROW(AMR_KF, 6), AMR_ROW(AMR_KF, 12), AMR_ROW(AMR_KF, 18),
                               AMR_ROW(AMR_KF, 24), AMR_ROW(AMR_KF, 30), AMR_KF(36)};
__constant__ float c_invDf[37] = {AMR_ROW(AMR_IKF, 0), AMR_ROW(AMR_IKF, 6), AMR_ROW(AMR_IKF, 12),
                                  AMR_ROW(AMR_IKF, 18), AMR_ROW(AMR_IKF, 24), AMR_ROW(AMR_IKF, 30), AMR_IKF(36)};

template <typename T> __device__ __forceinline__ T tabD(int k);
template <> __device__ __forceinline__ double tabD<double>(int k) { return c_D[k]; }
template <> __device__ __forceinline__ float tabD<float>(int k) { return c_Df[k]; }
template <typename T> __device__ __forceinline__ T tabInvD(int k);
template <> __device__ __forceinline__ double tabInvD<double>(int k) { return c_invD[k]; }
template <> __device__ __forceinline__ float tabInvD<float>(int k) { return c_invDf[k]; }

__host__ __device__ inline int64_t pad_index(const Grid &g, int i, int j, int k)
{
    return (int64_t)(k - g.lo[2] + 1) * g.sz + (int64_t)(j - g.lo[1] + 1) * g.sy + (i - g.lo[0] + 1);
}

dim3 cell_grid(const Grid &g)
{
    return dim3((unsigned)((g.n[0] - 2 + BX - 1) / BX), (unsigned)((g.n[1] - 2 + BY - 1) / BY),
                (unsigned)(g.n[2] - 2));
}

// One thread per cell of one colour: half the row extent in x.
dim3 colour_grid(const Grid &g)
{
    int half = (g.n[0] - 2 + 1) / 2;
    return dim3((unsigned)((half + BX - 1) / BX), (unsigned)((g.n[1] - 2 + BY - 1) / BY), (unsigned)(g.n[2] - 2));
}

// S and the face code k of the split above, for an active cell p.  All 32
// lanes of the warp must call it (inactive lanes with act = false): the
// fast path is taken when every active lane has six plain neighbours.
template <bool COMP, typename T>
__device__ __forceinline__ void stencil_S(const Grid &g, const T *__restrict__ u, int64_t p, bool act, T &S, int &k)
{
    const int64_t off[6] = {-1, 1, -g.sy, g.sy, -g.sz, g.sz};
    uint8_t m[6] = {1, 1, 1, 1, 1, 1};
    bool fast = true;
    if (act) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            m[f] = g.mask[p + off[f]];
            fast &= COMP ? (m[f] == 1) : (m[f] != 0);
        }
    }
    if (__all_sync(0xffffffffu, fast)) {
        k = 18;
        S = act ? (((u[p - 1] + u[p + 1]) + (u[p - g.sy] + u[p + g.sy])) + (u[p - g.sz] + u[p + g.sz])) : T(0);
        return;
    }
    T s = T(0);
    int kk = 0;
    if (act) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            uint8_t mn = m[f];
            if (COMP ? (mn == 1) : (mn != 0)) {
                s += u[p + off[f]];
                kk += 3;
            } else if (mn == 0) {
                if (g.dirichlet) {
                    kk += 6;
                } else {
                    s -= T(kFifth) * u[p - off[f]];
                    kk += 1;
                }
            }
        }
    }
    S = s;
    k = kk;
}

// Face code from the masks alone (for the first sweep from a zero iterate).
__device__ __forceinline__ int face_code(const Grid &g, int64_t p)
{
    const int64_t off[6] = {-1, 1, -g.sy, g.sy, -g.sz, g.sz};
    int kk = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        uint8_t mn = g.mask[p + off[f]];
        kk += mn != 0 ? 3 : (g.dirichlet ? 6 : 1);
    }
    return kk;
}

// ---------------------------------------------------------------- kernels

template <typename T>
__global__ void k_residual(Grid g, const T *__restrict__ rho, const T *__restrict__ u, T *__restrict__ r, int comp,
                           int zero_covered)
{
    pdl_begin();
    int a = 1 + blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (b >= g.n[1] - 1) return; // uniform per warp
    bool in = a < g.n[0] - 1;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + (in ? a : 1);
    uint8_t m = in ? g.mask[p] : 0;
    if (comp && m == 2 && zero_covered) r[p] = T(0);
    bool act = m == 1 || (!comp && m == 2);
    T S;
    int k;
    if (comp)
        stencil_S<true>(g, u, p, act, S, k);
    else
        stencil_S<false>(g, u, p, act, S, k);
    if (act) r[p] = rho[p] + T(g.ih2) * (S - tabD<T>(k) * u[p]);
}

template <typename T>
__global__ void k_rbgs(Grid g, T *__restrict__ x, const T *__restrict__ rhs, int colour, int mode, T *__restrict__ e,
                       T *__restrict__ phi)
{
    pdl_begin();
    int tx = blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (b >= g.n[1] - 1) return; // uniform per warp
    int base = g.lo[0] + g.lo[1] + g.lo[2] + b + c - 3;
    int a = 1 + 2 * tx + ((colour + 1 + base) & 1);
    bool in = a < g.n[0] - 1;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + (in ? a : 1);
    bool act = in && g.mask[p] != 0;
    T S;
    int k;
    stencil_S<false>(g, x, p, act, S, k);
    if (act) {
        T v = (S + T(g.h2) * rhs[p]) * tabInvD<T>(k);
        x[p] = v;
        if (mode == 1) {
            e[p] += v;
            phi[p] += v;
        } else if (mode == 2) {
            phi[p] += v;
        }
    }
}

// Red pass from a zero iterate: red cells get h^2 b / D (their neighbours
// are black, i.e. zero), black cells are set to zero.  One thread per cell.
template <typename T>
__global__ void k_rbgs_first(Grid g, T *__restrict__ x, const T *__restrict__ rhs, int mode, T *__restrict__ e,
                             T *__restrict__ phi)
{
    pdl_begin();
    int a = 1 + blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (a >= g.n[0] - 1 || b >= g.n[1] - 1) return;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
    if (g.mask[p] == 0) return;
    if (((g.lo[0] + g.lo[1] + g.lo[2] + a + b + c - 3) & 1) != 0) {
        x[p] = T(0);
        return;
    }
    T v = T(g.h2) * rhs[p] * tabInvD<T>(face_code(g, p));
    x[p] = v;
    if (mode == 1) {
        e[p] += v;
        phi[p] += v;
    } else if (mode == 2) {
        phi[p] += v;
    }
}

// Alg. 3 after the pre-smooth, one thread per covered coarse cell P of
// level l-1: for the 8 children f, t_f = r_f - (A_nf e)_f (homogeneous
// coarse-fine ghosts, e^{l-1} = 0), stored back into r_f; phi_f += e_f;
// r^{l-1}_P = mean of t_f (the 8-cell average R).
template <typename T>
__global__ void k_restrict_amr(Grid gf, Grid gc, int clo0, int clo1, int clo2, int cn0, int cn1, int cn2,
                               T *__restrict__ rf, const T *__restrict__ ef, T *__restrict__ phif, T *__restrict__ rc)
{
    pdl_begin();
    int ci = clo0 + blockIdx.x * BX + threadIdx.x;
    int cj = clo1 + blockIdx.y * BY + threadIdx.y;
    int ck = clo2 + blockIdx.z;
    if (cj >= clo1 + cn1) return; // uniform per warp
    bool in = ci < clo0 + cn0;
    int64_t P = pad_index(gc, in ? ci : clo0, cj, ck);
    bool act = in && gc.mask[P] == 2;
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int64_t f = act ? pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2)) : 0;
        T S;
        int k;
        stencil_S<false>(gf, ef, f, act, S, k);
        if (act) {
            T ev = ef[f];
            T t = rf[f] + T(gf.ih2) * (S - tabD<T>(k) * ev);
            rf[f] = t;
            phif[f] += ev;
            acc += t;
        }
    }
    if (act) rc[P] = T(0.125) * acc;
}

// Alg. 3 prolongation and residual update, one thread per valid fine cell:
// v = I e^{l-1} (piecewise constant); e_f += v_f; phi_f += v_f (so that phi
// ends as phi_save + e without a saved copy); r_f -= (A_nf v)_f.
template <typename T>
__global__ void k_prolong_amr(Grid gf, Grid gc, T *__restrict__ ef, T *__restrict__ rf, T *__restrict__ phif,
                              const T *__restrict__ ec)
{
    pdl_begin();
    int a = 1 + blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (b >= gf.n[1] - 1) return;
    bool in = a < gf.n[0] - 1;
    int64_t p = (int64_t)c * gf.sz + (int64_t)b * gf.sy + (in ? a : 1);
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
        res = s - tabD<T>(kk) * vp;
    }
    if (act) {
        ef[p] += vp;
        phif[p] += vp;
        rf[p] += T(gf.ih2) * res;
    }
}

// e += de; phi += de (used only when there is no post-smoothing sweep).
template <typename T>
__global__ void k_finish(int64_t n, T *__restrict__ e, const T *__restrict__ de, T *__restrict__ phi)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        T v = de[t];
        e[t] += v;
        phi[t] += v;
    }
}

// Coarse part of every coarse-fine ghost of a level: cp = sum of the
// (8/15)-weighted step-1 stencil over uc, one thread per face, accumulated
// in FP64 whatever the field's precision.
template <typename T>
__global__ void k_cp(int nface, const int8_t *__restrict__ cnt, const int *__restrict__ cidx,
                     const double *__restrict__ cw, const T *__restrict__ uc, double *__restrict__ cp)
{
    pdl_begin();
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nface) return;
    int n = cnt[q];
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += cw[q * kMaxStencil + k] * (double)uc[cidx[q * kMaxStencil + k]];
    cp[q] = acc;
}

template <typename T>
struct SurfaceArgs {
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

// Interface corrections, accumulated in FP64 whatever the field precision.
template <typename T>
__global__ void k_surface(SurfaceArgs<T> A)
{
    pdl_begin();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < A.ncell) {
        double acc = 0.0;
        for (int q = A.cell_ptr[t]; q < A.cell_ptr[t + 1]; ++q) acc += A.cp_f[q];
        int f = A.cell_f[t];
        A.rf[f] = (T)((double)A.rf[f] + A.scale_f * acc);
        return;
    }
    t -= A.ncell;
    if (t < A.ncrse) {
        double acc = 0.0;
        for (int q = A.crse_ptr[t]; q < A.crse_ptr[t + 1]; ++q) {
            int face = A.crse_face[q];
            acc += (kThird * (double)A.uf[A.ff[face]] + kFifth * (double)A.uf[A.ff1[face]]) - A.cp_c[face];
        }
        int C = A.crse_c[t];
        A.rc[C] = (T)((double)A.rc[C] + A.scale_c * acc);
    }
}

// Mixed precision: the FP32 right-hand side of the correction equation is
// the FP64 composite residual; the FP32 correction starts at zero.
__global__ void k_to32(int64_t n, const double *__restrict__ r64, float *__restrict__ rho32, float *__restrict__ res32,
                       float *__restrict__ phi32)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float v = (float)r64[t];
        rho32[t] = v;
        res32[t] = v;
        phi32[t] = 0.0f;
    }
}

// phi (FP64) += the FP32 correction.
__global__ void k_add32(int64_t n, double *__restrict__ phi, const float *__restrict__ d32)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        phi[t] += (double)d32[t];
}

// E_d = -(u_{+d} - u_{-d}) / (2h) on valid cells; coarse-fine ghosts get
// their fine part here and their coarse part from k_cf_grad.
__global__ void k_grad(Grid g, const double *__restrict__ u, double *__restrict__ e0, double *__restrict__ e1,
                       double *__restrict__ e2)
{
    pdl_begin();
    int a = 1 + blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (a >= g.n[0] - 1 || b >= g.n[1] - 1) return;
    int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
    if (g.mask[p] == 0) return;
    const int64_t st[3] = {1, g.sy, g.sz};
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
            else if (g.dirichlet)
                side[s] = -up;
            else
                side[s] = (2.0 * kThird) * up - kFifth * u[p - o];
        }
        out[d] = -(side[1] - side[0]) * (0.5 / g.h);
    }
    e0[p] = out[0];
    e1[p] = out[1];
    e2[p] = out[2];
}

__global__ void k_cf_grad(int ncell, const int *__restrict__ cell_f, const int *__restrict__ cell_ptr,
                          const int8_t *__restrict__ dir, const double *__restrict__ cp, double *__restrict__ e0,
                          double *__restrict__ e1, double *__restrict__ e2, double inv2h)
{
    pdl_begin();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = cell_ptr[i]; q < cell_ptr[i + 1]; ++q) {
        int d = dir[q] >> 1;
        double s = (dir[q] & 1) ? 1.0 : -1.0;
        acc[d] -= s * cp[q] * inv2h;
    }
    int f = cell_f[i];
    e0[f] += acc[0];
    e1[f] += acc[1];
    e2[f] += acc[2];
}

// Average down: covered coarse cells <- mean of their 8 children.
__global__ void k_avgdown(Grid gf, Grid gc, int clo0, int clo1, int clo2, int cn0, int cn1, int cn2,
                          const double *__restrict__ uf, double *__restrict__ uc)
{
    pdl_begin();
    int ci = clo0 + blockIdx.x * BX + threadIdx.x;
    int cj = clo1 + blockIdx.y * BY + threadIdx.y;
    int ck = clo2 + blockIdx.z;
    if (ci >= clo0 + cn0 || cj >= clo1 + cn1 || ck >= clo2 + cn2) return;
    int64_t P = pad_index(gc, ci, cj, ck);
    if (gc.mask[P] != 2) return;
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) acc += uf[pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2))];
    uc[P] = 0.125 * acc;
}

struct NormArgs {
    int nslots;
    int64_t n[2 * kMaxLevels];
    const uint8_t *mask[2 * kMaxLevels];
    const double *v[2 * kMaxLevels];
    int covered_too[2 * kMaxLevels];
};

// Per-block partials of sum v^2, sum |v| and max |v| over the cells with
// mask == 1 (or >= 1 when covered_too), one slot per blockIdx.y: fixed
// thread-to-cell assignment and a fixed shuffle tree, so the result is
// bitwise reproducible.
__global__ void k_norms(NormArgs A, double *__restrict__ part)
{
    pdl_begin();
    int slot = blockIdx.y;
    const uint8_t *mask = A.mask[slot];
    const double *v = A.v[slot];
    int64_t n = A.n[slot];
    int cov = A.covered_too[slot];
    double s2 = 0.0, s1 = 0.0, mx = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = mask[t];
        if (m == 1 || (cov && m == 2)) {
            double x = v[t];
            s2 += x * x;
            s1 += fabs(x);
            mx = fmax(mx, fabs(x));
        }
    }
    __shared__ double sh[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][w] = s2;
        sh[1][w] = s1;
        sh[2][w] = mx;
    }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        s2 = lane < nw ? sh[0][lane] : 0.0;
        s1 = lane < nw ? sh[1][lane] : 0.0;
        mx = lane < nw ? sh[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            double *p = part + (int64_t)slot * 3 * kPartialBlocks;
            p[blockIdx.x] = s2;
            p[kPartialBlocks + blockIdx.x] = s1;
            p[2 * kPartialBlocks + blockIdx.x] = mx;
        }
    }
}

// Convergence test of Alg. 2 on the device: fixed-order sums of the
// partials, rel^l = ||r^l||_p / ||rho^l||_p (a zero ||rho^l|| uses the
// largest one), iteration count, and the graph condition "another V-cycle".
__global__ void k_check(const double *__restrict__ part, int nlev, int with_rho, int is_body,
                        const SolveParams *__restrict__ prm, SolveState *__restrict__ st,
                        cudaGraphConditionalHandle cond, int use_cond)
{
    pdl_begin();
    __shared__ double tot[2 * kMaxLevels][3];
    __shared__ double sh[3][32];
    int nslots = with_rho ? 2 * nlev : nlev;
    for (int slot = 0; slot < nslots; ++slot) {
        const double *p = part + (int64_t)slot * 3 * kPartialBlocks;
        double s2 = 0.0, s1 = 0.0, mx = 0.0;
        for (int t = threadIdx.x; t < kPartialBlocks; t += blockDim.x) {
            s2 += p[t];
            s1 += p[kPartialBlocks + t];
            mx = fmax(mx, p[2 * kPartialBlocks + t]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            sh[0][w] = s2;
            sh[1][w] = s1;
            sh[2][w] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int nw = blockDim.x >> 5;
            double a = 0.0, b = 0.0, c = 0.0;
            for (int q = 0; q < nw; ++q) {
                a += sh[0][q];
                b += sh[1][q];
                c = fmax(c, sh[2][q]);
            }
            tot[slot][0] = a;
            tot[slot][1] = b;
            tot[slot][2] = c;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    int pn = prm->norm;
    auto pick = [pn](const double *v) { return pn == AMR_NORM_2 ? sqrt(v[0]) : (pn == AMR_NORM_1 ? v[1] : v[2]); };
    if (with_rho)
        for (int l = 0; l < nlev; ++l) st->rhon[l] = pick(tot[nlev + l]);
    double bmax = 0.0;
    for (int l = 0; l < nlev; ++l) bmax = fmax(bmax, st->rhon[l]);
    double worst = 0.0;
    for (int l = 0; l < nlev; ++l) {
        double b = st->rhon[l] > 0.0 ? st->rhon[l] : bmax;
        double r = pick(tot[l]);
        double rel = b > 0.0 ? r / b : r;
        st->rel[l] = rel;
        worst = fmax(worst, rel);
    }
    st->worst = worst;
    int it = is_body ? st->iters + 1 : 0;
    st->iters = it;
    int go = (worst > prm->eps) && (it < prm->max_iter);
    st->go = go;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// Level-0 multigrid restriction, one thread per coarse cell:
// r_c = mean over the children of (r_f - A e_f); e_c = 0.
template <typename T>
__global__ void k_mg_restrict(Grid gf, Grid gc, const T *__restrict__ ef, const T *__restrict__ rf, T *__restrict__ rc,
                              T *__restrict__ ec)
{
    pdl_begin();
    int a = 1 + blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (b >= gc.n[1] - 1) return;
    bool act = a < gc.n[0] - 1;
    int ci = gc.lo[0] + a - 1, cj = gc.lo[1] + b - 1, ck = gc.lo[2] + c - 1;
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int64_t f = act ? pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2)) : 0;
        T S;
        int k;
        stencil_S<false>(gf, ef, f, act, S, k);
        if (act) acc += rf[f] + T(gf.ih2) * (S - tabD<T>(k) * ef[f]);
    }
    if (act) {
        int64_t P = (int64_t)c * gc.sz + (int64_t)b * gc.sy + a;
        rc[P] = T(0.125) * acc;
        ec[P] = T(0);
    }
}

// Level-0 multigrid trilinear prolongation of the correction, one thread
// per fine cell: weights 3/4 and 1/4 per axis on the two nearest coarse
// centres; outside the domain the coarse ghost is the Dirichlet mirror.
template <typename T>
__global__ void k_mg_prolong(Grid gf, Grid gc, T *__restrict__ ef, const T *__restrict__ ec)
{
    pdl_begin();
    int a = 1 + blockIdx.x * BX + threadIdx.x;
    int b = 1 + blockIdx.y * BY + threadIdx.y;
    int c = 1 + blockIdx.z;
    if (a >= gf.n[0] - 1 || b >= gf.n[1] - 1) return;
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
        bool neg = false;
        int Q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            w *= sel[d] ? T(0.25) : T(0.75);
            int q = I[d] + (sel[d] ? O[d] : 0);
            if (q < 0 || q >= nc[d]) {
                neg = !neg;
                q = I[d];
            }
            Q[d] = q;
        }
        T v = ec[pad_index(gc, Q[0], Q[1], Q[2])];
        acc += w * (neg ? -v : v);
    }
    ef[p] += acc;
}

// Coarsest grid of the level-0 multigrid: e = M r with the dense FP64
// inverse M (order m), accumulated in FP64; one warp per row, r staged in
// shared memory.
template <typename T>
__global__ void k_coarse_solve(Grid g, int m, const double *__restrict__ M, const T *__restrict__ r, T *__restrict__ e)
{
    pdl_begin();
    extern __shared__ double rs[];
    int nx = g.n[0] - 2, ny = g.n[1] - 2;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        int i = t % nx, j = (t / nx) % ny, k = t / (nx * ny);
        rs[t] = (double)r[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)];
    }
    __syncthreads();
    int warps = blockDim.x >> 5;
    int row = blockIdx.x * warps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= m) return;
    double acc = 0.0;
    for (int c = lane; c < m; c += 32) acc += M[(int64_t)row * m + c] * rs[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        int i = row % nx, j = (row / nx) % ny, k = row / (nx * ny);
        e[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)] = (T)acc;
    }
}

struct DepositArgs {
    int nlev;
    Grid g[kMaxLevels];
    double *rho[kMaxLevels];
    int *outside;
    double inv_eps0;
};

// Cloud-in-cell deposit, one thread per particle, every level: node (cell
// centre) i at (i + 1/2) h, linear weights per axis, density q w / h^3.
__global__ void k_deposit(DepositArgs A, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const double *__restrict__ q, int64_t n)
{
    pdl_begin();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double px = x[t], py = y[t], pz = z[t], pq = q[t] * A.inv_eps0;
    for (int l = 0; l < A.nlev; ++l) {
        const Grid &g = A.g[l];
        double s[3] = {px / g.h - 0.5, py / g.h - 0.5, pz / g.h - 0.5};
        // keep far-away or non-finite positions in int range (they deposit nothing)
#pragma unroll
        for (int d = 0; d < 3; ++d) s[d] = fmin(fmax(s[d], -4.0), 1.0 / g.h + 4.0);
        int loc[3];
        double w1[3];
        bool inside = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double f = floor(s[d]);
            w1[d] = s[d] - f;
            loc[d] = (int)f - g.lo[d] + 1; // padded local index of the lower node
            inside &= (loc[d] >= 0 && loc[d] + 1 < g.n[d]);
        }
        if (l == 0 && A.outside) {
            // all nodes must be valid cells of level 0 (not the ring)
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) ok &= (loc[d] >= 1 && loc[d] + 1 <= g.n[d] - 2);
            if (!ok) atomicAdd(A.outside, 1);
        }
        double wq = pq / (g.h * g.h * g.h);
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            int da = o & 1, db = (o >> 1) & 1, dc = o >> 2;
            int a = loc[0] + da, b = loc[1] + db, c = loc[2] + dc;
            if (!inside && (a < 0 || b < 0 || c < 0 || a >= g.n[0] || b >= g.n[1] || c >= g.n[2])) continue;
            double w = (da ? w1[0] : 1.0 - w1[0]) * (db ? w1[1] : 1.0 - w1[1]) * (dc ? w1[2] : 1.0 - w1[2]);
            atomicAdd(A.rho[l] + (int64_t)c * g.sz + (int64_t)b * g.sy + a, wq * w);
        }
    }
}

struct GatherArgs {
    int nlev;
    Grid g[kMaxLevels];
    const double *e[kMaxLevels][3];
    const double *phi[kMaxLevels];
};

__global__ void k_gather(GatherArgs A, const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, int64_t n, double *__restrict__ ex, double *__restrict__ ey,
                         double *__restrict__ ez, double *__restrict__ phio)
{
    pdl_begin();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double px = x[t], py = y[t], pz = z[t];
    double E[3] = {0.0, 0.0, 0.0}, ph = 0.0;
    for (int l = A.nlev - 1; l >= 0; --l) {
        const Grid &g = A.g[l];
        double s[3] = {px / g.h - 0.5, py / g.h - 0.5, pz / g.h - 0.5};
#pragma unroll
        for (int d = 0; d < 3; ++d) s[d] = fmin(fmax(s[d], -4.0), 1.0 / g.h + 4.0);
        int loc[3];
        double w1[3];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double f = floor(s[d]);
            w1[d] = s[d] - f;
            loc[d] = (int)f - g.lo[d] + 1;
            ok &= (loc[d] >= 0 && loc[d] + 1 < g.n[d]);
        }
        if (!ok) continue;
        int64_t base = (int64_t)loc[2] * g.sz + (int64_t)loc[1] * g.sy + loc[0];
        const int64_t co[8] = {0, 1, g.sy, g.sy + 1, g.sz, g.sz + 1, g.sz + g.sy, g.sz + g.sy + 1};
#pragma unroll
        for (int o = 0; o < 8; ++o) ok &= (g.mask[base + co[o]] != 0);
        if (!ok) continue;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            int da = o & 1, db = (o >> 1) & 1, dc = o >> 2;
            double w = (da ? w1[0] : 1.0 - w1[0]) * (db ? w1[1] : 1.0 - w1[1]) * (dc ? w1[2] : 1.0 - w1[2]);
            int64_t p = base + co[o];
            E[0] += w * A.e[l][0][p];
            E[1] += w * A.e[l][1][p];
            E[2] += w * A.e[l][2][p];
            if (phio) ph += w * A.phi[l][p];
        }
        break;
    }
    ex[t] = E[0];
    ey[t] = E[1];
    ez[t] = E[2];
    if (phio) phio[t] = ph;
}

template <typename T>
__global__ void k_fill(T *p, T v, int64_t n)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        p[t] = v;
}

template <typename T>
__global__ void k_axpy(T *__restrict__ y, const T *__restrict__ x, T a, int64_t n)
{
    pdl_begin();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] += a * x[t];
}

unsigned elem_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Coarse footprint box of fine level l in level l-1 index space.
void footprint(const Hierarchy &H, int l, int lo[3], int n[3])
{
    for (int d = 0; d < 3; ++d) {
        lo[d] = H.L[l].vlo[d] >> 1;
        n[d] = (H.L[l].vhi[d] >> 1) - lo[d] + 1;
    }
}

// Counts the launch and, when the timers are on (and no graph is being
// captured), brackets it with a pair of events on the hierarchy's stream.
struct Launch {
    Hierarchy &H;
    int kind;
    double bytes;
    int ev = -1;
    Launch(Hierarchy &h, int k, double b) : H(h), kind(k), bytes(b)
    {
        if (!H.prof || H.capturing) return;
        if (H.evnext + 2 > (int)H.evpool.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                H.evpool.push_back(e);
            }
        }
        ev = H.evnext;
        H.evnext += 2;
        cudaEventRecord(H.evpool[ev], H.stream);
    }
    ~Launch()
    {
        H.launches++;
        if (ev < 0) return;
        cudaEventRecord(H.evpool[ev + 1], H.stream);
        H.pending.push_back({kind, ev, bytes});
    }
};

double valid_cells(const Hierarchy &H, const Grid &g)
{
    for (int l = 0; l < H.nlev; ++l)
        if (H.L[l].g.mask == g.mask) return (double)H.L[l].nvalid;
    return (double)(g.n[0] - 2) * (g.n[1] - 2) * (g.n[2] - 2);
}

} // namespace

int prof_resolve(Hierarchy &H)
{
    if (H.pending.empty()) return AMR_OK;
    cudaError_t e = cudaStreamSynchronize(H.stream);
    if (e != cudaSuccess) return cuda_fail(e, "profile");
    for (const ProfRecord &r : H.pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, H.evpool[r.ev], H.evpool[r.ev + 1]);
        H.kind_ms[r.kind] += ms;
        H.kind_bytes[r.kind] += r.bytes;
        H.kind_launches[r.kind]++;
    }
    H.pending.clear();
    H.evnext = 0;
    return AMR_OK;
}

const char *kind_name(int kind)
{
    static const char *names[K_NUM] = {"deposit",   "gather",     "residual",    "rbgs",       "restrict",
                                       "prolong",   "finish",     "cf_correct",  "flux",       "grad",
                                       "average_down", "norms",   "mg_restrict", "mg_prolong", "coarse_solve",
                                       "elementwise", "coarse_part", "check"};
    return (kind >= 0 && kind < K_NUM) ? names[kind] : "";
}

// ------------------------------------------------------------- launchers

template <typename... KArgs, typename... Args>
void launch(Hierarchy &H, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = H.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = H.pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename T>
void launch_residual(Hierarchy &H, const Grid &g, const T *rho, const T *phi, T *res, int comp, int zero_covered)
{
    Launch L(H, K_RESIDUAL, 3.0 * sizeof(T) * valid_cells(H, g));
    launch(H, k_residual<T>, cell_grid(g), dim3(BX, BY), 0, g, rho, phi, res, comp, zero_covered);
}

template <typename T>
void launch_rbgs(Hierarchy &H, const Grid &g, T *x, const T *b, int colour, int first, int mode, T *e, T *phi)
{
    double cells = valid_cells(H, g);
    double bytes = (first ? 1.5 : 2.0) * sizeof(T) * cells;
    if (mode == 1) bytes += 2.0 * sizeof(T) * cells;
    if (mode == 2) bytes += 1.0 * sizeof(T) * cells;
    Launch L(H, K_RBGS, bytes);
    if (first)
        launch(H, k_rbgs_first<T>, cell_grid(g), dim3(BX, BY), 0, g, x, b, mode, e, phi);
    else
        launch(H, k_rbgs<T>, colour_grid(g), dim3(BX, BY), 0, g, x, b, colour, mode, e, phi);
}

template <typename T>
void launch_restrict_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l], &C = H.L[l - 1];
    Fields<T> ff = fields<T>(F), fc = fields<T>(C);
    int lo[3], n[3];
    footprint(H, l, lo, n);
    dim3 grid((unsigned)((n[0] + BX - 1) / BX), (unsigned)((n[1] + BY - 1) / BY), (unsigned)n[2]);
    Launch L(H, K_RESTRICT, (5.0 + 1.0 / 8) * sizeof(T) * (double)F.nvalid);
    launch(H, k_restrict_amr<T>, grid, dim3(BX, BY), 0, F.g, C.g, lo[0], lo[1], lo[2], n[0], n[1], n[2], ff.res,
           (const T *)ff.err, ff.phi, fc.res);
}

template <typename T>
void launch_prolong_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l], &C = H.L[l - 1];
    Fields<T> ff = fields<T>(F), fc = fields<T>(C);
    Launch L(H, K_PROLONG, (6.0 + 1.0 / 8) * sizeof(T) * (double)F.nvalid);
    launch(H, k_prolong_amr<T>, cell_grid(F.g), dim3(BX, BY), 0, F.g, C.g, ff.err, ff.res, ff.phi,
           (const T *)fc.err);
}

template <typename T>
void launch_finish_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l];
    Fields<T> ff = fields<T>(F);
    Launch L(H, K_FINISH, 5.0 * sizeof(T) * (double)F.nvalid);
    launch(H, k_finish<T>, elem_blocks(F.g.ncell), 256, 0, F.g.ncell, ff.err, (const T *)ff.de, ff.phi);
}

template <typename T>
void launch_cp(Hierarchy &H, int l, const T *uc)
{
    CfTable &T_ = H.L[l].cf;
    if (T_.nface == 0) return;
    Launch L(H, K_CP, T_.nface * (8.0 + 9 * (12.0 + sizeof(T))));
    launch(H, k_cp<T>, (T_.nface + 127) / 128, 128, 0, T_.nface, (const int8_t *)T_.cnt, (const int *)T_.cidx,
           (const double *)T_.cw, uc, T_.cp);
}

template <typename T>
void launch_surface(Hierarchy &H, int lf, T *rf, int lc, const T *uf, T *rc)
{
    SurfaceArgs<T> A{};
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
    launch(H, k_surface<T>, (n + 127) / 128, 128, 0, A);
}

void launch_to32(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    Launch Lc(H, K_ELEMENTWISE, 20.0 * (double)L.g.ncell);
    launch(H, k_to32, elem_blocks(L.g.ncell), 256, 0, L.g.ncell, (const double *)L.res, L.rho32, L.res32, L.phi32);
}

void launch_add32(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    Launch Lc(H, K_ELEMENTWISE, 20.0 * (double)L.g.ncell);
    launch(H, k_add32, elem_blocks(L.g.ncell), 256, 0, L.g.ncell, L.phi, (const float *)L.phi32);
}

void launch_grad(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    Launch Lc(H, K_GRAD, 32.0 * (double)L.nvalid);
    launch(H, k_grad, cell_grid(L.g), dim3(BX, BY), 0, L.g, L.phi, L.ef[0], L.ef[1], L.ef[2]);
}

void launch_cf_grad(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    CfTable &T = L.cf;
    if (T.ncell == 0) return;
    Launch Lc(H, K_CF, 48.0 * T.ncell + 8.0 * T.nface);
    launch(H, k_cf_grad, (T.ncell + 127) / 128, 128, 0, T.ncell, T.cell_f, T.cell_ptr, T.dir, T.cp, L.ef[0],
                                                           L.ef[1], L.ef[2], 0.5 / L.g.h);
}

void launch_average_down(Hierarchy &H, int l)
{
    Level &F = H.L[l + 1], &C = H.L[l];
    int lo[3], n[3];
    footprint(H, l + 1, lo, n);
    dim3 grid((unsigned)((n[0] + BX - 1) / BX), (unsigned)((n[1] + BY - 1) / BY), (unsigned)n[2]);
    Launch Lc(H, K_AVGDOWN, 9.0 * (double)F.nvalid);
    launch(H, k_avgdown, grid, dim3(BX, BY), 0, F.g, C.g, lo[0], lo[1], lo[2], n[0], n[1], n[2], F.phi, C.phi);
}

void launch_norms_check(Hierarchy &H, int with_rho, int is_body, unsigned long long cond, int use_cond)
{
    NormArgs A{};
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
    {
        Launch Lc(H, K_NORMS, bytes);
        launch(H, k_norms, dim3(kPartialBlocks, ns), 256, 0, A, H.partials);
    }
    Launch Lc(H, K_CHECK, 24.0 * kPartialBlocks * ns);
    launch(H, k_check, 1, 256, 0, H.partials, H.nlev, with_rho, is_body, H.params, H.state,
                                     (cudaGraphConditionalHandle)cond, use_cond);
}

template <typename T>
void launch_mg_restrict(Hierarchy &H, int g)
{
    MgGrid &F = H.mg[g], &C = H.mg[g + 1];
    Launch Lc(H, K_MG_RESTRICT, 2.0 * sizeof(T) * (valid_cells(H, F.g) + valid_cells(H, C.g)));
    launch(H, k_mg_restrict<T>, cell_grid(C.g), dim3(BX, BY), 0, F.g, C.g, (const T *)mg_e<T>(F),
           (const T *)mg_r<T>(F), mg_r<T>(C), mg_e<T>(C));
}

template <typename T>
void launch_mg_prolong(Hierarchy &H, int g)
{
    MgGrid &F = H.mg[g], &C = H.mg[g + 1];
    Launch Lc(H, K_MG_PROLONG, 2.0 * sizeof(T) * valid_cells(H, F.g) + sizeof(T) * valid_cells(H, C.g));
    launch(H, k_mg_prolong<T>, cell_grid(F.g), dim3(BX, BY), 0, F.g, C.g, mg_e<T>(F), (const T *)mg_e<T>(C));
}

template <typename T>
void launch_mg_coarse_solve(Hierarchy &H)
{
    MgGrid &G = H.mg[H.nmg - 1];
    int m = H.ncoarse;
    int threads = 256, warps = threads / 32;
    unsigned blocks = (unsigned)((m + warps - 1) / warps);
    Launch Lc(H, K_COARSE, 8.0 * (double)m * m + 2.0 * sizeof(T) * m);
    launch(H, k_coarse_solve<T>, blocks, threads, sizeof(double) * (size_t)m, G.g, m, (const double *)H.coarse_inv,
           (const T *)mg_r<T>(G), mg_e<T>(G));
}

void launch_deposit(Hierarchy &H, const double *x, const double *y, const double *z, const double *q, int64_t n,
                    int level_only)
{
    if (n <= 0) return;
    DepositArgs A{};
    int l0 = level_only >= 0 ? level_only : 0, l1 = level_only >= 0 ? level_only + 1 : H.nlev;
    A.nlev = l1 - l0;
    for (int l = l0; l < l1; ++l) {
        A.g[l - l0] = H.L[l].g;
        A.rho[l - l0] = H.L[l].rho;
    }
    A.outside = (l0 == 0) ? H.outside : nullptr;
    A.inv_eps0 = 1.0 / H.eps0;
    double cells = 0.0;
    for (int l = l0; l < l1; ++l) cells += (double)H.L[l].nvalid;
    Launch Lc(H, K_DEPOSIT, 32.0 * (double)n + 8.0 * cells);
    launch(H, k_deposit, (unsigned)((n + 255) / 256), 256, 0, A, x, y, z, q, n);
}

void launch_gather(Hierarchy &H, const double *x, const double *y, const double *z, int64_t n, double *ex,
                   double *ey, double *ez, double *phi)
{
    if (n <= 0) return;
    GatherArgs A{};
    A.nlev = H.nlev;
    for (int l = 0; l < H.nlev; ++l) {
        A.g[l] = H.L[l].g;
        for (int d = 0; d < 3; ++d) A.e[l][d] = H.L[l].ef[d];
        A.phi[l] = H.L[l].phi;
    }
    Launch Lc(H, K_GATHER, (phi ? 64.0 : 48.0) * (double)n);
    launch(H, k_gather, (unsigned)((n + 255) / 256), 256, 0, A, x, y, z, n, ex, ey, ez, phi);
}

template <typename T>
void launch_fill(Hierarchy &H, T *p, T v, int64_t n)
{
    Launch Lc(H, K_ELEMENTWISE, sizeof(T) * (double)n);
    launch(H, k_fill<T>, elem_blocks(n), 256, 0, p, v, n);
}

template <typename T>
void launch_axpy(Hierarchy &H, T *y, const T *x, T a, int64_t n)
{
    Launch Lc(H, K_ELEMENTWISE, 3.0 * sizeof(T) * (double)n);
    launch(H, k_axpy<T>, elem_blocks(n), 256, 0, y, x, a, n);
}

#define AMR_INSTANTIATE(T)                                                                                  \
    template void launch_residual<T>(Hierarchy &, const Grid &, const T *, const T *, T *, int, int);                \
    template void launch_rbgs<T>(Hierarchy &, const Grid &, T *, const T *, int, int, int, T *, T *);                \
    template void launch_restrict_amr<T>(Hierarchy &, int);                                                          \
    template void launch_prolong_amr<T>(Hierarchy &, int);                                                           \
    template void launch_finish_amr<T>(Hierarchy &, int);                                                            \
    template void launch_cp<T>(Hierarchy &, int, const T *);                                                         \
    template void launch_surface<T>(Hierarchy &, int, T *, int, const T *, T *);                                     \
    template void launch_mg_restrict<T>(Hierarchy &, int);                                                           \
    template void launch_mg_prolong<T>(Hierarchy &, int);                                                            \
    template void launch_mg_coarse_solve<T>(Hierarchy &);                                                            \
    template void launch_fill<T>(Hierarchy &, T *, T, int64_t);                                                      \
    template void launch_axpy<T>(Hierarchy &, T *, const T *, T, int64_t);
AMR_INSTANTIATE(double)
AMR_INSTANTIATE(float)
#undef AMR_INSTANTIATE

} // namespace amr
