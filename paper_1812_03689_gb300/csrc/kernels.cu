// Device kernels of the AMR multigrid solve (sm_103a, FP64).
//
// Every stencil kernel works on the dense padded level boxes described in
// amr_internal.h, one thread per cell, x fastest (coalesced rows of 32
// cells per warp).  Operator conventions: A = -L, residual r = b - A u, and
// for a cell p the 7-point flux-differenced stencil (Eq. lap_flux_differencing
// with the coarse fluxes of Eq. coarse_fluxes) is split as
//     (L u)_p = (S - D u_p) / h^2,
// where each face contributes
//     neighbour valid on the level          S += u_n,            D += 1
//     physical boundary (Dirichlet 0)       ghost -u_p:           D += 2
//     coarse-fine face (level l >= 1)       ghost (2/3) u_p - (1/5) u_o + C:
//                                           S -= u_o / 5,        D += 1/3
// (u_o the inward neighbour opposite the face; C the coarse part, the
// (8/15)-weighted step-1 interpolation of Eq. 2d_lagrange, added by the
// coarse-fine kernels).  In composite mode a face towards a covered cell
// contributes nothing here: the flux-matching kernel adds the fine-averaged
// flux of Eq. flux_differencing.
#include <cuda_runtime.h>

#include "amr_internal.h"

namespace amr {

namespace {

constexpr int BX = 32, BY = 4;
constexpr double kThird = 1.0 / 3.0;
constexpr double kFifth = 0.2;

__host__ __device__ inline int64_t pad_index(const Grid &g, int i, int j, int k)
{
    return (int64_t)(k - g.lo[2] + 1) * g.sz + (int64_t)(j - g.lo[1] + 1) * g.sy + (i - g.lo[0] + 1);
}

dim3 cell_grid(const Grid &g)
{
    return dim3((unsigned)((g.n[0] - 2 + BX - 1) / BX), (unsigned)((g.n[1] - 2 + BY - 1) / BY),
                (unsigned)(g.n[2] - 2));
}

// Local padded coordinates of this thread's cell; false if outside the box.
__device__ inline bool cell_coords(const Grid &g, int &a, int &b, int &c, int64_t &p)
{
    a = 1 + blockIdx.x * BX + threadIdx.x;
    b = 1 + blockIdx.y * BY + threadIdx.y;
    c = 1 + blockIdx.z;
    if (a >= g.n[0] - 1 || b >= g.n[1] - 1) return false;
    p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
    return true;
}

__device__ inline int parity(const Grid &g, int a, int b, int c)
{
    return (g.lo[0] + g.lo[1] + g.lo[2] + a + b + c - 3) & 1;
}

// S and D of the stencil split above.  Returns true on the fast path (all
// six neighbours are plain valid cells: D = 6).
template <bool COMP>
__device__ inline bool stencil(const Grid &g, const double *__restrict__ u, int64_t p, double &S, double &D)
{
    const int64_t off[6] = {-1, 1, -g.sy, g.sy, -g.sz, g.sz};
    uint8_t m[6];
    bool fast = true;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        m[f] = g.mask[p + off[f]];
        fast &= COMP ? (m[f] == 1) : (m[f] != 0);
    }
    if (fast) {
        S = ((u[p - 1] + u[p + 1]) + (u[p - g.sy] + u[p + g.sy])) + (u[p - g.sz] + u[p + g.sz]);
        D = 6.0;
        return true;
    }
    double s = 0.0;
    int nv = 0, nd = 0, nc = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        uint8_t mn = m[f];
        if (mn == 1 || (!COMP && mn == 2)) {
            s += u[p + off[f]];
            ++nv;
        } else if (mn == 0) {
            if (g.dirichlet) {
                ++nd;
            } else {
                s -= kFifth * u[p - off[f]];
                ++nc;
            }
        }
    }
    S = s;
    D = (double)(3 * nv + 6 * nd + nc) * kThird;
    return false;
}

// ---------------------------------------------------------------- kernels

__global__ void k_residual(Grid g, const double *__restrict__ rho, const double *__restrict__ u,
                           double *__restrict__ r, int comp, int zero_covered)
{
    int a, b, c;
    int64_t p;
    if (!cell_coords(g, a, b, c, p)) return;
    uint8_t m = g.mask[p];
    if (m == 0) return;
    if (comp && m == 2) {
        if (zero_covered) r[p] = 0.0;
        return;
    }
    double S, D;
    if (comp)
        stencil<true>(g, u, p, S, D);
    else
        stencil<false>(g, u, p, S, D);
    r[p] = rho[p] + g.ih2 * (S - D * u[p]);
}

__global__ void k_rbgs(Grid g, double *__restrict__ x, const double *__restrict__ rhs, int colour)
{
    int a, b, c;
    int64_t p;
    if (!cell_coords(g, a, b, c, p)) return;
    if (parity(g, a, b, c) != colour || g.mask[p] == 0) return;
    double S, D;
    if (stencil<false>(g, x, p, S, D))
        x[p] = (S + g.h2 * rhs[p]) * (1.0 / 6.0);
    else
        x[p] = (S + g.h2 * rhs[p]) / D;
}

// Alg. 3 after the pre-smooth, one thread per covered coarse cell P of
// level l-1: for the 8 children f, t_f = r_f - (A_nf e)_f (the homogeneous
// coarse-fine ghosts: e^{l-1} = 0), stored back into r_f; phi_f += e_f;
// r^{l-1}_P = mean of t_f (the 8-cell average R).
__global__ void k_restrict_amr(Grid gf, Grid gc, int clo0, int clo1, int clo2, int cn0, int cn1, int cn2,
                               double *__restrict__ rf, const double *__restrict__ ef, double *__restrict__ phif,
                               double *__restrict__ rc)
{
    int ci = clo0 + blockIdx.x * BX + threadIdx.x;
    int cj = clo1 + blockIdx.y * BY + threadIdx.y;
    int ck = clo2 + blockIdx.z;
    if (ci >= clo0 + cn0 || cj >= clo1 + cn1 || ck >= clo2 + cn2) return;
    int64_t P = pad_index(gc, ci, cj, ck);
    if (gc.mask[P] != 2) return;
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int64_t f = pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2));
        double S, D;
        stencil<false>(gf, ef, f, S, D);
        double t = rf[f] + gf.ih2 * (S - D * ef[f]);
        rf[f] = t;
        phif[f] += ef[f];
        acc += t;
    }
    rc[P] = 0.125 * acc;
}

// Alg. 3 prolongation and residual update, one thread per valid fine cell:
// e_f += I e^{l-1} (piecewise constant), r_f -= (A_nf I e^{l-1})_f.
__global__ void k_prolong_amr(Grid gf, Grid gc, double *__restrict__ ef, double *__restrict__ rf,
                              const double *__restrict__ ec)
{
    int a, b, c;
    int64_t p;
    if (!cell_coords(gf, a, b, c, p)) return;
    if (gf.mask[p] == 0) return;
    int i = gf.lo[0] + a - 1, j = gf.lo[1] + b - 1, k = gf.lo[2] + c - 1;
    auto v = [&](int di, int dj, int dk) {
        return ec[pad_index(gc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1)];
    };
    double vp = v(0, 0, 0);
    const int64_t off[6] = {-1, 1, -gf.sy, gf.sy, -gf.sz, gf.sz};
    const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
    double s = 0.0;
    int nv = 0, nc = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        uint8_t mn = gf.mask[p + off[f]];
        if (mn != 0) {
            s += v(di[f], dj[f], dk[f]);
            ++nv;
        } else {
            s -= kFifth * v(-di[f], -dj[f], -dk[f]);
            ++nc;
        }
    }
    double D = (nc == 0) ? 6.0 : (double)(3 * nv + nc) * kThird;
    ef[p] += vp;
    rf[p] += gf.ih2 * (s - D * vp);
}

// e += de; phi = phi_save + e (whole padded box; cells outside the level
// hold zeros in all three arrays).
__global__ void k_finish(int64_t n, double *__restrict__ e, const double *__restrict__ de,
                         double *__restrict__ phi, const double *__restrict__ phisave)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double v = e[t] + de[t];
        e[t] = v;
        phi[t] = phisave[t] + v;
    }
}

// Fine-side coarse part of the ghosts: t_f += scale * sum over the cell's
// coarse-fine faces of the (8/15)-weighted step-1 interpolation of uc.
__global__ void k_cf_correct(int ncell, const int *__restrict__ cell_f, const int *__restrict__ cell_ptr,
                             const int8_t *__restrict__ cnt, const int *__restrict__ cidx,
                             const double *__restrict__ cw, const double *__restrict__ uc, double *__restrict__ t,
                             double scale)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    double acc = 0.0;
    for (int q = cell_ptr[i]; q < cell_ptr[i + 1]; ++q) {
        int n = cnt[q];
        for (int k = 0; k < n; ++k) acc += cw[q * kMaxStencil + k] * uc[cidx[q * kMaxStencil + k]];
    }
    t[cell_f[i]] += scale * acc;
}

// Coarse rows next to the finer level l (flux matching, Eq.
// flux_differencing): r_C += 1/(2 h_c^2) * sum over the fine faces of C of
// (u_f - ghost_f) = (1/3) u_f + (1/5) u_f1 - coarse part.
__global__ void k_flux(int ncrse, const int *__restrict__ crse_c, const int *__restrict__ crse_ptr,
                       const int *__restrict__ crse_face, const int *__restrict__ ff, const int *__restrict__ ff1,
                       const int8_t *__restrict__ cnt, const int *__restrict__ cidx, const double *__restrict__ cw,
                       const double *__restrict__ uc, const double *__restrict__ uf, double *__restrict__ r,
                       double scale)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncrse) return;
    double acc = 0.0;
    for (int q = crse_ptr[i]; q < crse_ptr[i + 1]; ++q) {
        int face = crse_face[q];
        double cp = 0.0;
        int n = cnt[face];
        for (int k = 0; k < n; ++k) cp += cw[face * kMaxStencil + k] * uc[cidx[face * kMaxStencil + k]];
        acc += (kThird * uf[ff[face]] + kFifth * uf[ff1[face]]) - cp;
    }
    r[crse_c[i]] += scale * acc;
}

// E_d = -(u_{+d} - u_{-d}) / (2h) on valid cells; coarse-fine ghosts get
// their fine part here and their coarse part from k_cf_grad.
__global__ void k_grad(Grid g, const double *__restrict__ u, double *__restrict__ e0, double *__restrict__ e1,
                       double *__restrict__ e2)
{
    int a, b, c;
    int64_t p;
    if (!cell_coords(g, a, b, c, p)) return;
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
                          const int8_t *__restrict__ dir, const int8_t *__restrict__ cnt,
                          const int *__restrict__ cidx, const double *__restrict__ cw, const double *__restrict__ uc,
                          double *__restrict__ e0, double *__restrict__ e1, double *__restrict__ e2, double inv2h)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = cell_ptr[i]; q < cell_ptr[i + 1]; ++q) {
        double cp = 0.0;
        int n = cnt[q];
        for (int k = 0; k < n; ++k) cp += cw[q * kMaxStencil + k] * uc[cidx[q * kMaxStencil + k]];
        int d = dir[q] >> 1;
        double s = (dir[q] & 1) ? 1.0 : -1.0;
        acc[d] -= s * cp * inv2h;
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

// Per-block partial sums of v^2, |v| and max |v| over cells with mask == 1
// (or mask >= 1 when covered_too): fixed thread-to-cell assignment and a
// fixed shuffle tree, so the result is bitwise reproducible.
__global__ void k_norms(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ v, int covered_too,
                        double *__restrict__ part)
{
    double s2 = 0.0, s1 = 0.0, mx = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = mask[t];
        if (m == 1 || (covered_too && m == 2)) {
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
            part[blockIdx.x] = s2;
            part[kPartialBlocks + blockIdx.x] = s1;
            part[2 * kPartialBlocks + blockIdx.x] = mx;
        }
    }
}

// One block per slot: fixed-order sum of the kPartialBlocks partials.
__global__ void k_norms_finish(const double *__restrict__ part, double *__restrict__ out)
{
    const double *p = part + (int64_t)blockIdx.x * 3 * kPartialBlocks;
    double s2 = 0.0, s1 = 0.0, mx = 0.0;
    for (int t = threadIdx.x; t < kPartialBlocks; t += blockDim.x) {
        s2 += p[t];
        s1 += p[kPartialBlocks + t];
        mx = fmax(mx, p[2 * kPartialBlocks + t]);
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
            out[3 * blockIdx.x] = s2;
            out[3 * blockIdx.x + 1] = s1;
            out[3 * blockIdx.x + 2] = mx;
        }
    }
}

// Level-0 multigrid restriction, one thread per coarse cell:
// r_c = mean over the children of (r_f - A e_f); e_c = 0.
__global__ void k_mg_restrict(Grid gf, Grid gc, const double *__restrict__ ef, const double *__restrict__ rf,
                              double *__restrict__ rc, double *__restrict__ ec)
{
    int a, b, c;
    int64_t P;
    if (!cell_coords(gc, a, b, c, P)) return;
    int ci = gc.lo[0] + a - 1, cj = gc.lo[1] + b - 1, ck = gc.lo[2] + c - 1;
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int64_t f = pad_index(gf, 2 * ci + (o & 1), 2 * cj + ((o >> 1) & 1), 2 * ck + (o >> 2));
        double S, D;
        stencil<false>(gf, ef, f, S, D);
        acc += rf[f] + gf.ih2 * (S - D * ef[f]);
    }
    rc[P] = 0.125 * acc;
    ec[P] = 0.0;
}

// Level-0 multigrid trilinear prolongation of the correction, one thread
// per fine cell: weights 3/4 and 1/4 per axis on the two nearest coarse
// centres; outside the domain the coarse ghost is the Dirichlet mirror.
__global__ void k_mg_prolong(Grid gf, Grid gc, double *__restrict__ ef, const double *__restrict__ ec)
{
    int a, b, c;
    int64_t p;
    if (!cell_coords(gf, a, b, c, p)) return;
    int i = gf.lo[0] + a - 1, j = gf.lo[1] + b - 1, k = gf.lo[2] + c - 1;
    int I[3] = {i >> 1, j >> 1, k >> 1};
    int O[3] = {(i & 1) ? 1 : -1, (j & 1) ? 1 : -1, (k & 1) ? 1 : -1};
    int nc[3] = {gc.n[0] - 2, gc.n[1] - 2, gc.n[2] - 2};
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int sel[3] = {o & 1, (o >> 1) & 1, o >> 2};
        double w = 1.0, sign = 1.0;
        int Q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            w *= sel[d] ? 0.25 : 0.75;
            int q = I[d] + (sel[d] ? O[d] : 0);
            if (q < 0 || q >= nc[d]) {
                sign = -sign;
                q = I[d];
            }
            Q[d] = q;
        }
        acc += sign * w * ec[pad_index(gc, Q[0], Q[1], Q[2])];
    }
    ef[p] += acc;
}

// Coarsest grid of the level-0 multigrid: e = M r with the dense inverse M
// (order m); one warp per row, r staged in shared memory.
__global__ void k_coarse_solve(Grid g, int m, const double *__restrict__ M, const double *__restrict__ r,
                               double *__restrict__ e)
{
    extern __shared__ double rs[];
    int nx = g.n[0] - 2, ny = g.n[1] - 2;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        int i = t % nx, j = (t / nx) % ny, k = t / (nx * ny);
        rs[t] = r[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)];
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
        e[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)] = acc;
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

__global__ void k_fill(double *p, double v, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        p[t] = v;
}

__global__ void k_copy(double *__restrict__ d, const double *__restrict__ s, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        d[t] = s[t];
}

__global__ void k_axpy(double *__restrict__ y, const double *__restrict__ x, double a, int64_t n)
{
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

// Counts the launch and, when the timers are on, brackets it with a pair
// of events on the hierarchy's stream.
struct Launch {
    Hierarchy &H;
    int kind;
    double bytes;
    int ev = -1;
    Launch(Hierarchy &h, int k, double b) : H(h), kind(k), bytes(b)
    {
        if (!H.prof) return;
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
    static const char *names[K_NUM] = {"deposit", "gather", "residual", "rbgs", "restrict", "prolong", "finish",
                                       "cf_correct", "flux", "grad", "average_down", "norms", "mg_restrict",
                                       "mg_prolong", "coarse_solve", "elementwise"};
    return (kind >= 0 && kind < K_NUM) ? names[kind] : "";
}

// ------------------------------------------------------------- launchers

void launch_residual(Hierarchy &H, const Grid &g, const double *rho, const double *phi, double *res, int comp,
                     int zero_covered)
{
    Launch L(H, K_RESIDUAL, 24.0 * valid_cells(H, g));
    k_residual<<<cell_grid(g), dim3(BX, BY), 0, H.stream>>>(g, rho, phi, res, comp, zero_covered);
}

void launch_rbgs(Hierarchy &H, const Grid &g, double *x, const double *b, int colour)
{
    Launch L(H, K_RBGS, 16.0 * valid_cells(H, g));
    k_rbgs<<<cell_grid(g), dim3(BX, BY), 0, H.stream>>>(g, x, b, colour);
}

void launch_restrict_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l], &C = H.L[l - 1];
    int lo[3], n[3];
    footprint(H, l, lo, n);
    dim3 grid((unsigned)((n[0] + BX - 1) / BX), (unsigned)((n[1] + BY - 1) / BY), (unsigned)n[2]);
    Launch L(H, K_RESTRICT, 41.0 * (double)F.nvalid);
    k_restrict_amr<<<grid, dim3(BX, BY), 0, H.stream>>>(F.g, C.g, lo[0], lo[1], lo[2], n[0], n[1], n[2], F.res,
                                                         F.err, F.phi, C.res);
}

void launch_prolong_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l], &C = H.L[l - 1];
    Launch L(H, K_PROLONG, 33.0 * (double)F.nvalid);
    k_prolong_amr<<<cell_grid(F.g), dim3(BX, BY), 0, H.stream>>>(F.g, C.g, F.err, F.res, C.err);
}

void launch_finish_amr(Hierarchy &H, int l)
{
    Level &F = H.L[l];
    Launch L(H, K_FINISH, 40.0 * (double)F.nvalid);
    k_finish<<<elem_blocks(F.g.ncell), 256, 0, H.stream>>>(F.g.ncell, F.err, F.de, F.phi, F.phisave);
}

void launch_cf_correct(Hierarchy &H, int l, const double *uc, double *t, double scale)
{
    CfTable &T = H.L[l].cf;
    if (T.ncell == 0) return;
    Launch L(H, K_CF, 16.0 * T.ncell + 8.0 * T.nface * 9);
    k_cf_correct<<<(T.ncell + 127) / 128, 128, 0, H.stream>>>(T.ncell, T.cell_f, T.cell_ptr, T.cnt, T.cidx, T.cw,
                                                              uc, t, scale);
}

void launch_flux_correct(Hierarchy &H, int l, const double *uc, const double *uf, double *r)
{
    CfTable &T = H.L[l].cf;
    if (T.ncrse == 0) return;
    double scale = 0.5 * H.L[l - 1].g.ih2;
    Launch L(H, K_FLUX, 16.0 * T.ncrse + 16.0 * T.nface + 8.0 * T.nface * 9);
    k_flux<<<(T.ncrse + 127) / 128, 128, 0, H.stream>>>(T.ncrse, T.crse_c, T.crse_ptr, T.crse_face, T.f, T.f1,
                                                        T.cnt, T.cidx, T.cw, uc, uf, r, scale);
}

void launch_grad(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    Launch Lc(H, K_GRAD, 32.0 * (double)L.nvalid);
    k_grad<<<cell_grid(L.g), dim3(BX, BY), 0, H.stream>>>(L.g, L.phi, L.ef[0], L.ef[1], L.ef[2]);
}

void launch_cf_grad(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    CfTable &T = L.cf;
    if (T.ncell == 0) return;
    Launch Lc(H, K_CF, 48.0 * T.ncell + 8.0 * T.nface * 9);
    k_cf_grad<<<(T.ncell + 127) / 128, 128, 0, H.stream>>>(T.ncell, T.cell_f, T.cell_ptr, T.dir, T.cnt, T.cidx,
                                                           T.cw, H.L[l - 1].phi, L.ef[0], L.ef[1], L.ef[2],
                                                           0.5 / L.g.h);
}

void launch_average_down(Hierarchy &H, int l)
{
    Level &F = H.L[l + 1], &C = H.L[l];
    int lo[3], n[3];
    footprint(H, l + 1, lo, n);
    dim3 grid((unsigned)((n[0] + BX - 1) / BX), (unsigned)((n[1] + BY - 1) / BY), (unsigned)n[2]);
    Launch Lc(H, K_AVGDOWN, 9.0 * (double)F.nvalid);
    k_avgdown<<<grid, dim3(BX, BY), 0, H.stream>>>(F.g, C.g, lo[0], lo[1], lo[2], n[0], n[1], n[2], F.phi, C.phi);
}

void launch_norms(Hierarchy &H, int l, const double *v, int slot, int covered_too)
{
    Level &L = H.L[l];
    Launch Lc(H, K_NORMS, 9.0 * (double)L.nvalid);
    k_norms<<<kPartialBlocks, 256, 0, H.stream>>>(L.g.ncell, L.mask, v, covered_too,
                                                  H.partials + (int64_t)slot * 3 * kPartialBlocks);
}

void launch_norms_finish(Hierarchy &H, int nslots)
{
    Launch Lc(H, K_NORMS, 24.0 * kPartialBlocks * nslots);
    k_norms_finish<<<nslots, 256, 0, H.stream>>>(H.partials, H.norms);
}

void launch_mg_restrict(Hierarchy &H, int g)
{
    MgGrid &F = H.mg[g], &C = H.mg[g + 1];
    Launch Lc(H, K_MG_RESTRICT, 16.0 * valid_cells(H, F.g) + 16.0 * valid_cells(H, C.g));
    k_mg_restrict<<<cell_grid(C.g), dim3(BX, BY), 0, H.stream>>>(F.g, C.g, F.e, F.r, C.r, C.e);
}

void launch_mg_prolong(Hierarchy &H, int g)
{
    MgGrid &F = H.mg[g], &C = H.mg[g + 1];
    Launch Lc(H, K_MG_PROLONG, 16.0 * valid_cells(H, F.g) + 8.0 * valid_cells(H, C.g));
    k_mg_prolong<<<cell_grid(F.g), dim3(BX, BY), 0, H.stream>>>(F.g, C.g, F.e, C.e);
}

void launch_mg_coarse_solve(Hierarchy &H)
{
    MgGrid &G = H.mg[H.nmg - 1];
    int m = H.ncoarse;
    int threads = 256, warps = threads / 32;
    unsigned blocks = (unsigned)((m + warps - 1) / warps);
    Launch Lc(H, K_COARSE, 8.0 * (double)m * m + 16.0 * m);
    k_coarse_solve<<<blocks, threads, sizeof(double) * (size_t)m, H.stream>>>(G.g, m, H.coarse_inv, G.r, G.e);
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
    k_deposit<<<(unsigned)((n + 255) / 256), 256, 0, H.stream>>>(A, x, y, z, q, n);
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
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, H.stream>>>(A, x, y, z, n, ex, ey, ez, phi);
}

void launch_fill(Hierarchy &H, double *p, double v, int64_t n)
{
    Launch Lc(H, K_ELEMENTWISE, 8.0 * (double)n);
    k_fill<<<elem_blocks(n), 256, 0, H.stream>>>(p, v, n);
}

void launch_copy(Hierarchy &H, double *dst, const double *src, int64_t n)
{
    Launch Lc(H, K_ELEMENTWISE, 16.0 * (double)n);
    k_copy<<<elem_blocks(n), 256, 0, H.stream>>>(dst, src, n);
}

void launch_axpy(Hierarchy &H, double *y, const double *x, double a, int64_t n)
{
    Launch Lc(H, K_ELEMENTWISE, 24.0 * (double)n);
    k_axpy<<<elem_blocks(n), 256, 0, H.stream>>>(y, x, a, n);
}

} // namespace amr
