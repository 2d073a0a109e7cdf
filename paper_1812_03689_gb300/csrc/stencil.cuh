// Device-side pieces of the 7-point cell-centred stencil shared by every
// translation unit that relaxes or applies the level operator.
//
// Split of the flux-differenced operator (Eq. lap_flux_differencing with
// the coarse-fine ghosts of Eq. 2d_lagrange and Eq. 1d_interp):
//     (L u)_p = (S - D u_p) / h^2,   D = k / 3,
// with one contribution c_f to S and one increment to k per face f:
//     neighbour valid on the level          c_f = u_n           k += 3
//     physical boundary (Dirichlet 0)       c_f = 0             k += 6
//     physical boundary (Robin, Eq. robin_bc) c_f = 0           k += 64
//     coarse-fine face                      c_f = -(1/5) u_o    k += 1
// (u_o the inward neighbour opposite the face).  Codes below 64 take D from
// the constant tables; a Robin face adds (1 - alpha), alpha = (2d-h)/(2d+h)
// depending on the grid's h, so codes >= 64 read the grid's RobinTab.  The six contributions are
// always summed in the same tree, ((c0 + c1) + (c2 + c3)) + (c4 + c5) over
// the faces -x, +x, -y, +y, -z, +z, with rounded operations that the
// compiler may not contract, so a cell's update has the same bits in every
// kernel that computes it (per-colour passes, fused sweeps, any warp mix).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "amr_internal.h"

namespace amr {
namespace {

constexpr double kFifth = 0.2;

// D = k/3 and 1/D = 3/k for the face codes k = 0..36 of the split above.
#define AMR_K(k) ((double)(k) / 3.0)
#define AMR_IK(k) ((k) ? 3.0 / (double)(k) : 0.0)
#define AMR_KF(k) ((float)(k) / 3.0f)
#define AMR_IKF(k) ((k) ? 3.0f / (float)(k) : 0.0f)
#define AMR_ROW(M, b) M(b), M(b + 1), M(b + 2), M(b + 3), M(b + 4), M(b + 5)
#define AMR_TAB(M) AMR_ROW(M, 0), AMR_ROW(M, 6), AMR_ROW(M, 12), AMR_ROW(M, 18), AMR_ROW(M, 24), AMR_ROW(M, 30), M(36)
__constant__ double c_D[37] = {AMR_TAB(AMR_K)};
__constant__ double c_invD[37] = {AMR_TAB(AMR_IK)};
__constant__ float c_Df[37] = {AMR_TAB(AMR_KF)};
__constant__ float c_invDf[37] = {AMR_TAB(AMR_IKF)};
#undef AMR_TAB
#undef AMR_ROW
#undef AMR_IKF
#undef AMR_KF
#undef AMR_IK
#undef AMR_K

template <typename T> __device__ __forceinline__ T tabD(int k);
template <> __device__ __forceinline__ double tabD<double>(int k) { return c_D[k]; }
template <> __device__ __forceinline__ float tabD<float>(int k) { return c_Df[k]; }
template <typename T> __device__ __forceinline__ T tabInvD(int k);
template <> __device__ __forceinline__ double tabInvD<double>(int k) { return c_invD[k]; }
template <> __device__ __forceinline__ float tabInvD<float>(int k) { return c_invDf[k]; }

template <typename T> __device__ __forceinline__ T robinD(const RobinTab *t, int k);
template <> __device__ __forceinline__ double robinD<double>(const RobinTab *t, int k) { return t->D[k]; }
template <> __device__ __forceinline__ float robinD<float>(const RobinTab *t, int k) { return t->Df[k]; }
template <typename T> __device__ __forceinline__ T robinInvD(const RobinTab *t, int k);
template <> __device__ __forceinline__ double robinInvD<double>(const RobinTab *t, int k) { return t->invD[k]; }
template <> __device__ __forceinline__ float robinInvD<float>(const RobinTab *t, int k) { return t->invDf[k]; }

// D and 1/D of face code k on grid g (codes >= kRobinFace only on grids
// with Robin faces).
template <typename T> __device__ __forceinline__ T diagD(const Grid &g, int k)
{
    return k < kRobinFace ? tabD<T>(k) : robinD<T>(g.robin, k);
}
template <typename T> __device__ __forceinline__ T diagInvD(const Grid &g, int k)
{
    return k < kRobinFace ? tabInvD<T>(k) : robinInvD<T>(g.robin, k);
}

template <typename T> __device__ __forceinline__ T gh2(const Grid &g);
template <> __device__ __forceinline__ double gh2<double>(const Grid &g) { return g.h2; }
template <> __device__ __forceinline__ float gh2<float>(const Grid &g) { return g.h2f; }
template <typename T> __device__ __forceinline__ T gih2(const Grid &g);
template <> __device__ __forceinline__ double gih2<double>(const Grid &g) { return g.ih2; }
template <> __device__ __forceinline__ float gih2<float>(const Grid &g) { return g.ih2f; }

// Rounded add / multiply that are never fused into an FMA.
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ T sum6(T c0, T c1, T c2, T c3, T c4, T c5)
{
    return radd(radd(radd(c0, c1), radd(c2, c3)), radd(c4, c5));
}

// Contribution of one face: mn the neighbour's mask, valid whether it takes
// part as a plain neighbour, un / uo the neighbour and the opposite cell,
// dirichlet the grid's domain-face code increment (0: coarse-fine faces).
template <typename T>
__device__ __forceinline__ T face_c(bool valid, uint8_t mn, int dirichlet, T un, T uo, int &k)
{
    if (valid) {
        k += 3;
        return un;
    }
    if (mn != 0) return T(0); // covered neighbour in composite mode: no term
    if (dirichlet) {
        k += dirichlet;
        return T(0);
    }
    k += 1;
    return -rmul(T(kFifth), uo);
}

// Gauss-Seidel update of one cell of grid g: u = (S + h^2 b) / D.
template <typename T>
__device__ __forceinline__ T gs_update(const Grid &g, T S, T h2, T b, int k)
{
    return rmul(fma(h2, b, S), diagInvD<T>(g, k));
}

} // namespace
} // namespace amr
