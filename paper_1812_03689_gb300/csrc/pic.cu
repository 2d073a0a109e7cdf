// The particle side of the space-charge step around the field solve
// (Sec. 4.1 domain transform, Fig. sc_workflow): mapping the particles into
// the computation cube, rescaling the solved potential and field back to
// particle space on the grid (Eqs. potential_transform and
// efield_transform), a kick-drift push with the gathered field, and the
// beam moments of Eqs. rms_sigma and halo.
//
// The transform, rescale and push are plain element-wise arithmetic written
// with rounded operations that are never contracted into FMAs, so their
// results are the same bits as the same formulas evaluated in FP64 on the
// host.  The moments are FP64 sums over the particles (atomic adds of
// per-block partials, so reproducible to rounding, not bitwise).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "amr_internal.h"

namespace amr {

namespace {

constexpr int kPThreads = 256;
constexpr int kPMaxBlocks = 152 * 8;

unsigned p_blocks(int64_t n)
{
    int64_t b = (n + kPThreads - 1) / kPThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kPMaxBlocks));
}

// max over particles and axes of |x_d - c_d| (non-negative: atomicMax on
// the bits orders like the values)
__global__ void k_extent(const double *x, const double *y, const double *z, int64_t n, double c0, double c1,
                         double c2, unsigned long long *mx)
{
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fmax(fabs(__dsub_rn(x[i], c0)), fmax(fabs(__dsub_rn(y[i], c1)), fabs(__dsub_rn(z[i], c2)))));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

// u = 1/2 + (x - c) * inv, per axis
__global__ void k_map(const double *x, const double *y, const double *z, int64_t n, double c0, double c1, double c2,
                      double inv, double *u, double *v, double *w)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = __dadd_rn(0.5, __dmul_rn(__dsub_rn(x[i], c0), inv));
        v[i] = __dadd_rn(0.5, __dmul_rn(__dsub_rn(y[i], c1), inv));
        w[i] = __dadd_rn(0.5, __dmul_rn(__dsub_rn(z[i], c2), inv));
    }
}

// a *= f over n values
__global__ void k_scale(double *a, int64_t n, double f)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = __dmul_rn(a[i], f);
}

// kick-drift: p += k E; x += d p (k = q/m dt, d = dt)
__global__ void k_push(double *x, double *y, double *z, double *px, double *py, double *pz, const double *ex,
                       const double *ey, const double *ez, int64_t n, double k, double d)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = __dadd_rn(px[i], __dmul_rn(k, ex[i]));
        const double b = __dadd_rn(py[i], __dmul_rn(k, ey[i]));
        const double c = __dadd_rn(pz[i], __dmul_rn(k, ez[i]));
        px[i] = a;
        py[i] = b;
        pz[i] = c;
        x[i] = __dadd_rn(x[i], __dmul_rn(d, a));
        y[i] = __dadd_rn(y[i], __dmul_rn(d, b));
        z[i] = __dadd_rn(z[i], __dmul_rn(d, c));
    }
}

// sums[a * 3 + w] of (coordinate w - m_w)^a for a = 1, 2, 4 (m = 0 on the
// first pass, the centroid on the second)
__global__ void k_moments(const double *x, const double *y, const double *z, int64_t n, const double *m,
                          double *sums)
{
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double *p[3] = {x, y, z};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int w = 0; w < 3; ++w) {
            const double d = p[w][i] - (m ? m[w] : 0.0), d2 = d * d;
            s[w] += d;
            s[3 + w] += d2;
            s[6 + w] += d2 * d2;
        }
    __shared__ double sh[9][kPThreads / 32];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
        if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = s[q];
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int k = 0; k < kPThreads / 32; ++k) t += sh[threadIdx.x][k];
        atomicAdd(&sums[threadIdx.x], t);
    }
}

} // namespace

} // namespace amr

using namespace amr;

extern "C" {

int amr_domain_transform(const double *x, const double *y, const double *z, int64_t n, const double centre_host[3],
                         double delta, double *u, double *v, double *w, double *scale_out_host, void *cuda_stream)
{
    set_error("");
    if (n < 0 || (n > 0 && (!x || !y || !z || !u || !v || !w)) || !centre_host || !scale_out_host ||
        !(delta >= 0.0 && delta <= 1e6)) {
        set_error("invalid domain-transform arguments");
        return AMR_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long *mx = nullptr;
    if (cudaMallocAsync((void **)&mx, sizeof(unsigned long long), st) != cudaSuccess) {
        set_error("out of memory");
        return AMR_ENOMEM;
    }
    cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st);
    if (n > 0)
        k_extent<<<p_blocks(n), kPThreads, 0, st>>>(x, y, z, n, centre_host[0], centre_host[1], centre_host[2], mx);
    unsigned long long bits = 0;
    cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(mx, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "domain transform");
    double ext;
    memcpy(&ext, &bits, sizeof(ext));
    if (!(ext > 0.0) || !std::isfinite(ext)) {
        set_error("the particles have no extent around the centre (or are not finite)");
        return AMR_EINVAL;
    }
    // s = (1 + delta) max Gamma with l = (1, 1, 1): the particles fill
    // [-1, 1]^3 / (1 + delta); the unit cube's edge is S = 2 s
    const double s = (1.0 + delta) * ext, S = 2.0 * s;
    if (n > 0) k_map<<<p_blocks(n), kPThreads, 0, st>>>(x, y, z, n, centre_host[0], centre_host[1], centre_host[2],
                                                        1.0 / S, u, v, w);
    *scale_out_host = S;
    e = cudaGetLastError();
    return e == cudaSuccess ? AMR_OK : cuda_fail(e, "domain transform");
}

int amr_rescale_fields(amr_hierarchy *h, double S)
{
    set_error("");
    if (!h || !(S > 0.0) || !std::isfinite(S)) {
        set_error("invalid rescale arguments");
        return AMR_EINVAL;
    }
    Hierarchy &H = *h->H;
    const double f1 = 1.0 / S, f2 = 1.0 / (S * S);
    for (int l = 0; l < H.nlev; ++l) {
        Level &L = H.L[l];
        const int64_t nc = L.g.ncell;
        k_scale<<<p_blocks(nc), kPThreads, 0, H.stream>>>(L.phi, nc, f1);
        for (int d = 0; d < 3; ++d) k_scale<<<p_blocks(nc), kPThreads, 0, H.stream>>>(L.ef[d], nc, f2);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMR_OK : cuda_fail(e, "rescale");
}

int amr_push(double *x, double *y, double *z, double *px, double *py, double *pz, const double *ex, const double *ey,
             const double *ez, int64_t n, double q_over_m, double dt, void *cuda_stream)
{
    set_error("");
    if (n < 0 || (n > 0 && (!x || !y || !z || !px || !py || !pz || !ex || !ey || !ez)) || !std::isfinite(q_over_m) ||
        !std::isfinite(dt)) {
        set_error("invalid push arguments");
        return AMR_EINVAL;
    }
    if (n == 0) return AMR_OK;
    const double k = q_over_m * dt;
    k_push<<<p_blocks(n), kPThreads, 0, (cudaStream_t)cuda_stream>>>(x, y, z, px, py, pz, ex, ey, ez, n, k, dt);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMR_OK : cuda_fail(e, "push");
}

int amr_moments(const double *x, const double *y, const double *z, int64_t n, double out_host[9], void *cuda_stream)
{
    set_error("");
    if (n <= 0 || !x || !y || !z || !out_host) {
        set_error("invalid moments arguments (n >= 1)");
        return AMR_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *buf = nullptr; // [0..8] first pass, [9..11] centroid, [12..20] second pass
    if (cudaMallocAsync((void **)&buf, 21 * sizeof(double), st) != cudaSuccess) {
        set_error("out of memory");
        return AMR_ENOMEM;
    }
    cudaMemsetAsync(buf, 0, 21 * sizeof(double), st);
    k_moments<<<p_blocks(n), kPThreads, 0, st>>>(x, y, z, n, nullptr, buf);
    double first[9];
    cudaMemcpyAsync(first, buf, sizeof(first), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return cuda_fail(e, "moments");
    }
    double m[3] = {first[0] / (double)n, first[1] / (double)n, first[2] / (double)n};
    cudaMemcpyAsync(buf + 9, m, sizeof(m), cudaMemcpyHostToDevice, st);
    k_moments<<<p_blocks(n), kPThreads, 0, st>>>(x, y, z, n, buf + 9, buf + 12);
    double c[9];
    cudaMemcpyAsync(c, buf + 12, sizeof(c), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "moments");
    for (int w = 0; w < 3; ++w) {
        const double m2 = c[3 + w] / (double)n, m4 = c[6 + w] / (double)n;
        out_host[w] = m[w];
        out_host[3 + w] = std::sqrt(m2);
        out_host[6 + w] = m2 > 0.0 ? m4 / (m2 * m2) : 0.0;
    }
    return AMR_OK;
}

} // extern "C"
