// Allocation-free variant of the masked norm reduction.
//
// The library's own norm reduction (used by amr_residual and the solve's
// convergence test) writes its per-block partial sums into scratch memory
// that amr_create_hierarchy allocates.  This entry point computes the same
// quantities for caller-supplied arrays without allocating anything: its
// scratch is a fixed file-scope device array that every GPU loading the
// library holds until the process exits.  It is meant for callers that
// cannot call cudaMalloc: code running while a CUDA graph is being captured
// on the current thread, callers that own a memory pool and forbid other
// allocations, or real-time loops where an allocation could synchronise the
// device.
#include <cuda_runtime.h>

#include <mutex>

#include "amr_internal.h"

namespace amr {

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1024;
// Largest n accepted: every thread of the at most kNaMaxBlocks blocks then
// reduces at most 256 elements.
constexpr int64_t kNaMaxN = (int64_t)kNaMaxBlocks * kNaThreads * 256;

// Per-block partials {sum v^2, sum |v|, max |v|} of one call (24 KiB).
static __device__ __align__(256) double g_norm_scratch[3 * kNaMaxBlocks];

// The max norm is taken on the bit pattern of |x|: for non-negative doubles
// the unsigned order of the bits is the numeric order and a NaN sorts above
// +inf, so a NaN element makes the max norm NaN (as it makes the sums NaN),
// exactly as the library's own norms do.
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__global__ void k_na_partials(int64_t n, const uint8_t *mask, const double *v, int covered_too, double *part)
{
    double s2 = 0.0, s1 = 0.0;
    unsigned long long mx = 0ull;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = mask ? mask[t] : 1;
        if (m == 1 || (covered_too && m == 2)) {
            double x = v[t];
            s2 += x * x;
            s1 += fabs(x);
            mx = max(mx, abs_bits(x));
        }
    }
    __shared__ double sh[2][kNaThreads / 32];
    __shared__ unsigned long long shm[kNaThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][w] = s2;
        sh[1][w] = s1;
        shm[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        unsigned long long c = 0ull;
        for (int q = 0; q < kNaThreads / 32; ++q) {
            a += sh[0][q];
            b += sh[1][q];
            c = max(c, shm[q]);
        }
        part[blockIdx.x] = a;
        part[kNaMaxBlocks + blockIdx.x] = b;
        part[2 * kNaMaxBlocks + blockIdx.x] = __longlong_as_double((long long)c);
    }
}

// One thread sums the nb partials in block order (fixed order: bitwise
// reproducible for a given n).
__global__ void k_na_final(int nb, const double *part, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    unsigned long long c = 0ull;
    for (int q = 0; q < nb; ++q) {
        a += part[q];
        b += part[kNaMaxBlocks + q];
        c = max(c, abs_bits(part[2 * kNaMaxBlocks + q]));
    }
    out[0] = a;
    out[1] = b;
    out[2] = __longlong_as_double((long long)c);
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in, never a device
// address).
std::mutex g_na_mu;
double *g_na_ptr[64] = {};

int scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc norms: current device");
    if (dev < 0 || dev >= 64) {
        set_error("no-alloc norms: device index out of range");
        return AMR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_norm_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "no-alloc norms: scratch address");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return AMR_OK;
}

} // namespace
} // namespace amr

extern "C" int amr_masked_norms_noalloc(const double *v, const uint8_t *mask, int64_t n, int covered_too,
                                        double *out3, void *cuda_stream)
{
    if (!v || !out3 || n < 0) {
        amr::set_error("invalid no-alloc norms arguments");
        return AMR_EINVAL;
    }
    if (n > amr::kNaMaxN) {
        amr::set_error("no-alloc norms: n exceeds the maximum of 67108864 elements");
        return AMR_EINVAL;
    }
    double *scratch = nullptr;
    int rc = amr::scratch_for_current_device(&scratch);
    if (rc != AMR_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int64_t want = (n + amr::kNaThreads - 1) / amr::kNaThreads;
    int nb = (int)(want < 1 ? 1 : (want > amr::kNaMaxBlocks ? amr::kNaMaxBlocks : want));
    amr::k_na_partials<<<nb, amr::kNaThreads, 0, s>>>(n, mask, v, covered_too, scratch);
    amr::k_na_final<<<1, 32, 0, s>>>(nb, scratch, out3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return amr::cuda_fail(e, "no-alloc norms launch");
    return AMR_OK;
}
