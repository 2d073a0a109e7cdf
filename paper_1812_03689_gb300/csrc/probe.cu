// FP64 arithmetic throughput probe: the denominator of the roofline of the
// FP64-bound kernels (this part runs FP64 at a small fraction of its FP32
// rate, so stencil sweeps, transforms, deposit and gather in FP64 are bound
// by the FP64 pipe rather than by HBM).
//
// Every thread runs kChains independent chains of dependent FMAs
// (x <- x * a + b, a slightly below 1 so the values stay bounded), enough
// chains per thread and resident warps per SM to keep the pipe busy; the
// result is written so that nothing is optimised away.
#include <cuda_runtime.h>

#include "amr_internal.h"

namespace amr {

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int64_t iters, double a, double b, double *out)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

} // namespace

} // namespace amr

extern "C" int amr_probe_fp64_fma(int64_t iters, double *gfma_per_s, double *ms_out, void *cuda_stream)
{
    if (iters <= 0 || iters > (int64_t)1 << 30 || !gfma_per_s) {
        amr::set_error("invalid probe arguments");
        return AMR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, amr::k_fma_probe, amr::kProbeThreads, 0);
    if (e != cudaSuccess) return amr::cuda_fail(e, "probe setup");
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMallocAsync((void **)&out, sizeof(double) * (size_t)blocks * amr::kProbeThreads, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        amr::k_fma_probe<<<blocks, amr::kProbeThreads, 0, s>>>(iters / 8 + 1, 0.9999999, 1e-7, out); // warm-up
        cudaEventRecord(e0, s);
        amr::k_fma_probe<<<blocks, amr::kProbeThreads, 0, s>>>(iters, 0.9999999, 1e-7, out);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (out) cudaFreeAsync(out, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return amr::cuda_fail(e, "probe");
    const double fmas = (double)blocks * amr::kProbeThreads * (double)iters * amr::kChains;
    *gfma_per_s = fmas / (ms * 1e-3) / 1e9;
    if (ms_out) *ms_out = ms;
    return AMR_OK;
}
