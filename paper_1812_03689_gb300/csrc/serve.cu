// Served form: a continuous-batching request loop over independent solves.
//
// Requests arrive over time (their arrival_s); the scheduler admits the
// oldest waiting request as soon as a slot is free and its estimated device
// bytes fit in the HBM budget, and hands it to the slot's worker thread.
// Each worker owns a non-blocking CUDA stream and particle buffers, so the
// work of all admitted requests overlaps on the device while hierarchy
// creation (host tagging and ghost tables) of one request overlaps with the
// kernels of others.  A request is: seeded particles generated on the
// device (or the caller's particles) -> hierarchy (tagged) -> deposit ->
// solve -> gather (into the caller's buffer when given) -> checksums of the
// gathered field; its hierarchy and multigrid state stay on the device for
// the whole request and are released at its end.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "amr_internal.h"

namespace amr {

bool dst_wanted(int n0, bool not_dirichlet); // hierarchy.cu

namespace {

// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of
// two 32x32->64 multiplications with the published multipliers and Weyl
// key increments.
struct U4 {
    unsigned x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, unsigned k0, unsigned k1)
{
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        U4 n{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        c = n;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// Uniform in (0, 1] from 32 random bits.
__device__ __forceinline__ double u01(unsigned a, unsigned b)
{
    unsigned long long v = ((unsigned long long)a << 21) ^ (unsigned long long)(b >> 11);
    v &= (1ull << 53) - 1;
    return ((double)v + 1.0) * (1.0 / 9007199254740992.0);
}

// Isotropic Gaussian bunch: particle t from counter (t, attempt), normals by
// the Box-Muller transform; samples outside [h0, 1 - h0]^3 are redrawn
// (bounded attempts, then clamped).  Equal charges 1 / n.
__global__ void k_gen_particles(int64_t n, unsigned long long seed, double sigma, double cx, double cy, double cz,
                                double h0, double *x, double *y, double *z, double *q)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    unsigned k0 = (unsigned)seed, k1 = (unsigned)(seed >> 32);
    double p[3] = {cx, cy, cz};
    const double c[3] = {cx, cy, cz};
    for (int att = 0; att < 32; ++att) {
        U4 r0 = philox4x32_10(U4{(unsigned)t, (unsigned)(t >> 32), (unsigned)att, 0u}, k0, k1);
        U4 r1 = philox4x32_10(U4{(unsigned)t, (unsigned)(t >> 32), (unsigned)att, 1u}, k0, k1);
        double u1 = u01(r0.x, r0.y), u2 = u01(r0.z, r0.w), u3 = u01(r1.x, r1.y), u4 = u01(r1.z, r1.w);
        double ra = sqrt(-2.0 * log(u1)), rb = sqrt(-2.0 * log(u3));
        const double tp = 6.283185307179586;
        double g[3] = {ra * cos(tp * u2), ra * sin(tp * u2), rb * cos(tp * u4)};
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            p[d] = c[d] + sigma * g[d];
            ok &= p[d] >= h0 && p[d] <= 1.0 - h0;
        }
        if (ok) break;
        if (att == 31)
            for (int d = 0; d < 3; ++d) p[d] = fmin(fmax(p[d], h0), 1.0 - h0);
    }
    x[t] = p[0];
    y[t] = p[1];
    z[t] = p[2];
    q[t] = 1.0 / (double)n;
}

// Fixed-order checksums of the gathered field: per-block partial sums of
// Ex, Ey, Ez and |E|, then one block sums the partials in order.
constexpr int kSumBlocks = 256;

__global__ void k_sum_partials(int64_t n, const double *ex, const double *ey, const double *ez, double *part)
{
    __shared__ double sh[4][256];
    double s[4] = {0, 0, 0, 0};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double a = ex[t], b = ey[t], c = ez[t];
        s[0] += a;
        s[1] += b;
        s[2] += c;
        s[3] += sqrt(a * a + b * b + c * c);
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[k * kSumBlocks + blockIdx.x] = sh[k][0];
}

__global__ void k_sum_final(const double *part, double *out)
{
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int b = 0; b < kSumBlocks; ++b) s += part[threadIdx.x * kSumBlocks + b];
        out[threadIdx.x] = s;
    }
}

struct Slot {
    cudaStream_t stream = nullptr;
    double *buf = nullptr; // x, y, z, q, ex, ey, ez (7 n)
    int64_t cap = 0;
    double *part = nullptr, *sums = nullptr, *sums_host = nullptr;
    std::thread th;
    int job = -1; // request index, -1 idle
};

// Budget accounting: in_use is the sum of the charges of the requests that
// hold (or may allocate) device memory.  A request is charged its estimate
// (times admit_fraction when that is in (0, 1)) when admitted and its
// hierarchy is created under that charge as a hard cap
// (amr_desc.max_device_bytes), so in_use never exceeds the budget.  A
// request whose tagged boxes turn out larger than its charge fails that
// creation (nothing of it stays allocated), gives its charge back, waits
// until twice the charge is free (at most the whole budget, which needs
// every other charge released) and is created again under the new charge;
// while a request waits, nothing new is admitted.  It is refused with
// AMR_ENOMEM if even the whole budget is too small.
struct Server {
    std::mutex mu;
    std::condition_variable cv_sched, cv_work;
    std::vector<Slot> slots;
    std::vector<int64_t> est, charge;
    int retry_waiters = 0; // requests waiting for a larger charge
    const amr_request *reqs = nullptr;
    amr_request_result *out = nullptr;
    amr_solve_opts opts{};
    int64_t budget = 0, in_use = 0;
    int done = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

// Device bytes of a request, an upper bound of what its hierarchy
// allocates (amr_device_bytes) plus its particle buffer: the level-0 box, the
// level-0 multigrid grids and their dense coarsest inverse, the exact bottom's
// arrays, refined boxes spanning about 2 x 2.5 sigma plus two bricks per axis,
// their coarse-fine face tables, the fused sweeps' second iterate, and the
// seven particle arrays of the slot.
int64_t estimate_bytes(const amr_request &r)
{
    const bool mixed = r.precision == AMR_MIXED;
    const double per_cell = 2.0 + 72.0 + (mixed ? 20.0 : 0.0); // mask, code, 9 FP64 (+ 5 FP32) fields
    const double n0 = (double)r.n0;
    const double c0 = std::pow(n0 + 2.0, 3.0);
    double bytes = c0 * per_cell, big = c0;
    // level-0 multigrid: halve while the extent is even and above 8; each
    // coarser grid holds mask, code, e and r (+ FP32 copies); the coarsest is
    // inverted densely
    int m = r.n0;
    while (m % 2 == 0 && m > 8) {
        m /= 2;
        bytes += std::pow((double)m + 2.0, 3.0) * (2.0 + 16.0 + (mixed ? 8.0 : 0.0));
    }
    const double mc = (double)m * m * m;
    // the coarsest grid: a dense inverse up to 11^3, else two work arrays of
    // its separable solve
    bytes += m <= 11 ? mc * mc * 8.0 : 2.0 * 8.0 * std::pow((double)m + 2.0, 3.0) + 3.0 * 8.0 * m * m;
    if (dst_wanted(r.n0, false)) bytes += 3.0 * 8.0 * c0 + 2.0 * 8.0 * n0 * n0 + 16.0 * n0;
    const double w = std::min(1.0, 5.0 * r.sigma + 0.05);
    for (int l = 1; l <= r.max_level; ++l) {
        const double nl = (double)((int64_t)r.n0 << l);
        const double side = std::min(nl, nl * w + 16.0) + 2.0, cells = side * side * side;
        // fields, cell list, the coarser level's covered-cell list, face tables
        bytes += cells * (per_cell + 4.5) + 6.0 * side * side * 160.0;
        big = std::max(big, cells);
    }
    bytes += 8.0 * big;                                 // second iterate of the fused sweeps
    bytes += (double)kMaxLevels * 6.0 * kPartialBlocks * 8.0 + (2 << 20);
    bytes += 56.0 * (double)r.n_particles;              // x, y, z, q, Ex, Ey, Ez
    return (int64_t)(bytes * 1.1) + (8 << 20);
}

void run_request(Server &S, Slot &slot, int i)
{
    const amr_request &r = S.reqs[i];
    amr_request_result &res = S.out[i];
    auto fail = [&](int code) {
        res.status = code;
        res.done_s = S.now();
    };
    if (r.n_particles <= 0 || r.n0 < 8) return fail(AMR_EINVAL);
    const bool given = r.x != nullptr;
    if (given && (!r.y || !r.z || !r.q)) return fail(AMR_EINVAL);
    if (slot.cap < r.n_particles) {
        // stream-ordered (pool) allocation: growing one slot's buffer does
        // not synchronise the device under the other slots
        if (slot.buf) cudaFreeAsync(slot.buf, slot.stream);
        slot.buf = nullptr;
        slot.cap = 0;
        if (cudaMallocAsync((void **)&slot.buf, sizeof(double) * 7 * (size_t)r.n_particles, slot.stream) !=
            cudaSuccess) {
            cudaGetLastError();
            return fail(AMR_ENOMEM);
        }
        slot.cap = r.n_particles;
    }
    int64_t n = r.n_particles;
    double *x = slot.buf, *y = x + n, *z = y + n, *q = z + n, *ex = q + n, *ey = ex + n, *ez = ey + n;
    double *phi_p = nullptr;
    if (r.field_out) {
        // the caller's buffer: Ex, Ey, Ez and phi at the particles
        ex = r.field_out;
        ey = ex + n;
        ez = ey + n;
        phi_p = ez + n;
    }
    if (given) {
        x = const_cast<double *>(r.x);
        y = const_cast<double *>(r.y);
        z = const_cast<double *>(r.z);
        q = const_cast<double *>(r.q);
    } else {
        k_gen_particles<<<(unsigned)((n + 255) / 256), 256, 0, slot.stream>>>(n, r.seed, r.sigma, r.centre[0],
                                                                            r.centre[1], r.centre[2], 1.0 / r.n0,
                                                                            x, y, z, q);
    }
    amr_desc d;
    amr_desc_default(&d);
    d.n0 = r.n0;
    d.max_level = r.max_level;
    d.precision = r.precision;
    const int64_t parts = 56 * n; // the slot's particle arrays, outside the hierarchy
    d.max_device_bytes = std::max<int64_t>(1, S.est[i] - parts);
    amr_hierarchy *h = nullptr;
    int rc = amr_create_hierarchy(&d, x, y, z, q, n, slot.stream, &h);
    // larger than its charge: give the charge back, wait until twice the
    // charge (at most the whole budget) is free, and create it again under
    // that cap; the whole budget is the last try
    int64_t want = S.charge[i];
    while (rc == AMR_ENOMEM && want < S.budget) {
        {
            std::unique_lock<std::mutex> lk(S.mu);
            S.in_use -= S.charge[i];
            S.charge[i] = 0;
            want = std::min<int64_t>(S.budget, 2 * want);
            S.retry_waiters++;
            S.cv_sched.notify_all();
            S.cv_work.wait(lk, [&] { return S.in_use + want <= S.budget; });
            S.retry_waiters--;
            S.charge[i] = want;
            S.in_use += want;
        }
        d.max_device_bytes = std::max<int64_t>(1, want - parts);
        res.retried = 1;
        rc = amr_create_hierarchy(&d, x, y, z, q, n, slot.stream, &h);
    }
    if (rc != AMR_OK) return fail(rc);
    amr_solve_stats st{};
    rc = amr_solve(h, &S.opts, &st);
    if (rc == AMR_OK || rc == AMR_ENOCONV) rc = amr_gather(h, x, y, z, n, ex, ey, ez, phi_p) == AMR_OK ? rc : AMR_ECUDA;
    if (rc == AMR_OK || rc == AMR_ENOCONV) {
        k_sum_partials<<<kSumBlocks, 256, 0, slot.stream>>>(n, ex, ey, ez, slot.part);
        k_sum_final<<<1, 32, 0, slot.stream>>>(slot.part, slot.sums);
        cudaMemcpyAsync(slot.sums_host, slot.sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, slot.stream);
        if (cudaStreamSynchronize(slot.stream) != cudaSuccess) rc = AMR_ECUDA;
        for (int k = 0; k < 4; ++k) res.checksum[k] = slot.sums_host[k];
    }
    int64_t bytes = 0;
    amr_device_bytes(h, &bytes);
    res.device_bytes = bytes;
    res.iters = st.iters;
    res.n_levels = st.n_levels;
    res.rel_res_max = 0.0;
    for (int l = 0; l < st.n_levels; ++l) res.rel_res_max = std::max(res.rel_res_max, st.rel_res[l]);
    amr_destroy(h);
    res.status = rc;
    res.done_s = S.now();
}

void worker(Server *S, int k)
{
    Slot &slot = S->slots[k];
    for (;;) {
        int job;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || slot.job >= 0; });
            if (slot.job < 0 && S->stop) return;
            job = slot.job;
        }
        run_request(*S, slot, job);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= S->charge[job];
            S->charge[job] = 0;
            S->done++;
            slot.job = -1;
        }
        S->cv_sched.notify_all();
        S->cv_work.notify_all();
    }
}

} // namespace

int serve(const amr_serve_config *cfg, const amr_request *reqs, int n, const amr_solve_opts *opts,
          amr_request_result *out)
{
    Server S;
    S.reqs = reqs;
    S.out = out;
    amr_solve_opts_default(&S.opts);
    if (opts) S.opts = *opts;
    S.budget = cfg->budget_bytes;
    int nslots = std::max(1, std::min(cfg->max_slots, 256));
    S.slots.resize(nslots);
    S.est.resize(n);
    S.charge.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        S.est[i] = estimate_bytes(reqs[i]);
        if (cfg->admit_fraction > 0.0 && cfg->admit_fraction < 1.0)
            S.est[i] = std::max<int64_t>(1, (int64_t)std::ceil(cfg->admit_fraction * (double)S.est[i]));
        memset(&out[i], 0, sizeof(out[i]));
        out[i].arrival_s = cfg->realtime ? reqs[i].arrival_s : 0.0;
        out[i].status = -1;
    }
    for (Slot &s : S.slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&s.part, sizeof(double) * 4 * kSumBlocks) != cudaSuccess ||
            cudaMalloc(&s.sums, sizeof(double) * 4) != cudaSuccess ||
            cudaMallocHost(&s.sums_host, sizeof(double) * 4) != cudaSuccess) {
            cudaGetLastError();
            set_error("out of memory (serve slots)");
            for (Slot &t : S.slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.part) cudaFree(t.part);
                if (t.sums) cudaFree(t.sums);
                if (t.sums_host) cudaFreeHost(t.sums_host);
            }
            return AMR_ENOMEM;
        }
    }
    S.t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < nslots; ++k) S.slots[k].th = std::thread(worker, &S, k);
    int next = 0;
    {
        std::unique_lock<std::mutex> lk(S.mu);
        while (S.done < n) {
            double t = S.now();
            // admit in arrival order while a slot is free and the budget allows
            while (next < n) {
                double arr = cfg->realtime ? reqs[next].arrival_s : 0.0;
                if (arr > t) break;
                if (S.est[next] > S.budget) {
                    out[next].status = AMR_ENOMEM;
                    out[next].admit_s = out[next].done_s = t;
                    S.done++;
                    ++next;
                    continue;
                }
                // nothing new while a request waits for a larger charge
                if (S.retry_waiters > 0) break;
                if (S.in_use + S.est[next] > S.budget) break;
                int free_slot = -1;
                for (int k = 0; k < nslots; ++k)
                    if (S.slots[k].job < 0) {
                        free_slot = k;
                        break;
                    }
                if (free_slot < 0) break;
                S.in_use += S.est[next];
                S.charge[next] = S.est[next];
                out[next].admit_s = t;
                S.slots[free_slot].job = next;
                ++next;
                S.cv_work.notify_all();
            }
            if (S.done >= n) break;
            double wait_s = 0.002;
            if (next < n && cfg->realtime) wait_s = std::min(wait_s, std::max(0.0, reqs[next].arrival_s - t));
            S.cv_sched.wait_for(lk, std::chrono::duration<double>(std::max(wait_s, 1e-4)));
        }
        S.stop = true;
    }
    S.cv_work.notify_all();
    for (Slot &s : S.slots) s.th.join();
    for (Slot &s : S.slots) {
        if (s.buf) cudaFreeAsync(s.buf, s.stream);
        cudaStreamSynchronize(s.stream);
        cudaFree(s.part);
        cudaFree(s.sums);
        cudaFreeHost(s.sums_host);
        cudaStreamDestroy(s.stream);
    }
    return AMR_OK;
}

int64_t request_bytes(const amr_request *r) { return estimate_bytes(*r); }

} // namespace amr

extern "C" {

int amr_serve(const amr_serve_config *cfg, const amr_request *reqs, int n, const amr_solve_opts *opts,
              amr_request_result *results)
{
    if (!cfg || !reqs || n <= 0 || !results || cfg->budget_bytes <= 0 || cfg->max_slots <= 0) {
        amr::set_error("invalid serve arguments");
        return AMR_EINVAL;
    }
    return amr::serve(cfg, reqs, n, opts, results);
}

int amr_request_bytes(const amr_request *r, int64_t *bytes_out)
{
    if (!r || !bytes_out) return AMR_EINVAL;
    *bytes_out = amr::request_bytes(r);
    return AMR_OK;
}

} // extern "C"
