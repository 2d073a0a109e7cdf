// Regrid (Sec. 4.2, AMR policies): the refined levels of a new hierarchy
// from the fields of an existing one, and the warm-start transfer of the
// potential into the new hierarchy.
//
// Tagging and block marking run on the device, one thread per cell of the
// tagged level: the level maxima the relative policies need are reduced
// first (atomicMax on the bit patterns of non-negative doubles, which order
// like the unsigned integers), then every tagged cell marks the aligned
// bc^3 blocks that its buffer neighbourhood touches.  Only the block marks
// (one byte per block of the level's bounding box) come back to the host,
// where each marked block is kept if it is properly nested in the new
// coarser level, exactly as when a hierarchy is created.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <unordered_set>
#include <vector>

#include "amr_internal.h"

namespace amr {

namespace {

constexpr int kRgThreads = 256;
constexpr int kRgMaxBlocks = 152 * 8;
constexpr int kNestCells = 2; // proper nesting margin, as at creation

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// Level maxima over the valid cells: max(rho, 0), |phi|, |E_x|, |E_y|, |E_z|.
__global__ void k_tag_max(int64_t ncell, const uint8_t *mask, const double *rho, const double *phi,
                          const double *ex, const double *ey, const double *ez, unsigned long long *mx)
{
    double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < ncell;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (mask[p] == 0) continue;
        m[0] = fmax(m[0], rho[p]);
        m[1] = fmax(m[1], fabs(phi[p]));
        m[2] = fmax(m[2], fabs(ex[p]));
        m[3] = fmax(m[3], fabs(ey[p]));
        m[4] = fmax(m[4], fabs(ez[p]));
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        for (int o = 16; o > 0; o >>= 1) m[q] = fmax(m[q], __shfl_xor_sync(0xffffffffu, m[q], o));
        if ((threadIdx.x & 31) == 0 && m[q] > 0.0) atomic_max_nonneg(&mx[q], m[q]);
    }
}

struct MarkA {
    Grid g;
    const uint8_t *mask;
    const double *rho, *phi, *ex, *ey, *ez;
    const unsigned long long *mx;
    int policy;
    double lambda, eps0;
    int buffer, bc, nl;
    int blo[3], nb[3];
    uint8_t *mark;
};

// The tag test of one cell (same arithmetic as at creation: one product,
// one comparison, in FP64).
__device__ __forceinline__ bool tagged(const MarkA &A, int64_t p)
{
    switch (A.policy) {
    case AMR_TAG_ABS_RHO:
        return fabs(A.rho[p] * A.eps0) >= A.lambda;
    case AMR_TAG_PHI: {
        const double m = __longlong_as_double((long long)A.mx[1]);
        return m > 0.0 && fabs(A.phi[p]) >= A.lambda * m;
    }
    case AMR_TAG_EFIELD: {
        const double *e[3] = {A.ex, A.ey, A.ez};
        bool t = false;
#pragma unroll
        for (int w = 0; w < 3; ++w) {
            const double m = __longlong_as_double((long long)A.mx[2 + w]);
            t |= m > 0.0 && fabs(e[w][p]) >= A.lambda * m;
        }
        return t;
    }
    default: {
        const double m = __longlong_as_double((long long)A.mx[0]);
        return m > 0.0 && A.rho[p] > A.lambda * m;
    }
    }
}

// Each tagged valid cell marks the blocks its buffer neighbourhood (clipped
// to the domain) touches.  Concurrent stores write the same byte value.
__global__ void k_tag_mark(const MarkA A)
{
    const Grid &g = A.g;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < g.ncell;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (A.mask[p] == 0 || !tagged(A, p)) continue;
        const int c = (int)(p / g.sz), b = (int)((p - (int64_t)c * g.sz) / g.sy);
        const int a = (int)(p - (int64_t)c * g.sz - (int64_t)b * g.sy);
        const int x[3] = {g.lo[0] + a - 1, g.lo[1] + b - 1, g.lo[2] + c - 1};
        int b0[3], b1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            b0[d] = max(x[d] - A.buffer, 0) / A.bc - A.blo[d];
            b1[d] = min(x[d] + A.buffer, A.nl - 1) / A.bc - A.blo[d];
        }
        for (int bk = b0[2]; bk <= b1[2]; ++bk)
            for (int bj = b0[1]; bj <= b1[1]; ++bj)
                for (int bi = b0[0]; bi <= b1[0]; ++bi)
                    A.mark[((int64_t)bk * A.nb[1] + bj) * A.nb[0] + bi] = 1;
    }
}

// Warm start: phi of dst level l from src level l where src holds the cell,
// else the parent's value on dst level l-1 (piecewise constant, the
// prolongation I of the V-cycle).
struct TransferA {
    Grid gd, gs, gp;  // dst level l, src level l, dst level l-1
    const uint8_t *md, *ms;
    const double *phis, *phip;
    double *phid;
    int has_src, has_parent;
};

__global__ void k_transfer_phi(const TransferA A)
{
    const Grid &g = A.gd;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < g.ncell;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (A.md[p] == 0) continue;
        const int c = (int)(p / g.sz), b = (int)((p - (int64_t)c * g.sz) / g.sy);
        const int a = (int)(p - (int64_t)c * g.sz - (int64_t)b * g.sy);
        const int x[3] = {g.lo[0] + a - 1, g.lo[1] + b - 1, g.lo[2] + c - 1};
        double v = 0.0;
        bool done = false;
        if (A.has_src) {
            const Grid &s = A.gs;
            const int sa = x[0] - s.lo[0] + 1, sb = x[1] - s.lo[1] + 1, sc = x[2] - s.lo[2] + 1;
            if (sa >= 1 && sb >= 1 && sc >= 1 && sa < s.n[0] - 1 && sb < s.n[1] - 1 && sc < s.n[2] - 1) {
                const int64_t q = (int64_t)sc * s.sz + (int64_t)sb * s.sy + sa;
                if (A.ms[q] != 0) {
                    v = A.phis[q];
                    done = true;
                }
            }
        }
        if (!done && A.has_parent) {
            const Grid &s = A.gp;
            const int64_t q = (int64_t)((x[2] >> 1) - s.lo[2] + 1) * s.sz +
                              (int64_t)((x[1] >> 1) - s.lo[1] + 1) * s.sy + ((x[0] >> 1) - s.lo[0] + 1);
            v = A.phip[q];
        }
        A.phid[p] = v;
    }
}

// Composite volume mean: sum of v h^3 over the cells with mask 1 (valid
// and uncovered: the composite domain; the unit cube has volume 1).
__global__ void k_mean(int64_t ncell, const uint8_t *mask, const double *v, double vol, double *sum)
{
    double s = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < ncell;
         p += (int64_t)gridDim.x * blockDim.x)
        if (mask[p] == 1) s += v[p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(sum, s * vol);
}

// v -= mean on every valid cell
__global__ void k_sub_mean(int64_t ncell, const uint8_t *mask, double *v, const double *mean)
{
    const double m = *mean;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < ncell;
         p += (int64_t)gridDim.x * blockDim.x)
        if (mask[p] != 0) v[p] -= m;
}

// Eroded mask: out[p] = 1 iff every cell within Chebyshev distance b of p
// lies in the padded box and is valid (mask != 0).
__global__ void k_erode(const Grid g, const uint8_t *mask, int b, uint8_t *out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < g.ncell;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(p / g.sz), bb = (int)((p - (int64_t)c * g.sz) / g.sy);
        const int a = (int)(p - (int64_t)c * g.sz - (int64_t)bb * g.sy);
        uint8_t ok = mask[p] != 0;
        if (ok && (a - b < 0 || bb - b < 0 || c - b < 0 || a + b >= g.n[0] || bb + b >= g.n[1] || c + b >= g.n[2]))
            ok = 0;
        for (int k = c - b; k <= c + b && ok; ++k)
            for (int j = bb - b; j <= bb + b && ok; ++j)
                for (int i = a - b; i <= a + b && ok; ++i)
                    if (mask[(int64_t)k * g.sz + (int64_t)j * g.sy + i] == 0) ok = 0;
        out[p] = ok;
    }
}

unsigned rg_blocks(int64_t n)
{
    int64_t b = (n + kRgThreads - 1) / kRgThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kRgMaxBlocks));
}

// Is every cell of [lo, hi] (level l, inclusive) inside the domain and valid
// on the new level l (level 0: the whole domain; l >= 1: a union of aligned
// bricks of edge `brick`)?
bool nested(int l, int nl, int brick, const std::unordered_set<int64_t> &bricks, const int lo[3], const int hi[3])
{
    for (int d = 0; d < 3; ++d)
        if (lo[d] < 0 || hi[d] > nl - 1) return false;
    if (l == 0) return true;
    const int64_t nbk = nl / brick;
    for (int k = lo[2] / brick; k <= hi[2] / brick; ++k)
        for (int j = lo[1] / brick; j <= hi[1] / brick; ++j)
            for (int i = lo[0] / brick; i <= hi[0] / brick; ++i)
                if (!bricks.count(((int64_t)k * nbk + j) * nbk + i)) return false;
    return true;
}

} // namespace

int regrid_boxes(Hierarchy &H, int policy, double lambda, int buffer, int max_level, std::vector<int> &out)
{
    out.clear();
    const int bc = H.brick / 2;
    unsigned long long *mx = nullptr;
    if (cudaMallocAsync((void **)&mx, 5 * sizeof(unsigned long long), H.stream) != cudaSuccess) {
        set_error("out of memory");
        return AMR_ENOMEM;
    }
    std::unordered_set<int64_t> bricks; // bricks of the new level l (l >= 1)
    int rc = AMR_OK;
    for (int l = 0; l < H.nlev && l + 1 <= max_level; ++l) {
        const Level &L = H.L[l];
        const int nl = H.n0 << l;
        MarkA A{};
        A.g = L.g;
        A.mask = L.mask;
        A.rho = L.rho;
        A.phi = L.phi;
        A.ex = L.ef[0];
        A.ey = L.ef[1];
        A.ez = L.ef[2];
        A.mx = mx;
        A.policy = policy;
        A.lambda = lambda;
        A.eps0 = H.eps0;
        A.buffer = buffer;
        A.bc = bc;
        A.nl = nl;
        int64_t nmark = 1;
        for (int d = 0; d < 3; ++d) {
            A.blo[d] = std::max(L.vlo[d] - buffer, 0) / bc;
            const int bhi = std::min(L.vhi[d] + buffer, nl - 1) / bc;
            A.nb[d] = bhi - A.blo[d] + 1;
            nmark *= A.nb[d];
        }
        uint8_t *mark = nullptr;
        if (cudaMallocAsync((void **)&mark, (size_t)nmark, H.stream) != cudaSuccess) {
            set_error("out of memory");
            rc = AMR_ENOMEM;
            break;
        }
        A.mark = mark;
        cudaMemsetAsync(mx, 0, 5 * sizeof(unsigned long long), H.stream);
        cudaMemsetAsync(mark, 0, (size_t)nmark, H.stream);
        const unsigned nb = rg_blocks(L.g.ncell);
        k_tag_max<<<nb, kRgThreads, 0, H.stream>>>(L.g.ncell, L.mask, L.rho, L.phi, L.ef[0], L.ef[1], L.ef[2], mx);
        k_tag_mark<<<nb, kRgThreads, 0, H.stream>>>(A);
        std::vector<uint8_t> hm((size_t)nmark);
        cudaMemcpyAsync(hm.data(), mark, (size_t)nmark, cudaMemcpyDeviceToHost, H.stream);
        cudaFreeAsync(mark, H.stream);
        cudaError_t e = cudaStreamSynchronize(H.stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "regrid tagging");
            break;
        }
        // keep the properly nested blocks, in (k, j, i) block order
        std::unordered_set<int64_t> next;
        const int nbk1 = (2 * nl) / H.brick;
        int kept = 0;
        for (int bk = 0; bk < A.nb[2]; ++bk)
            for (int bj = 0; bj < A.nb[1]; ++bj)
                for (int bi = 0; bi < A.nb[0]; ++bi) {
                    if (!hm[((size_t)bk * A.nb[1] + bj) * A.nb[0] + bi]) continue;
                    const int b3[3] = {A.blo[0] + bi, A.blo[1] + bj, A.blo[2] + bk};
                    int lo[3], hi[3];
                    for (int d = 0; d < 3; ++d) {
                        lo[d] = b3[d] * bc - kNestCells;
                        hi[d] = b3[d] * bc + bc - 1 + kNestCells;
                    }
                    if (!nested(l, nl, H.brick, bricks, lo, hi)) continue;
                    out.push_back(l + 1);
                    for (int d = 0; d < 3; ++d) out.push_back(2 * bc * b3[d]);
                    for (int d = 0; d < 3; ++d) out.push_back(2 * bc * b3[d] + 2 * bc - 1);
                    next.insert(((int64_t)b3[2] * nbk1 + b3[1]) * nbk1 + b3[0]);
                    ++kept;
                }
        if (!kept) break;
        bricks.swap(next);
    }
    cudaFreeAsync(mx, H.stream);
    cudaError_t e = cudaStreamSynchronize(H.stream);
    if (rc == AMR_OK && e != cudaSuccess) rc = cuda_fail(e, "regrid");
    return rc;
}

void launch_remove_mean(Hierarchy &H, int which)
{
    cudaMemsetAsync(H.pmean, 0, sizeof(double), H.stream);
    for (int l = 0; l < H.nlev; ++l) {
        const Level &L = H.L[l];
        const double h = L.g.h;
        k_mean<<<rg_blocks(L.g.ncell), kRgThreads, 0, H.stream>>>(L.g.ncell, L.mask, which ? L.phi : L.rho,
                                                                  h * h * h, H.pmean);
    }
    for (int l = 0; l < H.nlev; ++l) {
        const Level &L = H.L[l];
        k_sub_mean<<<rg_blocks(L.g.ncell), kRgThreads, 0, H.stream>>>(L.g.ncell, L.mask, which ? L.phi : L.rho,
                                                                      H.pmean);
    }
}

int set_gather_buffer(Hierarchy &H, int b)
{
    if (b == 0) {
        H.gather_buffer = 0;
        return AMR_OK;
    }
    // every level's eroded mask first; the buffer takes effect only once all
    // are built, so a failure leaves the previous setting in force
    for (int l = 1; l < H.nlev; ++l) {
        Level &L = H.L[l];
        if (!L.gmask) {
            if (cudaMallocAsync((void **)&L.gmask, (size_t)L.g.ncell, H.stream) != cudaSuccess) {
                cudaGetLastError();
                L.gmask = nullptr;
                set_error("out of memory");
                return AMR_ENOMEM;
            }
            H.allocs.push_back(L.gmask);
            H.device_bytes += L.g.ncell;
        }
    }
    // a previous buffer's masks are rebuilt in place: stream order keeps
    // gathers issued earlier on the old ones
    for (int l = 1; l < H.nlev; ++l) {
        Level &L = H.L[l];
        k_erode<<<rg_blocks(L.g.ncell), kRgThreads, 0, H.stream>>>(L.g, L.mask, b, L.gmask);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gather buffer");
    H.gather_buffer = b;
    return AMR_OK;
}

int transfer_phi(const Hierarchy &S, Hierarchy &D)
{
    for (int l = 0; l < D.nlev; ++l) {
        TransferA A{};
        A.gd = D.L[l].g;
        A.md = D.L[l].mask;
        A.phid = D.L[l].phi;
        A.has_src = l < S.nlev;
        if (A.has_src) {
            A.gs = S.L[l].g;
            A.ms = S.L[l].mask;
            A.phis = S.L[l].phi;
        }
        A.has_parent = l > 0;
        if (A.has_parent) {
            A.gp = D.L[l - 1].g;
            A.phip = D.L[l - 1].phi;
        }
        k_transfer_phi<<<rg_blocks(A.gd.ncell), kRgThreads, 0, D.stream>>>(A);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMR_OK : cuda_fail(e, "phi transfer");
}

} // namespace amr

extern "C" {

int amr_regrid_boxes(amr_hierarchy *h, int policy, double lambda, int buffer_cells, int max_level, int *boxes_host,
                     int cap, int *n_boxes_out)
{
    amr::set_error("");
    if (!h || !n_boxes_out || (cap > 0 && !boxes_host) || cap < 0 || buffer_cells < 0 || max_level < 0 ||
        max_level >= AMR_MAX_LEVELS || !std::isfinite(lambda) ||
        (policy != AMR_TAG_REL_RHO && policy != AMR_TAG_ABS_RHO && policy != AMR_TAG_PHI &&
         policy != AMR_TAG_EFIELD)) {
        amr::set_error("invalid regrid arguments");
        return AMR_EINVAL;
    }
    std::vector<int> boxes;
    int rc = amr::regrid_boxes(*h->H, policy, lambda, buffer_cells, max_level, boxes);
    if (rc != AMR_OK) return rc;
    const int n = (int)(boxes.size() / 7);
    *n_boxes_out = n;
    if (n > cap) {
        amr::set_error("boxes_host holds " + std::to_string(cap) + " boxes, the regrid made " + std::to_string(n));
        return AMR_EINVAL;
    }
    std::copy(boxes.begin(), boxes.end(), boxes_host);
    return AMR_OK;
}

int amr_set_gather_buffer(amr_hierarchy *h, int buffer_cells)
{
    amr::set_error("");
    if (!h || buffer_cells < 0 || buffer_cells > 8) {
        amr::set_error("gather buffer must be 0..8 cells");
        return AMR_EINVAL;
    }
    return amr::set_gather_buffer(*h->H, buffer_cells);
}

int amr_transfer_phi(const amr_hierarchy *src, amr_hierarchy *dst)
{
    amr::set_error("");
    if (!src || !dst || src->H->n0 != dst->H->n0) {
        amr::set_error("transfer needs two hierarchies with the same base grid");
        return AMR_EINVAL;
    }
    if (src->H->stream != dst->H->stream) cudaStreamSynchronize(src->H->stream);
    return amr::transfer_phi(*src->H, *dst->H);
}

} // extern "C"
