// Host side of hierarchy creation: tagging and bricks (Sec. 4.2, Eq.
// tag_charge), proper nesting (Sec. 3, Fig. amr), coarse-fine ghost tables
// with the pattern selection of Sec. 5.1 (Tab. bit_pattern, Tab.
// Lagrange_2d_linear), the level-0 multigrid grids, and device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "amr_internal.h"

namespace amr {

// Two-cell proper-nesting margin: the footprint of level l+1 grown by two
// cells of level l lies inside the domain and inside level l.  It keeps
// every uncovered cell of level l from lying between a face that leaves
// level l and a covered cell, and every 5x5 ghost surface of level l+1
// inside level l.
constexpr int kNest = 2;

namespace {

// ---------------------------------------------------------------- memory

// Stream-ordered allocation from the device's default pool (kept in the
// pool between hierarchies, so creating and destroying hierarchies does not
// synchronise the device under other streams' work).
void pool_setup()
{
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
}

template <typename T>
T *dalloc(Hierarchy &H, int64_t count)
{
    if (count <= 0) count = 1;
    void *p = nullptr;
    size_t bytes = sizeof(T) * (size_t)count;
    if (H.max_bytes > 0 && H.device_bytes + (int64_t)bytes > H.max_bytes) {
        H.over_limit = true; // the caller's cap (amr_desc.max_device_bytes)
        return nullptr;
    }
    pool_setup();
    if (cudaMallocAsync(&p, bytes, H.stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemsetAsync(p, 0, bytes, H.stream);
    H.allocs.push_back(p);
    H.device_bytes += (int64_t)bytes;
    return (T *)p;
}

template <typename T>
T *upload(Hierarchy &H, const std::vector<T> &v)
{
    T *d = dalloc<T>(H, (int64_t)v.size());
    if (d && !v.empty()) cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, H.stream);
    return d;
}

Grid make_grid(const int vlo[3], const int vhi[3], double h, int dirichlet)
{
    Grid g{};
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = vlo[d];
        g.n[d] = vhi[d] - vlo[d] + 3;
    }
    g.sy = g.n[0];
    g.sz = (int64_t)g.n[0] * g.n[1];
    g.ncell = g.sz * g.n[2];
    g.h = h;
    g.h2 = h * h;
    g.ih2 = 1.0 / (h * h);
    g.h2f = (float)g.h2;
    g.ih2f = (float)g.ih2;
    g.dirichlet = dirichlet ? 6 : 0; // Robin and periodic grids are switched later
    g.periodic = 0;
    g.robin = nullptr;
    return g;
}

int64_t hidx(const Grid &g, int i, int j, int k)
{
    int a = i - g.lo[0] + 1, b = j - g.lo[1] + 1, c = k - g.lo[2] + 1;
    if (a < 0 || b < 0 || c < 0 || a >= g.n[0] || b >= g.n[1] || c >= g.n[2]) return -1;
    return (int64_t)c * g.sz + (int64_t)b * g.sy + a;
}

uint8_t hmask_at(const Level &L, int i, int j, int k)
{
    int64_t p = hidx(L.g, i, j, k);
    return p < 0 ? 0 : L.hmask[p];
}

// Allocate the device arrays of a level whose host mask is final.
int alloc_level(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    int64_t n = L.g.ncell;
    L.mask = dalloc<uint8_t>(H, n);
    L.rho = dalloc<double>(H, n);
    L.phi = dalloc<double>(H, n);
    L.res = dalloc<double>(H, n);
    L.err = dalloc<double>(H, n);
    L.phisave = dalloc<double>(H, n);
    L.de = dalloc<double>(H, n);
    for (int d = 0; d < 3; ++d) L.ef[d] = dalloc<double>(H, n);
    if (!L.mask || !L.rho || !L.phi || !L.res || !L.err || !L.phisave || !L.de || !L.ef[0] || !L.ef[1] ||
        !L.ef[2])
        return AMR_ENOMEM;
    if (H.precision == AMR_MIXED) {
        L.rho32 = dalloc<float>(H, n);
        L.phi32 = dalloc<float>(H, n);
        L.res32 = dalloc<float>(H, n);
        L.err32 = dalloc<float>(H, n);
        L.de32 = dalloc<float>(H, n);
        if (!L.rho32 || !L.phi32 || !L.res32 || !L.err32 || !L.de32) return AMR_ENOMEM;
    }
    L.g.mask = L.mask;
    return AMR_OK;
}

// Valid interior cells of refined level l as padded indices, those of
// colour 0 (red: global i + j + k even) first.  The colour passes then run
// one thread per valid cell: a refined level's box is often less than half
// valid, and an FP64 instruction costs a warp the same pipe time whatever
// the number of its lanes that have a cell.  AMR_CELL_LISTS=0 keeps the
// passes on the whole box (the same bits either way).
int build_cell_list(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    Grid &g = L.g;
    const char *env = getenv("AMR_CELL_LISTS");
    if ((env && env[0] == '0') || g.ncell >= (int64_t)INT32_MAX) return AMR_OK;
    std::vector<int> lst[2];
    const int par0 = g.lo[0] + g.lo[1] + g.lo[2] - 3;
    for (int c = 1; c < g.n[2] - 1; ++c)
        for (int b = 1; b < g.n[1] - 1; ++b) {
            const int64_t row = (int64_t)c * g.sz + (int64_t)b * g.sy;
            for (int a = 1; a < g.n[0] - 1; ++a)
                if (L.hmask[row + a]) lst[(par0 + a + b + c) & 1].push_back((int)(row + a));
        }
    const size_t n0 = lst[0].size(), n1 = lst[1].size();
    int *d = dalloc<int>(H, (int64_t)std::max<size_t>(1, n0 + n1));
    if (!d) return AMR_ENOMEM;
    if (n0) cudaMemcpyAsync(d, lst[0].data(), sizeof(int) * n0, cudaMemcpyHostToDevice, H.stream);
    if (n1) cudaMemcpyAsync(d + n0, lst[1].data(), sizeof(int) * n1, cudaMemcpyHostToDevice, H.stream);
    g.clist = d;
    g.ccnt[0] = (int)n0;
    g.ccnt[1] = (int)n1;
    return AMR_OK;
}

// Covered cells (mask 2) of level l as padded indices in box order: the
// restriction from level l + 1 then runs one thread per covered cell
// instead of one per cell of level l + 1's footprint box, in which the
// covered cells come in runs of half a brick (partly filled warps would
// issue the FP64 work of their empty lanes all the same).
int build_cov_list(Hierarchy &H, int l)
{
    Level &L = H.L[l];
    const Grid &g = L.g;
    const char *env = getenv("AMR_CELL_LISTS");
    if ((env && env[0] == '0') || g.ncell >= (int64_t)INT32_MAX) return AMR_OK;
    std::vector<int> cov;
    for (int64_t p = 0; p < g.ncell; ++p)
        if (L.hmask[p] == 2) cov.push_back((int)p);
    if (cov.empty()) return AMR_OK;
    int *d = dalloc<int>(H, (int64_t)cov.size());
    if (!d) return AMR_ENOMEM;
    cudaMemcpyAsync(d, cov.data(), sizeof(int) * cov.size(), cudaMemcpyHostToDevice, H.stream);
    L.cov = d;
    L.ncov = (int)cov.size();
    return AMR_OK;
}

// ------------------------------------------------------- ghost patterns

// Sec. 5.1: bit patterns of the nine quadratic configurations (5x5
// surface, bit i + 5 j) and the four linear ones (3x3 surface, bit i + 3 j),
// in the order the paper tries them.
const uint32_t kQuad[9] = {473536u, 14798u, 236768u, 15153152u, 947072u, 29596u, 7399u, 7576576u, 30306304u};
const uint32_t kLin[4] = {27u, 216u, 432u, 54u};

struct Pattern {
    uint32_t bits;
    int oi, oj; // offset of the stencil's first node from the centre cell
    int m;      // nodes per axis
};

std::vector<Pattern> decode(const uint32_t *tab, int n, int w, int m)
{
    std::vector<Pattern> out;
    for (int c = 0; c < n; ++c) {
        int i0 = w, j0 = w;
        for (int b = 0; b < w * w; ++b)
            if (tab[c] >> b & 1u) {
                i0 = std::min(i0, b % w);
                j0 = std::min(j0, b / w);
            }
        out.push_back({tab[c], i0 - w / 2, j0 - w / 2, m});
    }
    return out;
}

// Lagrange weights of nodes o, o+1, ..., o+m-1 at t.
void lagrange(int o, int m, double t, double *w)
{
    for (int a = 0; a < m; ++a) {
        double num = 1.0, den = 1.0;
        for (int b = 0; b < m; ++b)
            if (b != a) {
                num *= t - (double)(o + b);
                den *= (double)(a - b);
            }
        w[a] = num / den;
    }
}

struct FaceEntry {
    int f, f1;
    int8_t dir, cnt;
    int c[kMaxStencil];
    double w[kMaxStencil];
    int C; // coarse cell across the face (padded index, level l-1)
};

// ------------------------------------------------------------- tagging

// Boxes of level l+1 from the charge density of level l: grown tags mark
// aligned bc^3 blocks of level l, kept under proper nesting.
std::vector<int> tag_boxes(const Hierarchy &H, int l, const std::vector<double> &rho, int mode, double lambda,
                           int buffer, int bc)
{
    const Level &L = H.L[l];
    const Grid &g = L.g;
    int nl = H.n0 << l;
    int nb = nl / bc;
    double mx = -INFINITY;
    for (int64_t p = 0; p < g.ncell; ++p)
        if (L.hmask[p]) mx = std::max(mx, rho[p]);
    std::vector<uint8_t> mark((size_t)nb * nb * nb, 0);
    for (int c = 1; c < g.n[2] - 1; ++c)
        for (int b = 1; b < g.n[1] - 1; ++b)
            for (int a = 1; a < g.n[0] - 1; ++a) {
                int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
                if (!L.hmask[p]) continue;
                double v = rho[p] * H.eps0;
                bool t = (mode == AMR_TAG_ABS_RHO) ? (std::fabs(v) >= lambda) : (mx > 0.0 && rho[p] > lambda * mx);
                if (!t) continue;
                int i = g.lo[0] + a - 1, j = g.lo[1] + b - 1, k = g.lo[2] + c - 1;
                for (int dk = -buffer; dk <= buffer; ++dk)
                    for (int dj = -buffer; dj <= buffer; ++dj)
                        for (int di = -buffer; di <= buffer; ++di) {
                            int x = i + di, y = j + dj, z = k + dk;
                            if (x < 0 || y < 0 || z < 0 || x >= nl || y >= nl || z >= nl) continue;
                            mark[((size_t)(z / bc) * nb + (y / bc)) * nb + (x / bc)] = 1;
                        }
            }
    std::vector<int> boxes;
    for (int bk = 0; bk < nb; ++bk)
        for (int bj = 0; bj < nb; ++bj)
            for (int bi = 0; bi < nb; ++bi) {
                if (!mark[((size_t)bk * nb + bj) * nb + bi]) continue;
                int lo[3] = {bi * bc, bj * bc, bk * bc};
                bool ok = true;
                for (int z = lo[2] - kNest; z < lo[2] + bc + kNest && ok; ++z)
                    for (int y = lo[1] - kNest; y < lo[1] + bc + kNest && ok; ++y)
                        for (int x = lo[0] - kNest; x < lo[0] + bc + kNest && ok; ++x)
                            if (x < 0 || y < 0 || z < 0 || x >= nl || y >= nl || z >= nl || !hmask_at(L, x, y, z))
                                ok = false;
                if (!ok) continue;
                for (int d = 0; d < 3; ++d) boxes.push_back(2 * lo[d]);
                for (int d = 0; d < 3; ++d) boxes.push_back(2 * lo[d] + 2 * bc - 1);
            }
    return boxes;
}

// Host mask of level l from its boxes (6 ints each); marks covered cells of
// level l-1 and checks alignment and nesting.
int build_level(Hierarchy &H, int l, const std::vector<int> &boxes)
{
    int nl = H.n0 << l;
    int nbox = (int)boxes.size() / 6;
    int vlo[3] = {1 << 30, 1 << 30, 1 << 30}, vhi[3] = {-1, -1, -1};
    for (int b = 0; b < nbox; ++b)
        for (int d = 0; d < 3; ++d) {
            int a = boxes[6 * b + d], e = boxes[6 * b + 3 + d];
            if (a < 0 || e >= nl || a > e || (a & 1) || !(e & 1)) {
                set_error("level " + std::to_string(l) + ": box " + std::to_string(b) +
                          " is outside the domain or not aligned to coarse cells");
                return AMR_ENESTING;
            }
            vlo[d] = std::min(vlo[d], a);
            vhi[d] = std::max(vhi[d], e);
        }
    Level &L = H.L[l];
    for (int d = 0; d < 3; ++d) {
        L.vlo[d] = vlo[d];
        L.vhi[d] = vhi[d];
    }
    L.g = make_grid(vlo, vhi, 1.0 / (double)nl, 0);
    if (L.g.ncell >= (int64_t)1 << 31) {
        set_error("level " + std::to_string(l) + " box exceeds 2^31 cells");
        return AMR_EINVAL;
    }
    L.hmask.assign((size_t)L.g.ncell, 0);
    for (int b = 0; b < nbox; ++b)
        for (int k = boxes[6 * b + 2]; k <= boxes[6 * b + 5]; ++k)
            for (int j = boxes[6 * b + 1]; j <= boxes[6 * b + 4]; ++j)
                for (int i = boxes[6 * b + 0]; i <= boxes[6 * b + 3]; ++i) L.hmask[hidx(L.g, i, j, k)] = 1;
    Level &C = H.L[l - 1];
    int nc = nl / 2;
    int64_t nvalid = 0;
    for (int64_t p = 0; p < L.g.ncell; ++p) nvalid += L.hmask[p] != 0;
    L.nvalid = nvalid;
    // every parent, grown by kNest, valid on level l-1 and in the domain
    for (int k = vlo[2] / 2; k <= vhi[2] / 2; ++k)
        for (int j = vlo[1] / 2; j <= vhi[1] / 2; ++j)
            for (int i = vlo[0] / 2; i <= vhi[0] / 2; ++i) {
                if (!hmask_at(L, 2 * i, 2 * j, 2 * k)) continue;
                for (int dk = -kNest; dk <= kNest; ++dk)
                    for (int dj = -kNest; dj <= kNest; ++dj)
                        for (int di = -kNest; di <= kNest; ++di) {
                            int x = i + di, y = j + dj, z = k + dk;
                            if (x < 0 || y < 0 || z < 0 || x >= nc || y >= nc || z >= nc || !hmask_at(C, x, y, z)) {
                                set_error("level " + std::to_string(l) + " is not properly nested in level " +
                                          std::to_string(l - 1));
                                return AMR_ENESTING;
                            }
                        }
                C.hmask[hidx(C.g, i, j, k)] = 2;
            }
    return AMR_OK;
}

// Coarse-fine face table of level l >= 1.
int build_cf(Hierarchy &H, int l)
{
    static std::vector<Pattern> quad = decode(kQuad, 9, 5, 3);
    static std::vector<Pattern> lin = decode(kLin, 4, 3, 2);
    Level &F = H.L[l], &C = H.L[l - 1];
    const Grid &g = F.g;
    int ncl = H.n0 << (l - 1);
    // step 2 weights: quadratic through the inward fine cell (-3/2 h_f), the
    // fine cell (-1/2 h_f) and the intermediate point (+h_f), at +1/2 h_f
    const double w_int = 8.0 / 15.0;
    std::vector<FaceEntry> faces;
    std::vector<int> cell_f, cell_ptr{0};
    const int64_t st[3] = {1, g.sy, g.sz};
    for (int c = 1; c < g.n[2] - 1; ++c)
        for (int b = 1; b < g.n[1] - 1; ++b)
            for (int a = 1; a < g.n[0] - 1; ++a) {
                int64_t p = (int64_t)c * g.sz + (int64_t)b * g.sy + a;
                if (!F.hmask[p]) continue;
                int fx[3] = {g.lo[0] + a - 1, g.lo[1] + b - 1, g.lo[2] + c - 1};
                int before = (int)faces.size();
                for (int d = 0; d < 3; ++d)
                    for (int s = -1; s <= 1; s += 2) {
                        int64_t q = p + s * st[d];
                        if (F.hmask[q]) continue;
                        FaceEntry e{};
                        e.f = (int)p;
                        e.f1 = (int)(p - s * st[d]);
                        if (!F.hmask[e.f1]) {
                            set_error("fine level one cell thick");
                            return AMR_ENESTING;
                        }
                        e.dir = (int8_t)(2 * d + (s > 0));
                        int Cc[3] = {fx[0] >> 1, fx[1] >> 1, fx[2] >> 1};
                        Cc[d] += s;
                        int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2; // transverse axes, increasing
                        double t0 = (fx[ta] & 1) ? 0.25 : -0.25, t1 = (fx[tb] & 1) ? 0.25 : -0.25;
                        auto avail = [&](int u, int v) {
                            int Q[3] = {Cc[0], Cc[1], Cc[2]};
                            Q[ta] += u;
                            Q[tb] += v;
                            if (Q[0] < 0 || Q[1] < 0 || Q[2] < 0 || Q[0] >= ncl || Q[1] >= ncl || Q[2] >= ncl)
                                return false;
                            return hmask_at(C, Q[0], Q[1], Q[2]) == 1;
                        };
                        auto cell_at = [&](int u, int v) {
                            int Q[3] = {Cc[0], Cc[1], Cc[2]};
                            Q[ta] += u;
                            Q[tb] += v;
                            return (int)hidx(C.g, Q[0], Q[1], Q[2]);
                        };
                        uint32_t m25 = 0;
                        for (int v = -2; v <= 2; ++v)
                            for (int u = -2; u <= 2; ++u)
                                if (avail(u, v)) m25 |= 1u << ((u + 2) + 5 * (v + 2));
                        uint32_t m9 = 0;
                        for (int v = -1; v <= 1; ++v)
                            for (int u = -1; u <= 1; ++u)
                                if (m25 >> ((u + 2) + 5 * (v + 2)) & 1u) m9 |= 1u << ((u + 1) + 3 * (v + 1));
                        const Pattern *pat = nullptr;
                        for (const Pattern &P : quad)
                            if ((m25 & P.bits) == P.bits) {
                                pat = &P;
                                break;
                            }
                        if (!pat)
                            for (const Pattern &P : lin)
                                if ((m9 & P.bits) == P.bits) {
                                    pat = &P;
                                    break;
                                }
                        if (pat) {
                            double wa[3], wb[3];
                            lagrange(pat->oi, pat->m, t0, wa);
                            lagrange(pat->oj, pat->m, t1, wb);
                            int n = 0;
                            for (int v = 0; v < pat->m; ++v)
                                for (int u = 0; u < pat->m; ++u) {
                                    e.c[n] = cell_at(pat->oi + u, pat->oj + v);
                                    e.w[n] = w_int * wa[u] * wb[v];
                                    ++n;
                                }
                            e.cnt = (int8_t)n;
                            F.cf.counts[pat->m == 3 ? 0 : 1]++;
                        } else {
                            e.c[0] = cell_at(0, 0);
                            e.w[0] = w_int;
                            e.cnt = 1;
                            F.cf.counts[2]++;
                        }
                        e.C = cell_at(0, 0);
                        for (int k2 = 0; k2 < e.cnt; ++k2)
                            if (e.c[k2] < 0) {
                                set_error("ghost stencil leaves the coarser level");
                                return AMR_ENESTING;
                            }
                        faces.push_back(e);
                    }
                if ((int)faces.size() > before) {
                    cell_f.push_back((int)p);
                    cell_ptr.push_back((int)faces.size());
                }
            }
    CfTable &T = F.cf;
    T.nface = (int)faces.size();
    T.ncell = (int)cell_f.size();
    std::vector<int> vf(T.nface), vf1(T.nface), vc((size_t)T.nface * kMaxStencil, 0);
    std::vector<int8_t> vdir(T.nface), vcnt(T.nface);
    std::vector<double> vw((size_t)T.nface * kMaxStencil, 0.0);
    std::map<int, std::vector<int>> by_coarse;
    for (int i = 0; i < T.nface; ++i) {
        const FaceEntry &e = faces[i];
        vf[i] = e.f;
        vf1[i] = e.f1;
        vdir[i] = e.dir;
        vcnt[i] = e.cnt;
        for (int k = 0; k < e.cnt; ++k) {
            vc[(size_t)i * kMaxStencil + k] = e.c[k];
            vw[(size_t)i * kMaxStencil + k] = e.w[k];
        }
        by_coarse[e.C].push_back(i);
    }
    std::vector<int> cc, cptr{0}, cface;
    for (auto &kv : by_coarse) {
        cc.push_back(kv.first);
        for (int i : kv.second) cface.push_back(i);
        cptr.push_back((int)cface.size());
    }
    T.ncrse = (int)cc.size();
    T.f = upload(H, vf);
    T.f1 = upload(H, vf1);
    T.dir = upload(H, vdir);
    T.cnt = upload(H, vcnt);
    T.cidx = upload(H, vc);
    T.cw = upload(H, vw);
    T.cell_f = upload(H, cell_f);
    T.cell_ptr = upload(H, cell_ptr);
    T.crse_c = upload(H, cc);
    T.crse_ptr = upload(H, cptr);
    T.crse_face = upload(H, cface);
    T.cp = dalloc<double>(H, T.nface);
    if (!T.f || !T.f1 || !T.dir || !T.cnt || !T.cidx || !T.cw || !T.cell_f || !T.cell_ptr || !T.crse_c ||
        !T.crse_ptr || !T.crse_face || !T.cp)
        return AMR_ENOMEM;
    return AMR_OK;
}

// Dense inverse of the m^3 7-point operator with h = 1 whose domain faces
// add bface to the diagonal (2 for the Dirichlet ghost -phi_0, 1 - alpha for
// the Robin ghost alpha phi_0), cached.  Periodic faces (bface < 0) couple
// to the opposite face instead; that operator is singular (constants), so
// the inverse is taken of A + 1 1^T, which maps a mean-free r to the
// mean-free solution of A e = r.
const std::vector<double> &coarse_inverse(int m, double bface)
{
    static std::mutex mu;
    static std::map<std::pair<int, double>, std::vector<double>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({m, bface});
    if (it != cache.end()) return it->second;
    const bool periodic = bface < 0.0;
    int N = m * m * m;
    std::vector<double> A((size_t)N * N, 0.0), X((size_t)N * N, 0.0);
    auto id = [m](int i, int j, int k) { return (k * m + j) * m + i; };
    for (int k = 0; k < m; ++k)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                int r = id(i, j, k);
                int c3[3] = {i, j, k};
                double diag = 0.0;
                for (int d = 0; d < 3; ++d)
                    for (int s = -1; s <= 1; s += 2) {
                        int q[3] = {c3[0], c3[1], c3[2]};
                        q[d] += s;
                        if ((q[d] < 0 || q[d] >= m) && !periodic)
                            diag += bface;
                        else {
                            q[d] = (q[d] + m) % m;
                            diag += 1.0;
                            A[(size_t)r * N + id(q[0], q[1], q[2])] -= 1.0;
                        }
                    }
                A[(size_t)r * N + r] += diag;
                X[(size_t)r * N + r] = 1.0;
            }
    if (periodic)
        for (size_t i = 0; i < (size_t)N * N; ++i) A[i] += 1.0;
    // Gauss-Jordan elimination (the matrix is symmetric positive definite,
    // so no pivoting is needed)
    for (int c = 0; c < N; ++c) {
        double inv = 1.0 / A[(size_t)c * N + c];
        for (int j = 0; j < N; ++j) {
            A[(size_t)c * N + j] *= inv;
            X[(size_t)c * N + j] *= inv;
        }
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            double f = A[(size_t)r * N + c];
            if (f == 0.0) continue;
            for (int j = 0; j < N; ++j) {
                A[(size_t)r * N + j] -= f * A[(size_t)c * N + j];
                X[(size_t)r * N + j] -= f * X[(size_t)c * N + j];
            }
        }
    }
    return cache[{m, bface}] = std::move(X);
}

// Ghost factor of a domain face on a grid of spacing h: phi_ghost = alpha
// phi_0; -1 for Dirichlet, (2d - h)/(2d + h) for Robin (Eq. robin_bc by
// central difference across the face).
double face_alpha(const Hierarchy &H, double h)
{
    if (H.robin_d <= 0.0) return -1.0;
    return (2.0 * H.robin_d - h) / (2.0 * H.robin_d + h);
}

// Switch a domain-face grid to Robin faces: its diagonal table for face
// codes k = base + 64 nb (nb Robin faces): D = base/3 + nb (1 - alpha).
int set_robin(Hierarchy &H, Grid &g)
{
    if (H.robin_d <= 0.0 || !g.dirichlet) return AMR_OK;
    std::vector<RobinTab> t(1);
    RobinTab &R = t[0];
    const double alpha = face_alpha(H, g.h);
    for (int k = 0; k < kRobinCodes; ++k) {
        const double D = (double)(k % kRobinFace) / 3.0 + (double)(k / kRobinFace) * (1.0 - alpha);
        R.D[k] = D;
        R.invD[k] = D > 0.0 ? 1.0 / D : 0.0;
        R.Df[k] = (float)D;
        R.invDf[k] = D > 0.0 ? (float)(1.0 / D) : 0.0f;
    }
    R.alpha = alpha;
    g.robin = upload(H, t);
    g.dirichlet = kRobinFace;
    return g.robin ? AMR_OK : AMR_ENOMEM;
}

// Largest coarsest multigrid extent solved with a dense inverse (order
// 11^3 = 1331); beyond it the coarsest grid is solved separably.
constexpr int kDenseCoarseMax = 11;

// Eigenvalues (ascending) and orthonormal eigenvectors (V[i n + m]: row i of
// eigenvector m) of a symmetric n x n matrix, by cyclic Jacobi rotations
// (Golub and Van Loan, Sec. 8.5): each rotation zeroes one off-diagonal
// pair; sweeps repeat until the off-diagonal mass is at rounding level.
void sym_eigen(int n, std::vector<double> A, std::vector<double> &V, std::vector<double> &lam)
{
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    double norm = 0.0;
    for (double x : A) norm += x * x;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a(p, q) * a(p, q);
        if (off <= 1e-32 * norm) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a(p, q);
                if (apq == 0.0) continue;
                const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) { // columns p, q
                    const double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - sn * akq;
                    a(k, q) = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { // rows p, q
                    const double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - sn * aqk;
                    a(q, k) = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    // ascending eigenvalues (the constant mode of periodic faces first)
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return a(x, x) < a(y, y); });
    std::vector<double> W((size_t)n * n);
    lam.assign(n, 0.0);
    for (int m = 0; m < n; ++m) {
        lam[m] = a(ord[m], ord[m]);
        for (int i = 0; i < n; ++i) W[(size_t)i * n + m] = V[(size_t)i * n + ord[m]];
    }
    V.swap(W);
}

int build_mg(Hierarchy &H)
{
    // grid 0 is level 0 itself; coarsen by 2 while the extent stays even
    // and above 8; the coarsest grid is solved with a dense inverse up to
    // 11^3 and separably beyond (n0 with a larger odd factor)
    H.nmg = 1;
    H.mg[0].g = H.L[0].g;
    H.mg[0].mask = H.L[0].mask;
    H.mg[0].e = H.L[0].err;
    H.mg[0].r = H.L[0].res;
    H.mg[0].e32 = H.L[0].err32;
    H.mg[0].r32 = H.L[0].res32;
    int n = H.n0;
    double h = 1.0 / H.n0;
    while (n % 2 == 0 && n > 8 && H.nmg < 16) {
        n /= 2;
        h *= 2.0;
        MgGrid &G = H.mg[H.nmg];
        int lo[3] = {0, 0, 0}, hi[3] = {n - 1, n - 1, n - 1};
        G.g = make_grid(lo, hi, h, 1);
        std::vector<uint8_t> m((size_t)G.g.ncell, 0);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) m[hidx(G.g, i, j, k)] = 1;
        G.mask = upload(H, m);
        G.g.mask = G.mask;
        G.e = dalloc<double>(H, G.g.ncell);
        G.r = dalloc<double>(H, G.g.ncell);
        G.owns = true;
        if (!G.mask || !G.e || !G.r) return AMR_ENOMEM;
        if (H.precision == AMR_MIXED) {
            G.e32 = dalloc<float>(H, G.g.ncell);
            G.r32 = dalloc<float>(H, G.g.ncell);
            if (!G.e32 || !G.r32) return AMR_ENOMEM;
        }
        H.nmg++;
    }
    H.ncoarse = n * n * n;
    const double bface = H.periodic ? -1.0 : 1.0 - face_alpha(H, h);
    if (n > kDenseCoarseMax && !getenv("AMR_COARSE_DENSE")) {
        // n0 with a large odd factor leaves a coarsest grid too large for a
        // dense inverse (its order n^3 reaches 30,000 for n0 = 248): solve it
        // separably.  The operator is T (x) I (x) I + I (x) T (x) I +
        // I (x) I (x) T with the 1-D operator T (ends 1 + bface, or the wrap
        // of periodic faces), so with T = V diag(lam) V^T,
        // e = h^2 (V (x) V (x) V) diag(1 / (lam_i + lam_j + lam_k)) (V (x) V (x) V)^T r;
        // periodic faces add n^3 to mode (0, 0, 0) (the constant mode, lam = 0:
        // the inverse of A + 1 1^T, as in the dense case).
        std::vector<double> T((size_t)n * n, 0.0), V, lam;
        for (int i = 0; i < n; ++i) {
            double d = 0.0;
            for (int s = -1; s <= 1; s += 2) {
                int q = i + s;
                if (q < 0 || q >= n) {
                    if (H.periodic) {
                        q = (q + n) % n;
                        T[(size_t)i * n + q] -= 1.0;
                        d += 1.0;
                    } else {
                        d += bface;
                    }
                } else {
                    T[(size_t)i * n + q] -= 1.0;
                    d += 1.0;
                }
            }
            T[(size_t)i * n + i] += d;
        }
        sym_eigen(n, T, V, lam);
        std::vector<double> vt((size_t)n * n);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) vt[(size_t)a * n + b] = V[(size_t)b * n + a];
        H.csep_n = n;
        H.csep_zero_add = H.periodic ? (double)n * n * n : 0.0;
        H.csep_v = upload(H, V);    // inverse pass: out_c = sum_q V[c][q] in_q
        H.csep_vt = upload(H, vt);  // forward pass: out_m = sum_q V[q][m] in_q
        H.csep_lam = upload(H, lam);
        H.csep_tmp[0] = dalloc<double>(H, H.mg[H.nmg - 1].g.ncell);
        H.csep_tmp[1] = dalloc<double>(H, H.mg[H.nmg - 1].g.ncell);
        return (H.csep_v && H.csep_vt && H.csep_lam && H.csep_tmp[0] && H.csep_tmp[1]) ? AMR_OK : AMR_ENOMEM;
    }
    const std::vector<double> &inv = coarse_inverse(n, bface);
    std::vector<double> scaled(inv.size());
    for (size_t i = 0; i < inv.size(); ++i) scaled[i] = inv[i] * h * h;
    H.coarse_inv = upload(H, scaled);
    return H.coarse_inv ? AMR_OK : AMR_ENOMEM;
}

} // namespace

void free_hierarchy(Hierarchy *H)
{
    if (!H) return;
    if (H->stream) cudaStreamSynchronize(H->stream);
    for (SolveGraph &G : H->graphs)
        if (G.exec) cudaGraphExecDestroy(G.exec);
    program_free(H->prog);
    for (void *p : H->allocs) cudaFreeAsync(p, H->stream);
    if (H->stage) cudaFree(H->stage);
    cudaStreamSynchronize(H->stream);
    if (H->cstream) {
        cudaStreamSynchronize(H->cstream);
        cudaStreamDestroy(H->cstream);
    }
    for (cudaEvent_t e : H->cev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : H->evpool) cudaEventDestroy(e);
    if (H->params_host) cudaFreeHost(H->params_host);
    if (H->state_host) cudaFreeHost(H->state_host);
    group_free(*H);
    delete H;
}

bool dst_wanted(int n0, bool robin);
bool fdst_size(int n0);
int build_dst(Hierarchy &H);

int create_hierarchy(const amr_desc *d, const double *x, const double *y, const double *z, const double *q,
                     int64_t n, void *stream, Hierarchy **out)
{
    if (!d || !out) {
        set_error("null descriptor or output");
        return AMR_EINVAL;
    }
    int brick = d->brick > 0 ? d->brick : 8;
    if (d->n0 < 8 || d->max_level < 0 || d->max_level >= kMaxLevels || brick < 4 || (brick & 1) ||
        d->n0 % (brick / 2) || d->buffer_cells < 0 || (d->precision != AMR_FP64 && d->precision != AMR_MIXED)) {
        set_error("invalid descriptor (n0 >= 8, 0 <= max_level < 6, even brick >= 4 dividing 2*n0)");
        return AMR_EINVAL;
    }
    if ((d->bc != AMR_BC_DIRICHLET && d->bc != AMR_BC_ROBIN && d->bc != AMR_BC_PERIODIC) ||
        (d->bc == AMR_BC_ROBIN && !(d->robin_d > 0.0 && d->robin_d <= 1e300))) {
        set_error("invalid boundary condition (bc Dirichlet or Robin with a positive finite robin_d)");
        return AMR_EINVAL;
    }
    if (d->tag_mode == AMR_TAG_BOXES) {
        if (d->n_boxes < 0 || (d->n_boxes > 0 && !d->boxes_host)) {
            set_error("boxes missing");
            return AMR_EINVAL;
        }
    } else if (d->tag_mode == AMR_TAG_REL_RHO || d->tag_mode == AMR_TAG_ABS_RHO) {
        if (d->max_level > 0 && (n <= 0 || !x || !y || !z || !q)) {
            set_error("tagging needs particles");
            return AMR_EINVAL;
        }
    } else {
        set_error("unknown tag_mode");
        return AMR_EINVAL;
    }
    Hierarchy *H = new Hierarchy();
    H->n0 = d->n0;
    H->eps0 = d->eps0 > 0.0 ? d->eps0 : 1.0;
    H->robin_d = d->bc == AMR_BC_ROBIN ? d->robin_d : 0.0;
    H->periodic = d->bc == AMR_BC_PERIODIC;
    H->precision = d->precision;
    H->brick = brick;
    H->max_bytes = d->max_device_bytes > 0 ? d->max_device_bytes : 0;
    H->stream = (cudaStream_t)stream;
    const char *pdl = getenv("AMR_PDL");
    H->pdl = !(pdl && pdl[0] == '0');
    int rc = AMR_OK;
    auto fail = [&](int code) {
        if (code == AMR_ENOMEM && H->over_limit)
            set_error("the hierarchy would exceed amr_desc.max_device_bytes");
        free_hierarchy(H);
        return code;
    };
    // scratch first (the tagging deposits count particles outside level 0)
    H->partials = dalloc<double>(*H, (int64_t)kMaxLevels * 2 * 3 * kPartialBlocks);
    H->params = dalloc<SolveParams>(*H, 1);
    H->state = dalloc<SolveState>(*H, 1);
    H->outside = dalloc<int>(*H, 1);
    H->nc_counter = dalloc<int>(*H, 1);
    if (!H->partials || !H->params || !H->state || !H->outside || !H->nc_counter ||
        cudaMallocHost((void **)&H->params_host, sizeof(SolveParams)) != cudaSuccess ||
        cudaMallocHost((void **)&H->state_host, sizeof(SolveState)) != cudaSuccess) {
        set_error("out of memory");
        return fail(AMR_ENOMEM);
    }
    // level 0
    {
        Level &L = H->L[0];
        int lo[3] = {0, 0, 0}, hi[3] = {d->n0 - 1, d->n0 - 1, d->n0 - 1};
        for (int e = 0; e < 3; ++e) {
            L.vlo[e] = lo[e];
            L.vhi[e] = hi[e];
        }
        L.g = make_grid(lo, hi, 1.0 / d->n0, 1);
        L.hmask.assign((size_t)L.g.ncell, 0);
        for (int k = 0; k < d->n0; ++k)
            for (int j = 0; j < d->n0; ++j)
                for (int i = 0; i < d->n0; ++i) L.hmask[hidx(L.g, i, j, k)] = 1;
        L.nvalid = (int64_t)d->n0 * d->n0 * d->n0;
        if ((rc = alloc_level(*H, 0)) != AMR_OK) {
            set_error("out of memory");
            return fail(rc);
        }
        cudaMemcpyAsync(L.mask, L.hmask.data(), L.hmask.size(), cudaMemcpyHostToDevice, H->stream);
    }
    H->nlev = 1;
    for (int l = 1; l <= d->max_level; ++l) {
        std::vector<int> boxes;
        if (d->tag_mode == AMR_TAG_BOXES) {
            for (int b = 0; b < d->n_boxes; ++b)
                if (d->boxes_host[7 * b] == l)
                    for (int e = 1; e < 7; ++e) boxes.push_back(d->boxes_host[7 * b + e]);
        } else {
            Level &P = H->L[l - 1];
            cudaMemcpyAsync(P.mask, P.hmask.data(), P.hmask.size(), cudaMemcpyHostToDevice, H->stream);
            launch_fill<double>(*H, P.rho, 0.0, P.g.ncell);
            launch_deposit(*H, x, y, z, q, n, l - 1);
            std::vector<double> rho((size_t)P.g.ncell);
            cudaMemcpyAsync(rho.data(), P.rho, sizeof(double) * rho.size(), cudaMemcpyDeviceToHost, H->stream);
            cudaError_t e = cudaStreamSynchronize(H->stream);
            if (e != cudaSuccess) return fail(cuda_fail(e, "tagging deposit"));
            boxes = tag_boxes(*H, l - 1, rho, d->tag_mode, d->tag_lambda, d->buffer_cells, brick / 2);
        }
        if (boxes.empty()) break;
        if ((rc = build_level(*H, l, boxes)) != AMR_OK) return fail(rc);
        if ((rc = alloc_level(*H, l)) != AMR_OK) {
            set_error("out of memory");
            return fail(rc);
        }
        H->nlev = l + 1;
    }
    for (int l = 0; l < H->nlev; ++l) {
        Level &L = H->L[l];
        cudaMemcpyAsync(L.mask, L.hmask.data(), L.hmask.size(), cudaMemcpyHostToDevice, H->stream);
    }
    for (int l = 1; l < H->nlev; ++l)
        if ((rc = build_cf(*H, l)) != AMR_OK) {
            if (rc == AMR_ENOMEM) set_error("out of memory");
            return fail(rc);
        }
    if ((rc = build_mg(*H)) != AMR_OK) {
        set_error("out of memory");
        return fail(rc);
    }
    // neighbour codes of every level and multigrid grid (grid 0 = level 0)
    for (int l = 0; l < H->nlev; ++l) {
        Level &L = H->L[l];
        L.code = dalloc<uint8_t>(*H, L.g.ncell);
        if (!L.code) {
            set_error("out of memory");
            return fail(AMR_ENOMEM);
        }
        launch_make_code(*H, L.g, L.code);
        L.g.code = L.code;
        if (l >= 1 && (rc = build_cell_list(*H, l)) != AMR_OK) {
            set_error("out of memory");
            return fail(rc);
        }
        if (l + 1 < H->nlev && (rc = build_cov_list(*H, l)) != AMR_OK) {
            set_error("out of memory");
            return fail(rc);
        }
    }
    H->mg[0].code = H->L[0].code;
    H->mg[0].g.code = H->L[0].code;
    for (int q = 1; q < H->nmg; ++q) {
        MgGrid &G = H->mg[q];
        G.code = dalloc<uint8_t>(*H, G.g.ncell);
        if (!G.code) {
            set_error("out of memory");
            return fail(AMR_ENOMEM);
        }
        launch_make_code(*H, G.g, G.code);
        G.g.code = G.code;
    }
    // periodic domain faces: level 0 and the grids of its multigrid (every
    // face of a cell then counts as a neighbour: face code increment 3)
    if (H->periodic) {
        H->L[0].g.periodic = 1;
        H->L[0].g.dirichlet = 3;
        for (int q = 1; q < H->nmg; ++q) {
            H->mg[q].g.periodic = 1;
            H->mg[q].g.dirichlet = 3;
        }
        H->pmean = dalloc<double>(*H, 1);
        if (!H->pmean) {
            set_error("out of memory");
            return fail(AMR_ENOMEM);
        }
    }
    // Robin domain faces: level 0 and the grids of its multigrid
    if ((rc = set_robin(*H, H->L[0].g)) != AMR_OK) {
        set_error("out of memory");
        return fail(rc);
    }
    H->mg[0].g.dirichlet = H->L[0].g.dirichlet;
    H->mg[0].g.periodic = H->L[0].g.periodic;
    H->mg[0].g.robin = H->L[0].g.robin;
    for (int q = 1; q < H->nmg; ++q)
        if ((rc = set_robin(*H, H->mg[q].g)) != AMR_OK) {
            set_error("out of memory");
            return fail(rc);
        }
    if ((rc = build_dst(*H)) != AMR_OK) {
        set_error("out of memory");
        return fail(rc);
    }
    {
        // second iterate of the out-of-place fused sweeps: the largest grid
        int64_t big = 0;
        for (int l = 0; l < H->nlev; ++l) big = std::max(big, H->L[l].g.ncell);
        for (int q = 0; q < H->nmg; ++q) big = std::max(big, H->mg[q].g.ncell);
        H->sweep_tmp = dalloc<double>(*H, big);
        if (!H->sweep_tmp) {
            set_error("out of memory");
            return fail(AMR_ENOMEM);
        }
        if ((rc = autotune_sweeps(*H)) != AMR_OK) return fail(rc);
        H->mg_bottom = mg_bottom_grid(*H);
    }
    if (n > 0 && x && y && z && q) {
        for (int l = 0; l < H->nlev; ++l) launch_fill<double>(*H, H->L[l].rho, 0.0, H->L[l].g.ncell);
        cudaMemsetAsync(H->outside, 0, sizeof(int), H->stream);
        launch_deposit(*H, x, y, z, q, n, -1);
    }
    cudaError_t e = cudaStreamSynchronize(H->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "hierarchy creation"));
    *out = H;
    return AMR_OK;
}

// Level-0 exact bottom solve.  With n0 = 128 the transforms are the fast
// ones (2 log2 n0 FP64 operations per value against 3 n0 / 8 FMAs for the
// folded matrix transforms); for n0 <= 64 and a multiple of 4, the matrix
// transforms (at these sizes their FMA chains run faster than the fast
// transforms' 2 log2 n0 synchronised stages); otherwise the level-0
// geometric multigrid.  AMR_BOTTOM=mg turns the exact solve off;
// AMR_BOTTOM=matrix (or dst) keeps the matrix transforms up to n0 = 128;
// AMR_BOTTOM=fast takes the fast transforms for every power of two from 32
// to 128.
bool dst_wanted(int n0, bool not_dirichlet)
{
    if (not_dirichlet) return false; // the sine basis diagonalises Dirichlet faces only
    const char *s = getenv("AMR_BOTTOM");
    if (s && !strcmp(s, "mg")) return false;
    if (n0 % 4) return false; // the folded transforms need n0 = 4k
    if (s && (!strcmp(s, "dst") || !strcmp(s, "matrix"))) return n0 <= 128;
    return n0 <= 64 || fdst_size(n0);
}

bool fdst_size(int n0)
{
    const char *s = getenv("AMR_BOTTOM");
    if (s && (!strcmp(s, "dst") || !strcmp(s, "matrix"))) return false;
    const bool pow2 = n0 >= 32 && n0 <= 128 && (n0 & (n0 - 1)) == 0;
    if (s && !strcmp(s, "fast")) return pow2;
    return pow2 && n0 >= 128;
}

int build_dst(Hierarchy &H)
{
    const int n = H.n0;
    if (!dst_wanted(n, H.robin_d > 0.0 || H.periodic)) return AMR_OK;
    const double pi = 3.14159265358979323846;
    std::vector<double> S((size_t)n * n), mf((size_t)n * n), mi((size_t)n * n), lam(n);
    for (int m = 0; m < n; ++m) {
        double c = m < n - 1 ? std::sqrt(2.0 / n) : std::sqrt(1.0 / n);
        for (int i = 0; i < n; ++i) S[(size_t)m * n + i] = c * std::sin(pi * (m + 1) * (i + 0.5) / n);
        double s = std::sin(pi * (m + 1) / (2.0 * n));
        lam[m] = 4.0 * s * s;
    }
    // forward table by output slot j (even modes m = 2j first, then odd
    // modes m = 2(j - n/2) + 1): mf[i n + j] = S[m(j)][i]; inverse table
    // mi[m n + i] = S[m][i]
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const int m = j < n / 2 ? 2 * j : 2 * (j - n / 2) + 1;
            mf[(size_t)i * n + j] = S[(size_t)m * n + i];
            mi[(size_t)i * n + j] = S[(size_t)i * n + j];
        }
    // fast transforms: the split factors 1 / (2 cos(pi (2i+1) / (2M))),
    // i < M/2, of block sizes M = n, n/2, ..., 2 at offset n - M; and per
    // (kx, ky) mode the factor h^2 c_kx^2 c_ky^2 that the tridiagonal solve
    // applies in place of h^2 (the basis scales c_m of the four transforms,
    // which the fast transforms leave out)
    std::vector<double> tab((size_t)n - 1), fm((size_t)n * n);
    for (int M = n; M >= 2; M >>= 1)
        for (int i = 0; i < M / 2; ++i) tab[(size_t)(n - M) + i] = 0.5 / std::cos(pi * (2 * i + 1) / (2.0 * M));
    {
        const double h2 = H.L[0].g.h2;
        auto c2 = [&](int m) { return m < n - 1 ? 2.0 / n : 1.0 / n; };
        for (int ky = 0; ky < n; ++ky)
            for (int kx = 0; kx < n; ++kx) fm[(size_t)ky * n + kx] = h2 * c2(kx) * c2(ky);
    }
    // reciprocal pivots of the two half systems (symmetric part: last
    // diagonal - 1, antisymmetric part: + 1), [part][k][mode]
    const int nm = n * n, h = n / 2;
    std::vector<double> iw((size_t)2 * h * nm);
    for (int part = 0; part < 2; ++part)
        for (int q = 0; q < nm; ++q) {
            double mu = lam[q % n] + lam[q / n];
            double w = 0.0;
            for (int k = 0; k < h; ++k) {
                double d = mu + (k == 0 ? 3.0 : 2.0);
                if (k == h - 1) d += part == 0 ? -1.0 : 1.0;
                w = k == 0 ? d : d - 1.0 / w;
                iw[((size_t)part * h + k) * nm + q] = 1.0 / w;
            }
        }
    H.dst_a = dalloc<double>(H, H.L[0].g.ncell);
    H.dst_b = dalloc<double>(H, H.L[0].g.ncell);
    H.dst_mf = upload(H, mf);
    H.dst_mi = upload(H, mi);
    H.dst_iw = upload(H, iw);
    if (!H.dst_a || !H.dst_b || !H.dst_mf || !H.dst_mi || !H.dst_iw) return AMR_ENOMEM;
    if (fdst_size(n)) {
        H.dst_tab = upload(H, tab);
        H.dst_fm = upload(H, fm);
        if (!H.dst_tab || !H.dst_fm) return AMR_ENOMEM;
        H.dst_fast = true;
    }
    H.dst_on = true;
    return AMR_OK;
}

int64_t hierarchy_bytes_estimate(const amr_desc *d, double fill)
{
    // fields of a level: mask and neighbour code (1 B each) + 9 float64
    // arrays per padded cell
    // (+ 5 float32 arrays in mixed precision)
    const int64_t per_cell = 2 + 9 * 8 + (d->precision == AMR_MIXED ? 5 * 4 : 0);
    int64_t n0 = d->n0;
    double big = std::pow((double)(n0 + 2), 3.0);
    int64_t bytes = (n0 + 2) * (n0 + 2) * (n0 + 2) * per_cell;
    for (int l = 1; l <= d->max_level; ++l) {
        double cells = std::pow((double)(n0 << l), 3.0) * std::min(1.0, fill);
        bytes += (int64_t)(cells * per_cell * 1.3);
        big = std::max(big, cells * 1.3);
    }
    bytes += (int64_t)(big * 8.0); // second iterate of the fused sweeps
    if (dst_wanted(d->n0, d->bc != AMR_BC_DIRICHLET)) bytes += (int64_t)(3.0 * 8.0 * std::pow((double)(n0 + 2), 3.0)); // exact bottom
    bytes += (int64_t)kMaxLevels * 6 * kPartialBlocks * 8 + (16 << 20);
    return bytes;
}

} // namespace amr
