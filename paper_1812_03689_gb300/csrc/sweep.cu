// Fused red-black Gauss-Seidel sweep: both colours of one sweep in a single
// launch, staged through shared memory.
//
// A block owns a TX x TY column tile of the padded box and a chunk of zc
// interior planes, and marches through the chunk plane by plane (2.5-D
// blocking).  Plane t of the iterate is kept in a ring of five
// shared-memory slots with a two-cell halo in x and y, and plane t of the
// right-hand side and of the neighbour codes in rings of three slots with a
// one-cell halo.  Load offsets and cell indices are computed once per block
// (the colour parity of a plane is one XOR).  Per plane t the block
//   - relaxes the red cells of plane t over the tile plus a one-cell halo
//     (the halo reds are recomputed, not exchanged: their black neighbours
//     are in the two-cell halo), then
//   - relaxes the black cells of plane t-1 over the tile (all their red
//     neighbours, planes t-2 .. t, are now new), and writes plane t-1 of the
//     tile, both colours, to global memory,
// while the loads of plane t+2 are in flight in registers.  Global traffic
// per sweep is one read of the iterate, the right-hand side and the code
// and one write of the iterate (plus the halo re-reads, which mostly hit
// L2), against two reads and one write per colour for per-colour passes.
//
// The sweep is out of place: it reads the previous iterate from x_in and
// writes the new one to x_out.  In place, a block's recomputed halo reds
// would read black cells that the neighbouring block may already have
// overwritten.  Each cell's update is the expression of the per-colour
// passes with the same summation tree (stencil.cuh), so a fused sweep and
// a red pass followed by a black pass give bitwise identical iterates.
//
// Cells are classified by their neighbour codes (Grid::code: which of the
// six neighbours and whether the cell itself are valid), so the codes need
// only the one-cell halo of the red region, and out-of-box cells (code 0)
// are never relaxed or written.  A coarse-fine face reads the cell opposite
// the face, which for levels l >= 1 (unions of refined coarse cells, at
// least two fine cells wide) is always a valid cell of the level.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "amr_internal.h"
#include "stencil.cuh"

namespace amr {

namespace {

constexpr int kSwThreads = 256;

template <typename T>
struct SweepA {
    Grid g;
    const T *xin; // previous iterate (unused for a sweep from zero)
    T *xout;      // new iterate
    const T *rhs;
    int mode;     // 1: e += x and phi += x; 2: phi += x (new values)
    T *e, *phi;
    int zc;       // interior planes per block
    const unsigned *list; // active blocks (null: the whole grid)
};

template <typename T, int TX, int TY>
struct SweepShape {
    static constexpr int RX = TX + 4, RY = TY + 4; // iterate planes (two-cell halo)
    static constexpr int PX = RX * RY;
    static constexpr int QX = TX + 2, QY = TY + 2; // rhs and code planes, red region
    static constexpr int PQ = QX * QY;
    static constexpr int NXS = 5, NQS = 3;         // ring slots
    static constexpr int LX = (PX + kSwThreads - 1) / kSwThreads;
    static constexpr int LQ = (PQ + kSwThreads - 1) / kSwThreads;
    static constexpr int NRED = (QX / 2) * QY;     // red cells of the red region
    static constexpr int NR = (NRED + kSwThreads - 1) / kSwThreads;
    static constexpr int NBLK = (TX / 2) * TY;     // black cells of the tile
    static constexpr int NB = (NBLK + kSwThreads - 1) / kSwThreads;
    static constexpr size_t smem = sizeof(T) * ((size_t)NXS * PX + (size_t)NQS * PQ) + (size_t)NQS * PQ;
    static_assert(TX % 2 == 0, "tile width must be even");
};

// S and k of one cell from shared memory: iterate planes Xm, X0, Xp (row
// length rx, cell index i) and the cell's neighbour code cd.
template <typename T>
__device__ __forceinline__ void smem_stencil(const T *Xm, const T *X0, const T *Xp, int i, int rx, unsigned cd,
                                             int dirichlet, T &S, int &k)
{
    T v[6] = {X0[i - 1], X0[i + 1], X0[i - rx], X0[i + rx], Xm[i], Xp[i]};
    if ((cd & 63u) == 63u) {
        k = 18;
        S = sum6(v[0], v[1], v[2], v[3], v[4], v[5]);
        return;
    }
    int kk = 0;
    T c[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        bool valid = (cd >> f) & 1u;
        c[f] = face_c(valid, (uint8_t)valid, dirichlet, v[f], v[f ^ 1], kk);
    }
    S = sum6(c[0], c[1], c[2], c[3], c[4], c[5]);
    k = kk;
}

template <typename T, int TX, int TY, bool FIRST>
__global__ void __launch_bounds__(kSwThreads) k_sweep(const __grid_constant__ SweepA<T> A)
{
    using Sh = SweepShape<T, TX, TY>;
    constexpr int RX = Sh::RX, PX = Sh::PX, QX = Sh::QX, PQ = Sh::PQ;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *xs = reinterpret_cast<T *>(sm_raw);
    T *bs = xs + Sh::NXS * PX;
    uint8_t *cs = reinterpret_cast<uint8_t *>(bs + Sh::NQS * PQ);

    const Grid &g = A.g;
    const int tid = threadIdx.x;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const int64_t sz = g.sz;
    const int sy = (int)g.sy;
    int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    if (A.list) {
        unsigned w = A.list[blockIdx.x];
        bx = (int)(w & 2047u);
        by = (int)((w >> 11) & 2047u);
        bz = (int)(w >> 22);
    }
    const int ax0 = 1 + bx * TX, by0 = 1 + by * TY;
    const int c0 = 1 + bz * A.zc;
    const int c1 = min(c0 + A.zc, n2 - 1); // planes [c0, c1) are this block's
    const int base = g.lo[0] + g.lo[1] + g.lo[2] - 3;
    const T h2 = gh2<T>(g);
    const int dir = g.dirichlet;
    const int mode = A.mode;

    // in-plane offsets of this thread's loads (-1: outside the box)
    int xoff[Sh::LX], qoff[Sh::LQ];
#pragma unroll
    for (int q = 0; q < Sh::LX; ++q) {
        int r = tid + q * kSwThreads;
        int ry = r / RX, rx = r - ry * RX;
        int a = ax0 - 2 + rx, b = by0 - 2 + ry;
        xoff[q] = (r < PX && a >= 0 && a < n0 && b >= 0 && b < n1) ? b * sy + a : -1;
    }
#pragma unroll
    for (int q = 0; q < Sh::LQ; ++q) {
        int r = tid + q * kSwThreads;
        int qy = r / QX, qx = r - qy * QX;
        int a = ax0 - 1 + qx, b = by0 - 1 + qy;
        qoff[q] = (r < PQ && a >= 0 && a < n0 && b >= 0 && b < n1) ? b * sy + a : -1;
    }
    // red cells of the red region (row qy, pair kx) and black cells of the
    // tile (row ty, pair kx): indices at parity 0 and the row's parity
    int rib[Sh::NR], rqb[Sh::NR], rpar[Sh::NR];
#pragma unroll
    for (int q = 0; q < Sh::NR; ++q) {
        int j = tid + q * kSwThreads;
        int qy = j / (QX / 2), kx = j - qy * (QX / 2);
        rib[q] = (qy + 1) * RX + 1 + 2 * kx;
        rqb[q] = qy * QX + 2 * kx;
        rpar[q] = j < Sh::NRED ? ((base + ax0 - 1 + by0 - 1 + qy) & 1) : -1;
    }
    int bib[Sh::NB], bqb[Sh::NB], bgo[Sh::NB], bpar[Sh::NB];
#pragma unroll
    for (int q = 0; q < Sh::NB; ++q) {
        int j = tid + q * kSwThreads;
        int ty = j / (TX / 2), kx = j - ty * (TX / 2);
        bib[q] = (ty + 2) * RX + 2 + 2 * kx;
        bqb[q] = (ty + 1) * QX + 1 + 2 * kx;
        bgo[q] = (by0 + ty) * sy + ax0 + 2 * kx;
        bpar[q] = j < Sh::NBLK ? ((base + ax0 + by0 + ty + 1) & 1) : -1;
    }

    T xr[Sh::LX];
    T br[Sh::LQ];
    unsigned cr[Sh::LQ];
    // per-plane base pointers: the in-plane offsets stay 32-bit
    auto fetch_x = [&](int c) {
        const bool cin = c >= 0 && c < n2;
        const T *xc = A.xin + (cin ? (int64_t)c * sz : 0);
#pragma unroll
        for (int q = 0; q < Sh::LX; ++q) xr[q] = (!FIRST && cin && xoff[q] >= 0) ? xc[xoff[q]] : T(0);
    };
    auto fetch_q = [&](int c) {
        const bool cin = c >= 0 && c < n2;
        const int64_t pc = cin ? (int64_t)c * sz : 0;
        const T *bc = A.rhs + pc;
        const uint8_t *kc = g.code + pc;
#pragma unroll
        for (int q = 0; q < Sh::LQ; ++q) {
            bool in = cin && qoff[q] >= 0;
            br[q] = in ? bc[qoff[q]] : T(0);
            cr[q] = in ? (unsigned)kc[qoff[q]] : 0u;
        }
    };
    auto store_x = [&](int slot) {
#pragma unroll
        for (int q = 0; q < Sh::LX; ++q) {
            int r = tid + q * kSwThreads;
            if (r < PX) xs[slot * PX + r] = xr[q];
        }
    };
    auto store_q = [&](int slot) {
#pragma unroll
        for (int q = 0; q < Sh::LQ; ++q) {
            int r = tid + q * kSwThreads;
            if (r < PQ) {
                bs[slot * PQ + r] = br[q];
                cs[slot * PQ + r] = (uint8_t)cr[q];
            }
        }
    };

    // prologue: planes c0-2 and c0-1 staged; plane c0 and rhs/codes of
    // plane c0-1 in flight
    const int t0 = c0 - 1;
    int sx_m2 = 0, sx_m1 = 1, sx_0 = 2, sx_p1 = 3, sx_p2 = 4; // iterate slots of planes t-2 .. t+2
    int sq_m1 = 0, sq_0 = 1, sq_p1 = 2;                       // rhs/code slots of planes t-1 .. t+1
    fetch_x(t0 - 1);
    store_x(sx_m1);
    fetch_x(t0);
    store_x(sx_0);
    fetch_x(t0 + 1);
    fetch_q(t0);

    for (int t = t0; t <= c1; ++t) {
        store_x(sx_p1);
        store_q(sq_0);
        __syncthreads();
        if (t < c1) {
            fetch_x(t + 2);
            fetch_q(t + 1);
        }
        // red cells of plane t over the tile plus a one-cell halo
        if (t >= 1 && t <= n2 - 2) {
            const T *Xm = xs + sx_m1 * PX, *Xp = xs + sx_p1 * PX;
            T *X0 = xs + sx_0 * PX;
            const T *B0 = bs + sq_0 * PQ;
            const uint8_t *C0 = cs + sq_0 * PQ;
#pragma unroll
            for (int q = 0; q < Sh::NR; ++q) {
                if (rpar[q] < 0) continue;
                int par = rpar[q] ^ (t & 1);
                unsigned cd = C0[rqb[q] + par];
                if (!(cd & 64u)) continue;
                int i = rib[q] + par;
                T S;
                int k;
                smem_stencil(Xm, X0, Xp, i, RX, cd, dir, S, k);
                X0[i] = gs_update(g, S, h2, B0[rqb[q] + par], k);
            }
        }
        __syncthreads();
        // black cells of plane t-1 over the tile; write plane t-1 out
        const int c = t - 1;
        if (c >= c0) {
            const T *Xm = xs + sx_m2 * PX, *X0 = xs + sx_m1 * PX, *Xp = xs + sx_0 * PX;
            const T *B0 = bs + sq_m1 * PQ;
            const uint8_t *C0 = cs + sq_m1 * PQ;
            const int64_t pc = (int64_t)c * sz;
            T *xo = A.xout + pc;
            T *eo = mode == 1 ? A.e + pc : nullptr;
            T *po = mode != 0 ? A.phi + pc : nullptr;
#pragma unroll
            for (int q = 0; q < Sh::NB; ++q) {
                if (bpar[q] < 0) continue;
                int par = bpar[q] ^ (c & 1); // black at pair offset par, red partner at 1 - par
                unsigned cb = C0[bqb[q] + par], cp = C0[bqb[q] + 1 - par];
                if (cb & 64u) {
                    int i = bib[q] + par;
                    T S;
                    int k;
                    smem_stencil(Xm, X0, Xp, i, RX, cb, dir, S, k);
                    T v = gs_update(g, S, h2, B0[bqb[q] + par], k);
                    const int p = bgo[q] + par;
                    xo[p] = v;
                    if (mode == 1) eo[p] += v;
                    if (mode != 0) po[p] += v;
                }
                if (cp & 64u) {
                    T v = X0[bib[q] + 1 - par];
                    const int p = bgo[q] + 1 - par;
                    xo[p] = v;
                    if (mode == 1) eo[p] += v;
                    if (mode != 0) po[p] += v;
                }
            }
        }
        // rotate the rings
        int s = sx_m2;
        sx_m2 = sx_m1;
        sx_m1 = sx_0;
        sx_0 = sx_p1;
        sx_p1 = sx_p2;
        sx_p2 = s;
        s = sq_m1;
        sq_m1 = sq_0;
        sq_0 = sq_p1;
        sq_p1 = s;
    }
}

// Tile shapes the autotuner chooses from (index = SweepTile::shape).
constexpr int kShapes = 5;
constexpr int kShapeTX[kShapes] = {32, 64, 32, 64, 32};
constexpr int kShapeTY[kShapes] = {8, 8, 16, 16, 32};

template <typename T, int TX, int TY, bool FIRST>
cudaError_t launch_shape(const SweepA<T> &A, dim3 grid, cudaStream_t s)
{
    using Sh = SweepShape<T, TX, TY>;
    auto fn = k_sweep<T, TX, TY, FIRST>;
    // the shared-memory limit is a per-device attribute of the function
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit);
    }
    fn<<<grid, kSwThreads, Sh::smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, bool FIRST>
cudaError_t launch_any(int shape, const SweepA<T> &A, dim3 grid, cudaStream_t s)
{
    switch (shape) {
    case 0: return launch_shape<T, 32, 8, FIRST>(A, grid, s);
    case 1: return launch_shape<T, 64, 8, FIRST>(A, grid, s);
    case 2: return launch_shape<T, 32, 16, FIRST>(A, grid, s);
    case 3: return launch_shape<T, 64, 16, FIRST>(A, grid, s);
    default: return launch_shape<T, 32, 32, FIRST>(A, grid, s);
    }
}

} // namespace

int sweep_num_shapes() { return kShapes; }

template <typename T>
void launch_sweep(Hierarchy &H, const Grid &g, const SweepTile &tile, const T *xin, T *xout, const T *b, int first,
                  int mode, T *e, T *phi)
{
    double cells = valid_cells(H, g);
    double bytes = ((first ? 2.0 : 3.0) * sizeof(T) + 1.0) * cells;
    if (mode == 1) bytes += 4.0 * sizeof(T) * cells;
    if (mode == 2) bytes += 2.0 * sizeof(T) * cells;
    // 8 flops (7 instructions) per red and per black update (a sweep from
    // zero: 3 flops, 2 instructions per red)
    Launch L(H, K_RBGS, bytes, (first ? 5.5 : 8.0) * cells, (first ? 4.5 : 7.0) * cells);
    SweepA<T> A{g, xin, xout, b, mode, e, phi, tile.zc, tile.list};
    int nx = g.n[0] - 2, ny = g.n[1] - 2, nz = g.n[2] - 2;
    int tx = kShapeTX[tile.shape], ty = kShapeTY[tile.shape];
    dim3 grid((unsigned)((nx + tx - 1) / tx), (unsigned)((ny + ty - 1) / ty), (unsigned)((nz + tile.zc - 1) / tile.zc));
    if (tile.list) grid = dim3((unsigned)tile.nlist);
    if (grid.x == 0) return;
    cudaError_t err = first ? launch_any<T, true>(tile.shape, A, grid, H.stream)
                            : launch_any<T, false>(tile.shape, A, grid, H.stream);
    if (err != cudaSuccess) cuda_fail(err, "fused sweep launch");
}

template void launch_sweep<double>(Hierarchy &, const Grid &, const SweepTile &, const double *, double *,
                                   const double *, int, int, double *, double *);
template void launch_sweep<float>(Hierarchy &, const Grid &, const SweepTile &, const float *, float *,
                                  const float *, int, int, float *, float *);

namespace {

// Autotuner cache: (precision, interior cells in half-octaves) -> shape.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, SweepTile> g_tune;
bool g_tune_file_read = false;

// AMR_SWEEP_TUNE_FILE=path keeps the tuned shapes across processes: lines
// "<bytes per value> <size class> <shape> <planes>" are read once per process
// and every newly tuned entry is appended, so a later run of the same
// program (a profiler run, say, whose own timings would be distorted) makes
// the same choices.  Called with g_tune_mu held.
const char *tune_file()
{
    const char *f = getenv("AMR_SWEEP_TUNE_FILE");
    return (f && *f) ? f : nullptr;
}

void tune_file_read_locked()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *fn = tune_file();
    if (!fn) return;
    FILE *fp = fopen(fn, "r");
    if (!fp) return;
    int t = 0, cls = 0, sh = 0, zc = 0;
    while (fscanf(fp, "%d %d %d %d", &t, &cls, &sh, &zc) == 4)
        if ((t == 4 || t == 8) && sh >= -1 && sh < kShapes && zc >= 0) g_tune[{t, cls}] = SweepTile{sh, zc};
    fclose(fp);
}

void tune_file_append_locked(int t, int cls, const SweepTile &v)
{
    const char *fn = tune_file();
    if (!fn) return;
    FILE *fp = fopen(fn, "a");
    if (!fp) return;
    fprintf(fp, "%d %d %d %d\n", t, cls, v.shape, v.zc);
    fclose(fp);
}

int size_class(const Grid &g)
{
    double cells = (double)(g.n[0] - 2) * (g.n[1] - 2) * (g.n[2] - 2);
    return (int)std::floor(2.0 * std::log2(std::max(cells, 1.0)));
}

// Which 8 x 8 x 2 blocks of a level's interior hold a valid cell (from the
// host mask).
struct Occupancy {
    int ox = 0, oy = 0, oz = 0;
    std::vector<uint8_t> b;
};

Occupancy occupancy(const Level &L)
{
    const Grid &g = L.g;
    const int nx = g.n[0] - 2, ny = g.n[1] - 2, nz = g.n[2] - 2;
    Occupancy O;
    O.ox = (nx + 7) / 8;
    O.oy = (ny + 7) / 8;
    O.oz = (nz + 1) / 2;
    O.b.assign((size_t)O.ox * O.oy * O.oz, 0);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            const uint8_t *row = L.hmask.data() + (size_t)((k + 1) * g.sz + (int64_t)(j + 1) * g.sy + 1);
            uint8_t *ob = O.b.data() + ((size_t)(k / 2) * O.oy + j / 8) * O.ox;
            for (int i = 0; i < nx; ++i)
                if (row[i]) ob[i / 8] = 1;
        }
    return O;
}

// Packed list of the blocks of tile (TX, TY, zc) that hold a valid cell;
// false when the grid exceeds the packing or when nearly every block is
// active (the full grid is launched then).
bool active_blocks(const Occupancy &O, const Grid &g, int TX, int TY, int zc, std::vector<unsigned> &out)
{
    const int nx = g.n[0] - 2, ny = g.n[1] - 2, nz = g.n[2] - 2;
    const int gx = (nx + TX - 1) / TX, gy = (ny + TY - 1) / TY, gz = (nz + zc - 1) / zc;
    out.clear();
    if (O.b.empty() || gx > 2048 || gy > 2048 || gz > 1024) return false;
    for (int bz = 0; bz < gz; ++bz) {
        const int z0 = bz * zc / 2, z1 = std::min(O.oz, (bz * zc + zc + 1) / 2);
        for (int by = 0; by < gy; ++by) {
            const int y0 = by * TY / 8, y1 = std::min(O.oy, (by * TY + TY + 7) / 8);
            for (int bx = 0; bx < gx; ++bx) {
                const int x0 = bx * TX / 8, x1 = std::min(O.ox, (bx * TX + TX + 7) / 8);
                bool any = false;
                for (int z = z0; z < z1 && !any; ++z)
                    for (int y = y0; y < y1 && !any; ++y)
                        for (int x = x0; x < x1 && !any; ++x) any = O.b[((size_t)z * O.oy + y) * O.ox + x] != 0;
                if (any) out.push_back((unsigned)bx | ((unsigned)by << 11) | ((unsigned)bz << 22));
            }
        }
    }
    return out.size() < (size_t)(0.9 * (double)gx * gy * gz);
}

// Mean time of `reps` sweeps of grid g with the candidate tile (shape < 0:
// two per-colour passes), after one untimed sweep.  The arrays hold zeros
// (right after creation), which the sweeps keep.
template <typename T>
float time_candidate(Hierarchy &H, const Grid &g, const SweepTile &c, T *x, const T *b, T *tmp, int reps,
                     cudaEvent_t e0, cudaEvent_t e1)
{
    auto one = [&]() {
        if (c.shape < 0) {
            launch_rbgs<T>(H, g, x, b, 0, 0, 0, nullptr, nullptr);
            launch_rbgs<T>(H, g, x, b, 1, 0, 0, nullptr, nullptr);
        } else {
            launch_sweep<T>(H, g, c, x, tmp, b, 0, 0, nullptr, nullptr);
        }
    };
    one();
    cudaEventRecord(e0, H.stream);
    for (int r = 0; r < reps; ++r) one();
    cudaEventRecord(e1, H.stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / (float)reps;
}

template <typename T>
SweepTile tune_grid(Hierarchy &H, const Grid &g, const Occupancy *occ, T *x, const T *b, cudaEvent_t e0,
                    cudaEvent_t e1)
{
    const int nz = g.n[2] - 2;
    std::vector<SweepTile> cand;
    cand.push_back(SweepTile{-1, 0});
    const int zcs[4] = {2, 8, 32, nz};
    for (int s = 0; s < kShapes; ++s)
        for (int zc : zcs) {
            int z = std::max(1, std::min(zc, nz));
            bool dup = false;
            for (auto &q : cand) dup |= (q.shape == s && q.zc == z);
            if (!dup) cand.push_back(SweepTile{s, z});
        }
    T *tmp = reinterpret_cast<T *>(H.sweep_tmp);
    SweepTile best = cand[0];
    float best_ms = 1e30f;
    const char *lg = getenv("AMR_SWEEP_LOG");
    bool log = lg && lg[0] == '1';
    std::vector<unsigned> lst;
    for (auto &c : cand) {
        unsigned *dl = nullptr;
        if (c.shape >= 0 && occ && active_blocks(*occ, g, kShapeTX[c.shape], kShapeTY[c.shape], c.zc, lst)) {
            if (cudaMallocAsync((void **)&dl, sizeof(unsigned) * std::max<size_t>(lst.size(), 1), H.stream) ==
                cudaSuccess) {
                cudaMemcpyAsync(dl, lst.data(), sizeof(unsigned) * lst.size(), cudaMemcpyHostToDevice, H.stream);
                c.list = dl;
                c.nlist = (int)lst.size();
            } else {
                cudaGetLastError();
                dl = nullptr;
            }
        }
        float ms = time_candidate<T>(H, g, c, x, b, tmp, 3, e0, e1);
        if (dl) cudaFreeAsync(dl, H.stream);
        c.list = nullptr;
        c.nlist = 0;
        if (log)
            fprintf(stderr, "sweep-tune fp%d grid %dx%dx%d shape %d zc %d: %.4f ms\n", (int)(8 * sizeof(T)),
                    g.n[0] - 2, g.n[1] - 2, g.n[2] - 2, c.shape, c.zc, ms);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    if (log)
        fprintf(stderr, "sweep-tune fp%d grid %dx%dx%d -> shape %d zc %d\n", (int)(8 * sizeof(T)), g.n[0] - 2,
                g.n[1] - 2, g.n[2] - 2, best.shape, best.zc);
    return best;
}

// AMR_SWEEP=colour forces per-colour passes, AMR_SWEEP=fused:<shape>:<zc>
// one fused shape; anything else (default) tunes (or reuses the tune file).
// AMR_SWEEP_LOG=1 prints every timed candidate to stderr.
bool forced_tile(SweepTile &t)
{
    const char *s = getenv("AMR_SWEEP");
    if (!s || !*s || !strcmp(s, "auto")) return false;
    if (!strcmp(s, "colour")) {
        t = SweepTile{-1, 0};
        return true;
    }
    int sh = 0, zc = 0;
    if (sscanf(s, "fused:%d:%d", &sh, &zc) == 2 && sh >= 0 && sh < kShapes && zc > 0) {
        t = SweepTile{sh, zc};
        return true;
    }
    return false;
}

// Device copy of a block list, owned by the hierarchy.
unsigned *dalloc_list(Hierarchy &H, const std::vector<unsigned> &v)
{
    void *p = nullptr;
    size_t bytes = sizeof(unsigned) * std::max<size_t>(v.size(), 1);
    if (cudaMallocAsync(&p, bytes, H.stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemcpyAsync(p, v.data(), sizeof(unsigned) * v.size(), cudaMemcpyHostToDevice, H.stream);
    H.allocs.push_back(p);
    H.device_bytes += (int64_t)bytes;
    return (unsigned *)p;
}

template <typename T>
int tune_all(Hierarchy &H)
{
    SweepTile forced;
    bool force = forced_tile(forced);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // choose (shape, zc), then attach the grid's active-block list
    auto pick = [&](const Grid &g, const Occupancy *occ, SweepTile &out, T *x, const T *b) {
        if (g.periodic) { // the fused sweep's tiles read the ring, not the periodic images
            out = SweepTile{};
            return;
        }
        bool found = false;
        if (force) {
            out = forced;
            found = true;
        } else {
            std::pair<int, int> key{(int)sizeof(T), size_class(g)};
            std::lock_guard<std::mutex> lk(g_tune_mu);
            tune_file_read_locked();
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                out = it->second;
                found = true;
            }
        }
        if (!found) {
            if (!e0) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
            }
            out = tune_grid<T>(H, g, occ, x, b, e0, e1);
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[{(int)sizeof(T), size_class(g)}] = out;
            tune_file_append_locked((int)sizeof(T), size_class(g), out);
        }
        out.zc = std::max(1, std::min(out.zc, g.n[2] - 2));
        out.list = nullptr;
        out.nlist = 0;
        std::vector<unsigned> lst;
        if (out.shape >= 0 && occ && active_blocks(*occ, g, kShapeTX[out.shape], kShapeTY[out.shape], out.zc, lst)) {
            unsigned *dl = dalloc_list(H, lst);
            if (dl) {
                out.list = dl;
                out.nlist = (int)lst.size();
            }
        }
    };
    for (int l = 1; l < H.nlev; ++l) {
        Fields<T> f = fields<T>(H.L[l]);
        Occupancy occ = occupancy(H.L[l]);
        pick(H.L[l].g, &occ, H.L[l].sw, f.err, f.res);
    }
    // (the multigrid grids are smoothed only when the bottom is not solved
    // exactly)
    for (int q = 0; q < H.nmg - 1 && !H.dst_on; ++q)
        pick(H.mg[q].g, nullptr, H.mg[q].sw, mg_e<T>(H.mg[q]), mg_r<T>(H.mg[q]));
    if (e0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaError_t e = cudaStreamSynchronize(H.stream);
    return e == cudaSuccess ? AMR_OK : cuda_fail(e, "sweep autotune");
}

} // namespace

int autotune_sweeps(Hierarchy &H)
{
    if (!H.sweep_tmp) return AMR_OK;
    return H.precision == AMR_MIXED ? tune_all<float>(H) : tune_all<double>(H);
}

} // namespace amr
