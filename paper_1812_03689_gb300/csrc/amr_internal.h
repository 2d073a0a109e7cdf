// Internal data structures of libamrmg (not part of the C ABI).
//
// Layout in HBM.  Every level l (and every coarsened grid of the level-0
// geometric multigrid) is a dense box: the bounding box of its valid cells
// plus a one-cell ring, x fastest.  Fields are separate float64 arrays over
// that padded box (structure of arrays, 8-byte aligned rows); a uint8 mask
// marks each cell as outside the level (0), valid and uncovered (1) or
// valid and covered by level l+1 (2).  The ring and the box cells outside
// the level hold no data: a neighbour with mask 0 is the physical boundary
// on level 0 (Dirichlet ghost) and a coarse-fine face on finer levels.
//
// Coarse-fine faces of level l >= 1 are a compact table (structure of
// arrays), one entry per (fine cell, face) whose neighbour lies outside
// level l, sorted by fine cell; each entry holds the fine cell, its inward
// neighbour and the step-1 coarse stencil (up to 9 cells of level l-1, with
// the weights already multiplied by the step-2 weight 8/15).  Two index
// lists over that table drive the kernels deterministically, one thread per
// cell: by fine cell (fine-side corrections) and by coarse cell (the
// flux-matched coarse rows).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/amrmg.h"

namespace amr {

constexpr int kMaxLevels = AMR_MAX_LEVELS;
constexpr int kStepChunks = 8; // particle chunks of amr_step's copy pipeline
constexpr int kMaxStencil = 9;

// Diagonal of the level operator for cells with Robin faces (Eq. robin_bc,
// d phi/dn + phi/d = 0 by central difference: ghost alpha phi_0 with
// alpha = (2d - h)/(2d + h)), indexed by the face code k of the stencil
// split (k = 3 per valid neighbour, 1 per coarse-fine face, 64 per Robin
// face): D = (k mod 64)/3 + (k / 64)(1 - alpha) and 1/D, for one grid.
constexpr int kRobinFace = 64;
constexpr int kRobinCodes = 3 * kRobinFace + 37;
struct RobinTab {
    double D[kRobinCodes], invD[kRobinCodes];
    float Df[kRobinCodes], invDf[kRobinCodes];
    double alpha;
};

// Device view of one dense level box (passed to kernels by value).
struct Grid {
    int lo[3];      // global index of the first valid-box cell (ring excluded)
    int n[3];       // padded extent (valid box + 2)
    int64_t sy, sz; // strides of j and k in the padded box
    int64_t ncell;  // padded cell count
    double h, h2, ih2;
    float h2f, ih2f; // h2 and ih2 rounded to FP32 (the FP32 operations' copies)
    // face code increment of a mask-0 neighbour, which is the domain face:
    // 0 none (a refined level: mask-0 neighbours are coarse-fine faces),
    // 6 homogeneous Dirichlet, kRobinFace Robin (then robin != nullptr)
    int dirichlet;
    int periodic; // 1: the neighbour across a domain face is the opposite face's cell
    const RobinTab *robin;
    const uint8_t *mask;
    // per cell: bit f (f = 0..5 for the faces -x, +x, -y, +y, -z, +z) set
    // when the neighbour across f has mask != 0, bit 6 when the cell itself
    // has (one byte replaces the six neighbour-mask reads of a stencil)
    const uint8_t *code;
    // valid interior cells of a refined level as padded indices, the cells
    // of colour 0 (red) first, then those of colour 1 (null: the colour
    // passes enumerate the whole box); colour = parity of the global i+j+k
    const int *clist;
    int ccnt[2];
};

// Coarse-fine face table of a level l >= 1 (device pointers).
struct CfTable {
    int nface = 0;
    int ncell = 0;             // fine cells with at least one such face
    int *f = nullptr;          // [nface] fine cell (padded index, level l)
    int *f1 = nullptr;         // [nface] inward neighbour of f
    int8_t *dir = nullptr;     // [nface] 2*d + (s > 0)
    int8_t *cnt = nullptr;     // [nface] stencil size (9, 4 or 1)
    int *cidx = nullptr;       // [nface*9] coarse cells (padded index, level l-1)
    double *cw = nullptr;      // [nface*9] step-1 weight * 8/15
    int *cell_ptr = nullptr;   // [ncell+1] faces of each fine cell
    int *cell_f = nullptr;     // [ncell] the fine cell
    // coarse side (rows of level l-1 next to level l)
    int ncrse = 0;
    int *crse_c = nullptr;     // [ncrse] coarse cell (padded index, level l-1)
    int *crse_ptr = nullptr;   // [ncrse+1]
    int *crse_face = nullptr;  // [4 * number of coarse faces] face ids
    double *cp = nullptr;      // [nface] coarse part of each ghost (scratch)
    int64_t counts[3] = {0, 0, 0}; // quadratic, linear, constant stencils
};

// Smoother launch shape of one grid, picked by the autotuner: shape < 0
// runs each red-black sweep as two per-colour passes; shape >= 0 runs it as
// one fused launch (sweep.cu) with tile shape `shape` and zc planes per
// block.
struct SweepTile {
    int shape = -1;
    int zc = 0;
    // the blocks that hold valid cells, packed bx | by << 11 | bz << 22
    // (device, owned by the hierarchy); null: every block of the grid
    const unsigned *list = nullptr;
    int nlist = 0;
};

struct Level {
    Grid g{};
    SweepTile sw;
    uint8_t *code = nullptr; // neighbour codes (Grid::code)
    int vlo[3], vhi[3]; // valid bounding box (global, inclusive)
    int64_t nvalid = 0;
    uint8_t *mask = nullptr;
    double *rho = nullptr, *phi = nullptr, *res = nullptr, *err = nullptr;
    double *phisave = nullptr, *de = nullptr, *ef[3] = {nullptr, nullptr, nullptr};
    // mixed precision: FP32 right-hand side, correction, residual, error and
    // post-smoothing increment of the inner V-cycle (allocated for AMR_MIXED)
    float *rho32 = nullptr, *phi32 = nullptr, *res32 = nullptr, *err32 = nullptr, *de32 = nullptr;
    CfTable cf;                 // faces of this level towards level l-1
    std::vector<uint8_t> hmask; // host copy of the mask
    // covered cells (mask 2) as padded indices, in box order (the
    // restriction from level l + 1 runs one thread per entry); null: none
    int *cov = nullptr;
    int ncov = 0;
    // gather buffer: 1 where every cell within Chebyshev distance
    // H.gather_buffer is valid (levels >= 1; null while the buffer is 0)
    uint8_t *gmask = nullptr;
};

// One grid of the level-0 geometric multigrid (g = 0 aliases level 0).
struct MgGrid {
    Grid g{};
    SweepTile sw;
    uint8_t *code = nullptr; // neighbour codes (grid 0: level 0's)
    uint8_t *mask = nullptr;
    double *e = nullptr, *r = nullptr;
    float *e32 = nullptr, *r32 = nullptr;
    bool owns = false;
};

// The V-cycle arrays of a level in one precision.
template <typename T>
struct Fields {
    T *rho, *phi, *res, *err, *de;
};
template <typename T>
inline Fields<T> fields(Level &L);
template <>
inline Fields<double> fields<double>(Level &L)
{
    return {L.rho, L.phi, L.res, L.err, L.de};
}
template <>
inline Fields<float> fields<float>(Level &L)
{
    return {L.rho32, L.phi32, L.res32, L.err32, L.de32};
}
template <typename T>
inline T *mg_e(MgGrid &G);
template <typename T>
inline T *mg_r(MgGrid &G);
template <>
inline double *mg_e<double>(MgGrid &G)
{
    return G.e;
}
template <>
inline float *mg_e<float>(MgGrid &G)
{
    return G.e32;
}
template <>
inline double *mg_r<double>(MgGrid &G)
{
    return G.r;
}
template <>
inline float *mg_r<float>(MgGrid &G)
{
    return G.r32;
}

// Convergence test state of a solve (device memory; see k_check).
struct SolveParams {
    double eps;
    int norm;
    int max_iter;
};

struct SolveState {
    double rhon[kMaxLevels]; // ||rho^l||_p
    double rel[kMaxLevels];  // ||r^l||_p / ||rho^l||_p
    double worst;
    int iters;
    int go; // 1 while another V-cycle is due
};

// A captured solve: init -> while (go) { V-cycle; residuals; test } -> field.
struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    int nu1 = -1, nu2 = -1, bottom = -1, warm = -1;
    int64_t n_init = 0, n_body = 0, n_tail = 0;
};

// Persistent programs (see k_program): recorded phases, zipped into rounds.
struct Phase; // one recorded operation (defined with the kernels)
struct ProgramRecorder;

// Grid barrier state: monotonic arrival counters (one per group of blocks
// and one for the groups), each on its own 128-byte line.
constexpr int kBarGroups = 16;
struct ProgramCtl {
    unsigned grp[kBarGroups][32];
    unsigned top[32];
    int err[32]; // err[0] = 1: a barrier wait ran out (timeout)
};

struct ProgramDesc {
    const void *phases;
    const int *round_ptr, *round_nvb;
    const int *ph_hier, *ph_nvb; // per phase: its hierarchy and virtual blocks
    int init_r0, init_r1, body_r0, body_r1, tail_r0, tail_r1;
    int nhier, max_loops;
    SolveState *const *states; // device array of the hierarchies' states
    ProgramCtl *ctl;
    unsigned long long limit_ns; // longest barrier wait before a timeout
    unsigned nblocks_expected;
};

struct Program {
    void *dev = nullptr;
    size_t bytes = 0;
    SolveState **states = nullptr;
    ProgramCtl *ctl = nullptr;
    ProgramDesc D{};
    size_t smem = 0;
    int blocks = 0;
    int64_t n_phases[3] = {0, 0, 0}; // recorded operations per segment
    int nu1 = -1, nu2 = -1, bottom = -1, warm = -1;
};

// Batched programs on thread-block clusters (see k_cluster_program): each
// hierarchy's recorded operations stay contiguous (init, body, tail), and a
// queue hands hierarchies (largest first) to clusters.
struct ClusterDesc {
    const void *phases;
    const int *hseg;  // [6 per hierarchy]: phase ranges of init, body, tail
    const int *order; // queue order: hierarchy indices by decreasing work
    int nhier, max_loops;
    SolveState *const *states;
    unsigned *queue;  // [0] next queue position, [1 + c] cluster c's hierarchy
};

struct ClusterProgram {
    void *dev = nullptr;
    size_t bytes = 0;
    SolveState **states = nullptr;
    unsigned *queue = nullptr;
    ClusterDesc D{};
    size_t smem = 0;
    int clusters = 0; // co-resident clusters launched
    int csize = 0;    // blocks per cluster
    int64_t n_phases = 0;
};

// Operations issued between group_begin and group_end must be independent
// (no operation reads what another writes, and they write disjoint cells);
// group_end launches them as one kernel (falling back to one launch each
// for a combination without a fused kernel).  A no-op while recording a
// program or while the per-launch timers are on.
void group_begin(struct Hierarchy &H);
void group_end(struct Hierarchy &H);
void group_free(struct Hierarchy &H);

ProgramRecorder *recorder_new(int nhier);
void recorder_delete(ProgramRecorder *R);
void record_begin(struct Hierarchy &H, ProgramRecorder *R, int hier, int segment);
void record_end(struct Hierarchy &H);
int program_compile(ProgramRecorder *R, SolveState *const *states_host, int nhier, cudaStream_t stream, Program &P);
int program_run(struct Hierarchy &H, Program &P, cudaStream_t stream, unsigned long long limit_ns, int expected_blocks);
void program_free(Program &P);
// work[h]: the queue's sort key of hierarchy h (larger first)
int cluster_compile(ProgramRecorder *R, SolveState *const *states_host, const double *work, int nhier,
                    cudaStream_t stream, ClusterProgram &P);
// Enqueues the queue reset and the cluster launch on stream (capturable).
int cluster_run(ClusterProgram &P, cudaStream_t stream);
void cluster_free(ClusterProgram &P);

// Kernel kinds for the per-launch event timers.
enum Kind {
    K_DEPOSIT, K_GATHER, K_RESIDUAL, K_RBGS, K_RESTRICT, K_PROLONG, K_FINISH, K_CF, K_FLUX, K_GRAD, K_AVGDOWN,
    K_NORMS, K_MG_RESTRICT, K_MG_PROLONG, K_COARSE, K_ELEMENTWISE, K_CP, K_CHECK, K_MG_BOTTOM, K_BIN,
    K_DST, K_TRIZ, K_NUM
};

struct ProfRecord {
    int kind;
    int ev;       // index of the start event in the pool (stop = ev + 1)
    double bytes; // algorithmic bytes of the launch
    double flops; // algorithmic floating-point operations (FMA = 2)
    double ops;   // algorithmic arithmetic instructions of the kernel's precision (FMA = 1)
    double share; // fraction of the timed interval charged to this record
                  // (1; an operation of a grouped launch gets its share of
                  // the group's algorithmic bytes)
};

struct Hierarchy {
    int n0 = 0;
    int nlev = 0;
    double eps0 = 1.0;
    int precision = AMR_FP64;
    int brick = 8;
    double robin_d = 0.0; // > 0: Robin domain faces with this distance d
    bool periodic = false; // periodic domain faces (singular operator, see solve)
    double *pmean = nullptr; // periodic: composite volume mean (1 double)
    int gather_buffer = 0;   // refined levels gathered from only this many cells inside
    cudaStream_t stream = nullptr;
    Level L[kMaxLevels];
    // level-0 geometric multigrid: grids 0..nmg-1, the last solved densely
    int nmg = 0;
    MgGrid mg[16];
    double *coarse_inv = nullptr; // dense inverse of the coarsest operator
    // coarsest grids above 11^3 (n0 with a large odd factor): solved
    // separably, e = V3 diag(h^2 / (lam_i + lam_j + lam_k)) V3^T r with the
    // eigenvectors V and eigenvalues lam of the 1-D operator (csep_n > 0)
    int csep_n = 0;
    double *csep_v = nullptr, *csep_vt = nullptr, *csep_lam = nullptr;
    double *csep_tmp[2] = {nullptr, nullptr};
    double csep_zero_add = 0.0;
    // exact level-0 bottom solve by sine transforms (n0 <= 64 by default):
    // two level-0-sized FP64 work arrays, the forward / inverse transform
    // matrices (n0 x n0, as MT[i n + m]) and the reciprocal pivots of the
    // z tridiagonal solves ([k][mode])
    bool dst_on = false;
    double *dst_a = nullptr, *dst_b = nullptr, *dst_mf = nullptr, *dst_mi = nullptr, *dst_iw = nullptr;
    // n0 a power of two (32..128): the same solve by fast transforms
    // (O(n log n) per line), their split factors in dst_tab and the
    // tridiagonal solve's per-mode factors (h^2 and the basis scales) in dst_fm
    bool dst_fast = false;
    double *dst_tab = nullptr, *dst_fm = nullptr;
    // second iterate for out-of-place fused sweeps (largest grid, FP64 size)
    double *sweep_tmp = nullptr;
    int mg_bottom = -1; // first grid of the one-launch multigrid bottom, -1: none
    int ncoarse = 0;              // its order
    // reduction scratch: per slot (residual of each level, then rho of each
    // level) and per block {sum v^2, sum |v|, max |v|}
    double *partials = nullptr;   // [2 * kMaxLevels * 3 * kPartialBlocks]
    SolveParams *params = nullptr, *params_host = nullptr;  // device / pinned
    SolveState *state = nullptr, *state_host = nullptr;     // device / pinned
    SolveGraph graphs[4];
    bool capturing = false;
    bool pdl = true; // programmatic dependent launch between kernels
    std::vector<Phase> *rec = nullptr; // recording a program instead of launching
    // grouping: independent operations issued between group_begin and
    // group_end run as ONE launch (see group_end)
    bool grouping = false;
    std::vector<Phase> *group = nullptr;
    int *nc_counter = nullptr; // arrival counter of the fused norms + check
    unsigned *bin_cnt = nullptr; // bucket counts / offsets of the particle binning
    int rec_hier = 0;
    Program prog;                      // persistent program of this hierarchy
    int *outside = nullptr;       // device counter of particles outside level 0
    // staging for amr_step, and its copy stream and chunk events (the
    // host-device copies of one chunk of particles overlap the deposit or
    // the gather of another)
    double *stage = nullptr;
    int64_t stage_n = 0;
    cudaStream_t cstream = nullptr;
    cudaEvent_t cev[2 * kStepChunks + 2] = {};
    int64_t device_bytes = 0;
    int64_t max_bytes = 0;   // > 0: allocations stop at this many device bytes
    bool over_limit = false; // an allocation was refused by max_bytes
    int64_t launches = 0;
    std::vector<void *> allocs;
    // per-launch event timers (off unless amr_profile enables them):
    // prof_mode 1 runs solves host-driven with an event pair around every
    // launch; prof_mode 2 runs each solve as a captured graph unrolled to
    // prof_iters V-cycles, the same kernels and grouped launches as the
    // solve graph, with event-record nodes around every kernel node
    bool prof = false;
    int prof_mode = 0;
    int prof_iters = 0;
    bool prof_capture = false;            // capturing the profiled graph
    std::vector<ProfRecord> group_prof;  // operations of the open group
    std::vector<cudaEvent_t> evpool;
    std::vector<ProfRecord> pending;
    int evnext = 0;
    double kind_ms[K_NUM] = {};
    double kind_bytes[K_NUM] = {};
    double kind_flops[K_NUM] = {};
    double kind_ops[K_NUM] = {};
    int64_t kind_launches[K_NUM] = {};
};

// Counts the launch and, when the timers are on (and nothing is being
// captured or recorded), brackets it with a pair of events.
struct Launch {
    Hierarchy &H;
    int kind;
    double bytes, flops, ops;
    int ev = -1;
    Launch(Hierarchy &h, int k, double b, double f = 0.0, double o = 0.0) : H(h), kind(k), bytes(b), flops(f), ops(o)
    {
        if (!H.prof || H.rec || (H.capturing && !H.prof_capture)) return;
        if (H.grouping) {
            // timed around the group's launch (group_end)
            H.group_prof.push_back({kind, -1, bytes, flops, ops, 0.0});
            return;
        }
        ev = prof_event_pair(H);
        prof_record(H, ev);
    }
    ~Launch()
    {
        if (!H.rec && !H.grouping) H.launches++;
        if (ev < 0) return;
        prof_record(H, ev + 1);
        H.pending.push_back({kind, ev, bytes, flops, ops, 1.0});
    }
    // next free pair of the event pool (grown outside captures: the
    // profiled graph's pool is reserved before its capture starts)
    static int prof_event_pair(Hierarchy &H)
    {
        if (H.evnext + 2 > (int)H.evpool.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                H.evpool.push_back(e);
            }
        }
        int e = H.evnext;
        H.evnext += 2;
        return e;
    }
    // an event on the stream, or an event-record node of the graph being
    // captured
    static void prof_record(Hierarchy &H, int e)
    {
        if (H.capturing)
            cudaEventRecordWithFlags(H.evpool[e], H.stream, cudaEventRecordExternal);
        else
            cudaEventRecord(H.evpool[e], H.stream);
    }
};

// valid cells of the level (or multigrid grid) whose mask g.mask is
double valid_cells(const Hierarchy &H, const Grid &g);

// Resolve pending event pairs into the per-kind totals (waits for them).
int prof_resolve(Hierarchy &H);
const char *kind_name(int kind);

constexpr int kPartialBlocks = 1024;

// ---- kernels and launchers (kernels.cu) -----------------------------------
void launch_deposit(Hierarchy &H, const double *x, const double *y, const double *z, const double *q,
                    int64_t n, int level_only);
void launch_gather(Hierarchy &H, const double *x, const double *y, const double *z, int64_t n, double *ex,
                   double *ey, double *ez, double *phi);
// r = rho - A phi on level l (bulk stencil; comp=1 skips covered faces and
// writes only uncovered cells, zeroing covered ones when zero_covered)
template <typename T>
void launch_residual(Hierarchy &H, const Grid &g, const T *rho, const T *phi, T *res, int comp, int zero_covered);
// One red-black colour pass.  first: the iterate starts from zero (red
// cells get h^2 b / D, black cells are zeroed).  mode 1 adds the new
// values to e and phi (end of a post-smooth), mode 2 adds them to phi.
template <typename T>
void launch_rbgs(Hierarchy &H, const Grid &g, T *x, const T *b, int colour, int first, int mode, T *e, T *phi);
template <typename T>
void launch_restrict_amr(Hierarchy &H, int l); // Alg. 3 pre-smooth update + restriction
template <typename T>
void launch_prolong_amr(Hierarchy &H, int l); // Alg. 3 prolongation + residual update
template <typename T>
void launch_finish_amr(Hierarchy &H, int l); // e += de; phi += de (when no post-smooth)
template <typename T>
void launch_cp(Hierarchy &H, int l, const T *uc); // coarse part of level l's ghosts from uc
// fine side: r^lf += ih2 * sum of cp over the cell's faces (level lf);
// coarse side: flux-matched rows of level lc-1 from level lc's faces.
template <typename T>
void launch_surface(Hierarchy &H, int lf, T *rf, int lc, const T *uf, T *rc);
void launch_to32(Hierarchy &H, int l);  // rho32 = res32 = r (FP64 residual), phi32 = 0
void launch_cp_zero(Hierarchy &H, int l); // coarse parts of level l <- 0
void launch_add32(Hierarchy &H, int l); // phi += phi32
void launch_grad(Hierarchy &H, int l);
void launch_cf_grad(Hierarchy &H, int l);
void launch_average_down(Hierarchy &H, int l); // phi^l covered <- R phi^{l+1}
// norms of the residual of every level (and of rho when with_rho) followed
// by the convergence test; sets the graph condition when cond != 0.
void launch_norms_check(Hierarchy &H, int with_rho, int is_body, unsigned long long cond, int use_cond);
template <typename T>
// r_{g+1} = R (r_g - A e_g); e_{g+1} = 0, or with first_red the first red
// pass from zero on grid g+1 (black cells 0)
void launch_mg_restrict(Hierarchy &H, int g, int first_red);
template <typename T>
void launch_mg_prolong(Hierarchy &H, int g); // e_g += P e_{g+1} (trilinear)
template <typename T>
void launch_mg_coarse_solve(Hierarchy &H);
// Exact solve of A_nf^0 e^0 = r^0 on level 0 by sine transforms (x, y),
// tridiagonal solves (z) and the inverse transforms; phi^0 += e^0.
template <typename T>
void launch_dst_bottom(Hierarchy &H);
// First multigrid grid g >= 1 from which the rest of the V-cycle runs as
// one cluster launch (launch_mg_bottom) when AMR_MG_BOTTOM=1, else -1.
int mg_bottom_grid(const Hierarchy &H);
// The V-cycle of grids gb .. coarsest (pre-smooth nu1 from zero,
// restriction, dense coarsest solve, prolongation, post-smooth nu2) as one
// launch of one thread-block cluster.
template <typename T>
void launch_mg_bottom(Hierarchy &H, int gb, int nu1, int nu2);
template <typename T>
void launch_fill(Hierarchy &H, T *p, T v, int64_t n);
template <typename T>
void launch_axpy(Hierarchy &H, T *y, const T *x, T a, int64_t n);

// One red-black sweep in a single launch, out of place (sweep.cu): reads
// the iterate xin (not read when first: the sweep starts from zero), writes
// the new iterate to xout; mode as in launch_rbgs.
template <typename T>
void launch_sweep(Hierarchy &H, const Grid &g, const SweepTile &tile, const T *xin, T *xout, const T *b, int first,
                  int mode, T *e, T *phi);
int sweep_num_shapes();
// Neighbour codes of grid g from its mask (Grid::code), on H.stream.
void launch_make_code(Hierarchy &H, const Grid &g, uint8_t *code);
// Picks the smoother launch shape of every grid of the hierarchy (timed on
// its stream, cached per grid size class and precision).
int autotune_sweeps(Hierarchy &H);

// Particle binning (amr_bin): keys, bucket counts, their prefix sum and the
// sorted permutation; bin_num_keys is the number of bricks of all levels.
int64_t bin_num_keys(const Hierarchy &H);
int launch_bin(Hierarchy &H, const double *x, const double *y, const double *z, int64_t n, uint32_t *keys,
               int64_t *perm);

// ---- error helpers ---------------------------------------------------------
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

int regrid_boxes(Hierarchy &H, int policy, double lambda, int buffer, int max_level, std::vector<int> &out);
int transfer_phi(const Hierarchy &src, Hierarchy &dst);
// Periodic faces: subtract the composite volume mean of rho (which = 0) or
// phi (which = 1) from every valid cell of every level, on H.stream.
void launch_remove_mean(Hierarchy &H, int which);
// The gather-buffer masks (Level::gmask) of levels >= 1 for buffer b.
int set_gather_buffer(Hierarchy &H, int b);

} // namespace amr

// The opaque C handle of a hierarchy.
struct amr_hierarchy {
    amr::Hierarchy *H;
};
