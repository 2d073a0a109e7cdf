// V-cycle driver (Alg. 1-3), the level-0 multigrid bottom solve, and the
// extern "C" entry points of libamrmg.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "amr_internal.h"

namespace amr {

int create_hierarchy(const amr_desc *d, const double *x, const double *y, const double *z, const double *q,
                     int64_t n, void *stream, Hierarchy **out);
void free_hierarchy(Hierarchy *H);
int64_t hierarchy_bytes_estimate(const amr_desc *d, double fill);

static thread_local std::string g_error;

void set_error(const std::string &msg) { g_error = msg; }

int cuda_fail(cudaError_t e, const char *what)
{
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    return AMR_ECUDA;
}

namespace {

struct Opts {
    int nu1, nu2, bottom_cycles;
};

// Alg. 1 RESIDUAL(l) for every level (FP64): bulk stencil, then the coarse
// parts of the ghosts from phi^{l-1} and the surface corrections
// (coarse-fine ghosts of level l, flux-matched rows of level l-1).  Leaves
// the coarse parts of all levels computed from phi^{l-1}, which the
// down-sweep of the next V-cycle reuses.
void residual_all(Hierarchy &H)
{
    // bulk residuals and coarse parts are independent (one launch); the
    // surface corrections of different levels write disjoint cells (proper
    // nesting keeps a level's coarse-side cells off the coarser level's own
    // coarse-fine cells), so they form a second launch
    int lmax = H.nlev - 1;
    group_begin(H);
    for (int l = 0; l <= lmax; ++l) {
        Level &L = H.L[l];
        launch_residual<double>(H, L.g, L.rho, L.phi, L.res, l < lmax, 1);
    }
    for (int l = 1; l <= lmax; ++l) launch_cp<double>(H, l, H.L[l - 1].phi);
    group_end(H);
    group_begin(H);
    for (int l = 1; l <= lmax; ++l) launch_surface<double>(H, l, H.L[l].res, l, H.L[l].phi, H.L[l - 1].res);
    group_end(H);
}

// nu red-black sweeps on A x = b; from_zero: the iterate starts at zero.
// mode (1 or 2) is applied to the last sweep (see launch_rbgs).  With a
// fused tile each sweep is one out-of-place launch, alternating between x
// and the scratch iterate so that the last sweep writes x; recorded
// programs and an odd sweep count on a given iterate use per-colour passes
// (the iterates are bitwise the same either way).
bool fused_smooth(const Hierarchy &H, const SweepTile &tile, int nu, bool from_zero)
{
    return tile.shape >= 0 && !H.rec && H.sweep_tmp && (from_zero || nu % 2 == 0);
}

// red_done: the red pass of the first sweep (from zero) has already been
// applied by the restriction that produced b (per-colour passes only).
template <typename T>
void smooth(Hierarchy &H, const Grid &g, const SweepTile &tile, T *x, const T *b, int nu, bool from_zero, int mode,
            T *e, T *phi, bool red_done = false)
{
    if (!fused_smooth(H, tile, nu, from_zero)) {
        for (int it = 0; it < nu; ++it) {
            int m = it == nu - 1 ? mode : 0;
            if (!(red_done && it == 0)) launch_rbgs<T>(H, g, x, b, 0, from_zero && it == 0, m, e, phi);
            launch_rbgs<T>(H, g, x, b, 1, 0, m, e, phi);
        }
        return;
    }
    T *tmp = reinterpret_cast<T *>(H.sweep_tmp);
    for (int it = 0; it < nu; ++it) {
        T *dst = ((nu - 1 - it) % 2 == 0) ? x : tmp;
        const T *src = it == 0 ? x : (dst == x ? tmp : x);
        int m = it == nu - 1 ? mode : 0;
        launch_sweep<T>(H, g, tile, src, dst, b, from_zero && it == 0, m, e, phi);
    }
}

// Geometric multigrid V-cycle on grid g of the level-0 hierarchy; the last
// post-smoothing sweep of the last cycle adds the correction to phi^0.
template <typename T>
void mg_vcycle(Hierarchy &H, int g, const Opts &o, bool first_cycle, bool last_cycle, bool red_done = false)
{
    MgGrid &G = H.mg[g];
    Fields<T> f0 = fields<T>(H.L[0]);
    T *ge = mg_e<T>(G), *gr = mg_r<T>(G);
    if (g == H.nmg - 1) {
        launch_mg_coarse_solve<T>(H);
        if (g == 0 && last_cycle) launch_axpy<T>(H, f0.phi, f0.err, T(1), H.L[0].g.ncell);
        return;
    }
    if (g > 0 && g == H.mg_bottom && !H.rec) {
        // the rest of the cycle in one cluster launch (same operations; e_g
        // is already zero from the restriction that produced r_g)
        launch_mg_bottom<T>(H, g, o.nu1, o.nu2);
        return;
    }
    bool from_zero = g > 0 || first_cycle;
    if (from_zero && o.nu1 == 0) launch_fill<T>(H, ge, T(0), G.g.ncell);
    smooth<T>(H, G.g, G.sw, ge, gr, o.nu1, from_zero, 0, nullptr, nullptr, red_done);
    // the next grid's first red pass rides on the restriction when that grid
    // is smoothed by per-colour passes (and not by the cluster bottom or
    // the dense coarsest solve)
    const int gn = g + 1;
    bool fuse = gn < H.nmg - 1 && o.nu1 > 0 && !(gn == H.mg_bottom && !H.rec) &&
                !fused_smooth(H, H.mg[gn].sw, o.nu1, true);
    launch_mg_restrict<T>(H, g, fuse ? 1 : 0);
    mg_vcycle<T>(H, gn, o, false, false, fuse);
    launch_mg_prolong<T>(H, g);
    int mode = (g == 0 && last_cycle) ? 2 : 0;
    if (o.nu2 > 0)
        smooth<T>(H, G.g, G.sw, ge, gr, o.nu2, false, mode, nullptr, f0.phi);
    else if (mode == 2)
        launch_axpy<T>(H, f0.phi, f0.err, T(1), H.L[0].g.ncell);
}

// Alg. 3 RELAX(l) in precision T.  On entry r^{l_max} and the coarse parts
// of every level hold Alg. 1's values for the current phi (the preceding
// residual evaluation), so the residual that Alg. 3 starts from is not
// recomputed.
template <typename T>
void relax(Hierarchy &H, int l, const Opts &o)
{
    Level &L = H.L[l];
    Fields<T> fl = fields<T>(L);
    if (l == 0 && H.dst_on) {
        // bottom: A_nf^0 e^0 = r^0 solved exactly (sine transforms), phi^0 += e^0
        launch_dst_bottom<T>(H);
        return;
    }
    if (l == 0) {
        // bottom: A_nf^0 e^0 = r^0 by geometric multigrid, phi^0 += e^0
        int cycles = H.nmg == 1 ? 1 : o.bottom_cycles;
        for (int c = 0; c < cycles; ++c) mg_vcycle<T>(H, 0, o, c == 0, c == cycles - 1);
        return;
    }
    Level &C = H.L[l - 1];
    Fields<T> fc = fields<T>(C);
    // e^{l-1} <- 0 is implicit: the pre-smooth runs with homogeneous
    // coarse-fine ghosts and relax(l-1) starts its own error from zero
    if (o.nu1 == 0) launch_fill<T>(H, fl.err, T(0), L.g.ncell);
    smooth<T>(H, L.g, L.sw, fl.err, fl.res, o.nu1, true, 0, nullptr, nullptr);
    // phi^l += e^l; r^l <- r^l - A_nf e^l; r^{l-1} <- R r^l on covered cells
    // (one launch with the next step: it writes the uncovered cells of l-1,
    // the restriction only covered ones, and reads neither's results)
    group_begin(H);
    launch_restrict_amr<T>(H, l);
    // uncovered cells of l-1: rho - A_comp phi^{l-1} - B_crse phi^{l-2} - B_fine phi^l
    launch_residual<T>(H, C.g, fc.rho, fc.phi, fc.res, 1, 0);
    group_end(H);
    launch_surface<T>(H, l - 1, fc.res, l, fl.phi, fc.res);
    relax<T>(H, l - 1, o);
    // e^l <- e^l + I e^{l-1} (phi^l too); r^l <- r^l - A_nf I e^{l-1} - B_crse e^{l-1}
    // (one launch with the coarse parts from e^{l-1}: both only read e^{l-1})
    group_begin(H);
    launch_prolong_amr<T>(H, l);
    launch_cp<T>(H, l, fc.err);
    group_end(H);
    launch_surface<T>(H, l, fl.res, -1, (const T *)nullptr, (T *)nullptr);
    // post-smooth delta e from zero; the last sweep adds it to e^l and phi^l
    if (o.nu2 > 0) smooth<T>(H, L.g, L.sw, fl.de, fl.res, o.nu2, true, 1, fl.err, fl.phi);
}

void field(Hierarchy &H)
{
    for (int l = H.nlev - 2; l >= 0; --l) launch_average_down(H, l);
    for (int l = 0; l < H.nlev; ++l) {
        launch_grad(H, l);
        if (l > 0) {
            launch_cp<double>(H, l, H.L[l - 1].phi);
            launch_cf_grad(H, l);
        }
    }
}

void init_part(Hierarchy &H, bool warm, unsigned long long cond, int use_cond)
{
    if (!warm)
        for (int l = 0; l < H.nlev; ++l) launch_fill<double>(H, H.L[l].phi, 0.0, H.L[l].g.ncell);
    residual_all(H);
    launch_norms_check(H, 1, 0, cond, use_cond);
}

// One iteration of Alg. 2.  FP64: an Alg. 3 V-cycle on phi.  Mixed
// precision: the same V-cycle in FP32 on the correction equation
// A^comp delta = r (r the FP64 composite residual, delta from zero, coarse
// parts zero), then phi += delta in FP64 (iterative refinement); the
// residual, interface corrections and the coarsest solve stay FP64.
void body_part(Hierarchy &H, const Opts &o, unsigned long long cond, int use_cond)
{
    if (H.precision == AMR_MIXED) {
        for (int l = 0; l < H.nlev; ++l) {
            launch_to32(H, l);
            if (l > 0) launch_cp_zero(H, l);
        }
        relax<float>(H, H.nlev - 1, o);
        for (int l = 0; l < H.nlev; ++l) launch_add32(H, l);
    } else {
        relax<double>(H, H.nlev - 1, o);
    }
    residual_all(H);
    launch_norms_check(H, 0, 1, cond, use_cond);
}

int check_launch(Hierarchy &H, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    (void)H;
    return AMR_OK;
}

#define AMR_TRY(call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

// Append the solve of H to graph g as one independent branch: init ->
// while (go) { V-cycle; residuals; test } -> field, the loop condition set
// on the device by k_check.  io: the branch also uploads the hierarchy's
// solve parameters first and reads its state back last (from and to its
// pinned host copies).  Capture runs on a private stream (the legacy default
// stream cannot be captured); launch counts per segment go to n[3].
int capture_solve_into(Hierarchy &H, cudaGraph_t g, const Opts &o, bool warm, bool io, int64_t n[3])
{
    cudaStream_t user = H.stream, cap = nullptr;
    AMR_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "graph stream");
    cudaGraphConditionalHandle hc;
    int rc = AMR_OK;
    int64_t c0 = H.launches;
    do {
        cudaError_t e = cudaGraphConditionalHandleCreate(&hc, g, 0, 0);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "graph capture begin");
            break;
        }
        H.stream = cap;
        H.capturing = true;
        if (io) cudaMemcpyAsync(H.params, H.params_host, sizeof(SolveParams), cudaMemcpyHostToDevice, cap);
        int64_t a = H.launches;
        init_part(H, warm, (unsigned long long)hc, 1);
        n[0] = H.launches - a;
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, &deps, nullptr, &nd);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wn = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&wn, cg, deps, nullptr, nd, &cp);
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cap, &wn, nullptr, 1, cudaStreamSetCaptureDependencies);
        a = H.launches;
        if (e == cudaSuccess) field(H);
        n[2] = H.launches - a;
        if (e == cudaSuccess && io)
            e = cudaMemcpyAsync(H.state_host, H.state, sizeof(SolveState), cudaMemcpyDeviceToHost, cap);
        cudaGraph_t gout = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &gout);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            rc = cuda_fail(e != cudaSuccess ? e : e2, "graph capture");
            break;
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        a = H.launches;
        if (e == cudaSuccess) body_part(H, o, (unsigned long long)hc, 1);
        n[1] = H.launches - a;
        e2 = cudaStreamEndCapture(cap, &body);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            rc = cuda_fail(e != cudaSuccess ? e : e2, "graph body capture");
            break;
        }
    } while (0);
    H.capturing = false;
    H.stream = user;
    H.launches = c0; // captured launches are counted when the graph runs
    cudaGetLastError();
    cudaStreamDestroy(cap);
    return rc;
}

// The solve of H as one captured graph (see capture_solve_into), launched
// on the hierarchy's stream.
int build_graph(Hierarchy &H, SolveGraph &G, const Opts &o, bool warm)
{
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    AMR_TRY(cudaGraphCreate(&g, 0), "graph create");
    int64_t n[3] = {0, 0, 0};
    int rc = capture_solve_into(H, g, o, warm, false, n);
    if (rc == AMR_OK) {
        cudaError_t e = cudaGraphInstantiate(&G.exec, g, 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "graph instantiate");
            G.exec = nullptr;
        }
    }
    cudaGraphDestroy(g);
    if (rc == AMR_OK) {
        G.n_init = n[0];
        G.n_body = n[1];
        G.n_tail = n[2];
        G.nu1 = o.nu1;
        G.nu2 = o.nu2;
        G.bottom = o.bottom_cycles;
        G.warm = warm;
    }
    return rc;
}

int get_graph(Hierarchy &H, const Opts &o, bool warm, SolveGraph **out)
{
    for (SolveGraph &G : H.graphs)
        if (G.exec && G.nu1 == o.nu1 && G.nu2 == o.nu2 && G.bottom == o.bottom_cycles && G.warm == (int)warm) {
            *out = &G;
            return AMR_OK;
        }
    SolveGraph *slot = &H.graphs[0];
    for (SolveGraph &G : H.graphs)
        if (!G.exec) {
            slot = &G;
            break;
        }
    int rc = build_graph(H, *slot, o, warm);
    *out = slot;
    return rc;
}

// The profiled solve (amr_profile mode 2): init, n V-cycle bodies and the
// tail captured straight (no conditional node, so every kernel node runs
// once per launch), with the same kernels and grouped launches as the solve
// graph and an event-record node before and after each kernel node.  The
// graph is launched once on the hierarchy's stream and destroyed.
int run_profiled_graph(Hierarchy &H, const Opts &o, bool warm, int n)
{
    // the event pool must not grow during the capture
    SolveGraph *G = nullptr;
    int rc = get_graph(H, o, warm, &G);
    if (rc != AMR_OK) return rc;
    const int64_t need = 2 * (G->n_init + G->n_tail + (int64_t)n * G->n_body) + 64;
    while ((int64_t)H.evpool.size() < H.evnext + need) {
        cudaEvent_t e;
        AMR_TRY(cudaEventCreate(&e), "profile events");
        H.evpool.push_back(e);
    }
    cudaStream_t user = H.stream, cap = nullptr;
    AMR_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "graph stream");
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    const size_t pend0 = H.pending.size();
    const int ev0 = H.evnext;
    int64_t c0 = H.launches;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        H.stream = cap;
        H.capturing = true;
        H.prof_capture = true;
        init_part(H, warm, 0, 0);
        for (int it = 0; it < n; ++it) body_part(H, o, 0, 0);
        field(H);
        H.prof_capture = false;
        H.capturing = false;
        H.stream = user;
        e = cudaStreamEndCapture(cap, &g);
    }
    H.launches = c0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, H.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H.stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        // drop this capture's records
        H.pending.resize(pend0);
        H.evnext = ev0;
        cudaGetLastError();
        return cuda_fail(e, "profiled graph");
    }
    H.launches += G->n_init + G->n_tail + (int64_t)n * G->n_body;
    return AMR_OK;
}

// Record the solve of one hierarchy (index hier of a program): init,
// V-cycle body, tail.
void record_solve(Hierarchy &H, ProgramRecorder *R, int hier, const Opts &o, bool warm)
{
    record_begin(H, R, hier, 0);
    init_part(H, warm, 0, 0);
    record_end(H);
    record_begin(H, R, hier, 1);
    body_part(H, o, 0, 0);
    record_end(H);
    record_begin(H, R, hier, 2);
    field(H);
    record_end(H);
}

int program_status(Program &P, cudaStream_t s)
{
    ProgramCtl ctl{};
    AMR_TRY(cudaMemcpyAsync(&ctl, P.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s), "program status");
    AMR_TRY(cudaStreamSynchronize(s), "program");
    if (ctl.err[0]) {
        set_error("a grid barrier of the persistent program ran out of time");
        return AMR_ETIMEOUT;
    }
    return AMR_OK;
}

int ensure_program(Hierarchy &H, const Opts &so, bool warm)
{
    Program &P = H.prog;
    if (P.dev && P.nu1 == so.nu1 && P.nu2 == so.nu2 && P.bottom == so.bottom_cycles && P.warm == (int)warm)
        return AMR_OK;
    ProgramRecorder *R = recorder_new(1);
    record_solve(H, R, 0, so, warm);
    SolveState *st = H.state;
    int rc = program_compile(R, &st, 1, H.stream, P);
    recorder_delete(R);
    if (rc == AMR_OK) {
        P.nu1 = so.nu1;
        P.nu2 = so.nu2;
        P.bottom = so.bottom_cycles;
        P.warm = warm;
    }
    return rc;
}

int read_state(Hierarchy &H)
{
    AMR_TRY(cudaMemcpyAsync(H.state_host, H.state, sizeof(SolveState), cudaMemcpyDeviceToHost, H.stream), "state");
    AMR_TRY(cudaStreamSynchronize(H.stream), "solve");
    return AMR_OK;
}

int solve(Hierarchy &H, const amr_solve_opts *opts, amr_solve_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    amr_solve_opts o;
    amr_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.nu_pre < 0 || o.nu_post < 0 || o.bottom_cycles < 1 ||
        (o.norm != AMR_NORM_INF && o.norm != AMR_NORM_1 && o.norm != AMR_NORM_2) || !(o.eps >= 0.0)) {
        set_error("invalid solve options");
        return AMR_EINVAL;
    }
    Opts so{o.nu_pre, o.nu_post, o.bottom_cycles};
    // periodic faces: the operator is singular (constants); solve with the
    // neutralised density rho - <rho> (a uniform background of opposite
    // charge) and return the mean-free potential
    if (H.periodic) launch_remove_mean(H, 0);
    H.params_host->eps = o.eps;
    H.params_host->norm = o.norm;
    H.params_host->max_iter = o.max_iter;
    AMR_TRY(cudaMemcpyAsync(H.params, H.params_host, sizeof(SolveParams), cudaMemcpyHostToDevice, H.stream),
            "solve parameters");
    int rc;
    bool warm = o.warm_start != 0;
    // (periodic faces: the program kernel has no periodic operations, so such
    // a hierarchy solves through its graph)
    if (o.persistent && !H.prof && !H.periodic) {
        if ((rc = ensure_program(H, so, warm)) != AMR_OK) return rc;
        if ((rc = program_run(H, H.prog, H.stream, 2000000000ull, 0)) != AMR_OK) return rc;
        if ((rc = program_status(H.prog, H.stream)) != AMR_OK) return rc;
        if ((rc = read_state(H)) != AMR_OK) return rc;
    } else if (o.use_graph && H.prof && H.prof_mode == 2 && H.prof_iters > 0) {
        if ((rc = run_profiled_graph(H, so, warm, H.prof_iters)) != AMR_OK) return rc;
        if ((rc = read_state(H)) != AMR_OK) return rc;
    } else if (o.use_graph && !H.prof) {
        SolveGraph *G = nullptr;
        if ((rc = get_graph(H, so, warm, &G)) != AMR_OK) return rc;
        AMR_TRY(cudaGraphLaunch(G->exec, H.stream), "graph launch");
        if ((rc = read_state(H)) != AMR_OK) return rc;
        H.launches += G->n_init + G->n_tail + (int64_t)H.state_host->iters * G->n_body;
    } else {
        init_part(H, warm, 0, 0);
        if ((rc = check_launch(H, "solve launch")) != AMR_OK) return rc;
        if ((rc = read_state(H)) != AMR_OK) return rc;
        while (H.state_host->go) {
            body_part(H, so, 0, 0);
            if ((rc = check_launch(H, "V-cycle launch")) != AMR_OK) return rc;
            if ((rc = read_state(H)) != AMR_OK) return rc;
        }
        field(H);
        if ((rc = read_state(H)) != AMR_OK) return rc;
    }
    if (H.periodic) {
        launch_remove_mean(H, 1);
        AMR_TRY(cudaStreamSynchronize(H.stream), "mean-free potential");
    }
    if (H.prof && (rc = prof_resolve(H)) != AMR_OK) return rc;
    const SolveState &st = *H.state_host;
    int status = st.worst <= o.eps ? AMR_OK : AMR_ENOCONV;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->iters = st.iters;
        stats->status = status;
        stats->n_levels = H.nlev;
        for (int l = 0; l < H.nlev; ++l) stats->rel_res[l] = st.rel[l];
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != AMR_OK) set_error("not converged within max_iter V-cycles");
    return status;
}

// Many independent hierarchies at once: each one's captured solve graph is
// launched on one of nstreams library streams (round robin), ordered after
// the work already queued on the hierarchy's own stream and before the work
// queued there later (events both ways).  Small hierarchies leave most SMs
// idle one at a time; side by side their graphs fill the GPU.  Hierarchies
// with periodic faces (mean removal around the graph) or with the per-launch
// timers on are solved by solve() afterwards.
int solve_many(Hierarchy *const *hs, int n, const amr_solve_opts *opts, int nstreams, amr_solve_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    amr_solve_opts o;
    amr_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.nu_pre < 0 || o.nu_post < 0 || o.bottom_cycles < 1 ||
        (o.norm != AMR_NORM_INF && o.norm != AMR_NORM_1 && o.norm != AMR_NORM_2) || !(o.eps >= 0.0)) {
        set_error("invalid solve options");
        return AMR_EINVAL;
    }
    Opts so{o.nu_pre, o.nu_post, o.bottom_cycles};
    const bool warm = o.warm_start != 0;
    nstreams = std::max(1, std::min(nstreams, 64));
    std::vector<SolveGraph *> G((size_t)n, nullptr);
    for (int i = 0; i < n; ++i) {
        Hierarchy &H = *hs[i];
        if (H.periodic || H.prof) continue;
        int rc = get_graph(H, so, warm, &G[i]);
        if (rc != AMR_OK) return rc;
    }
    std::vector<cudaStream_t> pool((size_t)nstreams, nullptr);
    std::vector<cudaEvent_t> ev((size_t)2 * n, nullptr);
    int rc = AMR_OK;
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t st : pool)
            if (st) cudaStreamDestroy(st);
    };
    for (cudaStream_t &st : pool)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            st = nullptr;
            cleanup();
            return cuda_fail(cudaGetLastError(), "solve streams");
        }
    // three passes, so that hierarchies sharing one stream do not chain
    // their graphs: every start event first, then the graphs, then the
    // waits of the hierarchies' streams on the graphs
    for (int i = 0; i < n && rc == AMR_OK; ++i) {
        if (!G[i]) continue;
        Hierarchy &H = *hs[i];
        H.params_host->eps = o.eps;
        H.params_host->norm = o.norm;
        H.params_host->max_iter = o.max_iter;
        cudaError_t e = cudaMemcpyAsync(H.params, H.params_host, sizeof(SolveParams), cudaMemcpyHostToDevice, H.stream);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[2 * i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[2 * i + 1], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i], H.stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "concurrent solve launch");
    }
    for (int i = 0; i < n && rc == AMR_OK; ++i) {
        if (!G[i]) continue;
        cudaStream_t st = pool[(size_t)i % nstreams];
        cudaError_t e = cudaStreamWaitEvent(st, ev[2 * i], 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(G[i]->exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], st);
        if (e != cudaSuccess) rc = cuda_fail(e, "concurrent solve launch");
    }
    for (int i = 0; i < n && rc == AMR_OK; ++i) {
        if (!G[i]) continue;
        Hierarchy &H = *hs[i];
        cudaError_t e = cudaStreamWaitEvent(H.stream, ev[2 * i + 1], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(H.state_host, H.state, sizeof(SolveState), cudaMemcpyDeviceToHost, H.stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "concurrent solve launch");
    }
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaStreamSynchronize(hs[i]->stream);
        if (e != cudaSuccess && rc == AMR_OK) rc = cuda_fail(e, "concurrent solve");
    }
    cleanup();
    if (rc != AMR_OK) return rc;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int status = AMR_OK;
    for (int i = 0; i < n; ++i) {
        Hierarchy &H = *hs[i];
        int s;
        if (!G[i]) {
            s = solve(H, &o, stats ? &stats[i] : nullptr);
            if (s != AMR_OK && s != AMR_ENOCONV) return s;
        } else {
            const SolveState &st = *H.state_host;
            H.launches += G[i]->n_init + G[i]->n_tail + (int64_t)st.iters * G[i]->n_body;
            s = st.worst <= o.eps ? AMR_OK : AMR_ENOCONV;
            if (stats) {
                amr_solve_stats &out = stats[i];
                memset(&out, 0, sizeof(out));
                out.iters = st.iters;
                out.status = s;
                out.n_levels = H.nlev;
                for (int l = 0; l < H.nlev; ++l) out.rel_res[l] = st.rel[l];
                out.ms_total = ms;
            }
        }
        if (s != AMR_OK) status = AMR_ENOCONV;
    }
    if (status != AMR_OK) set_error("a hierarchy did not converge within max_iter V-cycles");
    return status;
}

int deposit(Hierarchy &H, const double *x, const double *y, const double *z, const double *q, int64_t n)
{
    for (int l = 0; l < H.nlev; ++l) launch_fill(H, H.L[l].rho, 0.0, H.L[l].g.ncell);
    launch_deposit(H, x, y, z, q, n, -1);
    return check_launch(H, "deposit");
}

// Dense level layout <-> padded device box.
int level_copy(Hierarchy &H, int level, int field, double *host, const double *hin)
{
    if (level < 0 || level >= H.nlev) {
        set_error("level out of range");
        return AMR_EINVAL;
    }
    Level &L = H.L[level];
    double *src = nullptr;
    switch (field) {
    case AMR_RHO: src = L.rho; break;
    case AMR_PHI: src = L.phi; break;
    case AMR_RES: src = L.res; break;
    case AMR_EX: src = L.ef[0]; break;
    case AMR_EY: src = L.ef[1]; break;
    case AMR_EZ: src = L.ef[2]; break;
    default: set_error("unknown field"); return AMR_EINVAL;
    }
    const Grid &g = L.g;
    std::vector<double> buf((size_t)g.ncell);
    cudaError_t e = cudaMemcpyAsync(buf.data(), src, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, H.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H.stream);
    if (e != cudaSuccess) return cuda_fail(e, "level copy");
    int nx = g.n[0] - 2, ny = g.n[1] - 2, nz = g.n[2] - 2;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t p = (int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1);
                int64_t o = ((int64_t)k * ny + j) * nx + i;
                bool valid = L.hmask[p] != 0;
                if (hin) {
                    if (valid) buf[p] = hin[o];
                } else {
                    host[o] = valid ? buf[p] : 0.0;
                }
            }
    if (hin) {
        e = cudaMemcpyAsync(src, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, H.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(H.stream);
        if (e != cudaSuccess) return cuda_fail(e, "level copy");
    }
    return AMR_OK;
}

} // namespace
} // namespace amr

using amr::Hierarchy;


extern "C" {

int amr_desc_default(amr_desc *d)
{
    if (!d) return AMR_EINVAL;
    memset(d, 0, sizeof(*d));
    d->n0 = 64;
    d->max_level = 0;
    d->brick = 8;
    d->tag_mode = AMR_TAG_REL_RHO;
    d->tag_lambda = 0.1;
    d->buffer_cells = 1;
    d->precision = AMR_FP64;
    d->eps0 = 1.0;
    d->bc = AMR_BC_DIRICHLET;
    d->robin_d = 0.0;
    return AMR_OK;
}

int amr_solve_opts_default(amr_solve_opts *o)
{
    if (!o) return AMR_EINVAL;
    o->eps = 1e-10;
    o->norm = AMR_NORM_2;
    o->max_iter = 100;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->bottom_cycles = 2;
    o->warm_start = 0;
    o->use_graph = 1;
    o->persistent = 0;
    return AMR_OK;
}

int amr_create_hierarchy(const amr_desc *desc, const double *x, const double *y, const double *z, const double *q,
                         int64_t n, void *cuda_stream, amr_hierarchy **out)
{
    amr::set_error("");
    if (!out) {
        amr::set_error("null output");
        return AMR_EINVAL;
    }
    *out = nullptr;
    Hierarchy *H = nullptr;
    int rc = amr::create_hierarchy(desc, x, y, z, q, n, cuda_stream, &H);
    if (rc != AMR_OK) return rc;
    int outside = 0;
    cudaMemcpyAsync(&outside, H->outside, sizeof(int), cudaMemcpyDeviceToHost, H->stream);
    cudaStreamSynchronize(H->stream);
    if (outside > 0 && n > 0) {
        amr::set_error(std::to_string(outside) + " particles have cloud-in-cell nodes outside level 0");
        amr::free_hierarchy(H);
        return AMR_EOUTSIDE;
    }
    *out = new amr_hierarchy{H};
    return AMR_OK;
}

void amr_destroy(amr_hierarchy *h)
{
    if (!h) return;
    amr::free_hierarchy(h->H);
    delete h;
}

int amr_deposit(amr_hierarchy *h, const double *x, const double *y, const double *z, const double *q, int64_t n)
{
    if (!h || n < 0 || (n > 0 && (!x || !y || !z || !q))) {
        amr::set_error("invalid deposit arguments");
        return AMR_EINVAL;
    }
    return amr::deposit(*h->H, x, y, z, q, n);
}

int amr_solve(amr_hierarchy *h, const amr_solve_opts *opts, amr_solve_stats *stats)
{
    if (!h) {
        amr::set_error("null hierarchy");
        return AMR_EINVAL;
    }
    return amr::solve(*h->H, opts, stats);
}

int amr_solve_many(amr_hierarchy *const *hs, int n, const amr_solve_opts *opts, int n_streams,
                   amr_solve_stats *stats)
{
    amr::set_error("");
    if (!hs || n <= 0 || n_streams < 1) {
        amr::set_error("invalid arguments (hierarchies, n >= 1, n_streams >= 1)");
        return AMR_EINVAL;
    }
    std::vector<Hierarchy *> v;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) {
            amr::set_error("null hierarchy");
            return AMR_EINVAL;
        }
        for (Hierarchy *p : v)
            if (p == hs[i]->H) {
                amr::set_error("a hierarchy appears twice");
                return AMR_EINVAL;
            }
        v.push_back(hs[i]->H);
    }
    return amr::solve_many(v.data(), n, opts, n_streams, stats);
}

int amr_gather(amr_hierarchy *h, const double *x, const double *y, const double *z, int64_t n, double *ex,
               double *ey, double *ez, double *phi)
{
    if (!h || n < 0 || (n > 0 && (!x || !y || !z || !ex || !ey || !ez))) {
        amr::set_error("invalid gather arguments");
        return AMR_EINVAL;
    }
    amr::launch_gather(*h->H, x, y, z, n, ex, ey, ez, phi);
    return amr::check_launch(*h->H, "gather");
}

int amr_bin(amr_hierarchy *h, const double *x, const double *y, const double *z, int64_t n, uint32_t *keys,
            int64_t *perm, int64_t *nkeys_out)
{
    if (!h || !nkeys_out || n < 0 || n > 0x7fffffffLL || (n > 0 && (!x || !y || !z || !keys || !perm))) {
        amr::set_error("invalid binning arguments");
        return AMR_EINVAL;
    }
    const int64_t nk = amr::bin_num_keys(*h->H);
    if (nk >= 0x7fffffffLL) {
        amr::set_error("binning: too many bricks");
        return AMR_EINVAL;
    }
    *nkeys_out = nk;
    int rc = amr::launch_bin(*h->H, x, y, z, n, keys, perm);
    if (rc != AMR_OK) return rc;
    return amr::check_launch(*h->H, "binning");
}

int amr_step(amr_hierarchy *h, const double *x_host, const double *y_host, const double *z_host,
             const double *q_host, int64_t n, const amr_solve_opts *opts, double *ex_host, double *ey_host,
             double *ez_host, amr_solve_stats *stats)
{
    if (!h || n <= 0 || !x_host || !y_host || !z_host || !q_host || !ex_host || !ey_host || !ez_host) {
        amr::set_error("invalid step arguments");
        return AMR_EINVAL;
    }
    Hierarchy &H = *h->H;
    if (H.stage_n < n) {
        if (H.stage) {
            cudaStreamSynchronize(H.stream);
            cudaFree(H.stage);
            H.device_bytes -= H.stage_n * 7 * (int64_t)sizeof(double);
            H.stage = nullptr;
            H.stage_n = 0;
        }
        if (cudaMalloc(&H.stage, sizeof(double) * 7 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            amr::set_error("out of memory (staging)");
            return AMR_ENOMEM;
        }
        H.stage_n = n;
        H.device_bytes += n * 7 * (int64_t)sizeof(double);
    }
    if (!H.cstream) {
        bool ok = cudaStreamCreateWithFlags(&H.cstream, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t &ev : H.cev) ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return amr::cuda_fail(cudaGetLastError(), "step streams");
    }
    double *d[7];
    for (int i = 0; i < 7; ++i) d[i] = H.stage + (size_t)i * n;
    // Copy pipeline: the particles travel in up to kStepChunks chunks on the
    // copy stream, and the deposit of chunk c (hierarchy stream) waits only
    // for chunk c, so the copy of chunk c + 1 runs under it; likewise E of
    // chunk c goes back while chunk c + 1 is gathered.  The deposit's FP64
    // sums take the particles in another order than one launch would (the
    // order of its atomic additions is unspecified either way).
    const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(amr::kStepChunks, n >> 20));
    const int64_t per = (n + nch - 1) / nch;
    cudaEvent_t *ev = H.cev;
    cudaEventRecord(ev[2 * amr::kStepChunks], H.stream); // earlier work on the staging arrays
    cudaStreamWaitEvent(H.cstream, ev[2 * amr::kStepChunks], 0);
    const double *src[4] = {x_host, y_host, z_host, q_host};
    for (int c = 0; c < nch; ++c) {
        const int64_t o = c * per, m = std::min<int64_t>(per, n - o);
        for (int i = 0; i < 4; ++i)
            cudaMemcpyAsync(d[i] + o, src[i] + o, sizeof(double) * m, cudaMemcpyHostToDevice, H.cstream);
        cudaEventRecord(ev[c], H.cstream);
    }
    cudaMemsetAsync(H.outside, 0, sizeof(int), H.stream);
    for (int l = 0; l < H.nlev; ++l) amr::launch_fill(H, H.L[l].rho, 0.0, H.L[l].g.ncell);
    for (int c = 0; c < nch; ++c) {
        const int64_t o = c * per, m = std::min<int64_t>(per, n - o);
        cudaStreamWaitEvent(H.stream, ev[c], 0);
        amr::launch_deposit(H, d[0] + o, d[1] + o, d[2] + o, d[3] + o, m, -1);
    }
    int rc = amr::check_launch(H, "deposit");
    if (rc != AMR_OK) return rc;
    int src_rc = amr::solve(H, opts, stats);
    if (src_rc != AMR_OK && src_rc != AMR_ENOCONV) return src_rc;
    double *dst[3] = {ex_host, ey_host, ez_host};
    for (int c = 0; c < nch; ++c) {
        const int64_t o = c * per, m = std::min<int64_t>(per, n - o);
        amr::launch_gather(H, d[0] + o, d[1] + o, d[2] + o, m, d[4] + o, d[5] + o, d[6] + o, nullptr);
        cudaEventRecord(ev[amr::kStepChunks + c], H.stream);
        cudaStreamWaitEvent(H.cstream, ev[amr::kStepChunks + c], 0);
        for (int i = 0; i < 3; ++i)
            cudaMemcpyAsync(dst[i] + o, d[4 + i] + o, sizeof(double) * m, cudaMemcpyDeviceToHost, H.cstream);
    }
    cudaEventRecord(ev[2 * amr::kStepChunks + 1], H.cstream);
    cudaStreamWaitEvent(H.stream, ev[2 * amr::kStepChunks + 1], 0);
    cudaError_t e = cudaStreamSynchronize(H.stream);
    if (e != cudaSuccess) return amr::cuda_fail(e, "step");
    int outside = 0;
    cudaMemcpyAsync(&outside, H.outside, sizeof(int), cudaMemcpyDeviceToHost, H.stream);
    cudaStreamSynchronize(H.stream);
    if (outside > 0) {
        amr::set_error(std::to_string(outside) + " particles have cloud-in-cell nodes outside level 0");
        return AMR_EOUTSIDE;
    }
    return src_rc;
}

int amr_residual(amr_hierarchy *h, int norm, double *rel_out_host)
{
    if (!h || !rel_out_host || (norm != AMR_NORM_INF && norm != AMR_NORM_1 && norm != AMR_NORM_2)) {
        amr::set_error("invalid residual arguments");
        return AMR_EINVAL;
    }
    Hierarchy &H = *h->H;
    H.params_host->eps = 0.0;
    H.params_host->norm = norm;
    H.params_host->max_iter = 0;
    cudaMemcpyAsync(H.params, H.params_host, sizeof(amr::SolveParams), cudaMemcpyHostToDevice, H.stream);
    amr::residual_all(H);
    amr::launch_norms_check(H, 1, 0, 0, 0);
    int rc = amr::check_launch(H, "residual");
    if (rc == AMR_OK) rc = amr::read_state(H);
    if (rc != AMR_OK) return rc;
    for (int l = 0; l < H.nlev; ++l) rel_out_host[l] = H.state_host->rel[l];
    return AMR_OK;
}

int amr_field_from_phi(amr_hierarchy *h)
{
    if (!h) return AMR_EINVAL;
    amr::field(*h->H);
    cudaError_t e = cudaStreamSynchronize(h->H->stream);
    return e == cudaSuccess ? AMR_OK : amr::cuda_fail(e, "field");
}

int amr_num_levels(const amr_hierarchy *h, int *n_levels)
{
    if (!h || !n_levels) return AMR_EINVAL;
    *n_levels = h->H->nlev;
    return AMR_OK;
}

int amr_level_box(const amr_hierarchy *h, int level, int lo[3], int hi[3], int64_t *n_valid)
{
    if (!h || level < 0 || level >= h->H->nlev || !lo || !hi) {
        amr::set_error("invalid level");
        return AMR_EINVAL;
    }
    const amr::Level &L = h->H->L[level];
    for (int d = 0; d < 3; ++d) {
        lo[d] = L.vlo[d];
        hi[d] = L.vhi[d];
    }
    if (n_valid) *n_valid = L.nvalid;
    return AMR_OK;
}

int amr_get_level(amr_hierarchy *h, int level, int field, double *out_host)
{
    if (!h || !out_host) return AMR_EINVAL;
    return amr::level_copy(*h->H, level, field, out_host, nullptr);
}

int amr_set_level(amr_hierarchy *h, int level, int field, const double *in_host)
{
    if (!h || !in_host) return AMR_EINVAL;
    return amr::level_copy(*h->H, level, field, nullptr, in_host);
}

int amr_get_mask(amr_hierarchy *h, int level, int8_t *out_host)
{
    if (!h || !out_host || level < 0 || level >= h->H->nlev) return AMR_EINVAL;
    const amr::Level &L = h->H->L[level];
    const amr::Grid &g = L.g;
    int nx = g.n[0] - 2, ny = g.n[1] - 2, nz = g.n[2] - 2;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                out_host[((int64_t)k * ny + j) * nx + i] =
                    (int8_t)L.hmask[(int64_t)(k + 1) * g.sz + (int64_t)(j + 1) * g.sy + (i + 1)];
    return AMR_OK;
}

int amr_ghost_stats(const amr_hierarchy *h, int64_t out_host[3])
{
    if (!h || !out_host) return AMR_EINVAL;
    for (int i = 0; i < 3; ++i) out_host[i] = 0;
    for (int l = 1; l < h->H->nlev; ++l)
        for (int i = 0; i < 3; ++i) out_host[i] += h->H->L[l].cf.counts[i];
    return AMR_OK;
}

int amr_hierarchy_bytes(const amr_desc *desc, double fill, int64_t *bytes_out)
{
    if (!desc || !bytes_out || !(fill > 0.0)) return AMR_EINVAL;
    *bytes_out = amr::hierarchy_bytes_estimate(desc, fill);
    return AMR_OK;
}

int amr_device_bytes(const amr_hierarchy *h, int64_t *bytes_out)
{
    if (!h || !bytes_out) return AMR_EINVAL;
    *bytes_out = h->H->device_bytes;
    return AMR_OK;
}

int amr_kernel_launches(const amr_hierarchy *h, int64_t *count_out)
{
    if (!h || !count_out) return AMR_EINVAL;
    *count_out = h->H->launches;
    return AMR_OK;
}

int amr_bottom_solver(const amr_hierarchy *h, int *kind_out)
{
    if (!h || !kind_out) return AMR_EINVAL;
    *kind_out = h->H->dst_on ? AMR_BOTTOM_EXACT : AMR_BOTTOM_GMG;
    return AMR_OK;
}

int amr_profile(amr_hierarchy *h, int enable)
{
    if (!h || enable < 0 || enable > 2) return AMR_EINVAL;
    Hierarchy &H = *h->H;
    int rc = amr::prof_resolve(H);
    if (rc != AMR_OK) return rc;
    H.prof_mode = enable;
    // mode 2 unrolls the profiled graph to the last solve's V-cycle count
    H.prof_iters = enable == 2 ? std::max(1, H.state_host ? H.state_host->iters : 1) : 0;
    if (enable) {
        for (int k = 0; k < amr::K_NUM; ++k) {
            H.kind_ms[k] = 0.0;
            H.kind_bytes[k] = 0.0;
            H.kind_flops[k] = 0.0;
            H.kind_ops[k] = 0.0;
            H.kind_launches[k] = 0;
        }
    }
    H.prof = enable != 0;
    return AMR_OK;
}

int amr_profile_num_kinds(void) { return amr::K_NUM; }

const char *amr_profile_kind_name(int kind) { return amr::kind_name(kind); }

int amr_profile_read_ops(amr_hierarchy *h, int kind, double *alg_ops)
{
    if (!h || !alg_ops || kind < 0 || kind >= amr::K_NUM) return AMR_EINVAL;
    Hierarchy &H = *h->H;
    int rc = amr::prof_resolve(H);
    if (rc != AMR_OK) return rc;
    *alg_ops = H.kind_ops[kind];
    return AMR_OK;
}

int amr_profile_read_flops(amr_hierarchy *h, int kind, double *alg_flops)
{
    if (!h || !alg_flops || kind < 0 || kind >= amr::K_NUM) return AMR_EINVAL;
    Hierarchy &H = *h->H;
    int rc = amr::prof_resolve(H);
    if (rc != AMR_OK) return rc;
    *alg_flops = H.kind_flops[kind];
    return AMR_OK;
}

int amr_profile_read(amr_hierarchy *h, int kind, double *ms_total, int64_t *launches, double *alg_bytes)
{
    if (!h || kind < 0 || kind >= amr::K_NUM) return AMR_EINVAL;
    Hierarchy &H = *h->H;
    int rc = amr::prof_resolve(H);
    if (rc != AMR_OK) return rc;
    if (ms_total) *ms_total = H.kind_ms[kind];
    if (launches) *launches = H.kind_launches[kind];
    if (alg_bytes) *alg_bytes = H.kind_bytes[kind];
    return AMR_OK;
}

// A batch is one CUDA graph captured at creation and replayed by every
// amr_batch_solve.  Default (AMR_BATCH unset or "graphs"): every
// hierarchy's captured solve -- parameter upload, init, the device-side
// V-cycle loop, field, state read-back -- as an independent branch of that
// graph, the same kernels as its own solve graph, the branches running side
// by side.  AMR_BATCH=clusters: the hierarchies' recorded solves as one
// persistent cluster program (k_cluster_program), the graph holding the
// uploads, the queue reset, the kernel and the read-backs.  AMR_BATCH=rounds:
// the cooperative program of lock-step rounds (k_program), launched
// directly.
enum BatchMode { kBatchGraphs = 0, kBatchClusters = 1, kBatchRounds = 2 };

struct amr_batch {
    std::vector<Hierarchy *> hs;
    amr::Program prog;
    amr::ClusterProgram cprog;
    int mode = kBatchGraphs;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> nfixed, nbody; // kernel nodes of each branch: outside and inside the loop
    amr_solve_opts opts;
    cudaStream_t stream;
};

namespace {

// The hierarchies' solves as independent branches of one graph (see
// amr_batch).
int batch_branches(amr_batch *b, const amr::Opts &so, bool warm)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return amr::cuda_fail(e, "batch graph");
    int rc = AMR_OK;
    for (Hierarchy *H : b->hs) {
        int64_t n[3] = {0, 0, 0};
        if ((rc = amr::capture_solve_into(*H, g, so, warm, true, n)) != AMR_OK) break;
        b->nfixed.push_back(n[0] + n[2]);
        b->nbody.push_back(n[1]);
    }
    if (rc == AMR_OK) {
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            rc = amr::cuda_fail(e, "batch graph instantiate");
        }
    }
    cudaGraphDestroy(g);
    return rc;
}

// Capture the cluster program's whole launch into b->exec (see amr_batch).
int batch_graph(amr_batch *b)
{
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return amr::cuda_fail(e, "batch graph stream");
    cudaGraph_t g = nullptr;
    int rc = AMR_OK;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (Hierarchy *H : b->hs)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(H->params, H->params_host, sizeof(amr::SolveParams), cudaMemcpyHostToDevice, cap);
        if (e == cudaSuccess) rc = amr::cluster_run(b->cprog, cap);
        for (Hierarchy *H : b->hs)
            if (e == cudaSuccess && rc == AMR_OK)
                e = cudaMemcpyAsync(H->state_host, H->state, sizeof(amr::SolveState), cudaMemcpyDeviceToHost, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && rc == AMR_OK) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (rc != AMR_OK) return rc;
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return amr::cuda_fail(e, "batch graph");
    }
    return AMR_OK;
}

} // namespace

int amr_batch_create(amr_hierarchy *const *hs, int n, const amr_solve_opts *opts, amr_batch **out)
{
    if (!hs || n <= 0 || !out) {
        amr::set_error("invalid batch arguments");
        return AMR_EINVAL;
    }
    *out = nullptr;
    amr_solve_opts o;
    amr_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.nu_pre < 0 || o.nu_post < 0 || o.bottom_cycles < 1 ||
        (o.norm != AMR_NORM_INF && o.norm != AMR_NORM_1 && o.norm != AMR_NORM_2) || !(o.eps >= 0.0)) {
        amr::set_error("invalid solve options");
        return AMR_EINVAL;
    }
    amr_batch *b = new amr_batch();
    b->opts = o;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) {
            delete b;
            amr::set_error("null hierarchy in batch");
            return AMR_EINVAL;
        }
        if (hs[i]->H->periodic) {
            delete b;
            amr::set_error("periodic hierarchies are solved one at a time (amr_solve), not in a batch");
            return AMR_EINVAL;
        }
        for (Hierarchy *p : b->hs)
            if (p == hs[i]->H) {
                delete b;
                amr::set_error("a hierarchy appears twice in the batch");
                return AMR_EINVAL;
            }
        b->hs.push_back(hs[i]->H);
    }
    b->stream = b->hs[0]->stream;
    const char *mode = getenv("AMR_BATCH");
    b->mode = !mode ? kBatchGraphs
                    : (!strcmp(mode, "rounds") ? kBatchRounds : (!strcmp(mode, "clusters") ? kBatchClusters : kBatchGraphs));
    amr::Opts so{o.nu_pre, o.nu_post, o.bottom_cycles};
    for (Hierarchy *H : b->hs) {
        H->params_host->eps = o.eps;
        H->params_host->norm = o.norm;
        H->params_host->max_iter = o.max_iter;
    }
    if (b->mode == kBatchGraphs) {
        int rc = batch_branches(b, so, o.warm_start != 0);
        if (rc != AMR_OK) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            delete b;
            return rc;
        }
        *out = b;
        return AMR_OK;
    }
    const bool clusters = b->mode == kBatchClusters;
    amr::ProgramRecorder *R = amr::recorder_new(n);
    std::vector<amr::SolveState *> states;
    std::vector<double> work;
    for (int i = 0; i < n; ++i) {
        amr::record_solve(*b->hs[i], R, i, so, o.warm_start != 0);
        states.push_back(b->hs[i]->state);
        double cells = 0.0;
        for (int l = 0; l < b->hs[i]->nlev; ++l) cells += (double)b->hs[i]->L[l].nvalid;
        work.push_back(cells);
    }
    int rc = clusters ? amr::cluster_compile(R, states.data(), work.data(), n, b->stream, b->cprog)
                      : amr::program_compile(R, states.data(), n, b->stream, b->prog);
    amr::recorder_delete(R);
    if (rc == AMR_OK && clusters) rc = batch_graph(b);
    if (rc != AMR_OK) {
        amr::cluster_free(b->cprog);
        amr::program_free(b->prog);
        delete b;
        return rc;
    }
    *out = b;
    return AMR_OK;
}

int amr_batch_solve(amr_batch *b, amr_solve_stats *stats)
{
    if (!b) {
        amr::set_error("null batch");
        return AMR_EINVAL;
    }
    auto t0 = std::chrono::steady_clock::now();
    for (Hierarchy *H : b->hs) {
        if (H->stream != b->stream) {
            cudaError_t e = cudaStreamSynchronize(H->stream);
            if (e != cudaSuccess) return amr::cuda_fail(e, "batch");
        }
        H->params_host->eps = b->opts.eps;
        H->params_host->norm = b->opts.norm;
        H->params_host->max_iter = b->opts.max_iter;
        if (b->mode == kBatchRounds)
            cudaMemcpyAsync(H->params, H->params_host, sizeof(amr::SolveParams), cudaMemcpyHostToDevice, b->stream);
    }
    if (b->mode != kBatchRounds) {
        // the captured launch reads the parameters from and writes the
        // states to the hierarchies' pinned host copies
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return amr::cuda_fail(e, "batch");
        if (b->mode == kBatchClusters) {
            b->hs[0]->launches++;
        } else {
            for (size_t i = 0; i < b->hs.size(); ++i)
                b->hs[i]->launches += b->nfixed[i] + b->nbody[i] * b->hs[i]->state_host->iters;
        }
    } else {
        int rc = amr::program_run(*b->hs[0], b->prog, b->stream, 2000000000ull, 0);
        if (rc != AMR_OK) return rc;
        if ((rc = amr::program_status(b->prog, b->stream)) != AMR_OK) return rc;
        for (size_t i = 0; i < b->hs.size(); ++i) {
            Hierarchy &H = *b->hs[i];
            cudaMemcpyAsync(H.state_host, H.state, sizeof(amr::SolveState), cudaMemcpyDeviceToHost, b->stream);
        }
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return amr::cuda_fail(e, "batch");
    }
    int status = AMR_OK;
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (size_t i = 0; i < b->hs.size(); ++i) {
        Hierarchy &H = *b->hs[i];
        const amr::SolveState &st = *H.state_host;
        int s = st.worst <= b->opts.eps ? AMR_OK : AMR_ENOCONV;
        if (s != AMR_OK) status = AMR_ENOCONV;
        if (stats) {
            amr_solve_stats &o = stats[i];
            memset(&o, 0, sizeof(o));
            o.iters = st.iters;
            o.status = s;
            o.n_levels = H.nlev;
            for (int l = 0; l < H.nlev; ++l) o.rel_res[l] = st.rel[l];
            o.ms_total = ms;
        }
    }
    if (status != AMR_OK) amr::set_error("a hierarchy of the batch did not converge within max_iter");
    return status;
}

void amr_batch_destroy(amr_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    amr::cluster_free(b->cprog);
    amr::program_free(b->prog);
    delete b;
}

int amr_selftest_barrier_timeout(amr_hierarchy *h, int limit_ms)
{
    if (!h || limit_ms <= 0 || limit_ms > 10000) {
        amr::set_error("invalid self-test arguments");
        return AMR_EINVAL;
    }
    Hierarchy &H = *h->H;
    amr_solve_opts o;
    amr_solve_opts_default(&o);
    amr::Opts so{o.nu_pre, o.nu_post, o.bottom_cycles};
    int rc = amr::ensure_program(H, so, false);
    if (rc != AMR_OK) return rc;
    // one block more than launched is expected at every barrier, so no
    // barrier completes and every wait runs out after limit_ms
    rc = amr::program_run(H, H.prog, H.stream, (unsigned long long)limit_ms * 1000000ull, 1 << 30);
    if (rc != AMR_OK) return rc;
    return amr::program_status(H.prog, H.stream);
}

const char *amr_last_error(void) { return amr::g_error.c_str(); }

} // extern "C"
