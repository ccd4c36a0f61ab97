// C ABI of the GSIS library: context, argument checking, mesh set-up, and the
// orchestration of one GSIS iteration (Sec. 3.1 steps; Sec. 3.4 for the
// adaptive start).  Every numerical step runs in the kernels of the other
// translation units; this file only moves descriptors and launches them.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include "sweep_device.cuh"

using namespace gsis;

namespace gsis {

gsis_status set_err(gsis_ctx* c, gsis_status s, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (s == GSIS_ERR_CUDA || s == GSIS_ERR_NONFINITE || s == GSIS_ERR_INTERNAL || s == GSIS_ERR_TIMEOUT)
            c->broken = true;
    }
    return s;
}

bool cuda_ok(gsis_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    set_err(c, GSIS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

void* dev_alloc(gsis_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (c->have_alloc) {
        p = c->alloc.alloc(bytes, (void*)c->stream, c->alloc.user);
    } else {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (p) c->allocations.push_back(p);
    return p;
}

void dev_free(gsis_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
    if (it == c->allocations.end()) return;
    c->allocations.erase(it);
    if (c->have_alloc) c->alloc.free(p, (void*)c->stream, c->alloc.user);
    else cudaFree(p);
}

size_t vdf_elem_bytes(int dtype) {
    switch (dtype) {
        case GSIS_F64: return 8;
        case GSIS_F32: return 4;
        default: return 2;
    }
}

}  // namespace gsis

namespace {

template <typename T>
T* upload(gsis_ctx* c, const std::vector<T>& h) {
    T* d = (T*)dev_alloc(c, h.size() * sizeof(T));
    if (!d) return nullptr;
    if (cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return nullptr;
    return d;
}

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Solve the dim x dim normal equations G x = b (Gaussian elimination, partial pivoting).
bool solve_small(int n, double G[3][3], double b[3], double x[3]) {
    double A[3][4];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) A[i][j] = G[i][j];
        A[i][n] = b[i];
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return false;
        if (piv != col)
            for (int k = 0; k <= n; ++k) std::swap(A[col][k], A[piv][k]);
        for (int r = col + 1; r < n; ++r) {
            const double m = A[r][col] / A[col][col];
            for (int k = col; k <= n; ++k) A[r][k] -= m * A[col][k];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = A[r][n];
        for (int k = r + 1; k < n; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return true;
}

void phase_begin(gsis_ctx* c, int ph) {
    if (c->events) cudaEventRecord(c->ev[2 * ph], c->stream);
}
void phase_end(gsis_ctx* c, int ph) {
    if (c->events) cudaEventRecord(c->ev[2 * ph + 1], c->stream);
}
void phase_collect(gsis_ctx* c, const bool* used) {
    if (!c->events) return;
    for (int ph = 0; ph < GSIS_NPHASE; ++ph) {
        if (!used[ph]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[2 * ph], c->ev[2 * ph + 1]) == cudaSuccess) c->phase_ms[ph] += ms;
    }
}

gsis_status check_ctx(gsis_ctx* c) {
    if (!c) return GSIS_ERR_ARG;
    if (c->broken) return set_err(c, GSIS_ERR_STATE, "context is unusable after an earlier error: " + c->err);
    return GSIS_OK;
}

// ---------------------------------------------------------------------------- start-up (Sec. 3.4 Steps 1-2)
gsis_status presolve(gsis_ctx* c) {
    const int N = c->m.N;
    cudaMemsetAsync(c->hot, 0, (size_t)N * HOTN * sizeof(double), c->stream);
    cudaMemsetAsync(c->wall_corr, 0, (size_t)N * 30 * sizeof(double), c->stream);   // plain NSF walls
    launch_prim_to_cons(c, c->W, c->U);
    cudaMemcpyAsync(c->Wm, c->W, (size_t)N * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    c->presolve_blocks = 0;
    *c->h_err = 0;
    for (int b = 0; b < c->p.presolve_max_blocks; ++b) {
        cudaMemcpyAsync(c->Wp, c->Wm, (size_t)N * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
        macro_block(c, c->p.macro_steps, false, false);
        launch_eps(c, c->Wm, c->Wp);
        cudaMemcpyAsync(c->h_eps, c->eps_buf, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "presolve")) return GSIS_ERR_CUDA;
        if (*c->h_err != 0)
            return set_err(c, GSIS_ERR_TIMEOUT, "a grid barrier of the synthetic solve ran out of spin_limit polls "
                                                "(NS presolve)");
        c->presolve_blocks = b + 1;
        if (c->h_eps[1] != 0.0) return set_err(c, GSIS_ERR_NONFINITE, "non-finite state in the NS presolve");
        if (c->h_eps[0] < c->p.tol) break;
    }
    cudaMemcpyAsync(c->W, c->Wm, (size_t)N * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    return GSIS_OK;
}

gsis_status start(gsis_ctx* c) {
    const int N = c->m.N;
    if (c->vg.reduced) {   // the reduced distributions assume a flow without z dependence and u_z = 0
        if (c->normal_components > 2)
            return set_err(c, GSIS_ERR_ARG, "reduced velocity grid needs a mesh whose faces have no z component");
        for (int q = 0; q < N; ++q)
            if (c->host_W0[(size_t)q * 5 + 3] != 0.0)
                return set_err(c, GSIS_ERR_ARG, "reduced velocity grid needs u_z = 0 in the initial state");
        for (int s = 0; s < 6; ++s)
            if (c->m.bc_type[s] == GSIS_BC_FARFIELD && c->m.bc_state[s][3] != 0.0)
                return set_err(c, GSIS_ERR_ARG, "reduced velocity grid needs u_z = 0 in the far-field states");
    }
    if (!cuda_ok(c, cudaMemcpyAsync(c->W, c->host_W0.data(), (size_t)N * 5 * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream), "upload W0"))
        return GSIS_ERR_CUDA;
    cudaMemsetAsync(c->hot, 0, (size_t)N * HOTN * sizeof(double), c->stream);
    launch_face_geometry(c);
    if (c->p.vdf_dtype != GSIS_F64) {   // FP32 copies of the boundary and ghost records for the FP32 sweep
        const size_t NT = c->vg.NT;
        c->recBC.tabf = (float*)dev_alloc(c, 6 * NTAB * NT * sizeof(float));
        c->recBC.scalf = (float*)dev_alloc(c, 6 * RS * sizeof(float));
        c->recGhost.tabf = (float*)dev_alloc(c, (size_t)N * NTAB * NT * sizeof(float));
        c->recGhost.scalf = (float*)dev_alloc(c, (size_t)N * RS * sizeof(float));
        if (!c->recBC.tabf || !c->recBC.scalf || !c->recGhost.tabf || !c->recGhost.scalf)
            return set_err(c, GSIS_ERR_OOM, "device allocation failed (FP32 record copies)");
    }
    launch_bc_records(c);
    launch_wall_den(c);
    phase_begin(c, GSIS_PH_PRESOLVE);
    if (c->p.presolve_max_blocks > 0) {   // Sec. 3.4 Step 1 (also starts an all-kinetic run)
        gsis_status s = presolve(c);
        if (s != GSIS_OK) return s;
    }
    phase_end(c, GSIS_PH_PRESOLVE);
    if (c->have_forced) {
        cudaMemcpyAsync(c->flag, c->forced_flags.data(), N, cudaMemcpyHostToDevice, c->stream);
    } else if (c->p.adaptive) {
        launch_kn_gll(c, c->W);
    } else {
        cudaMemsetAsync(c->flag, 1, N, c->stream);
    }
    {
        std::vector<int> m1(N, -1);
        cudaMemcpyAsync(c->cell2dvm, m1.data(), N * sizeof(int), cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
    }
    if (build_region(c) < 0) return c->broken ? GSIS_ERR_CUDA : GSIS_ERR_OOM;
    launch_moments(c, c->W, c->mom);
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "start")) return GSIS_ERR_CUDA;
    c->started = true;
    return GSIS_OK;
}

// ---------------------------------------------------------------------------- one GSIS iteration
// The iteration is split in stages so that the batched driver can record the
// same launches for many solves into one CUDA graph.

// 1. reference distributions, tau, interface ghosts, wall densities
void stage_cell_eq(gsis_ctx* c) {
    if (c->n_ghost > 0) {
        launch_nsf(c, c->W, c->nsf);
        launch_ghost_records(c);
    }
    launch_cell_eq(c);
}

// 3. moments of f^{n+1/2} -> W^{n+1/2}, wall fluxes, HoT; set up the synthetic solve
void stage_moments(gsis_ctx* c) {
    const int N = c->m.N;
    cudaMemcpyAsync(c->Wmom, c->W, (size_t)N * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    launch_moments(c, c->Wmom, c->momh);
    launch_wall_flux(c);
    launch_half_state(c);
    launch_nsf(c, c->Wh, c->nsf);   // leaves the gradients of W^{n+1/2} in gu, gT
    launch_hot(c);
    if (c->has_wall) launch_wall_corr(c);
    launch_prim_to_cons(c, c->Wh, c->U);
    launch_prim_to_cons(c, c->W, c->Un);
    cudaMemcpyAsync(c->Wm, c->Wh, (size_t)N * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

// 6. under-relaxation of the synthetic correction and the residual between
// W^{n+1} (Wm) and W^n (W); with fixed_buffers the new state is copied into W
// (the buffers a recorded graph refers to stay the same), else swapped.
void stage_residual(gsis_ctx* c, bool fixed_buffers) {
    if (c->p.relax != 1.0) launch_blend(c, c->Wh, c->p.relax, c->Wm);
    launch_eps(c, c->Wm, c->W);
    if (fixed_buffers) {
        cudaMemcpyAsync(c->W, c->Wm, (size_t)c->m.N * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    } else {
        cudaMemcpyAsync(c->h_eps, c->eps_buf, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        std::swap(c->W, c->Wm);   // W = W^{n+1}
    }
}

// 5. Eq. updatef in DVM cells, and moments of f^{n+1} about u^{n+1}
void stage_correct(gsis_ctx* c) {
    launch_correction_records(c);
    launch_correct(c);
}

gsis_status gsis_step(gsis_ctx* c, double* eps_out, bool* used) {
    *c->h_err = 0;   // barrier error word of a persistent synthetic-solve launch (written back by it)
    if (c->p.adaptive && c->iteration == c->p.adapt_every && !c->have_forced) {
        used[GSIS_PH_ADAPT] = true;
        phase_begin(c, GSIS_PH_ADAPT);
        launch_kn_gll(c, c->W);
        if (build_region(c) < 0) return c->broken ? GSIS_ERR_CUDA : GSIS_ERR_OOM;
        launch_moments(c, c->W, c->mom);
        phase_end(c, GSIS_PH_ADAPT);
    }
    used[GSIS_PH_CELLEQ] = true;
    phase_begin(c, GSIS_PH_CELLEQ);
    stage_cell_eq(c);
    phase_end(c, GSIS_PH_CELLEQ);
    // (re)tune the sweep tile for a new region; a re-identification that changes the DVM cell
    // count by less than a quarter keeps the shape (the timings hardly move)
    const bool retune = c->sweep_shape < 0 || c->tuned_Nd <= 0 ||
                        std::llabs(c->Nd - c->tuned_Nd) * 4 > c->tuned_Nd;
    if (!c->sweep_forced && retune) {
        gsis_status st = tune_sweep(c);
        if (st != GSIS_OK) return st;
    }
    // 2. kinetic step: backward (towards the low-index walls) then forward Gauss-Seidel pass
    used[GSIS_PH_SWEEP] = true;
    phase_begin(c, GSIS_PH_SWEEP);
    launch_sweep(c, 1);
    launch_wall_rho(c);
    launch_sweep(c, 0);
    phase_end(c, GSIS_PH_SWEEP);
    used[GSIS_PH_MOMENTS] = true;
    phase_begin(c, GSIS_PH_MOMENTS);
    stage_moments(c);
    phase_end(c, GSIS_PH_MOMENTS);
    // 4. synthetic solve over all cells from W^{n+1/2}
    used[GSIS_PH_MACRO] = true;
    phase_begin(c, GSIS_PH_MACRO);
    macro_block(c, c->p.macro_steps, true, c->p.dt > 0.0);
    phase_end(c, GSIS_PH_MACRO);
    used[GSIS_PH_RESID] = true;
    phase_begin(c, GSIS_PH_RESID);
    stage_residual(c, false);
    phase_end(c, GSIS_PH_RESID);
    used[GSIS_PH_CORRECT] = true;
    phase_begin(c, GSIS_PH_CORRECT);
    stage_correct(c);
    phase_end(c, GSIS_PH_CORRECT);
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "GSIS iteration")) return GSIS_ERR_CUDA;
    if (!cuda_ok(c, cudaGetLastError(), "kernel launch")) return GSIS_ERR_CUDA;
    if (*c->h_err != 0)
        return set_err(c, GSIS_ERR_TIMEOUT, "a grid barrier of the synthetic solve ran out of spin_limit polls "
                                            "in iteration " + std::to_string(c->iteration));
    if (c->h_eps[1] != 0.0)
        return set_err(c, GSIS_ERR_NONFINITE, "non-finite or non-positive density/temperature after iteration " +
                                                  std::to_string(c->iteration));
    *eps_out = c->h_eps[0];
    c->iteration++;
    return GSIS_OK;
}


// ---------------------------------------------------------------------------- batched solves
// Many independent solves advanced together: per GSIS iteration, the
// per-solve stages of every solve, ONE persistent sweep launch over all
// (solve, velocity tile) items, and ONE fused synthetic-solve launch (one CTA
// per solve), recorded once into a CUDA graph and replayed.  The graph refers
// to fixed buffers, so in batched mode the new state is copied into W instead
// of swapping the W / Wm buffers.
struct BatchPlan {
    std::vector<gsis_ctx*> ctxs;
    std::vector<const double*> W_at_capture;   // W buffer of each solve when the graph was recorded
    gsis_ctx* owner = nullptr;                  // plan allocations go through this context
    cudaStream_t stream = nullptr;              // capture and replay stream
    bool own_stream = false;                    // created here (the solves run on the legacy default stream)
    BatchSolve* d_solves = nullptr;
    int2* d_items = nullptr;
    int n_items = 0;
    int* d_ticket = nullptr;
    MacroJob* d_jobs = nullptr;
    int n_jobs = 0;
    std::vector<int> big;                       // solves too large for the fused synthetic-solve kernel
    int nc = 1, shape = 1, grid = 0;
    int macro_cluster = 1;                      // CTAs per solve of the fused synthetic-solve launch
    bool tuned = false;
    std::vector<double> tune_ms;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // around the sweep and the whole iteration
    // Branch streams of the recorded graph: the per-solve stages of different
    // solves are independent, so they are recorded on BATCH_BRANCHES streams
    // forked from and joined back into the capture stream, which makes them
    // parallel branches of the graph (small solves' launches fill the GPU together).
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> branch_ev;        // [0]: fork, [1 + j]: join of branch j
    long long launches_per_iter = 0;
    std::string info;
};
constexpr int BATCH_BRANCHES = 16;

std::mutex& batch_mutex() {
    static std::mutex m;
    return m;
}
std::map<std::vector<gsis_ctx*>, BatchPlan*>& batch_plans() {
    static std::map<std::vector<gsis_ctx*>, BatchPlan*> m;
    return m;
}
std::map<std::string, int>& tuned_shapes() {   // autotuner cache: batch signature -> tile shape
    static std::map<std::string, int> m;
    return m;
}
int& forced_batch_shape() {   // gsis_debug_set_batch_tile: -1 = autotune
    static int s = -1;
    return s;
}

void destroy_plan(BatchPlan* P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    for (cudaEvent_t& e : P->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : P->branch_ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t st : P->branch)
        if (st) cudaStreamDestroy(st);
    if (P->own_stream && P->stream) {
        cudaStreamSynchronize(P->stream);
        cudaStreamDestroy(P->stream);
    }
    gsis_ctx* o = P->owner;
    for (void* p : {(void*)P->d_solves, (void*)P->d_items, (void*)P->d_ticket, (void*)P->d_jobs})
        if (p) dev_free(o, p);
    delete P;
}

// Items of the batch for a tile shape: all velocity tiles of each solve, the
// solves with the most DVM cells (the longest items) first.
std::vector<int2> batch_items(const std::vector<gsis_ctx*>& cs, int shape) {
    const int vt = batch_shape_vtile(shape);
    std::vector<int> order(cs.size());
    for (size_t i = 0; i < cs.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cs[a]->Nd > cs[b]->Nd; });
    std::vector<int2> items;
    for (int s : order) {
        if (cs[s]->Nd == 0) continue;
        const long long nt = (cs[s]->vg.Nv + vt - 1) / vt;
        for (long long t = 0; t < nt; ++t) items.push_back(make_int2(s, (int)t));
    }
    return items;
}

std::string batch_signature(const std::vector<gsis_ctx*>& cs, int nc) {
    std::vector<std::string> parts;
    for (gsis_ctx* c : cs)
        parts.push_back(std::to_string(c->Nd) + "x" + std::to_string(c->vg.Nv) + "x" + std::to_string(c->p.vdf_dtype) +
                        "x" + std::to_string(c->m.H));
    std::sort(parts.begin(), parts.end());
    std::string s = "nc" + std::to_string(nc);
    for (auto& p : parts) s += "|" + p;
    return s;
}

// Autotuner: time every tile shape on the batch itself (one warm-up and two
// timed launches each) on a snapshot of the VDFs, restore them, keep the
// fastest.  Cached per batch signature for the life of the process.
gsis_status tune_batch(BatchPlan* P) {
    gsis_ctx* o = P->owner;
    if (forced_batch_shape() >= 0) {   // test hook: the named shape, if this batch can run it
        bool pairs_ok = true;
        for (gsis_ctx* c : P->ctxs) pairs_ok = pairs_ok && c->p.vdf_dtype != GSIS_F64 && c->vg.nx % 2 == 0;
        if (!batch_shape_pair(forced_batch_shape()) || pairs_ok) {
            P->shape = forced_batch_shape();
            P->tuned = false;
            return GSIS_OK;
        }
        return set_err(o, GSIS_ERR_ARG, "the forced batch tile needs FP32/BF16/FP16 members with an even nx");
    }
    const std::string sig = batch_signature(P->ctxs, P->nc);
    auto hit = tuned_shapes().find(sig);
    if (hit != tuned_shapes().end()) {
        P->shape = hit->second;
        P->tuned = true;
        return GSIS_OK;
    }
    std::vector<void*> snap(P->ctxs.size(), nullptr);
    std::vector<size_t> bytes(P->ctxs.size(), 0);
    bool ok = true;
    for (size_t i = 0; i < P->ctxs.size() && ok; ++i) {
        gsis_ctx* c = P->ctxs[i];
        bytes[i] = (size_t)c->Nd * c->vg.Nv * vdf_elem_bytes(c->p.vdf_dtype);
        if (bytes[i] == 0) continue;
        snap[i] = dev_alloc(o, bytes[i]);
        if (!snap[i]) { ok = false; break; }
        cudaMemcpyAsync(snap[i], c->f, bytes[i], cudaMemcpyDeviceToDevice, P->stream);
    }
    if (!ok) {   // not enough memory for a snapshot: keep the default shape
        for (void* p : snap) if (p) dev_free(o, p);
        P->shape = 1;
        P->tuned = false;
        return GSIS_OK;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int ns = batch_num_shapes();
    P->tune_ms.assign(ns, -1.0);   // -1: shape not eligible for this batch
    int best = 1;
    double best_ms = 1e300;
    int2* d_it = nullptr;
    bool pairs_ok = true;   // the pair shapes need FP32 / BF16 / FP16 storage and an even nx in every member
    for (gsis_ctx* c : P->ctxs) pairs_ok = pairs_ok && c->p.vdf_dtype != GSIS_F64 && c->vg.nx % 2 == 0;
    for (int sh = 0; sh < ns; ++sh) {
        if (batch_shape_pair(sh) && !pairs_ok) continue;
        std::vector<int2> it = batch_items(P->ctxs, sh);
        d_it = (int2*)dev_alloc(o, std::max<size_t>(1, it.size()) * sizeof(int2));
        if (!d_it) break;
        cudaMemcpyAsync(d_it, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice, P->stream);
        const int grid = batch_grid(sh, P->nc);
        launch_sweep_batch(sh, P->nc, P->d_solves, d_it, (int)it.size(), P->d_ticket, grid, P->stream, 0, 2);
        cudaEventRecord(e0, P->stream);
        for (int r = 0; r < 2; ++r)
            launch_sweep_batch(sh, P->nc, P->d_solves, d_it, (int)it.size(), P->d_ticket, grid, P->stream, 0, 2);
        cudaEventRecord(e1, P->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        P->tune_ms[sh] = ms / 2.0;
        if (ms / 2.0 < best_ms) { best_ms = ms / 2.0; best = sh; }
        dev_free(o, d_it);
        d_it = nullptr;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t i = 0; i < P->ctxs.size(); ++i)
        if (snap[i]) cudaMemcpyAsync(P->ctxs[i]->f, snap[i], bytes[i], cudaMemcpyDeviceToDevice, P->stream);
    cudaStreamSynchronize(P->stream);
    for (void* p : snap) if (p) dev_free(o, p);
    if (!cuda_ok(o, cudaGetLastError(), "batch autotuning")) return GSIS_ERR_CUDA;
    P->shape = best;
    P->tuned = true;
    tuned_shapes()[sig] = best;
    return GSIS_OK;
}

gsis_status build_plan(BatchPlan* P) {
    gsis_ctx* o = P->owner;
    const int n = (int)P->ctxs.size();
    for (gsis_ctx* c : P->ctxs) stage_cell_eq(c);   // valid records for the autotuning sweeps
    for (gsis_ctx* c : P->ctxs)
        if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "batch set-up")) return GSIS_ERR_CUDA;
    std::vector<BatchSolve> hs(n);
    std::vector<MacroJob> jobs;
    P->nc = 1;
    for (int i = 0; i < n; ++i) {
        gsis_ctx* c = P->ctxs[i];
        hs[i].a = sweep_args(c);
        hs[i].f = c->f;
        hs[i].dtype = c->p.vdf_dtype;
        if (c->normal_components > 1) P->nc = 3;
        if (c->m.N <= MACRO_FUSED_MAX_CELLS)
            jobs.push_back(macro_job(c, c->p.macro_steps, c->p.dt > 0.0));
        else
            P->big.push_back(i);
        P->W_at_capture.push_back(c->W);
    }
    P->n_jobs = (int)jobs.size();
    {   // spread the fused synthetic solves over the SMs: clusters of up to 8 CTAs, at most one
        // resident CTA per SM (its 512 threads use the register file)
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int want = P->n_jobs > 0 ? std::max(1, sms / P->n_jobs) : 1;
        P->macro_cluster = fused_cluster_size(want);
    }
    P->d_solves = (BatchSolve*)dev_alloc(o, n * sizeof(BatchSolve));
    P->d_ticket = (int*)dev_alloc(o, sizeof(int));
    P->d_jobs = (MacroJob*)dev_alloc(o, std::max(1, P->n_jobs) * sizeof(MacroJob));
    if (!P->d_solves || !P->d_ticket || !P->d_jobs) return set_err(o, GSIS_ERR_OOM, "batch plan allocation failed");
    cudaMemcpyAsync(P->d_solves, hs.data(), n * sizeof(BatchSolve), cudaMemcpyHostToDevice, P->stream);
    if (P->n_jobs)
        cudaMemcpyAsync(P->d_jobs, jobs.data(), jobs.size() * sizeof(MacroJob), cudaMemcpyHostToDevice, P->stream);
    if (!cuda_ok(o, cudaStreamSynchronize(P->stream), "batch plan upload")) return GSIS_ERR_CUDA;
    gsis_status st = tune_batch(P);
    if (st != GSIS_OK) return st;
    std::vector<int2> items = batch_items(P->ctxs, P->shape);
    P->n_items = (int)items.size();
    P->d_items = (int2*)dev_alloc(o, std::max<size_t>(1, items.size()) * sizeof(int2));
    if (!P->d_items) return set_err(o, GSIS_ERR_OOM, "batch item list allocation failed");
    cudaMemcpyAsync(P->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, P->stream);
    P->grid = batch_grid(P->shape, P->nc);
    if (!cuda_ok(o, cudaStreamSynchronize(P->stream), "batch item upload")) return GSIS_ERR_CUDA;
    // record one GSIS iteration of every solve
    std::vector<cudaStream_t> saved(n);
    long long l0 = 0;
    for (int i = 0; i < n; ++i) {
        saved[i] = P->ctxs[i]->stream;
        P->ctxs[i]->stream = P->stream;
        l0 += P->ctxs[i]->launches;
    }
    for (cudaEvent_t& e : P->ev)
        if (!e && cudaEventCreate(&e) != cudaSuccess) return set_err(o, GSIS_ERR_CUDA, "batch timing events");
    const int nbr = std::min(n, BATCH_BRANCHES);
    while ((int)P->branch.size() < nbr) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return set_err(o, GSIS_ERR_CUDA, "batch branch stream");
        P->branch.push_back(st);
    }
    while ((int)P->branch_ev.size() < nbr + 1) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return set_err(o, GSIS_ERR_CUDA, "batch branch event");
        P->branch_ev.push_back(e);
    }
    // Record fn(solve i) for the given solves on the branch streams (solve i on
    // branch i mod nbr), between a fork from and a join into the capture stream.
    // main() is recorded on the capture stream between the fork and the join.
    auto branched = [&](const std::vector<int>& solves, auto fn, auto main) {
        cudaEventRecord(P->branch_ev[0], P->stream);
        for (int j = 0; j < nbr; ++j) cudaStreamWaitEvent(P->branch[j], P->branch_ev[0], 0);
        main();
        for (size_t t = 0; t < solves.size(); ++t) {
            gsis_ctx* c = P->ctxs[solves[t]];
            c->stream = P->branch[t % nbr];
            fn(c);
            c->stream = P->stream;
        }
        for (int j = 0; j < nbr; ++j) {
            cudaEventRecord(P->branch_ev[1 + j], P->branch[j]);
            cudaStreamWaitEvent(P->stream, P->branch_ev[1 + j], 0);
        }
    };
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    auto none = []() {};
    cudaError_t ce = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        cudaEventRecordWithFlags(P->ev[2], P->stream, cudaEventRecordExternal);
        branched(all, [](gsis_ctx* c) { stage_cell_eq(c); }, none);
        cudaEventRecordWithFlags(P->ev[0], P->stream, cudaEventRecordExternal);
        bool walls = false;
        for (gsis_ctx* c : P->ctxs) walls = walls || c->has_wall;
        if (walls) {   // wall densities refreshed between the passes
            launch_sweep_batch(P->shape, P->nc, P->d_solves, P->d_items, P->n_items, P->d_ticket, P->grid, P->stream,
                               0, 1);
            branched(all, [](gsis_ctx* c) { launch_wall_rho(c); }, none);
            launch_sweep_batch(P->shape, P->nc, P->d_solves, P->d_items, P->n_items, P->d_ticket, P->grid, P->stream,
                               1, 2);
        } else {   // both passes in one launch
            launch_sweep_batch(P->shape, P->nc, P->d_solves, P->d_items, P->n_items, P->d_ticket, P->grid, P->stream,
                               0, 2);
        }
        cudaEventRecordWithFlags(P->ev[1], P->stream, cudaEventRecordExternal);
        branched(all, [](gsis_ctx* c) { stage_moments(c); }, none);
        // the fused launch of the small solves, the large solves' synthetic solves beside it
        branched(P->big, [](gsis_ctx* c) { macro_block(c, c->p.macro_steps, true, c->p.dt > 0.0, true); },
                 [&]() {
                     if (P->n_jobs) launch_macro_fused(P->d_jobs, P->n_jobs, P->stream, P->macro_cluster);
                 });
        branched(all, [](gsis_ctx* c) {
            stage_residual(c, true);
            stage_correct(c);
        }, none);
        cudaEventRecordWithFlags(P->ev[3], P->stream, cudaEventRecordExternal);
        ce = cudaStreamEndCapture(P->stream, &P->graph);
    }
    long long l1 = 0;
    for (int i = 0; i < n; ++i) {
        l1 += P->ctxs[i]->launches;
        P->ctxs[i]->stream = saved[i];
    }
    if (ce != cudaSuccess) return set_err(o, GSIS_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&P->exec, P->graph, 0);
    if (ce != cudaSuccess)
        return set_err(o, GSIS_ERR_CUDA, std::string("batch graph instantiation: ") + cudaGetErrorString(ce));
    P->launches_per_iter = (l1 - l0) + 1 + (P->n_jobs ? 1 : 0);
    size_t nodes = 0;
    cudaGraphGetNodes(P->graph, nullptr, &nodes);
    P->info = std::string("solves=") + std::to_string(n) + " items=" + std::to_string(P->n_items) +
              " tile=" + batch_shape_name(P->shape) + (P->tuned ? " (autotuned" : " (default") +
              ") grid=" + std::to_string(P->grid) + " fused_macro=" + std::to_string(P->n_jobs) + "x" +
              std::to_string(P->macro_cluster) +
              " graph_nodes=" + std::to_string(nodes) + " kernels_per_iteration=" + std::to_string(P->launches_per_iter);
    if (!P->tune_ms.empty()) {
        P->info += " tune_ms=";
        for (int sh = 0; sh < (int)P->tune_ms.size(); ++sh)
            P->info += std::string(sh ? "," : "") + batch_shape_name(sh) + ":" + std::to_string(P->tune_ms[sh]);
    }
    return GSIS_OK;
}

void drop_plans_with(gsis_ctx* c) {
    std::lock_guard<std::mutex> lk(batch_mutex());
    auto& m = batch_plans();
    for (auto it = m.begin(); it != m.end();) {
        if (std::find(it->first.begin(), it->first.end(), c) != it->first.end()) {
            destroy_plan(it->second);
            it = m.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace

namespace {
// The kinetic update divides by 1/tau + sum_s max(xi.S_s, 0)/V.  The FP64
// sweep seeds that quotient with an FP32 reciprocal of the denominator moved
// into the FP32 exponent range by an integer rebias, and the FP32 sweep uses
// the fast FP32 quotient: both need the denominator inside the normal FP32
// range (2^-126 .. 2^127).  The host keeps it far inside: the outflow part is
// at most max|xi| * max_c sum_s |S_s|/V_c <= 2^100, and 1/tau = rho T^(1-omega)
// / mu(T0) with mu(T0) = Kn sqrt(2/pi) stays above 2^-100 for Kn <= 1e15 and
// rho T^(1-omega) >= 1e-15 (below 2^100 for Kn >= 1e-15 and rho T^(1-omega)
// <= 1e15).
constexpr double KN_MIN = 1e-15, KN_MAX = 1e15;
constexpr double QUOTIENT_OUTFLOW_MAX = 1.2676506002282294e30;   // 2^100
constexpr const char* quotient_range_msg =
    "max|xi| * max over cells of sum |S|/V exceeds 2^100: the sweep's quotient needs its denominator "
    "inside the FP32 exponent range";
bool quotient_range_ok(double max_sv, double max_xi) { return max_sv * max_xi <= QUOTIENT_OUTFLOW_MAX; }
}  // namespace

// ============================================================================ C ABI
extern "C" {

const char* gsis_version(void) { return "gsis-gb300 0.1 (sm_103a)"; }

gsis_status gsis_init(const gsis_params* params, const gsis_allocator* alloc, void* cuda_stream, gsis_ctx** out) {
    if (!out || !params) return GSIS_ERR_ARG;
    *out = nullptr;
    const gsis_params& p = *params;
    if (!(p.Kn > 0.0) || !std::isfinite(p.Kn) || !(p.omega >= 0.0) || p.macro_steps < 0 || p.k_sub < 0 ||
        !(p.cfl > 0.0) || !(p.dt >= 0.0) || p.vdf_dtype < GSIS_F64 || p.vdf_dtype > GSIS_F16 ||
        p.presolve_max_blocks < 0 || p.wall_layers < 0 || p.adapt_every < 0 || !(p.tol >= 0.0) ||
        !(p.relax >= 0.0 && p.relax <= 1.0))
        return GSIS_ERR_ARG;
    if (!(p.Kn >= KN_MIN && p.Kn <= KN_MAX)) return GSIS_ERR_UNSUPPORTED;   // see quotient_range_ok
    if (p.d_r < 0) return GSIS_ERR_ARG;
    if (p.d_r > 0) return GSIS_ERR_UNSUPPORTED;   // the two-VDF model of Eq. general_model is not built
    if (alloc && (!alloc->alloc || !alloc->free)) return GSIS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GSIS_ERR_CUDA;
    }
    gsis_ctx* c = new (std::nothrow) gsis_ctx();
    if (!c) return GSIS_ERR_OOM;
    c->p = p;
    if (c->p.relax == 0.0) c->p.relax = 1.0;
    if (c->p.spin_limit == 0) c->p.spin_limit = 1ull << 24;   // with 32 ns sleeps: about a second
    if (alloc) { c->alloc = *alloc; c->have_alloc = true; }
    c->stream = (cudaStream_t)cuda_stream;
    c->device = dev;
    c->mu0 = p.Kn * 1.0 * 1.0 / std::sqrt(PI / 2.0);   // Kn = mu(T0)/(p0 L) sqrt(pi R T0 / 2), p0 = L = T0 = 1
    for (int i = 0; i < GSIS_NPHASE; ++i) c->phase_ms[i] = 0.0;
    bool ev_ok = true;
    for (int i = 0; i < 2 * GSIS_NPHASE; ++i) ev_ok = ev_ok && cudaEventCreate(&c->ev[i]) == cudaSuccess;
    c->events = ev_ok;
    if (cudaMallocHost(&c->h_eps, 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_count, 4 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        gsis_free(c);
        return GSIS_ERR_CUDA;
    }
    *out = c;
    return GSIS_OK;
}

gsis_status gsis_set_mesh(gsis_ctx* c, const gsis_mesh_desc* md) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!md) return set_err(c, GSIS_ERR_ARG, "NULL mesh descriptor");
    if (c->started) return set_err(c, GSIS_ERR_STATE, "mesh cannot change after the first iterate");
    const int ni = md->ni, nj = md->nj, nk = md->nk;
    if (ni < 1 || nj < 1 || nk < 1 || md->dim < 1 || md->dim > 3)
        return set_err(c, GSIS_ERR_ARG, "mesh sizes must be >= 1 and dim in 1..3");
    if ((long long)ni * nj * nk > (1ll << 30)) return set_err(c, GSIS_ERR_ARG, "too many cells");
    if (!md->centers || !md->volumes || !md->W0 || !md->S[0] || !md->S[1] || !md->S[2] || !md->xf[0] ||
        !md->xf[1] || !md->xf[2])
        return set_err(c, GSIS_ERR_ARG, "NULL mesh array");
    const int n3[3] = {ni, nj, nk};
    bool per[3];
    for (int d = 0; d < 3; ++d) {
        const int lo = md->bc_type[2 * d], hi = md->bc_type[2 * d + 1];
        for (int s : {lo, hi})
            if (s < GSIS_BC_NONE || s > GSIS_BC_PERIODIC) return set_err(c, GSIS_ERR_ARG, "unknown boundary type");
        if ((lo == GSIS_BC_PERIODIC) != (hi == GSIS_BC_PERIODIC))
            return set_err(c, GSIS_ERR_ARG, "periodic sides must come in pairs");
        per[d] = lo == GSIS_BC_PERIODIC;
        if (per[d] && n3[d] < 3) return set_err(c, GSIS_ERR_ARG, "a periodic direction needs at least 3 cells");
    }
    for (int s = 0; s < 6; ++s) {
        if (md->bc_type[s] == GSIS_BC_FARFIELD &&
            (!(md->bc_state[s][0] > 0.0) || !(md->bc_state[s][4] > 0.0) || !finite_all(md->bc_state[s], 5)))
            return set_err(c, GSIS_ERR_ARG, "far-field state must be finite with rho, T > 0");
        if (md->bc_type[s] == GSIS_BC_WALL && !(md->bc_state[s][4] > 0.0))
            return set_err(c, GSIS_ERR_ARG, "wall temperature must be > 0");
    }
    const int N = ni * nj * nk;
    if (!finite_all(md->centers, (size_t)N * 3) || !finite_all(md->W0, (size_t)N * 5))
        return set_err(c, GSIS_ERR_ARG, "non-finite mesh centres or initial state");
    for (int q = 0; q < N; ++q) {
        if (!(md->volumes[q] > 0.0)) return set_err(c, GSIS_ERR_ARG, "cell volumes must be > 0");
        if (!(md->W0[q * 5] > 0.0) || !(md->W0[q * 5 + 4] > 0.0))
            return set_err(c, GSIS_ERR_ARG, "initial rho and T must be > 0");
    }
    const size_t nf[3] = {(size_t)(ni + 1) * nj * nk, (size_t)ni * (nj + 1) * nk, (size_t)ni * nj * (nk + 1)};
    for (int d = 0; d < 3; ++d)
        if (!finite_all(md->S[d], nf[d] * 3) || !finite_all(md->xf[d], nf[d] * 3))
            return set_err(c, GSIS_ERR_ARG, "non-finite face geometry");

    // connectivity, outward area vectors, face centres
    std::vector<int> nbr((size_t)N * 6), side_bc((size_t)N * 6), hyper(N);
    std::vector<double> Sout((size_t)N * 18), xf((size_t)N * 18), lsq((size_t)N * 18, 0.0);
    auto face_index = [&](int d, int i, int j, int k, int fi) -> size_t {
        if (d == 0) return ((size_t)k * nj + j) * (ni + 1) + fi;
        if (d == 1) return ((size_t)k * (nj + 1) + fi) * ni + i;
        return ((size_t)fi * nj + j) * ni + i;
    };
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) {
                const int cc = i + ni * (j + nj * k);
                hyper[cc] = i + j + k;
                const int idx[3] = {i, j, k};
                for (int d = 0; d < 3; ++d)
                    for (int hs = 0; hs < 2; ++hs) {
                        const int s = 2 * d + hs;
                        const int m = idx[d];
                        int fi = hs ? m + 1 : m;
                        if (per[d] && fi == n3[d]) fi = 0;
                        const size_t f = face_index(d, i, j, k, fi);
                        const double sg = hs ? 1.0 : -1.0;
                        for (int q = 0; q < 3; ++q) {
                            Sout[((size_t)cc * 6 + s) * 3 + q] = sg * md->S[d][f * 3 + q];
                            xf[((size_t)cc * 6 + s) * 3 + q] = md->xf[d][f * 3 + q];
                        }
                        int mm = m + (hs ? 1 : -1);
                        int nb = -1;
                        if (mm >= 0 && mm < n3[d]) nb = 0;
                        else if (per[d]) { mm = (mm + n3[d]) % n3[d]; nb = 0; }
                        if (nb == 0) {
                            int id2[3] = {i, j, k};
                            id2[d] = mm;
                            nb = id2[0] + ni * (id2[1] + nj * id2[2]);
                        }
                        nbr[(size_t)cc * 6 + s] = nb;
                        side_bc[(size_t)cc * 6 + s] = nb >= 0 ? -1 : md->bc_type[s];
                    }
            }
    // largest outflow factor sum_s |S_s| / V of a cell (bound on the sweep's denominator, see quotient_range)
    double max_sv = 0.0;
    for (int cc = 0; cc < N; ++cc) {
        double sv = 0.0;
        for (int s = 0; s < 6; ++s) {
            const double* v = &Sout[((size_t)cc * 6 + s) * 3];
            sv += std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        }
        max_sv = std::max(max_sv, sv / md->volumes[cc]);
    }
    if (c->vgrid_set && !quotient_range_ok(max_sv, c->max_xi))
        return set_err(c, GSIS_ERR_UNSUPPORTED, quotient_range_msg);
    c->max_sv = max_sv;
    // face-normal components that are nonzero on some flux-carrying face
    {
        bool any_y = false, any_z = false;
        int max_dir = 0;
        for (int cc = 0; cc < N; ++cc)
            for (int s = 0; s < 6; ++s) {
                const bool active = nbr[(size_t)cc * 6 + s] >= 0 || side_bc[(size_t)cc * 6 + s] == GSIS_BC_FARFIELD ||
                                    side_bc[(size_t)cc * 6 + s] == GSIS_BC_WALL;
                if (!active) continue;
                max_dir = std::max(max_dir, s / 2 + 1);
                any_y = any_y || Sout[((size_t)cc * 6 + s) * 3 + 1] != 0.0;
                any_z = any_z || Sout[((size_t)cc * 6 + s) * 3 + 2] != 0.0;
            }
        // directions 0..D-1 carry flux and normal components 0..D-1 can be nonzero
        c->normal_components = std::max(max_dir, any_z ? 3 : (any_y ? 2 : 1));
        // the face flux may also drop the other gradient components when the LSQ gradients have none
        // (dim) and neighbouring cell centres differ in no other coordinate
        const int nc = c->normal_components;
        bool flat = nc < 3 && md->dim <= nc;
        for (int cc = 0; flat && cc < N; ++cc)
            for (int s = 0; s < 6; ++s) {
                const int nb = nbr[(size_t)cc * 6 + s];
                if (nb < 0) continue;
                for (int k = nc; k < 3; ++k)
                    if (md->centers[(size_t)nb * 3 + k] != md->centers[(size_t)cc * 3 + k]) flat = false;
            }
        c->face_nd = flat ? nc : 3;
    }
    // least-squares weights over the first dim coordinates
    const int dim = md->dim;
    for (int cc = 0; cc < N; ++cc) {
        double rows[6][3];
        int used[6], nr = 0;
        for (int s = 0; s < 6; ++s) {
            const int nb = nbr[(size_t)cc * 6 + s];
            const int bc = side_bc[(size_t)cc * 6 + s];
            if (nb >= 0) {
                for (int q = 0; q < 3; ++q) rows[nr][q] = md->centers[(size_t)nb * 3 + q] - md->centers[(size_t)cc * 3 + q];
            } else if (bc == GSIS_BC_FARFIELD || bc == GSIS_BC_WALL) {
                for (int q = 0; q < 3; ++q) rows[nr][q] = xf[((size_t)cc * 6 + s) * 3 + q] - md->centers[(size_t)cc * 3 + q];
            } else {
                continue;
            }
            used[nr++] = s;
        }
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int r = 0; r < nr; ++r)
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) G[a][b] += rows[r][a] * rows[r][b];
        for (int r = 0; r < nr; ++r) {
            double rhs[3] = {0, 0, 0}, x[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) rhs[a] = rows[r][a];
            double Gc[3][3];
            std::memcpy(Gc, G, sizeof(G));
            if (!solve_small(dim, Gc, rhs, x))
                return set_err(c, GSIS_ERR_ARG, "degenerate least-squares stencil at cell " + std::to_string(cc));
            for (int a = 0; a < dim; ++a) lsq[((size_t)cc * 6 + used[r]) * 3 + a] = x[a];
        }
    }

    Mesh& m = c->m;
    m.ni = ni; m.nj = nj; m.nk = nk; m.dim = dim; m.N = N; m.H = ni + nj + nk - 2;
    std::memcpy(m.bc_type, md->bc_type, sizeof(m.bc_type));
    std::memcpy(m.bc_state, md->bc_state, sizeof(m.bc_state));
    std::vector<double> cen(md->centers, md->centers + (size_t)N * 3), vol(md->volumes, md->volumes + N);
    m.cen = upload(c, cen);
    m.vol = upload(c, vol);
    m.Sout = upload(c, Sout);
    m.xf = upload(c, xf);
    m.lsq_w = upload(c, lsq);
    m.nbr = upload(c, nbr);
    m.side_bc = upload(c, side_bc);
    m.hyper = upload(c, hyper);
    {
        std::vector<int> bs;
        for (int cc = 0; cc < N; ++cc)
            for (int s = 0; s < 6; ++s) {
                const int b = side_bc[(size_t)cc * 6 + s];
                if (nbr[(size_t)cc * 6 + s] < 0 && (b == GSIS_BC_FARFIELD || b == GSIS_BC_WALL)) bs.push_back(cc * 6 + s);
            }
        m.nbside = (int)bs.size();
        if (bs.empty()) bs.push_back(0);   // a valid pointer, never read
        m.bside = upload(c, bs);
    }
    std::vector<int> bct(md->bc_type, md->bc_type + 6);
    std::vector<double> bcs(&md->bc_state[0][0], &md->bc_state[0][0] + 30);
    c->d_bc_type = upload(c, bct);
    c->d_bc_state = upload(c, bcs);
    c->host_W0.assign(md->W0, md->W0 + (size_t)N * 5);
    const size_t N5 = (size_t)N * 5 * sizeof(double);
    c->W = (double*)dev_alloc(c, N5); c->Wh = (double*)dev_alloc(c, N5); c->Wp = (double*)dev_alloc(c, N5);
    c->Wm = (double*)dev_alloc(c, N5); c->U = (double*)dev_alloc(c, N5); c->Un = (double*)dev_alloc(c, N5);
    c->Wmom = (double*)dev_alloc(c, N5);
    c->dU = (double*)dev_alloc(c, N5); c->dU2 = (double*)dev_alloc(c, N5); c->R = (double*)dev_alloc(c, N5);
    c->D = (double*)dev_alloc(c, N * sizeof(double));
    c->lamS = (double*)dev_alloc(c, (size_t)N * 6 * sizeof(double));
    c->Fbnd = (double*)dev_alloc(c, (size_t)N * 36 * sizeof(double));
    c->Ff = (double*)dev_alloc(c, (size_t)N * 15 * sizeof(double));
    c->lamf = (double*)dev_alloc(c, (size_t)N * 3 * sizeof(double));
    c->F0 = (double*)dev_alloc(c, (size_t)N * 15 * sizeof(double));
    c->dFa = (double*)dev_alloc(c, (size_t)N * 15 * sizeof(double));
    c->dFb = (double*)dev_alloc(c, (size_t)N * 15 * sizeof(double));
    c->fgeo = (double*)dev_alloc(c, (size_t)N * 3 * 8 * sizeof(double));
    c->bgeo = (double*)dev_alloc(c, (size_t)N * 6 * 8 * sizeof(double));
    c->acell = (double*)dev_alloc(c, (size_t)N * sizeof(double));
    c->fields = (double*)dev_alloc(c, (size_t)N * FIELDS_N * sizeof(double));
    c->gu = (double*)dev_alloc(c, (size_t)N * 9 * sizeof(double));
    c->gT = (double*)dev_alloc(c, (size_t)N * 3 * sizeof(double));
    c->grho = (double*)dev_alloc(c, (size_t)N * 3 * sizeof(double));
    c->gU = (double*)dev_alloc(c, (size_t)N * 3 * sizeof(double));
    c->hot = (double*)dev_alloc(c, (size_t)N * HOTN * sizeof(double));
    c->kin = (double*)dev_alloc(c, (size_t)N * HOTN * sizeof(double));
    c->nsf = (double*)dev_alloc(c, (size_t)N * HOTN * sizeof(double));
    c->kn_gll = (double*)dev_alloc(c, N * sizeof(double));
    c->wall_den = (double*)dev_alloc(c, (size_t)N * 6 * sizeof(double));
    c->wall_in = (double*)dev_alloc(c, (size_t)N * 30 * sizeof(double));
    c->wall_kin = (double*)dev_alloc(c, (size_t)N * 30 * sizeof(double));
    c->wall_corr = (double*)dev_alloc(c, (size_t)N * 30 * sizeof(double));
    c->has_wall = false;
    for (int s = 0; s < 6; ++s) c->has_wall = c->has_wall || md->bc_type[s] == GSIS_BC_WALL;
    c->eps_buf = (double*)dev_alloc(c, 4 * sizeof(double));
    c->flag = (uint8_t*)dev_alloc(c, N);
    c->cell2dvm = (int*)dev_alloc(c, N * sizeof(int));
    c->old_cell2dvm = (int*)dev_alloc(c, N * sizeof(int));
    c->ghost_id = (int*)dev_alloc(c, N * sizeof(int));
    c->ghost_cell = (int*)dev_alloc(c, N * sizeof(int));
    c->enter_list = (int*)dev_alloc(c, N * sizeof(int));
    c->hp_off = (int*)dev_alloc(c, (m.H + 1) * sizeof(int));
    c->hp_cnt = (int*)dev_alloc(c, (m.H + 1) * sizeof(int));
    c->d_count = (int*)dev_alloc(c, 4 * sizeof(int));
    c->d_job = (gsis::MacroJob*)dev_alloc(c, sizeof(gsis::MacroJob));
    c->d_bar = (gsis::GridBarrier*)dev_alloc(c, sizeof(gsis::GridBarrier));
    c->specs = (RecSpec*)dev_alloc(c, (size_t)std::max(N, 6) * sizeof(RecSpec));
    c->recGhost.scal = (double*)dev_alloc(c, (size_t)N * RS * sizeof(double));
    c->recBC.scal = (double*)dev_alloc(c, 6 * RS * sizeof(double));
    if (!c->d_job || !c->d_bar || !m.cen || !m.vol || !m.Sout || !m.xf || !m.lsq_w || !m.nbr || !m.side_bc || !m.hyper || !m.bside || !c->Fbnd || !c->W || !c->Wmom ||
        !c->Wh || !c->fgeo || !c->bgeo || !c->acell || !c->fields ||
        !c->Wp || !c->Wm || !c->U || !c->Un || !c->dU || !c->dU2 || !c->R || !c->D || !c->lamS || !c->Ff ||
        !c->lamf || !c->F0 || !c->dFa || !c->dFb || !c->gu || !c->gT ||
        !c->grho || !c->gU || !c->hot || !c->kin || !c->nsf || !c->kn_gll || !c->wall_den || !c->wall_in ||
        !c->wall_kin || !c->wall_corr || !c->eps_buf || !c->flag ||
        !c->cell2dvm || !c->old_cell2dvm || !c->ghost_id || !c->ghost_cell || !c->enter_list || !c->hp_off ||
        !c->hp_cnt || !c->d_count || !c->specs || !c->recGhost.scal || !c->recBC.scal || !c->d_bc_type ||
        !c->d_bc_state)
        return set_err(c, GSIS_ERR_OOM, "device allocation failed in gsis_set_mesh");
    cudaMemsetAsync(c->wall_den, 0, (size_t)N * 6 * sizeof(double), c->stream);
    cudaMemsetAsync(c->wall_in, 0, (size_t)N * 30 * sizeof(double), c->stream);
    cudaMemsetAsync(c->wall_kin, 0, (size_t)N * 30 * sizeof(double), c->stream);
    cudaMemsetAsync(c->wall_corr, 0, (size_t)N * 30 * sizeof(double), c->stream);
    cudaMemsetAsync(c->kn_gll, 0, (size_t)N * sizeof(double), c->stream);
    c->mesh_set = true;
    if (c->vgrid_set) {
        c->recGhost.tab = (double*)dev_alloc(c, (size_t)N * NTAB * c->vg.NT * sizeof(double));
        if (!c->recGhost.tab) return set_err(c, GSIS_ERR_OOM, "device allocation failed (ghost tables)");
    }
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "gsis_set_mesh")) return GSIS_ERR_CUDA;
    return GSIS_OK;
}

gsis_status gsis_set_velocity_grid(gsis_ctx* c, const gsis_vgrid_desc* vd) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!vd) return set_err(c, GSIS_ERR_ARG, "NULL velocity-grid descriptor");
    if (c->started) return set_err(c, GSIS_ERR_STATE, "velocity grid cannot change after the first iterate");
    if (vd->reduced != 0 && vd->reduced != 1) return set_err(c, GSIS_ERR_ARG, "reduced must be 0 or 1");
    const bool red = vd->reduced == 1;
    const int naxes = red ? 2 : 3;   // the reduced grid's z "axis" is its two planes G and H
    for (int d = 0; d < naxes; ++d)
        if (vd->n[d] < 1 || !(vd->hi[d] > vd->lo[d]) || !std::isfinite(vd->lo[d]) || !std::isfinite(vd->hi[d]))
            return set_err(c, GSIS_ERR_ARG, "velocity grid needs n >= 1 and hi > lo on every axis");
    const int n3[3] = {vd->n[0], vd->n[1], red ? 2 : vd->n[2]};
    const long long Nv = (long long)n3[0] * n3[1] * n3[2];
    if (Nv > (1ll << 31)) return set_err(c, GSIS_ERR_ARG, "too many velocities");
    double max_xi = 0.0;
    for (int d = 0; d < naxes; ++d) max_xi = std::max(max_xi, std::max(std::fabs(vd->lo[d]), std::fabs(vd->hi[d])));
    if (c->mesh_set && !quotient_range_ok(c->max_sv, max_xi))
        return set_err(c, GSIS_ERR_UNSUPPORTED, quotient_range_msg);
    c->max_xi = max_xi;
    std::vector<double> xi;
    double w = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (red && d == 2) {   // planes G and H: xi_z = 0 in every flux, weight 1
            xi.push_back(0.0);
            xi.push_back(0.0);
        } else {
            const double h = (vd->hi[d] - vd->lo[d]) / vd->n[d];
            for (int q = 0; q < vd->n[d]; ++q) xi.push_back(vd->lo[d] + (q + 0.5) * h);
            w *= h;
        }
        c->nv3[d] = n3[d];
        c->vlo[d] = vd->lo[d];
        c->vhi[d] = vd->hi[d];
    }
    if (c->d_xi) dev_free(c, c->d_xi);
    if (c->recBC.tab) dev_free(c, c->recBC.tab);
    if (c->recGhost.tab) dev_free(c, c->recGhost.tab);
    c->recGhost.tab = nullptr;
    c->d_xi = upload(c, xi);
    c->vg.nx = n3[0]; c->vg.ny = n3[1]; c->vg.nz = n3[2];
    c->vg.NT = n3[0] + n3[1] + n3[2];
    c->vg.reduced = red ? 1 : 0;
    c->vg.vscale = c->p.vdf_dtype == GSIS_F16 ? 4096.0 : 1.0;
    c->vg.Nv = Nv;
    c->vg.w = w;
    c->vg.xi = c->d_xi;
    c->recBC.tab = (double*)dev_alloc(c, 6 * NTAB * c->vg.NT * sizeof(double));
    if (c->mesh_set) c->recGhost.tab = (double*)dev_alloc(c, (size_t)c->m.N * NTAB * c->vg.NT * sizeof(double));
    if (!c->d_xi || !c->recBC.tab || (c->mesh_set && !c->recGhost.tab))
        return set_err(c, GSIS_ERR_OOM, "device allocation failed in gsis_set_velocity_grid");
    c->cap_Nd = 0;   // record tables depend on NT: reallocate the DVM arrays at the next region build
    c->vgrid_set = true;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "gsis_set_velocity_grid")) return GSIS_ERR_CUDA;
    return GSIS_OK;
}

gsis_status gsis_debug_set_region(gsis_ctx* c, const uint8_t* flags) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!c->mesh_set) return set_err(c, GSIS_ERR_STATE, "set the mesh before forcing a region");
    if (c->started) return set_err(c, GSIS_ERR_STATE, "the region can only be forced before the first iterate");
    if (!flags) return set_err(c, GSIS_ERR_ARG, "NULL flags");
    c->forced_flags.assign(flags, flags + c->m.N);
    for (auto& v : c->forced_flags) v = v ? 1 : 0;
    c->have_forced = true;
    return GSIS_OK;
}

gsis_status gsis_iterate(gsis_ctx* c, int max_iter, gsis_report* rep) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!c->mesh_set || !c->vgrid_set) return set_err(c, GSIS_ERR_STATE, "set the mesh and velocity grid first");
    if (max_iter < 0) return set_err(c, GSIS_ERR_ARG, "max_iter must be >= 0");
    for (int i = 0; i < GSIS_NPHASE; ++i) c->phase_ms[i] = 0.0;
    const long long l0 = c->launches, s0 = c->sweep_launches;
    bool used[GSIS_NPHASE] = {false};
    if (!c->started) {
        used[GSIS_PH_PRESOLVE] = true;
        st = start(c);
        if (st != GSIS_OK) return st;
        phase_collect(c, used);
        used[GSIS_PH_PRESOLVE] = false;
    }
    int done = 0;
    double eps = rep ? rep->eps : 0.0;
    bool converged = false;
    for (int it = 0; it < max_iter; ++it) {
        for (bool& u : used) u = false;
        st = gsis_step(c, &eps, used);
        if (st != GSIS_OK) return st;
        phase_collect(c, used);
        ++done;
        if (eps < c->p.tol) { converged = true; break; }
    }
    if (rep) {
        rep->iterations = done;
        rep->total_iterations = c->iteration;
        rep->eps = eps;
        rep->converged = converged ? 1 : 0;
        rep->n_dvm = c->Nd;
        rep->n_v = c->vg.Nv;
        rep->vdf_bytes = c->Nd * c->vg.Nv * (long long)vdf_elem_bytes(c->p.vdf_dtype);
        rep->presolve_blocks = c->presolve_blocks;
        for (int i = 0; i < GSIS_NPHASE; ++i) rep->phase_ms[i] = c->phase_ms[i];
        rep->sweep_launches = c->sweep_launches - s0;
        rep->kernel_launches = c->launches - l0;
    }
    return GSIS_OK;
}

gsis_status gsis_moments(gsis_ctx* c, unsigned mask, double* dst, int dst_is_device) {
    if (!c) return GSIS_ERR_ARG;
    if (!dst) return set_err(c, GSIS_ERR_ARG, "NULL destination");
    if (!c->mesh_set) return set_err(c, GSIS_ERR_STATE, "no mesh");
    if (mask == 0 || mask >= (1u << GSIS_NFIELDS)) return set_err(c, GSIS_ERR_ARG, "bad field mask");
    const unsigned derived = ~((1u << 16) - 1) & ((1u << GSIS_NFIELDS) - 1);   // WALL_Q and above
    if ((mask & derived) && !c->started)
        return set_err(c, GSIS_ERR_STATE, "derived fields need the first gsis_iterate");
    const int N = c->m.N;
    std::vector<double> W((size_t)N * 5), hot((size_t)N * HOTN), kn(N, 0.0), fl;
    std::vector<int> c2d(N, -1);
    if (c->started) {
        const unsigned wall_bits = GSIS_FIELD_WALL_Q | GSIS_FIELD_WALL_P | GSIS_FIELD_WALL_TX | GSIS_FIELD_WALL_TY |
                                   GSIS_FIELD_WALL_TZ;
        const bool wall = (mask & wall_bits) != 0, cons = (mask & derived & ~wall_bits) != 0;
        if (wall || cons) {
            launch_fields(c, wall, cons);
            fl.resize((size_t)N * FIELDS_N);
            cudaMemcpyAsync(fl.data(), c->fields, fl.size() * 8, cudaMemcpyDeviceToHost, c->stream);
        }
        cudaMemcpyAsync(W.data(), c->W, W.size() * 8, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(hot.data(), c->hot, hot.size() * 8, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(kn.data(), c->kn_gll, kn.size() * 8, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(c2d.data(), c->cell2dvm, c2d.size() * 4, cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GSIS_ERR_CUDA, "gsis_moments copy failed");
        }
    } else {
        W = c->host_W0;
        std::fill(hot.begin(), hot.end(), 0.0);
    }
    int nsel = 0;
    for (int b = 0; b < GSIS_NFIELDS; ++b) nsel += (mask >> b) & 1;
    std::vector<double> out((size_t)N * nsel);
    for (int cc = 0; cc < N; ++cc) {
        int o = 0;
        for (int b = 0; b < GSIS_NFIELDS; ++b) {
            if (!((mask >> b) & 1)) continue;
            double v;
            if (b < 5) v = W[(size_t)cc * 5 + b];
            else if (b < 14) v = hot[(size_t)cc * HOTN + (b - 5)];
            else if (b == 14) v = kn[cc];
            else if (b == 15) v = c2d[cc] >= 0 ? 1.0 : 0.0;
            else if (b == 16) v = fl[(size_t)cc * FIELDS_N + FIELD_WALL];                 // wall heat flux
            else if (b < 27) v = fl[(size_t)cc * FIELDS_N + (b - 17)];                    // sigma, q, p
            else v = fl[(size_t)cc * FIELDS_N + FIELD_WALL + 1 + (b - 27)];               // wall p, shear
            out[(size_t)cc * nsel + o++] = v;
        }
    }
    if (dst_is_device) {
        if (cudaMemcpy(dst, out.data(), out.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, GSIS_ERR_ARG, "destination is not device memory");
        }
    } else {
        std::memcpy(dst, out.data(), out.size() * 8);
    }
    return GSIS_OK;
}

gsis_status gsis_get_vdf(gsis_ctx* c, double* dst, int* cells, long long capacity) {
    if (!c) return GSIS_ERR_ARG;
    if (!c->started) return set_err(c, GSIS_ERR_STATE, "no VDF before the first iterate");
    const long long n = c->Nd * c->vg.Nv;
    if (!dst || capacity < n) return set_err(c, GSIS_ERR_ARG, "destination too small");
    const size_t eb = vdf_elem_bytes(c->p.vdf_dtype);
    std::vector<unsigned char> raw((size_t)n * eb);
    cudaMemcpyAsync(raw.data(), c->f, raw.size(), cudaMemcpyDeviceToHost, c->stream);
    std::vector<int> dc(c->Nd);
    if (c->Nd) cudaMemcpyAsync(dc.data(), c->dvm_cell, dc.size() * 4, cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, GSIS_ERR_CUDA, "gsis_get_vdf copy failed");
    }
    const double iscale = 1.0 / c->vg.vscale;   // stored values carry the VDF storage scale
    for (long long i = 0; i < n; ++i) {
        double v;
        switch (c->p.vdf_dtype) {
            case GSIS_F64: std::memcpy(&v, &raw[(size_t)i * 8], 8); break;
            case GSIS_F32: { float x; std::memcpy(&x, &raw[(size_t)i * 4], 4); v = x; break; }
            case GSIS_BF16: { uint16_t h; std::memcpy(&h, &raw[(size_t)i * 2], 2); uint32_t b = (uint32_t)h << 16;
                              float x; std::memcpy(&x, &b, 4); v = x; break; }
            default: { uint16_t h; std::memcpy(&h, &raw[(size_t)i * 2], 2);
                       __half_raw hr; hr.x = h; v = (double)__half2float(__half(hr)); break; }
        }
        dst[i] = v * iscale;
    }
    if (cells) std::memcpy(cells, dc.data(), dc.size() * 4);
    return GSIS_OK;
}

gsis_status gsis_two_vdf_reference(gsis_ctx* c, const double* S, int n, int d_r, double Z_r, const double* A,
                                   double* g_out) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!S || !A || !g_out || n < 0) return set_err(c, GSIS_ERR_ARG, "NULL argument or n < 0");
    if (n > 65535) return set_err(c, GSIS_ERR_ARG, "at most 65535 states per call");
    if (d_r < 0 || !(Z_r >= 1.0) || !std::isfinite(Z_r) || !finite_all(A, 4))
        return set_err(c, GSIS_ERR_ARG, "need d_r >= 0, finite Z_r >= 1 and a finite A matrix");
    if (!c->vgrid_set) return set_err(c, GSIS_ERR_STATE, "velocity grid not set");
    if (c->vg.reduced) return set_err(c, GSIS_ERR_UNSUPPORTED, "two-VDF reference pair: full 3D velocity grids only");
    if (n == 0) return GSIS_OK;
    // the states are few: check them on the host before any launch
    std::vector<double> h((size_t)n * 12);
    if (!cuda_ok(c, cudaMemcpyAsync(h.data(), S, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                 "gsis_two_vdf_reference") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "gsis_two_vdf_reference"))
        return GSIS_ERR_CUDA;
    if (!finite_all(h.data(), h.size())) return set_err(c, GSIS_ERR_ARG, "non-finite state");
    for (int k = 0; k < n; ++k) {
        const double* s = &h[(size_t)k * 12];
        if (!(s[0] > 0.0) || !(s[4] > 0.0) || (d_r > 0 && !(s[5] > 0.0)))
            return set_err(c, GSIS_ERR_ARG, "states need rho > 0, T_t > 0 and (d_r > 0) T_r > 0");
    }
    const int NT = c->vg.NT;
    RecSpec* specs = (RecSpec*)dev_alloc(c, (size_t)4 * n * sizeof(RecSpec));
    Records rec{};
    rec.scal = (double*)dev_alloc(c, (size_t)4 * n * RS * sizeof(double));
    rec.tab = (double*)dev_alloc(c, (size_t)4 * n * NTAB * NT * sizeof(double));
    gsis_status out = GSIS_OK;
    if (!specs || !rec.scal || !rec.tab) {
        out = set_err(c, GSIS_ERR_OOM, "device allocation failed in gsis_two_vdf_reference");
    } else {
        TwoVdfGas g{d_r, Z_r, {A[0], A[1], A[2], A[3]}};
        launch_two_vdf_reference(c, S, n, g, specs, rec, g_out);
        if (!cuda_ok(c, cudaGetLastError(), "gsis_two_vdf_reference launch") ||
            !cuda_ok(c, cudaStreamSynchronize(c->stream), "gsis_two_vdf_reference"))
            out = GSIS_ERR_CUDA;
    }
    dev_free(c, specs);
    dev_free(c, rec.scal);
    dev_free(c, rec.tab);
    return out;
}

gsis_status gsis_two_vdf_moments(gsis_ctx* c, const double* F, int n, int d_r, double* out) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!F || !out || n < 0 || d_r < 0) return set_err(c, GSIS_ERR_ARG, "NULL argument, n < 0 or d_r < 0");
    if (n > 65535) return set_err(c, GSIS_ERR_ARG, "at most 65535 pairs per call");
    if (!c->vgrid_set) return set_err(c, GSIS_ERR_STATE, "velocity grid not set");
    if (c->vg.reduced) return set_err(c, GSIS_ERR_UNSUPPORTED, "two-VDF moments: full 3D velocity grids only");
    if (n == 0) return GSIS_OK;
    launch_two_vdf_moments(c, F, n, d_r, out);
    if (!cuda_ok(c, cudaGetLastError(), "gsis_two_vdf_moments launch") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "gsis_two_vdf_moments"))
        return GSIS_ERR_CUDA;
    return GSIS_OK;
}

const char* gsis_last_error(const gsis_ctx* c) {
    if (!c) return "NULL context";
    return c->err.c_str();
}

gsis_status gsis_iterate_batch(gsis_ctx** ctxs, int n, int iterations, gsis_report* reports) {
    if (!ctxs || n <= 0 || iterations < 0) return GSIS_ERR_ARG;
    std::vector<gsis_ctx*> cs(ctxs, ctxs + n);
    for (int i = 0; i < n; ++i) {
        if (!cs[i]) return GSIS_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (cs[j] == cs[i]) return set_err(cs[i], GSIS_ERR_ARG, "a context appears twice in the batch");
    }
    int dev0 = cs[0]->device;
    for (gsis_ctx* c : cs) {
        gsis_status st = check_ctx(c);
        if (st != GSIS_OK) return st;
        if (!c->mesh_set || !c->vgrid_set) return set_err(c, GSIS_ERR_STATE, "set the mesh and velocity grid first");
        if (c->device != dev0) return set_err(c, GSIS_ERR_ARG, "batched solves must share one device");
        if (c->p.adaptive && !c->have_forced)
            return set_err(c, GSIS_ERR_UNSUPPORTED, "batched solves run with a fixed DVM region (adaptive = 0)");
    }
    for (gsis_ctx* c : cs) {
        if (!c->started) {
            gsis_status st = start(c);
            if (st != GSIS_OK) return st;
        }
    }
    for (gsis_ctx* c : cs)   // the batch stream is ordered after each solve's own work
        if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "batch start")) return GSIS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(batch_mutex());
    auto& plans = batch_plans();
    BatchPlan* P = nullptr;
    auto found = plans.find(cs);
    if (found != plans.end()) {
        P = found->second;
        bool stale = false;   // a solve stepped on its own since the graph was recorded (buffers swapped)
        for (int i = 0; i < n; ++i) stale = stale || (P->W_at_capture[i] != cs[i]->W);
        if (stale) {
            destroy_plan(P);
            plans.erase(found);
            P = nullptr;
        }
    }
    if (!P) {
        P = new (std::nothrow) BatchPlan();
        if (!P) return GSIS_ERR_OOM;
        P->ctxs = cs;
        P->owner = cs[0];
        P->stream = cs[0]->stream;
        if (!P->stream) {   // the legacy default stream cannot be captured
            if (!cuda_ok(cs[0], cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking), "batch stream")) {
                delete P;
                return GSIS_ERR_CUDA;
            }
            P->own_stream = true;
        }
        gsis_status st = build_plan(P);
        if (st != GSIS_OK) {
            destroy_plan(P);
            return st;
        }
        plans[cs] = P;
    }
    for (int it = 0; it < iterations; ++it)
        if (!cuda_ok(P->owner, cudaGraphLaunch(P->exec, P->stream), "batch graph launch")) return GSIS_ERR_CUDA;
    if (!cuda_ok(P->owner, cudaStreamSynchronize(P->stream), "batched GSIS iterations")) return GSIS_ERR_CUDA;
    float sweep_ms = 0.f, iter_ms = 0.f;   // of the last replayed iteration (event-record nodes of the graph)
    if (iterations > 0) {
        if (!cuda_ok(P->owner, cudaEventElapsedTime(&sweep_ms, P->ev[0], P->ev[1]), "batch sweep timing") ||
            !cuda_ok(P->owner, cudaEventElapsedTime(&iter_ms, P->ev[2], P->ev[3]), "batch iteration timing"))
            return GSIS_ERR_CUDA;
    }
    if (!cuda_ok(P->owner, cudaGetLastError(), "batched iteration")) return GSIS_ERR_CUDA;
    gsis_status result = GSIS_OK;
    for (int i = 0; i < n; ++i) {
        gsis_ctx* c = cs[i];
        double e[2] = {0.0, 0.0};
        if (!cuda_ok(c, cudaMemcpy(e, c->eps_buf, 2 * sizeof(double), cudaMemcpyDeviceToHost), "read epsilon"))
            return GSIS_ERR_CUDA;
        c->iteration += iterations;
        c->launches += P->launches_per_iter * iterations / n;
        if (iterations > 0 && e[1] != 0.0 && result == GSIS_OK)
            result = set_err(c, GSIS_ERR_NONFINITE, "non-finite or non-positive density/temperature in a batched solve");
        if (reports) {
            gsis_report& r = reports[i];
            std::memset(&r, 0, sizeof(r));
            r.iterations = iterations;
            r.total_iterations = c->iteration;
            r.eps = e[0];
            r.converged = (iterations > 0 && e[0] < c->p.tol) ? 1 : 0;
            r.n_dvm = c->Nd;
            r.n_v = c->vg.Nv;
            r.vdf_bytes = c->Nd * c->vg.Nv * (long long)vdf_elem_bytes(c->p.vdf_dtype);
            r.presolve_blocks = c->presolve_blocks;
            r.sweep_launches = iterations;   // one persistent launch per iteration for the whole batch
            r.kernel_launches = P->launches_per_iter * iterations;
            r.phase_ms[GSIS_PH_SWEEP] = sweep_ms;           // the batched sweep of the last iteration
            r.phase_ms[GSIS_PH_MACRO] = iter_ms - sweep_ms;  // everything else of the last iteration
        }
    }
    return result;
}

gsis_status gsis_debug_set_sweep_tile(gsis_ctx* c, const char* name) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!name) return set_err(c, GSIS_ERR_ARG, "tile name is NULL");
    if (!c->started) {
        if (!c->mesh_set || !c->vgrid_set) return set_err(c, GSIS_ERR_STATE, "set the mesh and velocity grid first");
        st = start(c);
        if (st != GSIS_OK) return st;
    }
    return force_sweep_shape(c, name);
}

gsis_status gsis_debug_vdf_moments(gsis_ctx* c, int direct, double* dst, long long capacity) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (!dst) return set_err(c, GSIS_ERR_ARG, "NULL destination");
    if (!c->started || c->iteration == 0) return set_err(c, GSIS_ERR_STATE, "no GSIS iteration yet");
    if (capacity < c->Nd * MOMN) return set_err(c, GSIS_ERR_ARG, "destination too small");
    if (c->Nd == 0) return GSIS_OK;
    // (momh is free between iterations: the next moments pass rewrites it before any use)
    if (direct) launch_moments(c, c->W, c->momh);
    if (!cuda_ok(c, cudaMemcpyAsync(dst, direct ? c->momh : c->mom, (size_t)c->Nd * MOMN * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream),
                 "moment copy") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "moment copy"))
        return GSIS_ERR_CUDA;
    return GSIS_OK;
}

gsis_status gsis_debug_set_macro_path(gsis_ctx* c, int path) {
    gsis_status st = check_ctx(c);
    if (st != GSIS_OK) return st;
    if (path < GSIS_MACRO_AUTO || path > GSIS_MACRO_PERSISTENT_STALL) return set_err(c, GSIS_ERR_ARG, "unknown path");
    c->macro_path = path;
    return GSIS_OK;
}

const char* gsis_tuning_info(gsis_ctx* c) {
    if (!c) return "";
    return c->sweep_info.c_str();
}

gsis_status gsis_debug_set_batch_tile(const char* name) {
    std::lock_guard<std::mutex> lk(batch_mutex());
    if (!name || !*name) {
        forced_batch_shape() = -1;
        return GSIS_OK;
    }
    for (int sh = 0; sh < batch_num_shapes(); ++sh)
        if (std::string(batch_shape_name(sh)) == name) {
            forced_batch_shape() = sh;
            return GSIS_OK;
        }
    return GSIS_ERR_ARG;
}

const char* gsis_batch_info(gsis_ctx** ctxs, int n) {
    static thread_local std::string out;
    if (!ctxs || n <= 0) return "";
    std::lock_guard<std::mutex> lk(batch_mutex());
    auto it = batch_plans().find(std::vector<gsis_ctx*>(ctxs, ctxs + n));
    out = it == batch_plans().end() ? std::string() : it->second->info;
    return out.c_str();
}

void gsis_free(gsis_ctx* c) {
    if (!c) return;
    drop_plans_with(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    cudaGetLastError();
    std::vector<void*> all = c->allocations;
    for (void* p : all) dev_free(c, p);
    if (c->events)
        for (int i = 0; i < 2 * GSIS_NPHASE; ++i) cudaEventDestroy(c->ev[i]);
    if (c->h_eps) cudaFreeHost(c->h_eps);
    if (c->h_count) cudaFreeHost(c->h_count);
    if (c->h_err) cudaFreeHost(c->h_err);
    delete c;
}

}  // extern "C"
