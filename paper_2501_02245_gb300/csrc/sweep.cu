// Kinetic step of Sec. 3.1 (the implicit finite-volume update of f towards
// f^{n+1/2}), steady form (dt -> infinity), on the compacted DVM cells.
//
// Scheme (identical to the CPU reference): for cell c and velocity xi,
//   (1/tau + sum_{F out} xi.S_F/V) f_c =
//        g~_c/tau - sum_{F out} (xi.S_F/V) (+-1/2) slope_c,d
//                 - sum_{F in}  (xi.S_F/V) f_F^in
// with slope = minmod(f_c - f_{c-d}, f_{c+d} - f_c) in index space when both
// neighbours along d are DVM cells (else 0), and f_F^in the neighbour's MUSCL
// face value, a Grad-13 interface distribution (NS neighbour), the far-field
// corrected Maxwellian, or rho_w M_w (diffuse wall).  One backward (pass = 1,
// decreasing hyperplane h = i+j+k, towards the low-index walls of the
// O-grids) and one forward (pass = 0) Gauss-Seidel pass; the wall densities
// are refreshed from the latest f between them.
//
// Parallel structure.  Every dependency of the update at (c, xi) is on the
// same velocity xi, and cells of one hyperplane never depend on each other.
// A block owns 32*VPT consecutive velocities: lane l of every warp handles
// the VPT velocities l, l+32, ..., so each warp-wide load reads 32
// consecutive values of a cell row (coalesced, velocity innermost).  The G
// warps of the block split the cells of each hyperplane and the block
// synchronises once per hyperplane.  A warp updates CB cells of a hyperplane
// at a time: the cells' metadata (read through the non-coherent path, so the
// compiler may load it ahead of the VDF stores), then the stencils of all
// CB x VPT points (own value, both neighbours and both second neighbours per
// direction), then the branch-free updates, then the stores -- so the memory
// latency of CB x VPT independent updates overlaps.
//
// Arithmetic type T: FP64 for an FP64 VDF (ALU-bound on GB300: 2 DFMA/clk/SM),
// FP32 for FP32 / BF16 / FP16 storage.  NC = number of index directions that
// carry flux and of face-normal components that can be nonzero (1, 2 or 3 for
// 1D, 2D and 3D meshes); the rest is skipped.
#include <map>
#include <string>
#include "sweep_pair.cuh"

namespace gsis {

template <typename S, typename T, int NC, int G, int VPT, int CB, bool FULL>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, S* __restrict__ f, int pass) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Vel<T, VPT, FULL> V;
    make_vel(a.vg, (long long)blockIdx.x * (32 * VPT), lane, V);
    for (int hh = 0; hh < a.H; ++hh) {
        const int h = pass ? (a.H - 1 - hh) : hh;
        const int kb = __ldg(a.hp_off + h), ke = __ldg(a.hp_off + h + 1);
        const int n = ke - kb;
        // warp w takes the cells w, w+G, w+2G, ... (in reverse order for the backward pass)
        for (int i0 = w; i0 < n; i0 += G * CB) {
            int kk[CB];
            bool kon[CB];
#pragma unroll
            for (int b = 0; b < CB; ++b) {
                const int i = i0 + b * G;
                kon[b] = i < n;
                kk[b] = pass ? (ke - 1 - i) : (kb + i);
            }
            update_cells<S, T, NC, VPT, CB>(a, f, kk, kon, V);
        }
        if (G > 1) __syncthreads();
    }
}

template <typename S, typename T, int NC, int G, int VPT, int CB>
__global__ void __launch_bounds__(32 * G) k_sweep(SweepArgs a, S* __restrict__ f, int pass) {
    if ((long long)(blockIdx.x + 1) * (32 * VPT) <= a.vg.Nv)   // tile inside the grid (uniform)
        sweep_tile<S, T, NC, G, VPT, CB, true>(a, f, pass);
    else
        sweep_tile<S, T, NC, G, VPT, CB, false>(a, f, pass);
}

// The same tile on pairs of velocities (FP32 arithmetic, sweep_pair.cuh): a
// block owns 64 * VPT consecutive velocities, lane l the pairs 2l + 64u.
template <typename S, int NC, int G, int VPT, int CB, bool FULL>
__device__ __forceinline__ void sweep_tile2(const SweepArgs& a, S* __restrict__ f, int pass) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Vel2<VPT, FULL> V;
    make_vel2(a.vg, (long long)blockIdx.x * (64 * VPT), lane, V);
    for (int hh = 0; hh < a.H; ++hh) {
        const int h = pass ? (a.H - 1 - hh) : hh;
        const int kb = __ldg(a.hp_off + h), ke = __ldg(a.hp_off + h + 1);
        const int n = ke - kb;
        for (int i0 = w; i0 < n; i0 += G * CB) {
            int kk[CB];
            bool kon[CB];
#pragma unroll
            for (int b = 0; b < CB; ++b) {
                const int i = i0 + b * G;
                kon[b] = i < n;
                kk[b] = pass ? (ke - 1 - i) : (kb + i);
            }
            update_cells2<S, NC, VPT, CB>(a, f, kk, kon, V);
        }
        if (G > 1) __syncthreads();
    }
}

template <typename S, int NC, int G, int VPT, int CB>
__global__ void __launch_bounds__(32 * G) k_sweep2(SweepArgs a, S* __restrict__ f, int pass) {
    if ((long long)(blockIdx.x + 1) * (64 * VPT) <= a.vg.Nv)
        sweep_tile2<S, NC, G, VPT, CB, true>(a, f, pass);
    else
        sweep_tile2<S, NC, G, VPT, CB, false>(a, f, pass);
}

template <typename S, int G, int VPT, int CB>
static void sweep2_t(gsis_ctx* c, const SweepArgs& a, int pass) {
    const unsigned blocks = (unsigned)((c->vg.Nv + 64 * VPT - 1) / (64 * VPT));
    S* f = (S*)c->f;
    if (c->normal_components == 2)
        k_sweep2<S, 2, G, VPT, CB><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass);
    else
        k_sweep2<S, 3, G, VPT, CB><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass);
}

template <typename S, typename T, int G, int VPT, int CB>
static void sweep_t(gsis_ctx* c, const SweepArgs& a, int pass) {
    const unsigned blocks = (unsigned)((c->vg.Nv + 32 * VPT - 1) / (32 * VPT));
    S* f = (S*)c->f;
    switch (c->normal_components) {
        case 1: k_sweep<S, T, 1, G, VPT, CB><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass); break;
        case 2: k_sweep<S, T, 2, G, VPT, CB><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass); break;
        default: k_sweep<S, T, 3, G, VPT, CB><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass); break;
    }
}

// ---------------------------------------------------------------------------- tile shapes
// Candidate (warps per block G, velocities per thread VPT, cells per warp
// step CB) of the 2D/3D sweep, timed by the autotuner on the solve itself.
// 1D meshes (one cell per hyperplane) use one warp per block.
struct SweepShape {
    int g, vpt, cb;
    const char* name;
};
// (The wide FP64 blocks serve small velocity grids -- the reduced distributions
// of 2D flows -- whose few velocity tiles leave SMs idle with narrow blocks.)
static const SweepShape kShapesF64[] = {
    {2, 1, 2, "g2_v1_c2"}, {1, 1, 2, "g1_v1_c2"}, {4, 1, 1, "g4_v1_c1"}, {2, 1, 1, "g2_v1_c1"},
    {8, 1, 1, "g8_v1_c1"}, {16, 1, 1, "g16_v1_c1"}};
// (FP32 arithmetic: the p shapes update pairs of velocities with packed FP32
// instructions, sweep_pair.cuh; they need an even nx and a 2D or 3D mesh.)
static const SweepShape kShapesF32[] = {
    {8, 1, 1, "g8_v1_c1"}, {4, 1, 1, "g4_v1_c1"}, {8, 2, 1, "g8_v2_c1"},
    {4, 4, 1, "g4_v4_c1"}, {8, 4, 1, "g8_v4_c1"}, {4, 2, 2, "g4_v2_c2"},
    {8, 1, 1, "p8_v1_c1"}, {4, 2, 1, "p4_v2_c1"}, {8, 2, 1, "p8_v2_c1"}, {4, 1, 1, "p4_v1_c1"},
    {5, 2, 1, "p5_v2_c1"}};
constexpr int kFirstPairShape = 6, kPairShapeEnd = 11;
static bool pair_shape(int dtype, int shape) {
    return dtype != GSIS_F64 && shape >= kFirstPairShape && shape < kPairShapeEnd;
}
static bool pair_ok(gsis_ctx* c) { return c->vg.nx % 2 == 0 && c->normal_components >= 2; }

// Candidates after the register-stencil shapes: the shared-memory window
// sweep (sweep_ring.cu) with 8 warps x 32, 4 warps x 32 and 8 warps x 64
// velocities (2D meshes whose hyperplane window fits in shared memory).
static const char* kRingNames[] = {"ring_w8_v32", "ring_w4_v32", "ring_w8_v64"};
constexpr int kRingShapes = 3;

static int base_shapes(int dtype) {
    return dtype == GSIS_F64 ? (int)(sizeof(kShapesF64) / sizeof(kShapesF64[0]))
                             : (int)(sizeof(kShapesF32) / sizeof(kShapesF32[0]));
}
int sweep_num_shapes(int dtype) { return base_shapes(dtype) + kRingShapes; }
const char* sweep_shape_name(int dtype, int shape) {
    if (shape < 0 || shape >= sweep_num_shapes(dtype)) return "?";
    if (shape >= base_shapes(dtype)) return kRingNames[shape - base_shapes(dtype)];
    return dtype == GSIS_F64 ? kShapesF64[shape].name : kShapesF32[shape].name;
}

template <typename S>
static void sweep_f32_shape(gsis_ctx* c, const SweepArgs& a, int pass, int shape) {
    if (c->normal_components == 1) { sweep_t<S, float, 1, 2, 1>(c, a, pass); return; }
    switch (shape) {
        case 1: sweep_t<S, float, 4, 1, 1>(c, a, pass); break;
        case 2: sweep_t<S, float, 8, 2, 1>(c, a, pass); break;
        case 3: sweep_t<S, float, 4, 4, 1>(c, a, pass); break;
        case 4: sweep_t<S, float, 8, 4, 1>(c, a, pass); break;
        case 5: sweep_t<S, float, 4, 2, 2>(c, a, pass); break;
        case 6: sweep2_t<S, 8, 1, 1>(c, a, pass); break;
        case 7: sweep2_t<S, 4, 2, 1>(c, a, pass); break;
        case 8: sweep2_t<S, 8, 2, 1>(c, a, pass); break;
        case 9: sweep2_t<S, 4, 1, 1>(c, a, pass); break;
        case 10: sweep2_t<S, 5, 2, 1>(c, a, pass); break;
        default: sweep_t<S, float, 8, 1, 1>(c, a, pass); break;
    }
}

static void sweep_f64_shape(gsis_ctx* c, const SweepArgs& a, int pass, int shape) {
    if (c->normal_components == 1) { sweep_t<double, double, 1, 1, 1>(c, a, pass); return; }
    switch (shape) {
        case 1: sweep_t<double, double, 1, 1, 2>(c, a, pass); break;
        case 2: sweep_t<double, double, 4, 1, 1>(c, a, pass); break;
        case 3: sweep_t<double, double, 2, 1, 1>(c, a, pass); break;
        case 4: sweep_t<double, double, 8, 1, 1>(c, a, pass); break;
        case 5: sweep_t<double, double, 16, 1, 1>(c, a, pass); break;
        default: sweep_t<double, double, 2, 1, 2>(c, a, pass); break;
    }
}

static void launch_sweep_shape(gsis_ctx* c, const SweepArgs& a, int pass, int shape) {
    const int nb = base_shapes(c->p.vdf_dtype);
    if (shape >= nb) {
        if (launch_sweep_ring(c, a, pass, shape - nb)) return;
        shape = 0;   // does not fit: register-stencil sweep
    }
    if (pair_shape(c->p.vdf_dtype, shape) && !pair_ok(c)) shape = 0;   // odd nx or 1D: single velocities
    switch (c->p.vdf_dtype) {
        case GSIS_F64: sweep_f64_shape(c, a, pass, shape); break;
        case GSIS_F32: sweep_f32_shape<float>(c, a, pass, shape); break;
        case GSIS_BF16: sweep_f32_shape<__nv_bfloat16>(c, a, pass, shape); break;
        default: sweep_f32_shape<__half>(c, a, pass, shape); break;
    }
}

SweepArgs sweep_args(gsis_ctx* c) {
    SweepArgs a;
    a.H = c->m.H;
    a.nc = c->normal_components;
    a.hp_off = c->hp_off;
    a.sdi = c->sd_int;
    a.sdv = c->sd_val;
    a.itau = c->itau;
    a.itauf = c->itauf;
    a.rho_w = c->rho_w;
    a.rho_wf = c->rho_wf;
    a.recGhost = c->recGhost;
    a.recBC = c->recBC;
    a.gx4 = c->gx4;
    a.gx1 = c->gx1;
    a.gy4 = c->gy4;
    a.gy1 = c->gy1;
    a.vg = c->vg;
    return a;
}

void launch_sweep(gsis_ctx* c, int pass) {
    if (c->Nd == 0) return;
    const SweepArgs a = sweep_args(c);
    launch_sweep_shape(c, a, pass, c->sweep_shape < 0 ? 0 : c->sweep_shape);
    c->launches++;
    c->sweep_launches++;
}

// Autotuner of the sweep's tile shape: each candidate runs one backward and
// one forward pass (after one untimed warm-up pair) on a snapshot of the VDF,
// which is restored afterwards; the fastest is kept and cached for the life
// of the process per (storage type, mesh dimension, DVM cells, velocities,
// hyperplanes).  Without memory for the snapshot the first shape is used.
static std::map<std::string, int>& sweep_cache() {
    static std::map<std::string, int> m;
    return m;
}

// Fix the sweep tile shape by name (a test hook: every shape must give the
// same result); GSIS_ERR_ARG if the name is unknown or the shape cannot run
// this problem.
gsis_status force_sweep_shape(gsis_ctx* c, const char* name) {
    const int ns = sweep_num_shapes(c->p.vdf_dtype), nb = base_shapes(c->p.vdf_dtype);
    for (int sh = 0; sh < ns; ++sh) {
        if (std::string(sweep_shape_name(c->p.vdf_dtype, sh)) != name) continue;
        if (sh >= nb) {
            const int which = sh - nb;
            if (ring_bytes(c, which == 2 ? 64 : 32) == 0 || (c->p.vdf_dtype == GSIS_F64 && which == 2))
                return set_err(c, GSIS_ERR_ARG, std::string("sweep tile ") + name + " does not fit this problem");
        }
        if (pair_shape(c->p.vdf_dtype, sh) && !pair_ok(c))
            return set_err(c, GSIS_ERR_ARG, std::string("sweep tile ") + name + " needs an even nx and a 2D/3D mesh");
        c->sweep_shape = sh;
        c->tuned_Nd = c->Nd;
        c->sweep_forced = true;
        c->sweep_info = std::string("tile ") + name + " (forced)";
        return GSIS_OK;
    }
    return set_err(c, GSIS_ERR_ARG, std::string("unknown sweep tile ") + (name ? name : "(null)"));
}

gsis_status tune_sweep(gsis_ctx* c) {
    c->tuned_Nd = c->Nd;
    if (c->Nd == 0 || c->normal_components == 1) {
        c->sweep_shape = 0;
        c->sweep_info = "1D or empty: fixed shape";
        return GSIS_OK;
    }
    const std::string key = std::to_string(c->p.vdf_dtype) + "/" + std::to_string(c->normal_components) + "/" +
                            std::to_string(c->Nd) + "/" + std::to_string(c->vg.Nv) + "/" + std::to_string(c->m.H);
    auto hit = sweep_cache().find(key);
    if (hit != sweep_cache().end()) {
        c->sweep_shape = hit->second;
        c->sweep_info = std::string("tile ") + sweep_shape_name(c->p.vdf_dtype, c->sweep_shape) + " (cached)";
        return GSIS_OK;
    }
    const size_t bytes = (size_t)c->Nd * c->vg.Nv * vdf_elem_bytes(c->p.vdf_dtype);
    void* snap = dev_alloc(c, bytes);
    if (!snap) {
        c->sweep_shape = 0;
        c->sweep_info = std::string("tile ") + sweep_shape_name(c->p.vdf_dtype, 0) + " (not tuned: no memory for a snapshot)";
        return GSIS_OK;
    }
    cudaMemcpyAsync(snap, c->f, bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const SweepArgs a = sweep_args(c);
    const int ns = sweep_num_shapes(c->p.vdf_dtype);
    int best = 0;
    float best_ms = 1e30f;
    std::string info = "tile timings (ms per pass pair):";
    for (int sh = 0; sh < ns; ++sh) {
        const int nb = base_shapes(c->p.vdf_dtype);
        if (sh >= nb && ring_bytes(c, sh - nb == 2 ? 64 : 32) == 0) continue;   // window does not fit
        if (pair_shape(c->p.vdf_dtype, sh) && !pair_ok(c)) continue;
        if (sh >= nb && c->p.vdf_dtype == GSIS_F64 && sh - nb == 2) continue;
        launch_sweep_shape(c, a, 1, sh);
        launch_sweep_shape(c, a, 0, sh);
        cudaEventRecord(e0, c->stream);
        launch_sweep_shape(c, a, 1, sh);
        launch_sweep_shape(c, a, 0, sh);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        info += std::string(" ") + sweep_shape_name(c->p.vdf_dtype, sh) + "=" + std::to_string(ms);
        if (ms < best_ms) { best_ms = ms; best = sh; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(c->f, snap, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "sweep autotuning")) return GSIS_ERR_CUDA;
    dev_free(c, snap);
    if (!cuda_ok(c, cudaGetLastError(), "sweep autotuning")) return GSIS_ERR_CUDA;
    c->sweep_shape = best;
    sweep_cache()[key] = best;
    c->sweep_info = std::string("tile ") + sweep_shape_name(c->p.vdf_dtype, best) + " (autotuned; " + info + ")";
    return GSIS_OK;
}

}  // namespace gsis
