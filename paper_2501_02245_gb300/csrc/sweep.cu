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
#include "sweep_device.cuh"

namespace gsis {

template <typename S, typename T, int NC, int G, int VPT, int CB>
__global__ void __launch_bounds__(32 * G) k_sweep(SweepArgs a, S* __restrict__ f, int pass) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Vel<T, VPT> V;
    make_vel<T, VPT>(a.vg, (long long)blockIdx.x * (32 * VPT), lane, V);
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

SweepArgs sweep_args(gsis_ctx* c) {
    SweepArgs a;
    a.H = c->m.H;
    a.hp_off = c->hp_off;
    a.kind = c->dside_kind;
    a.ref = c->dside_ref;
    a.nb2 = c->dside_nb2;
    a.SoV = c->SoV;
    a.SoVf = c->SoVf;
    a.itau = c->itau;
    a.itauf = c->itauf;
    a.rho_w = c->rho_w;
    a.rho_wf = c->rho_wf;
    a.recG = c->recG;
    a.recGhost = c->recGhost;
    a.recBC = c->recBC;
    a.vg = c->vg;
    return a;
}

void launch_sweep(gsis_ctx* c, int pass) {
    if (c->Nd == 0) return;
    const SweepArgs a = sweep_args(c);
    switch (c->p.vdf_dtype) {
        case GSIS_F64: sweep_t<double, double, 2, 1, 2>(c, a, pass); break;
        case GSIS_F32: sweep_t<float, float, 4, 2, 2>(c, a, pass); break;
        case GSIS_BF16: sweep_t<__nv_bfloat16, float, 4, 2, 2>(c, a, pass); break;
        default: sweep_t<__half, float, 4, 2, 2>(c, a, pass); break;
    }
    c->launches++;
    c->sweep_launches++;
}

}  // namespace gsis
