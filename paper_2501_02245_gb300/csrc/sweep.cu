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
// corrected Maxwellian, or rho_w M_w (diffuse wall).  One forward and one
// backward Gauss-Seidel pass over hyperplanes h = i+j+k.
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
#include "gsis_device.cuh"

namespace gsis {

struct SweepArgs {
    int H;
    const int* hp_off;
    const int* kind;      // [Nd][6]
    const int* ref;       // [Nd][6]
    const int* nb2;       // [Nd][6]
    const double* SoV;    // [Nd][6][3]
    const float* SoVf;
    const double* itau;   // [Nd] 1/tau
    const float* itauf;
    const double* rho_w;  // [Nd][6]
    const float* rho_wf;
    Records recG, recGhost, recBC;
    VGridDev vg;
};

// minmod(a, b): 0 unless a and b share a sign, else the one nearer zero.
template <typename T>
__device__ __forceinline__ T minmod_t(T a, T b) {
    const T m = fabs(a) < fabs(b) ? a : b;
    return a * b > T(0) ? m : T(0);
}

template <typename T>
__device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

// per-thread velocity data
template <typename T, int VPT>
struct Vel {
    long long v[VPT];
    int ix[VPT], iy[VPT], iz[VPT];
    T x0[VPT], x1[VPT], x2[VPT];
    bool on[VPT];
};

// metadata of one DVM cell
template <typename T, int NC>
struct CellMeta {
    int kd[2 * NC], rf[2 * NC], n2[2 * NC];
    T it;
    T S[2 * NC][NC];
    T wall[2 * NC];
};

template <typename T, int NC>
__device__ __forceinline__ void load_meta(const SweepArgs& a, int k, CellMeta<T, NC>& m) {
    const T* So = pick<T>(a.SoV, a.SoVf) + (long long)k * 18;
    const T* rw = pick<T>(a.rho_w, a.rho_wf) + (long long)k * 6;
#pragma unroll
    for (int s = 0; s < 2 * NC; ++s) {
        m.kd[s] = __ldg(a.kind + (long long)k * 6 + s);
        m.rf[s] = __ldg(a.ref + (long long)k * 6 + s);
        m.n2[s] = __ldg(a.nb2 + (long long)k * 6 + s);
#pragma unroll
        for (int q = 0; q < NC; ++q) m.S[s][q] = __ldg(So + 3 * s + q);
        m.wall[s] = __ldg(rw + s);
    }
    m.it = __ldg(pick<T>(a.itau, a.itauf) + k);
}

template <typename S, typename T, int NC, int VPT, int CB>
__device__ __forceinline__ void update_cells(const SweepArgs& a, S* __restrict__ f, const int* kk, const bool* kon,
                                             const Vel<T, VPT>& V) {
    const long long Nv = a.vg.Nv;
    const int NT = a.vg.NT, nx = a.vg.nx, ny = a.vg.ny;
    CellMeta<T, NC> m[CB];
#pragma unroll
    for (int b = 0; b < CB; ++b)
        if (kon[b]) load_meta<T, NC>(a, kk[b], m[b]);
    // ---- gather
    T fc[CB][VPT];
    T lo[CB][NC][VPT], hi[CB][NC][VPT], lo2[CB][NC][VPT], hi2[CB][NC][VPT];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const S* fk = f + (long long)kk[b] * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u) fc[b][u] = V.on[u] ? ldT<T, S>(fk + V.v[u]) : T(0);
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const bool dl = m[b].kd[2 * d] == SK_DVM, dh = m[b].kd[2 * d + 1] == SK_DVM;
            const bool dl2 = dl && m[b].n2[2 * d] >= 0, dh2 = dh && m[b].n2[2 * d + 1] >= 0;
            const S* pl = f + (long long)m[b].rf[2 * d] * Nv;
            const S* ph = f + (long long)m[b].rf[2 * d + 1] * Nv;
            const S* pl2 = f + (long long)m[b].n2[2 * d] * Nv;
            const S* ph2 = f + (long long)m[b].n2[2 * d + 1] * Nv;
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                const bool on = V.on[u];
                lo[b][d][u] = (dl && on) ? ldT<T, S>(pl + V.v[u]) : fc[b][u];
                hi[b][d][u] = (dh && on) ? ldT<T, S>(ph + V.v[u]) : fc[b][u];
                lo2[b][d][u] = (dl2 && on) ? ldT<T, S>(pl2 + V.v[u]) : lo[b][d][u];
                hi2[b][d][u] = (dh2 && on) ? ldT<T, S>(ph2 + V.v[u]) : hi[b][d][u];
            }
        }
    }
    // ---- compute and store
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const int k = kk[b];
        const T* gs = RecT<T>::scal(a.recG, k);
        const T* gt = RecT<T>::tab(a.recG, k, NT);
        T den[VPT], num[VPT];
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
            den[u] = m[b].it;
            num[u] = eval_recT<T>(gs, gt, NT, nx, ny, V.ix[u], V.iy[u], V.iz[u]) * m[b].it;
        }
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const int kl = m[b].kd[2 * d], kh = m[b].kd[2 * d + 1];
            if (kl == SK_NONE && kh == SK_NONE) continue;
            const bool both = kl == SK_DVM && kh == SK_DVM;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int s = 2 * d + side;
                const int kq = side ? kh : kl;
                if (kq == SK_NONE) continue;
                const T hs = side ? T(0.5) : T(-0.5);
                const bool has2 = m[b].n2[s] >= 0;
                const T* bs = nullptr;
                const T* bt = nullptr;
                T scale = T(1);
                if (kq == SK_GHOST) {
                    bs = RecT<T>::scal(a.recGhost, m[b].rf[s]);
                    bt = RecT<T>::tab(a.recGhost, m[b].rf[s], NT);
                } else if (kq == SK_FAR || kq == SK_WALL) {
                    bs = RecT<T>::scal(a.recBC, m[b].rf[s]);
                    bt = RecT<T>::tab(a.recBC, m[b].rf[s], NT);
                    if (kq == SK_WALL) scale = m[b].wall[s];
                }
#pragma unroll
                for (int u = 0; u < VPT; ++u) {
                    T xn = V.x0[u] * m[b].S[s][0];
                    if (NC >= 2) xn += V.x1[u] * m[b].S[s][NC >= 2 ? 1 : 0];
                    if (NC >= 3) xn += V.x2[u] * m[b].S[s][NC >= 3 ? 2 : 0];
                    const T own = both ? minmod_t<T>(fc[b][u] - lo[b][d][u], hi[b][d][u] - fc[b][u]) : T(0);
                    T fin;
                    if (kq == SK_DVM) {
                        const T fn = side ? hi[b][d][u] : lo[b][d][u];
                        const T sn = has2 ? (side ? minmod_t<T>(fn - fc[b][u], hi2[b][d][u] - fn)
                                                  : minmod_t<T>(fn - lo2[b][d][u], fc[b][u] - fn))
                                          : T(0);
                        fin = fn - hs * sn;
                    } else {
                        fin = scale * eval_recT<T>(bs, bt, NT, nx, ny, V.ix[u], V.iy[u], V.iz[u]);
                    }
                    const bool out = xn > T(0);
                    den[u] += out ? xn : T(0);
                    num[u] -= out ? xn * hs * own : xn * fin;
                }
            }
        }
        S* fk = f + (long long)k * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u)
            if (V.on[u]) stT<T, S>(fk + V.v[u], num[u] / den[u]);
    }
}

template <typename S, typename T, int NC, int G, int VPT, int CB>
__global__ void __launch_bounds__(32 * G) k_sweep(SweepArgs a, S* __restrict__ f, int pass) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Vel<T, VPT> V;
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
        V.v[u] = (long long)blockIdx.x * (32 * VPT) + 32 * u + lane;
        V.on[u] = V.v[u] < a.vg.Nv;
        int ix = 0, iy = 0, iz = 0;
        if (V.on[u]) vsplit(V.v[u], a.vg.nx, a.vg.ny, ix, iy, iz);
        V.ix[u] = ix; V.iy[u] = iy; V.iz[u] = iz;
        V.x0[u] = (T)a.vg.xi[ix];
        V.x1[u] = (T)a.vg.xi[a.vg.nx + iy];
        V.x2[u] = (T)a.vg.xi[a.vg.nx + a.vg.ny + iz];
    }
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

void launch_sweep(gsis_ctx* c, int pass) {
    if (c->Nd == 0) return;
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
