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
// A block owns 32 consecutive velocities (one per lane, so a warp reads 32
// consecutive values of a cell row: coalesced, velocity innermost) and G
// warps; warp w updates the cells k = w, w+G, ... of each hyperplane, and the
// block synchronises once per hyperplane.  Each update first gathers all the
// values of its stencil (own value, both neighbours and both second
// neighbours along each direction) and then computes without branches on the
// sign of xi.n, so the loads of consecutive cells overlap.
//
// Arithmetic type T: FP64 for an FP64 VDF (ALU-bound on GB300: 2 DFMA/clk/SM),
// FP32 for FP32 / BF16 / FP16 storage (HBM-bound).  Face-normal components
// that are zero on every face of the mesh are skipped (NC).
#include "gsis_device.cuh"

namespace gsis {

template <typename T> struct Meta;
template <> struct Meta<double> {
    static __device__ __forceinline__ const double* sov(const double* d, const float*) { return d; }
};
template <> struct Meta<float> {
    static __device__ __forceinline__ const float* sov(const double*, const float* f) { return f; }
};

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

template <int NC, typename T>
__device__ __forceinline__ T normal_speed(T x0, T x1, T x2, const T* S) {
    if (NC == 1) return x0 * S[0];
    if (NC == 2) return x0 * S[0] + x1 * S[1];
    return x0 * S[0] + x1 * S[1] + x2 * S[2];
}

template <typename T>
__device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

// Values of the stencil of one (cell, velocity) point along direction d.
template <typename T>
struct Stencil {
    T lo, hi, lo2, hi2;
};

template <typename S, typename T, int NC>
__device__ __forceinline__ void update_point(const SweepArgs& a, S* __restrict__ f, int k, long long v, int ix, int iy,
                                             int iz, T x0, T x1, T x2) {
    const long long Nv = a.vg.Nv;
    const int NT = a.vg.NT, nx = a.vg.nx, ny = a.vg.ny;
    const int* kind = a.kind + (long long)k * 6;
    const int* ref = a.ref + (long long)k * 6;
    const int* nb2 = a.nb2 + (long long)k * 6;
    constexpr int ND = 3;    // index directions (a direction whose sides are NONE costs only integer tests)
    // ---- gather
    S* fk = f + (long long)k * Nv + v;
    const T fc = ldT<T, S>(fk);
    Stencil<T> st[3];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const bool dl = kind[2 * d] == SK_DVM, dh = kind[2 * d + 1] == SK_DVM;
        st[d].lo = dl ? ldT<T, S>(f + (long long)ref[2 * d] * Nv + v) : fc;
        st[d].hi = dh ? ldT<T, S>(f + (long long)ref[2 * d + 1] * Nv + v) : fc;
        st[d].lo2 = (dl && nb2[2 * d] >= 0) ? ldT<T, S>(f + (long long)nb2[2 * d] * Nv + v) : st[d].lo;
        st[d].hi2 = (dh && nb2[2 * d + 1] >= 0) ? ldT<T, S>(f + (long long)nb2[2 * d + 1] * Nv + v) : st[d].hi;
    }
    // ---- compute
    const T it = pick<T>(a.itau, a.itauf)[k];
    T den = it;
    T num = eval_recT<T>(RecT<T>::scal(a.recG, k), RecT<T>::tab(a.recG, k, NT), NT, nx, ny, ix, iy, iz) * it;
    const T* So = pick<T>(a.SoV, a.SoVf) + (long long)k * 18;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const int kl = kind[2 * d], kh = kind[2 * d + 1];
        // own limited slope (both neighbours DVM), else 0; unused neighbour values equal fc
        const T own = (kl == SK_DVM && kh == SK_DVM) ? minmod_t<T>(fc - st[d].lo, st[d].hi - fc) : T(0);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int s = 2 * d + side;
            const int kd = side ? kh : kl;
            if (kd == SK_NONE) continue;
            const T xn = normal_speed<NC, T>(x0, x1, x2, So + 3 * s);
            const T hs = side ? T(0.5) : T(-0.5);
            T fin;
            if (kd == SK_DVM) {
                const T fn = side ? st[d].hi : st[d].lo;
                const bool has2 = nb2[s] >= 0;
                const T sn = has2 ? (side ? minmod_t<T>(fn - fc, st[d].hi2 - fn) : minmod_t<T>(fn - st[d].lo2, fc - fn))
                                  : T(0);
                fin = fn - hs * sn;
            } else if (kd == SK_GHOST) {
                fin = eval_recT<T>(RecT<T>::scal(a.recGhost, ref[s]), RecT<T>::tab(a.recGhost, ref[s], NT), NT, nx, ny,
                                   ix, iy, iz);
            } else if (kd == SK_FAR) {
                fin = eval_recT<T>(RecT<T>::scal(a.recBC, ref[s]), RecT<T>::tab(a.recBC, ref[s], NT), NT, nx, ny, ix,
                                   iy, iz);
            } else {
                fin = pick<T>(a.rho_w, a.rho_wf)[(long long)k * 6 + s] *
                      eval_recT<T>(RecT<T>::scal(a.recBC, ref[s]), RecT<T>::tab(a.recBC, ref[s], NT), NT, nx, ny, ix,
                                   iy, iz);
            }
            const bool out = xn > T(0);
            den += out ? xn : T(0);
            num -= out ? xn * hs * own : xn * fin;
        }
    }
    stT<T, S>(fk, num / den);
}

template <typename S, typename T, int NC, int G>
__global__ void __launch_bounds__(32 * G) k_sweep(SweepArgs a, S* __restrict__ f, int pass) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long v = (long long)blockIdx.x * 32 + lane;
    const bool active = v < a.vg.Nv;
    int ix = 0, iy = 0, iz = 0;
    if (active) vsplit(v, a.vg.nx, a.vg.ny, ix, iy, iz);
    const T x0 = (T)a.vg.xi[ix], x1 = (T)a.vg.xi[a.vg.nx + iy], x2 = (T)a.vg.xi[a.vg.nx + a.vg.ny + iz];
    for (int hh = 0; hh < a.H; ++hh) {
        const int h = pass ? (a.H - 1 - hh) : hh;
        const int kb = a.hp_off[h], ke = a.hp_off[h + 1];
        if (active) {
            if (pass == 0) {
                for (int k = kb + w; k < ke; k += G) update_point<S, T, NC>(a, f, k, v, ix, iy, iz, x0, x1, x2);
            } else {
                for (int k = ke - 1 - w; k >= kb; k -= G) update_point<S, T, NC>(a, f, k, v, ix, iy, iz, x0, x1, x2);
            }
        }
        if (G > 1) __syncthreads();
    }
}

template <typename S, typename T, int G>
static void sweep_t(gsis_ctx* c, const SweepArgs& a, int pass) {
    const unsigned blocks = (unsigned)((c->vg.Nv + 31) / 32);
    S* f = (S*)c->f;
    switch (c->normal_components) {
        case 1: k_sweep<S, T, 1, G><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass); break;
        case 2: k_sweep<S, T, 2, G><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass); break;
        default: k_sweep<S, T, 3, G><<<blocks, 32 * G, 0, c->stream>>>(a, f, pass); break;
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
        case GSIS_F64: sweep_t<double, double, 2>(c, a, pass); break;
        case GSIS_F32: sweep_t<float, float, 4>(c, a, pass); break;
        case GSIS_BF16: sweep_t<__nv_bfloat16, float, 4>(c, a, pass); break;
        default: sweep_t<__half, float, 4>(c, a, pass); break;
    }
    c->launches++;
    c->sweep_launches++;
}

}  // namespace gsis
