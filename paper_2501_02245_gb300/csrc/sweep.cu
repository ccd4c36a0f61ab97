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
// Every dependency of the update at (c, xi) is on the same velocity xi, so one
// thread owns one velocity and marches through all DVM cells in hyperplane
// order: the whole pass is a single launch without barriers, and a warp reads
// 32 consecutive velocities of one cell row (coalesced, velocity innermost).
#include "gsis_device.cuh"

namespace gsis {

struct SweepArgs {
    int H;
    const int* hp_off;
    const int* kind;      // [Nd][6]
    const int* ref;       // [Nd][6]
    const int* nb2;       // [Nd][6]
    const double* SoV;    // [Nd][6][3]
    const double* tau;    // [Nd]
    const double* rho_w;  // [Nd][6]
    Records recG, recGhost, recBC;
    VGridDev vg;
};

template <typename S>
__device__ __forceinline__ void update_point(const SweepArgs& a, S* __restrict__ f, int k, long long v, int ix, int iy,
                                             int iz, double x0, double x1, double x2) {
    const long long Nv = a.vg.Nv;
    const int NT = a.vg.NT, nx = a.vg.nx, ny = a.vg.ny;
    S* fk = f + (long long)k * Nv + v;
    const double fc = Store<S>::ld(fk);
    const double tau = a.tau[k];
    double den = 1.0 / tau;
    double num = eval_rec(rec_scal(a.recG, k), rec_tab(a.recG, k, NT), NT, nx, ny, ix, iy, iz) / tau;
    const int* kind = a.kind + (long long)k * 6;
    const int* ref = a.ref + (long long)k * 6;
    const int* nb2 = a.nb2 + (long long)k * 6;
    const double* So = a.SoV + (long long)k * 18;
    double own_slope[3] = {0.0, 0.0, 0.0};
    bool have[3] = {false, false, false};
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int kd = kind[s];
        if (kd == SK_NONE) continue;
        const double xn = x0 * So[3 * s] + x1 * So[3 * s + 1] + x2 * So[3 * s + 2];
        const int d = s >> 1;
        const double hs = (s & 1) ? 0.5 : -0.5;
        if (xn > 0.0) {
            if (!have[d]) {
                double sl = 0.0;
                if (kind[2 * d] == SK_DVM && kind[2 * d + 1] == SK_DVM) {
                    const double flo = Store<S>::ld(f + (long long)ref[2 * d] * Nv + v);
                    const double fhi = Store<S>::ld(f + (long long)ref[2 * d + 1] * Nv + v);
                    sl = minmod(fc - flo, fhi - fc);
                }
                own_slope[d] = sl;
                have[d] = true;
            }
            den += xn;
            num -= xn * hs * own_slope[d];
        } else {
            double fin;
            if (kd == SK_DVM) {
                const double fn = Store<S>::ld(f + (long long)ref[s] * Nv + v);
                double sn = 0.0;
                if (nb2[s] >= 0) {
                    const double f2 = Store<S>::ld(f + (long long)nb2[s] * Nv + v);
                    sn = (s & 1) ? minmod(fn - fc, f2 - fn) : minmod(fn - f2, fc - fn);
                }
                fin = fn - hs * sn;
            } else if (kd == SK_GHOST) {
                fin = eval_rec(rec_scal(a.recGhost, ref[s]), rec_tab(a.recGhost, ref[s], NT), NT, nx, ny, ix, iy, iz);
            } else if (kd == SK_FAR) {
                fin = eval_rec(rec_scal(a.recBC, ref[s]), rec_tab(a.recBC, ref[s], NT), NT, nx, ny, ix, iy, iz);
            } else {
                fin = a.rho_w[(long long)k * 6 + s] *
                      eval_rec(rec_scal(a.recBC, ref[s]), rec_tab(a.recBC, ref[s], NT), NT, nx, ny, ix, iy, iz);
            }
            num -= xn * fin;
        }
    }
    Store<S>::st(fk, num / den);
}

template <typename S>
__global__ void __launch_bounds__(128) k_sweep(SweepArgs a, S* __restrict__ f, int pass) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.vg.Nv) return;
    int ix, iy, iz;
    vsplit(v, a.vg.nx, a.vg.ny, ix, iy, iz);
    const double x0 = a.vg.xi[ix], x1 = a.vg.xi[a.vg.nx + iy], x2 = a.vg.xi[a.vg.nx + a.vg.ny + iz];
    for (int hh = 0; hh < a.H; ++hh) {
        const int h = pass ? (a.H - 1 - hh) : hh;
        const int kb = a.hp_off[h], ke = a.hp_off[h + 1];
        if (pass == 0) {
            for (int k = kb; k < ke; ++k) update_point<S>(a, f, k, v, ix, iy, iz, x0, x1, x2);
        } else {
            for (int k = ke - 1; k >= kb; --k) update_point<S>(a, f, k, v, ix, iy, iz, x0, x1, x2);
        }
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
    a.tau = c->tau;
    a.rho_w = c->rho_w;
    a.recG = c->recG;
    a.recGhost = c->recGhost;
    a.recBC = c->recBC;
    a.vg = c->vg;
    const int threads = 128;
    const long long blocks = (c->vg.Nv + threads - 1) / threads;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: k_sweep<double><<<(unsigned)blocks, threads, 0, c->stream>>>(a, (double*)c->f, pass); break;
        case GSIS_F32: k_sweep<float><<<(unsigned)blocks, threads, 0, c->stream>>>(a, (float*)c->f, pass); break;
        case GSIS_BF16:
            k_sweep<__nv_bfloat16><<<(unsigned)blocks, threads, 0, c->stream>>>(a, (__nv_bfloat16*)c->f, pass);
            break;
        default: k_sweep<__half><<<(unsigned)blocks, threads, 0, c->stream>>>(a, (__half*)c->f, pass); break;
    }
    c->launches++;
    c->sweep_launches++;
}

}  // namespace gsis
