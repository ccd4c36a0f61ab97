// Device building blocks of the kinetic step shared by the single-solve
// sweep (sweep.cu) and the batched persistent sweep (batch.cu): argument
// block, per-thread velocity data, per-cell metadata and the update of CB
// cells x VPT velocities of one hyperplane.
#pragma once
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
    const double* yzd;    // [Nd][5][ny*nz] y-z factors of the reference distribution (FP64 sweep)
    const float* yzf;     // the same in FP32 (FP32 sweep)
    VGridDev vg;
};

// minmod(a, b): 0 unless a and b share a sign, else the one nearer zero.
template <typename T>
__device__ __forceinline__ T minmod_t(T a, T b) {
    const T m = fabs(a) < fabs(b) ? a : b;
    return a * b > T(0) ? m : T(0);
}

// minmod(a, b) and x > 0 with the decisions taken on the bit patterns: for
// FP64 this keeps the comparisons and the sign product off the FP64 pipe
// (GB300 issues FP64 at 1/64 of the FP32 rate), with the same result as
// minmod_t for finite values (magnitudes of IEEE doubles order like their
// bit patterns with the sign bit cleared; +-0 never shares a sign).
template <typename T> __device__ __forceinline__ T mm_t(T a, T b);
template <> __device__ __forceinline__ float mm_t<float>(float a, float b) { return minmod_t<float>(a, b); }
template <> __device__ __forceinline__ double mm_t<double>(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    const bool same = (ia ^ ib) >= 0 && ma != 0 && mb != 0;
    return same ? (ma < mb ? a : b) : 0.0;
}
template <typename T> __device__ __forceinline__ bool pos_t(T x);
template <> __device__ __forceinline__ bool pos_t<float>(float x) { return x > 0.0f; }
template <> __device__ __forceinline__ bool pos_t<double>(double x) { return __double_as_longlong(x) > 0; }

// n / d for d > 0 in the normal range.  FP64: one Newton-Raphson step
// r <- r (2 - d r) on a single-precision reciprocal seed (relative error
// ~2^-23 -> ~2^-46) and q = n r: relative error below 2e-14, far inside the
// tolerance of the scheme's FP64 results, for three FP64 operations.  FP32:
// IEEE division.
template <typename T> __device__ __forceinline__ T div_t(T n, T d);
template <> __device__ __forceinline__ float div_t<float>(float n, float d) { return n / d; }
template <> __device__ __forceinline__ double div_t<double>(double n, double d) {
    double r = (double)__frcp_rn(__double2float_rn(d));
    r = r * fma(-d, r, 2.0);
    return n * r;
}

template <typename T>
__device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

// Reference distribution of a cell at velocity (ix, q = iy + ny iz), divided
// by tau, from the x-tables of its record and its y-z factors (k_build_yz,
// whose E_yz carries 1/tau):
//   g/tau = E_x E_yz (D_yz + B_x + (R_x + R_yz)(C2_x + C2_yz) + C_x A_yz),
// the record's E_x E_y E_z (p0 + sum B + sum R sum C2 + 2 sum_{i<j} P2_ij C_i C_j)
// with the y-z sums formed once per cell instead of once per velocity.
template <typename T>
__device__ __forceinline__ T eval_g_yz(const T* __restrict__ tab, const T* __restrict__ yz, int NT, int nyz, int ix,
                                       int q) {
    const T E = __ldg(tab + ix), B = __ldg(tab + NT + ix), C = __ldg(tab + 2 * NT + ix);
    const T C2 = __ldg(tab + 3 * NT + ix), R = __ldg(tab + 4 * NT + ix);
    const T Eyz = __ldg(yz + q), D = __ldg(yz + nyz + q), Ryz = __ldg(yz + 2 * nyz + q);
    const T Cyz = __ldg(yz + 3 * nyz + q), A = __ldg(yz + 4 * nyz + q);
    const T poly = (D + B) + (R + Ryz) * (C2 + Cyz) + C * A;
    return (E * Eyz) * poly;
}

// per-thread velocity data
template <typename T, int VPT>
struct Vel {
    long long v[VPT];
    int ix[VPT], iy[VPT], iz[VPT], q[VPT];   // q = iy + ny iz
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

// The implicit update of CB cells x VPT velocities from their gathered
// stencils (own value fc, neighbours lo/hi and second neighbours lo2/hi2 per
// direction; a missing neighbour repeats the nearer value): new values in fo.
template <typename T, int NC, int VPT, int CB>
__device__ __forceinline__ void compute_cells(const SweepArgs& a, const int* kk, const bool* kon,
                                              const Vel<T, VPT>& V, const CellMeta<T, NC>* m, const T (*fc)[VPT],
                                              const T (*lo)[NC][VPT], const T (*hi)[NC][VPT],
                                              const T (*lo2)[NC][VPT], const T (*hi2)[NC][VPT], T (*fo)[VPT]) {
    const int NT = a.vg.NT, nx = a.vg.nx, ny = a.vg.ny;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const int k = kk[b];
        const T* gt = RecT<T>::tab(a.recG, k, NT);
        const int nyz = ny * a.vg.nz;
        const T* yz = pick<T>(a.yzd, a.yzf) + (long long)k * 5 * nyz;
        T den[VPT], num[VPT];
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
            den[u] = m[b].it;
            num[u] = eval_g_yz<T>(gt, yz, NT, nyz, V.ix[u], V.q[u]);   // g~ / tau
        }
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const int kl = m[b].kd[2 * d], kh = m[b].kd[2 * d + 1];
            if (kl == SK_NONE && kh == SK_NONE) continue;
            const bool both = kl == SK_DVM && kh == SK_DVM;
            const bool l2 = m[b].n2[2 * d] >= 0, h2 = m[b].n2[2 * d + 1] >= 0;
            // interface / boundary distributions of the non-DVM sides (the side
            // kinds are the same for every lane of the warp: uniform branches)
            const T *bsl = nullptr, *btl = nullptr, *bsh = nullptr, *bth = nullptr;
            T scl = T(1), sch = T(1);
            if (kl == SK_GHOST || kl == SK_FAR || kl == SK_WALL) {
                const Records& R = kl == SK_GHOST ? a.recGhost : a.recBC;
                bsl = RecT<T>::scal(R, m[b].rf[2 * d]);
                btl = RecT<T>::tab(R, m[b].rf[2 * d], NT);
                if (kl == SK_WALL) scl = m[b].wall[2 * d];
            }
            if (kh == SK_GHOST || kh == SK_FAR || kh == SK_WALL) {
                const Records& R = kh == SK_GHOST ? a.recGhost : a.recBC;
                bsh = RecT<T>::scal(R, m[b].rf[2 * d + 1]);
                bth = RecT<T>::tab(R, m[b].rf[2 * d + 1], NT);
                if (kh == SK_WALL) sch = m[b].wall[2 * d + 1];
            }
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                const T c0 = fc[b][u], vl = lo[b][d][u], vh = hi[b][d][u];
                // half the cell's own limited slope (outgoing face values c0 -+ hown)
                const T hown = both ? T(0.5) * mm_t<T>(c0 - vl, vh - c0) : T(0);
                if (kl != SK_NONE) {
                    T xn = V.x0[u] * m[b].S[2 * d][0];
                    if (NC >= 2) xn += V.x1[u] * m[b].S[2 * d][NC >= 2 ? 1 : 0];
                    if (NC >= 3) xn += V.x2[u] * m[b].S[2 * d][NC >= 3 ? 2 : 0];
                    T fin;
                    if (kl == SK_DVM)   // neighbour's face value: its value plus half its limited slope
                        fin = fma(T(0.5), l2 ? mm_t<T>(vl - lo2[b][d][u], c0 - vl) : T(0), vl);
                    else
                        fin = scl * eval_recT<T>(bsl, btl, NT, nx, ny, V.ix[u], V.iy[u], V.iz[u]);
                    const bool out = pos_t<T>(xn);
                    den[u] += out ? xn : T(0);
                    num[u] -= xn * (out ? -hown : fin);
                }
                if (kh != SK_NONE) {
                    T xn = V.x0[u] * m[b].S[2 * d + 1][0];
                    if (NC >= 2) xn += V.x1[u] * m[b].S[2 * d + 1][NC >= 2 ? 1 : 0];
                    if (NC >= 3) xn += V.x2[u] * m[b].S[2 * d + 1][NC >= 3 ? 2 : 0];
                    T fin;
                    if (kh == SK_DVM)
                        fin = fma(T(-0.5), h2 ? mm_t<T>(vh - c0, hi2[b][d][u] - vh) : T(0), vh);
                    else
                        fin = sch * eval_recT<T>(bsh, bth, NT, nx, ny, V.ix[u], V.iy[u], V.iz[u]);
                    const bool out = pos_t<T>(xn);
                    den[u] += out ? xn : T(0);
                    num[u] -= xn * (out ? hown : fin);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < VPT; ++u) fo[b][u] = div_t<T>(num[u], den[u]);
    }
}

template <typename S, typename T, int NC, int VPT, int CB>
__device__ __forceinline__ void update_cells(const SweepArgs& a, S* __restrict__ f, const int* kk, const bool* kon,
                                             const Vel<T, VPT>& V) {
    const long long Nv = a.vg.Nv;
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
    T fo[CB][VPT];
    compute_cells<T, NC, VPT, CB>(a, kk, kon, V, m, fc, lo, hi, lo2, hi2, fo);
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        S* fk = f + (long long)kk[b] * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u)
            if (V.on[u]) stT<T, S>(fk + V.v[u], fo[b][u]);
    }
}

// Velocities vbase + 32 u + lane (u < VPT) of the grid: flat index, axis
// indices and node values.
template <typename T, int VPT>
__device__ __forceinline__ void make_vel(const VGridDev& vg, long long vbase, int lane, Vel<T, VPT>& V) {
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
        V.v[u] = vbase + 32 * u + lane;
        V.on[u] = V.v[u] < vg.Nv;
        int ix = 0, iy = 0, iz = 0;
        if (V.on[u]) vsplit(V.v[u], vg.nx, vg.ny, ix, iy, iz);
        V.ix[u] = ix; V.iy[u] = iy; V.iz[u] = iz; V.q[u] = iy + vg.ny * iz;
        V.x0[u] = (T)vg.xi[ix];
        V.x1[u] = (T)vg.xi[vg.nx + iy];
        V.x2[u] = (T)vg.xi[vg.nx + vg.ny + iz];
    }
}

SweepArgs sweep_args(gsis_ctx* c);

// One solve of a batched sweep.
struct BatchSolve {
    SweepArgs a;
    void* f;      // VDF rows of this solve
    int dtype;    // GSIS_F64 / F32 / BF16 / F16
};

}  // namespace gsis
