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
        V.ix[u] = ix; V.iy[u] = iy; V.iz[u] = iz;
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
