// The FP32-arithmetic kinetic sweep on pairs of velocities (FP32 / BF16 /
// FP16 storage): the same update as compute_cells in sweep_device.cuh, with
// each thread owning two consecutive velocities (ix, ix + 1) of one x-row
// instead of one.  The pair is loaded and stored as one 8-byte (FP32) or
// 4-byte (BF16 / FP16) word, shares its y-z factors of g~/tau, and is updated
// with the packed FP32 instructions of sm_103a (fma / add / sub / mul
// .rn.f32x2, two lanes per instruction); only the limiter (minmod), the
// outflow tests and their selects act per component.  Every operation and
// rounding is that of the single-velocity update, so the results are the
// same.  Needs an even nx (a pair never crosses an x-row).
#pragma once
#include "sweep_device.cuh"

namespace gsis {

// ---------------------------------------------------------------- packed FP32 arithmetic
__device__ __forceinline__ unsigned long long pk(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {   // a * b + c, each rounded once
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 hmm2(float2 a, float2 b) {
    return make_float2(hmm_t<float>(a.x, b.x), hmm_t<float>(a.y, b.y));
}

// ---------------------------------------------------------------- paired storage access
template <typename S> __device__ __forceinline__ float2 ld2(const S* p);
template <> __device__ __forceinline__ float2 ld2<float>(const float* p) { return *reinterpret_cast<const float2*>(p); }
template <> __device__ __forceinline__ float2 ld2<__nv_bfloat16>(const __nv_bfloat16* p) {
    const unsigned w = *reinterpret_cast<const unsigned*>(p);   // element 0 in the low half
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <> __device__ __forceinline__ float2 ld2<__half>(const __half* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
}
template <typename S> __device__ __forceinline__ void st2(S* p, float2 v);
template <> __device__ __forceinline__ void st2<float>(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
template <> __device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
}
template <> __device__ __forceinline__ void st2<__half>(__half* p, float2 v) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.x, v.y);
}

// Pairs (v, v + 1), v = vbase + 64 u + 2 lane (u < VPT): v even, so the pair
// lies in one x-row (ix, ix + 1) and shares iy, iz.  In the ragged last tile
// the pairs past the end are clamped to the last pair and not stored.
template <int VPT, bool FULL>
struct Vel2 {
    int v[VPT];
    int ix[VPT], q[VPT];
    float2 x0[VPT];          // xi_x of both velocities
    float x1[VPT], x2[VPT];  // xi_y, xi_z (shared)
    bool on[VPT];
    __device__ __forceinline__ int idx(int u) const { return FULL ? v[0] + 64 * u : v[u]; }
    __device__ __forceinline__ bool active(int u) const { return FULL || on[u]; }
};

template <int VPT, bool FULL>
__device__ __forceinline__ void make_vel2(const VGridDev& vg, long long vbase, int lane, Vel2<VPT, FULL>& V) {
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
        const long long v = vbase + 64 * u + 2 * lane;
        V.on[u] = FULL || v < vg.Nv;
        V.v[u] = (int)(V.on[u] ? v : vg.Nv - 2);
        int ix, iy, iz;
        vsplit(V.v[u], vg.nx, vg.ny, ix, iy, iz);
        V.ix[u] = ix;
        V.q[u] = iy + vg.ny * iz;
        V.x0[u] = make_float2((float)vg.xi[ix], (float)vg.xi[ix + 1]);
        V.x1[u] = (float)vg.xi[vg.nx + iy];
        V.x2[u] = (float)vg.xi[vg.nx + vg.ny + iz];
    }
}

// g~ / tau at (ix, q) and (ix + 1, q): the five products of the x and y-z
// factor vectors (eval_g), the y-z factors shared by the pair.
__device__ __forceinline__ float2 eval_g2(const SweepArgs& a, int k, int ix, int q) {
    const int kx = k * a.vg.nx + ix, ky = k * (a.vg.ny * a.vg.nz) + q;
    const float* gx4 = static_cast<const float*>(a.gx4) + 4 * (long long)kx;
    const V4<float> xa = ld4(gx4), xb = ld4(gx4 + 4);
    const V4<float> y = ld4(static_cast<const float*>(a.gy4) + 4 * (long long)ky);
    const float2 x1 = __ldg(reinterpret_cast<const float2*>(static_cast<const float*>(a.gx1) + kx));
    const float y1 = __ldg(static_cast<const float*>(a.gy1) + ky);
    float2 g = f2mul(x1, bc2(y1));
    g = f2fma(make_float2(xa.x, xb.x), bc2(y.x), g);
    g = f2fma(make_float2(xa.y, xb.y), bc2(y.y), g);
    g = f2fma(make_float2(xa.z, xb.z), bc2(y.z), g);
    return f2fma(make_float2(xa.w, xb.w), bc2(y.w), g);
}

// xi . S for both velocities of the pair
template <int NC, int VPT, bool FULL>
__device__ __forceinline__ float2 normal2(const Vel2<VPT, FULL>& V, int u, const float* S) {
    float2 xn = f2mul(V.x0[u], bc2(S[0]));
    if constexpr (NC >= 2) xn = f2fma(bc2(V.x1[u]), bc2(S[NC >= 2 ? 1 : 0]), xn);
    if constexpr (NC >= 3) xn = f2fma(bc2(V.x2[u]), bc2(S[NC >= 3 ? 2 : 0]), xn);
    return xn;
}

// The implicit update of CB cells x VPT pairs (compute_cells with T = float).
template <int NC, int VPT, int CB, bool INTERIOR, bool FULL>
__device__ __forceinline__ void compute_cells2(const SweepArgs& a, const int* kk, const bool* kon,
                                               const Vel2<VPT, FULL>& V, const CellMeta<float, NC>* m,
                                               const float2 (*fc)[VPT], const float2 (*lo)[NC][VPT],
                                               const float2 (*hi)[NC][VPT], const float2 (*lo2)[NC][VPT],
                                               const float2 (*hi2)[NC][VPT], float2 (*fo)[VPT]) {
    const int NT = a.vg.NT, nx = a.vg.nx, ny = a.vg.ny;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const int k = kk[b];
        float2 den[VPT], num[VPT];
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
            den[u] = bc2(m[b].it);
            num[u] = eval_g2(a, k, V.ix[u], V.q[u]);
        }
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const int kl = INTERIOR ? SK_DVM : side_kind(m[b].kinds, 2 * d);
            const int kh = INTERIOR ? SK_DVM : side_kind(m[b].kinds, 2 * d + 1);
            if (kl == SK_NONE && kh == SK_NONE) continue;
            const float *bsl = nullptr, *btl = nullptr, *bsh = nullptr, *bth = nullptr;
            float scl = 1.0f, sch = 1.0f;
            if (!INTERIOR) {
                if (kl == SK_GHOST || kl == SK_FAR || kl == SK_WALL) {
                    const Records& R = kl == SK_GHOST ? a.recGhost : a.recBC;
                    bsl = RecT<float>::scal(R, m[b].rf[2 * d]);
                    btl = RecT<float>::tab(R, m[b].rf[2 * d], NT);
                    if (kl == SK_WALL) scl = __ldg(a.rho_wf + (long long)k * 6 + 2 * d);
                }
                if (kh == SK_GHOST || kh == SK_FAR || kh == SK_WALL) {
                    const Records& R = kh == SK_GHOST ? a.recGhost : a.recBC;
                    bsh = RecT<float>::scal(R, m[b].rf[2 * d + 1]);
                    bth = RecT<float>::tab(R, m[b].rf[2 * d + 1], NT);
                    if (kh == SK_WALL) sch = __ldg(a.rho_wf + (long long)k * 6 + 2 * d + 1);
                }
            }
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                const float2 c0 = fc[b][u], vl = lo[b][d][u], vh = hi[b][d][u];
                const float2 dl = f2sub(c0, vl), dh = f2sub(vh, c0);
                const float2 hown = hmm2(dl, dh);
                if (kl != SK_NONE) {
                    const float2 xn = normal2<NC>(V, u, m[b].S[2 * d]);
                    float2 fin;
                    if (kl == SK_DVM) {
                        fin = f2add(vl, hmm2(f2sub(vl, lo2[b][d][u]), dl));
                    } else {
                        const int iz = V.q[u] / ny, iy = V.q[u] - ny * iz;
                        fin = make_float2(scl * eval_recT<float>(bsl, btl, NT, nx, ny, V.ix[u], iy, iz),
                                          scl * eval_recT<float>(bsl, btl, NT, nx, ny, V.ix[u] + 1, iy, iz));
                    }
                    const bool ox = xn.x > 0.0f, oy = xn.y > 0.0f;
                    den[u] = f2add(den[u], make_float2(ox ? xn.x : 0.0f, oy ? xn.y : 0.0f));
                    // num - xn * (out ? -hown : fin)
                    num[u] = f2fma(make_float2(-xn.x, -xn.y), make_float2(ox ? -hown.x : fin.x, oy ? -hown.y : fin.y),
                                   num[u]);
                }
                if (kh != SK_NONE) {
                    const float2 xn = normal2<NC>(V, u, m[b].S[2 * d + 1]);
                    float2 fin;
                    if (kh == SK_DVM) {
                        fin = f2sub(vh, hmm2(dh, f2sub(hi2[b][d][u], vh)));
                    } else {
                        const int iz = V.q[u] / ny, iy = V.q[u] - ny * iz;
                        fin = make_float2(sch * eval_recT<float>(bsh, bth, NT, nx, ny, V.ix[u], iy, iz),
                                          sch * eval_recT<float>(bsh, bth, NT, nx, ny, V.ix[u] + 1, iy, iz));
                    }
                    const bool ox = xn.x > 0.0f, oy = xn.y > 0.0f;
                    den[u] = f2add(den[u], make_float2(ox ? xn.x : 0.0f, oy ? xn.y : 0.0f));
                    num[u] = f2fma(make_float2(-xn.x, -xn.y), make_float2(ox ? hown.x : fin.x, oy ? hown.y : fin.y),
                                   num[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < VPT; ++u) fo[b][u] = make_float2(__fdividef(num[u].x, den[u].x), __fdividef(num[u].y, den[u].y));
    }
}

// Gather, update and store CB cells of one hyperplane on pairs of velocities.
template <typename S, int NC, int VPT, int CB, bool INTERIOR, bool FULL>
__device__ __forceinline__ void update_cells2_k(const SweepArgs& a, S* __restrict__ f, const int* kk, const bool* kon,
                                                const Vel2<VPT, FULL>& V, const CellMeta<float, NC>* m) {
    const int Nv = (int)a.vg.Nv;
    float2 fc[CB][VPT];
    float2 lo[CB][NC][VPT], hi[CB][NC][VPT], lo2[CB][NC][VPT], hi2[CB][NC][VPT];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const S* fk = f + (long long)kk[b] * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u) fc[b][u] = ld2<S>(fk + V.idx(u));
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const bool dl = INTERIOR || side_kind(m[b].kinds, 2 * d) == SK_DVM;
            const bool dh = INTERIOR || side_kind(m[b].kinds, 2 * d + 1) == SK_DVM;
            const S* pl = f + (long long)m[b].rf[2 * d] * Nv;
            const S* ph = f + (long long)m[b].rf[2 * d + 1] * Nv;
            const S* pl2 = f + (long long)m[b].n2[2 * d] * Nv;
            const S* ph2 = f + (long long)m[b].n2[2 * d + 1] * Nv;
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                lo[b][d][u] = dl ? ld2<S>(pl + V.idx(u)) : fc[b][u];
                hi[b][d][u] = dh ? ld2<S>(ph + V.idx(u)) : fc[b][u];
                lo2[b][d][u] = dl ? ld2<S>(pl2 + V.idx(u)) : lo[b][d][u];
                hi2[b][d][u] = dh ? ld2<S>(ph2 + V.idx(u)) : hi[b][d][u];
            }
        }
    }
    float2 fo[CB][VPT];
    compute_cells2<NC, VPT, CB, INTERIOR>(a, kk, kon, V, m, fc, lo, hi, lo2, hi2, fo);
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        S* fk = f + (long long)kk[b] * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u)
            if (V.active(u)) st2<S>(fk + V.idx(u), fo[b][u]);
    }
}

template <typename S, int NC, int VPT, int CB, bool FULL>
__device__ __forceinline__ void update_cells2(const SweepArgs& a, S* __restrict__ f, const int* kk, const bool* kon,
                                             const Vel2<VPT, FULL>& V) {
    CellMeta<float, NC> m[CB];
    bool interior = a.nc == NC;
#pragma unroll
    for (int b = 0; b < CB; ++b)
        if (kon[b]) {
            load_meta<float, NC>(a, kk[b], m[b]);
            interior = interior && m[b].kinds < 0;
        }
    if (interior)
        update_cells2_k<S, NC, VPT, CB, true, FULL>(a, f, kk, kon, V, m);
    else
        update_cells2_k<S, NC, VPT, CB, false, FULL>(a, f, kk, kon, V, m);
}

}  // namespace gsis
