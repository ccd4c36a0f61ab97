// Device building blocks of the kinetic step shared by the single-solve
// sweep (sweep.cu) and the batched persistent sweep (batch.cu): argument
// block, per-thread velocity data, per-cell metadata and the update of CB
// cells x VPT velocities of one hyperplane.
#pragma once
#include <type_traits>
#include "gsis_device.cuh"

namespace gsis {

// Packed per-cell data of the sweep (k_sweep_desc, rebuilt with the DVM
// region).  Integers, SD_INTS per cell: [0..3] neighbour row (DVM side) or
// record index (ghost / boundary side) of sides 0..3, [4..7] second-neighbour
// rows of sides 0..3, [8..9] / [10..11] the same for sides 4..5, [12] the side
// kinds (3 bits per side) with bit 31 set when every side that carries flux
// is a DVM side.  Where a DVM side has no second neighbour its entry repeats
// the neighbour's row: the slope test then sees a zero difference and gives a
// zero slope, the value the scheme prescribes there, without a branch.
// Values, SD_VALS per cell in the arithmetic type: S/V component-major,
// [q * 8 + s] for component q < 3 of side s < 6.
// (SD_INTS = 16, SD_VALS = 24: gsis_internal.h.)
struct SweepArgs {
    int H;
    int nc;               // index directions of the mesh that carry flux (the all-DVM bit refers to these)
    const int* hp_off;
    const int* sdi;       // [Nd][SD_INTS]
    const void* sdv;      // [Nd][SD_VALS], double (FP64 sweep) or float
    const double* itau;   // [Nd] 1/tau
    const float* itauf;
    const double* rho_w;  // [Nd][6]
    const float* rho_wf;
    Records recGhost, recBC;
    // factor vectors of the reference distribution (k_build_gtab), in the
    // arithmetic type: gx4/gx1 [Nd][nx] (4-vector, scalar), gy4/gy1 [Nd][ny*nz]
    const void *gx4, *gx1, *gy4, *gy1;
    VGridDev vg;
};

// -x if s else x (FP64: a flip of the sign bit on the integer pipe).
template <typename T> __device__ __forceinline__ T neg_if(T x, bool s);
template <> __device__ __forceinline__ float neg_if<float>(float x, bool s) {
    return __uint_as_float(__float_as_uint(x) ^ ((unsigned)s << 31));
}
template <> __device__ __forceinline__ double neg_if<double>(double x, bool s) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)s << 63));
}
// x > 0 (FP64: on the bit pattern, integer pipe).
template <typename T> __device__ __forceinline__ bool pos_t(T x);
template <> __device__ __forceinline__ bool pos_t<float>(float x) { return x > 0.0f; }
template <> __device__ __forceinline__ bool pos_t<double>(double x) { return __double_as_longlong(x) > 0; }

// n / d for d > 0 with d and 1/d within the normal single-precision range
// (the denominators of the sweep, 1/tau plus outflow terms, are).
// FP64: a single-precision reciprocal seed, then one Newton-Raphson step
// r <- r (2 - d r) and q = n r.  The seed moves d into single precision and
// back on the integer pipe: the sign-less exponent and top 23 fraction bits
// of d, shifted into place, with the exponent rebias 1023 - 127 = 896 folded
// into one subtraction (d truncated: relative error < 2^-23), and the
// approximate hardware reciprocal (rcp.approx.ftz.f32, within 1 ulp).  The
// seed's relative error is below 2^-21.9, after the Newton step below
// 2^-43.8 plus rounding: under 1e-13, far inside the tolerance of the
// scheme's FP64 results, for three FP64 operations and none of the
// double <-> float conversions (which occupy the FP64 pipe).
// FP32: the fast single-precision quotient (__fdividef, within 2 ulp).
template <typename T> __device__ __forceinline__ T div_t(T n, T d);
template <> __device__ __forceinline__ float div_t<float>(float n, float d) { return __fdividef(n, d); }
template <> __device__ __forceinline__ double div_t<double>(double n, double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned fb = (unsigned)(b >> 29) - 0xC0000000u;   // (exponent - 896) << 23 | top 23 fraction bits
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(fb)));
    const unsigned long long rb = ((unsigned long long)__float_as_uint(rf) << 29) + (896ULL << 52);
    double r = __longlong_as_double((long long)rb);
    r = r * fma(-d, r, 2.0);
    return n * r;
}

template <typename T>
__device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

template <typename T> struct V4 { T x, y, z, w; };
__device__ __forceinline__ V4<float> ld4(const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
    const double2 u = __ldg(reinterpret_cast<const double2*>(p)), v = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {u.x, u.y, v.x, v.y};
}

// Reference distribution of cell k at velocity (ix, q = iy + ny iz), divided
// by tau.  The record's E_x E_y E_z (p0 + sum B + sum R sum C2
// + 2 sum_{i<j} P2_ij C_i C_j), split into its x and y-z parts, is the sum of
// five products x_i y_i (k_build_gtab):
//   x = (E_x, E_x (B_x + R_x C2_x), E_x R_x, E_x C2_x, E_x C_x)
//   y = E_yz/tau (D + R_yz C2_yz, 1, C2_yz, R_yz, A)
// with E_yz = E_y E_z, D = p0 + B_y + B_z + 2 P2_yz C_y C_z, R_yz = R_y + R_z,
// C2_yz = C2_y + C2_z and A = 2 (P2_xy C_y + P2_xz C_z).
template <typename T>
__device__ __forceinline__ T eval_g(const SweepArgs& a, int k, int ix, int q) {
    const int kx = k * a.vg.nx + ix, ky = k * (a.vg.ny * a.vg.nz) + q;
    const V4<T> x = ld4(static_cast<const T*>(a.gx4) + 4 * (long long)kx);
    const V4<T> y = ld4(static_cast<const T*>(a.gy4) + 4 * (long long)ky);
    T g = __ldg(static_cast<const T*>(a.gx1) + kx) * __ldg(static_cast<const T*>(a.gy1) + ky);
    g = fma(x.x, y.x, g);
    g = fma(x.y, y.y, g);
    g = fma(x.z, y.z, g);
    return fma(x.w, y.w, g);
}

// per-thread velocity data.  In the ragged last tile of the grid the
// velocities past the end are clamped to the last one: their loads stay in
// bounds and their results are not stored.  FULL: the tile lies inside the
// grid, so slot u is velocity v[0] + 32 u (the loads of a row then share one
// address plus constant offsets) and every result is stored.
template <typename T, int VPT, bool FULL = false>
struct Vel {
    int v[VPT];             // flat velocity index (clamped)
    int ix[VPT], q[VPT];    // q = iy + ny iz
    T x0[VPT], x1[VPT], x2[VPT];
    bool on[VPT];
    __device__ __forceinline__ int idx(int u) const { return FULL ? v[0] + 32 * u : v[u]; }
    __device__ __forceinline__ bool active(int u) const { return FULL || on[u]; }
};

// metadata of one DVM cell
template <typename T, int NC>
struct CellMeta {
    int kinds;              // packed side kinds, bit 31: every flux side is a DVM side
    int rf[2 * NC], n2[2 * NC];
    T S[2 * NC][NC];
    T it;
};

__device__ __forceinline__ int side_kind(int kinds, int s) { return (kinds >> (3 * s)) & 7; }

template <typename T>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b) {
    a = __ldg(p);
    b = __ldg(p + 1);
}

template <typename T, int NC>
__device__ __forceinline__ void load_meta(const SweepArgs& a, int k, CellMeta<T, NC>& m) {
    const int* p = a.sdi + (long long)k * SD_INTS;
    const int4 r = __ldg(reinterpret_cast<const int4*>(p)), r2 = __ldg(reinterpret_cast<const int4*>(p) + 1);
    m.kinds = __ldg(p + 12);
    m.rf[0] = r.x; m.rf[1] = r.y; m.n2[0] = r2.x; m.n2[1] = r2.y;
    if constexpr (NC >= 2) { m.rf[2] = r.z; m.rf[3] = r.w; m.n2[2] = r2.z; m.n2[3] = r2.w; }
    if constexpr (NC >= 3) {
        const int4 r3 = __ldg(reinterpret_cast<const int4*>(p) + 2);
        m.rf[4] = r3.x; m.rf[5] = r3.y; m.n2[4] = r3.z; m.n2[5] = r3.w;
    }
    const T* sv = static_cast<const T*>(a.sdv) + (long long)k * SD_VALS;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        if constexpr (NC == 1) {
            ld2<T>(sv, m.S[0][0], m.S[1][0]);
        } else {
            const V4<T> v = ld4(sv + 8 * q);
            m.S[0][q] = v.x; m.S[1][q] = v.y; m.S[2][q] = v.z; m.S[3][q] = v.w;
            if constexpr (NC >= 3) ld2<T>(sv + 8 * q + 4, m.S[4][q], m.S[5][q]);
        }
    }
    m.it = __ldg(pick<T>(a.itau, a.itauf) + k);
}

// The implicit update of CB cells x VPT velocities from their gathered
// stencils (own value fc, neighbours lo/hi and second neighbours lo2/hi2 per
// direction; a side that is not a DVM side repeats the own value, a missing
// second neighbour the neighbour's): new values in fo.  INTERIOR: every flux
// side of every cell is a DVM side (compiled without the side-kind branches).
template <typename T, int NC, int VPT, int CB, bool INTERIOR, typename VelT>
__device__ __forceinline__ void compute_cells(const SweepArgs& a, const int* kk, const bool* kon,
                                              const VelT& V, const CellMeta<T, NC>* m, const T (*fc)[VPT],
                                              const T (*lo)[NC][VPT], const T (*hi)[NC][VPT],
                                              const T (*lo2)[NC][VPT], const T (*hi2)[NC][VPT], T (*fo)[VPT]) {
    const int NT = a.vg.NT, nx = a.vg.nx, ny = a.vg.ny;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const int k = kk[b];
        T den[VPT], num[VPT];
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
            den[u] = m[b].it;
            num[u] = eval_g<T>(a, k, V.ix[u], V.q[u]);   // g~ / tau
        }
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const int kl = INTERIOR ? SK_DVM : side_kind(m[b].kinds, 2 * d);
            const int kh = INTERIOR ? SK_DVM : side_kind(m[b].kinds, 2 * d + 1);
            if (kl == SK_NONE && kh == SK_NONE) continue;
            // interface / boundary distributions of the non-DVM sides (the side
            // kinds are the same for every lane of the warp: uniform branches)
            const T *bsl = nullptr, *btl = nullptr, *bsh = nullptr, *bth = nullptr;
            T scl = T(1), sch = T(1);
            if (!INTERIOR) {
                if (kl == SK_GHOST || kl == SK_FAR || kl == SK_WALL) {
                    const Records& R = kl == SK_GHOST ? a.recGhost : a.recBC;
                    bsl = RecT<T>::scal(R, m[b].rf[2 * d]);
                    btl = RecT<T>::tab(R, m[b].rf[2 * d], NT);
                    if (kl == SK_WALL) scl = __ldg(pick<T>(a.rho_w, a.rho_wf) + (long long)k * 6 + 2 * d);
                }
                if (kh == SK_GHOST || kh == SK_FAR || kh == SK_WALL) {
                    const Records& R = kh == SK_GHOST ? a.recGhost : a.recBC;
                    bsh = RecT<T>::scal(R, m[b].rf[2 * d + 1]);
                    bth = RecT<T>::tab(R, m[b].rf[2 * d + 1], NT);
                    if (kh == SK_WALL) sch = __ldg(pick<T>(a.rho_w, a.rho_wf) + (long long)k * 6 + 2 * d + 1);
                }
            }
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                const T c0 = fc[b][u], vl = lo[b][d][u], vh = hi[b][d][u];
                const T dl = c0 - vl, dh = vh - c0;
                // half the cell's own limited slope (outgoing face values c0 -+ hown);
                // zero next to a side that is not a DVM side (its value repeats c0)
                const T hown = hmm_t<T>(dl, dh);
                if constexpr (INTERIOR && std::is_same<T, double>::value) {
                    // (FP64 arithmetic, where the FP64 pipe bounds the sweep; in FP32
                    // the votes and selects cost more issue slots than they save.)
                    // Both sides are DVM sides.  Usually one face of the pair is an
                    // inflow face and the other an outflow face (the radial faces of
                    // an O-grid cell always are): then only the inflow side's MUSCL
                    // face value is needed, formed once from operands selected by
                    // the outflow test of the low side.  Lanes whose two faces are
                    // both inflow (one more face value) or both outflow (one more
                    // outflow term) are fixed up under warp-uniform branches.  Every
                    // case takes the operations and summation order of the general
                    // update below, so the results are the same.
                    T xL = V.x0[u] * m[b].S[2 * d][0];
                    if constexpr (NC >= 2) xL = fma(V.x1[u], m[b].S[2 * d][NC >= 2 ? 1 : 0], xL);
                    if constexpr (NC >= 3) xL = fma(V.x2[u], m[b].S[2 * d][NC >= 3 ? 2 : 0], xL);
                    T xH = V.x0[u] * m[b].S[2 * d + 1][0];
                    if constexpr (NC >= 2) xH = fma(V.x1[u], m[b].S[2 * d + 1][NC >= 2 ? 1 : 0], xH);
                    if constexpr (NC >= 3) xH = fma(V.x2[u], m[b].S[2 * d + 1][NC >= 3 ? 2 : 0], xH);
                    const bool oL = pos_t<T>(xL), oH = pos_t<T>(xH);
                    // face value of the low side (vl + h, low side inflow) or of the
                    // high side (vh - h, low side outflow)
                    // (operands selected first: one subtraction, vh2 - vh or vl - vl2)
                    const T e = (oL ? hi2[b][d][u] : vl) - (oL ? vh : lo2[b][d][u]);
                    const T h = hmm_t<T>(e, oL ? dh : dl);
                    const T fin = (oL ? vh : vl) + neg_if<T>(h, oL);
                    T selH = oH ? hown : fin;
                    const bool both_in = !oL && !oH, both_out = oL && oH;
                    if (__any_sync(0xffffffffu, both_in)) {
                        const T fH = vh - hmm_t<T>(dh, hi2[b][d][u] - vh);
                        if (both_in) selH = fH;
                    }
                    den[u] += oL ? xL : (oH ? xH : T(0));
                    num[u] = fma(-xL, oL ? -hown : fin, num[u]);
                    if (__any_sync(0xffffffffu, both_out)) {
                        if (both_out) den[u] += xH;
                    }
                    num[u] = fma(-xH, selH, num[u]);
                    continue;
                }
                if (kl != SK_NONE) {
                    T xn = V.x0[u] * m[b].S[2 * d][0];
                    if constexpr (NC >= 2) xn = fma(V.x1[u], m[b].S[2 * d][NC >= 2 ? 1 : 0], xn);
                    if constexpr (NC >= 3) xn = fma(V.x2[u], m[b].S[2 * d][NC >= 3 ? 2 : 0], xn);
                    T fin;
                    if (kl == SK_DVM) {   // neighbour's face value: its value plus half its limited slope
                        fin = vl + hmm_t<T>(vl - lo2[b][d][u], dl);
                    } else {
                        const int iz = V.q[u] / ny;
                        fin = scl * eval_recT<T>(bsl, btl, NT, nx, ny, V.ix[u], V.q[u] - ny * iz, iz);
                    }
                    const bool out = pos_t<T>(xn);
                    den[u] += out ? xn : T(0);
                    num[u] = fma(-xn, out ? -hown : fin, num[u]);
                }
                if (kh != SK_NONE) {
                    T xn = V.x0[u] * m[b].S[2 * d + 1][0];
                    if constexpr (NC >= 2) xn = fma(V.x1[u], m[b].S[2 * d + 1][NC >= 2 ? 1 : 0], xn);
                    if constexpr (NC >= 3) xn = fma(V.x2[u], m[b].S[2 * d + 1][NC >= 3 ? 2 : 0], xn);
                    T fin;
                    if (kh == SK_DVM) {
                        fin = vh - hmm_t<T>(dh, hi2[b][d][u] - vh);
                    } else {
                        const int iz = V.q[u] / ny;
                        fin = sch * eval_recT<T>(bsh, bth, NT, nx, ny, V.ix[u], V.q[u] - ny * iz, iz);
                    }
                    const bool out = pos_t<T>(xn);
                    den[u] += out ? xn : T(0);
                    num[u] = fma(-xn, out ? hown : fin, num[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < VPT; ++u) fo[b][u] = div_t<T>(num[u], den[u]);
    }
}

// Gather, update and store CB cells of one hyperplane (cells with kon false
// are skipped).
template <typename S, typename T, int NC, int VPT, int CB, bool INTERIOR, typename VelT>
__device__ __forceinline__ void update_cells_k(const SweepArgs& a, S* __restrict__ f, const int* kk, const bool* kon,
                                               const VelT& V, const CellMeta<T, NC>* m) {
    const int Nv = (int)a.vg.Nv;
    T fc[CB][VPT];
    T lo[CB][NC][VPT], hi[CB][NC][VPT], lo2[CB][NC][VPT], hi2[CB][NC][VPT];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        const S* fk = f + (long long)kk[b] * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u) fc[b][u] = ldT<T, S>(fk + V.idx(u));
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
                lo[b][d][u] = dl ? ldT<T, S>(pl + V.idx(u)) : fc[b][u];
                hi[b][d][u] = dh ? ldT<T, S>(ph + V.idx(u)) : fc[b][u];
                lo2[b][d][u] = dl ? ldT<T, S>(pl2 + V.idx(u)) : lo[b][d][u];
                hi2[b][d][u] = dh ? ldT<T, S>(ph2 + V.idx(u)) : hi[b][d][u];
            }
        }
    }
    T fo[CB][VPT];
    compute_cells<T, NC, VPT, CB, INTERIOR>(a, kk, kon, V, m, fc, lo, hi, lo2, hi2, fo);
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!kon[b]) continue;
        S* fk = f + (long long)kk[b] * Nv;
#pragma unroll
        for (int u = 0; u < VPT; ++u)
            if (V.active(u)) stT<T, S>(fk + V.idx(u), fo[b][u]);
    }
}

template <typename S, typename T, int NC, int VPT, int CB, typename VelT>
__device__ __forceinline__ void update_cells(const SweepArgs& a, S* __restrict__ f, const int* kk, const bool* kon,
                                             const VelT& V) {
    CellMeta<T, NC> m[CB];
    // the branch-free update needs every one of the kernel's NC directions to
    // be a flux direction of the mesh (a batch runs lower-dimensional solves
    // in a 3-direction kernel: those take the general update)
    bool interior = a.nc == NC;
#pragma unroll
    for (int b = 0; b < CB; ++b)
        if (kon[b]) {
            load_meta<T, NC>(a, kk[b], m[b]);
            interior = interior && m[b].kinds < 0;
        }
    if (interior)
        update_cells_k<S, T, NC, VPT, CB, true>(a, f, kk, kon, V, m);
    else
        update_cells_k<S, T, NC, VPT, CB, false>(a, f, kk, kon, V, m);
}

// Velocities vbase + 32 u + lane (u < VPT) of the grid: flat index, axis
// indices and node values.
template <typename T, int VPT, bool FULL>
__device__ __forceinline__ void make_vel(const VGridDev& vg, long long vbase, int lane, Vel<T, VPT, FULL>& V) {
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
        const long long v = vbase + 32 * u + lane;
        V.on[u] = FULL || v < vg.Nv;
        V.v[u] = (int)(V.on[u] ? v : vg.Nv - 1);
        int ix, iy, iz;
        vsplit(V.v[u], vg.nx, vg.ny, ix, iy, iz);
        V.ix[u] = ix; V.q[u] = iy + vg.ny * iz;
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
