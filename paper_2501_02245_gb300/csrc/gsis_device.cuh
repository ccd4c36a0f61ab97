// Device helpers shared by the GSIS kernels.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "gsis_internal.h"

namespace gsis {

constexpr double GAMMA = 5.0 / 3.0;
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- storage conversion
template <typename S> struct Store;
template <> struct Store<double> {
    static __device__ __forceinline__ double ld(const double* p) { return *p; }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
    static __device__ __forceinline__ float ldf(const double* p) { return (float)*p; }
    static __device__ __forceinline__ void stf(double* p, float v) { *p = (double)v; }
};
template <> struct Store<float> {
    static __device__ __forceinline__ double ld(const float* p) { return (double)*p; }
    static __device__ __forceinline__ void st(float* p, double v) { *p = (float)v; }
    static __device__ __forceinline__ float ldf(const float* p) { return *p; }
    static __device__ __forceinline__ void stf(float* p, float v) { *p = v; }
};
// BF16 -> FP32 is exact: the 16 stored bits followed by 16 zero bits (an
// integer shift, where the conversion instruction is slower in the sweep)
__device__ __forceinline__ float bf16_to_f(const __nv_bfloat16* p) {
    return __uint_as_float((unsigned)__bfloat16_as_ushort(*p) << 16);
}
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ double ld(const __nv_bfloat16* p) { return (double)bf16_to_f(p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }
    static __device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return bf16_to_f(p); }
    static __device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ double ld(const __half* p) { return (double)__half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, double v) { *p = __float2half_rn((float)v); }
    static __device__ __forceinline__ float ldf(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void stf(__half* p, float v) { *p = __float2half_rn(v); }
};

// load / store in the arithmetic type T (double or float)
template <typename T, typename S> __device__ __forceinline__ T ldT(const S* p);
template <> __device__ __forceinline__ double ldT<double, double>(const double* p) { return *p; }
template <typename T, typename S> __device__ __forceinline__ void stT(S* p, T v);
template <> __device__ __forceinline__ void stT<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ float ldT<float, float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ldT<float, __nv_bfloat16>(const __nv_bfloat16* p) { return bf16_to_f(p); }
template <> __device__ __forceinline__ float ldT<float, __half>(const __half* p) { return __half2float(*p); }
template <> __device__ __forceinline__ void stT<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void stT<float, __nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ void stT<float, __half>(__half* p, float v) { *p = __float2half_rn(v); }

// One 16-byte load of VEC16<S> consecutive stored values (p 16-byte aligned),
// converted to the arithmetic type T.
template <typename S> struct Vec16 { static constexpr int N = 16 / (int)sizeof(S); };
template <typename T, typename S> __device__ __forceinline__ void ld16(const S* p, T* out);
template <> __device__ __forceinline__ void ld16<double, double>(const double* p, double* out) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    out[0] = v.x; out[1] = v.y;
}
template <> __device__ __forceinline__ void ld16<float, float>(const float* p, float* out) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
__device__ __forceinline__ void bf16x2_to_f(unsigned w, float* o) {   // element 0 in the low half
    o[0] = __uint_as_float(w << 16);
    o[1] = __uint_as_float(w & 0xffff0000u);
}
__device__ __forceinline__ void f16x2_to_f(unsigned w, float* o) {
    const float2 t = __half22float2(*reinterpret_cast<const __half2*>(&w));
    o[0] = t.x;
    o[1] = t.y;
}
template <> __device__ __forceinline__ void ld16<float, __nv_bfloat16>(const __nv_bfloat16* p, float* out) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    bf16x2_to_f(v.x, out); bf16x2_to_f(v.y, out + 2); bf16x2_to_f(v.z, out + 4); bf16x2_to_f(v.w, out + 6);
}
template <> __device__ __forceinline__ void ld16<float, __half>(const __half* p, float* out) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    f16x2_to_f(v.x, out); f16x2_to_f(v.y, out + 2); f16x2_to_f(v.z, out + 4); f16x2_to_f(v.w, out + 6);
}

// ---------------------------------------------------------------- small math
// minmod(a, b): 0 unless a and b share a sign, else the one nearer zero.
template <typename T>
__device__ __forceinline__ T minmod_t(T a, T b) {
    const T m = fabs(a) < fabs(b) ? a : b;
    return a * b > T(0) ? m : T(0);
}

// Half the minmod, 0.5 minmod(a, b).  FP64: decisions on the bit patterns and the halving as a decrement of the exponent field, all on the
// integer pipe (GB300 issues FP64 at 1/64 of the FP32 rate).  Magnitudes of
// IEEE doubles order like their bit patterns with the sign bit cleared, and
// +-0 never shares a sign, so the result equals 0.5 minmod_t(a, b) for every
// result of magnitude >= 2^-1021; a smaller one (300 orders of magnitude
// below any value of the scheme) gives 0.
template <typename T> __device__ __forceinline__ T hmm_t(T a, T b);
template <> __device__ __forceinline__ float hmm_t<float>(float a, float b) { return 0.5f * minmod_t<float>(a, b); }
template <> __device__ __forceinline__ double hmm_t<double>(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    const bool a_smaller = ma < mb;
    const long long m = a_smaller ? ia : ib, mm = a_smaller ? ma : mb;
    const bool ok = (ia ^ ib) >= 0 && mm >= (2LL << 52);   // same sign, |result| >= 2^-1021 (so nonzero)
    return ok ? __longlong_as_double(m - (1LL << 52)) : 0.0;
}

// mu0 T^omega as exp(omega ln T): within a few ulp of the power (relative
// error below 1e-15 for the temperatures of the workloads), at about half
// the FP64 operations of pow, which carries its logarithm in extended
// precision; evaluated once per face per pseudo-step of the synthetic solve.
__device__ __forceinline__ double viscosity(double T, double mu0, double omega) {
    return mu0 * exp(omega * log(T));
}

// ---------------------------------------------------------------- velocity index
__device__ __forceinline__ void vsplit(long long v, int nx, int ny, int& ix, int& iy, int& iz) {
    ix = (int)(v % nx);
    long long t = v / nx;
    iy = (int)(t % ny);
    iz = (int)(t / ny);
}

// Weights of (mass, x/y/z momentum, energy) carried by the value at velocity
// node (x0, x1, x2) of z node iz: (1, xi, |xi|^2/2) on a 3D grid; on the
// reduced grid the G plane carries mass, x/y momentum and (x0^2 + x1^2)/2 of
// energy, the H plane (int xi_z^2 f) the remaining 1/2 of energy.
__device__ __forceinline__ void psi_node(const VGridDev& vg, double x0, double x1, double x2, int iz, double* psi) {
    if (vg.reduced) {
        const double g = iz == 0 ? 1.0 : 0.0;
        psi[0] = g;
        psi[1] = g * x0;
        psi[2] = g * x1;
        psi[3] = 0.0;
        psi[4] = iz == 0 ? 0.5 * (x0 * x0 + x1 * x1) : 0.5;
        return;
    }
    psi[0] = 1.0;
    psi[1] = x0;
    psi[2] = x1;
    psi[3] = x2;
    psi[4] = 0.5 * (x0 * x0 + x1 * x1 + x2 * x2);
}

// ---------------------------------------------------------------- distribution records
// value at node (ix, iy, iz): E_x E_y E_z * (p0 + B_x+B_y+B_z + (R_x+R_y+R_z)(C2_x+C2_y+C2_z)
//                                              + 2 (P2xy cx cy + P2xz cx cz + P2yz cy cz))
__device__ __forceinline__ double eval_rec(const double* __restrict__ scal, const double* __restrict__ tab,
                                           int NT, int nx, int ny, int ix, int iy, int iz) {
    const int jy = nx + iy, jz = nx + ny + iz;
    double e = tab[ix] * tab[jy] * tab[jz];
    const double* B = tab + NT;
    const double* C2 = tab + 3 * NT;
    const double* Rr = tab + 4 * NT;
    double poly = scal[RS_P0] + (B[ix] + B[jy] + B[jz]) + (Rr[ix] + Rr[jy] + Rr[jz]) * (C2[ix] + C2[jy] + C2[jz]);
    if (scal[RS_OFFD] != 0.0) {
        const double* C = tab + 2 * NT;
        double cx = C[ix], cy = C[jy], cz = C[jz];
        poly += 2.0 * (scal[RS_P2XY] * cx * cy + scal[RS_P2XZ] * cx * cz + scal[RS_P2YZ] * cy * cz);
    }
    return e * poly;
}

__device__ __forceinline__ const double* rec_scal(const Records& r, long long i) { return r.scal + i * RS; }
__device__ __forceinline__ const double* rec_tab(const Records& r, long long i, int NT) {
    return r.tab + i * (long long)(NTAB * NT);
}

// Record access in the arithmetic type T (the FP32 copies for T = float).
template <typename T> struct RecT;
template <> struct RecT<double> {
    static __device__ __forceinline__ const double* scal(const Records& r, long long i) { return r.scal + i * RS; }
    static __device__ __forceinline__ const double* tab(const Records& r, long long i, int NT) {
        return r.tab + i * (long long)(NTAB * NT);
    }
};
template <> struct RecT<float> {
    static __device__ __forceinline__ const float* scal(const Records& r, long long i) { return r.scalf + i * RS; }
    static __device__ __forceinline__ const float* tab(const Records& r, long long i, int NT) {
        return r.tabf + i * (long long)(NTAB * NT);
    }
};

// Record tables are read-only while the kernels that evaluate them run, so
// they are read through the non-coherent path (__ldg): this also tells the
// compiler they cannot alias the VDF being updated.
template <typename T>
__device__ __forceinline__ T eval_recT(const T* __restrict__ scal, const T* __restrict__ tab, int NT, int nx, int ny,
                                       int ix, int iy, int iz) {
    const int jy = nx + iy, jz = nx + ny + iz;
    T e = __ldg(tab + ix) * __ldg(tab + jy) * __ldg(tab + jz);
    const T* B = tab + NT;
    const T* C2 = tab + 3 * NT;
    const T* Rr = tab + 4 * NT;
    T poly = __ldg(scal + RS_P0) + (__ldg(B + ix) + __ldg(B + jy) + __ldg(B + jz)) +
             (__ldg(Rr + ix) + __ldg(Rr + jy) + __ldg(Rr + jz)) * (__ldg(C2 + ix) + __ldg(C2 + jy) + __ldg(C2 + jz));
    if (__ldg(scal + RS_OFFD) != T(0)) {
        const T* C = tab + 2 * NT;
        T cx = __ldg(C + ix), cy = __ldg(C + jy), cz = __ldg(C + jz);
        poly += T(2) * (__ldg(scal + RS_P2XY) * cx * cy + __ldg(scal + RS_P2XZ) * cx * cz +
                        __ldg(scal + RS_P2YZ) * cy * cz);
    }
    return e * poly;
}

// ---------------------------------------------------------------- deterministic reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of K values per thread (blockDim.x a multiple of 32, <= 1024).
// Result valid in thread 0 (returned there; other threads get partial values).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* [32*K] */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) smem[wid * K + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += smem[w * K + k];
            v[k] = s;
        }
    }
    __syncthreads();
}

}  // namespace gsis
