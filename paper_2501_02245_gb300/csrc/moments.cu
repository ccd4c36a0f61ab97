// Velocity-moment reductions (Eq. getmoment), high-order terms
// (Eq. full_constitutive) and the VDF correction of Eq. updatef.
//
// One block per DVM cell reduces over all discrete velocities in a fixed
// order, so results are bitwise reproducible.  Moments are taken about a
// reference velocity u_ref (the cell's current macroscopic velocity) to
// avoid cancellation:
//   m[0] = sum w f, m[1..3] = sum w c f, m[4..9] = sum w c_i c_j f
//   (xx, yy, zz, xy, xz, yz), m[10..12] = sum w c^2 c f,  c = xi - u_ref,
//   m[13+s] = sum_{xi.S_s > 0} w (xi.S_s) f for wall sides s (outgoing mass
//   flux through the wall face, for the diffuse-wall density).
//
// Row factoring: a thread owns whole x-rows (fixed iy, iz) of the cell's VDF,
// read as 16-byte loads where the rows are aligned (a warp's scalar loads
// would touch 32 rows each and cost one L1 wavefront per row per value).
// Per point it accumulates only sum f c_x^k, k = 0..3 (c_x^k from shared
// memory), and folds the row sums into the 13 moments with the row constants
// c_y, c_z once per row.  The correction pass (k_correct) gets the moments of
// the corrected VDF without a second reduction (see there).
//
// Arithmetic type T: FP64 for an FP64 VDF; for FP32/BF16/FP16 storage the
// per-row work (row sums over at most nx <= 64 nodes, the correction) is
// FP32 and every sum across rows and cells is FP64.  The FP32 row sum of
// n terms carries a relative rounding error below n * 2^-24 (< 4e-6 for
// n = 64) of the sum of |terms|, far under the storage rounding of BF16/FP16
// (2^-9 / 2^-12 per value) and comparable to FP32 storage rounding.
#include <type_traits>
#include "gsis_device.cuh"

namespace gsis {

// n consecutive T values from shared memory as 16-byte loads (p 16-byte
// aligned, n a multiple of 16 / sizeof(T)): a warp reading the same address
// gets it by broadcast in one instruction per 16 bytes.
template <typename T, int N>
__device__ __forceinline__ void lds16(const T* p, T* o) {
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 q = *reinterpret_cast<const float4*>(p + i);
            o[i] = q.x; o[i + 1] = q.y; o[i + 2] = q.z; o[i + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const double2 q = *reinterpret_cast<const double2*>(p + i);
            o[i] = q.x; o[i + 1] = q.y;
        }
    }
}

// ---------------------------------------------------------------- outgoing wall sums by rows
// On one x-row (fixed xi_y, xi_z) the normal speed through a wall side of area
// vector S is xi.S = xi_x S_x + r with r = xi_y S_y + xi_z S_z, monotone in ix
// (xi_x increases with ix), so the outgoing nodes (xi.S > 0) form one range
// [lo, hi) of ix, found by bisection.  Over the row, with A_j = sum_range xi_x^j f,
//   sum_range (xi.S) f = S_x A_1 + r A_0 = m_0,
//   sum_range (xi.S) xi_x^j f = S_x A_{j+1} + r A_j = m_j,
// so a row costs one to four sums per outgoing node and no FP64 per node.
__device__ __forceinline__ void out_range(const double* __restrict__ xi, int nx, double Sx, double r, int& lo,
                                          int& hi) {
    int a = 0, b = nx;
    if (Sx > 0.0) {          // first node with xi.S > 0
        while (a < b) {
            const int m = (a + b) >> 1;
            if (fma(xi[m], Sx, r) > 0.0) b = m; else a = m + 1;
        }
        lo = a; hi = nx;
    } else if (Sx < 0.0) {   // first node with xi.S <= 0
        while (a < b) {
            const int m = (a + b) >> 1;
            if (fma(xi[m], Sx, r) > 0.0) a = m + 1; else b = m;
        }
        lo = 0; hi = a;
    } else {
        lo = 0; hi = r > 0.0 ? nx : 0;
    }
}

// The conserved-quantity weights psi (mass, momentum x/y/z, energy) on row
// (xi_y = x1, xi_z = x2, plane iz) as a + b xi_x + c xi_x^2: (1, xi_x, xi_y,
// xi_z, |xi|^2 / 2) on the 3D grid and the G plane of the reduced grid (whose
// xi_z entries are 0), (0, 0, 0, 0, 1/2) on the H plane.
__device__ __forceinline__ void psi_row(const VGridDev& vg, double x1, double x2, int iz, double* a, double* b,
                                        double* c) {
#pragma unroll
    for (int q = 0; q < 5; ++q) a[q] = b[q] = c[q] = 0.0;
    if (vg.reduced && iz != 0) {
        a[4] = 0.5;
        return;
    }
    a[0] = 1.0;
    b[1] = 1.0;
    a[2] = x1;
    a[3] = x2;
    a[4] = 0.5 * (x1 * x1 + x2 * x2);
    c[4] = 0.5;
}

template <typename S, typename T>
__global__ void __launch_bounds__(256, 3) k_moments(int Nd, const int* __restrict__ dvm_cell,
                                                 const double* __restrict__ Wref, const int* __restrict__ side_bc,
                                                 const double* __restrict__ Sout, const S* __restrict__ f, VGridDev vg,
                                                 double* __restrict__ mom) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    extern __shared__ double sh_raw[];
    T* sh = reinterpret_cast<T*>(sh_raw);
    __shared__ double red[32 * MOMN];
    const int nx = vg.nx, ny = vg.ny, nz = vg.nz;
    const int c = dvm_cell[k];
    const double ux = Wref[c * 5 + 1], uy = Wref[c * 5 + 2], uz = Wref[c * 5 + 3];
    T* scx = sh;                 // c_x, c_x^2, c_x^3, xi_x
    T* scx2 = sh + nx;
    T* scx3 = sh + 2 * nx;
    T* sxi = sh + 3 * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double cx = vg.xi[i] - ux;
        scx[i] = (T)cx;
        scx2[i] = (T)(cx * cx);
        scx3[i] = (T)(cx * cx * cx);
        sxi[i] = (T)vg.xi[i];
    }
    __syncthreads();
    int wall_mask = 0;
    for (int s = 0; s < 6; ++s)
        if (side_bc[c * 6 + s] == GSIS_BC_WALL) wall_mask |= 1 << s;
    // this thread's sums live in its row of the reduction buffer (shared memory),
    // not in registers: they are touched once per plane
    double* part = sh_raw + (4 * nx * (int)sizeof(T) + 7) / 8;
    double* acc = part + threadIdx.x * MOMN;
#pragma unroll
    for (int q = 0; q < MOMN; ++q) acc[q] = 0.0;
    const S* fk = f + (long long)k * vg.Nv;
    const int rows = ny * nz;
    // Rows start on 16-byte boundaries when nx is a multiple of the values per
    // 16 bytes (the VDF allocation is 256-byte aligned and a cell holds whole rows).
    constexpr int V = Vec16<S>::N;
    const bool vec = nx % V == 0;
    // Each thread takes a contiguous run of rows, so that its rows share the
    // plane iz: per row it folds the row sums d_a with the powers of c_y only
    // (Y sums), and once per plane with the plane's c_z weights z_k (c_z^k on
    // the 3D grid, the G/H plane weights on the reduced grid):
    //   m = sum_planes sum_a,b Y_{a,b} z_k
    double Y[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // d0 (1, cy, cy^2, cy^3), d1 (1, cy, cy^2), d2 (1, cy), d3
    const int per = (rows + blockDim.x - 1) / blockDim.x;
    const int r0 = threadIdx.x * per, r1 = min(rows, r0 + per);
    for (int rp = r0; rp < r1;) {   // the thread's rows plane by plane
      const int iz = rp / ny, rend = min(r1, (iz + 1) * ny);
#pragma unroll
      for (int q = 0; q < 10; ++q) Y[q] = 0.0;
      for (int r = rp; r < rend; ++r) {
        const int iy = r - iz * ny;
        const double cy = vg.xi[nx + iy] - uy;
        const S* row = fk + (long long)r * nx;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        if (vec) {   // the row as 16-byte loads (same order of the sums)
            for (int ix0 = 0; ix0 < nx; ix0 += V) {
                T fv[V], x1[V], x2[V], x3[V];
                ld16<T, S>(row + ix0, fv);
                lds16<T, V>(scx + ix0, x1);
                lds16<T, V>(scx2 + ix0, x2);
                lds16<T, V>(scx3 + ix0, x3);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    s0 += fv[j];
                    s1 += fv[j] * x1[j];
                    s2 += fv[j] * x2[j];
                    s3 += fv[j] * x3[j];
                }
            }
        } else {
            for (int ix = 0; ix < nx; ++ix) {
                const T fv = ldT<T, S>(row + ix);
                s0 += fv;
                s1 += fv * scx[ix];
                s2 += fv * scx2[ix];
                s3 += fv * scx3[ix];
            }
        }
        const double d0 = s0, d1 = s1, d2 = s2, d3 = s3;
        const double cy2 = cy * cy, cy3 = cy2 * cy;
        Y[0] += d0;
        Y[1] = fma(d0, cy, Y[1]);
        Y[2] = fma(d0, cy2, Y[2]);
        Y[3] = fma(d0, cy3, Y[3]);
        Y[4] += d1;
        Y[5] = fma(d1, cy, Y[5]);
        Y[6] = fma(d1, cy2, Y[6]);
        Y[7] += d2;
        Y[8] = fma(d2, cy, Y[8]);
        Y[9] += d3;
      }
      {   // fold the plane's Y sums with its c_z weights
        double z0, z1, z2, z3;
        const double cz = vg.xi[nx + ny + iz] - uz;
        if (vg.reduced) {
            z0 = zpow(vg, iz, cz, 0); z1 = zpow(vg, iz, cz, 1);
            z2 = zpow(vg, iz, cz, 2); z3 = zpow(vg, iz, cz, 3);
        } else {
            z0 = 1.0; z1 = cz; z2 = cz * cz; z3 = z2 * cz;
        }
        acc[0] += Y[0] * z0;
        acc[1] += Y[4] * z0;
        acc[2] += Y[1] * z0;
        acc[3] += Y[0] * z1;
        acc[4] += Y[7] * z0;
        acc[5] += Y[2] * z0;
        acc[6] += Y[0] * z2;
        acc[7] += Y[5] * z0;
        acc[8] += Y[4] * z1;
        acc[9] += Y[1] * z1;
        acc[10] += (Y[9] + Y[6]) * z0 + Y[4] * z2;   // c_x c^2
        acc[11] += (Y[8] + Y[3]) * z0 + Y[1] * z2;   // c_y c^2
        acc[12] += (Y[7] + Y[2]) * z1 + Y[0] * z3;   // c_z c^2
      }
      rp = rend;
    }
    if (wall_mask) {   // outgoing mass flux through each wall side, row by row (mass rows only)
        double wsum[6] = {0, 0, 0, 0, 0, 0};
        const int mrows = vg.reduced ? ny : rows;
        for (int r = threadIdx.x; r < mrows; r += blockDim.x) {
            const double xy = vg.xi[nx + r % ny], xz = vg.xi[nx + ny + r / ny];
            const S* row = fk + (long long)r * nx;
            for (int s = 0; s < 6; ++s) {
                if (!((wall_mask >> s) & 1)) continue;
                const double* Sw = Sout + ((long long)c * 6 + s) * 3;
                const double rr = xy * Sw[1] + xz * Sw[2];
                int lo, hi;
                out_range(vg.xi, nx, Sw[0], rr, lo, hi);
                T a0 = T(0), a1 = T(0);
                for (int ix = lo; ix < hi; ++ix) {
                    const T fv = ldT<T, S>(row + ix);
                    a0 += fv;
                    a1 += fv * sxi[ix];
                }
                wsum[s] += Sw[0] * (double)a1 + rr * (double)a0;
            }
        }
#pragma unroll
        for (int s = 0; s < 6; ++s) acc[13 + s] = wsum[s];
    }
    // Block reduction over the rows of the buffer: lane q of each warp adds
    // moment q over the warp's threads
    // (31 FP64 additions per warp instead of MOMN five-step shuffle trees), and
    // thread q adds the warps' totals.
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane < MOMN) {
        const double* pw = part + w * 32 * MOMN + lane;
        double t = 0.0;
        for (int j = 0; j < 32; ++j) t += pw[j * MOMN];
        red[w * MOMN + lane] = t;
    }
    __syncthreads();
    if (threadIdx.x < MOMN) {
        double t = 0.0;
        for (int j = 0; j < nw; ++j) t += red[j * MOMN + threadIdx.x];
        const double wv = vg.w / vg.vscale;   // stored values carry the VDF storage scale
        mom[(long long)k * MOMN + threadIdx.x] = t * wv;
    }
}

// 1D sums of one axis table of a record about velocity u, on the lanes of
// one warp: s[a] = sum_j c^a E_j and s[4 + a] = sum_j c^a E_j B_j, a = 0..3,
// c = xi_j - u (valid in lane 0).
// On the reduced grid's z axis (zplanes) c^a is the plane weight of xi_z^a.
__device__ void axis_sums(const double* __restrict__ tab, int NT, const double* __restrict__ xi, int off, int n,
                          double u, int lane, double* s, const VGridDev* zplanes = nullptr) {
    double p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = lane; j < n; j += 32) {
        const double c = xi[off + j] - u, E = tab[off + j], EB = E * tab[NT + off + j];
        double ca = 1.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double wa = zplanes ? zpow(*zplanes, j, 0.0, a) : ca;
            p[a] += wa * E;
            p[4 + a] += wa * EB;
            ca *= c;
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) p[a] = warp_sum(p[a]);
    if (lane == 0)
        for (int a = 0; a < 8; ++a) s[a] = p[a];
}

// Moment c_x^a c_y^b c_z^c of a record whose value at a node is
// E_x E_y E_z (p0 + B_x + B_y + B_z), from its axis sums X, Y, Z (axis_sums).
__device__ __forceinline__ double rec_moment(const double* X, const double* Y, const double* Z, double p0, int a,
                                             int b, int c) {
    return (p0 * X[a] + X[4 + a]) * Y[b] * Z[c] + X[a] * (Y[4 + b] * Z[c] + Y[b] * Z[4 + c]);
}

// The 13 moments (layout of k_moments) of a record about the velocity its
// axis sums were taken about.
__device__ void rec_moments13(const double* X, const double* Y, const double* Z, double p0, double* m) {
    m[0] = rec_moment(X, Y, Z, p0, 0, 0, 0);
    m[1] = rec_moment(X, Y, Z, p0, 1, 0, 0);
    m[2] = rec_moment(X, Y, Z, p0, 0, 1, 0);
    m[3] = rec_moment(X, Y, Z, p0, 0, 0, 1);
    m[4] = rec_moment(X, Y, Z, p0, 2, 0, 0);
    m[5] = rec_moment(X, Y, Z, p0, 0, 2, 0);
    m[6] = rec_moment(X, Y, Z, p0, 0, 0, 2);
    m[7] = rec_moment(X, Y, Z, p0, 1, 1, 0);
    m[8] = rec_moment(X, Y, Z, p0, 1, 0, 1);
    m[9] = rec_moment(X, Y, Z, p0, 0, 1, 1);
    m[10] = rec_moment(X, Y, Z, p0, 3, 0, 0) + rec_moment(X, Y, Z, p0, 1, 2, 0) + rec_moment(X, Y, Z, p0, 1, 0, 2);
    m[11] = rec_moment(X, Y, Z, p0, 2, 1, 0) + rec_moment(X, Y, Z, p0, 0, 3, 0) + rec_moment(X, Y, Z, p0, 0, 1, 2);
    m[12] = rec_moment(X, Y, Z, p0, 2, 0, 1) + rec_moment(X, Y, Z, p0, 0, 2, 1) + rec_moment(X, Y, Z, p0, 0, 0, 3);
}

// The 13 moments (layout of k_moments) of a distribution taken about u,
// re-expressed about u + d: with c' = c - d,
//   m1' = m1 - d m0,  M' = M - d m1^T - m1 d^T + d d^T m0,
//   Q'_i = Q_i - 2 (M d)_i + |d|^2 m1_i - d_i tr M + 2 d_i (d.m1) - |d|^2 d_i m0.
__device__ void shift_moments13(const double* m, const double d[3], double* o) {
    const double m0 = m[0], m1[3] = {m[1], m[2], m[3]};
    const double M[3][3] = {{m[4], m[7], m[8]}, {m[7], m[5], m[9]}, {m[8], m[9], m[6]}};
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double dm1 = d[0] * m1[0] + d[1] * m1[1] + d[2] * m1[2];
    const double trM = M[0][0] + M[1][1] + M[2][2];
    double Mp[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mp[i][j] = M[i][j] - d[i] * m1[j] - m1[i] * d[j] + d[i] * d[j] * m0;
    o[0] = m0;
    for (int i = 0; i < 3; ++i) o[1 + i] = m1[i] - d[i] * m0;
    o[4] = Mp[0][0]; o[5] = Mp[1][1]; o[6] = Mp[2][2];
    o[7] = Mp[0][1]; o[8] = Mp[0][2]; o[9] = Mp[1][2];
    for (int i = 0; i < 3; ++i) {
        const double Md = M[i][0] * d[0] + M[i][1] * d[1] + M[i][2] * d[2];
        o[10 + i] = m[10 + i] - 2.0 * Md + dd * m1[i] - d[i] * trM + 2.0 * d[i] * dm1 - dd * d[i] * m0;
    }
}

// Eq. updatef in the DVM cells, f^{n+1} = f^{n+1/2} + M~(W^{n+1}) - M~(W^{n+1/2}),
// one block per DVM cell, and the outgoing half-range wall sums of f^{n+1}.
//
// The update is one coalesced pass over the cell's row.  Both records are
// conservation-corrected Maxwellians, E_x E_y E_z (p0 + B_x + B_y + B_z), so
// with per-x values (E, E B) and per-(y, z) values e = E_y E_z,
// p = p0 + B_y + B_z held in shared memory each point costs
//   a_N = E_x p_N + (E B)_x,  a_H likewise,  f += e_N a_N - e_H a_H
// (five operations).  Where the x-rows hold whole 16-byte chunks a thread
// loads and stores 16 bytes (2 to 8 values) at a time, two chunks in flight,
// else four scalar points; every thread loads before it stores (the loads and
// stores go through the same pointer, so the compiler would not move a load
// above an earlier store).  Both forms compute the same values in the same
// order (bitwise equal results).  A wall
// cell adds the correction's outgoing wall sums to those of f^{n+1/2}.
constexpr int CORR_UNROLL = 4;
constexpr int CORR_VEC_UNROLL = 2;

// Storage of the corrected value f + delta.  Near convergence delta is far
// below half a unit in the last place of a BF16 or FP16 value, so rounding
// to nearest would drop it every time (a systematic bias: the correction of
// Eq. updatef would stop acting).  Reduced-precision storage therefore
// rounds stochastically here: up with probability equal to the fraction of
// the unit in the last place that the value carries, so the stored value is
// unbiased and the increments survive on average over the velocities.  The
// random bits come from a hash of the cell, the velocity and the new value's
// own bits (deterministic, different from iteration to iteration because
// the values change; no seed, so the same launch can be replayed in a graph).
__device__ __forceinline__ unsigned mix32(unsigned x) {   // integer hash (avalanche), bits well mixed
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
template <typename T, typename S>
__device__ __forceinline__ S rounded(T v, unsigned key) {
    S o;
    stT<T, S>(&o, v);
    return o;
}
template <>
__device__ __forceinline__ __nv_bfloat16 rounded<float, __nv_bfloat16>(float v, unsigned key) {
    unsigned b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return __float2bfloat16_rn(v);   // inf / nan: nearest
    const unsigned r = mix32(key ^ b) & 0xffffu;   // uniform below the 16 dropped bits of the magnitude
    b += r;
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
}
template <>
__device__ __forceinline__ __half rounded<float, __half>(float v, unsigned key) {
    // Both roundings are formed and one is selected (Maxwellian tails put
    // normal and subnormal results in most warps, where a branch runs both
    // anyway); one hash serves both.
    const unsigned b = __float_as_uint(v);
    const unsigned mag = b & 0x7fffffffu;
    const unsigned h = mix32(key ^ b);
    // |v| in FP16's normal range (2^-14 up to the last binade below 65504): FP16
    // keeps the top 10 of FP32's 23 fraction bits, so adding 13 uniform random
    // bits below them and truncating toward zero rounds up with probability
    // equal to the dropped fraction (as for BF16)
    const __half hn = __float2half_rz(__uint_as_float(b + (h & 0x1fffu)));
    // below 2^-14: FP16's subnormals, m 2^-24 for m = 0..1023, so |v| 2^24 (exact)
    // splits into the lower m and the fraction that rounds up (m + 1 = 1024 is
    // the smallest normal, whose bits follow on); clamped so that the
    // conversion stays in range where this result is not the one selected
    const float r = fminf(__uint_as_float(mag) * 16777216.0f, 2048.0f);
    const unsigned m = (unsigned)r;
    const float frac = r - (float)m;
    const float u = (float)(h >> 8) * (1.0f / 16777216.0f);
    const __half hs = __ushort_as_half((unsigned short)(((b >> 16) & 0x8000u) | (m + (u < frac ? 1u : 0u))));
    // beyond the largest finite FP16, inf, nan: nearest
    const __half ho = __float2half_rn(v);
    return mag < 0x38800000u ? hs : (mag < 0x477fe000u ? hn : ho);
}
__device__ __forceinline__ unsigned corr_key(int k, int v) {
    return (unsigned)k * 0x9e3779b9u ^ (unsigned)v * 0x85ebca6bu;
}

template <typename S, typename T>
__global__ void __launch_bounds__(256) k_correct(int Nd, const int* __restrict__ dvm_cell,
                                                 const int* __restrict__ side_bc, const double* __restrict__ Sout,
                                                 S* __restrict__ f, Records recNew, Records recHalf, VGridDev vg,
                                                 const double* __restrict__ momh, double* __restrict__ mom) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    extern __shared__ double sh_raw[];
    const int nx = vg.nx, ny = vg.ny, NT = vg.NT, nyz = ny * vg.nz;
    T* xa = reinterpret_cast<T*>(sh_raw);   // [4][nx]: E_N, (E B)_N, E_H, (E B)_H
    T* rv = xa + 4 * nx;                     // [4][nyz]: e_N, p_N, e_H, p_H
    __shared__ double red[32 * 6];
    const int c = dvm_cell[k];
    const T* TN = RecT<T>::tab(recNew, k, NT);
    const T* TH = RecT<T>::tab(recHalf, k, NT);
    const T p0N = RecT<T>::scal(recNew, k)[RS_P0], p0H = RecT<T>::scal(recHalf, k)[RS_P0];
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        xa[i] = TN[i];
        xa[nx + i] = TN[i] * TN[NT + i];
        xa[2 * nx + i] = TH[i];
        xa[3 * nx + i] = TH[i] * TH[NT + i];
    }
    for (int q = threadIdx.x; q < nyz; q += blockDim.x) {
        const int jy = nx + q % ny, jz = nx + ny + q / ny;
        rv[q] = TN[jy] * TN[jz];
        rv[nyz + q] = p0N + (TN[NT + jy] + TN[NT + jz]);
        rv[2 * nyz + q] = TH[jy] * TH[jz];
        rv[3 * nyz + q] = p0H + (TH[NT + jy] + TH[NT + jz]);
    }
    int wall_mask = 0;
    for (int s = 0; s < 6; ++s)
        if (side_bc[c * 6 + s] == GSIS_BC_WALL) wall_mask |= 1 << s;
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    S* fk = f + (long long)k * vg.Nv;
    const int Nv = (int)vg.Nv, step = blockDim.x;
    // the increment at velocity (ix, q) and the outgoing wall sums of it
    auto delta = [&](int ix, int q) -> T {
        const T aN = fma(xa[ix], rv[nyz + q], xa[nx + ix]);
        const T aH = fma(xa[2 * nx + ix], rv[3 * nyz + q], xa[3 * nx + ix]);
        const T dlt = fma(rv[q], aN, -(rv[2 * nyz + q] * aH));
        if (wall_mask && (!vg.reduced || q < ny)) {   // mass flux: the G plane on the reduced grid
            const int iz = q / ny, iy = q - iz * ny;
            const double x0 = vg.xi[ix], x1 = vg.xi[nx + iy], x2 = vg.xi[nx + ny + iz];
            for (int s = 0; s < 6; ++s) {
                if (!((wall_mask >> s) & 1)) continue;
                const double* Sw = Sout + ((long long)c * 6 + s) * 3;
                const double xn = x0 * Sw[0] + x1 * Sw[1] + x2 * Sw[2];
                if (xn > 0.0) acc[s] += xn * (double)dlt;
            }
        }
        return dlt;
    };
    constexpr int V = Vec16<S>::N;
    if (nx % V == 0) {
        // 16-byte chunks of V consecutive velocities (one x-row holds whole chunks;
        // rows start on 16-byte boundaries), two chunks in flight per thread
        const int nch = Nv / V;
        for (int ch0 = threadIdx.x; ch0 < nch; ch0 += CORR_VEC_UNROLL * step) {
            T fv[CORR_VEC_UNROLL][V];
#pragma unroll
            for (int u = 0; u < CORR_VEC_UNROLL; ++u) {
                const int ch = ch0 + u * step;
                if (ch < nch) ld16<T, S>(fk + (long long)ch * V, fv[u]);
            }
#pragma unroll
            for (int u = 0; u < CORR_VEC_UNROLL; ++u) {
                const int ch = ch0 + u * step;
                if (ch >= nch) continue;
                const int v0 = ch * V, q = v0 / nx, ix0 = v0 - q * nx;
                alignas(16) S out[V];
#pragma unroll
                for (int j = 0; j < V; ++j)
                    out[j] = rounded<T, S>(fv[u][j] + delta(ix0 + j, q), corr_key(k, v0 + j));
                *reinterpret_cast<uint4*>(fk + (long long)v0) = *reinterpret_cast<const uint4*>(out);
            }
        }
    } else {
        const int sx = step % nx, sq = step / nx;
        int ix = threadIdx.x % nx, q = threadIdx.x / nx;
        for (int v0 = threadIdx.x; v0 < Nv; v0 += CORR_UNROLL * step) {
            T fv[CORR_UNROLL];
#pragma unroll
            for (int j = 0; j < CORR_UNROLL; ++j) {
                const int v = v0 + j * step;
                fv[j] = v < Nv ? ldT<T, S>(fk + v) : T(0);
            }
#pragma unroll
            for (int j = 0; j < CORR_UNROLL; ++j) {
                const int v = v0 + j * step;
                if (v < Nv) fk[v] = rounded<T, S>(fv[j] + delta(ix, q), corr_key(k, v));
                ix += sx;
                q += sq;
                if (ix >= nx) { ix -= nx; ++q; }
            }
        }
    }
    if (wall_mask) block_sum<6>(acc, red);
    if (threadIdx.x == 0) {
        const double* mh = momh + (long long)k * MOMN;
        double* m = mom + (long long)k * MOMN;
        // (the increment is in stored units: its record copies carry the VDF storage scale)
        const double wv = std::is_same<T, double>::value ? vg.w : vg.w / vg.vscale;
        for (int s = 0; s < 6; ++s) m[13 + s] = mh[13 + s] + (((wall_mask >> s) & 1) ? wv * acc[s] : 0.0);
    }
}

// The 13 velocity moments of f^{n+1} about u^{n+1} that the next
// cell-equilibrium step reads (its heat flux), one block of six warps per
// DVM cell, with no reduction over the velocities: the moments of f^{n+1/2}
// (taken about u^n = Wmom by the moments pass, momh) moved to u^{n+1}, plus
// those of the two corrected Maxwellians of Eq. updatef, which factor into 1D
// sums over each axis (warp 3 r + d: record r, axis d).
__global__ void __launch_bounds__(192) k_corr_moments(int Nd, const int* __restrict__ dvm_cell,
                                                      const double* __restrict__ Wnew,
                                                      const double* __restrict__ Wmom, Records recNew,
                                                      Records recHalf, VGridDev vg, const double* __restrict__ momh,
                                                      double* __restrict__ mom) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    __shared__ double axs[2][3][8];
    const int c = dvm_cell[k];
    const int nx = vg.nx, ny = vg.ny, nz = vg.nz, NT = vg.NT;
    const int w = threadIdx.x >> 5;
    if (w < 6) {
        const int r = w / 3, d = w % 3;
        const double* tab = (r == 0 ? recNew.tab : recHalf.tab) + (long long)k * NTAB * NT;
        const int off = d == 0 ? 0 : (d == 1 ? nx : nx + ny), n = d == 0 ? nx : (d == 1 ? ny : nz);
        axis_sums(tab, NT, vg.xi, off, n, Wnew[c * 5 + 1 + d], threadIdx.x & 31, axs[r][d],
                  (vg.reduced && d == 2) ? &vg : nullptr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double* mh = momh + (long long)k * MOMN;
        double* m = mom + (long long)k * MOMN;
        const double d[3] = {Wnew[c * 5 + 1] - Wmom[c * 5 + 1], Wnew[c * 5 + 2] - Wmom[c * 5 + 2],
                             Wnew[c * 5 + 3] - Wmom[c * 5 + 3]};
        double sh[13], mN[13], mH[13];
        shift_moments13(mh, d, sh);
        rec_moments13(axs[0][0], axs[0][1], axs[0][2], recNew.scal[(long long)k * RS + RS_P0], mN);
        rec_moments13(axs[1][0], axs[1][1], axs[1][2], recHalf.scal[(long long)k * RS + RS_P0], mH);
        for (int i = 0; i < 13; ++i) m[i] = sh[i] + vg.w * (mN[i] - mH[i]);
    }
}

template <typename S, typename T>
static void correct_t(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    const long long nyz = (long long)c->vg.ny * c->vg.nz;
    const size_t smem = (size_t)4 * (c->vg.nx + nyz) * sizeof(T);
    static size_t configured = 0;   // per instantiation: the largest dynamic size set so far
    if (smem > configured) {
        if (cudaFuncSetAttribute(k_correct<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            set_err(c, GSIS_ERR_UNSUPPORTED, "velocity grid too large for the correction pass's tables");
            c->broken = true;
            return;
        }
        configured = smem;
    }
    k_correct<S, T><<<Nd, 256, smem, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout, (S*)c->f, c->recNew,
                                                   c->recHalf, c->vg, c->momh, c->mom);
    k_corr_moments<<<Nd, 192, 0, c->stream>>>(Nd, c->dvm_cell, c->W, c->Wmom, c->recNew, c->recHalf, c->vg, c->momh,
                                              c->mom);
    c->launches += 2;
}

// Eq. updatef on the DVM cells and the moments of f^{n+1} about u^{n+1}
// (records recNew / recHalf; momh holds the moments of f^{n+1/2} about Wmom).
void launch_correct(gsis_ctx* c) {
    if (c->Nd == 0) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: correct_t<double, double>(c); break;
        case GSIS_F32: correct_t<float, float>(c); break;
        case GSIS_BF16: correct_t<__nv_bfloat16, float>(c); break;
        default: correct_t<__half, float>(c); break;
    }
}

// Diffuse-wall densities from the current VDF of each DVM wall cell:
// rho_w[k][s] = sum_{xi.S_s > 0} w (xi.S_s) f / wall_den[c][s].  Run between
// the forward and the backward pass, so that each pass emits from the wall
// with the latest outgoing half of f (the forward pass takes the values of
// the cell-equilibrium step, computed from f^n).  One block per DVM cell;
// cells without a wall side return at once.
template <typename S, typename T>
__global__ void __launch_bounds__(256) k_wall_rho(int Nd, const int* __restrict__ dvm_cell,
                                                  const int* __restrict__ side_bc, const double* __restrict__ Sout,
                                                  const S* __restrict__ f, VGridDev vg,
                                                  const double* __restrict__ wall_den, double* __restrict__ rho_w,
                                                  float* __restrict__ rho_wf) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    const int c = dvm_cell[k];
    int wall_mask = 0;
    for (int s = 0; s < 6; ++s)
        if (side_bc[c * 6 + s] == GSIS_BC_WALL) wall_mask |= 1 << s;
    if (!wall_mask) return;
    __shared__ double red[32 * 6];
    extern __shared__ double sh_raw[];
    T* sxi = reinterpret_cast<T*>(sh_raw);   // xi_x
    const int nx = vg.nx, ny = vg.ny;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) sxi[i] = (T)vg.xi[i];
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const S* fk = f + (long long)k * vg.Nv;
    const int rows = vg.reduced ? ny : ny * vg.nz;   // mass: the G plane if reduced
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double x1 = vg.xi[nx + r % ny], x2 = vg.xi[nx + ny + r / ny];
        const S* row = fk + (long long)r * nx;
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            if (!((wall_mask >> s) & 1)) continue;
            const double* Sw = Sout + ((long long)c * 6 + s) * 3;
            const double rr = x1 * Sw[1] + x2 * Sw[2];
            int lo, hi;
            out_range(vg.xi, nx, Sw[0], rr, lo, hi);
            T a0 = T(0), a1 = T(0);
            for (int ix = lo; ix < hi; ++ix) {
                const T fv = ldT<T, S>(row + ix);
                a0 += fv;
                a1 += fv * sxi[ix];
            }
            acc[s] += Sw[0] * (double)a1 + rr * (double)a0;
        }
    }
    block_sum<6>(acc, red);
    if (threadIdx.x == 0) {
        for (int s = 0; s < 6; ++s) {
            if ((wall_mask >> s) & 1) {
                const double v = acc[s] * (vg.w / vg.vscale) / wall_den[c * 6 + s];
                rho_w[(long long)k * 6 + s] = v;
                if (rho_wf) rho_wf[(long long)k * 6 + s] = (float)v;
            }
        }
    }
}

template <typename S, typename T>
static void wall_rho_t(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    k_wall_rho<S, T><<<Nd, 256, c->vg.nx * sizeof(T), c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                                   (const S*)c->f, c->vg, c->wall_den, c->rho_w,
                                                                   c->rho_wf);
    c->launches++;
}

void launch_wall_rho(gsis_ctx* c) {
    if (c->Nd == 0 || !c->has_wall) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: wall_rho_t<double, double>(c); break;
        case GSIS_F32: wall_rho_t<float, float>(c); break;
        case GSIS_BF16: wall_rho_t<__nv_bfloat16, float>(c); break;
        default: wall_rho_t<__half, float>(c); break;
    }
}

template <typename S, typename T>
static void moments_t(gsis_ctx* c, const double* Wref, double* out) {
    const int Nd = (int)c->Nd;
    // threads own whole x-rows: a block size that divides the rows evenly keeps
    // every warp busy until the final reduction (256 unless 192 or 128 fits better)
    const int rows = c->vg.ny * c->vg.nz;
    int tb = 256;
    for (int b : {256, 192, 128})
        if ((rows + b - 1) / b * b - rows < (rows + tb - 1) / tb * tb - rows) tb = b;
    // c_x tables, then one row of MOMN sums per thread for the block reduction
    const size_t smem = ((size_t)4 * c->vg.nx * sizeof(T) + 7) / 8 * 8 + (size_t)tb * MOMN * sizeof(double);
    k_moments<S, T><<<Nd, tb, smem, c->stream>>>(Nd, c->dvm_cell, Wref, c->m.side_bc, c->m.Sout, (const S*)c->f,
                                                  c->vg, out);
    c->launches++;
}

// Moments of f about Wref into `out` ([Nd][MOMN]).
void launch_moments(gsis_ctx* c, const double* Wref, double* out) {
    if (c->Nd == 0) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: moments_t<double, double>(c, Wref, out); break;
        case GSIS_F32: moments_t<float, float>(c, Wref, out); break;
        case GSIS_BF16: moments_t<__nv_bfloat16, float>(c, Wref, out); break;
        default: moments_t<__half, float>(c, Wref, out); break;
    }
}

// W^{n+1/2} and the kinetic stress / heat flux of Eq. getmoment from the
// moments of f^{n+1/2} taken about u^n: with delta = u^{n+1/2} - u^n,
//   P_ij = M_ij - rho d_i d_j,  T = tr(P)/(3 rho),  sigma = P - tr(P)/3 I,
//   q_i = 1/2 (T_i - 2 sum_j d_j M_ij - d_i tr M + 2 rho |d|^2 d_i).
// NS cells keep W^n and zero kinetic terms.
__global__ void k_half_state(int N, const int* __restrict__ cell2dvm, const double* __restrict__ W,
                             const double* __restrict__ momh, double* __restrict__ Wh, double* __restrict__ kin) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int k = cell2dvm[c];
    if (k < 0) {
        for (int q = 0; q < 5; ++q) Wh[c * 5 + q] = W[c * 5 + q];
        for (int q = 0; q < HOTN; ++q) kin[(long long)c * HOTN + q] = 0.0;
        return;
    }
    const double* m = momh + (long long)k * MOMN;
    const double rho = m[0];
    const double d[3] = {m[1] / rho, m[2] / rho, m[3] / rho};
    const double M[3][3] = {{m[4], m[7], m[8]}, {m[7], m[5], m[9]}, {m[8], m[9], m[6]}};
    double P[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i][j] = M[i][j] - rho * d[i] * d[j];
    const double tr = P[0][0] + P[1][1] + P[2][2];
    const double T = tr / (3.0 * rho);
    const double trM = M[0][0] + M[1][1] + M[2][2];
    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double q[3];
    for (int i = 0; i < 3; ++i)
        q[i] = 0.5 * (m[10 + i] - 2.0 * (d[0] * M[i][0] + d[1] * M[i][1] + d[2] * M[i][2]) - d[i] * trM +
                      2.0 * rho * d2 * d[i]);
    Wh[c * 5 + 0] = rho;
    for (int i = 0; i < 3; ++i) Wh[c * 5 + 1 + i] = W[c * 5 + 1 + i] + d[i];
    Wh[c * 5 + 4] = T;
    double* o = kin + (long long)c * HOTN;
    o[0] = P[0][0] - tr / 3.0;
    o[1] = P[1][1] - tr / 3.0;
    o[2] = P[2][2] - tr / 3.0;
    o[3] = P[0][1];
    o[4] = P[0][2];
    o[5] = P[1][2];
    o[6] = q[0];
    o[7] = q[1];
    o[8] = q[2];
}

void launch_half_state(gsis_ctx* c) {
    const int N = c->m.N;
    k_half_state<<<(N + 127) / 128, 128, 0, c->stream>>>(N, c->cell2dvm, c->W, c->momh, c->Wh, c->kin);
    c->launches++;
}

// Kinetic flux of (mass, momentum, energy) through each diffuse-wall face of a
// DVM cell, carried by the face distribution of f^{n+1/2}: the cell's values
// for outgoing velocities and rho_w M_w (rho_w from zero net mass flux) for
// incoming ones: F = sum_{xi.S>0} w (xi.S) psi f + rho_w wall_in.
template <typename S, typename T>
__global__ void __launch_bounds__(256) k_wall_flux(int Nd, const int* __restrict__ dvm_cell,
                                                   const int* __restrict__ side_bc, const double* __restrict__ Sout,
                                                   const S* __restrict__ f, VGridDev vg,
                                                   const double* __restrict__ wall_den,
                                                   const double* __restrict__ wall_in, double* __restrict__ wall_kin) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    const int c = dvm_cell[k];
    int wall_mask = 0;
    for (int s = 0; s < 6; ++s)
        if (side_bc[c * 6 + s] == GSIS_BC_WALL) wall_mask |= 1 << s;
    if (!wall_mask) return;
    __shared__ double sm[32 * 5];
    extern __shared__ double sh_raw[];
    T* sx1 = reinterpret_cast<T*>(sh_raw);   // xi_x, xi_x^2, xi_x^3
    T* sx2 = sx1 + vg.nx;
    T* sx3 = sx2 + vg.nx;
    const int nx = vg.nx, ny = vg.ny, rows = ny * vg.nz;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double x = vg.xi[i];
        sx1[i] = (T)x;
        sx2[i] = (T)(x * x);
        sx3[i] = (T)(x * x * x);
    }
    __syncthreads();
    const S* fk = f + (long long)k * vg.Nv;
    for (int s = 0; s < 6; ++s) {
        if (!((wall_mask >> s) & 1)) continue;
        const double* Sw = Sout + ((long long)c * 6 + s) * 3;
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            const int iy = r % ny, iz = r / ny;
            const double x1 = vg.xi[nx + iy], x2 = vg.xi[nx + ny + iz];
            const double rr = x1 * Sw[1] + x2 * Sw[2];
            int lo, hi;
            out_range(vg.xi, nx, Sw[0], rr, lo, hi);
            const S* row = fk + (long long)r * nx;
            T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
            for (int ix = lo; ix < hi; ++ix) {
                const T fv = ldT<T, S>(row + ix);
                a0 += fv;
                a1 += fv * sx1[ix];
                a2 += fv * sx2[ix];
                a3 += fv * sx3[ix];
            }
            const double m0 = Sw[0] * (double)a1 + rr * (double)a0;
            const double m1 = Sw[0] * (double)a2 + rr * (double)a1;
            const double m2 = Sw[0] * (double)a3 + rr * (double)a2;
            double pa[5], pb[5], pc[5];
            psi_row(vg, x1, x2, iz, pa, pb, pc);
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q] += pa[q] * m0 + pb[q] * m1 + pc[q] * m2;
        }
        block_sum<5>(acc, sm);
        if (threadIdx.x == 0) {
            const long long o = ((long long)c * 6 + s) * 5;
            const double wv = vg.w / vg.vscale;   // stored values carry the VDF storage scale
            const double rw = acc[0] * wv / wall_den[c * 6 + s];
            for (int q = 0; q < 5; ++q) wall_kin[o + q] = acc[q] * wv + rw * wall_in[o + q];
        }
        __syncthreads();   // sm is reused by the next wall side
    }
}

template <typename S, typename T>
static void wall_flux_t(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    k_wall_flux<S, T><<<Nd, 256, 3 * c->vg.nx * sizeof(T), c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                                        (const S*)c->f, c->vg, c->wall_den,
                                                                        c->wall_in, c->wall_kin);
    c->launches++;
}

void launch_wall_flux(gsis_ctx* c) {
    if (c->Nd == 0 || !c->has_wall) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: wall_flux_t<double, double>(c); break;
        case GSIS_F32: wall_flux_t<float, float>(c); break;
        case GSIS_BF16: wall_flux_t<__nv_bfloat16, float>(c); break;
        default: wall_flux_t<__half, float>(c); break;
    }
}

// HoT = kinetic - NSF(W^{n+1/2}) in DVM cells, zero in NS cells (Eq. full_constitutive).
__global__ void k_hot(int N, const int* __restrict__ cell2dvm, const double* __restrict__ kin,
                      const double* __restrict__ nsf, double* __restrict__ hot) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const bool dvm = cell2dvm[c] >= 0;
    for (int q = 0; q < HOTN; ++q) {
        hot[(long long)c * HOTN + q] = dvm ? kin[(long long)c * HOTN + q] - nsf[(long long)c * HOTN + q] : 0.0;
    }
}

void launch_hot(gsis_ctx* c) {
    const int N = c->m.N;
    k_hot<<<(N + 127) / 128, 128, 0, c->stream>>>(N, c->cell2dvm, c->kin, c->nsf, c->hot);
    c->launches++;
}

// ---------------------------------------------------------------------------- two-VDF moments
// Eq. getmoment for the two-VDF model, one block per state of F[n][2][Nv]
// (f0 then f1 on a full 3D grid): rho, u from f0; then, about u, the
// pressure tensor P and heat flux q_t = 1/2 sum w c |c|^2 f0, and
// q_r = sum w c f1, d_r/2 rho T_r = sum w f1.  out[k][18] = rho, u (3), T_t,
// T_r, sigma (xx, yy, zz, xy, xz, yz), q_t (3), q_r (3); T_t = tr P/(3 rho),
// sigma = P - tr P/3 I, T_r = T_t when d_r = 0.  FP64 sums in a fixed order
// (block reduction through shared memory).
constexpr int TWO_VDF_THREADS = 256;

__device__ static void block_sum(double* v, int m, double* sh) {
    // sums v[0..m) over the block into sh[0..m) (m <= 16); every thread gets the result in v
    for (int i = 0; i < m; ++i) sh[i * TWO_VDF_THREADS + threadIdx.x] = v[i];
    __syncthreads();
    for (int stride = TWO_VDF_THREADS / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride)
            for (int i = 0; i < m; ++i)
                sh[i * TWO_VDF_THREADS + threadIdx.x] += sh[i * TWO_VDF_THREADS + threadIdx.x + stride];
        __syncthreads();
    }
    for (int i = 0; i < m; ++i) v[i] = sh[i * TWO_VDF_THREADS];
    __syncthreads();
}

__global__ void __launch_bounds__(TWO_VDF_THREADS) k_two_vdf_moments(int n, const double* __restrict__ F, int d_r,
                                                                     VGridDev vg, double* __restrict__ out) {
    __shared__ double sh[16 * TWO_VDF_THREADS];
    const int k = blockIdx.x;
    if (k >= n) return;
    const long long Nv = vg.Nv;
    const int nx = vg.nx, ny = vg.ny;
    const double* f0 = F + (long long)k * 2 * Nv;
    const double* f1 = f0 + Nv;
    double a[16];
    for (int i = 0; i < 4; ++i) a[i] = 0.0;
    for (long long v = threadIdx.x; v < Nv; v += TWO_VDF_THREADS) {
        const int ix = (int)(v % nx);
        const long long rr = v / nx;
        const int iy = (int)(rr % ny), iz = (int)(rr / ny);
        const double f = f0[v];
        a[0] += f;
        a[1] += vg.xi[ix] * f;
        a[2] += vg.xi[nx + iy] * f;
        a[3] += vg.xi[nx + ny + iz] * f;
    }
    block_sum(a, 4, sh);
    const double rho = vg.w * a[0];
    const double u[3] = {vg.w * a[1] / rho, vg.w * a[2] / rho, vg.w * a[3] / rho};
    for (int i = 0; i < 14; ++i) a[i] = 0.0;
    for (long long v = threadIdx.x; v < Nv; v += TWO_VDF_THREADS) {
        const int ix = (int)(v % nx);
        const long long rr = v / nx;
        const int iy = (int)(rr % ny), iz = (int)(rr / ny);
        const double c0 = vg.xi[ix] - u[0], c1 = vg.xi[nx + iy] - u[1], c2 = vg.xi[nx + ny + iz] - u[2];
        const double f = f0[v], g = f1[v];
        const double c2f = (c0 * c0 + c1 * c1 + c2 * c2) * f;
        a[0] += c0 * c0 * f; a[1] += c1 * c1 * f; a[2] += c2 * c2 * f;
        a[3] += c0 * c1 * f; a[4] += c0 * c2 * f; a[5] += c1 * c2 * f;
        a[6] += c0 * c2f; a[7] += c1 * c2f; a[8] += c2 * c2f;
        a[9] += g; a[10] += c0 * g; a[11] += c1 * g; a[12] += c2 * g;
    }
    block_sum(a, 13, sh);
    if (threadIdx.x != 0) return;
    const double w = vg.w;
    const double P[6] = {w * a[0], w * a[1], w * a[2], w * a[3], w * a[4], w * a[5]};
    const double tr = P[0] + P[1] + P[2];
    const double Tt = tr / (3.0 * rho);
    double* o = out + (long long)k * 18;
    o[0] = rho; o[1] = u[0]; o[2] = u[1]; o[3] = u[2];
    o[4] = Tt;
    o[5] = d_r > 0 ? 2.0 * w * a[9] / (d_r * rho) : Tt;
    o[6] = P[0] - tr / 3.0; o[7] = P[1] - tr / 3.0; o[8] = P[2] - tr / 3.0;
    o[9] = P[3]; o[10] = P[4]; o[11] = P[5];
    o[12] = 0.5 * w * a[6]; o[13] = 0.5 * w * a[7]; o[14] = 0.5 * w * a[8];
    o[15] = w * a[10]; o[16] = w * a[11]; o[17] = w * a[12];
}

void launch_two_vdf_moments(gsis_ctx* c, const double* F, int n, int d_r, double* out) {
    if (n <= 0) return;
    k_two_vdf_moments<<<n, TWO_VDF_THREADS, 0, c->stream>>>(n, F, d_r, c->vg, out);
    c->launches++;
}

}  // namespace gsis
