// Distribution records: reference distributions of the kinetic model, their
// conservation correction, Grad-13 interface distributions and boundary
// Maxwellians, all in the separable form
//     D(xi) = A e_x(ix) e_y(iy) e_z(iz) * P(c),   c = xi - u,
//     e_d = exp(-c_d^2 / (2T)),  P = p0 + p.c + c.P2.c + (r.c) c^2,
// so that one exp per 1D node (not per 3D node) is evaluated.
//
//  * Shakhov reference g_0t of Sec. 2 (Eq. general_model with d_r = 0):
//      p0 = 1, p = -5T s q, r = s q, s = 1/(15 p T^2)
//  * Grad-13 distribution of Eq. G13_VDF:
//      p0 = 1, p = -q/(rho T^2), P2 = sigma/(2 rho T^2), r = q/(5 rho T^3)
//  * conservation correction (the Lagrange-multiplier form of Gamba and
//    Tharkabhushanam, J. Comput. Phys. 228 (2009), Maxwellian weighted):
//      D <- D + M (a0 + a.xi + a4 |xi|^2) with the 5x5 system
//      sum_v w psi phi^T M a = U - sum_v w psi D,  psi = (1, xi, |xi|^2/2),
//      phi = (1, xi, |xi|^2),
//    whose sums are assembled exactly from 1D sums C_d[k] = sum_i e_d c_d^k.
#include <algorithm>
#include <type_traits>
#include "gsis_device.cuh"

namespace gsis {

struct Term { double c; int a, b, d; };

__device__ static int psi_terms(int row, const double* u, Term* t, double scale) {
    // psi_row in powers of c (c = xi - u); scale = 1 for psi, 2 for phi_4 only
    switch (row) {
        case 0: t[0] = {1.0, 0, 0, 0}; return 1;
        case 1: t[0] = {1.0, 1, 0, 0}; t[1] = {u[0], 0, 0, 0}; return 2;
        case 2: t[0] = {1.0, 0, 1, 0}; t[1] = {u[1], 0, 0, 0}; return 2;
        case 3: t[0] = {1.0, 0, 0, 1}; t[1] = {u[2], 0, 0, 0}; return 2;
        default: {
            double h = 0.5 * scale;
            t[0] = {h, 2, 0, 0}; t[1] = {h, 0, 2, 0}; t[2] = {h, 0, 0, 2};
            t[3] = {scale * u[0], 1, 0, 0}; t[4] = {scale * u[1], 0, 1, 0}; t[5] = {scale * u[2], 0, 0, 1};
            t[6] = {h * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]), 0, 0, 0};
            return 7;
        }
    }
}

// Terms of the base polynomial with a nonzero coefficient (a Maxwellian has only
// p0; skipping the zero terms leaves its moment sums 19 times shorter, and a
// zero term contributes exactly zero to them).
__device__ static int base_terms(const RecSpec& s, Term* t) {
    const Term all[19] = {
        {s.p0, 0, 0, 0},
        {s.p[0], 1, 0, 0}, {s.p[1], 0, 1, 0}, {s.p[2], 0, 0, 1},
        {s.P2[0], 2, 0, 0}, {s.P2[1], 0, 2, 0}, {s.P2[2], 0, 0, 2},
        {2.0 * s.P2[3], 1, 1, 0}, {2.0 * s.P2[4], 1, 0, 1}, {2.0 * s.P2[5], 0, 1, 1},
        {s.r[0], 3, 0, 0}, {s.r[0], 1, 2, 0}, {s.r[0], 1, 0, 2},
        {s.r[1], 2, 1, 0}, {s.r[1], 0, 3, 0}, {s.r[1], 0, 1, 2},
        {s.r[2], 2, 0, 1}, {s.r[2], 0, 2, 1}, {s.r[2], 0, 0, 3}};
    int n = 0;
    for (int i = 0; i < 19; ++i)
        if (all[i].c != 0.0) t[n++] = all[i];
    return n;
}

__device__ static double poly_moment(const Term* t1, int n1, const Term* t2, int n2, const double (*Cs)[6]) {
    double s = 0.0;
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
            s += t1[i].c * t2[j].c * (Cs[0][t1[i].a + t2[j].a] * Cs[1][t1[i].b + t2[j].b] * Cs[2][t1[i].d + t2[j].d]);
    return s;
}

// Solve A x = b (5x5) by Gaussian elimination with partial pivoting.
__device__ static void solve5(double A[5][5], double b[5], double x[5]) {
    for (int col = 0; col < 5; ++col) {
        int piv = col;
        double best = fabs(A[col][col]);
        for (int r = col + 1; r < 5; ++r)
            if (fabs(A[r][col]) > best) { best = fabs(A[r][col]); piv = r; }
        if (piv != col) {
            for (int k = 0; k < 5; ++k) { double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < 5; ++r) {
            double m = A[r][col] / A[col][col];
            for (int k = col; k < 5; ++k) A[r][k] -= m * A[col][k];
            b[r] -= m * b[col];
        }
    }
    for (int r = 4; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 5; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
}

// Four records per warp, eight lanes (a "group") per record: the FP64
// operations of a warp instruction cost the same whatever the number of active
// lanes, so the per-record serial parts (the 5 x 5 solve, the reductions) run
// for four records at once.  Lanes of a group split the 1D nodes and the 30
// entries of the correction system; every shuffle is segmented to the group.
constexpr int REC_LANES = 8;
constexpr int REC_PER_WARP = 32 / REC_LANES;

__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = REC_LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, REC_LANES);
    return v;
}

__global__ void k_build_records(const RecSpec* __restrict__ specs, int nrec, Records out, VGridDev vg) {
    const int lane = threadIdx.x & 31, sl = lane & (REC_LANES - 1);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp * REC_PER_WARP >= nrec) return;   // the whole warp is past the last record
    const int r0 = warp * REC_PER_WARP + (lane / REC_LANES);
    const bool valid = r0 < nrec;              // groups past the end compute a copy and store nothing
    const int r = valid ? r0 : nrec - 1;
    const RecSpec s = specs[r];
    const int NT = vg.NT, nx = vg.nx, ny = vg.ny;
    double* tab = out.tab + (long long)r * NTAB * NT;
    double* scal = out.scal + (long long)r * RS;
    const double T = s.T;
    const double A = s.rho * pow(2.0 * PI * T, -1.5);
    double part[3][6];
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < 6; ++k) part[d][k] = 0.0;
    // reduced grid: the z "nodes" are the planes G (p = 0) and H (p = 1); integrating the separable form
    // over xi_z (u_z = r_z = 0 and no xz / yz stress in a flow without z dependence) leaves the same form
    // with the plane values E_z = int xi_z^{2p} e_z dxi_z = sqrt(2 pi T) (1, T), C_z = 0 and
    // C2_z = (2p + 1) T, the ratio of the Gaussian moments 3T^2 / T and T / 1
    const double sq2piT = sqrt(2.0 * PI * T);
    const double i2T = 0.5 / T;   // exp(-c^2 / (2T)) as exp(-c^2 * i2T): one division per record, not per node
#pragma unroll
    for (int d = 0; d < 3; ++d) {   // the axes' node ranges in turn (static axis index for the sums)
        const int lo = d == 0 ? 0 : (d == 1 ? nx : nx + ny), hi = d == 0 ? nx : (d == 1 ? nx + ny : NT);
        for (int idx = lo + sl; idx < hi; idx += REC_LANES) {
            if (vg.reduced && d == 2) {
                const int p = idx - nx - ny;
                if (valid) {
                    tab[idx] = p ? sq2piT * T : sq2piT;
                    tab[2 * NT + idx] = 0.0;
                    tab[3 * NT + idx] = p ? 3.0 * T : T;
                }
                continue;
            }
            const double c = vg.xi[idx] - s.u[d];
            const double e = exp(-(c * c) * i2T);
            if (valid) {
                tab[idx] = e;
                tab[2 * NT + idx] = c;
                tab[3 * NT + idx] = c * c;
            }
            double pw = e;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                part[d][k] += pw;
                pw *= c;
            }
        }
    }
    double Cs[3][6];
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < 6; ++k) Cs[d][k] = group_sum(part[d][k]);
    if (vg.reduced) {   // exact xi_z integrals int c_z^k e_z dxi_z of the Gaussian (k = 0..5)
        const double zk[6] = {1.0, 0.0, T, 0.0, 3.0 * T * T, 0.0};
        for (int k = 0; k < 6; ++k) Cs[2][k] = sq2piT * zk[k];
    }

    // the 5 right-hand sides (entries 0-4) and 25 matrix entries (5-29) of the
    // correction system, entry e on lane e % 8 of the group (slot e / 8), gathered
    // on the group's first lane
    double mine[4] = {0.0, 0.0, 0.0, 0.0};
    if (s.correct) {
        Term tp[7], tq[19];
        const double wa = vg.w * A;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = sl + REC_LANES * m;
            if (e < 5) {
                const int na = psi_terms(e, s.u, tp, 1.0);
                const int nb = base_terms(s, tq);
                mine[m] = s.U[e] - wa * poly_moment(tp, na, tq, nb, Cs);
            } else if (e < 30) {
                const int ra = (e - 5) / 5, rb = (e - 5) % 5;
                const int na = psi_terms(ra, s.u, tp, 1.0);
                const int nbb = psi_terms(rb, s.u, tq, rb == 4 ? 2.0 : 1.0);
                mine[m] = wa * poly_moment(tp, na, tq, nbb, Cs);
            }
        }
    }
    double Am[5][5], rhs[5];
#pragma unroll
    for (int e = 0; e < 30; ++e) {
        const double v = __shfl_sync(0xffffffffu, mine[e / REC_LANES], e % REC_LANES, REC_LANES);
        if (e < 5) rhs[e] = v;
        else Am[(e - 5) / 5][(e - 5) % 5] = v;
    }
    double coef[7];   // p0', p'(3), P2'(diag 3)
    if (sl == 0) {
        double pp[3] = {s.p[0], s.p[1], s.p[2]};
        double p2d[3] = {s.P2[0], s.P2[1], s.P2[2]};
        double p0 = s.p0;
        double alpha[5] = {0, 0, 0, 0, 0};
        if (s.correct) {
            solve5(Am, rhs, alpha);
            const double ua = alpha[1] * s.u[0] + alpha[2] * s.u[1] + alpha[3] * s.u[2];
            const double u2 = s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2];
            p0 = s.p0 + alpha[0] + ua + alpha[4] * u2;
            for (int d = 0; d < 3; ++d) {
                pp[d] = s.p[d] + alpha[1 + d] + 2.0 * alpha[4] * s.u[d];
                p2d[d] = s.P2[d] + alpha[4];
            }
        }
        coef[0] = p0;
        for (int d = 0; d < 3; ++d) { coef[1 + d] = pp[d]; coef[4 + d] = p2d[d]; }
        if (valid) {
            scal[RS_P0] = p0;
            scal[RS_P2XY] = s.P2[3];
            scal[RS_P2XZ] = s.P2[4];
            scal[RS_P2YZ] = s.P2[5];
            scal[RS_OFFD] = (s.P2[3] != 0.0 || s.P2[4] != 0.0 || s.P2[5] != 0.0) ? 1.0 : 0.0;
            scal[RS_UX] = s.u[0];
            scal[RS_UY] = s.u[1];
            scal[RS_UZ] = s.u[2];
            for (int k = 0; k < 5; ++k) scal[RS_ALPHA0 + k] = alpha[k];
            for (int q = RS_ALPHA0 + 5; q < RS; ++q) scal[q] = 0.0;
        }
    }
    for (int k = 0; k < 7; ++k) coef[k] = __shfl_sync(0xffffffffu, coef[k], 0, REC_LANES);
    __syncwarp();   // the table values of the first loop, written by other lanes of the group, are read below
    if (valid) {
        for (int idx = sl; idx < NT; idx += REC_LANES) {
            const int d = idx < nx ? 0 : (idx < nx + ny ? 1 : 2);
            const double c = tab[2 * NT + idx];
            tab[NT + idx] = coef[1 + d] * c + coef[4 + d] * tab[3 * NT + idx];   // C2 = c^2 (plane value if reduced)
            tab[4 * NT + idx] = s.r[d] * c;
            if (d == 0) tab[idx] *= A;
            if (out.tabf) {   // FP32 copies in stored units: E_x carries the VDF storage scale once
                float* tf = out.tabf + (long long)r * NTAB * NT;
                for (int t = 0; t < NTAB; ++t)
                    tf[t * NT + idx] = (float)(t == 0 && d == 0 ? tab[idx] * vg.vscale : tab[t * NT + idx]);
            }
        }
        if (out.scalf)
            for (int q = sl; q < RS; q += REC_LANES) out.scalf[(long long)r * RS + q] = (float)scal[q];
    }
}

// Context-free launcher of the record builder (caller supplies every buffer).
void build_records_raw(const RecSpec* d_specs, int nrec, const Records& out, const VGridDev& vg, cudaStream_t st) {
    if (nrec <= 0) return;
    const int threads = 128;
    const int warps = (nrec + REC_PER_WARP - 1) / REC_PER_WARP;
    const int blocks = (warps * 32 + threads - 1) / threads;
    k_build_records<<<blocks, threads, 0, st>>>(d_specs, nrec, out, vg);
}

void launch_build_records(gsis_ctx* c, const Records& out, int nrec, const RecSpec* d_specs) {
    if (nrec <= 0) return;
    const int threads = 128;
    const int warps = (nrec + REC_PER_WARP - 1) / REC_PER_WARP;
    const int blocks = (warps * 32 + threads - 1) / threads;
    k_build_records<<<blocks, threads, 0, c->stream>>>(d_specs, nrec, out, c->vg);
    c->launches++;
}

// ---------------------------------------------------------------------------- spec builders
__device__ static void cons_of(double rho, const double* u, double T, double* U) {
    U[0] = rho;
    U[1] = rho * u[0]; U[2] = rho * u[1]; U[3] = rho * u[2];
    U[4] = rho * (1.5 * T + 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
}

__device__ static void spec_maxwellian(RecSpec& s, double rho, const double* u, double T, int correct) {
    s.rho = rho; s.T = T;
    for (int d = 0; d < 3; ++d) { s.u[d] = u[d]; s.p[d] = 0.0; s.r[d] = 0.0; }
    for (int k = 0; k < 6; ++k) s.P2[k] = 0.0;
    s.p0 = 1.0;
    cons_of(rho, u, T, s.U);
    s.correct = correct;
}

// Shakhov reference state of each DVM cell from W^n and the heat flux of f^n
// about u^n (third moment stored by the moments pass), tau = mu(T)/p, and the
// diffuse-wall densities from the lagged outgoing half-range fluxes.
__global__ void k_cell_eq(int Nd, const int* __restrict__ dvm_cell, const double* __restrict__ W,
                          const double* __restrict__ mom, const int* __restrict__ side_bc,
                          const double* __restrict__ wall_den, double mu0, double omega,
                          RecSpec* specs, double* itau, double* rho_w, float* itauf, float* rho_wf) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nd) return;
    const int c = dvm_cell[k];
    const double rho = W[c * 5], T = W[c * 5 + 4];
    const double u[3] = {W[c * 5 + 1], W[c * 5 + 2], W[c * 5 + 3]};
    const double* m = mom + (long long)k * MOMN;
    const double q[3] = {0.5 * m[10], 0.5 * m[11], 0.5 * m[12]};
    const double p = rho * T;
    const double sc = 1.0 / (15.0 * p * T * T);
    RecSpec s;
    spec_maxwellian(s, rho, u, T, 1);
    for (int d = 0; d < 3; ++d) { s.p[d] = -5.0 * T * sc * q[d]; s.r[d] = sc * q[d]; }
    specs[k] = s;
    itau[k] = p / viscosity(T, mu0, omega);   // 1/tau, tau = mu(T)/p
    if (itauf) itauf[k] = (float)itau[k];
    for (int sd = 0; sd < 6; ++sd) {
        double v = 0.0;
        if (side_bc[c * 6 + sd] == GSIS_BC_WALL) v = m[13 + sd] / wall_den[c * 6 + sd];
        rho_w[(long long)k * 6 + sd] = v;
        if (rho_wf) rho_wf[(long long)k * 6 + sd] = (float)v;
    }
}

// Factor vectors of g~/tau for the sweep (eval_g in sweep_device.cuh), one
// block per DVM cell, from the cell's record (Eq. updatef's corrected
// Maxwellian tables) and 1/tau; formed in FP64 and stored in the sweep's
// arithmetic type T:
//   x(ix) = (E, E (B + R C2), E R, E C2 ; E C)             [gx4 ; gx1]
//   y(q)  = E_yz/tau (D + R_yz C2_yz, 1, C2_yz, R_yz ; A)   [gy4 ; gy1]
// so that g~/tau = sum of the five products x_i y_i.
template <typename T>
__global__ void k_build_gtab(int Nd, Records rec, VGridDev vg, const double* __restrict__ itau,
                             const float* __restrict__ itauf, T* __restrict__ gx4, T* __restrict__ gx1,
                             T* __restrict__ gy4, T* __restrict__ gy1) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    const int NT = vg.NT, nx = vg.nx, ny = vg.ny, nyz = vg.ny * vg.nz;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 arithmetic for FP32 factor vectors, from the FP32 record copies
        // (whose E_x carries the storage scale; the FP64 form below puts it on
        // the y-z part): the same products rounded once to FP32 become a few
        // rounding steps in FP32, far under the storage rounding, and the FP64
        // pipe (the bound of the FP64 form) is left alone.
        const float* tf = rec.tabf + (long long)k * NTAB * NT;
        const float* sf = rec.scalf + (long long)k * RS;
        const float p0 = sf[RS_P0], pxy = sf[RS_P2XY], pxz = sf[RS_P2XZ], pyz = sf[RS_P2YZ];
        const float it = itauf[k];
        for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
            const float E = tf[ix], B = tf[NT + ix], C = tf[2 * NT + ix], C2 = tf[3 * NT + ix], R = tf[4 * NT + ix];
            *reinterpret_cast<float4*>(gx4 + ((long long)k * nx + ix) * 4) =
                make_float4(E, E * (B + R * C2), E * R, E * C2);
            gx1[(long long)k * nx + ix] = E * C;
        }
        for (int q = threadIdx.x; q < nyz; q += blockDim.x) {
            const int iz = q / ny, jy = nx + q - iz * ny, jz = nx + ny + iz;
            const float Cy = tf[2 * NT + jy], Cz = tf[2 * NT + jz];
            const float Eyz = tf[jy] * tf[jz] * it;
            const float D = p0 + (tf[NT + jy] + tf[NT + jz]) + 2.0f * pyz * Cy * Cz;
            const float Ryz = tf[4 * NT + jy] + tf[4 * NT + jz];
            const float C2yz = tf[3 * NT + jy] + tf[3 * NT + jz];
            const float A = 2.0f * (pxy * Cy + pxz * Cz);
            *reinterpret_cast<float4*>(gy4 + ((long long)k * nyz + q) * 4) =
                make_float4(Eyz * (D + Ryz * C2yz), Eyz, Eyz * C2yz, Eyz * Ryz);
            gy1[(long long)k * nyz + q] = Eyz * A;
        }
        return;
    }
    const double* tab = rec.tab + (long long)k * NTAB * NT;
    const double* sc = rec.scal + (long long)k * RS;
    const double p0 = sc[RS_P0], pxy = sc[RS_P2XY], pxz = sc[RS_P2XZ], pyz = sc[RS_P2YZ];
    const double it = itau[k];
    for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
        const double E = tab[ix], B = tab[NT + ix], C = tab[2 * NT + ix], C2 = tab[3 * NT + ix], R = tab[4 * NT + ix];
        T* o = gx4 + ((long long)k * nx + ix) * 4;
        o[0] = (T)E;
        o[1] = (T)(E * (B + R * C2));
        o[2] = (T)(E * R);
        o[3] = (T)(E * C2);
        gx1[(long long)k * nx + ix] = (T)(E * C);
    }
    for (int q = threadIdx.x; q < nyz; q += blockDim.x) {
        const int jy = nx + q % ny, jz = nx + ny + q / ny;
        const double Cy = tab[2 * NT + jy], Cz = tab[2 * NT + jz];
        const double Eyz = tab[jy] * tab[jz] * it * vg.vscale;   // g~/tau in stored units
        const double D = p0 + (tab[NT + jy] + tab[NT + jz]) + 2.0 * pyz * Cy * Cz;
        const double Ryz = tab[4 * NT + jy] + tab[4 * NT + jz];
        const double C2yz = tab[3 * NT + jy] + tab[3 * NT + jz];
        const double A = 2.0 * (pxy * Cy + pxz * Cz);
        T* o = gy4 + ((long long)k * nyz + q) * 4;
        o[0] = (T)(Eyz * (D + Ryz * C2yz));
        o[1] = (T)Eyz;
        o[2] = (T)(Eyz * C2yz);
        o[3] = (T)(Eyz * Ryz);
        gy1[(long long)k * nyz + q] = (T)(Eyz * A);
    }
}

void launch_cell_eq(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    if (Nd == 0) return;
    k_cell_eq<<<(Nd + 127) / 128, 128, 0, c->stream>>>(Nd, c->dvm_cell, c->W, c->mom, c->m.side_bc, c->wall_den,
                                                        c->mu0, c->p.omega, c->specs, c->itau, c->rho_w, c->itauf,
                                                        c->rho_wf);
    c->launches++;
    launch_build_records(c, c->recG, Nd, c->specs);
    if (c->p.vdf_dtype == GSIS_F64)
        k_build_gtab<double><<<Nd, 128, 0, c->stream>>>(Nd, c->recG, c->vg, c->itau, c->itauf, (double*)c->gx4,
                                                        (double*)c->gx1, (double*)c->gy4, (double*)c->gy1);
    else
        k_build_gtab<float><<<Nd, 128, 0, c->stream>>>(Nd, c->recG, c->vg, c->itau, c->itauf, (float*)c->gx4,
                                                       (float*)c->gx1, (float*)c->gy4, (float*)c->gy1);
    c->launches++;
}

// Boundary records: far field -> conservation-corrected Maxwellian of the
// boundary state; wall -> unit-density Maxwellian at rest at T_w (emission
// shape, scaled by rho_w in the sweep).
__global__ void k_bc_specs(RecSpec* specs, const int* bc_type, const double* bc_state) {
    const int s = threadIdx.x;
    if (s >= 6) return;
    const double* st = bc_state + s * 5;
    RecSpec r;
    if (bc_type[s] == GSIS_BC_FARFIELD) {
        spec_maxwellian(r, st[0], st + 1, st[4], 1);
    } else if (bc_type[s] == GSIS_BC_WALL) {
        const double z[3] = {0.0, 0.0, 0.0};
        spec_maxwellian(r, 1.0, z, st[4], 0);
    } else {
        const double z[3] = {0.0, 0.0, 0.0};
        spec_maxwellian(r, 1.0, z, 1.0, 0);
    }
    specs[s] = r;
}

void launch_bc_records(gsis_ctx* c) {
    k_bc_specs<<<1, 32, 0, c->stream>>>(c->specs, c->d_bc_type, c->d_bc_state);
    c->launches++;
    launch_build_records(c, c->recBC, 6, c->specs);
}

// Denominator of the diffuse-wall density: sum over incoming velocities
// (xi . S_out <= 0) of w |xi . S_out| M_w, one block per (cell, wall side).
// Also the incoming half-range moments of the wall Maxwellian,
// wall_in[c][s] = sum_{xi.S <= 0} w (xi.S) (1, xi, |xi|^2/2) M_w, so that the
// kinetic wall flux of a face is (outgoing moments) + rho_w * wall_in.
__global__ void k_wall_den(int N, const int* __restrict__ side_bc, const double* __restrict__ Sout,
                           Records bc, VGridDev vg, double* wall_den, double* wall_in) {
    const int c = blockIdx.x;
    __shared__ double sm[32 * 6];
    for (int s = 0; s < 6; ++s) {
        if (side_bc[c * 6 + s] != GSIS_BC_WALL) continue;
        const double* S = Sout + ((long long)c * 6 + s) * 3;
        const double* sc = rec_scal(bc, s);
        const double* tb = rec_tab(bc, s, vg.NT);
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (long long v = threadIdx.x; v < vg.Nv; v += blockDim.x) {
            int ix, iy, iz;
            vsplit(v, vg.nx, vg.ny, ix, iy, iz);
            const double x0 = vg.xi[ix], x1 = vg.xi[vg.nx + iy], x2 = vg.xi[vg.nx + vg.ny + iz];
            const double xn = x0 * S[0] + x1 * S[1] + x2 * S[2];
            if (!(xn > 0.0)) {
                const double m = eval_rec(sc, tb, vg.NT, vg.nx, vg.ny, ix, iy, iz);
                const double g = xn * m;
                double psi[5];
                psi_node(vg, x0, x1, x2, iz, psi);
                acc[0] += -g * psi[0];
                acc[1] += g * psi[0];
                acc[2] += g * psi[1];
                acc[3] += g * psi[2];
                acc[4] += g * psi[3];
                acc[5] += g * psi[4];
            }
        }
        block_sum<6>(acc, sm);
        if (threadIdx.x == 0) {
            wall_den[c * 6 + s] = acc[0] * vg.w;
            for (int q = 0; q < 5; ++q) wall_in[((long long)c * 6 + s) * 5 + q] = acc[1 + q] * vg.w;
        }
    }
}

void launch_wall_den(gsis_ctx* c) {
    k_wall_den<<<c->m.N, 256, 0, c->stream>>>(c->m.N, c->m.side_bc, c->m.Sout, c->recBC, c->vg, c->wall_den,
                                              c->wall_in);
    c->launches++;
}

// Grad-13 interface distributions (Eq. G13_VDF) of NS cells next to DVM
// cells, from W^n and the NSF stress / heat flux at W^n, conservation-corrected.
__device__ static void spec_grad13(RecSpec& s, const double* Wc, const double* nsf9) {
    const double rho = Wc[0], T = Wc[4];
    const double u[3] = {Wc[1], Wc[2], Wc[3]};
    spec_maxwellian(s, rho, u, T, 1);
    const double rT2 = rho * T * T;
    for (int d = 0; d < 3; ++d) {
        const double q = nsf9[6 + d];
        s.p[d] = -q / rT2;
        s.r[d] = q / (5.0 * rT2 * T);
    }
    for (int k = 0; k < 6; ++k) s.P2[k] = nsf9[k] / (2.0 * rT2);
}

__global__ void k_ghost_specs(int ng, const int* __restrict__ ghost_cell, const double* __restrict__ W,
                              const double* __restrict__ nsf, RecSpec* specs) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int c = ghost_cell[g];
    RecSpec s;
    spec_grad13(s, W + c * 5, nsf + (long long)c * HOTN);
    specs[g] = s;
}

void launch_ghost_records(gsis_ctx* c) {
    if (c->n_ghost == 0) return;
    k_ghost_specs<<<(c->n_ghost + 127) / 128, 128, 0, c->stream>>>(c->n_ghost, c->ghost_cell, c->W, c->nsf, c->specs);
    c->launches++;
    launch_build_records(c, c->recGhost, c->n_ghost, c->specs);
}

// M~(W^{n+1}) and M~(W^{n+1/2}) for Eq. updatef.
__global__ void k_corr_specs(int Nd, const int* __restrict__ dvm_cell, const double* __restrict__ Wa,
                             RecSpec* specs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nd) return;
    const double* w = Wa + dvm_cell[k] * 5;
    const double u[3] = {w[1], w[2], w[3]};
    RecSpec s;
    spec_maxwellian(s, w[0], u, w[4], 1);
    specs[k] = s;
}

void launch_correction_records(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    if (Nd == 0) return;
    k_corr_specs<<<(Nd + 127) / 128, 128, 0, c->stream>>>(Nd, c->dvm_cell, c->W, c->specs);
    c->launches++;
    launch_build_records(c, c->recNew, Nd, c->specs);
    k_corr_specs<<<(Nd + 127) / 128, 128, 0, c->stream>>>(Nd, c->dvm_cell, c->Wh, c->specs);
    c->launches++;
    launch_build_records(c, c->recHalf, Nd, c->specs);
}

// Seed distributions for cells entering the DVM region: Grad-13 from W and
// its NSF stress / heat flux (adaptive start, Sec. 3.2) or the corrected
// Maxwellian M~(W) (all-kinetic start), into recNew slots of the new list.
__global__ void k_seed_specs(int ne, const int* __restrict__ enter, const int* __restrict__ dvm_cell,
                             const double* __restrict__ W, const double* __restrict__ nsf, int grad13,
                             RecSpec* specs) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int c = dvm_cell[enter[e]];
    RecSpec s;
    if (grad13) {
        spec_grad13(s, W + c * 5, nsf + (long long)c * HOTN);
    } else {
        const double u[3] = {W[c * 5 + 1], W[c * 5 + 2], W[c * 5 + 3]};
        spec_maxwellian(s, W[c * 5], u, W[c * 5 + 4], 1);
    }
    specs[e] = s;
}

void launch_seed_records(gsis_ctx* c, int ne, int grad13) {
    if (ne == 0) return;
    k_seed_specs<<<(ne + 127) / 128, 128, 0, c->stream>>>(ne, c->enter_list, c->dvm_cell, c->W, c->nsf, grad13,
                                                           c->specs);
    c->launches++;
    launch_build_records(c, c->recNew, ne, c->specs);
}


// ---------------------------------------------------------------------------- two-VDF reference pair
// Reference pair of Eq. general_model, g = (1 - 1/Z_r) g_t + g_r / Z_r for
// f0 and f1, for states S[n][12] = (rho, u (3), T_t, T_r, q_t (3), q_r (3)) on
// a full 3D grid.  Four conservation-corrected records per state: the
// Shakhov forms g_0t at (T_t, q_t) and g_0r at (T, q0), each corrected to its
// own translational energy, and the Maxwellians M~ at T_t and at T; per node
//   g0 = a g_0t + b g_0r,
//   g1 = a [(d_r/2) T_r g_0t + M~_t (q_r.c)/(rho T_t)] + b [(d_r/2) T g_0r + M~_T (q1.c)/(rho T)],
// a = 1 - 1/Z_r, b = 1/Z_r, T = (3 T_t + d_r T_r)/(3 + d_r) and (q0, q1) the
// mixing of (q_t, q_r) of Sec. 2 (g_1t and g_1r with R = 1: their
// Maxwellian factor is rho^-1 times that of g_0t, g_0r).
__device__ static void two_vdf_mix(const TwoVdfGas& g, const double* qt, const double* qr, double* q0, double* q1) {
    const double m00 = (2.0 - 3.0 * g.A[0]) * g.Zr + 1.0, m01 = -3.0 * g.A[1] * g.Zr;
    const double m10 = -g.A[2] * g.Zr, m11 = -g.A[3] * g.Zr + 1.0;
    for (int d = 0; d < 3; ++d) {
        q0[d] = m00 * qt[d] + m01 * qr[d];
        q1[d] = m10 * qt[d] + m11 * qr[d];
    }
}

__device__ static RecSpec spec_shakhov(double rho, const double* u, double T, const double* q) {
    RecSpec s;
    spec_maxwellian(s, rho, u, T, 1);
    const double sc = 1.0 / (15.0 * rho * T * T * T);   // 1/(15 p T^2), p = rho T
    for (int d = 0; d < 3; ++d) { s.p[d] = -5.0 * T * sc * q[d]; s.r[d] = sc * q[d]; }
    return s;
}

__global__ void k_two_vdf_specs(int n, const double* __restrict__ S, TwoVdfGas g, RecSpec* __restrict__ specs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* s = S + (long long)k * 12;
    const double rho = s[0], Tt = s[4], Tr = s[5];
    const double T = (3.0 * Tt + g.d_r * Tr) / (3.0 + g.d_r);
    double q0[3], q1[3];
    two_vdf_mix(g, s + 6, s + 9, q0, q1);
    RecSpec m;
    specs[4 * k + 0] = spec_shakhov(rho, s + 1, Tt, s + 6);
    specs[4 * k + 1] = spec_shakhov(rho, s + 1, T, q0);
    spec_maxwellian(m, rho, s + 1, Tt, 1);
    specs[4 * k + 2] = m;
    spec_maxwellian(m, rho, s + 1, T, 1);
    specs[4 * k + 3] = m;
}

// grid (x: velocity blocks, y: state); out[k][0][v] = g0, out[k][1][v] = g1
__global__ void k_two_vdf_eval(int n, const double* __restrict__ S, TwoVdfGas g, Records rec, VGridDev vg,
                               double* __restrict__ out) {
    const int k = blockIdx.y;
    if (k >= n) return;
    const long long Nv = vg.Nv;
    const int nx = vg.nx, ny = vg.ny, NT = vg.NT;
    const double* s = S + (long long)k * 12;
    const double rho = s[0], Tt = s[4], Tr = s[5];
    const double T = (3.0 * Tt + g.d_r * Tr) / (3.0 + g.d_r);
    double q0[3], q1[3];
    two_vdf_mix(g, s + 6, s + 9, q0, q1);
    const double a = 1.0 - 1.0 / g.Zr, b = 1.0 / g.Zr;
    const double* sc = rec.scal + (long long)4 * k * RS;
    const double* tb = rec.tab + (long long)4 * k * NTAB * NT;
    const long long TS = (long long)NTAB * NT;
    double* o0 = out + (long long)k * 2 * Nv;
    double* o1 = o0 + Nv;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < Nv; v += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(v % nx);
        const long long rr = v / nx;
        const int iy = (int)(rr % ny), iz = (int)(rr / ny);
        const double c0 = vg.xi[ix] - s[1], c1 = vg.xi[nx + iy] - s[2], c2 = vg.xi[nx + ny + iz] - s[3];
        const double G0t = eval_rec(sc, tb, NT, nx, ny, ix, iy, iz);
        const double G0r = eval_rec(sc + RS, tb + TS, NT, nx, ny, ix, iy, iz);
        const double Mt = eval_rec(sc + 2 * RS, tb + 2 * TS, NT, nx, ny, ix, iy, iz);
        const double Mr = eval_rec(sc + 3 * RS, tb + 3 * TS, NT, nx, ny, ix, iy, iz);
        const double qrc = s[9] * c0 + s[10] * c1 + s[11] * c2;
        const double q1c = q1[0] * c0 + q1[1] * c1 + q1[2] * c2;
        o0[v] = a * G0t + b * G0r;
        o1[v] = a * (0.5 * g.d_r * Tr * G0t + Mt * qrc / (rho * Tt)) + b * (0.5 * g.d_r * T * G0r + Mr * q1c / (rho * T));
    }
}

void launch_two_vdf_reference(gsis_ctx* c, const double* S, int n, const TwoVdfGas& g, RecSpec* specs,
                              const Records& rec, double* out) {
    if (n <= 0) return;
    k_two_vdf_specs<<<(n + 127) / 128, 128, 0, c->stream>>>(n, S, g, specs);
    c->launches++;
    launch_build_records(c, rec, 4 * n, specs);
    const long long Nv = c->vg.Nv;
    const int bx = (int)std::min<long long>((Nv + 255) / 256, 64);
    k_two_vdf_eval<<<dim3(bx, n), 256, 0, c->stream>>>(n, S, g, rec, c->vg, out);
    c->launches++;
}

}  // namespace gsis
