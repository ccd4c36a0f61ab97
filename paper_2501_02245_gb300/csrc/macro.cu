// Macroscopic synthetic solve (Eq. macro with the constitutive relations of
// Eq. full_constitutive and Eq. NSF_constitutive), monatomic gas, on ALL cells.
//
// Flux and relaxation choices (the paper defers them to another work; the
// same choices are made in the CPU reference):
//  * inviscid: kinetic flux-vector splitting (the Euler flux the
//    discrete-velocity upwind scheme carries for Maxwellian states, in closed
//    form) on index-space MUSCL-minmod states of (rho, u, p), first order
//    next to boundaries;
//  * viscous: NSF from the mean of the two cells' least-squares gradients
//    corrected along the line of centres, at the mean cell u and T, plus the
//    mean of the two cells' HoT;
//  * far field: the same splitting against the boundary state plus the
//    cell's HoT;
//    wall: cell pressure, no mass flux, NSF at u = 0 and T = T_w from a
//    one-sided gradient; at the wall of a DVM cell plus the frozen difference
//    between the kinetic wall flux of f^{n+1/2} and that NSF wall flux at
//    W^{n+1/2};
//  * DP-LUR pseudo-time relaxation (Wright, Candler & Bose 1998): scalar
//    diagonal (1/CFL + 1/2) sum lambda |S| (+ V/dt with the time term of
//    Eq. macro), k_sub Jacobi sweeps over Rusanov-split Euler flux changes.
// Every interior face flux is evaluated once, by one thread (face kernel),
// and gathered by both cells in a fixed order (cell kernel), so the scheme is
// exactly conservative and deterministic.
#include <algorithm>
#include <cooperative_groups.h>
#include "gsis_device.cuh"

namespace cg = cooperative_groups;

namespace gsis {


static MacroArgs margs(gsis_ctx* c) {
    MacroArgs a;
    a.N = c->m.N;
    a.nbr = c->m.nbr;
    a.side_bc = c->m.side_bc;
    a.Sout = c->m.Sout;
    a.xf = c->m.xf;
    a.cen = c->m.cen;
    a.vol = c->m.vol;
    a.lsq_w = c->m.lsq_w;
    a.bc_state = c->d_bc_state;
    a.fgeo = c->fgeo;
    a.bgeo = c->bgeo;
    a.bside = c->m.bside;
    a.nbside = c->m.nbside;
    a.nd = c->normal_components;
    a.fnd = c->face_nd;
    a.mu0 = c->mu0;
    a.omega = c->p.omega;
    return a;
}

// ---------------------------------------------------------------------------- gradients
// Least-squares gradient (face neighbours plus boundary face centres with the
// boundary value: far field -> boundary state; wall -> u = 0, |u| = 0, T = T_w,
// rho = cell value).  gu[c][j][i] = d u_j / d x_i.  ND: the LSQ weights have
// components 0..ND-1 only (MacroArgs::fnd); the others are written as zero.
template <int ND>
__device__ __forceinline__ void gradients_nd(const MacroArgs& a, const double* Wp, int with_rho_U, double* gu,
                                             double* gT, double* grho, double* gU, double* acell, int c) {
    const double* wc = Wp + c * 5;
    if (acell) acell[c] = sqrt(GAMMA * wc[4]);
    const double Uc = with_rho_U ? sqrt(wc[1] * wc[1] + wc[2] * wc[2] + wc[3] * wc[3]) : 0.0;
    double g[6][3];
    for (int q = 0; q < 6; ++q) g[q][0] = g[q][1] = g[q][2] = 0.0;
    for (int s = 0; s < 6; ++s) {
        const int n = a.nbr[c * 6 + s];
        const int bc = a.side_bc[c * 6 + s];
        double val[6];   // ux, uy, uz, T, rho, U
        if (n >= 0) {
            const double* wn = Wp + n * 5;
            val[0] = wn[1]; val[1] = wn[2]; val[2] = wn[3]; val[3] = wn[4]; val[4] = wn[0];
            val[5] = with_rho_U ? sqrt(wn[1] * wn[1] + wn[2] * wn[2] + wn[3] * wn[3]) : 0.0;
        } else if (bc == GSIS_BC_FARFIELD) {
            const double* st = a.bc_state + s * 5;
            val[0] = st[1]; val[1] = st[2]; val[2] = st[3]; val[3] = st[4]; val[4] = st[0];
            val[5] = with_rho_U ? sqrt(st[1] * st[1] + st[2] * st[2] + st[3] * st[3]) : 0.0;
        } else if (bc == GSIS_BC_WALL) {
            const double* st = a.bc_state + s * 5;
            val[0] = 0.0; val[1] = 0.0; val[2] = 0.0; val[3] = st[4]; val[4] = wc[0]; val[5] = 0.0;
        } else {
            continue;
        }
        const double phic[6] = {wc[1], wc[2], wc[3], wc[4], wc[0], Uc};
        const double* w = a.lsq_w + ((long long)c * 6 + s) * 3;
        const int nq = with_rho_U ? 6 : 4;
        for (int q = 0; q < nq; ++q) {
            const double dphi = val[q] - phic[q];
#pragma unroll
            for (int i = 0; i < ND; ++i) g[q][i] += w[i] * dphi;
        }
    }
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) gu[(long long)c * 9 + j * 3 + i] = g[j][i];
    for (int i = 0; i < 3; ++i) gT[(long long)c * 3 + i] = g[3][i];
    if (with_rho_U) {
        for (int i = 0; i < 3; ++i) {
            grho[(long long)c * 3 + i] = g[4][i];
            gU[(long long)c * 3 + i] = g[5][i];
        }
    }
}

__device__ __forceinline__ void gradients_cell(const MacroArgs& a, const double* Wp, int with_rho_U, double* gu,
                                               double* gT, double* grho, double* gU, double* acell, int c) {
    switch (a.fnd) {
        case 1: gradients_nd<1>(a, Wp, with_rho_U, gu, gT, grho, gU, acell, c); break;
        case 2: gradients_nd<2>(a, Wp, with_rho_U, gu, gT, grho, gU, acell, c); break;
        default: gradients_nd<3>(a, Wp, with_rho_U, gu, gT, grho, gU, acell, c); break;
    }
}

__global__ void k_gradients(MacroArgs a, const double* __restrict__ Wp, int with_rho_U, double* __restrict__ gu,
                            double* __restrict__ gT, double* __restrict__ grho, double* __restrict__ gU,
                            double* __restrict__ acell) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.N) gradients_cell(a, Wp, with_rho_U, gu, gT, grho, gU, acell, c);
}

void launch_gradients(gsis_ctx* c, const double* Wprim, bool with_rho_U) {
    const int N = c->m.N;
    k_gradients<<<(N + 63) / 64, 64, 0, c->stream>>>(margs(c), Wprim, with_rho_U ? 1 : 0, c->gu, c->gT, c->grho,
                                                     c->gU, c->acell);
    c->launches++;
}

// ---------------------------------------------------------------------------- NSF
__device__ __forceinline__ void nsf_of(double mu, const double* gu /*[j][i]*/, const double* gT, double* sig,
                                       double* q) {
    // G[i][j] = d u_j / d x_i = gu[j*3 + i]
    const double div = gu[0] + gu[4] + gu[8];
    const double two3 = 2.0 / 3.0;
    sig[0] = -mu * (2.0 * gu[0] - two3 * div);
    sig[1] = -mu * (2.0 * gu[4] - two3 * div);
    sig[2] = -mu * (2.0 * gu[8] - two3 * div);
    sig[3] = -mu * (gu[0 * 3 + 1] + gu[1 * 3 + 0]);   // xy: du_x/dy + du_y/dx
    sig[4] = -mu * (gu[0 * 3 + 2] + gu[2 * 3 + 0]);   // xz
    sig[5] = -mu * (gu[1 * 3 + 2] + gu[2 * 3 + 1]);   // yz
    const double kap = 3.75 * mu;
    q[0] = -kap * gT[0];
    q[1] = -kap * gT[1];
    q[2] = -kap * gT[2];
}

__global__ void k_nsf(int N, const double* __restrict__ Wp, const double* __restrict__ gu,
                      const double* __restrict__ gT, double mu0, double omega, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const double mu = viscosity(Wp[c * 5 + 4], mu0, omega);
    nsf_of(mu, gu + (long long)c * 9, gT + (long long)c * 3, out + (long long)c * HOTN, out + (long long)c * HOTN + 6);
}

void launch_nsf(gsis_ctx* c, const double* Wprim, double* out) {
    launch_gradients(c, Wprim, false);
    const int N = c->m.N;
    k_nsf<<<(N + 127) / 128, 128, 0, c->stream>>>(N, Wprim, c->gu, c->gT, c->mu0, c->p.omega, out);
    c->launches++;
}

// ---------------------------------------------------------------------------- conversions
__global__ void k_prim_to_cons(int N, const double* __restrict__ Wp, double* __restrict__ U) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const double r = Wp[c * 5], ux = Wp[c * 5 + 1], uy = Wp[c * 5 + 2], uz = Wp[c * 5 + 3], T = Wp[c * 5 + 4];
    U[c * 5] = r;
    U[c * 5 + 1] = r * ux;
    U[c * 5 + 2] = r * uy;
    U[c * 5 + 3] = r * uz;
    U[c * 5 + 4] = r * (1.5 * T + 0.5 * (ux * ux + uy * uy + uz * uz));
}

// (One FP64 division per state, its reciprocal reused: on GB300 a division
// costs about ten FP64-pipe operations.)
__device__ __forceinline__ void cons_to_prim(const double* U, double* Wp) {
    const double r = U[0], ir = 1.0 / r;
    const double ux = U[1] * ir, uy = U[2] * ir, uz = U[3] * ir;
    Wp[0] = r;
    Wp[1] = ux;
    Wp[2] = uy;
    Wp[3] = uz;
    Wp[4] = (2.0 * U[4] * ir - (ux * ux + uy * uy + uz * uz)) * (1.0 / 3.0);
}

__global__ void k_cons_to_prim(int N, const double* __restrict__ U, double* __restrict__ Wp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    cons_to_prim(U + c * 5, Wp + c * 5);
}

// Face geometry of the synthetic solve, computed once per mesh: for the high
// face of each direction |S|, n = S/|S|, the unit vector e between the cell
// centres and their distance; for every side |S|, n and the unit vector from
// the cell centre to the face centre and its length.
__global__ void k_face_geometry(MacroArgs a, double* __restrict__ fgeo, double* __restrict__ bgeo) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    for (int s = 0; s < 6; ++s) {
        const double* So = a.Sout + ((long long)c * 6 + s) * 3;
        const double Sabs = sqrt(So[0] * So[0] + So[1] * So[1] + So[2] * So[2]);
        double eb[3];
        for (int i = 0; i < 3; ++i) eb[i] = a.xf[((long long)c * 6 + s) * 3 + i] - a.cen[c * 3 + i];
        const double bd = sqrt(eb[0] * eb[0] + eb[1] * eb[1] + eb[2] * eb[2]);
        double* B = bgeo + ((long long)c * 6 + s) * 8;
        B[0] = Sabs;
        for (int i = 0; i < 3; ++i) B[1 + i] = Sabs > 0.0 ? So[i] / Sabs : 0.0;
        for (int i = 0; i < 3; ++i) B[4 + i] = bd > 0.0 ? eb[i] / bd : 0.0;
        B[7] = bd;
        if (s & 1) {
            const int d = s >> 1;
            const int R = a.nbr[c * 6 + s];
            double* G = fgeo + ((long long)c * 3 + d) * 8;
            for (int q = 0; q < 8; ++q) G[q] = 0.0;
            if (R >= 0) {
                double e[3];
                for (int i = 0; i < 3; ++i) e[i] = a.cen[R * 3 + i] - a.cen[c * 3 + i];
                const double dist = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
                G[0] = Sabs;
                for (int i = 0; i < 3; ++i) G[1 + i] = So[i] / Sabs;
                for (int i = 0; i < 3; ++i) G[4 + i] = e[i] / dist;
                G[7] = dist;
            }
        }
    }
}

void launch_face_geometry(gsis_ctx* c) {
    const int N = c->m.N;
    k_face_geometry<<<(N + 127) / 128, 128, 0, c->stream>>>(margs(c), c->fgeo, c->bgeo);
    c->launches++;
}

// W <- Wh + w (W - Wh): under-relaxed synthetic correction of the primitives.
__global__ void k_blend(int N, const double* __restrict__ Wh, double w, double* __restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 5) return;
    const double h = Wh[i];
    W[i] = h + w * (W[i] - h);
}

void launch_blend(gsis_ctx* c, const double* Wh, double w, double* W) {
    const int n = c->m.N * 5;
    k_blend<<<(n + 255) / 256, 256, 0, c->stream>>>(c->m.N, Wh, w, W);
    c->launches++;
}

void launch_prim_to_cons(gsis_ctx* c, const double* Wprim, double* Ucons) {
    const int N = c->m.N;
    k_prim_to_cons<<<(N + 127) / 128, 128, 0, c->stream>>>(N, Wprim, Ucons);
    c->launches++;
}

void launch_cons_to_prim(gsis_ctx* c, const double* Ucons, double* Wprim) {
    const int N = c->m.N;
    k_cons_to_prim<<<(N + 127) / 128, 128, 0, c->stream>>>(N, Ucons, Wprim);
    c->launches++;
}

// ---------------------------------------------------------------------------- fluxes
// Flux carried by the molecules of the Maxwellian (r, u, T) that cross a
// face of unit normal n in the direction sign*n (half-range moments of the
// normal Gaussian N(u.n, T); tangential thermal motion in closed form),
// added to F.
// (ND: the normal has components 0..ND-1 only; the others are exact zeros,
// so the terms they multiply are left out.)
template <int ND>
__device__ __forceinline__ void half_range_add(double r, const double* u, double T, const double* n, double sign,
                                               double* F) {
    double un = u[0] * n[0];
#pragma unroll
    for (int i = 1; i < ND; ++i) un += u[i] * n[i];
    // s = un / sqrt(T) and sqrt(T) = T / sqrt(T) from one reciprocal square root
    // (instead of a square root and two FP64 divisions)
    const double ist = rsqrt(T), st = T * ist, s = un * ist;
    const double P = 0.5 * (1.0 + sign * erf(s * 0.7071067811865476));        // 1/sqrt(2)
    const double D = sign * st * exp(-0.5 * s * s) * 0.3989422804014327;       // 1/sqrt(2 pi)
    const double M0 = un * P + D;
    const double M1 = (un * un + T) * P + un * D;
    const double M2 = (un * un * un + 3.0 * un * T) * P + (un * un + 2.0 * T) * D;
    double ut[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ut[i] = i < ND ? u[i] - un * n[i] : u[i];
    F[0] += r * M0;
#pragma unroll
    for (int i = 0; i < 3; ++i) F[1 + i] += r * (i < ND ? M1 * n[i] + ut[i] * M0 : ut[i] * M0);
    F[4] += 0.5 * r * (M2 + (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2] + 2.0 * T) * M0);
}

// Kinetic flux-vector splitting per unit area through the unit normal n: the
// left Maxwellian's molecules moving along +n plus the right one's moving
// along -n -- the Euler flux that the discrete-velocity upwind scheme carries
// for Maxwellian states.
template <int ND = 3>
__device__ void kfvs(double rL, const double* uL, double pL, double rR, const double* uR, double pR,
                     const double* n, double* F) {
    for (int q = 0; q < 5; ++q) F[q] = 0.0;
    half_range_add<ND>(rL, uL, pL / rL, n, 1.0, F);
    half_range_add<ND>(rR, uR, pR / rR, n, -1.0, F);
}

// Euler flux tensor of conserved state U: F[q * 3 + i] = flux of component q
// along axis i (so that F.S is euler_flux_dot(U, S)), one division.  Only the
// axes i < ND are formed: on a mesh whose face normals have no component
// along the others (ND = normal_components), F.S never reads them.
template <int ND>
__device__ __forceinline__ void euler_tensor(const double* U, double* F) {
    const double r = U[0], ir = 1.0 / r;
    const double u[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const double p = (GAMMA - 1.0) * (U[4] - 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
#pragma unroll
    for (int i = 0; i < ND; ++i) {
        F[i] = U[1 + i];
#pragma unroll
        for (int j = 0; j < 3; ++j) F[(1 + j) * 3 + i] = U[1 + j] * u[i] + (i == j ? p : 0.0);
        F[12 + i] = (U[4] + p) * u[i];
    }
}

// Change of the Euler flux tensor of cell c for the relaxation increment
// dU_c, F(U_c + dU_c) - F(U_c), with F(U_c) kept in F0 for the pseudo-step:
// each neighbour then reads the values instead of evaluating both fluxes
// (and their divisions) itself.
template <int ND>
__device__ __forceinline__ void flux_change(const double* U, const double* dU, const double* F0, double* dF, int c) {
    double Up[5], F1[15];
#pragma unroll
    for (int q = 0; q < 5; ++q) Up[q] = U[c * 5 + q] + dU[c * 5 + q];
    euler_tensor<ND>(Up, F1);
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int i = 0; i < ND; ++i) dF[(long long)c * 15 + q * 3 + i] = F1[q * 3 + i] - F0[(long long)c * 15 + q * 3 + i];
}

__device__ __forceinline__ void prim5(const double* w, double* q) {   // (rho, u, p)
    q[0] = w[0]; q[1] = w[1]; q[2] = w[2]; q[3] = w[3]; q[4] = w[0] * w[4];
}

// Interior face between L = cell c and R = its neighbour across side 2d+1
// (area vector S pointing L -> R).  Writes the total face flux (inviscid +
// viscous + HoT) F.S to Ff[c][d][5] and lambda |S| to lamf[c][d]; faces that
// do not exist (boundary) get lamf = -1.
// ND: on a mesh whose face normals, cell-to-cell vectors and LSQ weights have
// components 0..ND-1 only (MacroArgs::fnd), the gradient entries along the
// other directions are exact zeros and are not formed or multiplied: the same
// values as the 3D expressions.  (Every velocity component keeps its gradient:
// the out-of-plane velocity of a 2D flow is zero only up to rounding -- and up
// to the storage noise of BF16/FP16 VDFs -- and its viscous stress is what
// damps it.)
template <int ND>
__device__ __forceinline__ void face_flux_nd(const MacroArgs& a, const double* Wm, const double* gu,
                                             const double* gT, const double* hot, const double* acell, int ndir,
                                             double* Ff, double* lamf, int t) {
    const int L = t / ndir, d = t % ndir;
    const int Rr = a.nbr[L * 6 + 2 * d + 1];
    double* F = Ff + ((long long)L * 3 + d) * 5;
    if (Rr < 0) {
        lamf[(long long)L * 3 + d] = -1.0;
        return;
    }
    const double* S = a.Sout + ((long long)L * 6 + 2 * d + 1) * 3;
    const double* G = a.fgeo + ((long long)L * 3 + d) * 8;
    const double Sabs = G[0];
    const double nn[3] = {G[1], G[2], G[3]};
    // MUSCL face states: q -/+ 0.5 minmod of the one-sided differences (the
    // halved limiter on the integer pipe), first order where the second
    // neighbour is missing
    double qL[5], qR[5], mL[5] = {0, 0, 0, 0, 0}, mR[5] = {0, 0, 0, 0, 0};
    prim5(Wm + L * 5, qL);
    prim5(Wm + Rr * 5, qR);
    {
        const int lo = a.nbr[L * 6 + 2 * d];
        if (lo >= 0) {
            double ql[5];
            prim5(Wm + lo * 5, ql);
            for (int q = 0; q < 5; ++q) mL[q] = hmm_t<double>(qL[q] - ql[q], qR[q] - qL[q]);
        }
    }
    {
        const int hi = a.nbr[Rr * 6 + 2 * d + 1];
        if (hi >= 0) {
            double qh[5];
            prim5(Wm + hi * 5, qh);
            for (int q = 0; q < 5; ++q) mR[q] = hmm_t<double>(qR[q] - qL[q], qh[q] - qR[q]);
        }
    }
    double fl[5], fr[5];
    for (int q = 0; q < 5; ++q) { fl[q] = qL[q] + mL[q]; fr[q] = qR[q] - mR[q]; }
    double Fv[5];
    kfvs<ND>(fl[0], fl + 1, fl[4], fr[0], fr + 1, fr[4], nn, Fv);
    for (int q = 0; q < 5; ++q) Fv[q] *= Sabs;
    // viscous + HoT
    const double* wL = Wm + L * 5;
    const double* wR = Wm + Rr * 5;
    const double uf[3] = {0.5 * (wL[1] + wR[1]), 0.5 * (wL[2] + wR[2]), 0.5 * (wL[3] + wR[3])};
    const double Tf = 0.5 * (wL[4] + wR[4]);
    const double muf = viscosity(Tf, a.mu0, a.omega);
    const double e[3] = {G[4], G[5], G[6]};
    const double dist = G[7], idist = 1.0 / dist;
    // face gradients: cell average corrected along the line of centres, for every
    // velocity component j and the directions i below ND (the others are zero:
    // the LSQ weights and the line of centres have no such component)
    double guf[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gTf[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double gav[3], ge = 0.0;
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            gav[i] = 0.5 * (gu[(long long)L * 9 + j * 3 + i] + gu[(long long)Rr * 9 + j * 3 + i]);
            ge = i == 0 ? gav[0] * e[0] : ge + gav[i] * e[i];
        }
        const double corr = (wR[1 + j] - wL[1 + j]) * idist - ge;
#pragma unroll
        for (int i = 0; i < ND; ++i) guf[j * 3 + i] = gav[i] + corr * e[i];
    }
    {
        double gav[3], ge = 0.0;
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            gav[i] = 0.5 * (gT[(long long)L * 3 + i] + gT[(long long)Rr * 3 + i]);
            ge = i == 0 ? gav[0] * e[0] : ge + gav[i] * e[i];
        }
        const double corr = (wR[4] - wL[4]) * idist - ge;
#pragma unroll
        for (int i = 0; i < ND; ++i) gTf[i] = gav[i] + corr * e[i];
    }
    // Eq. NSF_constitutive (nsf_of) with the zero gradient entries (directions
    // i >= ND) not multiplied: the same values
    double sig[6], qf[3];
    {
        double div = guf[0];
        if (ND > 1) div += guf[4];
        if (ND > 2) div += guf[8];
        const double two3 = 2.0 / 3.0, t = two3 * div;
        sig[0] = -muf * (2.0 * guf[0] - t);
        sig[1] = ND > 1 ? -muf * (2.0 * guf[4] - t) : -muf * (-t);
        sig[2] = ND > 2 ? -muf * (2.0 * guf[8] - t) : -muf * (-t);
        sig[3] = -muf * (ND > 1 ? guf[1] + guf[3] : guf[3]);   // du_x/dy + du_y/dx
        sig[4] = -muf * (ND > 2 ? guf[2] + guf[6] : guf[6]);   // du_x/dz + du_z/dx
        sig[5] = ND > 1 ? -muf * (ND > 2 ? guf[5] + guf[7] : guf[7]) : 0.0;   // du_y/dz + du_z/dy
        const double kap = 3.75 * muf;
#pragma unroll
        for (int i = 0; i < 3; ++i) qf[i] = i < ND ? -kap * gTf[i] : 0.0;
    }
    const double* hL = hot + (long long)L * HOTN;
    const double* hR = hot + (long long)Rr * HOTN;
    double Sg[6], Q[3];
    for (int q = 0; q < 6; ++q) Sg[q] = sig[q] + 0.5 * (hL[q] + hR[q]);
    for (int q = 0; q < 3; ++q) Q[q] = qf[q] + 0.5 * (hL[6 + q] + hR[6 + q]);
    // sigma . S and q . S over the normal's components 0..ND-1
    const double row[3][3] = {{Sg[0], Sg[3], Sg[4]}, {Sg[3], Sg[1], Sg[5]}, {Sg[4], Sg[5], Sg[2]}};
    double SigS[3], QS = Q[0] * S[0];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        double v = row[r][0] * S[0];
#pragma unroll
        for (int k = 1; k < ND; ++k) v += row[r][k] * S[k];
        SigS[r] = v;
    }
#pragma unroll
    for (int k = 1; k < ND; ++k) QS += Q[k] * S[k];
    F[0] = Fv[0];
    F[1] = Fv[1] + SigS[0];
    F[2] = Fv[2] + SigS[1];
    F[3] = Fv[3] + SigS[2];
    F[4] = Fv[4] + ((SigS[0] * uf[0] + SigS[1] * uf[1] + SigS[2] * uf[2]) + QS);
    const double aL = acell[L], aR = acell[Rr];
    double un = uf[0] * nn[0];
#pragma unroll
    for (int k = 1; k < ND; ++k) un += uf[k] * nn[k];
    const double lam = fabs(un) + 0.5 * (aL + aR) + 5.0 * muf / (0.5 * (wL[0] + wR[0]) * dist);
    lamf[(long long)L * 3 + d] = lam * Sabs;
}

__device__ __forceinline__ void face_flux_one(const MacroArgs& a, const double* Wm, const double* gu,
                                              const double* gT, const double* hot, const double* acell, int ndir,
                                              double* Ff, double* lamf, int t) {
    switch (a.fnd) {
        case 1: face_flux_nd<1>(a, Wm, gu, gT, hot, acell, ndir, Ff, lamf, t); break;
        case 2: face_flux_nd<2>(a, Wm, gu, gT, hot, acell, ndir, Ff, lamf, t); break;
        default: face_flux_nd<3>(a, Wm, gu, gT, hot, acell, ndir, Ff, lamf, t); break;
    }
}

// NSF flux through wall side s of cell c at state w (prim) with cell gradients
// gu, gT: no mass flux, cell pressure, NSF stress and heat flux at u = 0,
// T = T_w from the cell gradient corrected along the cell-to-face line.
__device__ void wall_nsf_flux(const MacroArgs& a, const double* w, const double* gu, const double* gT, int c, int s,
                              double* Fb) {
    const double* So = a.Sout + ((long long)c * 6 + s) * 3;
    const double Tw = a.bc_state[s * 5 + 4];
    const double* G = a.bgeo + ((long long)c * 6 + s) * 8;
    const double eb[3] = {G[4], G[5], G[6]};
    const double bdist = G[7];
    double guw[9], gTw[3];
    for (int j = 0; j < 3; ++j) {
        const double* gc = gu + j * 3;
        const double corr = (0.0 - w[1 + j]) / bdist - (gc[0] * eb[0] + gc[1] * eb[1] + gc[2] * eb[2]);
        for (int i = 0; i < 3; ++i) guw[j * 3 + i] = gc[i] + corr * eb[i];
    }
    {
        const double corr = (Tw - w[4]) / bdist - (gT[0] * eb[0] + gT[1] * eb[1] + gT[2] * eb[2]);
        for (int i = 0; i < 3; ++i) gTw[i] = gT[i] + corr * eb[i];
    }
    double sig[6], qw[3];
    nsf_of(viscosity(Tw, a.mu0, a.omega), guw, gTw, sig, qw);
    const double p = w[0] * w[4];
    const double SigS[3] = {sig[0] * So[0] + sig[3] * So[1] + sig[4] * So[2],
                            sig[3] * So[0] + sig[1] * So[1] + sig[5] * So[2],
                            sig[4] * So[0] + sig[5] * So[1] + sig[2] * So[2]};
    Fb[0] = 0.0;
    Fb[1] = p * So[0] + SigS[0];
    Fb[2] = p * So[1] + SigS[1];
    Fb[3] = p * So[2] + SigS[2];
    Fb[4] = qw[0] * So[0] + qw[1] * So[1] + qw[2] * So[2];
}

// Wall correction of the synthetic solve: for each wall side of a DVM cell,
// the kinetic wall flux of f^{n+1/2} minus the NSF wall flux at W^{n+1/2}
// (gradients of W^{n+1/2} in gu, gT); zero elsewhere.
__global__ void k_wall_corr(MacroArgs a, const int* __restrict__ cell2dvm, const double* __restrict__ Wh,
                            const double* __restrict__ gu, const double* __restrict__ gT,
                            const double* __restrict__ wall_kin, double* __restrict__ wall_corr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    for (int s = 0; s < 6; ++s) {
        double* o = wall_corr + ((long long)c * 6 + s) * 5;
        if (a.nbr[c * 6 + s] < 0 && a.side_bc[c * 6 + s] == GSIS_BC_WALL && cell2dvm[c] >= 0) {
            double F[5];
            wall_nsf_flux(a, Wh + c * 5, gu + (long long)c * 9, gT + (long long)c * 3, c, s, F);
            const double* kin = wall_kin + ((long long)c * 6 + s) * 5;
            for (int q = 0; q < 5; ++q) o[q] = kin[q] - F[q];
        } else {
            for (int q = 0; q < 5; ++q) o[q] = 0.0;
        }
    }
}

void launch_wall_corr(gsis_ctx* c) {
    const int N = c->m.N;
    k_wall_corr<<<(N + 63) / 64, 64, 0, c->stream>>>(margs(c), c->cell2dvm, c->Wh, c->gu, c->gT, c->wall_kin,
                                                     c->wall_corr);
    c->launches++;
}

// Wall loads per unit wall area for every cell with wall sides, written to
// out[c * FIELDS_N + FIELD_WALL + (0: heat flux into the wall, 1: pressure,
// 2..4: shear vector)]: the wall fluxes F (kinetic, wall_kin of the current f,
// for DVM cells; the NSF wall flux at the current state for NS cells), with
// pressure F_m.n and shear F_m - (F_m.n) n of the momentum part F_m, summed
// over the wall sides and divided by their area.
__global__ void k_wall_loads(MacroArgs a, const int* __restrict__ cell2dvm, const double* __restrict__ W,
                             const double* __restrict__ gu, const double* __restrict__ gT,
                             const double* __restrict__ wall_kin, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    double num[5] = {0, 0, 0, 0, 0}, area = 0.0;
    for (int s = 0; s < 6; ++s) {
        if (a.nbr[c * 6 + s] >= 0 || a.side_bc[c * 6 + s] != GSIS_BC_WALL) continue;
        double F[5];
        if (cell2dvm[c] >= 0) {
            for (int q = 0; q < 5; ++q) F[q] = wall_kin[((long long)c * 6 + s) * 5 + q];
        } else {
            wall_nsf_flux(a, W + c * 5, gu + (long long)c * 9, gT + (long long)c * 3, c, s, F);
        }
        const double* G = a.bgeo + ((long long)c * 6 + s) * 8;   // |S|, unit normal
        const double Fn = F[1] * G[1] + F[2] * G[2] + F[3] * G[3];
        num[0] += F[4];
        num[1] += Fn;
        for (int i = 0; i < 3; ++i) num[2 + i] += F[1 + i] - Fn * G[1 + i];
        area += G[0];
    }
    double* o = out + (long long)c * FIELDS_N + FIELD_WALL;
    for (int q = 0; q < 5; ++q) o[q] = area > 0.0 ? num[q] / area : 0.0;
}

// Eq. full_constitutive at the current state, out[c * FIELDS_N + 0..8]:
// sigma = sigma_NSF(W) + HoT_sigma (xx, yy, zz, xy, xz, yz), q = q_NSF(W) +
// HoT_q, with the HoT of the last kinetic step (zero in NS cells); and the
// pressure rho T at index 9.
__global__ void k_constitutive(int N, const double* __restrict__ W, const double* __restrict__ gu,
                               const double* __restrict__ gT, const double* __restrict__ hot, double mu0,
                               double omega, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    double sig[6], q[3];
    nsf_of(viscosity(W[c * 5 + 4], mu0, omega), gu + (long long)c * 9, gT + (long long)c * 3, sig, q);
    double* o = out + (long long)c * FIELDS_N;
    const double* h = hot + (long long)c * HOTN;
    for (int k = 0; k < 6; ++k) o[k] = sig[k] + h[k];
    for (int k = 0; k < 3; ++k) o[6 + k] = q[k] + h[6 + k];
    o[9] = W[c * 5] * W[c * 5 + 4];
}

void launch_fields(gsis_ctx* c, bool wall, bool cons) {
    const int N = c->m.N;
    if (wall && c->has_wall) launch_wall_flux(c);   // kinetic wall fluxes of the current f
    launch_gradients(c, c->W, false);               // gradients of the current state
    if (wall) {
        k_wall_loads<<<(N + 127) / 128, 128, 0, c->stream>>>(margs(c), c->cell2dvm, c->W, c->gu, c->gT,
                                                            c->wall_kin, c->fields);
        c->launches++;
    }
    if (cons) {
        k_constitutive<<<(N + 127) / 128, 128, 0, c->stream>>>(N, c->W, c->gu, c->gT, c->hot, c->mu0, c->p.omega,
                                                               c->fields);
        c->launches++;
    }
}

// Flux F.S_out through boundary side s of cell c and lambda |S| of the side,
// into Fbnd[c][s][0..5]: far field, the kinetic flux-vector splitting against
// the far-field state with the cell's HoT; wall, the NSF wall flux plus the
// wall correction.  Formed in the face phase (boundary side j of a.bside), so
// that the residual phase only gathers.
__device__ __forceinline__ void boundary_flux_one(const MacroArgs& a, const double* Wm, const double* gu,
                                                  const double* gT, const double* hot, const double* wall_corr,
                                                  double* Fbnd, int j) {
    const int cs = a.bside[j], c = cs / 6, s = cs - 6 * c;
    const int bc = a.side_bc[cs];
    const double* wc = Wm + c * 5;
    const double rho_c = wc[0], T_c = wc[4], p_c = rho_c * T_c;
    const double u_c[3] = {wc[1], wc[2], wc[3]};
    const double* So = a.Sout + (long long)cs * 3;
    const double* st = a.bc_state + s * 5;
    const double* G = a.bgeo + (long long)cs * 8;
    const double Sabs = G[0];
    const double nn[3] = {G[1], G[2], G[3]};
    const double* h = hot + (long long)c * HOTN;
    double Fb[5];
    const double bdist = G[7];
    if (bc == GSIS_BC_FARFIELD) {
        kfvs(rho_c, u_c, p_c, st[0], st + 1, st[0] * st[4], nn, Fb);
        for (int q = 0; q < 5; ++q) Fb[q] *= Sabs;
        const double SigS[3] = {h[0] * So[0] + h[3] * So[1] + h[4] * So[2],
                                h[3] * So[0] + h[1] * So[1] + h[5] * So[2],
                                h[4] * So[0] + h[5] * So[1] + h[2] * So[2]};
        const double ufb[3] = {0.5 * (u_c[0] + st[1]), 0.5 * (u_c[1] + st[2]), 0.5 * (u_c[2] + st[3])};
        Fb[1] += SigS[0];
        Fb[2] += SigS[1];
        Fb[3] += SigS[2];
        Fb[4] += (SigS[0] * ufb[0] + SigS[1] * ufb[1] + SigS[2] * ufb[2]) +
                 (h[6] * So[0] + h[7] * So[1] + h[8] * So[2]);
    } else {
        wall_nsf_flux(a, wc, gu + (long long)c * 9, gT + (long long)c * 3, c, s, Fb);
        const double* wcr = wall_corr + (long long)cs * 5;
        for (int q = 0; q < 5; ++q) Fb[q] += wcr[q];
    }
    const double a_c = sqrt(GAMMA * p_c / rho_c);
    const double mu_c = viscosity(T_c, a.mu0, a.omega);
    const double lam = fabs(u_c[0] * nn[0] + u_c[1] * nn[1] + u_c[2] * nn[2]) + a_c +
                       5.0 * mu_c / (rho_c * 2.0 * bdist);
    double* o = Fbnd + (long long)cs * 6;
    for (int q = 0; q < 5; ++q) o[q] = Fb[q];
    o[5] = lam * Sabs;
}

// Face phase of the per-phase kernels: interior faces (N * ndir threads), then
// the far-field and wall sides.
__global__ void k_face_flux(MacroArgs a, const double* __restrict__ Wm, const double* __restrict__ gu,
                            const double* __restrict__ gT, const double* __restrict__ hot,
                            const double* __restrict__ acell, int ndir, double* __restrict__ Ff,
                            double* __restrict__ lamf, const double* __restrict__ wall_corr,
                            double* __restrict__ Fbnd) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nf = a.N * ndir;
    if (t < nf) face_flux_one(a, Wm, gu, gT, hot, acell, ndir, Ff, lamf, t);
    else if (t < nf + a.nbside) boundary_flux_one(a, Wm, gu, gT, hot, wall_corr, Fbnd, t - nf);
}

// Cell residual R_c = -sum_F F.S_out (gathering the face fluxes in side
// order: interior faces from Ff, far-field and wall sides from Fbnd), lambda|S|
// per side, the reciprocal 1/D of the diagonal (in D) and dU0 = R/D.
__device__ __forceinline__ void cell_residual_one(const MacroArgs& a, const double* Wm, const double* U,
                                                  const double* Un, const double* gu, const double* gT,
                                                  const double* hot, const double* Ff, const double* lamf,
                                                  const double* Fbnd, double cfl, double dt, double* R, double* D,
                                                  double* lamS, double* dU, double* F0, double* dF, int c) {
    double Rc[5] = {0, 0, 0, 0, 0};
    double lam_sum = 0.0;
    for (int s = 0; s < 6; ++s) {
        const int n = a.nbr[c * 6 + s];
        const int bc = a.side_bc[c * 6 + s];
        const int d = s >> 1;
        if (n >= 0) {
            const bool isL = (s & 1) != 0;
            const int L = isL ? c : n;
            const double* F = Ff + ((long long)L * 3 + d) * 5;
            const double sgn = isL ? -1.0 : 1.0;
            for (int q = 0; q < 5; ++q) Rc[q] += sgn * F[q];
            const double ls = lamf[(long long)L * 3 + d];
            lamS[(long long)c * 6 + s] = ls;
            lam_sum += ls;
        } else if (bc == GSIS_BC_FARFIELD || bc == GSIS_BC_WALL) {   // formed in the face phase
            const double* Fb = Fbnd + ((long long)c * 6 + s) * 6;
            for (int q = 0; q < 5; ++q) Rc[q] -= Fb[q];
            lamS[(long long)c * 6 + s] = Fb[5];
            lam_sum += Fb[5];
        } else {
            lamS[(long long)c * 6 + s] = 0.0;
        }
    }
    double Dc = (1.0 / cfl + 0.5) * lam_sum;
    if (dt > 0.0) {
        const double Vdt = a.vol[c] / dt;
        for (int q = 0; q < 5; ++q) Rc[q] -= Vdt * (U[c * 5 + q] - Un[c * 5 + q]);
        Dc += Vdt;
    }
    const double iD = 1.0 / Dc;
    D[c] = iD;   // the relaxation sweeps multiply by the reciprocal
    for (int q = 0; q < 5; ++q) {
        R[c * 5 + q] = Rc[q];
        dU[c * 5 + q] = Rc[q] * iD;
    }
    if (dF) {   // relaxation sweeps follow: the flux tensor of U_c and its change for dU_c
        switch (a.nd) {
            case 1: euler_tensor<1>(U + c * 5, F0 + (long long)c * 15); flux_change<1>(U, dU, F0, dF, c); break;
            case 2: euler_tensor<2>(U + c * 5, F0 + (long long)c * 15); flux_change<2>(U, dU, F0, dF, c); break;
            default: euler_tensor<3>(U + c * 5, F0 + (long long)c * 15); flux_change<3>(U, dU, F0, dF, c); break;
        }
    }
}

__global__ void k_cell_residual(MacroArgs a, const double* __restrict__ Wm, const double* __restrict__ U,
                                const double* __restrict__ Un, const double* __restrict__ gu,
                                const double* __restrict__ gT, const double* __restrict__ hot,
                                const double* __restrict__ Ff, const double* __restrict__ lamf,
                                const double* __restrict__ Fbnd, double cfl, double dt,
                                double* __restrict__ R, double* __restrict__ D, double* __restrict__ lamS,
                                double* __restrict__ dU, double* __restrict__ F0, double* __restrict__ dF) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.N) cell_residual_one(a, Wm, U, Un, gu, gT, hot, Ff, lamf, Fbnd, cfl, dt, R, D, lamS, dU, F0, dF, c);
}

// One Jacobi sweep: dU_new = (R - 1/2 sum_j [dF_j . S_out - lambda|S| dU_j]) / D,
// dF_j = F(U_j + dU_j) - F(U_j) read from the neighbour's flux-change tensor
// (dFin); with dFout the cell's own tensor for dU_new follows for the next sweep.
// The two sums are accumulated apart (FMA chains over the normal components
// that can be nonzero) and combined once.
template <int ND>
__device__ __forceinline__ void relax_nd(const MacroArgs& a, const double* U, const double* R, const double* D,
                                         const double* lamS, const double* dUin, double* dUout, const double* dFin,
                                         double* dFout, const double* F0, int c) {
    double fs[5] = {0, 0, 0, 0, 0}, ld[5] = {0, 0, 0, 0, 0};
    for (int s = 0; s < 6; ++s) {
        const int n = a.nbr[c * 6 + s];
        if (n < 0) continue;
        const double* So = a.Sout + ((long long)c * 6 + s) * 3;
        const double* dF = dFin + (long long)n * 15;
        const double ls = lamS[(long long)c * 6 + s];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double t = fs[q];
#pragma unroll
            for (int i = 0; i < ND; ++i) t = fma(dF[q * 3 + i], So[i], t);
            fs[q] = t;
            ld[q] = fma(ls, dUin[n * 5 + q], ld[q]);
        }
    }
    const double iD = D[c];   // 1 / D
#pragma unroll
    for (int q = 0; q < 5; ++q) dUout[c * 5 + q] = (R[c * 5 + q] - 0.5 * (fs[q] - ld[q])) * iD;
    if (dFout) flux_change<ND>(U, dUout, F0, dFout, c);
}

__device__ __forceinline__ void relax_one(const MacroArgs& a, const double* U, const double* R, const double* D,
                                          const double* lamS, const double* dUin, double* dUout, const double* dFin,
                                          double* dFout, const double* F0, int c) {
    switch (a.nd) {
        case 1: relax_nd<1>(a, U, R, D, lamS, dUin, dUout, dFin, dFout, F0, c); break;
        case 2: relax_nd<2>(a, U, R, D, lamS, dUin, dUout, dFin, dFout, F0, c); break;
        default: relax_nd<3>(a, U, R, D, lamS, dUin, dUout, dFin, dFout, F0, c); break;
    }
}

__global__ void k_relax(MacroArgs a, const double* __restrict__ U, const double* __restrict__ R,
                        const double* __restrict__ D, const double* __restrict__ lamS, const double* __restrict__ dUin,
                        double* __restrict__ dUout, const double* __restrict__ dFin, double* __restrict__ dFout,
                        const double* __restrict__ F0) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.N) relax_one(a, U, R, D, lamS, dUin, dUout, dFin, dFout, F0, c);
}


__device__ __forceinline__ void update_one(double* U, const double* dU, double* Wm, int c) {
    for (int q = 0; q < 5; ++q) U[c * 5 + q] += dU[c * 5 + q];
    cons_to_prim(U + c * 5, Wm + c * 5);
}

__global__ void k_update(int N, double* __restrict__ U, const double* __restrict__ dU, double* __restrict__ Wm) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) update_one(U, dU, Wm, c);
}

// The last Jacobi sweep of a pseudo-step followed by the update of the
// cell's own state (U += dU, primitive Wm): the sweep reads U only through the
// flux change, which the last sweep does not form, so each cell may update
// its state in place (one launch instead of two, the same values).
__global__ void k_relax_update(MacroArgs a, double* __restrict__ U, const double* __restrict__ R,
                               const double* __restrict__ D, const double* __restrict__ lamS,
                               const double* __restrict__ dUin, double* __restrict__ dUout,
                               const double* __restrict__ dFin, double* __restrict__ Wm) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    relax_one(a, U, R, D, lamS, dUin, dUout, dFin, nullptr, nullptr, c);
    update_one(U, dUout, Wm, c);
}

// The whole pseudo-time block of one solve in one thread-block cluster of
// `cs` CTAs (meshes up to a few thousand cells: the 1D shocks, solve
// batches).  The same per-cell and per-face functions as the multi-block
// kernels, separated by cluster barriers (release/acquire at cluster scope,
// so every CTA of the cluster sees the others' global-memory writes of the
// previous phase), so the result is identical.  A batch of solves uses
// clusters to occupy the SMs its solves alone would leave idle (64 solves:
// clusters of two, 5 % faster).  Jobs are clusters 0, 1, ... of the grid.
__device__ __forceinline__ void fused_sync(int cs) {
    if (cs > 1)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

__global__ void __launch_bounds__(MACRO_FUSED_THREADS, 1) k_macro_fused(const MacroJob* __restrict__ jobs, int cs) {
    const MacroJob& J = jobs[blockIdx.x / cs];
    const int first = (blockIdx.x % cs) * blockDim.x + threadIdx.x, stride = cs * blockDim.x;
    const MacroArgs a = J.a;
    const int N = a.N;
    for (int it = 0; it < J.steps; ++it) {
        for (int c = first; c < N; c += stride)
            gradients_cell(a, J.Wm, 0, J.gu, J.gT, nullptr, nullptr, J.acell, c);
        fused_sync(cs);
        for (int t = first; t < N * J.ndir + a.nbside; t += stride) {
            if (t < N * J.ndir) face_flux_one(a, J.Wm, J.gu, J.gT, J.hot, J.acell, J.ndir, J.Ff, J.lamf, t);
            else boundary_flux_one(a, J.Wm, J.gu, J.gT, J.hot, J.wall_corr, J.Fbnd, t - N * J.ndir);
        }
        fused_sync(cs);
        for (int c = first; c < N; c += stride)
            cell_residual_one(a, J.Wm, J.U, J.Un, J.gu, J.gT, J.hot, J.Ff, J.lamf, J.Fbnd, J.cfl, J.dt, J.R,
                              J.D, J.lamS, J.dU, J.F0, J.k_sub > 0 ? J.dFa : nullptr, c);
        fused_sync(cs);
        double* din = J.dU;
        double* dout = J.dU2;
        for (int s = 0; s < J.k_sub; ++s) {
            double* fin = (s & 1) ? J.dFb : J.dFa;
            double* fout = s + 1 < J.k_sub ? ((s & 1) ? J.dFa : J.dFb) : nullptr;
            for (int c = first; c < N; c += stride) relax_one(a, J.U, J.R, J.D, J.lamS, din, dout, fin, fout, J.F0, c);
            fused_sync(cs);
            double* t = din; din = dout; dout = t;
        }
        for (int c = first; c < N; c += stride) update_one(J.U, din, J.Wm, c);
        fused_sync(cs);
    }
}

// Largest usable cluster size <= want (a power of two, at most 8) for the
// fused kernel on the current device; 1 if clusters cannot be resident.
int fused_cluster_size(int want) {
    static int cached[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int cs = 1;
    while (cs * 2 <= want && cs * 2 <= 8) cs *= 2;
    for (; cs > 1; cs /= 2) {
        if (cached[cs] == 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(MACRO_FUSED_THREADS);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cs;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_macro_fused, &cfg) != cudaSuccess) {
                cudaGetLastError();
                n = 0;
            }
            cached[cs] = n > 0 ? 1 : -1;
        }
        if (cached[cs] > 0) return cs;
    }
    return 1;
}

MacroJob macro_job(gsis_ctx* c, int steps, bool time_term) {
    MacroJob J;
    J.a = margs(c);
    J.steps = steps;
    J.ndir = c->normal_components;
    J.k_sub = c->p.k_sub;
    J.cfl = c->p.cfl;
    J.dt = time_term ? c->p.dt : 0.0;
    J.Wm = c->Wm; J.U = c->U; J.Un = c->Un; J.gu = c->gu; J.gT = c->gT; J.hot = c->hot; J.Ff = c->Ff;
    J.lamf = c->lamf; J.wall_corr = c->wall_corr; J.R = c->R; J.D = c->D; J.lamS = c->lamS; J.dU = c->dU;
    J.dU2 = c->dU2;
    J.acell = c->acell;
    J.F0 = c->F0;
    J.dFa = c->dFa;
    J.dFb = c->dFb;
    J.Fbnd = c->Fbnd;
    return J;
}

// cs: cluster size from fused_cluster_size (called before any stream capture).
void launch_macro_fused(const MacroJob* d_jobs, int njobs, cudaStream_t stream, int cs) {
    if (cs > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(njobs * cs);
        cfg.blockDim = dim3(MACRO_FUSED_THREADS);
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_macro_fused, d_jobs, cs);
        return;
    }
    k_macro_fused<<<njobs, MACRO_FUSED_THREADS, 0, stream>>>(d_jobs, 1);
}

// Cluster size for one fused solve alone: one CTA (measured on the 200-cell
// shock: a cluster of two CTAs was 8 % slower -- the phases are bound by
// their dependent loads and the barriers, not by one SM's FP64 rate).
int fused_cluster_for(int N) {
    (void)N;
    return 1;
}

// ---------------------------------------------------------------------------- persistent kernel
// The whole block of pseudo-steps of one solve in ONE cooperative launch
// over all SMs (meshes above MACRO_FUSED_MAX_CELLS cells: the cylinder, the
// sphere).  The same per-cell and per-face functions as the per-phase
// kernels, separated by a grid-wide barrier, so the result is identical;
// what goes away is the launch latency of the ~(4 + k_sub) kernels per
// pseudo-step.  Every wait of the barrier is bounded by spin_limit polls:
// a block that runs out records the error and returns, and every other
// block returns at its next barrier (the host reports GSIS_ERR_TIMEOUT).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Returns false when the barrier failed (this block's wait ran out, or
// another block's did): the caller returns at once.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned expected, unsigned long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_gpu(&bar->gen);   // read before arriving: gen cannot move before we arrive
        __threadfence();                                // this block's writes before its arrival
        const unsigned arrived = atomicAdd(&bar->count, 1u);
        if (arrived == expected - 1) {
            bar->count = 0;                             // reset for the next barrier before releasing
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned long long polls = 0;
            while (ld_acquire_gpu(&bar->gen) == g) {
                if (++polls > spin_limit || ld_relaxed_gpu(&bar->err) != 0) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (!ok) atomicExch(&bar->err, 1);
        __threadfence();                                // the other blocks' writes before ours
        s_ok = ok && ld_relaxed_gpu(&bar->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(MACRO_PERSISTENT_THREADS, 2)
    k_macro_persistent(MacroJob J, GridBarrier* bar, unsigned long long spin_limit, int stall) {
    const MacroArgs a = J.a;
    const int N = a.N;
    const int first = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    // stall (test hook): the barrier waits for one block more than the grid
    // holds, so its wait can only end by running out of spin_limit polls
    const unsigned expected = gridDim.x + (stall ? 1u : 0u);
    for (int it = 0; it < J.steps; ++it) {
        for (int c = first; c < N; c += stride)
            gradients_cell(a, J.Wm, 0, J.gu, J.gT, nullptr, nullptr, J.acell, c);
        if (!grid_barrier(bar, expected, spin_limit)) return;
        for (int t = first; t < N * J.ndir + a.nbside; t += stride) {
            if (t < N * J.ndir) face_flux_one(a, J.Wm, J.gu, J.gT, J.hot, J.acell, J.ndir, J.Ff, J.lamf, t);
            else boundary_flux_one(a, J.Wm, J.gu, J.gT, J.hot, J.wall_corr, J.Fbnd, t - N * J.ndir);
        }
        if (!grid_barrier(bar, expected, spin_limit)) return;
        for (int c = first; c < N; c += stride)
            cell_residual_one(a, J.Wm, J.U, J.Un, J.gu, J.gT, J.hot, J.Ff, J.lamf, J.Fbnd, J.cfl, J.dt, J.R,
                              J.D, J.lamS, J.dU, J.F0, J.k_sub > 0 ? J.dFa : nullptr, c);
        if (!grid_barrier(bar, expected, spin_limit)) return;
        double* din = J.dU;
        double* dout = J.dU2;
        for (int s = 0; s < J.k_sub; ++s) {
            double* fin = (s & 1) ? J.dFb : J.dFa;
            double* fout = s + 1 < J.k_sub ? ((s & 1) ? J.dFa : J.dFb) : nullptr;
            for (int c = first; c < N; c += stride) relax_one(a, J.U, J.R, J.D, J.lamS, din, dout, fin, fout, J.F0, c);
            if (!grid_barrier(bar, expected, spin_limit)) return;
            double* t = din; din = dout; dout = t;
        }
        for (int c = first; c < N; c += stride) update_one(J.U, din, J.Wm, c);
        if (!grid_barrier(bar, expected, spin_limit)) return;
    }
}

// Co-resident CTAs of the persistent kernel on this device (0 if a
// cooperative launch is not possible).
static int persistent_capacity(gsis_ctx* c) {
    if (c->pers_grid != 0) return c->pers_grid;
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_macro_persistent, MACRO_PERSISTENT_THREADS, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    c->pers_grid = (coop && per_sm > 0) ? per_sm * sms : -1;
    return c->pers_grid;
}

// One cooperative launch for `steps` pseudo-steps; the barrier's error word
// is copied to c->h_err (read by the host after its next synchronisation).
static bool launch_macro_persistent(gsis_ctx* c, const MacroJob& J, bool stall) {
    const int cap = persistent_capacity(c);
    if (cap <= 0) return false;
    // every co-resident CTA: the phases are bound by the FP64 pipes of all SMs (a grid sized to the work
    // alone left SMs idle), capped where some CTAs would find no item in any phase
    const long long work = std::max<long long>((long long)J.a.N * J.ndir, J.a.N);
    const int grid = (int)std::min<long long>(cap, std::max<long long>(1, work / 32));
    cudaMemsetAsync(c->d_bar, 0, sizeof(GridBarrier), c->stream);
    MacroJob Jc = J;
    GridBarrier* bar = c->d_bar;
    unsigned long long spin = c->p.spin_limit;
    int st = stall ? 1 : 0;
    void* args[] = {&Jc, &bar, &spin, &st};
    if (cudaLaunchCooperativeKernel((const void*)k_macro_persistent, dim3(grid), dim3(MACRO_PERSISTENT_THREADS), args,
                                    0, c->stream) != cudaSuccess)
        return false;
    cudaMemcpyAsync(c->h_err, &c->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    c->launches++;
    return true;
}

// `steps` DP-LUR pseudo-steps on c->U / c->Wm (prim kept in step), HoT from
// c->hot, time term against c->Un when time_term.  Small meshes run the fused
// one-CTA kernel (one launch per block of steps), larger ones the persistent
// cooperative kernel (one launch per block of steps); inside a graph capture
// and where a cooperative launch is not available the per-phase kernels run
// over the whole grid.  Every path computes the same result.
void macro_block(gsis_ctx* c, int steps, bool with_hot, bool time_term, bool capturing) {
    (void)with_hot;
    const int N = c->m.N;
    if (steps <= 0) return;
    // automatic choice: the per-phase kernels above the fused kernel's limit (measured on the 16,384-cell
    // cylinder, 100 pseudo-steps: per-phase kernels 11.1 ms, persistent kernel 13.0 ms with one CTA on
    // each of 128 SMs and 23.8 ms with every co-resident CTA -- its 600 grid barriers cost more than
    // the launches they replace, the phases being bound by the FP64 special functions of the fluxes)
    int path = c->macro_path;
    if (path == MACRO_AUTO) path = N <= MACRO_FUSED_MAX_CELLS ? MACRO_FUSED : MACRO_MULTI;
    if (capturing && (path == MACRO_PERSISTENT || path == MACRO_PERSISTENT_STALL)) path = MACRO_MULTI;
    if (path == MACRO_FUSED) {
        MacroJob J = macro_job(c, steps, time_term);
        cudaMemcpyAsync(c->d_job, &J, sizeof(MacroJob), cudaMemcpyHostToDevice, c->stream);
        launch_macro_fused(c->d_job, 1, c->stream, fused_cluster_for(N));
        c->launches++;
        return;
    }
    if (path == MACRO_PERSISTENT || path == MACRO_PERSISTENT_STALL) {
        if (launch_macro_persistent(c, macro_job(c, steps, time_term), path == MACRO_PERSISTENT_STALL)) return;
        cudaGetLastError();   // no cooperative launch here: fall through to the per-phase kernels
    }
    const int TB = 64;
    const int nb = (N + TB - 1) / TB;
    const int ndir = c->normal_components;   // index directions that carry flux
    const int nf = (N * ndir + c->m.nbside + TB - 1) / TB;   // faces, then the boundary sides
    MacroArgs a = margs(c);
    const double dt = time_term ? c->p.dt : 0.0;
    for (int it = 0; it < steps; ++it) {
        launch_gradients(c, c->Wm, false);
        k_face_flux<<<nf, TB, 0, c->stream>>>(a, c->Wm, c->gu, c->gT, c->hot, c->acell, ndir, c->Ff, c->lamf,
                                               c->wall_corr, c->Fbnd);
        k_cell_residual<<<nb, TB, 0, c->stream>>>(a, c->Wm, c->U, c->Un, c->gu, c->gT, c->hot, c->Ff, c->lamf,
                                                  c->Fbnd, c->p.cfl, dt, c->R, c->D, c->lamS, c->dU, c->F0,
                                                  c->p.k_sub > 0 ? c->dFa : nullptr);
        c->launches += 2;
        double* din = c->dU;
        double* dout = c->dU2;
        for (int s = 0; s < c->p.k_sub; ++s) {
            double* fin = (s & 1) ? c->dFb : c->dFa;
            if (s + 1 < c->p.k_sub) {
                double* fout = (s & 1) ? c->dFa : c->dFb;
                k_relax<<<nb, TB, 0, c->stream>>>(a, c->U, c->R, c->D, c->lamS, din, dout, fin, fout, c->F0);
            } else {
                k_relax_update<<<nb, TB, 0, c->stream>>>(a, c->U, c->R, c->D, c->lamS, din, dout, fin, c->Wm);
            }
            c->launches++;
            double* t = din; din = dout; dout = t;
        }
        if (c->p.k_sub == 0) {
            k_update<<<nb, TB, 0, c->stream>>>(N, c->U, din, c->Wm);
            c->launches++;
        }
    }
}

// ---------------------------------------------------------------------------- residual epsilon
// Convergence criterion of Sec. 4: max over {rho, u (as a vector), T} of
// sqrt(sum (Wn - Wp)^2 vol / sum Wp^2 vol), quantities with a zero denominator
// left out.  out[0] = epsilon, out[1] = number of cells with non-finite or
// non-positive rho / T in Wn.
__global__ void k_eps(int N, const double* __restrict__ Wn, const double* __restrict__ Wp,
                      const double* __restrict__ vol, double* __restrict__ out) {
    __shared__ double sm[32 * 7];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const double V = vol[c];
        const double* a = Wn + c * 5;
        const double* b = Wp + c * 5;
        const double dr = a[0] - b[0];
        acc[0] += dr * dr * V;
        acc[1] += b[0] * b[0] * V;
        double du = 0.0, uu = 0.0;
        for (int i = 1; i < 4; ++i) { du += (a[i] - b[i]) * (a[i] - b[i]); uu += b[i] * b[i]; }
        acc[2] += du * V;
        acc[3] += uu * V;
        const double dT = a[4] - b[4];
        acc[4] += dT * dT * V;
        acc[5] += b[4] * b[4] * V;
        bool bad = !(a[0] > 0.0) || !(a[4] > 0.0) || !isfinite(a[0]) || !isfinite(a[4]);
        for (int i = 1; i < 4; ++i) bad = bad || !isfinite(a[i]);
        acc[6] += bad ? 1.0 : 0.0;
    }
    block_sum<7>(acc, sm);
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int q = 0; q < 3; ++q)
            if (acc[2 * q + 1] > 0.0) e = fmax(e, sqrt(acc[2 * q] / acc[2 * q + 1]));
        out[0] = e;
        out[1] = acc[6];
    }
}

void launch_eps(gsis_ctx* c, const double* Wn, const double* Wp) {
    k_eps<<<1, 1024, 0, c->stream>>>(c->m.N, Wn, Wp, c->m.vol, c->eps_buf);
    c->launches++;
}

}  // namespace gsis
