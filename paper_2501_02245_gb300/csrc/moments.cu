// Velocity-moment reductions (Eq. getmoment), high-order terms
// (Eq. full_constitutive) and the VDF correction of Eq. updatef.
//
// One block per DVM cell reduces over all discrete velocities in a fixed
// order (per-thread strided partial sums, then a warp-shuffle tree and a
// block tree), so results are bitwise reproducible.  Moments are taken about
// a reference velocity u_ref (the cell's current macroscopic velocity) to
// avoid cancellation:
//   m[0] = sum w f, m[1..3] = sum w c f, m[4..9] = sum w c_i c_j f
//   (xx, yy, zz, xy, xz, yz), m[10..12] = sum w c^2 c f,  c = xi - u_ref,
//   m[13+s] = sum_{xi.S_s > 0} w (xi.S_s) f for wall sides s (outgoing mass
//   flux through the wall face, for the diffuse-wall density).
#include "gsis_device.cuh"

namespace gsis {

template <typename S, bool CORRECT>
__global__ void __launch_bounds__(256) k_moments(int Nd, const int* __restrict__ dvm_cell,
                                                 const double* __restrict__ Wref, const int* __restrict__ side_bc,
                                                 const double* __restrict__ Sout, S* __restrict__ f, Records recNew,
                                                 Records recHalf, VGridDev vg, double* __restrict__ mom) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    __shared__ double sm[32 * MOMN];
    const int c = dvm_cell[k];
    const double ux = Wref[c * 5 + 1], uy = Wref[c * 5 + 2], uz = Wref[c * 5 + 3];
    const int NT = vg.NT, nx = vg.nx, ny = vg.ny;
    int wall_s[6];
    int nwall = 0;
    for (int s = 0; s < 6; ++s)
        if (side_bc[c * 6 + s] == GSIS_BC_WALL) wall_s[nwall++] = s;
    double acc[MOMN];
#pragma unroll
    for (int q = 0; q < MOMN; ++q) acc[q] = 0.0;
    S* fk = f + (long long)k * vg.Nv;
    const double* sN = CORRECT ? rec_scal(recNew, k) : nullptr;
    const double* tN = CORRECT ? rec_tab(recNew, k, NT) : nullptr;
    const double* sH = CORRECT ? rec_scal(recHalf, k) : nullptr;
    const double* tH = CORRECT ? rec_tab(recHalf, k, NT) : nullptr;
    for (long long v = threadIdx.x; v < vg.Nv; v += blockDim.x) {
        int ix, iy, iz;
        vsplit(v, nx, ny, ix, iy, iz);
        double fv = Store<S>::ld(fk + v);
        if (CORRECT) {
            fv = fv + (eval_rec(sN, tN, NT, nx, ny, ix, iy, iz) - eval_rec(sH, tH, NT, nx, ny, ix, iy, iz));
            Store<S>::st(fk + v, fv);
            fv = Store<S>::ld(fk + v);   // moments of the stored value
        }
        const double x0 = vg.xi[ix], x1 = vg.xi[nx + iy], x2 = vg.xi[nx + ny + iz];
        const double cx = x0 - ux, cy = x1 - uy, cz = x2 - uz;
        const double c2 = cx * cx + cy * cy + cz * cz;
        acc[0] += fv;
        acc[1] += fv * cx;
        acc[2] += fv * cy;
        acc[3] += fv * cz;
        acc[4] += fv * cx * cx;
        acc[5] += fv * cy * cy;
        acc[6] += fv * cz * cz;
        acc[7] += fv * cx * cy;
        acc[8] += fv * cx * cz;
        acc[9] += fv * cy * cz;
        acc[10] += fv * c2 * cx;
        acc[11] += fv * c2 * cy;
        acc[12] += fv * c2 * cz;
        for (int q = 0; q < nwall; ++q) {
            const double* Sw = Sout + ((long long)c * 6 + wall_s[q]) * 3;
            const double xn = x0 * Sw[0] + x1 * Sw[1] + x2 * Sw[2];
            if (xn > 0.0) acc[13 + q] += xn * fv;
        }
    }
    block_sum<MOMN>(acc, sm);
    if (threadIdx.x == 0) {
        double* m = mom + (long long)k * MOMN;
        for (int q = 0; q < 13; ++q) m[q] = acc[q] * vg.w;
        for (int s = 0; s < 6; ++s) m[13 + s] = 0.0;
        for (int q = 0; q < nwall; ++q) m[13 + wall_s[q]] = acc[13 + q] * vg.w;
    }
}

template <typename S>
static void moments_t(gsis_ctx* c, const double* Wref, bool correct, double* out) {
    const int Nd = (int)c->Nd;
    if (correct)
        k_moments<S, true><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, Wref, c->m.side_bc, c->m.Sout, (S*)c->f,
                                                       c->recNew, c->recHalf, c->vg, out);
    else
        k_moments<S, false><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, Wref, c->m.side_bc, c->m.Sout, (S*)c->f,
                                                        c->recNew, c->recHalf, c->vg, out);
    c->launches++;
}

// correct_pass = 0: moments of f about Wref into `out`.
// correct_pass = 1: f += M~(W^{n+1}) - M~(W^{n+1/2}) (records recNew/recHalf),
//                   then moments of the corrected f about Wref into `out`.
void launch_moments(gsis_ctx* c, const double* Wref, int correct_pass, double* out) {
    if (c->Nd == 0) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: moments_t<double>(c, Wref, correct_pass != 0, out); break;
        case GSIS_F32: moments_t<float>(c, Wref, correct_pass != 0, out); break;
        case GSIS_BF16: moments_t<__nv_bfloat16>(c, Wref, correct_pass != 0, out); break;
        default: moments_t<__half>(c, Wref, correct_pass != 0, out); break;
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

// HoT = kinetic - NSF(W^{n+1/2}) in DVM cells, zero in NS cells (Eq. full_constitutive).
__global__ void k_hot(int N, const int* __restrict__ cell2dvm, const double* __restrict__ kin,
                      const double* __restrict__ nsf, double* __restrict__ hot) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const bool dvm = cell2dvm[c] >= 0;
    for (int q = 0; q < HOTN; ++q)
        hot[(long long)c * HOTN + q] = dvm ? kin[(long long)c * HOTN + q] - nsf[(long long)c * HOTN + q] : 0.0;
}

void launch_hot(gsis_ctx* c) {
    const int N = c->m.N;
    k_hot<<<(N + 127) / 128, 128, 0, c->stream>>>(N, c->cell2dvm, c->kin, c->nsf, c->hot);
    c->launches++;
}

}  // namespace gsis
