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
// Row factoring: a thread owns whole x-rows (fixed iy, iz) of the cell's VDF.
// Per point it accumulates only sum f c_x^k, k = 0..3 (c_x^k from shared
// memory), and folds the row sums into the 13 moments with the row constants
// c_y, c_z once per row.  In the correction pass the two corrected
// Maxwellians are evaluated with their y/z factors hoisted out of the row.
//
// Arithmetic type T: FP64 for an FP64 VDF; for FP32/BF16/FP16 storage the
// per-row work (row sums over at most nx <= 64 nodes, the correction) is
// FP32 and every sum across rows and cells is FP64.  The FP32 row sum of
// n terms carries a relative rounding error below n * 2^-24 (< 4e-6 for
// n = 64) of the sum of |terms|, far under the storage rounding of BF16/FP16
// (2^-9 / 2^-12 per value) and comparable to FP32 storage rounding.
#include "gsis_device.cuh"

namespace gsis {

template <typename S, typename T, bool CORRECT>
__global__ void __launch_bounds__(256) k_moments(int Nd, const int* __restrict__ dvm_cell,
                                                 const double* __restrict__ Wref, const int* __restrict__ side_bc,
                                                 const double* __restrict__ Sout, S* __restrict__ f, Records recNew,
                                                 Records recHalf, VGridDev vg, double* __restrict__ mom) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    extern __shared__ double sh_raw[];
    T* sh = reinterpret_cast<T*>(sh_raw);
    __shared__ double red[32 * MOMN];
    const int nx = vg.nx, ny = vg.ny, nz = vg.nz, NT = vg.NT;
    const int c = dvm_cell[k];
    const double ux = Wref[c * 5 + 1], uy = Wref[c * 5 + 2], uz = Wref[c * 5 + 3];
    T* scx = sh;                 // c_x, c_x^2, c_x^3
    T* scx2 = sh + nx;
    T* scx3 = sh + 2 * nx;
    T* tN = sh + 3 * nx;         // x-tables E, B, C2, R of M~(W^{n+1})
    T* tH = sh + 7 * nx;         // x-tables of M~(W^{n+1/2})
    const T* TN = CORRECT ? RecT<T>::tab(recNew, k, NT) : nullptr;
    const T* TH = CORRECT ? RecT<T>::tab(recHalf, k, NT) : nullptr;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double cx = vg.xi[i] - ux;
        scx[i] = (T)cx;
        scx2[i] = (T)(cx * cx);
        scx3[i] = (T)(cx * cx * cx);
        if (CORRECT) {
            tN[i] = TN[i]; tN[nx + i] = TN[NT + i]; tN[2 * nx + i] = TN[3 * NT + i]; tN[3 * nx + i] = TN[4 * NT + i];
            tH[i] = TH[i]; tH[nx + i] = TH[NT + i]; tH[2 * nx + i] = TH[3 * NT + i]; tH[3 * nx + i] = TH[4 * NT + i];
        }
    }
    __syncthreads();
    T p0N = T(0), p0H = T(0);
    if (CORRECT) {
        p0N = RecT<T>::scal(recNew, k)[RS_P0];
        p0H = RecT<T>::scal(recHalf, k)[RS_P0];
    }
    int wall_mask = 0;
    for (int s = 0; s < 6; ++s)
        if (side_bc[c * 6 + s] == GSIS_BC_WALL) wall_mask |= 1 << s;
    double acc[MOMN];
#pragma unroll
    for (int q = 0; q < MOMN; ++q) acc[q] = 0.0;
    S* fk = f + (long long)k * vg.Nv;
    const int rows = ny * nz;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int iy = r % ny, iz = r / ny;
        const int jy = nx + iy, jz = nx + ny + iz;
        const double xy = vg.xi[jy], xz = vg.xi[jz];
        const double cy = xy - uy, cz = xz - uz;
        T eN = T(0), bN = T(0), eH = T(0), bH = T(0);
        if (CORRECT) {
            eN = TN[jy] * TN[jz]; bN = TN[NT + jy] + TN[NT + jz];
            eH = TH[jy] * TH[jz]; bH = TH[NT + jy] + TH[NT + jz];
        }
        S* row = fk + (long long)r * nx;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        for (int ix = 0; ix < nx; ++ix) {
            T fv = ldT<T, S>(row + ix);
            if (CORRECT) {
                // the correction records are conservation-corrected Maxwellians: their
                // cubic (r.c) c^2 term is identically zero, so P = p0 + B
                const T vN = (tN[ix] * eN) * (p0N + (tN[nx + ix] + bN));
                const T vH = (tH[ix] * eH) * (p0H + (tH[nx + ix] + bH));
                stT<T, S>(row + ix, fv + (vN - vH));
                fv = ldT<T, S>(row + ix);   // moments of the stored value
            }
            s0 += fv;
            s1 += fv * scx[ix];
            s2 += fv * scx2[ix];
            s3 += fv * scx3[ix];
            if (wall_mask) {
#pragma unroll
                for (int s = 0; s < 6; ++s) {
                    if ((wall_mask >> s) & 1) {
                        const double* Sw = Sout + ((long long)c * 6 + s) * 3;
                        const double xn = vg.xi[ix] * Sw[0] + xy * Sw[1] + xz * Sw[2];
                        if (xn > 0.0) acc[13 + s] += xn * (double)fv;
                    }
                }
            }
        }
        const double d0 = s0, d1 = s1, d2 = s2, d3 = s3;
        const double t = cy * cy + cz * cz;
        acc[0] += d0;
        acc[1] += d1;
        acc[2] += d0 * cy;
        acc[3] += d0 * cz;
        acc[4] += d2;
        acc[5] += d0 * (cy * cy);
        acc[6] += d0 * (cz * cz);
        acc[7] += d1 * cy;
        acc[8] += d1 * cz;
        acc[9] += d0 * (cy * cz);
        acc[10] += d3 + d1 * t;
        acc[11] += cy * (d2 + d0 * t);
        acc[12] += cz * (d2 + d0 * t);
    }
    block_sum<MOMN>(acc, red);
    if (threadIdx.x == 0) {
        double* m = mom + (long long)k * MOMN;
        for (int q = 0; q < MOMN; ++q) m[q] = acc[q] * vg.w;
    }
}

// Diffuse-wall densities from the current VDF of each DVM wall cell:
// rho_w[k][s] = sum_{xi.S_s > 0} w (xi.S_s) f / wall_den[c][s].  Run between
// the forward and the backward pass, so that each pass emits from the wall
// with the latest outgoing half of f (the forward pass takes the values of
// the cell-equilibrium step, computed from f^n).  One block per DVM cell;
// cells without a wall side return at once.
template <typename S>
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
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const S* fk = f + (long long)k * vg.Nv;
    for (long long v = threadIdx.x; v < vg.Nv; v += blockDim.x) {
        int ix, iy, iz;
        vsplit(v, vg.nx, vg.ny, ix, iy, iz);
        const double x0 = vg.xi[ix], x1 = vg.xi[vg.nx + iy], x2 = vg.xi[vg.nx + vg.ny + iz];
        const double fv = Store<S>::ld(fk + v);
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            if ((wall_mask >> s) & 1) {
                const double* Sw = Sout + ((long long)c * 6 + s) * 3;
                const double xn = x0 * Sw[0] + x1 * Sw[1] + x2 * Sw[2];
                if (xn > 0.0) acc[s] += xn * fv;
            }
        }
    }
    block_sum<6>(acc, red);
    if (threadIdx.x == 0) {
        for (int s = 0; s < 6; ++s) {
            if ((wall_mask >> s) & 1) {
                const double v = acc[s] * vg.w / wall_den[c * 6 + s];
                rho_w[(long long)k * 6 + s] = v;
                if (rho_wf) rho_wf[(long long)k * 6 + s] = (float)v;
            }
        }
    }
}

void launch_wall_rho(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    if (Nd == 0 || !c->has_wall) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64:
            k_wall_rho<double><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout, (const double*)c->f,
                                                          c->vg, c->wall_den, c->rho_w, c->rho_wf);
            break;
        case GSIS_F32:
            k_wall_rho<float><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout, (const float*)c->f,
                                                         c->vg, c->wall_den, c->rho_w, c->rho_wf);
            break;
        case GSIS_BF16:
            k_wall_rho<__nv_bfloat16><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                                 (const __nv_bfloat16*)c->f, c->vg, c->wall_den,
                                                                 c->rho_w, c->rho_wf);
            break;
        default:
            k_wall_rho<__half><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                          (const __half*)c->f, c->vg, c->wall_den, c->rho_w,
                                                          c->rho_wf);
            break;
    }
    c->launches++;
}

template <typename S, typename T>
static void moments_t(gsis_ctx* c, const double* Wref, bool correct, double* out) {
    const int Nd = (int)c->Nd;
    const size_t smem = (size_t)(correct ? 11 : 3) * c->vg.nx * sizeof(T);
    if (correct)
        k_moments<S, T, true><<<Nd, 256, smem, c->stream>>>(Nd, c->dvm_cell, Wref, c->m.side_bc, c->m.Sout,
                                                             (S*)c->f, c->recNew, c->recHalf, c->vg, out);
    else
        k_moments<S, T, false><<<Nd, 256, smem, c->stream>>>(Nd, c->dvm_cell, Wref, c->m.side_bc, c->m.Sout,
                                                              (S*)c->f, c->recNew, c->recHalf, c->vg, out);
    c->launches++;
}

// correct_pass = 0: moments of f about Wref into `out`.
// correct_pass = 1: f += M~(W^{n+1}) - M~(W^{n+1/2}) (records recNew/recHalf),
//                   then moments of the corrected f about Wref into `out`.
void launch_moments(gsis_ctx* c, const double* Wref, int correct_pass, double* out) {
    if (c->Nd == 0) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64: moments_t<double, double>(c, Wref, correct_pass != 0, out); break;
        case GSIS_F32: moments_t<float, float>(c, Wref, correct_pass != 0, out); break;
        case GSIS_BF16: moments_t<__nv_bfloat16, float>(c, Wref, correct_pass != 0, out); break;
        default: moments_t<__half, float>(c, Wref, correct_pass != 0, out); break;
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
template <typename S>
__global__ void __launch_bounds__(256) k_wall_flux(int Nd, const int* __restrict__ dvm_cell,
                                                   const int* __restrict__ side_bc, const double* __restrict__ Sout,
                                                   const S* __restrict__ f, VGridDev vg,
                                                   const double* __restrict__ wall_den,
                                                   const double* __restrict__ wall_in, double* __restrict__ wall_kin) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    const int c = dvm_cell[k];
    __shared__ double sm[32 * 5];
    for (int s = 0; s < 6; ++s) {
        if (side_bc[c * 6 + s] != GSIS_BC_WALL) continue;
        const double* Sw = Sout + ((long long)c * 6 + s) * 3;
        const S* fk = f + (long long)k * vg.Nv;
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (long long v = threadIdx.x; v < vg.Nv; v += blockDim.x) {
            int ix, iy, iz;
            vsplit(v, vg.nx, vg.ny, ix, iy, iz);
            const double x0 = vg.xi[ix], x1 = vg.xi[vg.nx + iy], x2 = vg.xi[vg.nx + vg.ny + iz];
            const double xn = x0 * Sw[0] + x1 * Sw[1] + x2 * Sw[2];
            if (xn > 0.0) {
                const double g = xn * Store<S>::ld(fk + v);
                acc[0] += g;
                acc[1] += g * x0;
                acc[2] += g * x1;
                acc[3] += g * x2;
                acc[4] += g * 0.5 * (x0 * x0 + x1 * x1 + x2 * x2);
            }
        }
        block_sum<5>(acc, sm);
        if (threadIdx.x == 0) {
            const long long o = ((long long)c * 6 + s) * 5;
            const double rw = acc[0] * vg.w / wall_den[c * 6 + s];
            for (int q = 0; q < 5; ++q) wall_kin[o + q] = acc[q] * vg.w + rw * wall_in[o + q];
        }
    }
}

void launch_wall_flux(gsis_ctx* c) {
    const int Nd = (int)c->Nd;
    if (Nd == 0 || !c->has_wall) return;
    switch (c->p.vdf_dtype) {
        case GSIS_F64:
            k_wall_flux<double><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                            (const double*)c->f, c->vg, c->wall_den, c->wall_in,
                                                            c->wall_kin);
            break;
        case GSIS_F32:
            k_wall_flux<float><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                           (const float*)c->f, c->vg, c->wall_den, c->wall_in,
                                                           c->wall_kin);
            break;
        case GSIS_BF16:
            k_wall_flux<__nv_bfloat16><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                                   (const __nv_bfloat16*)c->f, c->vg, c->wall_den,
                                                                   c->wall_in, c->wall_kin);
            break;
        default:
            k_wall_flux<__half><<<Nd, 256, 0, c->stream>>>(Nd, c->dvm_cell, c->m.side_bc, c->m.Sout,
                                                            (const __half*)c->f, c->vg, c->wall_den, c->wall_in,
                                                            c->wall_kin);
            break;
    }
    c->launches++;
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

}  // namespace gsis
