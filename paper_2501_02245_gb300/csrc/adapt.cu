// Adaptation (Sec. 3.2, Sec. 3.4 Steps 2-3): gradient-length local Knudsen
// number (Eq. Kn_Gll), the DVM-region rule, forced wall layers, and the
// on-device compaction of the kinetic cells into a list sorted by hyperplane
// h = i + j + k (then by flat index), with the cell-indirection maps, the
// per-side connectivity the sweep needs, the Grad-13 ghost list and the remap
// of the VDF rows (survivors copied, entering cells seeded).
#include <algorithm>
#include <vector>
#include "gsis_device.cuh"

namespace gsis {

// Kn_Gll = lambda max(|grad rho|/rho, |grad U|/max(U, a), |grad T|/T),
// lambda = mu(T)/p sqrt(pi T/2) (the Kn definition of Sec. 2 with local
// values), a = sqrt(gamma T) keeps stagnation points finite.  flag = Kn_Gll >=
// Kn_ref, or the cell lies within wall_layers of a wall side.
__global__ void k_kn_gll(int N, int ni, int nj, int nk, const int* __restrict__ bc_type,
                         const double* __restrict__ Wp, const double* __restrict__ grho,
                         const double* __restrict__ gU, const double* __restrict__ gT, double mu0, double omega,
                         double Kn_ref, int wall_layers, double* __restrict__ kn, uint8_t* __restrict__ flag) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const double rho = Wp[c * 5], T = Wp[c * 5 + 4];
    const double ux = Wp[c * 5 + 1], uy = Wp[c * 5 + 2], uz = Wp[c * 5 + 3];
    const double U = sqrt(ux * ux + uy * uy + uz * uz);
    const double a = sqrt(GAMMA * T);
    const double lam = viscosity(T, mu0, omega) / (rho * T) * sqrt(PI * T / 2.0);
    auto nrm = [](const double* g) { return sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]); };
    const double r = fmax(fmax(nrm(grho + c * 3) / rho, nrm(gU + c * 3) / fmax(U, a)), nrm(gT + c * 3) / T);
    const double k = lam * r;
    kn[c] = k;
    bool f = k >= Kn_ref;
    if (wall_layers > 0) {
        const int idx[3] = {c % ni, (c / ni) % nj, c / (ni * nj)};
        const int n[3] = {ni, nj, nk};
        for (int d = 0; d < 3; ++d) {
            if (bc_type[2 * d] == GSIS_BC_WALL && idx[d] < wall_layers) f = true;
            if (bc_type[2 * d + 1] == GSIS_BC_WALL && n[d] - 1 - idx[d] < wall_layers) f = true;
        }
    }
    flag[c] = f ? 1 : 0;
}

void launch_kn_gll(gsis_ctx* c, const double* Wprim) {
    launch_gradients(c, Wprim, true);
    const int N = c->m.N;
    k_kn_gll<<<(N + 127) / 128, 128, 0, c->stream>>>(N, c->m.ni, c->m.nj, c->m.nk, c->d_bc_type, Wprim, c->grho,
                                                     c->gU, c->gT, c->mu0, c->p.omega, c->p.Kn_ref,
                                                     c->p.wall_layers, c->kn_gll, c->flag);
    c->launches++;
}

// ---------------------------------------------------------------------------- compaction
// Cells of hyperplane h in flat-index order: (k, j) lexicographic, i = h - j - k.
__device__ __forceinline__ int hp_cell(int h, int p, int ni, int nj, int nk) {
    const int j = p % nj, k = p / nj;
    const int i = h - j - k;
    if (i < 0 || i >= ni) return -1;
    return i + ni * (j + nj * k);
}

__global__ void k_hp_count(int ni, int nj, int nk, const uint8_t* __restrict__ flag, int* __restrict__ cnt) {
    const int h = blockIdx.x;
    __shared__ double sm[32];
    double acc[1] = {0.0};
    for (int p = threadIdx.x; p < nj * nk; p += blockDim.x) {
        const int c = hp_cell(h, p, ni, nj, nk);
        if (c >= 0 && flag[c]) acc[0] += 1.0;
    }
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) cnt[h] = (int)acc[0];
}

__global__ void k_hp_scan(int H, const int* __restrict__ cnt, int* __restrict__ off, int* __restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int s = 0;
    for (int h = 0; h < H; ++h) { off[h] = s; s += cnt[h]; }
    off[H] = s;
    total[0] = s;
}

// Ordered scatter of the flagged cells of hyperplane h (block-wide exclusive scan).
__global__ void k_hp_scatter(int ni, int nj, int nk, const uint8_t* __restrict__ flag, const int* __restrict__ off,
                             int* __restrict__ dvm_cell, int* __restrict__ cell2dvm) {
    const int h = blockIdx.x;
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = off[h];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p0 = 0; p0 < nj * nk; p0 += blockDim.x) {
        const int p = p0 + threadIdx.x;
        const int c = (p < nj * nk) ? hp_cell(h, p, ni, nj, nk) : -1;
        const int v = (c >= 0 && flag[c]) ? 1 : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        int wbase = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) wbase += warp_tot[w];
            tot += warp_tot[w];
        }
        if (v) {
            const int pos = base + wbase + x - 1;
            dvm_cell[pos] = c;
            cell2dvm[c] = pos;
        }
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
}

__global__ void k_fill_int(int n, int* a, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// NS cells with at least one DVM face neighbour receive a ghost record slot.
__global__ void k_ghost_mark(int N, const int* __restrict__ nbr, const int* __restrict__ cell2dvm,
                             int* __restrict__ ghost_id, int* __restrict__ ghost_cell, int* __restrict__ counter) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    ghost_id[c] = -1;
    if (cell2dvm[c] >= 0) return;
    bool need = false;
    for (int s = 0; s < 6; ++s) {
        const int n = nbr[c * 6 + s];
        if (n >= 0 && cell2dvm[n] >= 0) need = true;
    }
    if (need) {
        const int g = atomicAdd(counter, 1);
        ghost_id[c] = g;
        ghost_cell[g] = c;
    }
}

__global__ void k_dvm_sides(int Nd, const int* __restrict__ dvm_cell, const int* __restrict__ cell2dvm,
                            const int* __restrict__ nbr, const int* __restrict__ side_bc,
                            const double* __restrict__ Sout, const double* __restrict__ vol,
                            const int* __restrict__ ghost_id, int* __restrict__ kind, int* __restrict__ ref,
                            int* __restrict__ nb2, double* __restrict__ SoV, float* __restrict__ SoVf) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nd) return;
    const int c = dvm_cell[k];
    const double V = vol[c];
    for (int s = 0; s < 6; ++s) {
        const int n = nbr[c * 6 + s];
        int kd = SK_NONE, r = -1, r2 = -1;
        if (n >= 0) {
            const int kn = cell2dvm[n];
            if (kn >= 0) {
                kd = SK_DVM;
                r = kn;
                const int n2 = nbr[n * 6 + s];
                if (n2 >= 0 && cell2dvm[n2] >= 0) r2 = cell2dvm[n2];
            } else {
                kd = SK_GHOST;
                r = ghost_id[n];
            }
        } else {
            const int bc = side_bc[c * 6 + s];
            if (bc == GSIS_BC_FARFIELD) { kd = SK_FAR; r = s; }
            else if (bc == GSIS_BC_WALL) { kd = SK_WALL; r = s; }
        }
        kind[(long long)k * 6 + s] = kd;
        ref[(long long)k * 6 + s] = r;
        nb2[(long long)k * 6 + s] = r2;
        for (int i = 0; i < 3; ++i) {
            const double v = Sout[((long long)c * 6 + s) * 3 + i] / V;
            SoV[((long long)k * 6 + s) * 3 + i] = v;
            if (SoVf) SoVf[((long long)k * 6 + s) * 3 + i] = (float)v;
        }
    }
}

// Packed per-cell data of the sweep (layout in sweep_device.cuh) from the
// side lists: rows, second-neighbour rows (the neighbour's own row where a
// DVM side has none), side kinds with the all-DVM bit over the nc flux
// directions, and S/V component-major in the arithmetic type T.
template <typename T>
__global__ void k_sweep_desc(int Nd, int nc, const int* __restrict__ kind, const int* __restrict__ ref,
                             const int* __restrict__ nb2, const double* __restrict__ SoV, int* __restrict__ sdi,
                             T* __restrict__ sdv) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nd) return;
    int w[SD_INTS];
    for (int i = 0; i < SD_INTS; ++i) w[i] = 0;
    unsigned kinds = 0;
    bool interior = true;
    for (int s = 0; s < 6; ++s) {
        const int kd = kind[(long long)k * 6 + s], r = ref[(long long)k * 6 + s];
        int r2 = nb2[(long long)k * 6 + s];
        if (kd != SK_DVM || r2 < 0) r2 = r;
        if (s < 2 * nc && kd != SK_DVM) interior = false;
        kinds |= (unsigned)kd << (3 * s);
        if (s < 4) { w[s] = r; w[4 + s] = r2; }
        else { w[8 + (s - 4)] = r; w[10 + (s - 4)] = r2; }
    }
    w[12] = (int)(kinds | (interior ? 0x80000000u : 0u));
    for (int i = 0; i < SD_INTS; ++i) sdi[(long long)k * SD_INTS + i] = w[i];
    for (int q = 0; q < 3; ++q)
        for (int s = 0; s < 8; ++s)
            sdv[(long long)k * SD_VALS + 8 * q + s] = s < 6 ? (T)SoV[((long long)k * 6 + s) * 3 + q] : T(0);
}

__global__ void k_enter_mark(int Nd, const int* __restrict__ dvm_cell, const int* __restrict__ old_c2d,
                             int* __restrict__ enter_list, int* __restrict__ enter_of, int* __restrict__ counter) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nd) return;
    enter_of[k] = -1;
    if (old_c2d[dvm_cell[k]] < 0) {
        const int e = atomicAdd(counter, 1);
        enter_list[e] = k;
        enter_of[k] = e;
    }
}

template <typename S>
__global__ void k_remap(int Nd, const int* __restrict__ dvm_cell, const int* __restrict__ old_c2d,
                        const int* __restrict__ enter_of, const S* __restrict__ f_old, S* __restrict__ f_new,
                        Records seed, VGridDev vg) {
    const int k = blockIdx.x;
    if (k >= Nd) return;
    const int old = old_c2d[dvm_cell[k]];
    S* dst = f_new + (long long)k * vg.Nv;
    if (old >= 0) {
        const S* src = f_old + (long long)old * vg.Nv;
        for (long long v = threadIdx.x; v < vg.Nv; v += blockDim.x) dst[v] = src[v];
    } else {
        const int e = enter_of[k];
        const double* sc = rec_scal(seed, e);
        const double* tb = rec_tab(seed, e, vg.NT);
        for (long long v = threadIdx.x; v < vg.Nv; v += blockDim.x) {
            int ix, iy, iz;
            vsplit(v, vg.nx, vg.ny, ix, iy, iz);
            Store<S>::st(dst + v, vg.vscale * eval_rec(sc, tb, vg.NT, vg.nx, vg.ny, ix, iy, iz));
        }
    }
}

static bool ensure_dvm_capacity(gsis_ctx* c, long long Nd) {
    if (Nd <= c->cap_Nd && c->dvm_cell != nullptr) return true;
    long long cap = Nd > 0 ? Nd : 1;
    const int NT = c->vg.NT;
    dev_free(c, c->dvm_cell); dev_free(c, c->dside_kind); dev_free(c, c->dside_ref); dev_free(c, c->dside_nb2);
    dev_free(c, c->SoV); dev_free(c, c->itau); dev_free(c, c->mom); dev_free(c, c->momh); dev_free(c, c->rho_w);
    dev_free(c, c->recG.scal); dev_free(c, c->recG.tab); dev_free(c, c->recHalf.scal); dev_free(c, c->recHalf.tab);
    dev_free(c, c->recNew.scal); dev_free(c, c->recNew.tab); dev_free(c, c->enter_of);
    dev_free(c, c->SoVf); dev_free(c, c->itauf); dev_free(c, c->rho_wf);
    dev_free(c, c->sd_int); dev_free(c, c->sd_val);
    dev_free(c, c->gx4); dev_free(c, c->gx1); dev_free(c, c->gy4); dev_free(c, c->gy1);
    c->sd_int = nullptr; c->sd_val = nullptr;
    c->gx4 = c->gx1 = c->gy4 = c->gy1 = nullptr;
    dev_free(c, c->recG.tabf); dev_free(c, c->recG.scalf); dev_free(c, c->recHalf.tabf);
    dev_free(c, c->recHalf.scalf); dev_free(c, c->recNew.tabf); dev_free(c, c->recNew.scalf);
    c->SoVf = nullptr; c->itauf = nullptr; c->rho_wf = nullptr;
    c->recG.tabf = c->recHalf.tabf = c->recNew.tabf = nullptr;
    c->recG.scalf = c->recHalf.scalf = c->recNew.scalf = nullptr;
    c->dvm_cell = (int*)dev_alloc(c, cap * sizeof(int));
    c->dside_kind = (int*)dev_alloc(c, cap * 6 * sizeof(int));
    c->dside_ref = (int*)dev_alloc(c, cap * 6 * sizeof(int));
    c->dside_nb2 = (int*)dev_alloc(c, cap * 6 * sizeof(int));
    c->SoV = (double*)dev_alloc(c, cap * 18 * sizeof(double));
    c->itau = (double*)dev_alloc(c, cap * sizeof(double));
    c->mom = (double*)dev_alloc(c, cap * MOMN * sizeof(double));
    c->momh = (double*)dev_alloc(c, cap * MOMN * sizeof(double));
    c->rho_w = (double*)dev_alloc(c, cap * 6 * sizeof(double));
    c->recG.scal = (double*)dev_alloc(c, cap * RS * sizeof(double));
    c->recG.tab = (double*)dev_alloc(c, cap * NTAB * NT * sizeof(double));
    c->recHalf.scal = (double*)dev_alloc(c, cap * RS * sizeof(double));
    c->recHalf.tab = (double*)dev_alloc(c, cap * NTAB * NT * sizeof(double));
    c->recNew.scal = (double*)dev_alloc(c, cap * RS * sizeof(double));
    c->recNew.tab = (double*)dev_alloc(c, cap * NTAB * NT * sizeof(double));
    c->enter_of = (int*)dev_alloc(c, cap * sizeof(int));
    {   // sweep data in the sweep's arithmetic type
        const long long nyz = (long long)c->vg.ny * c->vg.nz;
        const size_t tb = c->p.vdf_dtype == GSIS_F64 ? sizeof(double) : sizeof(float);
        c->sd_int = (int*)dev_alloc(c, cap * SD_INTS * sizeof(int));
        c->sd_val = dev_alloc(c, cap * SD_VALS * tb);
        c->gx4 = dev_alloc(c, cap * c->vg.nx * 4 * tb);
        c->gx1 = dev_alloc(c, cap * c->vg.nx * tb);
        c->gy4 = dev_alloc(c, cap * nyz * 4 * tb);
        c->gy1 = dev_alloc(c, cap * nyz * tb);
        if (!c->sd_int || !c->sd_val || !c->gx4 || !c->gx1 || !c->gy4 || !c->gy1) return false;
    }
    if (c->p.vdf_dtype != GSIS_F64) {
        c->SoVf = (float*)dev_alloc(c, cap * 18 * sizeof(float));
        c->itauf = (float*)dev_alloc(c, cap * sizeof(float));
        c->rho_wf = (float*)dev_alloc(c, cap * 6 * sizeof(float));
        c->recG.tabf = (float*)dev_alloc(c, cap * NTAB * NT * sizeof(float));
        c->recG.scalf = (float*)dev_alloc(c, cap * RS * sizeof(float));
        c->recHalf.tabf = (float*)dev_alloc(c, cap * NTAB * NT * sizeof(float));
        c->recHalf.scalf = (float*)dev_alloc(c, cap * RS * sizeof(float));
        c->recNew.tabf = (float*)dev_alloc(c, cap * NTAB * NT * sizeof(float));
        c->recNew.scalf = (float*)dev_alloc(c, cap * RS * sizeof(float));
        if (!c->SoVf || !c->itauf || !c->rho_wf || !c->recG.tabf || !c->recG.scalf || !c->recHalf.tabf ||
            !c->recHalf.scalf || !c->recNew.tabf || !c->recNew.scalf)
            return false;
    }
    if (!c->dvm_cell || !c->dside_kind || !c->dside_ref || !c->dside_nb2 || !c->SoV || !c->itau || !c->mom ||
        !c->momh || !c->rho_w || !c->recG.scal || !c->recG.tab || !c->recHalf.scal || !c->recHalf.tab ||
        !c->recNew.scal || !c->recNew.tab || !c->enter_of)
        return false;
    c->cap_Nd = cap;
    return true;
}

// Build the DVM region from c->flag (already set), remap f.  Returns the new
// number of DVM cells, or -1 on failure (error recorded on the context).
int build_region(gsis_ctx* c) {
    const int N = c->m.N, H = c->m.H;
    const int nb = (N + 127) / 128;
    // keep the old indirection for the remap
    cudaMemcpyAsync(c->old_cell2dvm, c->cell2dvm, N * sizeof(int), cudaMemcpyDeviceToDevice, c->stream);
    k_hp_count<<<H, 256, 0, c->stream>>>(c->m.ni, c->m.nj, c->m.nk, c->flag, c->hp_cnt);
    k_hp_scan<<<1, 32, 0, c->stream>>>(H, c->hp_cnt, c->hp_off, c->d_count);
    c->launches += 2;
    cudaMemcpyAsync(c->h_count, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "region count")) return -1;
    const long long Nd_new = c->h_count[0];
    const long long Nd_old = c->Nd;
    void* f_old = c->f;
    // the old list is only needed through old_cell2dvm (cell -> old row)
    if (!ensure_dvm_capacity(c, Nd_new)) {
        set_err(c, GSIS_ERR_OOM, "allocation of the DVM lists failed");
        return -1;
    }
    const size_t eb = vdf_elem_bytes(c->p.vdf_dtype);
    void* f_new = nullptr;
    if (Nd_new > 0) {
        f_new = dev_alloc(c, (size_t)Nd_new * (size_t)c->vg.Nv * eb);
        if (!f_new) {
            set_err(c, GSIS_ERR_OOM, "allocation of the VDF array failed");
            return -1;
        }
    }
    k_fill_int<<<nb, 128, 0, c->stream>>>(N, c->cell2dvm, -1);
    k_hp_scatter<<<H, 256, 0, c->stream>>>(c->m.ni, c->m.nj, c->m.nk, c->flag, c->hp_off, c->dvm_cell, c->cell2dvm);
    cudaMemsetAsync(c->d_count, 0, 2 * sizeof(int), c->stream);
    k_ghost_mark<<<nb, 128, 0, c->stream>>>(N, c->m.nbr, c->cell2dvm, c->ghost_id, c->ghost_cell, c->d_count);
    c->launches += 3;
    if (Nd_new > 0) {
        const int kb = (int)((Nd_new + 127) / 128);
        k_dvm_sides<<<kb, 128, 0, c->stream>>>((int)Nd_new, c->dvm_cell, c->cell2dvm, c->m.nbr, c->m.side_bc,
                                               c->m.Sout, c->m.vol, c->ghost_id, c->dside_kind, c->dside_ref,
                                               c->dside_nb2, c->SoV, c->SoVf);
        if (c->p.vdf_dtype == GSIS_F64)
            k_sweep_desc<double><<<kb, 128, 0, c->stream>>>((int)Nd_new, c->normal_components, c->dside_kind,
                                                            c->dside_ref, c->dside_nb2, c->SoV, c->sd_int,
                                                            (double*)c->sd_val);
        else
            k_sweep_desc<float><<<kb, 128, 0, c->stream>>>((int)Nd_new, c->normal_components, c->dside_kind,
                                                           c->dside_ref, c->dside_nb2, c->SoV, c->sd_int,
                                                           (float*)c->sd_val);
        k_enter_mark<<<kb, 128, 0, c->stream>>>((int)Nd_new, c->dvm_cell, c->old_cell2dvm, c->enter_list,
                                                c->enter_of, c->d_count + 1);
        c->launches += 3;
    }
    cudaMemcpyAsync(c->h_count, c->d_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "region lists")) return -1;
    c->n_ghost = c->h_count[0];
    const int n_enter = c->h_count[1];
    c->Nd = Nd_new;
    {   // most DVM cells in one hyperplane (shared-memory window of the sweep)
        std::vector<int> off(H + 1);
        if (!cuda_ok(c, cudaMemcpy(off.data(), c->hp_off, (H + 1) * sizeof(int), cudaMemcpyDeviceToHost),
                     "hyperplane offsets"))
            return -1;
        int mx = 0;
        for (int h = 0; h < H; ++h) mx = std::max(mx, off[h + 1] - off[h]);
        c->max_hp = mx;
    }
    if (n_enter > 0) {
        const int grad13 = c->p.adaptive ? 1 : 0;
        if (grad13) launch_nsf(c, c->W, c->nsf);
        launch_seed_records(c, n_enter, grad13);
    }
    if (Nd_new > 0) {
        switch (c->p.vdf_dtype) {
            case GSIS_F64:
                k_remap<double><<<(unsigned)Nd_new, 256, 0, c->stream>>>((int)Nd_new, c->dvm_cell, c->old_cell2dvm,
                                                                         c->enter_of, (const double*)f_old,
                                                                         (double*)f_new, c->recNew, c->vg);
                break;
            case GSIS_F32:
                k_remap<float><<<(unsigned)Nd_new, 256, 0, c->stream>>>((int)Nd_new, c->dvm_cell, c->old_cell2dvm,
                                                                        c->enter_of, (const float*)f_old,
                                                                        (float*)f_new, c->recNew, c->vg);
                break;
            case GSIS_BF16:
                k_remap<__nv_bfloat16><<<(unsigned)Nd_new, 256, 0, c->stream>>>(
                    (int)Nd_new, c->dvm_cell, c->old_cell2dvm, c->enter_of, (const __nv_bfloat16*)f_old,
                    (__nv_bfloat16*)f_new, c->recNew, c->vg);
                break;
            default:
                k_remap<__half><<<(unsigned)Nd_new, 256, 0, c->stream>>>((int)Nd_new, c->dvm_cell, c->old_cell2dvm,
                                                                         c->enter_of, (const __half*)f_old,
                                                                         (__half*)f_new, c->recNew, c->vg);
                break;
        }
        c->launches++;
    }
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "region remap")) return -1;
    if (f_old) dev_free(c, f_old);
    c->f = f_new;
    (void)Nd_old;
    return (int)Nd_new;
}

}  // namespace gsis
