// Kinetic sweep with the hyperplane window staged in shared memory (2D meshes).
//
// The same Gauss-Seidel pass and the same per-point arithmetic as k_sweep
// (compute_cells), with a different memory schedule.  A block owns a tile of
// VT = 32*VPT velocities and walks the hyperplanes in pass order.  The update
// of hyperplane h reads hyperplanes h-2 .. h+2 (neighbours and second
// neighbours of a structured mesh lie one or two hyperplanes away), so the
// block keeps a ring of R = 7 hyperplane slots in shared memory: rows
// [cell of the hyperplane][VT velocities] in the storage type.  While it
// updates position t of the pass it already has t+1 .. t+3 in flight and
// issues the asynchronous copies (cp.async, 16 bytes per thread and copy)
// of position t+4 into the slot that held t-3.  Each VDF value is thus read
// from HBM once per pass and written once (the new value goes to the slot,
// for the hyperplanes after it, and to global memory); the global loads of
// the neighbour stencils, which made k_sweep latency bound, become shared
// loads.  Neighbours across a periodic seam are in far hyperplanes: they
// are read from global memory, which holds their latest value (the block
// stored every value it updated).
//
// Requirements (checked on the host): a 2D mesh (flux in two index
// directions), at most `maxc` DVM cells per hyperplane with
// R * maxc * VT * sizeof(storage) bytes of shared memory available, and
// 16-byte aligned velocity rows (N_v * sizeof(storage) a multiple of 16).
#include "sweep_device.cuh"

namespace gsis {

constexpr int RING = 7;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename S, typename T, int VPT, int NW>
__global__ void __launch_bounds__(32 * NW) k_sweep_ring(SweepArgs a, S* __restrict__ f, int pass, int maxc) {
    constexpr int NC = 2;
    constexpr int VT = 32 * VPT;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    S* ring = reinterpret_cast<S*>(sm_raw);   // [RING][maxc][VT]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long Nv = a.vg.Nv;
    const long long v0 = (long long)blockIdx.x * VT;
    const int vcount = (int)min((long long)VT, Nv - v0);
    const int chunks = vcount * (int)sizeof(S) / 16;   // 16-byte copies per row
    Vel<T, VPT> V;
    make_vel(a.vg, v0, lane, V);
    const int H = a.H;

    auto hyp = [&](int t) { return pass ? (H - 1 - t) : t; };
    auto issue = [&](int t) {   // copies of the rows of pass position t into its slot
        if (t < H) {
            const int h = hyp(t);
            const int kb = __ldg(a.hp_off + h), n = __ldg(a.hp_off + h + 1) - kb;
            S* slot = ring + (size_t)(t % RING) * maxc * VT;
            for (int q = threadIdx.x; q < n * chunks; q += 32 * NW) {
                const int r = q / chunks, c = q - r * chunks;
                cp_async16(reinterpret_cast<char*>(slot + (size_t)r * VT) + 16 * c,
                           reinterpret_cast<const char*>(f + (long long)(kb + r) * Nv + v0) + 16 * c);
            }
        }
        cp_async_commit();
    };
    for (int t = 0; t < 4; ++t) issue(t);

    for (int t = 0; t < H; ++t) {
        issue(t + 4);
        cp_async_wait<2>();   // positions up to t+2 have landed (t+3, t+4 may be in flight)
        __syncthreads();
        const int h = hyp(t);
        // hyperplane offsets h-2 .. h+3 (DVM rows of neighbour hyperplanes)
        int off[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int hq = h - 2 + q;
            off[q] = (hq >= 0 && hq <= H) ? __ldg(a.hp_off + hq) : (hq < 0 ? 0 : 0x7fffffff);
        }
        const int kb = off[2], n = off[3] - off[2];
        // ring slot of hyperplane h + dh (dh = -2..2), or nullptr if it is outside the window
        auto slot_of = [&](int dh) -> const S* {
            const int tt = t + (pass ? -dh : dh);
            if (tt < 0 || tt >= H) return nullptr;
            return ring + (size_t)(tt % RING) * maxc * VT;
        };
        for (int i = w; i < n; i += NW) {
            const int k = kb + i;
            CellMeta<T, NC> m[1];
            load_meta<T, NC>(a, k, m[0]);
            T fc[1][VPT], lo[1][NC][VPT], hi[1][NC][VPT], lo2[1][NC][VPT], hi2[1][NC][VPT];
            const S* own = ring + ((size_t)(t % RING) * maxc + i) * VT;
#pragma unroll
            for (int u = 0; u < VPT; ++u) fc[0][u] = V.on[u] ? ldT<T, S>(own + 32 * u + lane) : T(0);
            // value row of DVM row kn expected in hyperplane h + dh: shared slot, else global
            auto row_of = [&](int kn, int dh) -> const S* {
                const S* sl = slot_of(dh);
                if (sl && kn >= off[2 + dh] && kn < off[3 + dh]) return sl + (size_t)(kn - off[2 + dh]) * VT;
                return nullptr;
            };
#pragma unroll
            for (int d = 0; d < NC; ++d) {
                const bool dl = side_kind(m[0].kinds, 2 * d) == SK_DVM, dh_ = side_kind(m[0].kinds, 2 * d + 1) == SK_DVM;
                const bool dl2 = dl, dh2 = dh_;   // (a missing second neighbour repeats the neighbour's row)
                const S* sl = dl ? row_of(m[0].rf[2 * d], -1) : nullptr;
                const S* sh = dh_ ? row_of(m[0].rf[2 * d + 1], 1) : nullptr;
                const S* sl2 = dl2 ? row_of(m[0].n2[2 * d], -2) : nullptr;
                const S* sh2 = dh2 ? row_of(m[0].n2[2 * d + 1], 2) : nullptr;
                const S* gl = f + (long long)m[0].rf[2 * d] * Nv + v0;
                const S* gh = f + (long long)m[0].rf[2 * d + 1] * Nv + v0;
                const S* gl2 = f + (long long)m[0].n2[2 * d] * Nv + v0;
                const S* gh2 = f + (long long)m[0].n2[2 * d + 1] * Nv + v0;
#pragma unroll
                for (int u = 0; u < VPT; ++u) {
                    const bool on = V.on[u];
                    const int j = 32 * u + lane;
                    lo[0][d][u] = (dl && on) ? (sl ? ldT<T, S>(sl + j) : ldT<T, S>(gl + j)) : fc[0][u];
                    hi[0][d][u] = (dh_ && on) ? (sh ? ldT<T, S>(sh + j) : ldT<T, S>(gh + j)) : fc[0][u];
                    lo2[0][d][u] = (dl2 && on) ? (sl2 ? ldT<T, S>(sl2 + j) : ldT<T, S>(gl2 + j)) : lo[0][d][u];
                    hi2[0][d][u] = (dh2 && on) ? (sh2 ? ldT<T, S>(sh2 + j) : ldT<T, S>(gh2 + j)) : hi[0][d][u];
                }
            }
            const int kk[1] = {k};
            const bool kon[1] = {true};
            T fo[1][VPT];
            compute_cells<T, NC, VPT, 1, false>(a, kk, kon, V, m, fc, lo, hi, lo2, hi2, fo);
            S* orow = const_cast<S*>(own);
            S* grow = f + (long long)k * Nv + v0;
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                if (!V.on[u]) continue;
                stT<T, S>(orow + 32 * u + lane, fo[0][u]);
                stT<T, S>(grow + 32 * u + lane, fo[0][u]);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------- host side
template <typename S, typename T, int VPT, int NW>
static bool ring_t(gsis_ctx* c, const SweepArgs& a, int pass, int maxc) {
    constexpr int VT = 32 * VPT;
    const size_t bytes = (size_t)RING * maxc * VT * sizeof(S);
    static int configured = 0;   // per instantiation: the largest dynamic size set so far
    if ((int)bytes > configured) {
        if (cudaFuncSetAttribute(k_sweep_ring<S, T, VPT, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        configured = (int)bytes;
    }
    const unsigned blocks = (unsigned)((c->vg.Nv + VT - 1) / VT);
    k_sweep_ring<S, T, VPT, NW><<<blocks, 32 * NW, bytes, c->stream>>>(a, (S*)c->f, pass, maxc);
    return true;
}

// Shared memory the ring sweep needs for velocity tile vt (0 if it cannot run).
size_t ring_bytes(gsis_ctx* c, int vt) {
    const size_t eb = vdf_elem_bytes(c->p.vdf_dtype);
    if (c->normal_components != 2 || c->max_hp <= 0) return 0;
    if ((c->vg.Nv * eb) % 16 != 0 || (vt * eb) % 16 != 0) return 0;
    const size_t bytes = (size_t)RING * c->max_hp * vt * eb;
    return bytes <= 220 * 1024 ? bytes : 0;
}

// Launch the ring sweep with shape index `which` (0: 8 warps x 32 velocities,
// 1: 4 warps x 32 velocities, 2: 8 warps x 64 velocities); false if the
// problem does not fit it.
bool launch_sweep_ring(gsis_ctx* c, const SweepArgs& a, int pass, int which) {
    const int vt = which == 2 ? 64 : 32;
    if (ring_bytes(c, vt) == 0) return false;
    const int maxc = c->max_hp;
    switch (c->p.vdf_dtype) {
        case GSIS_F64:
            if (which == 2) return false;
            return which == 1 ? ring_t<double, double, 1, 4>(c, a, pass, maxc) : ring_t<double, double, 1, 8>(c, a, pass, maxc);
        case GSIS_F32:
            return which == 2 ? ring_t<float, float, 2, 8>(c, a, pass, maxc)
                              : (which == 1 ? ring_t<float, float, 1, 4>(c, a, pass, maxc)
                                            : ring_t<float, float, 1, 8>(c, a, pass, maxc));
        case GSIS_BF16:
            return which == 2 ? ring_t<__nv_bfloat16, float, 2, 8>(c, a, pass, maxc)
                              : (which == 1 ? ring_t<__nv_bfloat16, float, 1, 4>(c, a, pass, maxc)
                                            : ring_t<__nv_bfloat16, float, 1, 8>(c, a, pass, maxc));
        default:
            return which == 2 ? ring_t<__half, float, 2, 8>(c, a, pass, maxc)
                              : (which == 1 ? ring_t<__half, float, 1, 4>(c, a, pass, maxc)
                                            : ring_t<__half, float, 1, 8>(c, a, pass, maxc));
    }
}

}  // namespace gsis
