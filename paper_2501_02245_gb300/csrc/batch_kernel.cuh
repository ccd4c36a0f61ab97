// Batched kinetic step: the sweeps of many independent solves (uneven meshes,
// velocity grids and VDF storage types) in ONE persistent launch.
//
// Work items are (solve, velocity tile) pairs.  Every dependency of the
// update at (cell, velocity) is on the same velocity, so one warp can take an
// item and run both Gauss-Seidel passes (one launch; with diffuse walls the
// passes are separate launches with the wall-density refresh between them)
// over all hyperplanes of its solve for
// its 32*VPT velocities on its own, with no barrier and no wait on any other
// warp: lane l only ever reads values that lane l itself wrote.  Warps draw
// items from a device ticket counter (atomicAdd), so long and short solves
// balance dynamically across the SMs; the host orders the items by decreasing
// cost.  The arithmetic is the single-solve sweep's own update (update_cells),
// so the result is identical to sweeping each solve alone.
//
// Tile shapes (velocities per thread VPT, cells per warp step CB, warps per
// CTA WPB) are template parameters; the host-side autotuner times the
// candidates listed here on the batch itself and keeps the fastest.
#pragma once
#include <algorithm>
#include "sweep_pair.cuh"

namespace gsis {

template <typename S, typename T, int NC, int VPT, int CB, bool FULL>
__device__ __forceinline__ void batch_item_t(const BatchSolve& B, int vtile, int lane, int pass0, int pass1) {
    const SweepArgs& a = B.a;
    Vel<T, VPT, FULL> V;
    make_vel(a.vg, (long long)vtile * (32 * VPT), lane, V);
    S* f = (S*)B.f;
    for (int step = pass0; step < pass1; ++step) {   // step 0: backward pass, step 1: forward pass
        const int pass = 1 - step;
        for (int hh = 0; hh < a.H; ++hh) {
            const int h = pass ? (a.H - 1 - hh) : hh;
            const int kb = __ldg(a.hp_off + h), ke = __ldg(a.hp_off + h + 1);
            const int n = ke - kb;
            for (int i0 = 0; i0 < n; i0 += CB) {
                int kk[CB];
                bool kon[CB];
#pragma unroll
                for (int b = 0; b < CB; ++b) {
                    const int i = i0 + b;
                    kon[b] = i < n;
                    kk[b] = pass ? (ke - 1 - i) : (kb + i);
                }
                update_cells<S, T, NC, VPT, CB>(a, f, kk, kon, V);
            }
        }
    }
}

template <typename S, typename T, int NC, int VPT, int CB>
__device__ __forceinline__ void batch_item(const BatchSolve& B, int vtile, int lane, int pass0, int pass1) {
    // tile inside the grid (warp-uniform); the 3-direction kernel (2D / 3D
    // members, rare in batches) keeps one variant to bound its compile time
    if constexpr (NC == 1) {
        if ((long long)(vtile + 1) * (32 * VPT) <= B.a.vg.Nv) {
            batch_item_t<S, T, NC, VPT, CB, true>(B, vtile, lane, pass0, pass1);
            return;
        }
    }
    batch_item_t<S, T, NC, VPT, CB, false>(B, vtile, lane, pass0, pass1);
}

template <int NC, int VPT, int CB, int WPB>
__global__ void __launch_bounds__(32 * WPB) k_sweep_batch(const BatchSolve* __restrict__ solves,
                                                          const int2* __restrict__ items, int n_items,
                                                          int* __restrict__ ticket, int pass0, int pass1) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_items) return;   // the counter only grows: every warp leaves after at most n_items draws
        const int2 it = items[t];
        const BatchSolve& B = solves[it.x];
        switch (B.dtype) {
            case GSIS_F64: batch_item<double, double, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
            case GSIS_F32: batch_item<float, float, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
            case GSIS_BF16: batch_item<__nv_bfloat16, float, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
            default: batch_item<__half, float, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
        }
    }
}

// The same persistent sweep on pairs of velocities (sweep_pair.cuh): items of
// 64 * VPT velocities, every member stored in FP32 / BF16 / FP16 with an even
// nx (the host offers these shapes only for such batches).
template <typename S, int NC, int VPT, int CB, bool FULL>
__device__ __forceinline__ void batch_item2_t(const BatchSolve& B, int vtile, int lane, int pass0, int pass1) {
    const SweepArgs& a = B.a;
    Vel2<VPT, FULL> V;
    make_vel2(a.vg, (long long)vtile * (64 * VPT), lane, V);
    S* f = (S*)B.f;
    for (int step = pass0; step < pass1; ++step) {
        const int pass = 1 - step;
        for (int hh = 0; hh < a.H; ++hh) {
            const int h = pass ? (a.H - 1 - hh) : hh;
            const int kb = __ldg(a.hp_off + h), ke = __ldg(a.hp_off + h + 1);
            const int n = ke - kb;
            for (int i0 = 0; i0 < n; i0 += CB) {
                int kk[CB];
                bool kon[CB];
#pragma unroll
                for (int b = 0; b < CB; ++b) {
                    const int i = i0 + b;
                    kon[b] = i < n;
                    kk[b] = pass ? (ke - 1 - i) : (kb + i);
                }
                update_cells2<S, NC, VPT, CB>(a, f, kk, kon, V);
            }
        }
    }
}

template <typename S, int NC, int VPT, int CB>
__device__ __forceinline__ void batch_item2(const BatchSolve& B, int vtile, int lane, int pass0, int pass1) {
    if constexpr (NC == 1) {
        if ((long long)(vtile + 1) * (64 * VPT) <= B.a.vg.Nv) {
            batch_item2_t<S, NC, VPT, CB, true>(B, vtile, lane, pass0, pass1);
            return;
        }
    }
    batch_item2_t<S, NC, VPT, CB, false>(B, vtile, lane, pass0, pass1);
}

template <int NC, int VPT, int CB, int WPB>
__global__ void __launch_bounds__(32 * WPB) k_sweep_batch2(const BatchSolve* __restrict__ solves,
                                                           const int2* __restrict__ items, int n_items,
                                                           int* __restrict__ ticket, int pass0, int pass1) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_items) return;
        const int2 it = items[t];
        const BatchSolve& B = solves[it.x];
        switch (B.dtype) {
            case GSIS_F32: batch_item2<float, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
            case GSIS_BF16: batch_item2<__nv_bfloat16, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
            case GSIS_F16: batch_item2<__half, NC, VPT, CB>(B, it.y, lane, pass0, pass1); break;
            default: break;   // FP64 members never reach the pair shapes
        }
    }
}

template <int NC, int VPT, int CB, int WPB>
static void launch_t2(const BatchSolve* d_solves, const int2* d_items, int n_items, int* d_ticket, int grid,
                      cudaStream_t st, int p0, int p1) {
    k_sweep_batch2<NC, VPT, CB, WPB><<<grid, 32 * WPB, 0, st>>>(d_solves, d_items, n_items, d_ticket, p0, p1);
}

template <int NC, int VPT, int CB, int WPB>
static int grid_t2() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_batch2<NC, VPT, CB, WPB>, 32 * WPB, 0);
    return std::max(1, sms * std::max(1, per));
}

template <int NC, int VPT, int CB, int WPB>
static void launch_t(const BatchSolve* d_solves, const int2* d_items, int n_items, int* d_ticket, int grid,
                     cudaStream_t st, int p0, int p1) {
    k_sweep_batch<NC, VPT, CB, WPB><<<grid, 32 * WPB, 0, st>>>(d_solves, d_items, n_items, d_ticket, p0, p1);
}

template <int NC, int VPT, int CB, int WPB>
static int grid_t() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_batch<NC, VPT, CB, WPB>, 32 * WPB, 0);
    return std::max(1, sms * std::max(1, per));
}

// One translation unit per mesh dimension class instantiates these.
template <int NC>
static void launch_nc(int shape, const BatchSolve* s, const int2* i, int n, int* t, int g, cudaStream_t st, int p0,
                      int p1) {
    switch (shape) {
        case 0: launch_t<NC, 1, 1, 4>(s, i, n, t, g, st, p0, p1); break;
        case 1: launch_t<NC, 2, 1, 4>(s, i, n, t, g, st, p0, p1); break;
        case 2: launch_t<NC, 4, 1, 4>(s, i, n, t, g, st, p0, p1); break;
        case 3: launch_t<NC, 2, 1, 8>(s, i, n, t, g, st, p0, p1); break;
        case 4: launch_t<NC, 2, 2, 4>(s, i, n, t, g, st, p0, p1); break;
        case 6: launch_t2<NC, 1, 1, 4>(s, i, n, t, g, st, p0, p1); break;
        case 7: launch_t2<NC, 2, 1, 4>(s, i, n, t, g, st, p0, p1); break;
        case 8: launch_t2<NC, 1, 1, 8>(s, i, n, t, g, st, p0, p1); break;
        default: launch_t<NC, 4, 2, 2>(s, i, n, t, g, st, p0, p1); break;
    }
}

template <int NC>
static int grid_nc(int shape) {
    switch (shape) {
        case 0: return grid_t<NC, 1, 1, 4>();
        case 1: return grid_t<NC, 2, 1, 4>();
        case 2: return grid_t<NC, 4, 1, 4>();
        case 3: return grid_t<NC, 2, 1, 8>();
        case 4: return grid_t<NC, 2, 2, 4>();
        case 6: return grid_t2<NC, 1, 1, 4>();
        case 7: return grid_t2<NC, 2, 1, 4>();
        case 8: return grid_t2<NC, 1, 1, 8>();
        default: return grid_t<NC, 4, 2, 2>();
    }
}

void batch_launch_nc1(int shape, const BatchSolve* s, const int2* i, int n, int* t, int g, cudaStream_t st, int p0,
                      int p1);
void batch_launch_nc3(int shape, const BatchSolve* s, const int2* i, int n, int* t, int g, cudaStream_t st, int p0,
                      int p1);
int batch_grid_nc1(int shape);
int batch_grid_nc3(int shape);

}  // namespace gsis
