// Measured arithmetic peaks of the current GPU: FP64 and FP32 fused
// multiply-add throughput of the CUDA cores, the denominators of the
// roofline of the FP64- and FP32-arithmetic kinetic sweeps.
//
// Every thread runs eight independent FMA chains (a <- a*b + c) for a given
// number of iterations; with eight CTAs of 256 threads per SM there are
// enough independent FMAs in flight to cover the pipeline latency of both
// precisions, so the launch is bound by the FMA issue rate.  b and c are
// kernel arguments and the chains end in a store the compiler cannot prove
// dead, so no FMA is removed.  flops = 2 per FMA.
#include <algorithm>
#include "gsis_device.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, T b, T c, T* __restrict__ out) {
    T a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == T(-1)) out[blockIdx.x] = s;   // never taken for the arguments used (all terms stay positive)
}

template <typename T>
gsis_status probe(cudaStream_t st, double* flops_per_s, double* ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return GSIS_ERR_CUDA;
    }
    const int grid = sms * 8;
    T* out = nullptr;   // never written (see the kernel); a valid address all the same
    if (cudaMalloc(&out, grid * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return GSIS_ERR_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T b = T(0.9999999), c = T(1e-7);
    // size the launch to about 40 ms from a short first run
    int iters = sizeof(T) == 8 ? 2000 : 100000;
    double best = 0.0, best_ms = 0.0;
    gsis_status status = GSIS_OK;
    for (int rep = 0; rep < 5 && status == GSIS_OK; ++rep) {
        cudaEventRecord(e0, st);
        k_fma_probe<T><<<grid, PROBE_THREADS, 0, st>>>(iters, b, c, out);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            status = GSIS_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * PROBE_CHAINS * (double)iters * grid * PROBE_THREADS;
        if (rep == 0) {   // calibration run
            iters = (int)std::min(2.0e9, std::max(1.0, iters * 40.0 / std::max(ms, 1e-3f)));
            continue;
        }
        const double rate = flops / (ms * 1e-3);
        if (rate > best) { best = rate; best_ms = ms; }
    }
    if (cudaGetLastError() != cudaSuccess) status = GSIS_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (status == GSIS_OK) {
        *flops_per_s = best;
        if (ms_out) *ms_out = best_ms;
    }
    return status;
}

}  // namespace

extern "C" gsis_status gsis_probe_fma_peak(int fp64, void* cuda_stream, double* flops_per_s, double* ms) {
    if (!flops_per_s) return GSIS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return fp64 ? probe<double>(st, flops_per_s, ms) : probe<float>(st, flops_per_s, ms);
}
