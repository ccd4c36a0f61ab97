// Allocation-free evaluation of conservation-corrected Maxwellian rows.
//
// For callers that must not allocate device memory themselves: hosts whose
// device memory is owned entirely by their own arena or pool and that forbid
// any other allocation, and latency-critical loops where a cudaMalloc (which
// may synchronise the device and take an unbounded time) is not acceptable.
// The caller passes the input states and the output rows; the intermediate
// distribution records live in one file-scope device array of fixed size,
// sized here once for every GPU that loads the library.
#include <algorithm>
#include <cmath>
#include <mutex>
#include "gsis_device.cuh"

namespace gsis {
void build_records_raw(const RecSpec* d_specs, int nrec, const Records& out, const VGridDev& vg, cudaStream_t st);
}

using namespace gsis;

namespace {

constexpr int NOALLOC_MAX_STATES = 256;   // rows per call
constexpr int NOALLOC_MAX_NODES = 384;    // nx + ny + nz
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t XI_BYTES = align256(NOALLOC_MAX_NODES * sizeof(double));
constexpr size_t SPEC_BYTES = align256(NOALLOC_MAX_STATES * sizeof(RecSpec));
constexpr size_t SCAL_BYTES = align256((size_t)NOALLOC_MAX_STATES * RS * sizeof(double));
constexpr size_t TAB_BYTES = align256((size_t)NOALLOC_MAX_STATES * NTAB * NOALLOC_MAX_NODES * sizeof(double));
constexpr size_t SCRATCH_BYTES = XI_BYTES + SPEC_BYTES + SCAL_BYTES + TAB_BYTES;   // about 3.9 MB

// Shared by every call on a device; its contents are whatever the last call left.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_addr[128] = {nullptr};   // device address of g_noalloc_scratch, per device ordinal

__global__ void k_noalloc_nodes(int nx, int ny, int nz, double lox, double loy, double loz, double hx, double hy,
                                double hz, double* xi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int NT = nx + ny + nz;
    if (i >= NT) return;
    if (i < nx) xi[i] = lox + (i + 0.5) * hx;
    else if (i < nx + ny) xi[i] = loy + (i - nx + 0.5) * hy;
    else xi[i] = loz + (i - nx - ny + 0.5) * hz;
}

__global__ void k_noalloc_specs(int n, const double* __restrict__ W, RecSpec* specs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* w = W + (long long)k * 5;
    RecSpec s;
    s.rho = w[0];
    s.T = w[4];
    for (int d = 0; d < 3; ++d) { s.u[d] = w[1 + d]; s.p[d] = 0.0; s.r[d] = 0.0; }
    for (int q = 0; q < 6; ++q) s.P2[q] = 0.0;
    s.p0 = 1.0;
    s.U[0] = w[0];
    for (int d = 0; d < 3; ++d) s.U[1 + d] = w[0] * w[1 + d];
    s.U[4] = w[0] * (1.5 * w[4] + 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
    s.correct = 1;
    specs[k] = s;
}

__global__ void k_noalloc_rows(int n, Records rec, VGridDev vg, double* __restrict__ out) {
    const int k = blockIdx.y;
    if (k >= n) return;
    const double* sc = rec_scal(rec, k);
    const double* tb = rec_tab(rec, k, vg.NT);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < vg.Nv;
         v += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        vsplit(v, vg.nx, vg.ny, ix, iy, iz);
        out[(long long)k * vg.Nv + v] = eval_rec(sc, tb, vg.NT, vg.nx, vg.ny, ix, iy, iz);
    }
}

// Device address of the scratch array on the current device (looked up once
// per device and cached for the life of the process; a cudaDeviceReset
// reloads the module and may move the array, so the cached address is only
// valid until the device is reset).
gsis_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return GSIS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return GSIS_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GSIS_OK;
}

}  // namespace

extern "C" gsis_status gsis_corrected_maxwellian_noalloc(const double* W, int n, const gsis_vgrid_desc* vgrid,
                                                         double* f_out, void* cuda_stream) {
    if (!W || !f_out || !vgrid || n < 0) return GSIS_ERR_ARG;
    if (n > NOALLOC_MAX_STATES) return GSIS_ERR_ARG;
    if (vgrid->reduced != 0) return GSIS_ERR_ARG;   // full 3D grids only
    // each axis is bounded before the node count is summed, so the sum cannot overflow
    long long Nv = 1, NTl = 0;
    for (int d = 0; d < 3; ++d) {
        if (vgrid->n[d] < 1 || vgrid->n[d] > NOALLOC_MAX_NODES) return GSIS_ERR_ARG;
        if (!(vgrid->hi[d] > vgrid->lo[d]) || !std::isfinite(vgrid->lo[d]) || !std::isfinite(vgrid->hi[d]))
            return GSIS_ERR_ARG;
        Nv *= vgrid->n[d];
        NTl += vgrid->n[d];
    }
    if (NTl > NOALLOC_MAX_NODES) return GSIS_ERR_ARG;
    const int NT = (int)NTl;
    if (n == 0) return GSIS_OK;
    // an error left by the caller's earlier asynchronous work is not this call's: leave it pending
    if (cudaPeekAtLastError() != cudaSuccess) return GSIS_ERR_CUDA;
    void* base = nullptr;
    gsis_status st = scratch_address(&base);
    if (st != GSIS_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* b = (unsigned char*)base;
    double* xi = (double*)b;
    RecSpec* specs = (RecSpec*)(b + XI_BYTES);
    Records rec;
    rec.scal = (double*)(b + XI_BYTES + SPEC_BYTES);
    rec.tab = (double*)(b + XI_BYTES + SPEC_BYTES + SCAL_BYTES);
    double h[3];
    double w = 1.0;
    for (int d = 0; d < 3; ++d) {
        h[d] = (vgrid->hi[d] - vgrid->lo[d]) / vgrid->n[d];
        w *= h[d];
    }
    VGridDev vg;
    vg.nx = vgrid->n[0];
    vg.ny = vgrid->n[1];
    vg.nz = vgrid->n[2];
    vg.NT = NT;
    vg.Nv = Nv;
    vg.w = w;
    vg.xi = xi;
    // Every scratch entry read below is written first in this call (nodes,
    // specs, record scalars and tables), so nothing needs clearing.  Each
    // launch is checked before the next one is queued.
    k_noalloc_nodes<<<(NT + 127) / 128, 128, 0, s>>>(vg.nx, vg.ny, vg.nz, vgrid->lo[0], vgrid->lo[1], vgrid->lo[2],
                                                     h[0], h[1], h[2], xi);
    if (cudaGetLastError() != cudaSuccess) return GSIS_ERR_CUDA;
    k_noalloc_specs<<<(n + 127) / 128, 128, 0, s>>>(n, W, specs);
    if (cudaGetLastError() != cudaSuccess) return GSIS_ERR_CUDA;
    build_records_raw(specs, n, rec, vg, s);
    if (cudaGetLastError() != cudaSuccess) return GSIS_ERR_CUDA;
    dim3 grid((unsigned)std::min<long long>((Nv + 255) / 256, 64), (unsigned)n);
    k_noalloc_rows<<<grid, 256, 0, s>>>(n, rec, vg, f_out);
    if (cudaGetLastError() != cudaSuccess) return GSIS_ERR_CUDA;
    return GSIS_OK;
}
