// Batched persistent sweep kernels for meshes with one flux direction (1D) (see batch_kernel.cuh).
#include "batch_kernel.cuh"

namespace gsis {

void batch_launch_nc1(int shape, const BatchSolve* s, const int2* i, int n, int* t, int g, cudaStream_t st, int p0,
                      int p1) {
    launch_nc<1>(shape, s, i, n, t, g, st, p0, p1);
}

int batch_grid_nc1(int shape) { return grid_nc<1>(shape); }

}  // namespace gsis
