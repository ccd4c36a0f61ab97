// Host side of the batched persistent sweep: the candidate tile shapes, the
// grid size of each (resident CTAs per SM x SMs) and the launch.  The kernel
// is in batch_kernel.cuh, instantiated in batch_nc1.cu and batch_nc3.cu.
#include "batch_kernel.cuh"

namespace gsis {

// ---------------------------------------------------------------------------- candidates
struct TileShape {
    int vpt, cb, wpb;
    bool pair;   // velocity pairs with packed FP32 arithmetic (FP32/BF16/FP16 members with an even nx only)
    const char* name;
};

static const TileShape kShapes[] = {
    {1, 1, 4, false, "vpt1_cb1_w4"}, {2, 1, 4, false, "vpt2_cb1_w4"}, {4, 1, 4, false, "vpt4_cb1_w4"},
    {2, 1, 8, false, "vpt2_cb1_w8"}, {2, 2, 4, false, "vpt2_cb2_w4"}, {4, 2, 2, false, "vpt4_cb2_w2"},
    {1, 1, 4, true, "pair1_cb1_w4"}, {2, 1, 4, true, "pair2_cb1_w4"}, {1, 1, 8, true, "pair1_cb1_w8"},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int batch_num_shapes() { return kNumShapes; }
const char* batch_shape_name(int s) { return (s >= 0 && s < kNumShapes) ? kShapes[s].name : "?"; }
int batch_shape_vtile(int s) { return (kShapes[s].pair ? 64 : 32) * kShapes[s].vpt; }
bool batch_shape_pair(int s) { return s >= 0 && s < kNumShapes && kShapes[s].pair; }

int batch_grid(int shape, int nc) { return nc == 1 ? batch_grid_nc1(shape) : batch_grid_nc3(shape); }

// Steps pass0 .. pass1-1 of every item: step 0 is the backward pass, step 1 the forward pass.
void launch_sweep_batch(int shape, int nc, const BatchSolve* d_solves, const int2* d_items, int n_items,
                        int* d_ticket, int grid, cudaStream_t st, int pass0, int pass1) {
    cudaMemsetAsync(d_ticket, 0, sizeof(int), st);
    if (nc == 1)
        batch_launch_nc1(shape, d_solves, d_items, n_items, d_ticket, grid, st, pass0, pass1);
    else
        batch_launch_nc3(shape, d_solves, d_items, n_items, d_ticket, grid, st, pass0, pass1);
}

}  // namespace gsis
