// Internal declarations of the GSIS library (not part of the public ABI).
//
// Device data layout (all FP64 unless stated):
//   mesh, per cell c (ncell = N):   vol[N], cen[N][3], hyper[N] (i+j+k, int)
//   mesh, per cell side s (0..5 = i-lo, i-hi, j-lo, j-hi, k-lo, k-hi):
//     nbr[N][6] (int, neighbour cell or -1), side_bc[N][6] (int),
//     Sout[N][6][3] (outward area vector), xf[N][6][3], lsq_w[N][6][3]
//   velocity grid: xi[NT] = x-nodes | y-nodes | z-nodes (NT = nx+ny+nz)
//   DVM list (compacted kinetic cells, sorted by hyperplane, then flat index):
//     dvm_cell[Nd] (int), cell2dvm[N] (int, -1 for NS cells), hp_off[H+1]
//     dside_kind[Nd][6], dside_ref[Nd][6], dside_nb2[Nd][6] (int)
//     SoV[Nd][6][3] = Sout/V of the DVM cell
//     f[Nd][Nv] in the storage type, velocity index innermost (x fastest)
//   distribution records (EqRec): scalar block [RS] + five axis tables [5][NT]
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/gsis.h"

namespace gsis {

constexpr int RS = 16;          // scalars per distribution record
constexpr int NTAB = 5;         // axis tables per record: E, B, C, C2, R
constexpr int MOMN = 19;        // 13 velocity moments + 6 wall half-range fluxes
constexpr int HOTN = 9;         // sigma xx,yy,zz,xy,xz,yz; q x,y,z
constexpr int FIELDS_N = 15;    // derived fields per cell: constitutive sigma (6), q (3), p; wall loads
constexpr int FIELD_WALL = 10;  // wall heat flux, pressure, shear x/y/z

// record scalar slots
enum { RS_P0 = 0, RS_P2XY = 1, RS_P2XZ = 2, RS_P2YZ = 3, RS_OFFD = 4, RS_UX = 5, RS_UY = 6, RS_UZ = 7,
       RS_ALPHA0 = 8 };

// DVM side kinds
enum { SK_NONE = 0, SK_DVM = 1, SK_GHOST = 2, SK_FAR = 3, SK_WALL = 4 };
// packed sweep data per DVM cell: integers and values (layout in sweep_device.cuh)
constexpr int SD_INTS = 16;
constexpr int SD_VALS = 24;

struct VGridDev {
    int nx, ny, nz, NT;
    long long Nv;
    double w;
    const double* xi;            // [NT]
    // 1: reduced distributions (xi_z integrated out): the z "nodes" are the
    // planes G (iz = 0) and H (iz = 1), their xi values are 0 (xi_z never
    // enters a face flux of a 2D mesh), and the xi_z^k weight of plane iz is
    // zpow(iz, k) (1 for G and k = 0, 1 for H and k = 2, else 0)
    int reduced = 0;
    // Storage scale of the VDF: stored value = vscale * f.  FP16 storage uses
    // 2^12 so that the Maxwellian tails that carry the heat flux stay above
    // FP16's subnormal range (its largest values, about 4 for a dense cold
    // cell, stay far below 65504); 1 for the other types.  The kinetic step
    // is linear in f: only its sources (g~/tau, boundary and interface
    // distributions) carry the scale; moments and wall sums divide it out.
    double vscale = 1.0;
};

// xi_z^k weight of z node iz for a moment: on a 3D grid the node value cz^k
// (cz = xi_z - u_z); on the reduced grid plane G carries k = 0 and plane H
// k = 2 (its values are int xi_z^2 f; odd powers vanish with u_z = 0).
__host__ __device__ __forceinline__ double zpow(const VGridDev& vg, int iz, double cz, int k) {
    if (vg.reduced) return (k == 0 && iz == 0) || (k == 2 && iz == 1) ? 1.0 : 0.0;
    double r = 1.0;
    for (int j = 0; j < k; ++j) r *= cz;
    return r;
}

struct Records {                 // R records
    double* scal;                // [R][RS]
    double* tab;                 // [R][NTAB][NT]
    float* tabf = nullptr;       // FP32 copy of tab (reduced-precision VDF storage only)
    float* scalf = nullptr;      // FP32 copy of scal
};

// Base polynomial of a record in c = xi - u:
//   p0 + p.c + c.P2.c + (r.c) c^2, optionally conservation-corrected to U.
struct RecSpec {
    double rho, u[3], T;         // Maxwellian factor
    double p0, p[3], P2[6], r[3];
    double U[5];                 // target conserved moments (rho, rho u, rho E)
    int correct;
};

struct Mesh {
    int ni = 0, nj = 0, nk = 0, dim = 0, N = 0, H = 0;
    int bc_type[6];
    double bc_state[6][5];
    double *vol = nullptr, *cen = nullptr, *Sout = nullptr, *xf = nullptr, *lsq_w = nullptr;
    int *nbr = nullptr, *side_bc = nullptr, *hyper = nullptr;
    int* bside = nullptr;   // far-field and wall sides, c * 6 + s (their fluxes are formed in the face phase)
    int nbside = 0;
};

struct Ctx;

// Mesh view of the synthetic solve.
struct MacroArgs {
    int N;
    const int* nbr;
    const int* side_bc;
    const double* Sout;
    const double* xf;
    const double* cen;
    const double* vol;
    const double* lsq_w;
    const double* bc_state;   // [6][5]
    const double* fgeo;       // [N][3][8] high face of each direction: |S|, n (3), e (3), distance of centres
    const double* bgeo;       // [N][6][8] each side: |S|, n (3), unit cell-to-face vector (3), its length
    const int* bside;         // [nbside] far-field and wall sides, c * 6 + s
    int nbside;
    int nd;                   // face normals have components 0..nd-1 only (normal_components)
    int fnd;                  // and cell-to-cell vectors and gradients too (face_nd; else 3)
    double mu0, omega;
};

// One block of pseudo-time steps of one solve, for the fused one-CTA kernel.
struct MacroJob {
    MacroArgs a;
    int steps, ndir, k_sub;
    double cfl, dt;
    double *Wm, *U;
    const double *Un, *hot, *wall_corr;
    double *gu, *gT, *Ff, *lamf, *R, *D, *lamS, *dU, *dU2, *acell;
    double *F0, *dFa, *dFb;   // Euler flux tensor of U and its changes for the relaxation increments [N][15]
    double* Fbnd;             // [N][6][6] boundary-side flux F.S_out (5) and lambda |S|
};

constexpr int MACRO_FUSED_THREADS = 512;
constexpr int MACRO_FUSED_MAX_CELLS = 4096;
constexpr int MACRO_PERSISTENT_THREADS = 256;

// Grid-wide barrier of the persistent synthetic-solve kernel: arrival count,
// generation, and an error word set by a block whose wait ran out of
// spin_limit iterations (then every block returns at its next barrier).
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

// Synthetic-solve implementation (gsis_debug_set_macro_path): AUTO picks the
// fused one-CTA kernel up to MACRO_FUSED_MAX_CELLS cells and the persistent
// cooperative kernel above (the per-phase kernels inside a batch graph).
enum { MACRO_AUTO = 0, MACRO_FUSED = 1, MACRO_MULTI = 2, MACRO_PERSISTENT = 3, MACRO_PERSISTENT_STALL = 4 };
}  // namespace gsis

struct gsis_ctx {
    gsis_params p{};
    gsis_allocator alloc{};
    bool have_alloc = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    bool broken = false;
    bool mesh_set = false, vgrid_set = false, started = false;
    std::vector<void*> allocations;
    double mu0 = 0.0;

    gsis::Mesh m;
    int normal_components = 3;     // 1: only x, 2: x and y, 3: x, y, z components of face normals are nonzero
    int face_nd = 3;               // normal_components when the LSQ gradients and the cell-to-cell vectors
                                   // have no other components either (mesh dim and cell centres), else 3
    bool has_wall = false;         // some boundary side is a diffuse wall
    double max_sv = 0.0;           // max over cells of sum_s |S_s| / V (set_mesh)
    double max_xi = 0.0;           // largest |velocity node| (set_velocity_grid)
    int* d_bc_type = nullptr;      // [6]
    double* d_bc_state = nullptr;  // [6][5]
    std::vector<double> host_W0;
    std::vector<uint8_t> forced_flags;
    bool have_forced = false;

    // velocity grid
    int nv3[3] = {0, 0, 0};
    double vlo[3], vhi[3];
    gsis::VGridDev vg{};
    double* d_xi = nullptr;

    // macro state
    double *W = nullptr, *Wh = nullptr, *Wp = nullptr, *Wm = nullptr, *U = nullptr, *Un = nullptr;
    double* Wmom = nullptr;        // [N][5] the state the moments of f^{n+1/2} (momh) were taken about
    double *dU = nullptr, *dU2 = nullptr, *R = nullptr, *D = nullptr, *lamS = nullptr;
    double* Fbnd = nullptr;                  // [N][6][6] boundary-side fluxes of the synthetic solve
    double *Ff = nullptr, *lamf = nullptr;   // interior face fluxes [N][3][5] and lambda|S| [N][3] (high faces)
    double *F0 = nullptr, *dFa = nullptr, *dFb = nullptr;   // [N][15] Euler flux tensor and its changes (relaxation)
    double *fgeo = nullptr, *bgeo = nullptr; // face geometry (see MacroArgs)
    double* acell = nullptr;                 // [N] sound speed of the current pseudo-time state
    double* fields = nullptr;                // [N][FIELDS_N] derived fields of gsis_moments
    double *gu = nullptr, *gT = nullptr, *grho = nullptr, *gU = nullptr;
    double *hot = nullptr, *kin = nullptr, *nsf = nullptr, *kn_gll = nullptr;
    double *eps_buf = nullptr, *h_eps = nullptr;
    gsis::GridBarrier* d_bar = nullptr;   // barrier of the persistent synthetic-solve kernel
    int* h_err = nullptr;          // pinned: barrier error word of the last persistent launch
    int macro_path = 0;            // gsis::MACRO_* (test hook; 0 = automatic)
    int pers_grid = 0;             // co-resident CTAs of the persistent kernel (0 = not queried yet)
    uint8_t* flag = nullptr;

    // DVM state
    long long Nd = 0, cap_Nd = 0;
    int *dvm_cell = nullptr, *cell2dvm = nullptr, *hp_off = nullptr, *hp_cnt = nullptr;
    int *dside_kind = nullptr, *dside_ref = nullptr, *dside_nb2 = nullptr;
    double* SoV = nullptr;
    float *SoVf = nullptr, *itauf = nullptr, *rho_wf = nullptr;   // FP32 mirrors for the FP32 sweep
    int* sd_int = nullptr;         // [Nd][SD_INTS] packed sweep data per DVM cell (k_sweep_desc)
    void* sd_val = nullptr;        // [Nd][SD_VALS] S/V of the sides, in the sweep's arithmetic type
    void *gx4 = nullptr, *gx1 = nullptr;   // [Nd][nx] x factor vectors of g~/tau (k_build_gtab)
    void *gy4 = nullptr, *gy1 = nullptr;   // [Nd][ny*nz] y-z factor vectors
    void* f = nullptr;
    double *itau = nullptr, *mom = nullptr, *rho_w = nullptr, *wall_den = nullptr;
    double *wall_in = nullptr;     // [N][6][5] incoming half-range moments of the wall Maxwellian
    double *wall_kin = nullptr;    // [N][6][5] kinetic wall flux of f^{n+1/2}
    double *wall_corr = nullptr;   // [N][6][5] kinetic minus NSF wall flux at W^{n+1/2} (0 for NS cells)
    gsis::Records recG{}, recHalf{}, recNew{}, recGhost{}, recBC{};
    int* ghost_id = nullptr;       // [N] ghost record index or -1
    int* ghost_cell = nullptr;     // [N] cell of each ghost record
    int n_ghost = 0;
    gsis::RecSpec* specs = nullptr;  // scratch, capacity N records
    double* momh = nullptr;        // [Nd][MOMN] moments of f^{n+1/2}
    int* old_cell2dvm = nullptr;   // [N] scratch for re-compaction
    int* enter_list = nullptr;     // [N] scratch: DVM indices entering the region
    int* enter_of = nullptr;       // [Nd] entering slot of each DVM cell or -1
    int* d_count = nullptr;        // scratch counters
    gsis::MacroJob* d_job = nullptr;   // device copy of this solve's fused macro job
    int sweep_shape = -1;          // autotuned sweep tile shape (-1: not tuned yet)
    int max_hp = 0;                // most DVM cells in one hyperplane (current region)
    bool sweep_forced = false;     // tile shape fixed by gsis_debug_set_sweep_tile
    long long tuned_Nd = -1;       // DVM cell count the shape was tuned for
    std::string sweep_info;        // tuning result, for gsis_tuning_info
    int* h_count = nullptr;

    // bookkeeping
    int iteration = 0;
    int presolve_blocks = 0;
    long long launches = 0, sweep_launches = 0;
    cudaEvent_t ev[2 * GSIS_NPHASE];
    bool events = false;
    double phase_ms[GSIS_NPHASE];
};

namespace gsis {

// ---------------------------------------------------------------------------- kernels (launchers)
// equilibrium.cu
void launch_build_records(gsis_ctx* c, const Records& out, int nrec, const RecSpec* d_specs);
void launch_cell_eq(gsis_ctx* c);
void launch_bc_records(gsis_ctx* c);
void launch_wall_den(gsis_ctx* c);
void launch_ghost_records(gsis_ctx* c);
void launch_correction_records(gsis_ctx* c);
void launch_seed_records(gsis_ctx* c, int n_enter, int grad13);
// Reference pair (g0, g1) of the two-VDF model for n states [n][12] (rho, u,
// T_t, T_r, q_t, q_r) into out[n][2][Nv]; specs [4n] and rec (4n records)
// are scratch of the caller.
struct TwoVdfGas { int d_r; double Zr; double A[4]; };
void launch_two_vdf_reference(gsis_ctx* c, const double* S, int n, const TwoVdfGas& g, RecSpec* specs,
                              const Records& rec, double* out);
// moments.cu: Eq. getmoment of n pairs F[n][2][Nv] into out[n][18]
void launch_two_vdf_moments(gsis_ctx* c, const double* F, int n, int d_r, double* out);
// sweep.cu
void launch_sweep(gsis_ctx* c, int pass);
gsis_status tune_sweep(gsis_ctx* c);
gsis_status force_sweep_shape(gsis_ctx* c, const char* name);
// sweep_ring.cu (shared-memory hyperplane window, 2D meshes)
struct SweepArgs;
size_t ring_bytes(gsis_ctx* c, int vt);
bool launch_sweep_ring(gsis_ctx* c, const SweepArgs& a, int pass, int which);
// batch.cu (persistent batched sweep; BatchSolve is declared in sweep_device.cuh)
struct BatchSolve;
int batch_num_shapes();
const char* batch_shape_name(int shape);
int batch_shape_vtile(int shape);
bool batch_shape_pair(int shape);
int batch_grid(int shape, int nc);
void launch_sweep_batch(int shape, int nc, const BatchSolve* d_solves, const int2* d_items, int n_items,
                        int* d_ticket, int grid, cudaStream_t st, int pass0, int pass1);
// moments.cu
void launch_moments(gsis_ctx* c, const double* Wref, double* out);
void launch_correct(gsis_ctx* c);
void launch_half_state(gsis_ctx* c);
void launch_hot(gsis_ctx* c);
void launch_wall_flux(gsis_ctx* c);
void launch_wall_rho(gsis_ctx* c);
void launch_wall_corr(gsis_ctx* c);
// macro.cu
void launch_gradients(gsis_ctx* c, const double* Wprim, bool with_rho_U);
void launch_nsf(gsis_ctx* c, const double* Wprim, double* out);
void launch_prim_to_cons(gsis_ctx* c, const double* Wprim, double* Ucons);
void launch_cons_to_prim(gsis_ctx* c, const double* Ucons, double* Wprim);
void launch_blend(gsis_ctx* c, const double* Wh, double w, double* W);
void launch_face_geometry(gsis_ctx* c);
// Derived per-cell fields of gsis_moments into c->fields: with wall, the wall
// loads (FIELD_WALL + heat flux, pressure, shear x/y/z); with cons, the
// constitutive stress and heat flux of Eq. full_constitutive and the pressure.
void launch_fields(gsis_ctx* c, bool wall, bool cons);
// capturing: the launches are being recorded into a CUDA graph (then the
// per-phase kernels replace the cooperative persistent launch)
void macro_block(gsis_ctx* c, int steps, bool with_hot, bool time_term, bool capturing = false);
MacroJob macro_job(gsis_ctx* c, int steps, bool time_term);
void launch_macro_fused(const MacroJob* d_jobs, int njobs, cudaStream_t stream, int cs);
int fused_cluster_size(int want);
int fused_cluster_for(int N);
void launch_eps(gsis_ctx* c, const double* Wn, const double* Wp);
// adapt.cu
void launch_kn_gll(gsis_ctx* c, const double* Wprim);
int  build_region(gsis_ctx* c);   // returns new Nd; builds lists and remaps f

// ---------------------------------------------------------------------------- host helpers
gsis_status set_err(gsis_ctx* c, gsis_status s, const std::string& msg);
void* dev_alloc(gsis_ctx* c, size_t bytes);
void dev_free(gsis_ctx* c, void* p);
size_t vdf_elem_bytes(int dtype);
bool cuda_ok(gsis_ctx* c, cudaError_t e, const char* what);

}  // namespace gsis

#define GSIS_LAUNCH_CHECK(ctx) do { (ctx)->launches++; } while (0)
