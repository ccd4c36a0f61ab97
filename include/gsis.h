/*
 * gsis.h -- C ABI of the GB300 (sm_103a) adaptive GSIS kinetic hot path.
 *
 * The library implements one iteration of the adaptive general synthetic
 * iterative scheme of Zhang, Zeng & Wu (arXiv 2501.02245) for a monatomic gas
 * (the d_r = 0 reduction of the model of Sec. 2, i.e. the Shakhov model with
 * Pr = 2/3) on a structured finite-volume mesh and a uniform discrete velocity
 * grid, restricted to a compacted list of kinetic (DVM) cells:
 *
 *   reference distribution  (Sec. 2, Eq. general_model and the g_0t formula)
 *   implicit upwind kinetic step           (Sec. 3.1, first equation)
 *   velocity moments + high-order terms    (Eq. getmoment, Eq. full_constitutive)
 *   macroscopic synthetic solve            (Eq. macro with Eq. NSF_constitutive)
 *   VDF correction                         (Eq. updatef)
 *   convergence criterion                  (Sec. 4, Eq. convergence_critertion)
 *   adaptation + Grad-13 reconstruction    (Sec. 3.2, Eq. Kn_Gll, Eq. G13_VDF;
 *                                           Sec. 3.4 Steps 1-3)
 *
 * Conventions
 *  - Every function returns gsis_status; no C++ exception crosses the ABI.
 *  - Non-dimensional units: R = 1, free-stream rho = T = 1; p = rho T.
 *  - Host pointers passed in are read during the call and copied; the caller
 *    keeps ownership.  The library owns all device memory it allocates,
 *    through the gsis_allocator callbacks when given, else cudaMalloc.
 *  - All device work of a context runs on the cuda stream given to gsis_init
 *    (NULL = the legacy default stream).  Calls on one context are not
 *    thread-safe; distinct contexts are independent.
 *  - On GSIS_ERR_ARG the context state is unchanged.  After GSIS_ERR_CUDA,
 *    GSIS_ERR_NONFINITE or GSIS_ERR_INTERNAL the context only accepts
 *    gsis_free, gsis_last_error and gsis_moments.
 */
#ifndef GSIS_H
#define GSIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSIS_OK = 0,
    GSIS_ERR_ARG = 1,          /* invalid argument or descriptor             */
    GSIS_ERR_STATE = 2,        /* call not allowed in the current state      */
    GSIS_ERR_OOM = 3,          /* allocation failed (callback returned NULL) */
    GSIS_ERR_CUDA = 4,         /* a CUDA runtime call failed                 */
    GSIS_ERR_NONFINITE = 5,    /* non-finite or non-positive rho/T detected  */
    GSIS_ERR_TIMEOUT = 6,      /* a bounded device wait ran out              */
    GSIS_ERR_UNSUPPORTED = 7,  /* valid but not implemented combination      */
    GSIS_ERR_INTERNAL = 8      /* device-side consistency check failed       */
} gsis_status;

/* VDF storage types (arithmetic: FP64 for GSIS_F64, FP32 otherwise; moments,
 * conservation correction and the synthetic solve are FP64 always). */
enum { GSIS_F64 = 0, GSIS_F32 = 1, GSIS_BF16 = 2, GSIS_F16 = 3 };

/* Boundary side types. */
enum { GSIS_BC_NONE = 0, GSIS_BC_FARFIELD = 1, GSIS_BC_WALL = 2, GSIS_BC_PERIODIC = 3 };

/* Fields returned by gsis_moments, one bit each; values are written per cell
 * in this order for the bits that are set. */
enum {
    GSIS_FIELD_RHO = 1 << 0, GSIS_FIELD_UX = 1 << 1, GSIS_FIELD_UY = 1 << 2, GSIS_FIELD_UZ = 1 << 3,
    GSIS_FIELD_T = 1 << 4,
    GSIS_FIELD_HOT_SXX = 1 << 5, GSIS_FIELD_HOT_SYY = 1 << 6, GSIS_FIELD_HOT_SZZ = 1 << 7,
    GSIS_FIELD_HOT_SXY = 1 << 8, GSIS_FIELD_HOT_SXZ = 1 << 9, GSIS_FIELD_HOT_SYZ = 1 << 10,
    GSIS_FIELD_HOT_QX = 1 << 11, GSIS_FIELD_HOT_QY = 1 << 12, GSIS_FIELD_HOT_QZ = 1 << 13,
    GSIS_FIELD_KN_GLL = 1 << 14, GSIS_FIELD_DVM = 1 << 15,
    GSIS_FIELD_WALL_Q = 1 << 16,   /* heat flux into the wall, per unit area (0 off the wall) */
    /* Eq. full_constitutive at the current state: sigma = sigma_NSF(W) + HoT_sigma, q = q_NSF(W) + HoT_q,
     * HoT of the last iteration (0 in NS cells) -- equal to the kinetic moments at a converged state */
    GSIS_FIELD_SXX = 1 << 17, GSIS_FIELD_SYY = 1 << 18, GSIS_FIELD_SZZ = 1 << 19,
    GSIS_FIELD_SXY = 1 << 20, GSIS_FIELD_SXZ = 1 << 21, GSIS_FIELD_SYZ = 1 << 22,
    GSIS_FIELD_QX = 1 << 23, GSIS_FIELD_QY = 1 << 24, GSIS_FIELD_QZ = 1 << 25,
    GSIS_FIELD_P = 1 << 26,        /* pressure rho T */
    /* force of the gas on the wall per unit wall area (0 off the wall): normal component (pressure) and
     * tangential vector (shear); from the same wall fluxes as GSIS_FIELD_WALL_Q */
    GSIS_FIELD_WALL_P = 1 << 27, GSIS_FIELD_WALL_TX = 1 << 28, GSIS_FIELD_WALL_TY = 1 << 29,
    GSIS_FIELD_WALL_TZ = 1 << 30,
    GSIS_NFIELDS = 31
};

/* Device-memory callbacks (for example a framework's caching allocator).
 * alloc must return memory aligned to at least 256 bytes, or NULL on failure
 * (reported as GSIS_ERR_OOM).  free(NULL) is never called. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void  (*free)(void* p, void* stream, void* user);
    void* user;
} gsis_allocator;

/* Run parameters. */
typedef struct {
    double Kn;            /* free-stream Knudsen number; mu(T0) from the Kn definition of Sec. 2 */
    double omega;         /* viscosity index: mu = mu(T0) (T/T0)^omega (Sec. 2)                  */
    int    adaptive;      /* 1: Sec. 3.4 Steps 2-3 (Kn_Gll region, re-identification); 0: all cells DVM */
    double Kn_ref;        /* reference Knudsen number of the DVM-region rule (Sec. 3.2)           */
    int    adapt_every;   /* the region is re-identified once, after this many GSIS iterations    */
    int    wall_layers;   /* cell layers next to a wall that are always DVM                        */
    int    vdf_dtype;     /* GSIS_F64 / GSIS_F32 / GSIS_BF16 / GSIS_F16                            */
    int    macro_steps;   /* pseudo-time steps of the synthetic solve per GSIS iteration           */
    double cfl;           /* pseudo-time CFL number of the synthetic solve                         */
    int    k_sub;         /* Jacobi sweeps of the data-parallel relaxation per pseudo-step         */
    double dt;            /* time step of Eq. macro; 0 = steady form (dt -> infinity)              */
    double tol;           /* convergence tolerance on epsilon (Sec. 4), also for the NS presolve   */
    int    presolve_max_blocks; /* Sec. 3.4 Step 1 NS presolve (HoT = 0): at most this many blocks of
                                   macro_steps steps, stopping when epsilon between blocks < tol;
                                   0 = start from W0 directly                                     */
    unsigned long long spin_limit; /* polls (about 32 ns apart) of any device-side wait before it gives
                                      up with GSIS_ERR_TIMEOUT: the grid barriers of the persistent
                                      synthetic-solve kernel (GSIS_MACRO_PERSISTENT);
                                      0 = default 2^24 (about a second)                              */
    double relax;         /* weight of the synthetic correction: W^{n+1} = W^{n+1/2} + relax *
                             (W_synthetic - W^{n+1/2}); 1 = the plain scheme, (0, 1]; 0 is read as 1 */
    int    d_r;           /* internal degrees of freedom of the gas (Sec. 2, Eq. general_model): 0 = monatomic,
                             the Shakhov model with Pr = 2/3, the only form implemented; d_r > 0 (the
                             two-VDF model, f_0 and f_1) returns GSIS_ERR_UNSUPPORTED, d_r < 0 GSIS_ERR_ARG */
    double Z_r;           /* internal collision number of Eq. general_model (read only when d_r > 0)         */
    double A[4];          /* heat-flux relaxation rates A_tt, A_tr, A_rt, A_rr of Eq. mu_kappa and the q_0/q_1
                             mixing (read only when d_r > 0)                                               */
} gsis_params;

/* Structured mesh: cells (i, j, k), flat index c = i + ni*(j + nj*k).
 * centers [ncell][3], volumes [ncell]; for direction d the faces normal to it:
 * S[d] and xf[d] of shape [nk'][nj'][ni'][3] with one extra face along d
 * (area vector pointing along +d, magnitude = area; face centre).  In a
 * periodic direction the face between the last and the first cell is face 0.
 * A periodic direction is taken as geometrically continuous (the angular
 * direction of an O-grid): the line of centres and the least-squares vectors
 * across its wrap are the plain differences of the given cell centres, so a
 * direction whose wrap is a translation (a periodic box) gets the distance
 * across the whole domain there.
 * bc_type/bc_state per side (i-lo, i-hi, j-lo, j-hi, k-lo, k-hi); bc_state is
 * (rho, ux, uy, uz, T) for a far field, T at index 4 is the wall temperature
 * for a wall.  W0 [ncell][5] is the initial (rho, ux, uy, uz, T).
 * Errors: GSIS_ERR_ARG for non-positive sizes or volumes, a periodic
 * direction with fewer than 3 cells, inconsistent periodic sides, non-finite
 * input or non-positive rho/T; GSIS_ERR_UNSUPPORTED when the velocity grid is
 * set and the mesh's largest sum_s |S_s|/V times max|xi| exceeds 2^100 (see
 * gsis_set_velocity_grid); GSIS_ERR_STATE after the first gsis_iterate. */
typedef struct {
    int ni, nj, nk;
    int dim;                    /* spatial directions carrying gradients (1, 2 or 3) */
    const double* centers;
    const double* volumes;
    const double* S[3];
    const double* xf[3];
    int    bc_type[6];
    double bc_state[6][5];
    const double* W0;
} gsis_mesh_desc;

/* Uniform midpoint velocity grid (Sec. 4.2: uniform discretisation of a
 * truncated box): n[d] nodes on [lo[d], hi[d]], node k at lo+(k+1/2)(hi-lo)/n,
 * weight prod_d (hi-lo)/n; flat index v = ix + nx*(iy + ny*iz).
 * reduced = 1 (2D flows, Sec. 3.3 and the 2D velocity grid of Sec. 4.2): the
 * xi_z direction is integrated out and the VDF of a cell is stored as two
 * reduced distributions on the n[0] x n[1] grid, G = int f dxi_z and
 * H = int xi_z^2 f dxi_z (flat index v = ix + nx*(iy + ny*p), p = 0 for G,
 * 1 for H; weight (hi[0]-lo[0])(hi[1]-lo[1])/(n[0] n[1]); n[2], lo[2], hi[2]
 * ignored).  Needs a mesh whose faces have no z component and a state with
 * u_z = 0 (GSIS_ERR_ARG at the first gsis_iterate otherwise). */
typedef struct {
    int    n[3];
    double lo[3];
    double hi[3];
    int    reduced;
} gsis_vgrid_desc;

/* Per-call report of gsis_iterate. Phase times are CUDA-event times on the
 * context stream, summed over the iterations of the call (milliseconds). */
enum { GSIS_PH_ADAPT = 0, GSIS_PH_CELLEQ = 1, GSIS_PH_SWEEP = 2, GSIS_PH_MOMENTS = 3,
       GSIS_PH_MACRO = 4, GSIS_PH_CORRECT = 5, GSIS_PH_RESID = 6, GSIS_PH_PRESOLVE = 7, GSIS_NPHASE = 8 };
typedef struct {
    int     iterations;          /* GSIS iterations run by this call                    */
    int     total_iterations;    /* since gsis_init                                     */
    double  eps;                 /* epsilon of the last iteration (Sec. 4)              */
    int     converged;           /* eps < tol                                           */
    long long n_dvm;             /* kinetic cells                                       */
    long long n_v;               /* discrete velocities                                 */
    long long vdf_bytes;         /* bytes of the compacted VDF array                    */
    int     presolve_blocks;     /* NS presolve blocks run (adaptive only)              */
    double  phase_ms[GSIS_NPHASE];
    long long sweep_launches;    /* sweep kernel launches in this call                  */
    long long kernel_launches;   /* all kernel launches in this call                    */
} gsis_report;

typedef struct gsis_ctx gsis_ctx;

/* Create a context.  params is copied.  alloc may be NULL (cudaMalloc/cudaFree).
 * cuda_stream is a cudaStream_t (NULL = default stream).
 * Errors: GSIS_ERR_ARG (NULL out/params, Kn <= 0, macro_steps < 0, k_sub < 0,
 * cfl <= 0, dt < 0, unknown vdf_dtype), GSIS_ERR_UNSUPPORTED (Kn outside
 * [1e-15, 1e15]: the kinetic update's quotient needs 1/tau + sum xi.S/V inside
 * the FP32 exponent range, see gsis_set_velocity_grid; d_r > 0),
 * GSIS_ERR_CUDA (no device). */
gsis_status gsis_init(const gsis_params* params, const gsis_allocator* alloc, void* cuda_stream,
                      gsis_ctx** out);

/* Upload the mesh (copied to the device). Must precede gsis_iterate. */
gsis_status gsis_set_mesh(gsis_ctx* ctx, const gsis_mesh_desc* mesh);

/* Set the velocity grid. Must precede gsis_iterate; GSIS_ERR_STATE afterwards.
 * Errors: GSIS_ERR_ARG for n[d] < 1 or hi[d] <= lo[d]; GSIS_ERR_UNSUPPORTED
 * when max|xi| times the mesh's largest sum_s |S_s|/V exceeds 2^100 (the
 * kinetic update divides by 1/tau + sum_s max(xi.S_s, 0)/V with an FP32
 * reciprocal seed, which needs that denominator inside the FP32 exponent
 * range; gsis_set_mesh refuses a mesh the same way once the grid is set). */
gsis_status gsis_set_velocity_grid(gsis_ctx* ctx, const gsis_vgrid_desc* vgrid);

/* Run up to max_iter GSIS iterations (Sec. 3.1 steps; Sec. 3.4 drives the
 * adaptive start on the first call).  max_iter = 0 performs only the start
 * (presolve, region, initial VDF).  Stops early when eps < tol.  Synchronises
 * the stream once per iteration to read eps (8 bytes device->host).
 * report may be NULL.  Errors: GSIS_ERR_STATE (mesh or grid missing),
 * GSIS_ERR_NONFINITE, GSIS_ERR_CUDA, GSIS_ERR_OOM, GSIS_ERR_TIMEOUT (with
 * the persistent synthetic solve selected: a grid barrier waited more than
 * spin_limit polls; every block of that launch returns, the CUDA context
 * stays usable, the state of this solve is lost). */
gsis_status gsis_iterate(gsis_ctx* ctx, int max_iter, gsis_report* report);

/* Write the selected per-cell fields (GSIS_FIELD_* bits, in bit order) of the
 * current state: [ncell][popcount(mask)] doubles to dst (host memory when
 * dst_is_device = 0, device memory on the context's device otherwise).  HoT
 * fields are those of the last kinetic step (zero in NS cells).
 * GSIS_FIELD_WALL_Q, for a cell with diffuse-wall sides: the energy flux
 * through those sides into the wall divided by their area -- for a DVM cell
 * carried by its current distribution (outgoing half of f, the re-emitted
 * half rho_w M(0, T_w) with zero net mass flux), for an NS cell the Fourier
 * heat flux of the NSF wall flux at the current state; 0 for other cells.
 * GSIS_FIELD_WALL_P / _TX.._TZ: the momentum components F_m of the same wall
 * fluxes (outward area vector S, unit normal n = S/|S|), pressure F_m.n and
 * shear F_m - (F_m.n) n, summed over the wall sides and divided by their area.
 * The derived fields (WALL_*, S*, Q*, P) are computed on the device at the
 * call; before the first gsis_iterate (state W0; HoT, Kn_Gll and the DVM flag
 * 0) they give GSIS_ERR_STATE. */
gsis_status gsis_moments(gsis_ctx* ctx, unsigned field_mask, double* dst, int dst_is_device);

/* Copy the compacted VDF of the DVM cells to host memory as FP64:
 * dst [n_dvm][n_v] in the order of the cell list returned through cells
 * (flat cell indices, n_dvm entries, may be NULL). */
gsis_status gsis_get_vdf(gsis_ctx* ctx, double* dst, int* cells, long long capacity);

/* Test hook: force the DVM region to the given per-cell flags (uint8, ncell)
 * instead of the Kn_Gll rule, for the start and for the re-identification.
 * Used to compare with a reference whose threshold decisions are taken
 * elsewhere.  Must be called before the first gsis_iterate. */
gsis_status gsis_debug_set_region(gsis_ctx* ctx, const uint8_t* flags);

/* Advance n independent solves together by `iterations` GSIS iterations each
 * (the batched form: many small solves, e.g. 1D shocks with uneven meshes,
 * velocity grids and VDF storage types, in one device pass per iteration).
 * Per iteration the per-solve stages run for every solve, the kinetic sweeps
 * of ALL solves run in one persistent launch that draws (solve, velocity
 * tile) work items from a device counter, and the synthetic solves of all
 * meshes up to 4096 cells run in one launch (one CTA each); one iteration of
 * the whole batch is recorded once into a CUDA graph and replayed.  The tile
 * shape of the persistent sweep is picked by timing the candidates on the
 * batch itself (on a snapshot of the VDFs, restored afterwards; skipped
 * without memory for the snapshot) and cached per batch shape for the life
 * of the process.  Results are identical to iterating each solve alone.
 *
 * ctxs: n distinct contexts on one device, each with mesh and velocity grid
 *       set, adaptive = 0 (or a region forced by gsis_debug_set_region);
 *       contexts not yet started are started (presolve included).
 * iterations: >= 0; exactly this many iterations run (no early stop: the
 *       residual is only read at the end); reports[i] (may be NULL) receives
 *       the residual of the last iteration and the sizes of solve i; its
 *       phase_ms[GSIS_PH_SWEEP] is the duration of the batched sweep launch of
 *       the last iteration (the whole batch, not solve i alone) and
 *       phase_ms[GSIS_PH_MACRO] the rest of that iteration.
 * The batch runs on ctxs[0]'s stream (a private stream when that is the
 * legacy default stream) after synchronising every context's stream, and
 * synchronises before returning.  The recorded graph is kept for the same
 * ordered context list and re-recorded when a context was iterated alone in
 * between; gsis_free of any member drops it.
 * Errors: GSIS_ERR_ARG (NULL, n <= 0, duplicates, mixed devices),
 * GSIS_ERR_UNSUPPORTED (adaptive context), GSIS_ERR_STATE, GSIS_ERR_OOM,
 * GSIS_ERR_CUDA; GSIS_ERR_NONFINITE if a solve ends non-finite (that context
 * becomes unusable).  The paper has no counterpart: it runs one solve at a
 * time. */
gsis_status gsis_iterate_batch(gsis_ctx** ctxs, int n, int iterations, gsis_report* reports);

/* Test hook: batch plans recorded from now on (in this process) use the named
 * tile shape of the persistent batched sweep instead of the autotuned one
 * (names as reported by gsis_batch_info, e.g. "vpt2_cb1_w4", or the
 * velocity-pair shapes "pair1_cb1_w4", "pair2_cb1_w4", "pair1_cb1_w8", which
 * need FP32/BF16/FP16 members with an even nx: gsis_iterate_batch then returns
 * GSIS_ERR_ARG for another batch).  NULL or "" restores autotuning.  Every
 * shape computes the same result.  GSIS_ERR_ARG for an unknown name.  The
 * paper has no counterpart. */
gsis_status gsis_debug_set_batch_tile(const char* name);

/* Test hook: run the kinetic sweep of this context with the named tile shape
 * from now on instead of the autotuned one (names as reported by
 * gsis_tuning_info, e.g. "g4_v1_c1", "ring_w8_v32"); starts the context
 * (presolve, region) if needed.  Every shape computes the same result.
 * GSIS_ERR_ARG for an unknown name or a shape that cannot run this problem
 * (the shared-memory window shapes need a 2D mesh whose hyperplane window
 * fits in shared memory).  The paper has no counterpart. */
gsis_status gsis_debug_set_sweep_tile(gsis_ctx* ctx, const char* name);

/* Test hook: velocity moments of the VDF of each DVM cell (Eq. getmoment,
 * the quadrature of Sec. 3.1), dst [n_dvm][19] doubles in host memory, in
 * the order of the cell list of gsis_get_vdf; capacity = entries of dst
 * (>= 19 n_dvm, else GSIS_ERR_ARG).  Per cell, with c = xi - u the peculiar
 * velocity about the cell's current macroscopic velocity u and w the
 * quadrature weight: sum w f; sum w c f (3); sum w c_i c_j f for xx, yy, zz,
 * xy, xz, yz; sum w c_i |c|^2 f (3); then for each of the six sides, on a
 * diffuse-wall side, the outgoing half-range sum of w (xi.S) f (S the
 * outward area vector), else 0.
 * direct = 0: the moments the last GSIS iteration carried forward (taken
 * without a pass over the velocities after the correction of Eq. updatef);
 * direct = 1: a fresh reduction over the current VDF.  Both describe the same
 * VDF, so they agree up to rounding (and, for reduced-precision storage, the
 * storage rounding of the corrected values).  GSIS_ERR_STATE before the
 * first iteration.  The paper has no counterpart. */
gsis_status gsis_debug_vdf_moments(gsis_ctx* ctx, int direct, double* dst, long long capacity);

/* Test hook: choose how the synthetic solve (Eq. macro) runs from now on.
 * GSIS_MACRO_AUTO (default): the fused one-CTA kernel for meshes of up to
 * 4096 cells, else the per-phase kernels (4 + k_sub launches per
 * pseudo-step).  GSIS_MACRO_FUSED, _MULTI and _PERSISTENT (one cooperative
 * launch per block of pseudo-steps, the phases separated by grid barriers
 * bounded by spin_limit; the per-phase kernels inside a batch graph capture
 * or where a cooperative launch is not available) force one
 * implementation; all compute the same result.
 * GSIS_MACRO_PERSISTENT_STALL (tests of the bounded wait only): the
 * persistent launch's barrier waits for one CTA more than the launch has, so
 * the wait can only end by running out of spin_limit polls; the next
 * gsis_iterate returns GSIS_ERR_TIMEOUT.  GSIS_ERR_ARG for another value.
 * The paper has no counterpart. */
enum { GSIS_MACRO_AUTO = 0, GSIS_MACRO_FUSED = 1, GSIS_MACRO_MULTI = 2, GSIS_MACRO_PERSISTENT = 3,
       GSIS_MACRO_PERSISTENT_STALL = 4 };
gsis_status gsis_debug_set_macro_path(gsis_ctx* ctx, int path);

/* Human-readable result of the sweep's tile-shape autotuning for this
 * context (chosen shape and the timing of every candidate), or "" before the
 * first iteration.  Each context times the candidate shapes of its kinetic
 * sweep once per DVM region (on a snapshot of its VDF, restored afterwards;
 * results cached per problem shape for the life of the process).  The string
 * is owned by the context. */
const char* gsis_tuning_info(gsis_ctx* ctx);

/* Human-readable description of the recorded batch plan for this ordered
 * context list (work items, autotuned tile shape and the timings of every
 * candidate, grid, graph nodes), or "" if none.  The string lives until the
 * next call from the same thread. */
const char* gsis_batch_info(gsis_ctx** ctxs, int n);

/* Reference distribution pair of the two-VDF model of a gas with d_r internal
 * degrees of freedom (Sec. 2, Eq. general_model): for each state, on the
 * context's velocity grid,
 *   g0 = (1 - 1/Z_r) g_0t + g_0r / Z_r,   g1 = (1 - 1/Z_r) g_1t + g_1r / Z_r,
 * with g_0t the Shakhov form at (T_t, q_t), g_0r the one at the equilibrium
 * temperature T = (3 T_t + d_r T_r)/(3 + d_r) and q0, g_1t = (d_r/2) T_r g_0t +
 * M_t (q_r.c)/(rho T_t), g_1r = (d_r/2) T g_0r + M_T (q1.c)/(rho T) (R = 1),
 * (q0, q1) the mixing of (q_t, q_r) by the A matrix.  g_0t and g_0r are
 * conservation-corrected (their discrete mass, momentum and translational
 * energy are exact), and so are the Maxwellians M_t, M_T of the q terms, so
 * that the pair conserves mass, momentum and total energy on the grid.  This
 * is the reference pair of the two-VDF kinetic step, which gsis_iterate does
 * not run (gsis_init refuses d_r > 0); it is evaluated here on its own.
 *
 * ctx:    a context whose velocity grid is set (full 3D grids only); its
 *         allocator and stream are used, and the call synchronises the stream.
 * S:      device pointer, [n][12] states: rho, u_x, u_y, u_z, T_t, T_r,
 *         q_t (3), q_r (3); rho, T_t > 0 and (d_r > 0) T_r > 0; 0 <= n <= 65535.
 * d_r, Z_r, A: the gas (A = A_tt, A_tr, A_rt, A_rr; host pointer); Z_r >= 1.
 * g_out:  device pointer, [n][2][Nv] doubles (x fastest): g0 then g1 of each
 *         state; written in full, owned by the caller.
 * Allocates scratch of 4 n (16 + 5 (nx + ny + nz)) doubles through the
 * context's allocator for the duration of the call.
 * Errors: GSIS_ERR_ARG (NULL, n out of range, bad gas, non-finite or
 * non-positive states; checked before any launch), GSIS_ERR_STATE (no
 * velocity grid), GSIS_ERR_UNSUPPORTED (reduced grid), GSIS_ERR_OOM,
 * GSIS_ERR_CUDA. */
gsis_status gsis_two_vdf_reference(gsis_ctx* ctx, const double* S, int n, int d_r, double Z_r, const double* A,
                                   double* g_out);

/* Moments of two-VDF distribution pairs (Sec. 2, Eq. getmoment) on the
 * context's velocity grid, the reduction of the two-VDF kinetic step
 * (evaluated on its own, as gsis_two_vdf_reference): rho and u from f0; about
 * u the traceless stress sigma = P - tr P/3 I and the heat flux
 * q_t = 1/2 sum w c |c|^2 f0 of f0, T_t = tr P/(3 rho); from f1
 * d_r/2 rho T_r = sum w f1 and q_r = sum w c f1 (T_r = T_t when d_r = 0).
 * FP64 sums.
 *
 * ctx:  a context whose velocity grid is set (full 3D grids only); its stream
 *       is used and synchronised.
 * F:    device pointer, [n][2][Nv] doubles (x fastest): f0 then f1 of each
 *       pair (as gsis_two_vdf_reference writes them); 0 <= n <= 65535.
 * out:  device pointer, [n][18] doubles: rho, u (3), T_t, T_r, sigma (xx, yy,
 *       zz, xy, xz, yz), q_t (3), q_r (3); owned by the caller.  The pairs
 *       are not inspected: a pair with zero mass gives non-finite moments.
 * Errors: GSIS_ERR_ARG (NULL, n or d_r out of range), GSIS_ERR_STATE (no
 * velocity grid), GSIS_ERR_UNSUPPORTED (reduced grid), GSIS_ERR_CUDA. */
gsis_status gsis_two_vdf_moments(gsis_ctx* ctx, const double* F, int n, int d_r, double* out);

/* Sweep levels of an unstructured mesh (host computation; no context, no
 * device work): the schedule under which a level-parallel kinetic sweep gives
 * the values of the sequential Gauss-Seidel sweep in the order (key, index).
 * In that order each cell's level is one more than the highest level of its
 * face neighbours that come before it (0 if none): face neighbours never
 * share a level, and every neighbour that precedes a cell lies on a lower
 * level (sweeping the levels downwards reproduces the reverse sweep).  On a
 * structured grid with key i + j + k the levels are its hyperplanes.
 *
 * ncell:      number of cells (>= 0).
 * offsets:    host, [ncell + 1], offsets[0] = 0, non-decreasing: the face
 *             neighbours of cell c are neighbours[offsets[c] .. offsets[c+1]).
 * neighbours: host, cell indices in [0, ncell), none equal to its own cell;
 *             the relation must be symmetric.
 * key:        host, [ncell] finite sweep-order keys.
 * level:      host, [ncell], written.  nlevels: host, number of levels.
 * Errors: GSIS_ERR_ARG (NULL where data are needed, bad offsets, an index
 * out of range or a self-neighbour, an asymmetric relation, a non-finite
 * key); nothing is written to level then. */
gsis_status gsis_sweep_levels(int ncell, const int* offsets, const int* neighbours, const double* key, int* level,
                              int* nlevels);

/* Human-readable description of the last error on this context (never NULL). */
const char* gsis_last_error(const gsis_ctx* ctx);

/* Release every resource of the context. NULL-safe; the pointer is invalid afterwards. */
void gsis_free(gsis_ctx* ctx);

/* Library version string. */
const char* gsis_version(void);

/* Measurement utility (the paper has no counterpart): the fused
 * multiply-add throughput of the CUDA cores of the current device in FP64
 * (fp64 != 0) or FP32, in flop/s (2 per FMA), the best of four launches of
 * about 40 ms each on cuda_stream (NULL = default stream; synchronises it).
 * It is the measured roof of the FP64- and FP32-arithmetic kinetic sweeps.
 * ms (may be NULL) receives the duration of the best launch.  Allocates and
 * frees a few KB of device memory.  Errors: GSIS_ERR_ARG (NULL
 * flops_per_s), GSIS_ERR_OOM, GSIS_ERR_CUDA. */
gsis_status gsis_probe_fma_peak(int fp64, void* cuda_stream, double* flops_per_s, double* ms);

/* Allocation-free evaluation of conservation-corrected discrete Maxwellians
 * (the paper has no counterpart; this is a library service).
 *
 * For callers that must not allocate device memory: applications whose device
 * memory is owned entirely by their own arena or pool and that forbid any
 * other allocation, and latency-critical loops where a cudaMalloc (which may
 * synchronise the device and take an unbounded time) is not allowed.  The
 * function allocates nothing: its intermediate data live in one fixed-size
 * array of device memory (about 3.9 MB) that every GPU loading the library
 * holds until the process exits.
 *
 * W:      device pointer, [n][5] states (rho, ux, uy, uz, T), rho > 0, T > 0.
 * vgrid:  host pointer, the velocity grid (as for gsis_set_velocity_grid;
 *         full 3D grids only: reduced = 1 gives GSIS_ERR_ARG).
 * f_out:  device pointer, [n][nx*ny*nz] doubles (x fastest): row k receives
 *         the Maxwellian of W[k] corrected so that its discrete mass,
 *         momentum and energy equal those of W[k] exactly (the same rows the
 *         all-kinetic start of gsis_iterate stores as the initial VDF).
 * cuda_stream: cudaStream_t on which the work is queued (NULL = default).
 * Limits: n <= 256 and nx + ny + nz <= 384 per call (each of nx, ny, nz
 * checked before they are summed), else GSIS_ERR_ARG; process more states in
 * several calls.  Other errors: GSIS_ERR_ARG for NULL pointers or an invalid
 * grid; GSIS_ERR_CUDA when a CUDA call fails, or on entry when an error of
 * earlier asynchronous work is already pending on the calling thread (that
 * error is left pending for its owner and nothing is queued).
 * The first call on a device looks up the address of the device array
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The address is cached for the life of the
 * process: after a cudaDeviceReset of that device the entry point must not be
 * called again in the same process.  All calls share the array and it keeps
 * the last call's contents, so calls whose device work overlaps (other
 * streams, other host threads) race on it: order them on one stream.
 * Asynchronous: returns after queueing the work. */
gsis_status gsis_corrected_maxwellian_noalloc(const double* W, int n, const gsis_vgrid_desc* vgrid,
                                              double* f_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GSIS_H */
