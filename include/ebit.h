/*
 * ebit.h -- C ABI of the GB300 (sm_103a) EBIT phase-change time step.
 *
 * Method: Long, Pan & Zaleski, "An Edge-based Interface Tracking (EBIT) Method for
 * Multiphase Flows with Phase Change", arXiv 2402.13677.  One call of ebit_step()
 * performs the five-step iteration of Sec. 2.5 on a uniform 2D Cartesian grid:
 *   1. energy advection (energy-advection equation, Sec. 2.4),
 *   2. EBIT interface advection (marker-motion equations, Sec. 2.1, Fig. 1) with the
 *      interfacial velocity of the jump condition (interfacial-velocity equation,
 *      Sec. 2.3, Fig. 2) and Color-Vertex reconnection (Sec. 2.1),
 *   3. energy diffusion with T = T_sat imposed sharply through ghost-fluid
 *      coefficients (ghost-temperature and Txx-ghost equations, Sec. 2.4),
 *   4. interface heat and mass flux (mass-flux and normal-gradient equations) and the
 *      ghost velocities (ghost-velocity equation, Sec. 2.3),
 *   5. momentum predictor and ghost-fluid projection (discretization equations 1-5
 *      and the ghost-fluid Poisson equation, Sec. 2.3).
 *
 * Conventions
 *   - Grid units: cell (i, j) covers [x0 + i h, x0 + (i+1) h] x [y0 + j h, ...].  All
 *     arrays are row-major with x fastest:
 *       cell fields        ny     x nx        (double, or double2 = {x, y} for vectors)
 *       x-faces            ny     x (nx + 1)  (normal velocity at x = x0 + i h)
 *       y-faces            (ny+1) x nx
 *       vertex colours     (ny+1) x (nx + 1)  (uint8: 1 liquid, 0 vapour)
 *       horizontal edges   (ny+1) x nx        (marker fraction from the left vertex)
 *       vertical edges     ny     x (nx + 1)  (marker fraction from the lower vertex)
 *     An edge carries a marker (is "cut") iff its two vertex colours differ (one marker
 *     per edge, Sec. 2.1); marker fractions of cut edges lie in [1e-9, 1 - 1e-9].
 *   - Pointers: "host" pointers are plain CPU memory; "device" pointers are CUDA global
 *     memory of the device that was current at ebit_init().  The caller owns every
 *     pointer it passes; the library keeps none of them after the call returns.
 *   - Streams: all device work of a context is ordered on the cudaStream_t given to
 *     ebit_init() (passed as void*; NULL = legacy default stream).  Calls that return
 *     data to the host (ebit_get_field with on_device = 0, ebit_get_diagnostics)
 *     synchronise that stream before returning; ebit_step() synchronises once per step to
 *     read the status word and the solver statistics (and, with graphs disabled, polls the
 *     solver convergence words every few iterations).
 *   - Errors: every call returns an ebit_status; on failure a message is kept for
 *     ebit_last_error().  EBIT_ENOCONV means a linear solve hit max_iter: the step is
 *     completed with its last iterate; iteration counts and final residuals are reported by
 *     ebit_get_diagnostics().  EBIT_ECUDA means a CUDA call failed, or a bounded device
 *     wait gave up; the context should then be destroyed.  EBIT_ENONFINITE means a NaN or
 *     an infinity reached a linear solve (each solve tests its residual norms and stops at
 *     the first non-finite one): the step is completed but its results are not usable.
 *   - Threads: a context may be used by one host thread at a time.
 */
#ifndef EBIT_H
#define EBIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ebit_ctx ebit_ctx;

typedef enum {
    EBIT_OK = 0,
    EBIT_EINVAL = -1,     /* bad argument or inconsistent input                        */
    EBIT_ENOMEM = -2,     /* device allocation failed                                  */
    EBIT_ENOCONV = -3,    /* a linear solve did not reach its tolerance in max_iter     */
    EBIT_ETOPO = -4,      /* marker set inconsistent with the vertex colours            */
    EBIT_ECUDA = -5,      /* CUDA runtime error                                        */
    EBIT_ECFL = -6,       /* a marker moved one cell or more in one sweep (CFL >= 1)   */
    EBIT_ENONFINITE = -7  /* a linear solve met a NaN or an infinity (in the state, a field
                             the caller set, or the system passed to a solve entry point) */
} ebit_status;

/* Boundary kinds (per side: 0 left, 1 right, 2 bottom, 3 top). */
enum { EBIT_BC_WALL = 0,      /* no-slip wall: u = 0, zero normal pressure gradient     */
       EBIT_BC_OUTFLOW = 1,   /* zero normal gradient of u and T, p = 0 on the face     */
       EBIT_BC_SYMMETRY = 2   /* normal u = 0, tangential u and T free                  */ };

/* Precision of the linear solves. */
enum { EBIT_FP64 = 0,         /* MG-preconditioned CG entirely in FP64                   */
       EBIT_MIXED = 1         /* FP32 MG-PCG inside an FP64 iterative-refinement loop;
                                 ghost-fluid coefficients, jump-condition velocities and
                                 the outer residuals stay FP64                           */ };

typedef struct {
    int nx, ny;               /* cells, each >= 4, nx * ny <= 2^29                        */
    double x0, y0, h;         /* origin and cell size (square cells)                      */
    int bc[4];                /* EBIT_BC_* per side                                       */
    int T_fixed[4];           /* 1: wall temperature T_wall[s] imposed (Dirichlet)        */
    double T_wall[4];
    double dt;                /* time step                                                */
    int precision;            /* EBIT_FP64 or EBIT_MIXED                                   */
    double rtol;              /* relative residual ||b - A x||_2 / ||b||_2 of every solve */
    int max_iter;             /* CG iterations (FP64) or outer refinements x inner (MIXED) */
    int extend_iters;         /* Jacobi sweeps of the narrow-band extension (paper: iterative) */
    double theta_min;         /* lower clamp of the ghost-fluid link fraction theta        */
    int sweep_order;          /* 0: x then y every step; 1: alternate x-y / y-x             */
    int energy;               /* 1: solve the energy equation; 0: impose mdot_fixed (Sec. 3.3) */
    double mdot_fixed;
    int one_fluid;            /* 0: ghost-fluid method (ghost-velocity equation, two velocity
                                 fields); 1: one-fluid variant (Sec. 2.3): one velocity field
                                 (the vapour arrays repeat the liquid ones; set the liquid ones),
                                 no ghost velocities, and the phase-change source of the
                                 pc-source equation in the projection, div u_f = S_pc with
                                 S_pc V = mdot S_Gamma (1/rho_v - 1/rho_l) in the cut cells     */
    int axisymmetric;         /* 0: planar (x, y), per unit depth; 1: axisymmetric (r, z) about the
                                 line x = 0 (the setting of Secs. 3.4-3.7): x is the radius, x0 >= 0,
                                 and with x0 == 0 the left side is the axis (bc[0] must be
                                 EBIT_BC_SYMMETRY).  Every integrated balance (the rows of the
                                 energy, viscous and Poisson systems, the divergence of the face
                                 velocities, the phase-change source) is weighted by the radius of
                                 its cell, face or interface segment, the radial velocity gets the
                                 hoop term mu u_r / r^2 of the viscous stress, the curvature gets
                                 its azimuthal part n_r / r, and the diagnostics report ring
                                 volumes, masses and fluxes (2 pi r times the planar measure)     */
} ebit_config;

typedef struct { double rho, mu, lambda, cp; } ebit_phase_props;

/* Optional device allocator: returns a device pointer of at least `bytes` bytes (aligned
 * to 256 B) or NULL; the library frees it through `free_fn` in ebit_destroy().  With
 * alloc == NULL the library uses cudaMalloc/cudaFree. */
typedef struct {
    void* (*alloc_fn)(size_t bytes, void* user);
    void (*free_fn)(void* ptr, void* user);
    void* user;
} ebit_allocator;

/* Field identifiers for ebit_set_field / ebit_get_field. */
enum {
    EBIT_F_T_L = 0, EBIT_F_T_V = 1,         /* cell temperature of each phase (ghost band included) */
    EBIT_F_U_L = 2, EBIT_F_U_V = 3,         /* cell velocity, double2                                */
    EBIT_F_UFX_L = 4, EBIT_F_UFX_V = 5,     /* x-face normal velocity                                */
    EBIT_F_UFY_L = 6, EBIT_F_UFY_V = 7,     /* y-face normal velocity                                */
    EBIT_F_P = 8,                           /* pressure                                              */
    EBIT_F_GC = 9,                          /* cell face-acceleration average, double2               */
    EBIT_F_MDOT = 10,                       /* mass flux on the narrow band                          */
    EBIT_F_VF = 11,                         /* liquid volume fraction (read only)                    */
    EBIT_F_CCOL = 12,                       /* uint8 centre colour f_C (read only)                   */
    EBIT_F_BAND = 13,                       /* uint8 narrow-band flag (read only)                    */
    EBIT_F_NB = 14,                         /* band normal, double2, liquid -> vapour (read only)    */
    EBIT_F_VCOL = 15,                       /* uint8 vertex colours                                  */
    EBIT_F_HX_POS = 16, EBIT_F_VY_POS = 17, /* marker fractions of horizontal / vertical edges       */
    EBIT_F_TSTAR_L = 18, EBIT_F_TSTAR_V = 19, /* advected temperature of the current step            */
    EBIT_F_CSEG = 20,                       /* uint16 per cell: nseg | P0<<2 | Q0<<4 | P1<<6 | Q1<<8  */
    EBIT_F_UG = 21,                         /* cell interfacial velocity u_Gamma of the last step,
                                               double2, on the cells within two of the interface  */
    EBIT_F_COUNT = 22
};

/* Stages for ebit_run_stage (one call of ebit_step runs STAGE_ADVECT_T .. STAGE_DIAGNOSTICS). */
enum {
    EBIT_STAGE_PREPARE = 0,          /* reconstruct, extend T, mdot, ghost velocities, gc      */
    EBIT_STAGE_RECONSTRUCT = 1,      /* Color-Vertex reconstruction + band (S0)                */
    EBIT_STAGE_ADVECT_T = 2,         /* S1: T* = WENO3 advection of T_l, T_v                    */
    EBIT_STAGE_EXTEND_TSTAR = 3,     /* S6: extend T* into the band of the current interface   */
    EBIT_STAGE_ADVANCE_INTERFACE = 4,/* S2-S5: u_Gamma, two sweeps, reconnection                */
    EBIT_STAGE_SOLVE_ENERGY = 5,     /* S7-S8: ghost-fluid coefficients and implicit diffusion  */
    EBIT_STAGE_EXTEND_T = 6,         /* ghost band of T after the diffusion solve               */
    EBIT_STAGE_MASS_FLUX = 7,        /* S9: mdot on cut cells, extended over the band           */
    EBIT_STAGE_GHOST_VELOCITY = 8,   /* S10                                                    */
    EBIT_STAGE_MOMENTUM = 9,         /* S11 + S12: predictor and projection                    */
    EBIT_STAGE_DIAGNOSTICS = 10,     /* S13, also advances t and the step counter               */
    EBIT_STAGE_COUNT = 11
};

/* Create a context for `batch` independent instances (cfgs[0..batch-1]); all instance
 * data is allocated here, once.  stream: cudaStream_t or NULL. */
ebit_status ebit_init(const ebit_config* cfgs, int batch, void* stream,
                      const ebit_allocator* alloc, ebit_ctx** out);

/* Material properties of instance `inst` (Sec. 2.2): liquid and vapour rho, mu, lambda,
 * cp; saturation temperature, latent heat h_lg, surface tension coefficient sigma >= 0,
 * gravity.  With sigma > 0 the step adds the surface-tension force f = sigma kappa delta_s n
 * of the momentum equation (discretization equations 1-5) in the well-balanced face form:
 * sigma kappa_f (H_j - H_i) / (h rho_f) on every interior face, H the liquid volume fraction,
 * kappa = div n (n from liquid into vapour) from the circles through each cut cell's markers
 * and their chain neighbours, so that the pressure jumps by p_liq - p_vap = sigma kappa across
 * the interface (pressure-jump equation). */
ebit_status ebit_set_phase_props(ebit_ctx* ctx, int inst, const ebit_phase_props* liq,
                                 const ebit_phase_props* vap, double T_sat, double h_lg,
                                 double sigma, double gx, double gy);

/* Interface of instance `inst`: vertex colours and marker fractions (layouts above).
 * Cut flags are implied by the colours; fractions of uncut edges are ignored. */
ebit_status ebit_set_interface(ebit_ctx* ctx, int inst, const uint8_t* vcol,
                               const double* hx_pos, const double* vy_pos, int on_device);

/* Copy one field in (set) or out (get); on_device selects device or host pointers. */
ebit_status ebit_set_field(ebit_ctx* ctx, int inst, int field, const void* src, int on_device);
ebit_status ebit_get_field(ebit_ctx* ctx, int inst, int field, void* dst, int on_device);

/* Copy n fields in (set) or out (get) in one call: field ids[k] from srcs[k] / to dsts[k]
 * (each laid out as for ebit_set_field / ebit_get_field).  The copies are issued back to back
 * on the context stream and, for host pointers, the stream is synchronised once after the
 * last of them (page-locked host buffers make the copies asynchronous).  Read-only fields
 * are rejected by ebit_set_fields; ebit_get_fields rejects EBIT_F_CCOL and EBIT_F_BAND (bits
 * of the flag byte: use ebit_get_field).  EBIT_EINVAL names the first bad entry; no copy is
 * issued then. */
ebit_status ebit_set_fields(ebit_ctx* ctx, int inst, int n, const int* ids, const void* const* srcs,
                            int on_device);
ebit_status ebit_get_fields(ebit_ctx* ctx, int inst, int n, const int* ids, void* const* dsts, int on_device);

/* Number of elements and element size of a field of instance `inst`. */
ebit_status ebit_field_shape(const ebit_ctx* ctx, int inst, int field, size_t* count, size_t* elem_bytes);

/* Set the time of instance `inst` (its step counter is reset to 0). */
ebit_status ebit_set_time(ebit_ctx* ctx, int inst, double t);

/* Run one stage on every instance (parity testing and profiling). */
ebit_status ebit_run_stage(ebit_ctx* ctx, int stage);

/* Advance every instance by nsteps time steps (ebit_run_stage(PREPARE) must have run). */
ebit_status ebit_step(ebit_ctx* ctx, int nsteps);

/* Diagnostics of the last step of instance `inst` (Sec. 3): up to n (<= 14) doubles of
 * { t, vapour volume, volume expected from sum mdot S dt / rho_v in the step, M_d (mass-in-
 *   domain equation), outlet mass in the step (mass-with-outflow equation), cut cells,
 *   solver iterations (energy, viscous, Poisson), final relative residuals (energy, viscous,
 *   Poisson), vapour volume that left through the outflow faces in the step (the V_bc of the
 *   film-boiling vapour volume, Sec. 3.7: (1 - H) u_f . n h dt over the outflow faces, H the
 *   boundary cell's volume fraction, u_f the face velocity of its phase), space-averaged
 *   Nusselt number of the fixed-temperature walls (Sec. 3.7: l / (T_w - T_sat) times the mean
 *   of 2 (T_w - T_i) / h over their faces, T_i the boundary cell's temperature of its phase,
 *   l = sqrt(sigma / (|rho_l - rho_v| |g|)) when sigma and g are nonzero, else 1) }.
 * Synchronises. */
ebit_status ebit_get_diagnostics(ebit_ctx* ctx, int inst, double* dst, int n);

/* Kernel launches issued since the context was created (all instances). */
uint64_t ebit_launch_count(const ebit_ctx* ctx);

/* Device-side timing of one kernel class while ebit_step runs (graph or not): each timed
 * launch records the span from its first block's start to its last block's end from the GPU
 * global timer.  kernel_class EBIT_KT_SMOOTH_L0: the finest-grid multigrid smoother kernels
 * (tiled red-black Gauss-Seidel "pre" and "post" kernels), the dominant kernels of the step.
 * ebit_timing_end synchronises and returns the summed kernel time, the number of timed
 * launches and the algorithmic bytes of an average launch (pre: b, diag, wl, wb read, x and a
 * quarter-size coarse b written; post: x, a quarter-size coarse x, b, diag, wl, wb read, x
 * written; one word per value, 4 bytes in the mixed mode, 8 in FP64, per right-hand side).  A
 * batched launch counts once, with the bytes of all its instances that had not converged. */
enum { EBIT_KT_SMOOTH_L0 = 1 };
ebit_status ebit_timing_begin(ebit_ctx* ctx, int kernel_class);
ebit_status ebit_timing_end(ebit_ctx* ctx, double* total_ms, uint64_t* launches, double* bytes_per_launch);

/* The library's multigrid-preconditioned CG (FP64, or FP32 inside FP64 refinement) applied
 * to a caller-supplied five-point system on instance `inst`'s grid (host pointers, cell
 * arrays of nx*ny doubles, layout above):
 *   (A x)_i = D_i x_i + wl_i (x_i - x_{i-1}) + wl_{i+1} (x_i - x_{i+1})
 *                     + wb_i (x_i - x_{i-nx}) + wb_{i+nx} (x_i - x_{i+nx}),
 * wl_i / wb_i the weights of cell i's left / bottom face (0 on domain faces), D_i >= 0, the
 * matrix symmetric positive definite.  nr = 1 or 2 right-hand sides interleaved per cell
 * (b and x hold nr*nx*ny doubles; x is the initial guess on entry, the solution on return).
 * Converges to ||b - A x||_2 <= rtol ||b||_2 per right-hand side; returns the iteration count
 * (CG iterations, or total inner FP32 iterations in refinement mode) and the final relative
 * residual.  This is the solver used by the energy, viscous and Poisson solves of ebit_step;
 * it overwrites that instance's operator scratch (not its state).  EBIT_ENOCONV if max_iter
 * is reached.  Synchronises. */
ebit_status ebit_solve_system(ebit_ctx* ctx, int inst, const double* D, const double* wl, const double* wb,
                              const double* b, double* x, int nr, int precision, double rtol, int max_iter,
                              int* iters, double* rel_res);

/* Allocation-free variant of ebit_solve_system, for callers that cannot allocate device
 * memory when they call: a host framework that owns the whole device memory through its own
 * pool and forbids other allocations, or a service loop that must not allocate per call.
 * No context: D, wl, wb, b and x are the caller's DEVICE arrays (same meaning and layout as in
 * ebit_solve_system, on an nx x ny grid; x holds the initial guess and receives the
 * solution); the work is ordered on `stream` (cudaStream_t, NULL = legacy default stream) and
 * the call synchronises it before returning.  Every scratch array of the solver lives in one
 * fixed 6 MiB __device__ array of the library, which every GPU that loads the library holds
 * until the process exits; grids above 128 x 128 cells (or whose coarsest multigrid level
 * has more than 1024 cells) are rejected with EBIT_EINVAL.  The call makes no device
 * allocation.  The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents (the solver clears what must start at zero);
 * calls whose work overlaps on the GPU (two streams, two host threads) race on the array.
 * The paper has no counterpart: this is a deployment variant of the library's own solver. */
ebit_status ebit_solve_system_noalloc(int nx, int ny, const double* D, const double* wl, const double* wb,
                                      const double* b, double* x, int nr, int precision, double rtol, int max_iter,
                                      void* stream, int* iters, double* rel_res);

/* Autotuning of the multigrid schedule (the paper has no counterpart; a deployment feature of
 * the library's solver).  For every batch of instances sharing launches, and every instance
 * stepped alone, times `trial_steps` graph-replayed steps (after one untimed step) of each
 * candidate schedule and keeps the fastest:
 *   - the size of the largest level solved inside the single-block kernel: 256, 1024 or 4096
 *     cells, the values that change the level split of this grid;
 *   - the relative tolerance of the refinement's inner FP32 solves: 1e-4 or 1e-5 (mixed
 *     precision only);
 *   - TMA staging of the tile regions on or off (instances stepped alone);
 *   - the coarse tiled levels and the single-block levels in one cooperative launch (grid
 *     barriers between the phases) or one launch per level (instances stepped alone).
 * The state of every instance (fields, markers, time, step counter) is restored afterwards
 * from a device snapshot of the largest unit's arena, which is allocated with cudaMalloc for
 * the duration of the call.  Needs graph mode.  EBIT_ENOMEM when the snapshot does not fit. */
ebit_status ebit_autotune(ebit_ctx* ctx, int trial_steps);
/* The schedule an instance uses: single-block level size, inner tolerance, TMA staging,
 * cooperative launches (EBIT_OPT_COOP's values). */
ebit_status ebit_get_schedule(ebit_ctx* ctx, int inst, int* small_max, double* inner_rtol, int* tma, int* coop);

/* Options:
 *   EBIT_OPT_GRAPH (default 1) replays each step as a CUDA graph captured on the context's
 *   stream (solver loops as conditional WHILE nodes, no host round trip inside a step); 0
 *   launches every kernel from the host.  Graph mode needs a non-default stream.
 *   EBIT_OPT_TMA (default 1) stages the tile regions of the multigrid smoother kernels into
 *   shared memory with tensor-memory-accelerator copies (cp.async.bulk.tensor); 0 loads them
 *   with ordinary loads.  Both give the same values; levels whose rows or base are not 16-byte
 *   aligned always use ordinary loads.  Changing it drops the captured step graphs.
 *   EBIT_OPT_COOP (default 1) runs the coarse tiled levels of each V-cycle (those whose tiles
 *   fit one per co-resident block) and the single-block levels in one cooperative launch with
 *   grid barriers between the phases; 0 launches each level separately.  Both give the same
 *   values.  2 (mixed precision) runs each whole inner FP32 solve of the refinement, every
 *   V-cycle and CG update until the inner tolerance, in one cooperative launch with bounded
 *   grid barriers between its phases (grids whose finest tiles fit the reduction slots; others
 *   fall back to 1); its dot products are grouped per block, so the iterates agree with the
 *   other forms to rounding, not bit for bit (measured 10-30 % slower than 0 or 1 on 512^2 and
 *   1024x2048 grids, where its one block per SM and the spills of its 128 registers outweigh
 *   the saved launches).  Instances stepped in batches always launch each level separately.
 *   EBIT_OPT_BARRIER_SPIN (default 0 = 2^22 polls) bounds the wait of each grid barrier of the
 *   cooperative launch, in polls of the arrival counter.  A fault-path test setting: a bound of
 *   a few polls makes the barriers give up before the other blocks arrive.  Changing it drops
 *   the captured step graphs.
 *   EBIT_OPT_EXT_BLOCK (default 1 on grids of at most 2^19 cells, 0 above) runs every Jacobi
 *   sweep of a narrow-band extension (extrapolation equation, Sec. 2.4) in one thread block per
 *   instance; 0 launches one kernel per sweep over the whole device.  Both give the same values.
 *   Changing it drops the captured step graphs.
 * A tile kernel that waits for its copies in vain, or a grid barrier that waits in vain, gives
 * up after a bounded wait and records a fault; ebit_step, ebit_solve_system and
 * ebit_solve_system_noalloc then return EBIT_ECUDA: every result of that launch (not only of
 * the instance) is invalid, and the context should be destroyed. */
enum { EBIT_OPT_GRAPH = 1, EBIT_OPT_TMA = 2, EBIT_OPT_COOP = 3, EBIT_OPT_BARRIER_SPIN = 4,
       EBIT_OPT_EXT_BLOCK = 5 };
ebit_status ebit_set_option(ebit_ctx* ctx, int option, int value);

const char* ebit_last_error(const ebit_ctx* ctx);
void ebit_destroy(ebit_ctx* ctx);

/* Library version string. */
const char* ebit_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EBIT_H */
