// C ABI of the EBIT phase-change step: context, memory, stage orchestration.
// The time iteration follows Sec. 2.5 of arXiv 2402.13677 (see include/ebit.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/ebit.h"
#include "common.cuh"
#include "kernels.h"
#include "solver.h"
#include "status.h"

using namespace ebit;

namespace {

std::atomic<uint64_t> g_launches{0};

struct Instance {
    ebit_config cfg;
    Grid g;
    Phys p;
    bool props_set = false;
    // interface
    uint8_t *vcol, *vcol_n;
    double *hpos, *hpos_n, *vpos, *vpos_n, *hdisp, *vdisp;
    uint16_t* cseg;
    uint8_t* flags;
    double* vf;
    double2 *nb, *uG;
    // fields
    double *T_l, *T_v, *Ts_l, *Ts_v, *P, *mdot;
    double2 *u_l, *u_v, *us_l, *us_v, *gc;
    double *ufx_l, *ufx_v, *ufy_l, *ufy_v;
    // linear systems
    double *op_cd, *op_dd, *op_wl, *op_wb, *op_b, *op_x;
    double *op2_cd, *op2_dd, *op2_wl, *op2_wb;   // the second viscous component's operator
    double2 *vbx, *vby, *vxx, *vxy;   // viscous RHS / solutions, liquid and vapour interleaved
    // band compaction + extension values
    int *band_list, *band_count, *band_idx;
    int *near_list, *near_count, *near_mark;   // cells within two of the interface (the sweeps)
    double *ext[4];
    double *face_ax, *face_ay;   // face accelerations of the projection
    double* kap;                 // interface curvature of the cut cells (surface tension)
    // diagnostics and status
    double *diag_partial, *diag_out, *clock;
    unsigned* diag_ticket;
    int* status;
    Solver solver;
    Solver solver2;          // the second viscous component's solve (runs beside the first in graphs)
    cudaStream_t side = nullptr;   // capture branch of the second viscous solve (the context's)
    cudaEvent_t e_fork = nullptr, e_join = nullptr;   // its fork / join while capturing
    void* arena = nullptr;
    size_t arena_bytes = 0;
    double t0 = 0.0;
    long long nstep = 0;
    double stats[6] = {0, 0, 0, 0, 0, 0};   // iterations and residuals: energy, viscous, poisson
    bool noconv = false;
    bool fault = false;   // a multigrid kernel gave up a bounded wait (TMA copies, grid barrier)
    bool nonfinite = false;   // a solve met a NaN or an infinity
    // CUDA graphs of one step, per sweep-order parity
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_launches[2] = {0, 0};   // kernel launches captured per graph (loop bodies once)
    unsigned solved = 0;                     // solve slots written since the last statistics read
    int batch = -1;                          // batch this instance belongs to (-1: stepped alone)
    int bz = 0;                              // its index inside the batch
};

// Instances that share grid, boundary conditions and solver settings are stepped together when
// the context replays graphs: their arenas lie `stride` bytes apart in one allocation, and one
// graph of batched launches (grid z = instance) steps all of them; `lead` is a copy of the first
// member whose Grid and Solver carry the batch stride, count and the device array of properties.
struct Batch {
    std::vector<int> members;
    size_t stride = 0;
    void* arena = nullptr;
    Phys* d_phys = nullptr;
    std::vector<Phys> h_phys;
    Instance lead;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_launches[2] = {0, 0};
};

}  // namespace

struct ebit_ctx {
    std::vector<Instance> inst;
    cudaStream_t stream = nullptr;
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};   // capture streams of the solvers' loop bodies
    cudaStream_t side = nullptr;   // capture branch of the second viscous solve
    // batched steps: instance b replays its step graph on workers[b % workers.size()], between a
    // fork event recorded on the context stream and the workers' join events
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    int* host_status = nullptr;   // pinned, one status word per instance
    std::vector<Batch> batches;
    ebit_allocator alloc{};
    bool has_alloc = false;
    SolveState* host_states = nullptr;   // pinned, Solver::NSLOT per instance
    std::string err;
    uint64_t launch0 = 0;
    int use_graph = 1;
};

static ebit_status fail(ebit_ctx* ctx, ebit_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

static ebit_status cuda_check(ebit_ctx* ctx, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return EBIT_OK;
}

static size_t field_count(const Grid& g, int f, size_t* elem) {
    size_t N = (size_t)g.nx * g.ny;
    size_t nfx = (size_t)g.ny * (g.nx + 1), nfy = (size_t)(g.ny + 1) * g.nx;
    switch (f) {
        case EBIT_F_T_L: case EBIT_F_T_V: case EBIT_F_P: case EBIT_F_MDOT: case EBIT_F_VF:
        case EBIT_F_TSTAR_L: case EBIT_F_TSTAR_V:
            *elem = 8; return N;
        case EBIT_F_U_L: case EBIT_F_U_V: case EBIT_F_GC: case EBIT_F_NB: case EBIT_F_UG:
            *elem = 16; return N;
        case EBIT_F_UFX_L: case EBIT_F_UFX_V: case EBIT_F_VY_POS:
            *elem = 8; return nfx;
        case EBIT_F_UFY_L: case EBIT_F_UFY_V: case EBIT_F_HX_POS:
            *elem = 8; return nfy;
        case EBIT_F_CCOL: case EBIT_F_BAND:
            *elem = 1; return N;
        case EBIT_F_VCOL:
            *elem = 1; return (size_t)(g.nx + 1) * (g.ny + 1);
        case EBIT_F_CSEG:
            *elem = 2; return N;
        default:
            *elem = 0; return 0;
    }
}

static void* field_ptr(Instance& I, int f) {
    switch (f) {
        case EBIT_F_T_L: return I.T_l;
        case EBIT_F_T_V: return I.T_v;
        case EBIT_F_U_L: return I.u_l;
        case EBIT_F_U_V: return I.u_v;
        case EBIT_F_UFX_L: return I.ufx_l;
        case EBIT_F_UFX_V: return I.ufx_v;
        case EBIT_F_UFY_L: return I.ufy_l;
        case EBIT_F_UFY_V: return I.ufy_v;
        case EBIT_F_P: return I.P;
        case EBIT_F_GC: return I.gc;
        case EBIT_F_MDOT: return I.mdot;
        case EBIT_F_VF: return I.vf;
        case EBIT_F_NB: return I.nb;
        case EBIT_F_VCOL: return I.vcol;
        case EBIT_F_HX_POS: return I.hpos;
        case EBIT_F_VY_POS: return I.vpos;
        case EBIT_F_TSTAR_L: return I.Ts_l;
        case EBIT_F_TSTAR_V: return I.Ts_v;
        case EBIT_F_CSEG: return I.cseg;
        case EBIT_F_UG: return I.uG;
        default: return nullptr;
    }
}

// ---------------------------------------------------------------------------------------
// memory layout of one instance (single arena, 256-byte aligned pieces)
// ---------------------------------------------------------------------------------------
template <class F>
static size_t layout(Instance& I, char* base, F&& assign) {
    const Grid& g = I.g;
    size_t N = (size_t)g.nx * g.ny;
    size_t nv = (size_t)(g.nx + 1) * (g.ny + 1);
    size_t nh = (size_t)(g.ny + 1) * g.nx, nve = (size_t)g.ny * (g.nx + 1);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* r = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return r;
    };
    assign(I, take, N, nv, nh, nve);
    char* sb = take(Solver::bytes(g.nx, g.ny));
    if (base) I.solver.bind(sb, g.nx, g.ny, false);   // capture streams come from the context
    char* sb2 = take(Solver::bytes(g.nx, g.ny));
    if (base) I.solver2.bind(sb2, g.nx, g.ny, false);
    return off;
}

static void assign_ptrs(Instance& I, const std::function<char*(size_t)>& take, size_t N, size_t nv, size_t nh,
                        size_t nve) {
    I.vcol = (uint8_t*)take(nv);
    I.vcol_n = (uint8_t*)take(nv);
    I.hpos = (double*)take(nh * 8);
    I.hpos_n = (double*)take(nh * 8);
    I.vpos = (double*)take(nve * 8);
    I.vpos_n = (double*)take(nve * 8);
    I.hdisp = (double*)take(nh * 8);
    I.vdisp = (double*)take(nve * 8);
    I.cseg = (uint16_t*)take(N * 2);
    I.flags = (uint8_t*)take(N);
    I.vf = (double*)take(N * 8);
    I.nb = (double2*)take(N * 16);
    I.uG = (double2*)take(N * 16);
    I.T_l = (double*)take(N * 8);
    I.T_v = (double*)take(N * 8);
    I.Ts_l = (double*)take(N * 8);
    I.Ts_v = (double*)take(N * 8);
    I.P = (double*)take(N * 8);
    I.mdot = (double*)take(N * 8);
    I.u_l = (double2*)take(N * 16);
    I.u_v = (double2*)take(N * 16);
    I.us_l = (double2*)take(N * 16);
    I.us_v = (double2*)take(N * 16);
    I.gc = (double2*)take(N * 16);
    I.ufx_l = (double*)take(nve * 8);
    I.ufx_v = (double*)take(nve * 8);
    I.ufy_l = (double*)take(nh * 8);
    I.ufy_v = (double*)take(nh * 8);
    I.face_ax = (double*)take(nve * 8);
    I.face_ay = (double*)take(nh * 8);
    I.op_cd = (double*)take(N * 8);
    I.op_dd = (double*)take(N * 8);
    I.op_wl = (double*)take(N * 8);
    I.op_wb = (double*)take(N * 8);
    I.op_b = (double*)take(N * 8);
    I.op_x = (double*)take(N * 8);
    I.op2_cd = (double*)take(N * 8);
    I.op2_dd = (double*)take(N * 8);
    I.op2_wl = (double*)take(N * 8);
    I.op2_wb = (double*)take(N * 8);
    I.vbx = (double2*)take(N * 16);
    I.vby = (double2*)take(N * 16);
    I.vxx = (double2*)take(N * 16);
    I.vxy = (double2*)take(N * 16);
    I.band_list = (int*)take(N * 4);
    I.band_count = (int*)take(256);
    I.band_idx = (int*)take(N * 4);
    I.near_list = (int*)take(N * 4);
    I.near_count = (int*)take(256);
    I.near_mark = (int*)take(N * 4);   // zero between steps (the arena starts zeroed)
    for (int k = 0; k < 4; ++k) I.ext[k] = (double*)take(N * 8);
    I.kap = (double*)take(N * 8);
    I.diag_partial = (double*)take(8 * 8 * 1024);
    I.diag_out = (double*)take(64 * 8);
    I.clock = (double*)take(256);
    I.diag_ticket = (unsigned*)take(256);
    I.status = (int*)take(256);
}

// ---------------------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------------------
static void count(int n) { g_launches += (uint64_t)n; }

static void reconstruct_full(Instance& I, cudaStream_t st) {
    launch_reconstruct(I.g, I.vcol, I.hpos, I.vpos, I.cseg, I.flags, I.vf, st);
    launch_band(I.g, I.cseg, I.hpos, I.vpos, I.flags, I.nb, st);
    launch_compact(I.g, I.flags, I.g.nx * I.g.ny, F_BAND, I.band_list, I.band_count, I.band_idx, st);
    count(3);   // + memset
}

// kernels of one narrow-band extension: one in a single block per instance, else one per sweep
static int extend_launches(const Instance& I) { return I.g.ext_block ? 1 : I.p.extend_iters; }

static void extend_T(Instance& I, double* Tl, double* Tv, cudaStream_t st) {
    launch_extend_T(I.g, I.p.extend_iters, I.band_list, I.band_count, I.flags, I.band_idx, I.nb, Tl, Tv, I.ext, st);
    count(extend_launches(I));
}

static void mass_flux(Instance& I, cudaStream_t st) {
    launch_mass_flux(I.g, I.p, I.cseg, I.hpos, I.vpos, I.T_l, I.T_v, I.mdot, st);
    launch_extend(I.g, 2, I.p.extend_iters, I.band_list, I.band_count, I.flags, I.band_idx, I.nb, I.mdot, I.ext[0],
                  I.ext[1], st);
    count(1 + extend_launches(I));
}

static void ghost_velocity(Instance& I, cudaStream_t st) {
    if (I.p.one_fluid) return;   // one velocity field: no ghost values
    launch_ghost_velocity(I.g, I.p, I.band_list, I.band_count, I.flags, I.mdot, I.nb, I.vcol, I.hpos, I.vpos, I.u_l,
                          I.u_v, I.ufx_l, I.ufx_v, I.ufy_l, I.ufy_v, st);
    count(1);
}

// S2-S5 over the cells within two of the interface: the narrow band of the start-of-step
// geometry dilated by one cell, u_Gamma on those cells, the two sweeps, the reconstruction
static void advance_interface(Instance& I, cudaStream_t st) {
    launch_band_dilate(I.g, I.band_list, I.band_count, I.near_mark, I.near_list, I.near_count, st);
    launch_ug_list(I.g, I.p, I.near_list, I.near_count, I.flags, I.u_l, I.u_v, I.mdot, I.nb, I.uG, st);
    count(2);
    double dth = I.p.dt / I.g.h;
    int first = (I.cfg.sweep_order == 0 || (I.nstep % 2) == 0) ? 0 : 1;
    for (int k = 0; k < 2; ++k) {
        int axis = k == 0 ? first : 1 - first;
        if (k == 1) {
            launch_reconstruct_list(I.g, I.near_list, I.near_count, I.vcol, I.hpos, I.vpos, I.cseg, I.flags, nullptr,
                                    st);
            count(1);
        }
        launch_sweep(I.g, axis, dth, I.near_list, I.near_count, I.vcol, I.hpos, I.vpos, I.cseg, I.uG, I.hdisp,
                     I.vdisp, I.vcol_n, I.hpos_n, I.vpos_n, I.status, st);
        count(3);
        std::swap(I.vcol, I.vcol_n);
        std::swap(I.hpos, I.hpos_n);
        std::swap(I.vpos, I.vpos_n);
    }
    launch_band_unmark(I.g, I.near_list, I.near_count, I.near_mark, st);
    // S5 over the near list (the cells the sweeps can change) and its neighbours (the new band)
    launch_reconstruct_list(I.g, I.near_list, I.near_count, I.vcol, I.hpos, I.vpos, I.cseg, I.flags, I.vf, st);
    launch_band_list(I.g, I.near_list, I.near_count, I.cseg, I.hpos, I.vpos, I.flags, I.nb, st);
    launch_compact(I.g, I.flags, I.g.nx * I.g.ny, F_BAND, I.band_list, I.band_count, I.band_idx, st);
    count(3);   // + memset
}

enum { SLOT_ENERGY = 0, SLOT_VISC_X = 1, SLOT_VISC_Y = 2, SLOT_POISSON = 3 };

static void do_solve(Instance& I, int slot, const double* b, double* x, int nr, cudaStream_t st) {
    I.solver.slot = slot;
    I.solved |= 1u << slot;
    long long l0 = I.solver.launches;
    I.solver.solve(I.op_cd, I.op_dd, I.op_wl, I.op_wb, b, x, nr, I.cfg.precision, I.cfg.rtol, I.cfg.max_iter, st);
    count((int)(I.solver.launches - l0));
}

// the second viscous component on its own solver and operator arrays
static void do_solve2(Instance& I, int slot, const double* b, double* x, int nr, cudaStream_t st) {
    I.solver2.slot = slot;
    I.solved |= 1u << slot;
    long long l0 = I.solver2.launches;
    I.solver2.solve(I.op2_cd, I.op2_dd, I.op2_wl, I.op2_wb, b, x, nr, I.cfg.precision, I.cfg.rtol, I.cfg.max_iter,
                    st);
    count((int)(I.solver2.launches - l0));
}

// solver statistics of the last step from the host copy of the solver slots (fetched by
// check_status before its synchronisation)
static void collect_stats(Instance& I, bool graph_step) {
    unsigned m = I.solved;
    I.solved = 0;
    if (!m) return;
    SolveResult r[4];
    bool ok = true;
    long long body = I.solver.body_size(I.cfg.precision), n = 0;
    for (int k = 0; k < 4; ++k) {
        if (!(m & (1u << k))) continue;
        r[k] = (k == SLOT_VISC_Y ? I.solver2 : I.solver).result_from_host(k, I.cfg.precision);
        ok = ok && r[k].converged;
        if (r[k].fault) I.fault = true;
        if (r[k].nonfinite) I.nonfinite = true;
        // kernels executed inside the conditional loop bodies of a graph step
        n += r[k].iters * body;
        if (I.cfg.precision == EBIT_MIXED) n += 2 * r[k].outer - 1;
    }
    if (graph_step && I.bz == 0) g_launches += (uint64_t)n;   // a batched launch counts once
    if (m & (1u << SLOT_ENERGY)) {
        I.stats[0] = r[SLOT_ENERGY].iters;
        I.stats[3] = r[SLOT_ENERGY].rel_res;
    }
    if (m & (1u << SLOT_VISC_X)) {
        I.stats[1] = r[SLOT_VISC_X].iters + ((m & (1u << SLOT_VISC_Y)) ? r[SLOT_VISC_Y].iters : 0);
        double w = r[SLOT_VISC_X].rel_res;
        if ((m & (1u << SLOT_VISC_Y)) && r[SLOT_VISC_Y].rel_res > w) w = r[SLOT_VISC_Y].rel_res;
        I.stats[4] = w;
    }
    if (m & (1u << SLOT_POISSON)) {
        I.stats[2] = r[SLOT_POISSON].iters;
        I.stats[5] = r[SLOT_POISSON].rel_res;
    }
    if (!ok) I.noconv = true;
}

static void solve_energy(Instance& I, cudaStream_t st) {
    launch_energy_operator(I.g, I.p, I.flags, I.cseg, I.hpos, I.vpos, I.Ts_l, I.Ts_v, I.op_cd, I.op_dd, I.op_wl,
                           I.op_wb, I.op_b, I.op_x, st);
    count(1);
    do_solve(I, SLOT_ENERGY, I.op_b, I.op_x, 1, st);
    launch_split_T(I.g, I.flags, I.op_x, I.Ts_l, I.Ts_v, I.T_l, I.T_v, st);
    count(1);
}

static void momentum(Instance& I, cudaStream_t st) {
    // S11: predictor; one two-RHS solve (liquid, vapour) per velocity component
    launch_mom_rhs(I.g, I.p, I.vf, I.u_l, I.u_v, I.gc, I.vbx, I.vby, I.vxx, I.vxy, st);
    count(1);
    // the two components are independent: while capturing a graph the y solve becomes a
    // parallel branch (forked and joined through events on the side stream)
    // both components' operators in one pass (their cell and face terms are shared)
    launch_visc_operator(I.g, I.p, I.vf, I.op_cd, I.op_dd, I.op_wl, I.op_wb, I.op2_cd, I.op2_dd, I.op2_wl, I.op2_wb,
                         st);
    count(1);
    bool fork = I.solver.use_graph && I.side;
    cudaStream_t s2 = fork ? I.side : st;
    if (fork) {
        if (!I.e_fork) cudaEventCreateWithFlags(&I.e_fork, cudaEventDisableTiming);
        if (!I.e_join) cudaEventCreateWithFlags(&I.e_join, cudaEventDisableTiming);
        cudaEventRecord(I.e_fork, st);
        cudaStreamWaitEvent(s2, I.e_fork, 0);
        I.solver2.use_graph = 1;
    }
    do_solve(I, SLOT_VISC_X, (const double*)I.vbx, (double*)I.vxx, 2, st);
    do_solve2(I, SLOT_VISC_Y, (const double*)I.vby, (double*)I.vxy, 2, s2);
    if (fork) {
        cudaEventRecord(I.e_join, s2);
        cudaStreamWaitEvent(st, I.e_join, 0);
        I.solver2.use_graph = 0;
    }
    if (I.p.sigma > 0.0) {   // curvature of the new interface for the surface-tension force
        launch_curvature(I.g, I.flags, I.cseg, I.hpos, I.vpos, I.kap, st);
        count(1);
    }
    launch_ustar(I.g, I.p, I.vxx, I.vxy, I.gc, I.kap, I.vf, I.us_l, I.us_v, I.ufx_l, I.ufx_v, I.ufy_l, I.ufy_v, st);
    count(2);
    // S12: projection
    launch_poisson_operator(I.g, I.p, I.vf, I.flags, I.cseg, I.hpos, I.vpos, I.mdot, I.ufx_l, I.ufx_v, I.ufy_l,
                            I.ufy_v, I.op_cd, I.op_dd, I.op_wl, I.op_wb, I.op_b, st);
    count(1);
    do_solve(I, SLOT_POISSON, I.op_b, I.P, 1, st);
    launch_project(I.g, I.p, I.P, I.vf, I.kap, I.op_wl, I.op_wb, I.face_ax, I.face_ay, I.ufx_l, I.ufx_v, I.ufy_l,
                   I.ufy_v, I.gc, I.us_l, I.us_v, I.u_l, I.u_v, st);
    count(2);
}

static void diagnostics(Instance& I, cudaStream_t st) {
    launch_diagnostics(I.g, I.p, I.vf, I.cseg, I.hpos, I.vpos, I.mdot, I.flags, I.ufx_l, I.ufx_v, I.ufy_l, I.ufy_v,
                       I.T_l, I.T_v, I.diag_partial, I.diag_ticket, I.clock, I.diag_out, st);
    count(1);
    I.nstep += 1;
}

static void prepare(Instance& I, cudaStream_t st) {
    if (I.p.one_fluid) {   // the one velocity field is the liquid one; the vapour arrays repeat it
        size_t N = (size_t)I.g.nx * I.g.ny, nfx = (size_t)I.g.ny * (I.g.nx + 1), nfy = (size_t)(I.g.ny + 1) * I.g.nx;
        cudaMemcpyAsync(I.u_v, I.u_l, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(I.ufx_v, I.ufx_l, nfx * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(I.ufy_v, I.ufy_l, nfy * 8, cudaMemcpyDeviceToDevice, st);
    }
    reconstruct_full(I, st);
    if (I.p.energy) extend_T(I, I.T_l, I.T_v, st);
    mass_flux(I, st);
    ghost_velocity(I, st);
    if (I.p.sigma > 0.0) {
        launch_curvature(I.g, I.flags, I.cseg, I.hpos, I.vpos, I.kap, st);
        count(1);
    }
    launch_project(I.g, I.p, I.P, I.vf, I.kap, nullptr, nullptr, I.face_ax, I.face_ay, nullptr, nullptr, nullptr,
                   nullptr, I.gc, nullptr, nullptr, nullptr, nullptr, st);
    count(2);
}

static ebit_status run_stage(ebit_ctx* ctx, Instance& I, int stage) {
    cudaStream_t st = ctx->stream;
    switch (stage) {
        case EBIT_STAGE_PREPARE: prepare(I, st); break;
        case EBIT_STAGE_RECONSTRUCT: reconstruct_full(I, st); break;
        case EBIT_STAGE_ADVECT_T:
            if (I.p.energy) {
                launch_advect_T(I.g, I.p, I.flags, I.T_l, I.T_v, I.u_l, I.u_v, I.Ts_l, I.Ts_v, st);
                count(1);
            }
            break;
        case EBIT_STAGE_EXTEND_TSTAR:
            if (I.p.energy) extend_T(I, I.Ts_l, I.Ts_v, st);
            break;
        case EBIT_STAGE_ADVANCE_INTERFACE: advance_interface(I, st); break;
        case EBIT_STAGE_SOLVE_ENERGY:
            if (I.p.energy) solve_energy(I, st);
            break;
        case EBIT_STAGE_EXTEND_T:
            if (I.p.energy) extend_T(I, I.T_l, I.T_v, st);
            break;
        case EBIT_STAGE_MASS_FLUX: mass_flux(I, st); break;
        case EBIT_STAGE_GHOST_VELOCITY: ghost_velocity(I, st); break;
        case EBIT_STAGE_MOMENTUM: momentum(I, st); break;
        case EBIT_STAGE_DIAGNOSTICS: diagnostics(I, st); break;
        default: return fail(ctx, EBIT_EINVAL, "unknown stage");
    }
    return cuda_check(ctx, "run_stage");
}

// status and solver statistics of every instance: all read-backs are queued on the context
// stream, then one synchronisation
static ebit_status check_status(ebit_ctx* ctx, bool graph_step = false) {
    for (size_t b = 0; b < ctx->inst.size(); ++b) {
        Instance& I = ctx->inst[b];
        if (I.solved) I.solver.fetch_states(ctx->stream);
        if (I.solved & (1u << SLOT_VISC_Y)) I.solver2.fetch_states(ctx->stream);
        cudaMemcpyAsync(ctx->host_status + b, I.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(e));
    ebit_status worst = EBIT_OK;
    for (size_t b = 0; b < ctx->inst.size(); ++b) {
        Instance& I = ctx->inst[b];
        collect_stats(I, graph_step);
        int s = ctx->host_status[b];
        std::string where = ctx->inst.size() > 1 ? " (instance " + std::to_string(b) + ")" : "";
        if (s & 1) return fail(ctx, EBIT_ECFL, "a marker moved one cell or more in one sweep (reduce dt)" + where);
        if (s & 2) return fail(ctx, EBIT_ETOPO, "too many marker candidates on one edge" + where);
        if (I.fault) {
            I.fault = false;
            return fail(ctx, EBIT_ECUDA,
                        "a multigrid kernel gave up a bounded wait (TMA copies or grid barrier)" + where);
        }
        if (I.nonfinite) {
            I.nonfinite = false;
            I.noconv = false;
            return fail(ctx, EBIT_ENONFINITE, "a linear solve met a NaN or an infinity in the state" + where);
        }
        if (I.noconv) {
            I.noconv = false;
            worst = fail(ctx, EBIT_ENOCONV, "a linear solve hit max_iter" + where);
        }
    }
    return worst;
}

// grids up to this many cells run each narrow-band extension in one CTA per instance (their
// bands are a few thousand cells); larger ones launch one kernel per Jacobi sweep
constexpr long long EXT_BLOCK_MAX_CELLS = 1LL << 19;

// two configurations can share batched launches: the same grid, boundaries and solver settings
// (the time step and the properties may differ)
static bool batchable(const ebit_config& a, const ebit_config& b) {
    if (a.nx != b.nx || a.ny != b.ny || a.h != b.h || a.x0 != b.x0 || a.y0 != b.y0) return false;
    for (int s = 0; s < 4; ++s)
        if (a.bc[s] != b.bc[s] || a.T_fixed[s] != b.T_fixed[s] || a.T_wall[s] != b.T_wall[s]) return false;
    return a.precision == b.precision && a.rtol == b.rtol && a.max_iter == b.max_iter &&
           a.extend_iters == b.extend_iters && a.theta_min == b.theta_min && a.sweep_order == b.sweep_order &&
           a.energy == b.energy && a.mdot_fixed == b.mdot_fixed && a.one_fluid == b.one_fluid &&
           a.axisymmetric == b.axisymmetric;
}

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

const char* ebit_version(void) { return "ebit-gb300 0.1 (sm_103a)"; }

ebit_status ebit_init(const ebit_config* cfgs, int batch, void* stream, const ebit_allocator* alloc, ebit_ctx** out) {
    if (!out || !cfgs || batch < 1) return EBIT_EINVAL;
    *out = nullptr;
    ebit_ctx* ctx = new ebit_ctx();
    ctx->stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc_fn) { ctx->alloc = *alloc; ctx->has_alloc = true; }
    ctx->inst.resize(batch);
    for (int b = 0; b < batch; ++b) {
        const ebit_config& c = cfgs[b];
        if (c.nx < 4 || c.ny < 4 || (long long)c.nx * c.ny > (1LL << 29) || !(c.h > 0) || !(c.dt > 0) ||
            c.extend_iters < 2 || c.extend_iters > 64 ||
            c.max_iter < 1 || !(c.rtol > 0) || (c.precision != EBIT_FP64 && c.precision != EBIT_MIXED)) {
            delete ctx;
            return EBIT_EINVAL;
        }
        for (int s = 0; s < 4; ++s)
            if (c.bc[s] < 0 || c.bc[s] > 2) { delete ctx; return EBIT_EINVAL; }
        if (!Solver::supported(c.nx, c.ny)) { delete ctx; return EBIT_EINVAL; }
        if (c.axisymmetric && (!(c.x0 >= 0.0) || (c.x0 == 0.0 && c.bc[0] != EBIT_BC_SYMMETRY))) {
            delete ctx;
            return EBIT_EINVAL;
        }
        Instance& I = ctx->inst[b];
        I.cfg = c;
        I.g.nx = c.nx; I.g.ny = c.ny; I.g.h = c.h; I.g.x0 = c.x0; I.g.y0 = c.y0; I.g.inv_h = 1.0 / c.h;
        I.g.axi = c.axisymmetric ? 1 : 0; I.g.r0 = c.x0 / c.h;
        I.g.ext_block = (long long)c.nx * c.ny <= EXT_BLOCK_MAX_CELLS ? 1 : 0;
        I.g.nz = 1; I.g.zs = 0; I.g.pz = nullptr;
        for (int s = 0; s < 4; ++s) {
            I.g.bc[s] = c.bc[s];
            I.g.Tfix[s] = c.T_fixed[s] ? 1 : 0;
            I.g.Tw[s] = c.T_wall[s];
        }
        std::memset(&I.p, 0, sizeof(I.p));
        I.p.dt = c.dt; I.p.theta_min = c.theta_min; I.p.extend_iters = c.extend_iters;
        I.p.energy = c.energy; I.p.mdot_fixed = c.mdot_fixed; I.p.one_fluid = c.one_fluid ? 1 : 0;
        phys_derive(I.p);
    }
    // group instances that can share batched launches (same grid, boundaries and solver settings)
    std::vector<int> group(batch, -1);
    std::vector<std::vector<int>> groups;
    for (int b = 0; b < batch; ++b) {
        if (group[b] >= 0) continue;
        group[b] = (int)groups.size();
        groups.push_back({b});
        for (int b2 = b + 1; b2 < batch; ++b2)
            if (group[b2] < 0 && batchable(cfgs[b], cfgs[b2])) {
                group[b2] = group[b];
                groups.back().push_back(b2);
            }
    }
    for (auto& gm : groups) {
        Instance& I0 = ctx->inst[gm[0]];
        size_t bytes = (layout(I0, nullptr, assign_ptrs) + 255) & ~size_t(255);
        size_t total = bytes * gm.size();
        void* mem = nullptr;
        if (ctx->has_alloc) mem = ctx->alloc.alloc_fn(total, ctx->alloc.user);
        else if (cudaMalloc(&mem, total) != cudaSuccess) mem = nullptr;
        if (!mem) { ebit_destroy(ctx); return EBIT_ENOMEM; }
        for (size_t z = 0; z < gm.size(); ++z) {
            Instance& I = ctx->inst[gm[z]];
            I.arena_bytes = bytes;
            layout(I, (char*)mem + z * bytes, assign_ptrs);
        }
        cudaMemsetAsync(mem, 0, total, ctx->stream);
        if (gm.size() == 1) {
            I0.arena = mem;
            continue;
        }
        Batch B;
        B.members = gm;
        B.stride = bytes;
        B.arena = mem;
        B.h_phys.resize(gm.size());
        if (cudaMalloc(&B.d_phys, gm.size() * sizeof(Phys)) != cudaSuccess) {
            ctx->batches.push_back(B);
            ebit_destroy(ctx);
            return EBIT_ENOMEM;
        }
        for (size_t z = 0; z < gm.size(); ++z) {
            ctx->inst[gm[z]].batch = (int)ctx->batches.size();
            ctx->inst[gm[z]].bz = (int)z;
        }
        ctx->batches.push_back(B);
    }
    if (cudaMallocHost(&ctx->host_states, 2 * batch * Solver::NSLOT * sizeof(SolveState)) != cudaSuccess ||
        cudaMallocHost(&ctx->host_status, batch * sizeof(int)) != cudaSuccess) {
        ebit_destroy(ctx);
        return EBIT_ENOMEM;
    }
    for (int k = 0; k < 3; ++k) cudaStreamCreateWithFlags(&ctx->aux[k], cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    for (int b = 0; b < batch; ++b) {
        Instance& I = ctx->inst[b];
        I.solver.st_host = ctx->host_states + b * Solver::NSLOT;
        I.solver2.st_host = ctx->host_states + (batch + b) * Solver::NSLOT;
        for (int k = 0; k < 3; ++k) I.solver.aux[k] = I.solver2.aux[k] = ctx->aux[k];
        I.side = ctx->side;
    }
    ctx->launch0 = g_launches.load();
    ebit_status s = cuda_check(ctx, "ebit_init");
    if (s != EBIT_OK) { ebit_destroy(ctx); return s; }
    *out = ctx;
    return EBIT_OK;
}

ebit_status ebit_set_phase_props(ebit_ctx* ctx, int inst, const ebit_phase_props* liq, const ebit_phase_props* vap,
                                 double T_sat, double h_lg, double sigma, double gx, double gy) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !liq || !vap) return fail(ctx, EBIT_EINVAL, "bad args");
    if (!(sigma >= 0.0) || !std::isfinite(sigma)) return fail(ctx, EBIT_EINVAL, "sigma must be finite and >= 0");
    if (!(liq->rho > 0 && vap->rho > 0 && liq->lambda > 0 && vap->lambda > 0 && liq->cp > 0 && vap->cp > 0 &&
          liq->mu > 0 && vap->mu > 0 && h_lg != 0.0))
        return fail(ctx, EBIT_EINVAL, "properties must be positive");
    Instance& I = ctx->inst[inst];
    Phys& p = I.p;
    // whether the step computes a curvature is decided when its graph is captured: a change
    // between no surface tension and some drops the captured graphs of the instance (or batch)
    if (I.props_set && (p.sigma > 0.0) != (sigma > 0.0)) {
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto& gx : I.graph)
            if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        if (I.batch >= 0)
            for (auto& gx : ctx->batches[I.batch].graph)
                if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
    }
    p.rho_l = liq->rho; p.mu_l = liq->mu; p.lam_l = liq->lambda; p.cp_l = liq->cp;
    p.rho_v = vap->rho; p.mu_v = vap->mu; p.lam_v = vap->lambda; p.cp_v = vap->cp;
    phys_derive(p);
    p.T_sat = T_sat; p.h_lg = h_lg; p.gx = gx; p.gy = gy; p.sigma = sigma;
    I.props_set = true;
    return EBIT_OK;
}

ebit_status ebit_set_interface(ebit_ctx* ctx, int inst, const uint8_t* vcol, const double* hx_pos,
                               const double* vy_pos, int on_device) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !vcol || !hx_pos || !vy_pos)
        return fail(ctx, EBIT_EINVAL, "bad args");
    Instance& I = ctx->inst[inst];
    const Grid& g = I.g;
    size_t nv = (size_t)(g.nx + 1) * (g.ny + 1), nh = (size_t)(g.ny + 1) * g.nx, nve = (size_t)g.ny * (g.nx + 1);
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!on_device) {
        // validated on the device: the upload lands in the sweep scratch arrays, is checked there
        // (colours 0/1, cut fractions inside [FMIN, 1 - FMIN]; uncut fractions zeroed) and only
        // then replaces the instance's interface, so a rejected upload leaves it unchanged
        int* err = I.status + 32;
        cudaMemcpyAsync(I.vcol_n, vcol, nv, k, ctx->stream);
        cudaMemcpyAsync(I.hpos_n, hx_pos, nh * 8, k, ctx->stream);
        cudaMemcpyAsync(I.vpos_n, vy_pos, nve * 8, k, ctx->stream);
        cudaMemsetAsync(err, 0, sizeof(int), ctx->stream);
        launch_check_interface(g, I.vcol_n, I.hpos_n, I.vpos_n, err, ctx->stream);
        int herr = 0;
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t ce = cudaStreamSynchronize(ctx->stream);
        if (ce != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(ce));
        if (herr & 1) return fail(ctx, EBIT_EINVAL, "vertex colours must be 0 or 1");
        if (herr & 2) return fail(ctx, EBIT_ETOPO, "cut edge with a marker fraction outside [1e-9, 1-1e-9]");
        cudaMemcpyAsync(I.vcol, I.vcol_n, nv, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemcpyAsync(I.hpos, I.hpos_n, nh * 8, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemcpyAsync(I.vpos, I.vpos_n, nve * 8, cudaMemcpyDeviceToDevice, ctx->stream);
    } else {
        cudaMemcpyAsync(I.vcol, vcol, nv, k, ctx->stream);
        cudaMemcpyAsync(I.hpos, hx_pos, nh * 8, k, ctx->stream);
        cudaMemcpyAsync(I.vpos, vy_pos, nve * 8, k, ctx->stream);
    }
    return cuda_check(ctx, "ebit_set_interface");
}

ebit_status ebit_field_shape(const ebit_ctx* ctx, int inst, int field, size_t* count_out, size_t* elem_bytes) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !count_out || !elem_bytes) return EBIT_EINVAL;
    size_t e;
    size_t n = field_count(ctx->inst[inst].g, field, &e);
    if (!n) return EBIT_EINVAL;
    *count_out = n;
    *elem_bytes = e;
    return EBIT_OK;
}

ebit_status ebit_set_field(ebit_ctx* ctx, int inst, int field, const void* src, int on_device) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !src) return fail(ctx, EBIT_EINVAL, "bad args");
    if (field == EBIT_F_VF || field == EBIT_F_CCOL || field == EBIT_F_BAND || field == EBIT_F_NB ||
        field == EBIT_F_CSEG || field == EBIT_F_UG)
        return fail(ctx, EBIT_EINVAL, "field is derived (read only)");
    Instance& I = ctx->inst[inst];
    size_t e;
    size_t n = field_count(I.g, field, &e);
    void* dst = field_ptr(I, field);
    if (!n || !dst) return fail(ctx, EBIT_EINVAL, "unknown field");
    cudaMemcpyAsync(dst, src, n * e, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
    if (!on_device) cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, "ebit_set_field");
}

ebit_status ebit_get_field(ebit_ctx* ctx, int inst, int field, void* dst, int on_device) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !dst) return fail(ctx, EBIT_EINVAL, "bad args");
    Instance& I = ctx->inst[inst];
    size_t e;
    size_t n = field_count(I.g, field, &e);
    if (!n) return fail(ctx, EBIT_EINVAL, "unknown field");
    if (field == EBIT_F_CCOL || field == EBIT_F_BAND) {
        std::vector<uint8_t> fl(n);
        cudaMemcpyAsync(fl.data(), I.flags, n, cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t er = cudaStreamSynchronize(ctx->stream);
        if (er != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(er));
        uint8_t mask = field == EBIT_F_CCOL ? F_CCOL : F_BAND;
        for (size_t k = 0; k < n; ++k) fl[k] = (fl[k] & mask) ? 1 : 0;
        if (on_device) cudaMemcpy(dst, fl.data(), n, cudaMemcpyHostToDevice);
        else std::memcpy(dst, fl.data(), n);
        return cuda_check(ctx, "ebit_get_field");
    }
    cudaMemcpyAsync(dst, field_ptr(I, field), n * e, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                    ctx->stream);
    cudaError_t er = cudaStreamSynchronize(ctx->stream);
    if (er != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(er));
    return cuda_check(ctx, "ebit_get_field");
}

ebit_status ebit_set_fields(ebit_ctx* ctx, int inst, int n, const int* ids, const void* const* srcs,
                            int on_device) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || n < 0 || (n > 0 && (!ids || !srcs)))
        return fail(ctx, EBIT_EINVAL, "bad args");
    Instance& I = ctx->inst[inst];
    for (int k = 0; k < n; ++k) {
        int f = ids[k];
        size_t e;
        if (f == EBIT_F_VF || f == EBIT_F_CCOL || f == EBIT_F_BAND || f == EBIT_F_NB || f == EBIT_F_CSEG ||
            f == EBIT_F_UG || !srcs[k] || !field_count(I.g, f, &e) || !field_ptr(I, f))
            return fail(ctx, EBIT_EINVAL, "ebit_set_fields: entry " + std::to_string(k) + " is not a writable field");
    }
    for (int k = 0; k < n; ++k) {
        size_t e;
        size_t cnt = field_count(I.g, ids[k], &e);
        cudaMemcpyAsync(field_ptr(I, ids[k]), srcs[k], cnt * e,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
    }
    if (!on_device) cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, "ebit_set_fields");
}

ebit_status ebit_get_fields(ebit_ctx* ctx, int inst, int n, const int* ids, void* const* dsts, int on_device) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || n < 0 || (n > 0 && (!ids || !dsts)))
        return fail(ctx, EBIT_EINVAL, "bad args");
    Instance& I = ctx->inst[inst];
    for (int k = 0; k < n; ++k) {
        int f = ids[k];
        size_t e;
        if (f == EBIT_F_CCOL || f == EBIT_F_BAND || !dsts[k] || !field_count(I.g, f, &e) || !field_ptr(I, f))
            return fail(ctx, EBIT_EINVAL, "ebit_get_fields: entry " + std::to_string(k) + " is not a readable field");
    }
    for (int k = 0; k < n; ++k) {
        size_t e;
        size_t cnt = field_count(I.g, ids[k], &e);
        cudaMemcpyAsync(dsts[k], field_ptr(I, ids[k]), cnt * e,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream);
    }
    cudaError_t er = cudaStreamSynchronize(ctx->stream);
    if (er != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(er));
    return cuda_check(ctx, "ebit_get_fields");
}

ebit_status ebit_set_time(ebit_ctx* ctx, int inst, double t) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size()) return EBIT_EINVAL;
    Instance& I = ctx->inst[inst];
    double c[2] = {t, 0.0};
    cudaMemcpyAsync(I.clock, c, sizeof(c), cudaMemcpyHostToDevice, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    I.nstep = 0;
    return cuda_check(ctx, "ebit_set_time");
}

ebit_status ebit_run_stage(ebit_ctx* ctx, int stage) {
    if (!ctx) return EBIT_EINVAL;
    for (auto& I : ctx->inst) {
        if (!I.props_set) return fail(ctx, EBIT_EINVAL, "ebit_set_phase_props not called");
        ebit_status s = run_stage(ctx, I, stage);
        if (s != EBIT_OK) return s;
    }
    return check_status(ctx);
}

static ebit_status step_eager(ebit_ctx* ctx, Instance& I) {
    for (int s = EBIT_STAGE_ADVECT_T; s <= EBIT_STAGE_DIAGNOSTICS; ++s) {
        ebit_status r = run_stage(ctx, I, s);
        if (r != EBIT_OK) return r;
    }
    return EBIT_OK;
}

// capture one whole step (stages ADVECT_T .. DIAGNOSTICS) into a graph; the solver loops
// become conditional WHILE nodes, so replaying the graph needs no host round trip
static ebit_status capture_step(ebit_ctx* ctx, Instance& I, cudaStream_t st, cudaGraphExec_t* out) {
    if (!st) return fail(ctx, EBIT_EINVAL, "graph mode needs a non-default stream");
    long long nstep = I.nstep;
    uint64_t l0 = g_launches.load();
    cudaGraph_t g;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return fail(ctx, EBIT_ECUDA, "cudaStreamBeginCapture failed");
    I.solver.use_graph = 1;
    cudaStream_t s = st;
    if (I.p.energy) {
        launch_advect_T(I.g, I.p, I.flags, I.T_l, I.T_v, I.u_l, I.u_v, I.Ts_l, I.Ts_v, s);
        extend_T(I, I.Ts_l, I.Ts_v, s);
    }
    advance_interface(I, s);
    if (I.p.energy) {
        solve_energy(I, s);
        extend_T(I, I.T_l, I.T_v, s);
    }
    mass_flux(I, s);
    ghost_velocity(I, s);
    momentum(I, s);
    diagnostics(I, s);
    I.solver.use_graph = 0;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    I.nstep = nstep;
    int par = (I.cfg.sweep_order == 0) ? 0 : (int)(nstep & 1);
    I.graph_launches[par] = (long long)(g_launches.load() - l0);
    g_launches -= (g_launches.load() - l0);   // counted at launch time instead
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return EBIT_OK;
}

// replay (capturing it first if needed) one instance's step graph on stream st
static ebit_status replay_step(ebit_ctx* ctx, Instance& I, cudaStream_t st) {
    int par = (I.cfg.sweep_order == 0) ? 0 : (int)(I.nstep & 1);
    if (!I.graph[par]) {
        ebit_status r = capture_step(ctx, I, st, &I.graph[par]);
        if (r != EBIT_OK) return r;
    }
    cudaGraphLaunch(I.graph[par], st);
    g_launches += (uint64_t)I.graph_launches[par];
    I.solved = (I.p.energy ? 1u : 0u) | 2u | 4u | 8u;
    I.nstep += 1;
    return EBIT_OK;
}

// a batch of instances: up to MAX_WORKERS instances run concurrently, each on a worker stream
// forked from the context stream and joined back before the status check
// (a process that sets CUDA_DEVICE_MAX_CONNECTIONS=32 before creating its CUDA context gives
// each of them its own hardware queue)
static constexpr int MAX_WORKERS = 32;

static ebit_status ensure_workers(ebit_ctx* ctx) {
    if (!ctx->workers.empty()) return EBIT_OK;
    int k = (int)ctx->inst.size() < MAX_WORKERS ? (int)ctx->inst.size() : MAX_WORKERS;
    ctx->workers.resize(k);
    ctx->joins.resize(k);
    for (int w = 0; w < k; ++w) {
        cudaStreamCreateWithFlags(&ctx->workers[w], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&ctx->joins[w], cudaEventDisableTiming);
    }
    cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
    return cuda_check(ctx, "worker streams");
}

// one step of a batch: refresh the members' properties on the device, capture the batched graph
// of the lead on first use, replay it on stream st
static ebit_status replay_batch(ebit_ctx* ctx, Batch& B, cudaStream_t st) {
    Instance& I0 = ctx->inst[B.members[0]];
    if (B.lead.batch < 0 || B.lead.g.nz == 1) {
        B.lead = I0;
        B.lead.g.nz = (int)B.members.size();
        B.lead.g.zs = (long long)B.stride;
        B.lead.g.pz = B.d_phys;
        for (Solver* sv : {&B.lead.solver, &B.lead.solver2}) {
            sv->nz = (int)B.members.size();
            sv->zs = (long long)B.stride;
            sv->use_tma = 0;    // descriptors hold one instance's addresses
            sv->use_coop = 0;   // a grid barrier per member would not fit one cooperative grid
        }
    }
    double smax = 0.0;
    for (size_t z = 0; z < B.members.size(); ++z) {
        B.h_phys[z] = ctx->inst[B.members[z]].p;
        smax = std::max(smax, B.h_phys[z].sigma);
    }
    B.lead.p.sigma = smax;   // launches the curvature kernel if any member has surface tension
    cudaMemcpyAsync(B.d_phys, B.h_phys.data(), B.h_phys.size() * sizeof(Phys), cudaMemcpyHostToDevice, st);
    B.lead.nstep = I0.nstep;
    int par = (I0.cfg.sweep_order == 0) ? 0 : (int)(I0.nstep & 1);
    if (!B.graph[par]) {
        ebit_status r = capture_step(ctx, B.lead, st, &B.graph[par]);
        if (r != EBIT_OK) return r;
        B.graph_launches[par] = B.lead.graph_launches[par];
    }
    cudaGraphLaunch(B.graph[par], st);
    g_launches += (uint64_t)B.graph_launches[par];
    for (int m : B.members) {
        Instance& I = ctx->inst[m];
        I.solved = (I.p.energy ? 1u : 0u) | 2u | 4u | 8u;
        I.nstep += 1;
    }
    return EBIT_OK;
}

ebit_status ebit_step(ebit_ctx* ctx, int nsteps) {
    if (!ctx || nsteps < 0) return EBIT_EINVAL;
    for (auto& I : ctx->inst)
        if (!I.props_set) return fail(ctx, EBIT_EINVAL, "ebit_set_phase_props not called");
    bool graph = ctx->use_graph && ctx->stream;
    bool batched = graph && ctx->inst.size() > 1;
    if (batched) {
        ebit_status r = ensure_workers(ctx);
        if (r != EBIT_OK) return r;
    }
    ebit_status worst = EBIT_OK;
    for (int n = 0; n < nsteps; ++n) {
        if (batched) {
            // batches and the instances stepped alone, round-robin over the worker streams
            int K = (int)ctx->workers.size(), w = 0;
            cudaEventRecord(ctx->fork, ctx->stream);
            for (int k = 0; k < K; ++k) cudaStreamWaitEvent(ctx->workers[k], ctx->fork, 0);
            for (auto& B : ctx->batches) {
                ebit_status r = replay_batch(ctx, B, ctx->workers[w++ % K]);
                if (r != EBIT_OK) return r;
            }
            for (auto& I : ctx->inst) {
                if (I.batch >= 0) continue;
                ebit_status r = replay_step(ctx, I, ctx->workers[w++ % K]);
                if (r != EBIT_OK) return r;
            }
            for (int k = 0; k < K; ++k) {
                cudaEventRecord(ctx->joins[k], ctx->workers[k]);
                cudaStreamWaitEvent(ctx->stream, ctx->joins[k], 0);
            }
        } else {
            for (auto& I : ctx->inst) {
                ebit_status r = graph ? replay_step(ctx, I, ctx->stream) : step_eager(ctx, I);
                if (r != EBIT_OK) return r;
            }
        }
        ebit_status s = check_status(ctx, graph);
        if (s == EBIT_ENOCONV) worst = s;
        else if (s != EBIT_OK) return s;
    }
    return worst;
}

// ---- autotuning of the multigrid schedule ------------------------------------------------
// A unit is a batch or an instance stepped alone; its arena, step counter and schedule.
struct Unit {
    std::vector<int> members;
    Batch* batch = nullptr;
    char* arena = nullptr;
    size_t bytes = 0;
};

static void apply_schedule(ebit_ctx* ctx, Unit& U, int small_max, double inner, int tma, int coop) {
    auto set = [&](Instance& I) {
        for (Solver* sv : {&I.solver, &I.solver2}) {
            sv->set_schedule(small_max, inner);
            sv->use_tma = tma;
            sv->use_coop = coop;
        }
        for (auto& gx : I.graph)
            if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
    };
    for (int m : U.members) set(ctx->inst[m]);
    if (U.batch) {
        for (auto& gx : U.batch->graph)
            if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        U.batch->lead.batch = -1;   // rebuilt from the first member on the next replay
    }
}

// one step of the unit on the context stream, with the status check of its members
static ebit_status step_unit(ebit_ctx* ctx, Unit& U) {
    ebit_status r = U.batch ? replay_batch(ctx, *U.batch, ctx->stream)
                            : replay_step(ctx, ctx->inst[U.members[0]], ctx->stream);
    if (r != EBIT_OK) return r;
    return check_status(ctx, true);
}

ebit_status ebit_autotune(ebit_ctx* ctx, int trial_steps) {
    if (!ctx || trial_steps < 1) return EBIT_EINVAL;
    if (!ctx->use_graph || !ctx->stream) return fail(ctx, EBIT_EINVAL, "autotuning times graph replays (graph mode)");
    for (auto& I : ctx->inst)
        if (!I.props_set) return fail(ctx, EBIT_EINVAL, "ebit_set_phase_props not called");
    std::vector<Unit> units;
    for (auto& B : ctx->batches) {
        Unit U;
        U.members = B.members;
        U.batch = &B;
        U.arena = (char*)B.arena;
        U.bytes = B.stride * B.members.size();
        units.push_back(U);
    }
    for (size_t b = 0; b < ctx->inst.size(); ++b) {
        Instance& I = ctx->inst[b];
        if (I.batch >= 0) continue;
        Unit U;
        U.members = {(int)b};
        U.arena = (char*)I.arena;
        U.bytes = I.arena_bytes;
        units.push_back(U);
    }
    size_t most = 0;
    for (auto& U : units) most = U.bytes > most ? U.bytes : most;
    void* snap = nullptr;
    if (cudaMalloc(&snap, most) != cudaSuccess) return fail(ctx, EBIT_ENOMEM, "no room for the autotuning snapshot");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ebit_status status = EBIT_OK;
    for (auto& U : units) {
        Instance& I0 = ctx->inst[U.members[0]];
        std::vector<long long> nstep0;
        for (int m : U.members) nstep0.push_back(ctx->inst[m].nstep);
        cudaMemcpyAsync(snap, U.arena, U.bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        auto restore = [&]() {
            cudaMemcpyAsync(U.arena, snap, U.bytes, cudaMemcpyDeviceToDevice, ctx->stream);
            for (size_t z = 0; z < U.members.size(); ++z) ctx->inst[U.members[z]].nstep = nstep0[z];
        };
        // candidates: single-block threshold x inner tolerance (mixed) x TMA staging (alone)
        std::vector<int> smalls;
        int last_nbig = -1;
        for (int sm : {256, 1024, 4096}) {
            Solver probe = I0.solver;
            probe.set_schedule(sm, 1e-5);
            if (probe.nbig_f != last_nbig) { smalls.push_back(sm); last_nbig = probe.nbig_f; }
        }
        std::vector<double> inners = I0.cfg.precision == EBIT_MIXED ? std::vector<double>{1e-4, 1e-5}
                                                                    : std::vector<double>{1e-5};
        std::vector<int> tmas = U.batch ? std::vector<int>{0} : std::vector<int>{1, 0};
        // cooperative launches: none or the coarse part of each V-cycle (a whole inner solve in
        // one launch measured slower at 512^2 and 1024x2048 and is not a candidate); batched
        // instances launch every kernel per level
        std::vector<int> coops = U.batch ? std::vector<int>{0} : std::vector<int>{1, 0};
        float best = 1e30f;
        int bs = I0.solver.small_max_f, bt = I0.solver.use_tma, bc = I0.solver.use_coop;
        double bi = I0.solver.inner_rtol;
        for (int sm : smalls)
            for (double in : inners)
                for (int tm : tmas)
                for (int co : coops) {
                    apply_schedule(ctx, U, sm, in, tm, co);
                    restore();
                    ebit_status r = step_unit(ctx, U);   // captures the graphs, warms up
                    if (r == EBIT_OK || r == EBIT_ENOCONV) {
                        cudaEventRecord(e0, ctx->stream);
                        for (int k = 0; k < trial_steps && (r == EBIT_OK || r == EBIT_ENOCONV); ++k)
                            r = U.batch ? replay_batch(ctx, *U.batch, ctx->stream)
                                        : replay_step(ctx, I0, ctx->stream);
                        cudaEventRecord(e1, ctx->stream);
                        ebit_status c = check_status(ctx, true);
                        float ms = 0.0f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if ((r == EBIT_OK || r == EBIT_ENOCONV) && c == EBIT_OK && ms < best) {
                            best = ms;
                            bs = sm;
                            bi = in;
                            bt = tm;
                            bc = co;
                        }
                    }
                }
        apply_schedule(ctx, U, bs, bi, bt, bc);
        restore();
        cudaStreamSynchronize(ctx->stream);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    if (status == EBIT_OK) status = cuda_check(ctx, "ebit_autotune");
    return status;
}

ebit_status ebit_get_schedule(ebit_ctx* ctx, int inst, int* small_max, double* inner_rtol, int* tma, int* coop) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !small_max || !inner_rtol || !tma || !coop)
        return EBIT_EINVAL;
    const Solver& s = ctx->inst[inst].solver;
    *small_max = s.small_max_f;
    *inner_rtol = s.inner_rtol;
    *tma = s.use_tma;
    *coop = s.use_coop;
    return EBIT_OK;
}

ebit_status ebit_solve_system(ebit_ctx* ctx, int inst, const double* D, const double* wl, const double* wb,
                              const double* b, double* x, int nr, int precision, double rtol, int max_iter,
                              int* iters, double* rel_res) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !D || !wl || !wb || !b || !x || (nr != 1 && nr != 2) ||
        (precision != EBIT_FP64 && precision != EBIT_MIXED) || !(rtol > 0) || max_iter < 1)
        return fail(ctx, EBIT_EINVAL, "bad args");
    Instance& I = ctx->inst[inst];
    size_t N = (size_t)I.g.nx * I.g.ny;
    cudaStream_t st = ctx->stream;
    // host operands -> the instance's operator arrays (cd = D, dd = 0) and viscous vectors
    cudaMemcpyAsync(I.op_cd, D, N * 8, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(I.op_dd, 0, N * 8, st);
    cudaMemcpyAsync(I.op_wl, wl, N * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(I.op_wb, wb, N * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(I.vbx, b, N * 8 * nr, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(I.vxx, x, N * 8 * nr, cudaMemcpyHostToDevice, st);
    I.solver.slot = 4;
    I.solver.use_graph = 0;
    long long l0 = I.solver.launches;
    I.solver.solve(I.op_cd, I.op_dd, I.op_wl, I.op_wb, (const double*)I.vbx, (double*)I.vxx, nr, precision, rtol,
                   max_iter, st);
    count((int)(I.solver.launches - l0));
    cudaError_t e = cudaSuccess;
    SolveResult r = I.solver.read_result(4, precision, st, &e);
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(e));
    cudaMemcpyAsync(x, I.vxx, N * 8 * nr, cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(e));
    if (iters) *iters = r.iters;
    if (rel_res) *rel_res = r.rel_res;
    ebit_status s = cuda_check(ctx, "ebit_solve_system");
    if (s != EBIT_OK) return s;
    s = solve_status(true, r.fault, r.nonfinite, r.converged);
    if (s == EBIT_ECUDA)
        return fail(ctx, s, "ebit_solve_system: a multigrid kernel gave up a bounded wait (result invalid)");
    if (s == EBIT_ENONFINITE) return fail(ctx, s, "ebit_solve_system: a NaN or an infinity in the system");
    if (s == EBIT_ENOCONV) return fail(ctx, s, "ebit_solve_system: max_iter reached");
    return EBIT_OK;
}

ebit_status ebit_set_option(ebit_ctx* ctx, int option, int value) {
    if (!ctx) return EBIT_EINVAL;
    if (option == EBIT_OPT_GRAPH) {
        ctx->use_graph = value ? 1 : 0;
        return EBIT_OK;
    }
    if (option == EBIT_OPT_EXT_BLOCK) {
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto& I : ctx->inst) {
            I.g.ext_block = value ? 1 : 0;
            for (auto& gx : I.graph)
                if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        }
        for (auto& B : ctx->batches) {
            B.lead.g.ext_block = value ? 1 : 0;
            for (auto& gx : B.graph)
                if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        }
        return cuda_check(ctx, "ebit_set_option");
    }
    if (option == EBIT_OPT_TMA || option == EBIT_OPT_COOP || option == EBIT_OPT_BARRIER_SPIN) {
        if (option == EBIT_OPT_BARRIER_SPIN && value < 0) return fail(ctx, EBIT_EINVAL, "negative spin bound");
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto& I : ctx->inst) {
            for (Solver* sv : {&I.solver, &I.solver2}) {
                if (option == EBIT_OPT_TMA) sv->use_tma = value ? 1 : 0;
                else if (option == EBIT_OPT_COOP) sv->use_coop = value <= 0 ? 0 : (value >= 2 ? 2 : 1);
                else sv->barrier_spin = value;
            }
            for (auto& gx : I.graph)
                if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        }
        for (auto& B : ctx->batches)
            for (auto& gx : B.graph)
                if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        return cuda_check(ctx, "ebit_set_option");
    }
    return fail(ctx, EBIT_EINVAL, "unknown option");
}

ebit_status ebit_get_diagnostics(ebit_ctx* ctx, int inst, double* dst, int n) {
    if (!ctx || inst < 0 || inst >= (int)ctx->inst.size() || !dst || n < 0) return EBIT_EINVAL;
    Instance& I = ctx->inst[inst];
    double d[14], o[8];
    cudaMemcpyAsync(o, I.diag_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t er = cudaStreamSynchronize(ctx->stream);
    if (er != cudaSuccess) return fail(ctx, EBIT_ECUDA, cudaGetErrorString(er));
    for (int k = 0; k < 6; ++k) d[k] = o[k];
    for (int k = 0; k < 6; ++k) d[6 + k] = I.stats[k];
    d[12] = o[6];
    d[13] = o[7];
    for (int k = 0; k < n && k < 14; ++k) dst[k] = d[k];
    return EBIT_OK;
}

uint64_t ebit_launch_count(const ebit_ctx* ctx) { return ctx ? g_launches.load() - ctx->launch0 : 0; }

ebit_status ebit_timing_begin(ebit_ctx* ctx, int kernel_class) {
    if (!ctx || kernel_class != EBIT_KT_SMOOTH_L0) return EBIT_EINVAL;
    for (auto& I : ctx->inst) {
        KTimer z[2];
        for (auto& t : z) {
            t.start = ~0ull; t.end = 0; t.ticket = 0; t.active = 0; t.total_ns = 0; t.launches = 0; t.bytes = 0.0;
        }
        cudaMemcpyAsync(I.solver.timer, z, sizeof(z), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(I.solver2.timer, z, sizeof(z), cudaMemcpyHostToDevice, ctx->stream);
    }
    cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, "ebit_timing_begin");
}

ebit_status ebit_timing_end(ebit_ctx* ctx, double* total_ms, uint64_t* launches, double* bytes_per_launch) {
    if (!ctx || !total_ms || !launches || !bytes_per_launch) return EBIT_EINVAL;
    double tot = 0.0, bytes = 0.0;
    uint64_t n = 0;
    std::vector<KTimer> t(4 * ctx->inst.size());
    for (size_t b = 0; b < ctx->inst.size(); ++b) {
        cudaMemcpyAsync(&t[4 * b], ctx->inst[b].solver.timer, 2 * sizeof(KTimer), cudaMemcpyDeviceToHost,
                        ctx->stream);
        cudaMemcpyAsync(&t[4 * b + 2], ctx->inst[b].solver2.timer, 2 * sizeof(KTimer), cudaMemcpyDeviceToHost,
                        ctx->stream);
    }
    cudaStreamSynchronize(ctx->stream);
    for (auto& k : t) {
        tot += k.total_ns * 1e-6;
        n += k.launches;
        bytes += k.bytes;
    }
    *total_ms = tot;
    *launches = n;
    *bytes_per_launch = n ? bytes / (double)n : 0.0;
    return cuda_check(ctx, "ebit_timing_end");
}

const char* ebit_last_error(const ebit_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void ebit_destroy(ebit_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (auto& I : ctx->inst) {
        if (!I.arena) continue;
        if (ctx->has_alloc) { if (ctx->alloc.free_fn) ctx->alloc.free_fn(I.arena, ctx->alloc.user); }
        else cudaFree(I.arena);
        I.arena = nullptr;
    }
    for (auto& I : ctx->inst)
        for (auto& gx : I.graph)
            if (gx) cudaGraphExecDestroy(gx);
    for (auto& B : ctx->batches) {
        for (auto& gx : B.graph)
            if (gx) cudaGraphExecDestroy(gx);
        if (B.arena) {
            if (ctx->has_alloc) { if (ctx->alloc.free_fn) ctx->alloc.free_fn(B.arena, ctx->alloc.user); }
            else cudaFree(B.arena);
        }
        if (B.d_phys) cudaFree(B.d_phys);
    }
    for (auto& s : ctx->aux)
        if (s) cudaStreamDestroy(s);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (auto& I : ctx->inst) {
        if (I.e_fork) cudaEventDestroy(I.e_fork);
        if (I.e_join) cudaEventDestroy(I.e_join);
    }
    for (auto& s : ctx->workers) cudaStreamDestroy(s);
    for (auto& e : ctx->joins) cudaEventDestroy(e);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->host_states) cudaFreeHost(ctx->host_states);
    if (ctx->host_status) cudaFreeHost(ctx->host_status);
    delete ctx;
}

}  // extern "C"
