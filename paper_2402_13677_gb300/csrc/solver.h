// Multigrid-preconditioned CG for the implicit solves of the step (FP64, or FP32 inside
// FP64 iterative refinement), with device-side loop control so that a whole solve can be
// captured into a CUDA graph (conditional WHILE nodes) or driven from the host.
#pragma once
#include <cuda.h>           // CUtensorMap (the encoder is fetched through the runtime)
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace ebit {

struct SolveResult {
    int iters;        // CG iterations (FP64) or total inner FP32 iterations (mixed)
    double rel_res;   // final ||r|| / ||b|| (max over right-hand sides)
    bool converged;
    int outer = 0;    // refinement sweeps (mixed)
    bool fault = false;   // a bounded wait (TMA copies, grid barrier) gave up: the result is not valid
    bool nonfinite = false;   // the system or the iterate held a NaN or an infinity
};

// device-resident timing of one kernel class (span from the first block's start to the
// last block's end, read from %globaltimer), accumulated over launches
struct KTimer {
    unsigned long long start;
    unsigned long long end;
    unsigned int ticket;
    unsigned int active;   // instances of the current launch that ran (not converged)
    unsigned long long total_ns;
    unsigned long long launches;
    double bytes;      // algorithmic bytes of the timed launches (each launch adds its own)
};

// device-side scalars of one solve; per right-hand side k < 2
struct SolveState {
    double rz[2], pq[2], alpha[2], beta[2], rr[2], bb[2], tol2[2];
    double orr[2], obb[2], otol2[2];   // outer (FP64) residual norms of the refinement loop
    int done, iters, odone, oiters, max_iters, max_outer, nr, itot;
    double inner_rtol;
    int fault;         // nonzero: a bounded wait gave up (TMA copies that never landed, a grid barrier)
    int nonfinite;     // nonzero: a residual norm was NaN or infinite (the solve stopped there)
    double scale[2];   // refinement: the inner FP32 system is solved for scale * r (a power of two)
    double scale_next[2];   // the scale the next refinement pass uses (from the latest residual norm)
};

// TMA descriptors of one tiled level (precision and right-hand-side count fixed): the level's
// right-hand side b, the pre-smoothed x (k_post), the next level's x (k_post), and D, wl, wb
struct TileMaps {
    CUtensorMap b, xin, xc, d, wl, wb;
};

struct Solver {
    static constexpr int MAXLEV = 16;
    int nx = 0, ny = 0;
    int nlev = 0;     // all levels
    int nbig = 0;     // levels [0, nbig) use the tiled kernels, [nbig, nlev) the one-block cycle
    int nbig_f = 0, nbig_d = 0;   // the same split for FP32 and FP64 level data
    int lnx[MAXLEV], lny[MAXLEV];
    size_t loff[MAXLEV];   // cell offset of level l in the packed per-level arrays
    size_t ncells_all = 0;
    // per-level operators, packed over levels (float and double copies): diag, wl, wb, cd, dd
    float *f_diag, *f_wl, *f_wb, *f_cd, *f_dd;
    double *d_diag, *d_wl, *d_wb, *d_cd, *d_dd;
    // per-level vectors (2 right-hand sides interleaved), packed: x (correction) and b (rhs)
    float *f_x, *f_b, *f_x2;    // x2: pre-smoothed x (written by k_pre, read by k_post)
    double *d_x, *d_b, *d_x2;
    // CG vectors at level 0 (2 RHS interleaved)
    float *f_r, *f_p, *f_q, *f_e;
    double *d_r, *d_p, *d_q;
    float* f_inv;      // dense inverse of the coarsest operator (at most 32 cells)
    double* d_inv;
    // reductions
    double* partial;   // [4][MAXBLK][2]
    unsigned* tickets; // 8
    static constexpr int NSLOT = 8;
    SolveState* st_base;   // device, one state per solve slot
    SolveState* st_host;   // pinned mirror of all slots (set by the owner)
    SolveState* st = nullptr;   // slot of the current solve
    int slot = 0;
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};   // capture streams of loop bodies
    KTimer* timer;     // device, [2]: tiled level-0 pre / post kernels
    int timing = 0;
    long long launches = 0;
    int use_graph = 0;     // set by the owner while capturing
    // TMA descriptors of the tiled levels, [precision][NR - 1][level], encoded on first use;
    // tma_ok false where a level's rows or base are not 16-byte aligned (plain loads then)
    std::vector<TileMaps> tmaps;
    std::vector<char> tma_ok;
    bool tma_ready = false;
    int use_tma = 1;       // 0: the tile kernels load their regions with plain loads
    int use_coop = 1;      // 0: no cooperative launch for the coarse part of the V-cycle
    int barrier_spin = 0;  // polls of the cooperative launch's grid barrier before it gives up (0: 2^22)
    // batched launches: this solver drives nz instances whose arenas lie zs bytes apart (the
    // solvers of instances 1..nz-1 are bound to their own arenas, read only for statistics)
    int nz = 1;
    long long zs = 0;
    // schedule (tunable): levels with at most small_max_f cells run in the single-block kernel
    // (FP32); the refinement's inner FP32 solves stop at inner_rtol
    int small_max_f = 0;   // 0: the default
    double inner_rtol = 1e-5;
    bool set_schedule(int small_max, double inner);

    void plan(int nx, int ny);
    static size_t bytes(int nx, int ny);
    // carve the arrays out of `base`; returns the first CUDA error of the set-up calls
    cudaError_t bind(void* base, int nx, int ny, bool make_streams = true, cudaStream_t init_stream = 0);
    // Solve A x = b for nr (1 or 2) interleaved right-hand sides.  The fine operator is given
    // cell-centred in FP64: cd (h^2 c), dd (Dirichlet terms), wl (left-face weight), wb
    // (bottom-face weight); x holds the initial guess.  In graph mode (use_graph) the loops
    // become conditional nodes of the graph being captured on `st`; the result is then only
    // available after the graph ran (read it with read_result).
    void solve(const double* cd, const double* dd, const double* wl, const double* wb, const double* b, double* x,
               int nr, int precision, double rtol, int max_iter, cudaStream_t st);
    // synchronises st; a failed copy or synchronisation is returned in *err (if given) and
    // gives a result with fault set
    SolveResult read_result(int slot, int precision, cudaStream_t st, cudaError_t* err = nullptr);
    // batched read-back: queue the copy of every slot's state to st_host (no synchronisation),
    // then, once the stream has been synchronised, read a slot from the host copy
    void fetch_states(cudaStream_t st);
    SolveResult result_from_host(int slot, int precision) const;
    static bool supported(int nx, int ny);
    int body_size(int precision) const;   // kernels of one CG iteration (V-cycle + apply + update)
};

}  // namespace ebit
