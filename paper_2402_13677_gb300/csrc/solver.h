// Multigrid-preconditioned CG (FP64, or FP32 inside FP64 iterative refinement).
#pragma once
#include <cuda_runtime.h>

namespace ebit {

struct SolveResult {
    int iters;        // CG iterations (FP64) or total inner FP32 iterations (mixed)
    double rel_res;   // final ||r|| / ||b|| (recursive residual for FP64, true FP64 residual for mixed)
    bool converged;
    int outer = 0;    // refinement sweeps (mixed)
};

struct Solver {
    static constexpr int MAXLEV = 16;
    int nlev = 0;
    int lnx[MAXLEV], lny[MAXLEV];
    double *cd[MAXLEV], *dd[MAXLEV], *wx64[MAXLEV], *wy64[MAXLEV];
    float *fdiag[MAXLEV], *fwx[MAXLEV], *fwy[MAXLEV], *fx[MAXLEV], *fb[MAXLEV];
    double *ddiag[MAXLEV], *dwx[MAXLEV], *dwy[MAXLEV], *dx[MAXLEV], *db[MAXLEV];
    double *r64, *z64, *p64, *q64;
    float *r32, *z32, *p32, *q32, *e32, *b32;
    double* ir_r64;
    double *partial, *partial2;
    unsigned* ticket;
    double *scal, *oscal, *beta;
    int* flags;
    int* host_flags;   // pinned, set by the owner
    int launches = 0;
    // optional CUDA-event timing of the level-0 smoother sweeps (the dominant kernel class)
    bool timing = false;
    int ev_cap = 0, ev_used = 0;
    long long timed_launches = 0;
    cudaEvent_t* ev = nullptr;
    void time_begin();
    void time_mark(cudaStream_t st);   // records one event (pairs: start, stop)
    double time_end_ms();               // synchronises, sums the recorded pairs

    void plan(int nx, int ny);
    static size_t bytes(int nx, int ny);
    void bind(void* base, int nx, int ny);
    // Solve A x = b; A given at the fine level by cd, dd, wx, wy (FP64); x holds the guess.
    SolveResult solve(const double* cd0, const double* dd0, const double* wx0, const double* wy0, const double* b,
                      double* x, int precision, double rtol, int max_iter, cudaStream_t st);
};

}  // namespace ebit
