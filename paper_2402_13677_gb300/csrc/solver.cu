// Matrix-free-coefficient multigrid-preconditioned conjugate gradients for the three
// implicit solves of the step (energy diffusion, viscous Helmholtz, ghost-fluid Poisson).
//
// All three operators have the integrated five-point form
//     (A x)_i = (cd_i + dd_i + sum_f w_f) x_i - sum_f w_f x_nbr(f)
// with cd the h^2 (rho cp / dt or rho / dt) term, dd the Dirichlet contributions
// (ghost-fluid interface links, fixed-temperature walls, no-slip walls, outflow pressure)
// and w the face conductances.  The preconditioner is a symmetric V(2,2)-cycle:
// red-black Gauss-Seidel (red-black before, black-red after), restriction = sum of the four
// children, prolongation = injection, coarse operators re-discretised (cd summed, dd summed
// and halved, face weights averaged along the coarse face), and a fixed symmetric sweep
// sequence on the coarsest grid, so CG sees a fixed SPD preconditioner.
//
// Precision modes (precision pattern of the method's GPU design):
//   FP64  : CG + V-cycle in double.
//   MIXED : iterative refinement: r = b - A x in FP64, correction A e = r solved in FP32 by
//           the same MG-PCG to a loose tolerance, x += e in FP64, until ||r|| <= rtol ||b||.
//
// Reductions are deterministic: per-block partial sums, the last block adds them in block
// order.  Scalars (alpha, beta, r.z, convergence flags) stay on the device; every kernel
// returns at once when the solve has converged, so the host may enqueue iterations ahead
// and only polls the convergence word every few iterations.
#include <cstdio>
#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace ebit {

constexpr int RB = 256;   // threads per block for reductions / stencils
constexpr int NRED = 608; // blocks of grid-stride kernels (4 x 152 SMs)

// scalar slots (double) and flag slots (int)
enum { S_RZ = 0, S_PQ, S_RR, S_TOL2, S_BB, S_RR0, S_COUNT };
enum { FL_DONE = 0, FL_ITERS, FL_ODONE, FL_OITERS, FL_COUNT };

template <typename T>
struct LevelView {
    int nx, ny;
    const T* diag;
    const T* wx;
    const T* wy;
};

template <typename T>
__device__ inline T nbr_sum(const LevelView<T>& L, const T* __restrict__ x, int i, int j) {
    T s = T(0);
    int c = j * L.nx + i;
    if (i > 0) s += L.wx[j * (L.nx + 1) + i] * x[c - 1];
    if (i < L.nx - 1) s += L.wx[j * (L.nx + 1) + i + 1] * x[c + 1];
    if (j > 0) s += L.wy[j * L.nx + i] * x[c - L.nx];
    if (j < L.ny - 1) s += L.wy[(j + 1) * L.nx + i] * x[c + L.nx];
    return s;
}

__device__ inline bool skip(const int* fl) { return fl[FL_DONE] != 0 || fl[FL_ODONE] != 0; }

// ---- block reductions ---------------------------------------------------------------
__device__ inline double bsum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// write this block's partial; returns true in thread 0 of the last block, with the total in *tot
__device__ inline bool reduce_finish(double v, double* partial, unsigned* ticket, double* tot) {
    __shared__ double sh[32];
    __shared__ bool last;
    double r = bsum(v, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile double*)partial)[b];
    s = bsum(s, sh);
    if (threadIdx.x == 0) { *tot = s; *ticket = 0u; }
    return threadIdx.x == 0;
}

// ---- operator setup -------------------------------------------------------------------
template <typename T>
__global__ void k_make_diag(int nx, int ny, const double* __restrict__ cd, const double* __restrict__ dd,
                            const double* __restrict__ wx, const double* __restrict__ wy, T* __restrict__ diag,
                            T* __restrict__ wx_o, T* __restrict__ wy_o) {
    int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int i = c % nx, j = c / nx;
        double a = wx[j * (nx + 1) + i], b = wx[j * (nx + 1) + i + 1];
        double d = wy[j * nx + i], e = wy[(j + 1) * nx + i];
        diag[c] = (T)(cd[c] + dd[c] + a + b + d + e);
        if (wx_o) {
            wx_o[j * (nx + 1) + i] = (T)a;
            if (i == nx - 1) wx_o[j * (nx + 1) + nx] = (T)b;
            wy_o[j * nx + i] = (T)d;
            if (j == ny - 1) wy_o[ny * nx + i] = (T)e;
        }
    }
}

// coarse operator from a fine one (cd summed, dd summed and halved, faces averaged)
template <typename Tc>
__global__ void k_coarsen(int fnx, int fny, const double* __restrict__ fcd, const double* __restrict__ fdd,
                          const double* __restrict__ fwx, const double* __restrict__ fwy, double* __restrict__ ccd,
                          double* __restrict__ cdd, double* __restrict__ cwx, double* __restrict__ cwy,
                          Tc* __restrict__ cdiag, Tc* __restrict__ cwx_t, Tc* __restrict__ cwy_t) {
    int nx = fnx / 2, ny = fny / 2;
    int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int I = c % nx, J = c / nx;
        int f00 = (2 * J) * fnx + 2 * I;
        double s_cd = fcd[f00] + fcd[f00 + 1] + fcd[f00 + fnx] + fcd[f00 + fnx + 1];
        double s_dd = 0.5 * (fdd[f00] + fdd[f00 + 1] + fdd[f00 + fnx] + fdd[f00 + fnx + 1]);
        auto fx = [&](int fi, int fj) { return fwx[fj * (fnx + 1) + fi]; };
        auto fy = [&](int fi, int fj) { return fwy[fj * fnx + fi]; };
        double wl = 0.5 * (fx(2 * I, 2 * J) + fx(2 * I, 2 * J + 1));
        double wr = 0.5 * (fx(2 * I + 2, 2 * J) + fx(2 * I + 2, 2 * J + 1));
        double wb = 0.5 * (fy(2 * I, 2 * J) + fy(2 * I + 1, 2 * J));
        double wt = 0.5 * (fy(2 * I, 2 * J + 2) + fy(2 * I + 1, 2 * J + 2));
        ccd[c] = s_cd;
        cdd[c] = s_dd;
        cwx[J * (nx + 1) + I] = wl;
        if (I == nx - 1) cwx[J * (nx + 1) + nx] = wr;
        cwy[J * nx + I] = wb;
        if (J == ny - 1) cwy[ny * nx + I] = wt;
        cdiag[c] = (Tc)(s_cd + s_dd + wl + wr + wb + wt);
        cwx_t[J * (nx + 1) + I] = (Tc)wl;
        if (I == nx - 1) cwx_t[J * (nx + 1) + nx] = (Tc)wr;
        cwy_t[J * nx + I] = (Tc)wb;
        if (J == ny - 1) cwy_t[ny * nx + I] = (Tc)wt;
    }
}

// ---- smoother, transfer, coarse solve --------------------------------------------------
template <typename T>
__global__ void k_smooth(LevelView<T> L, const T* __restrict__ b, T* __restrict__ x, int color, int zero,
                         const int* __restrict__ fl) {
    if (skip(fl)) return;
    int N = L.nx * L.ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int i = c % L.nx, j = c / L.nx;
        if (((i + j) & 1) != color) {
            if (zero) x[c] = T(0);
            continue;
        }
        T s = zero ? T(0) : nbr_sum(L, x, i, j);
        x[c] = (b[c] + s) / L.diag[c];
    }
}

template <typename T>
__global__ void k_restrict_residual(LevelView<T> F, const T* __restrict__ b, const T* __restrict__ x,
                                    T* __restrict__ bc, const int* __restrict__ fl) {
    if (skip(fl)) return;
    int nx = F.nx / 2, ny = F.ny / 2;
    int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int I = c % nx, J = c / nx;
        T s = T(0);
        for (int b2 = 0; b2 < 2; ++b2)
            for (int a2 = 0; a2 < 2; ++a2) {
                int i = 2 * I + a2, j = 2 * J + b2;
                int f = j * F.nx + i;
                s += b[f] - (F.diag[f] * x[f] - nbr_sum(F, x, i, j));
            }
        bc[c] = s;
    }
}

template <typename T>
__global__ void k_prolong(int fnx, int fny, const T* __restrict__ xc, T* __restrict__ x, const int* __restrict__ fl) {
    if (skip(fl)) return;
    int N = fnx * fny;
    int cnx = fnx / 2;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int i = c % fnx, j = c / fnx;
        x[c] += xc[(j >> 1) * cnx + (i >> 1)];
    }
}

// coarsest grid, one block: `pairs` red-black sweeps then `pairs` black-red sweeps from zero
template <typename T>
__global__ void k_coarse_solve(LevelView<T> L, const T* __restrict__ b, T* __restrict__ x, int pairs,
                               const int* __restrict__ fl) {
    if (skip(fl)) return;
    extern __shared__ unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    int N = L.nx * L.ny;
    for (int c = threadIdx.x; c < N; c += blockDim.x) xs[c] = T(0);
    __syncthreads();
    for (int sweep = 0; sweep < 4 * pairs; ++sweep) {
        int color = sweep < 2 * pairs ? (sweep & 1) : 1 - (sweep & 1);
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            int i = c % L.nx, j = c / L.nx;
            if (((i + j) & 1) != color) continue;
            xs[c] = (b[c] + nbr_sum(L, xs, i, j)) / L.diag[c];
        }
        __syncthreads();
    }
    for (int c = threadIdx.x; c < N; c += blockDim.x) x[c] = xs[c];
}

// ---- CG kernels -------------------------------------------------------------------------
// q = A p, pq = p.q
template <typename T>
__global__ void k_apply_dot(LevelView<T> L, const T* __restrict__ p, T* __restrict__ q, double* partial,
                            unsigned* ticket, double* scal, const int* fl) {
    if (skip(fl)) return;
    int N = L.nx * L.ny;
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int i = c % L.nx, j = c / L.nx;
        T pc = p[c];
        T v = L.diag[c] * pc - nbr_sum(L, p, i, j);
        q[c] = v;
        acc += (double)pc * (double)v;
    }
    double tot;
    if (reduce_finish(acc, partial, ticket, &tot)) scal[S_PQ] = tot;
}

// x += alpha p, r -= alpha q, rr = r.r, convergence test
template <typename T>
__global__ void k_cg_update(int N, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                            const T* __restrict__ q, double* partial, unsigned* ticket, double* scal, int* fl,
                            int iter_slot) {
    if (skip(fl)) return;
    double pq = scal[S_PQ];
    T alpha = (T)(pq != 0.0 ? scal[S_RZ] / pq : 0.0);
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        x[c] += alpha * p[c];
        T rv = r[c] - alpha * q[c];
        r[c] = rv;
        acc += (double)rv * (double)rv;
    }
    double tot;
    if (reduce_finish(acc, partial, ticket, &tot)) {
        scal[S_RR] = tot;
        fl[iter_slot] += 1;
        if (tot <= scal[S_TOL2]) fl[FL_DONE] = 1;
    }
}

// rz_new = r.z; beta = rz_new / rz; p = z + beta p is done by k_update_p
template <typename T>
__global__ void k_dot_rz(int N, const T* __restrict__ r, const T* __restrict__ z, double* partial, unsigned* ticket,
                         double* scal, const int* fl, double* beta_out) {
    if (skip(fl)) return;
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
        acc += (double)r[c] * (double)z[c];
    double tot;
    if (reduce_finish(acc, partial, ticket, &tot)) {
        double old = scal[S_RZ];
        *beta_out = old != 0.0 ? tot / old : 0.0;
        scal[S_RZ] = tot;
    }
}

template <typename T>
__global__ void k_update_p(int N, const T* __restrict__ z, T* __restrict__ p, const double* __restrict__ beta,
                           int first, const int* __restrict__ fl) {
    if (skip(fl)) return;
    T bt = first ? T(0) : (T)(*beta);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
        p[c] = z[c] + bt * p[c];
}

// r = b - A x, rr = r.r, bb = b.b; sets the tolerance (rtol^2 bb) and the done flag
template <typename T>
__global__ void k_cg_init(LevelView<T> L, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r,
                          double* partial, double* partial2, unsigned* ticket, unsigned* ticket2, double* scal,
                          int* fl, double rtol2) {
    int N = L.nx * L.ny;
    double acc = 0.0, accb = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int i = c % L.nx, j = c / L.nx;
        T bv = b[c];
        T rv = bv - (L.diag[c] * x[c] - nbr_sum(L, x, i, j));
        r[c] = rv;
        acc += (double)rv * (double)rv;
        accb += (double)bv * (double)bv;
    }
    double tot, totb;
    bool l1 = reduce_finish(accb, partial2, ticket2, &totb);
    if (l1) scal[S_BB] = totb;
    if (reduce_finish(acc, partial, ticket, &tot)) {
        // both reductions finish in the same (last) block for the first one only if ordering
        // matches; the tolerance is therefore set by k_cg_tol below
        scal[S_RR] = tot;
        scal[S_RR0] = tot;
    }
    (void)rtol2;
    (void)fl;
}

__global__ void k_cg_tol(double* scal, int* fl, double rtol2, int reset_outer) {
    double bb = scal[S_BB];
    double tol2 = rtol2 * (bb > 1e-300 ? bb : 1e-300);
    scal[S_TOL2] = tol2;
    fl[FL_DONE] = scal[S_RR] <= tol2 ? 1 : 0;
    fl[FL_ITERS] = 0;
    if (reset_outer) { fl[FL_ODONE] = 0; fl[FL_OITERS] = 0; }
}

// mixed precision: r64 = b - A64 x64 and its norm; r32 = r64; outer convergence test
__global__ void k_ir_residual(LevelView<double> L, const double* __restrict__ b, const double* __restrict__ x,
                              double* __restrict__ r64, float* __restrict__ r32, float* __restrict__ e32,
                              double* partial, unsigned* ticket, double* oscal, int* fl) {
    if (fl[FL_ODONE]) return;
    int N = L.nx * L.ny;
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int i = c % L.nx, j = c / L.nx;
        double rv = b[c] - (L.diag[c] * x[c] - nbr_sum(L, x, i, j));
        r64[c] = rv;
        r32[c] = (float)rv;
        e32[c] = 0.0f;
        acc += rv * rv;
    }
    double tot;
    if (reduce_finish(acc, partial, ticket, &tot)) {
        oscal[S_RR] = tot;
        fl[FL_OITERS] += 1;
        if (tot <= oscal[S_TOL2]) fl[FL_ODONE] = 1;
        fl[FL_DONE] = 0;
        fl[FL_ITERS] = 0;
    }
}

__global__ void k_ir_update(int N, double* __restrict__ x, const float* __restrict__ e, const int* __restrict__ fl) {
    if (fl[FL_ODONE]) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) x[c] += (double)e[c];
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static inline int nblocks(long long n) {
    long long b = (n + RB - 1) / RB;
    return (int)(b < NRED ? (b < 1 ? 1 : b) : NRED);
}

void Solver::plan(int nx, int ny) {
    nlev = 0;
    int x = nx, y = ny;
    while (true) {
        lnx[nlev] = x;
        lny[nlev] = y;
        ++nlev;
        if (nlev == MAXLEV) break;
        if ((x & 1) || (y & 1) || (long long)x * y <= 64 || x < 4 || y < 4) break;
        x /= 2;
        y /= 2;
    }
}

size_t Solver::bytes(int nx, int ny) {
    Solver s;
    s.plan(nx, ny);
    size_t total = 0;
    auto add = [&](size_t b) { total += (b + 255) & ~size_t(255); };
    for (int l = 0; l < s.nlev; ++l) {
        size_t n = (size_t)s.lnx[l] * s.lny[l];
        size_t nfx = (size_t)s.lny[l] * (s.lnx[l] + 1), nfy = (size_t)(s.lny[l] + 1) * s.lnx[l];
        if (l > 0) { add(n * 8); add(n * 8); add(nfx * 8); add(nfy * 8); }   // cd, dd, wx, wy (FP64 coarsening)
        for (int t = 0; t < 2; ++t) {                                        // float and double views
            size_t e = t == 0 ? 4 : 8;
            add(n * e); add(nfx * e); add(nfy * e);                          // diag, wx, wy
            add(n * e); add(n * e);                                          // x, b
        }
    }
    size_t n0 = (size_t)nx * ny;
    add(n0 * 8 * 4);   // r, z, p, q double
    add(n0 * 4 * 6);   // r, z, p, q, e, b float
    add(n0 * 8);       // r64 (IR)
    add(NRED * 8 * 4); add(64); add(64 * 8); add(64 * 4); add(64);
    return total;
}

void Solver::bind(void* base, int nx, int ny) {
    plan(nx, ny);
    char* p = (char*)base;
    auto take = [&](size_t b) { void* r = p; p += (b + 255) & ~size_t(255); return r; };
    for (int l = 0; l < nlev; ++l) {
        size_t n = (size_t)lnx[l] * lny[l];
        size_t nfx = (size_t)lny[l] * (lnx[l] + 1), nfy = (size_t)(lny[l] + 1) * lnx[l];
        if (l > 0) {
            cd[l] = (double*)take(n * 8); dd[l] = (double*)take(n * 8);
            wx64[l] = (double*)take(nfx * 8); wy64[l] = (double*)take(nfy * 8);
        }
        fdiag[l] = (float*)take(n * 4); fwx[l] = (float*)take(nfx * 4); fwy[l] = (float*)take(nfy * 4);
        fx[l] = (float*)take(n * 4); fb[l] = (float*)take(n * 4);
        ddiag[l] = (double*)take(n * 8); dwx[l] = (double*)take(nfx * 8); dwy[l] = (double*)take(nfy * 8);
        dx[l] = (double*)take(n * 8); db[l] = (double*)take(n * 8);
    }
    size_t n0 = (size_t)nx * ny;
    r64 = (double*)take(n0 * 8 * 4);
    z64 = r64 + n0; p64 = z64 + n0; q64 = p64 + n0;
    r32 = (float*)take(n0 * 4 * 6);
    z32 = r32 + n0; p32 = z32 + n0; q32 = p32 + n0; e32 = q32 + n0; b32 = e32 + n0;
    ir_r64 = (double*)take(n0 * 8);
    partial = (double*)take(NRED * 8 * 4);
    partial2 = partial + NRED;
    ticket = (unsigned*)take(64);
    scal = (double*)take(64 * 8);
    oscal = scal + 16;
    beta = scal + 32;
    flags = (int*)take(64 * 4);
    host_flags = nullptr;
}

template <typename T>
static LevelView<T> view(const Solver& s, int l);
template <>
LevelView<float> view<float>(const Solver& s, int l) { return {s.lnx[l], s.lny[l], s.fdiag[l], s.fwx[l], s.fwy[l]}; }
template <>
LevelView<double> view<double>(const Solver& s, int l) {
    return {s.lnx[l], s.lny[l], s.ddiag[l], s.dwx[l], s.dwy[l]};
}
template <typename T> static T* lx(const Solver& s, int l);
template <> float* lx<float>(const Solver& s, int l) { return s.fx[l]; }
template <> double* lx<double>(const Solver& s, int l) { return s.dx[l]; }
template <typename T> static T* lb(const Solver& s, int l);
template <> float* lb<float>(const Solver& s, int l) { return s.fb[l]; }
template <> double* lb<double>(const Solver& s, int l) { return s.db[l]; }

// Build the hierarchy for the fine operator (cd0, dd0, wx0, wy0 in FP64).
template <typename T>
static void setup_hierarchy(Solver& s, const double* cd0, const double* dd0, const double* wx0, const double* wy0,
                            cudaStream_t st, int& launches) {
    int N0 = s.lnx[0] * s.lny[0];
    // FP64 level 0 always (outer residual / FP64 CG)
    k_make_diag<double><<<nblocks(N0), RB, 0, st>>>(s.lnx[0], s.lny[0], cd0, dd0, wx0, wy0, s.ddiag[0], s.dwx[0],
                                                    s.dwy[0]);
    ++launches;
    if (sizeof(T) == 4) {
        k_make_diag<float><<<nblocks(N0), RB, 0, st>>>(s.lnx[0], s.lny[0], cd0, dd0, wx0, wy0, s.fdiag[0], s.fwx[0],
                                                       s.fwy[0]);
        ++launches;
    }
    const double *fcd = cd0, *fdd = dd0, *fwx = wx0, *fwy = wy0;
    for (int l = 1; l < s.nlev; ++l) {
        int n = s.lnx[l] * s.lny[l];
        T* cdiag = sizeof(T) == 4 ? (T*)s.fdiag[l] : (T*)s.ddiag[l];
        T* cwx = sizeof(T) == 4 ? (T*)s.fwx[l] : (T*)s.dwx[l];
        T* cwy = sizeof(T) == 4 ? (T*)s.fwy[l] : (T*)s.dwy[l];
        k_coarsen<T><<<nblocks(n), RB, 0, st>>>(s.lnx[l - 1], s.lny[l - 1], fcd, fdd, fwx, fwy, s.cd[l], s.dd[l],
                                               s.wx64[l], s.wy64[l], cdiag, cwx, cwy);
        ++launches;
        fcd = s.cd[l]; fdd = s.dd[l]; fwx = s.wx64[l]; fwy = s.wy64[l];
    }
}

void Solver::time_begin() {
    if (!ev) {
        ev_cap = 8192;
        ev = new cudaEvent_t[ev_cap];
        for (int k = 0; k < ev_cap; ++k) cudaEventCreate(&ev[k]);
    }
    ev_used = 0;
    timed_launches = 0;
    timing = true;
}

void Solver::time_mark(cudaStream_t st) {
    if (ev_used < ev_cap) cudaEventRecord(ev[ev_used], st);
    ++ev_used;
}

double Solver::time_end_ms() {
    timing = false;
    double tot = 0.0;
    int n = ev_used < ev_cap ? ev_used : ev_cap;
    if (n >= 2) cudaEventSynchronize(ev[n - 1]);
    for (int k = 0; k + 1 < n; k += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
        tot += ms;
    }
    timed_launches = n / 2;
    return tot;
}

// z = M r (one V(2,2)-cycle), level-0 input b0 = r and output x0 = z
template <typename T>
static void vcycle(Solver& s, const T* r, T* z, cudaStream_t st, int& launches) {
    const int nu = 2;
    const T* b = r;
    T* x = z;
    for (int l = 0; l < s.nlev - 1; ++l) {
        LevelView<T> L = view<T>(s, l);
        int n = L.nx * L.ny;
        bool tm = s.timing && l == 0;
        for (int k = 0; k < nu; ++k) {
            if (tm) s.time_mark(st);
            k_smooth<T><<<nblocks(n), RB, 0, st>>>(L, b, x, 0, k == 0, s.flags);
            if (tm) { s.time_mark(st); s.time_mark(st); }
            k_smooth<T><<<nblocks(n), RB, 0, st>>>(L, b, x, 1, 0, s.flags);
            if (tm) s.time_mark(st);
            launches += 2;
        }
        T* bc = lb<T>(s, l + 1);
        k_restrict_residual<T><<<nblocks(n / 4), RB, 0, st>>>(L, b, x, bc, s.flags);
        ++launches;
        b = bc;
        x = lx<T>(s, l + 1);
    }
    {
        int l = s.nlev - 1;
        LevelView<T> L = view<T>(s, l);
        int n = L.nx * L.ny;
        if (n <= 4096) {
            int threads = n < 1024 ? ((n + 31) / 32) * 32 : 1024;
            k_coarse_solve<T><<<1, threads, n * sizeof(T), st>>>(L, b, x, 16, s.flags);
            ++launches;
        } else {
            for (int k = 0; k < 64; ++k) {
                k_smooth<T><<<nblocks(n), RB, 0, st>>>(L, b, x, k < 32 ? (k & 1) : 1 - (k & 1), k == 0, s.flags);
                ++launches;
            }
        }
    }
    for (int l = s.nlev - 2; l >= 0; --l) {
        LevelView<T> L = view<T>(s, l);
        int n = L.nx * L.ny;
        T* xl = l == 0 ? z : lx<T>(s, l);
        const T* bl = l == 0 ? r : lb<T>(s, l);
        k_prolong<T><<<nblocks(n), RB, 0, st>>>(L.nx, L.ny, lx<T>(s, l + 1), xl, s.flags);
        ++launches;
        bool tm = s.timing && l == 0;
        for (int k = 0; k < nu; ++k) {
            if (tm) s.time_mark(st);
            k_smooth<T><<<nblocks(n), RB, 0, st>>>(L, bl, xl, 1, 0, s.flags);
            if (tm) { s.time_mark(st); s.time_mark(st); }
            k_smooth<T><<<nblocks(n), RB, 0, st>>>(L, bl, xl, 0, 0, s.flags);
            if (tm) s.time_mark(st);
            launches += 2;
        }
    }
}

// poll the convergence flags (pinned host copy)
static void poll_flags(Solver& s, cudaStream_t st, int* out) {
    cudaMemcpyAsync(s.host_flags, s.flags, FL_COUNT * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (int k = 0; k < FL_COUNT; ++k) out[k] = s.host_flags[k];
}

// PCG on A x = b at level 0 in precision T (x holds the initial guess)
template <typename T>
static int pcg(Solver& s, const T* b, T* x, T* r, T* z, T* p, T* q, double rtol, int max_iter, int poll_every,
               bool reset_outer, cudaStream_t st, int& launches) {
    LevelView<T> L = view<T>(s, 0);
    int N = L.nx * L.ny;
    k_cg_init<T><<<nblocks(N), RB, 0, st>>>(L, b, x, r, s.partial, s.partial2, s.ticket, s.ticket + 1, s.scal,
                                            s.flags, rtol * rtol);
    k_cg_tol<<<1, 1, 0, st>>>(s.scal, s.flags, rtol * rtol, reset_outer ? 1 : 0);
    vcycle<T>(s, r, z, st, launches);
    k_dot_rz<T><<<nblocks(N), RB, 0, st>>>(N, r, z, s.partial, s.ticket, s.scal, s.flags, s.beta);
    k_update_p<T><<<nblocks(N), RB, 0, st>>>(N, z, p, s.beta, 1, s.flags);
    launches += 4;
    int hf[FL_COUNT];
    for (int it = 0; it < max_iter; ++it) {
        k_apply_dot<T><<<nblocks(N), RB, 0, st>>>(L, p, q, s.partial, s.ticket, s.scal, s.flags);
        k_cg_update<T><<<nblocks(N), RB, 0, st>>>(N, x, r, p, q, s.partial, s.ticket, s.scal, s.flags, FL_ITERS);
        vcycle<T>(s, r, z, st, launches);
        k_dot_rz<T><<<nblocks(N), RB, 0, st>>>(N, r, z, s.partial, s.ticket, s.scal, s.flags, s.beta);
        k_update_p<T><<<nblocks(N), RB, 0, st>>>(N, z, p, s.beta, 0, s.flags);
        launches += 4;
        if ((it + 1) % poll_every == 0 || it == max_iter - 1) {
            poll_flags(s, st, hf);
            if (hf[FL_DONE] || hf[FL_ODONE]) return hf[FL_ITERS];
        }
    }
    return -1;
}

SolveResult Solver::solve(const double* cd0, const double* dd0, const double* wx0, const double* wy0, const double* b,
                          double* x, int precision, double rtol, int max_iter, cudaStream_t st) {
    SolveResult res{0, 0.0, true};
    int N = lnx[0] * lny[0];
    if (precision == 0) {
        setup_hierarchy<double>(*this, cd0, dd0, wx0, wy0, st, launches);
        int it = pcg<double>(*this, b, x, r64, z64, p64, q64, rtol, max_iter, 4, true, st, launches);
        int hf[FL_COUNT];
        poll_flags(*this, st, hf);
        double sc[S_COUNT];
        cudaMemcpy(sc, scal, sizeof(sc), cudaMemcpyDeviceToHost);
        res.iters = hf[FL_ITERS];
        res.converged = hf[FL_DONE] != 0;
        res.rel_res = sqrt(sc[S_RR] / (sc[S_BB] > 1e-300 ? sc[S_BB] : 1e-300));
        (void)it;
        return res;
    }
    // mixed: FP64 outer residual, FP32 inner MG-PCG
    setup_hierarchy<float>(*this, cd0, dd0, wx0, wy0, st, launches);
    LevelView<double> L64 = view<double>(*this, 0);
    // ||b||^2 and tolerance for the outer loop (reuse k_cg_init on x to get b.b)
    k_cg_init<double><<<nblocks(N), RB, 0, st>>>(L64, b, x, ir_r64, partial, partial2, ticket, ticket + 1, oscal,
                                                 flags, 0.0);
    k_cg_tol<<<1, 1, 0, st>>>(oscal, flags, rtol * rtol, 1);
    launches += 2;
    int max_outer = max_iter > 0 ? (max_iter + 19) / 20 + 4 : 8;
    int hf[FL_COUNT];
    int inner_total = 0;
    for (int o = 0; o < max_outer; ++o) {
        k_ir_residual<<<nblocks(N), RB, 0, st>>>(L64, b, x, ir_r64, r32, e32, partial, ticket, oscal, flags);
        ++launches;
        int it = pcg<float>(*this, r32, e32, b32, z32, p32, q32, 1e-4, 60, 6, false, st, launches);
        (void)it;
        poll_flags(*this, st, hf);
        if (hf[FL_ODONE]) break;
        inner_total += hf[FL_ITERS];
        k_ir_update<<<nblocks(N), RB, 0, st>>>(N, x, e32, flags);
        ++launches;
    }
    poll_flags(*this, st, hf);
    double sc[S_COUNT];
    cudaMemcpy(sc, oscal, sizeof(sc), cudaMemcpyDeviceToHost);
    res.iters = inner_total;
    res.outer = hf[FL_OITERS];
    res.converged = hf[FL_ODONE] != 0;
    res.rel_res = sqrt(sc[S_RR] / (sc[S_BB] > 1e-300 ? sc[S_BB] : 1e-300));
    return res;
}

}  // namespace ebit
