// Multigrid-preconditioned conjugate gradients for the implicit solves of the step
// (energy diffusion, viscous Helmholtz, ghost-fluid Poisson).
//
// Operator (integrated five-point form, cell-centred coefficients), applied in flux form:
//     (A x)_i = D_i x_i + wl_i (x_i - x_{i-1}) + wl_{i+1} (x_i - x_{i+1})
//                       + wb_i (x_i - x_{i-nx}) + wb_{i+nx} (x_i - x_{i+nx}),   D_i = cd_i + dd_i
// The flux form keeps the zero row sum of the conductance part exact in any precision: a
// diagonal stored as cd + dd + sum w and rounded to FP32 separately from the w would add a
// spurious diagonal of relative size 6e-8, above the smallest eigenvalue of a 4096^2 Poisson
// operator (condition number ~1e9), and the FP32 solve would stall.  Smoothers use
// diag = D + sum w computed on the fly.
// with cd the h^2 (rho cp / dt or rho / dt) term, dd the Dirichlet contributions (ghost-fluid
// interface links, fixed-temperature or no-slip walls, outflow pressure), wl/wb the left and
// bottom face conductances (zero on domain faces).
//
// Preconditioner: one symmetric V(2,2)-cycle.  Red-black Gauss-Seidel (red-black before,
// black-red after), restriction = sum of the four children, prolongation = injection, coarse
// operators re-discretised (cd summed, dd summed and halved, face weights averaged along the
// coarse face), a fixed symmetric sweep sequence on the coarsest grid.
//
// Kernel structure (few launches per CG iteration):
//   * large levels: k_pre  = 2 red-black sweeps from zero + residual + restriction, and
//                   k_post = prolongation + 2 black-red sweeps (+ r.z at the finest level),
//     each a shared-memory tile with a halo of recomputed cells, so one launch performs
//     several Gauss-Seidel half-sweeps; halo cells are recomputed from the same inputs with
//     the same formula, so the result equals global red-black Gauss-Seidel exactly;
//   * every level of at most 1024 cells: one single-block kernel (k_small) runs the rest of
//     the V-cycle in shared memory;
//   * CG: k_apply (p = z + beta p fused into q = A p, p.q) and k_update (x, r, r.r, test).
// Loop control lives on the device (SolveState); kernels can drive CUDA-graph conditional
// WHILE nodes (cudaGraphSetConditional), or the host can poll the state.
//
// Precision modes:
//   FP64  : CG + V-cycle in double.
//   MIXED : iterative refinement: r = b - A x in FP64, correction A e = r solved in FP32 by
//           the same MG-PCG to a relative 1e-5, x += e in FP64, until ||r|| <= rtol ||b||.
//
// Reductions are deterministic: per-block partial sums, the last block adds them in block order.
#include <vector>
#include <cfloat>
#include <cstdio>
#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace ebit {

constexpr int RB = 256;          // threads of grid-stride kernels
constexpr int NRED = 608;        // blocks of grid-stride kernels (4 x 152 SMs)
constexpr int SMALL_MAX_F = 1024; // default: levels with at most this many cells run inside k_small (FP32)
constexpr int SMALL_MAX_F_LIMIT = 4096;   // the shared memory of k_small holds at most this level
constexpr int SMALL_MAX_D = 1024; // (FP64: half the shared memory per value)
constexpr int SMALL_THREADS = 1024;
constexpr int TX = 32, TY = 32;  // tile of the large-level kernels
constexpr int NU = 2;            // smoothing sweeps (red-black pairs) before and after
constexpr int NU_SMALL = 2;      // the same on the levels of the single-block kernel
// halo of the tile kernels: every half-sweep after the first leaves one more ring of the region
// stale.  Pre-smoothing starts from x = 0, so its first half-sweep needs no neighbours and is
// exact up to the region edge: 2 NU - 1 further half-sweeps and the residual need 2 NU rings.
// Post-smoothing: 2 NU half-sweeps, then the core only.
constexpr int HPRE = 2 * NU, HPOST = 2 * NU;
constexpr int COARSE_PAIRS = 12; // symmetric sweeps on the coarsest grid (at most 16 cells)

template <typename T, int NR>
struct alignas(sizeof(T) * NR) Vec {
    T v[NR];
};

template <typename T>
struct Lev {
    int nx, ny;
    const T* diag;
    const T* wl;
    const T* wb;
    long long zs;   // byte stride between the instances of a batched launch (0: one instance)
};

// correctly rounded reciprocal (the same value as 1 / v)
// reciprocal of a smoother's diagonal.  FP32 (the preconditioner of the inner solves): the
// hardware approximation (one MUFU instruction, within about an ulp; the diagonals are normal
// numbers), the same in every kernel, so that the tile, cooperative and single-block paths stay
// identical; a preconditioner need only be fixed and symmetric, not correctly rounded.  FP64:
// correctly rounded.
__device__ inline float rcp_diag(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ inline double rcp_diag(double v) { return __drcp_rn(v); }

__device__ inline bool skip(const SolveState* s) { return s->done != 0 || s->odone != 0; }

__device__ inline unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Device timing of a tile-kernel launch (one timer per launch; the instances of a batched launch
// share their lead's).  Every block arrives once: a block that runs records its start and end
// (and the first block of each instance counts that instance as active), a block of a converged
// instance only arrives.  The last block to arrive adds the launch's span (first start to last
// end), its launch and the algorithmic bytes of its active instances, and resets the timer.
__device__ inline void timer_begin(KTimer* tm) {
    if (tm && threadIdx.x == 0) {
        atomicMin(&tm->start, gtimer());
        if (blockIdx.x == 0 && blockIdx.y == 0) atomicAdd(&tm->active, 1u);
    }
}
__device__ inline void timer_arrive(KTimer* tm, double bytes_per_instance, bool ran) {
    if (!tm) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ran) atomicMax(&tm->end, gtimer());
        __threadfence();
        unsigned int n = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(&tm->ticket, 1u) == n - 1) {
            __threadfence();
            unsigned long long s = atomicAdd(&tm->start, 0ull), e = atomicAdd(&tm->end, 0ull);
            unsigned act = atomicAdd(&tm->active, 0u);
            if (act > 0) {
                tm->total_ns += e > s ? e - s : 0ull;
                tm->launches += 1;
                tm->bytes += bytes_per_instance * act;
            }
            tm->start = ~0ull;
            tm->end = 0ull;
            tm->ticket = 0u;
            tm->active = 0u;
        }
    }
}
__device__ inline void timer_end(KTimer* tm, double bytes_per_instance) { timer_arrive(tm, bytes_per_instance, true); }

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

// Grid reductions in a fixed order.  block_partial writes the block sum of NV per-thread values
// into slot `slot` of partial (partial[k * nslot + slot], thread 0); once every block of the grid
// has written its slots, last_block_total returns true in thread 0 of the last block to arrive,
// with the totals over the nslot slots in tot[0..NV).
template <int NV>
__device__ inline void block_partial(const double* v, double* partial, int nslot, int slot) {
    __shared__ double sh[32];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double r = bsum(v[k], sh);
        if (threadIdx.x == 0) partial[k * nslot + slot] = r;
    }
}
// the same block sum in the solver precision T, converted once (thread 0): the r.z of a tile's
// FP32 cells is summed in FP32 (its slot then joins the FP64 total in tile order), so the tile
// kernels issue no FP64 shuffles
template <typename T>
__device__ inline T bsum_t(T v, T* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = T(0);
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return f2d(v); }
template <typename T, int NV>
__device__ inline void block_partial_t(const T* v, double* partial, int nslot, int slot) {
    __shared__ T sh[32];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T r = bsum_t(v[k], sh);
        if (threadIdx.x == 0) partial[k * nslot + slot] = widen(r);
    }
}
template <int NV>
__device__ inline bool last_block_total(double* partial, int nslot, unsigned* ticket, double* tot) {
    __shared__ double sh[32];
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nslot; b += blockDim.x) s += ((volatile double*)partial)[k * nslot + b];
        s = bsum(s, sh);
        if (threadIdx.x == 0) tot[k] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return threadIdx.x == 0;
}
// one slot per block; partial has room for NV x (number of blocks) doubles
template <int NV>
__device__ inline bool grid_reduce(const double* v, double* partial, unsigned* ticket, double* tot) {
    int nb = gridDim.x * gridDim.y;
    block_partial<NV>(v, partial, nb, blockIdx.y * gridDim.x + blockIdx.x);
    return last_block_total<NV>(partial, nb, ticket, tot);
}

// use 1: the loop condition is this solve's own (assigned); use 2: a batched launch, where the
// condition is the OR over the instances (reset to 0 at the top of each loop body by
// k_cond_reset, raised to 1 by every instance that continues)
__device__ inline void set_cond(cudaGraphConditionalHandle h, int use, unsigned v) {
    if (use == 1 || (use == 2 && v)) cudaGraphSetConditional(h, v);
}

__global__ void k_cond_reset(cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1, int two) {
    if (threadIdx.x == 0) {
        cudaGraphSetConditional(h0, 0u);
        if (two) cudaGraphSetConditional(h1, 0u);
    }
}

// ---- operator setup -------------------------------------------------------------------
template <typename T>
__device__ inline void coarsen_cell(int fnx, const T* fcd, const T* fdd, const T* fwl, const T* fwb, int nx, int ny,
                                    int I, int J, T* ccd, T* cdd, T* cwl, T* cwb, T* cdiag) {
    int f = (2 * J) * fnx + 2 * I;
    T s_cd = fcd[f] + fcd[f + 1] + fcd[f + fnx] + fcd[f + fnx + 1];
    T s_dd = T(0.5) * (fdd[f] + fdd[f + 1] + fdd[f + fnx] + fdd[f + fnx + 1]);
    T wl = T(0.5) * (fwl[f] + fwl[f + fnx]);
    T wb = T(0.5) * (fwb[f] + fwb[f + 1]);
    int c = J * nx + I;
    ccd[c] = s_cd;
    cdd[c] = s_dd;
    cwl[c] = wl;
    cwb[c] = wb;
    cdiag[c] = s_cd + s_dd;
    (void)ny;
}

// ---- large-level kernels: tiles with recomputed halos ------------------------------------
// A tile kernel owns a TX x TY block of cells and recomputes a halo of H cells around it, so one
// launch performs several red-black half-sweeps with no exchange between blocks (halo cells
// are recomputed from the same inputs with the same formula, so the result equals global
// red-black Gauss-Seidel exactly).
//
// Thread (k, seg) owns the cells of region columns 2k and 2k + 1 in the two rows 2 seg and
// 2 seg + 1; in every row exactly one of its two cells has the colour being swept.  A thread
// keeps its four cells' coefficients (b, the reciprocal of the full diagonal, the four face
// weights, D) in registers; only x lives in shared memory, split by colour.  The region starts
// at an even global cell (tile origins are multiples of TX, TY and the halos are even), so
// region cell (rx, ry) has colour c = (rx + ry) & 1, known at compile time for each of a
// thread's cells, and sits in column k = rx >> 1 of row ry of colour c's array (HX = SX / 2
// columns).  A colour-c cell with
// e = rx & 1 finds its left / right neighbours (colour 1 - c) in columns k - 1 + e / k + e of
// its row and its lower / upper neighbours in column k of rows ry -+ 1.
template <typename T, int NR, int H>
struct Region {
    static constexpr int SX = TX + 2 * H, SY = TY + 2 * H, HX = SX / 2, NC = SY * HX;
    static constexpr int NSEG = SY / 2, THREADS = HX * NSEG;
    static_assert(SX % 2 == 0 && SY % 2 == 0, "region sides must be even");
    // the FP64 tile kernels restrict through shared memory (their residuals in registers
    // would spill at the register count their occupancy allows); the FP32 ones in registers
    static constexpr bool RES_SMEM = sizeof(T) == 8;
    T* x0;   // x of colour 0 (NR per cell), then colour 1; then the core residuals (FP64 k_pre)
    __device__ Region(unsigned char* base) { x0 = (T*)base; }
    __device__ T* x(int c) const { return x0 + c * (NR * NC); }
    __device__ T* res() const { return x0 + 2 * NR * NC; }
    static constexpr size_t BYTES = ((size_t)2 * NC + (RES_SMEM ? TX * TY : 0)) * NR * sizeof(T);
    __host__ __device__ static constexpr size_t bytes() { return BYTES; }
};
template <int H>
constexpr int tile_block() { return (((TX + 2 * H) / 2) * ((TY + 2 * H) / 2) + 31) / 32 * 32; }
// blocks per SM the FP32 tile kernels are compiled for (register budget: two blocks, 72
// registers, measured 1.2 % faster on the 4096^2 film than three blocks with spills); the FP64
// ones keep the compiler's choice
template <typename T, int NR>
constexpr int tile_min_blocks() { return sizeof(T) == 4 ? 2 : 1; }

// ---- TMA staging of the tile regions ------------------------------------------------------
// One elected thread issues a 2-D tensor copy (cp.async.bulk.tensor) per operand array into
// dense shared-memory boxes and arms an mbarrier with their byte count; every thread waits on
// the barrier (bounded) and then reads its cells from the boxes.  A copy must start at an x
// coordinate whose byte offset is a multiple of 16, so each box starts up to A - 1 cells left
// of the region (A = 16 / bytes per cell) and the region indexes it from that offset; cells
// outside the grid are filled with zeros by the copy.
__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// wait for the phase of the barrier with the given parity; false if it did not complete within
// the bound
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity = 0) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// order this thread's earlier generic-proxy accesses to shared memory (the block's reads of a
// box, made visible to it by a block barrier) before its next async-proxy (TMA) writes there
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__host__ __device__ constexpr int pmod(int a, int m) { return ((a % m) + m) % m; }
__host__ __device__ constexpr int floordiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }
__host__ __device__ constexpr int round_up(int a, int m) { return (a + m - 1) / m * m; }
__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~size_t(127); }

// box geometry of a tile kernel with halo H; POST: k_post (also the pre-smoothed x and the
// coarse x)
template <typename T, int NR, int H, bool POST>
struct Stage {
    static constexpr int SX = TX + 2 * H, SY = TY + 2 * H;
    static constexpr int AS = 16 / (int)sizeof(T);          // x alignment of D, wl, wb (cells)
    static constexpr int AV = 16 / (NR * (int)sizeof(T));   // x alignment of the NR-vector arrays
    static constexpr int OXS = pmod(-H, AS), OXV = pmod(-H, AV), OXC = pmod(floordiv2(-H), AV);
    static constexpr int BWS = round_up(OXS + SX + 1, AS), BHS = SY + 1;   // +1: right / upper faces
    static constexpr int BWV = round_up(OXV + SX, AV), BHV = SY;
    static constexpr int BWC = round_up(OXC + SX / 2 + 1, AV), BHC = SY / 2 + 1;
    static constexpr size_t SB = (size_t)BWS * BHS * sizeof(T);
    static constexpr size_t VB = (size_t)BWV * NR * BHV * sizeof(T);
    static constexpr size_t CB = (size_t)BWC * NR * BHC * sizeof(T);
    static constexpr size_t OFF_D = 0, OFF_WL = align128(SB), OFF_WB = 2 * align128(SB), OFF_B = 3 * align128(SB);
    static constexpr size_t OFF_XIN = OFF_B + align128(VB), OFF_XC = OFF_XIN + (POST ? align128(VB) : 0);
    static constexpr size_t OFF_BAR = OFF_XC + (POST ? align128(CB) : 0);
    static constexpr size_t BYTES = OFF_BAR + 128;
    static constexpr uint32_t TX_BYTES = (uint32_t)(3 * SB + VB + (POST ? VB + CB : 0));
    static_assert(BWS <= 256 && BWV * NR <= 256 && BWC * NR <= 256 && BHS <= 256, "TMA box too large");
};

// the copies of one region into the boxes (thread 0): arms the barrier with their byte count
template <typename T, int NR, int H, bool POST>
__device__ inline void stage_issue(unsigned char* sbase, const TileMaps& M, int gx0, int gy0) {
    using Sg = Stage<T, NR, H, POST>;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sbase + Sg::OFF_BAR);
    mbar_expect_tx(bar, Sg::TX_BYTES);
    int xs = gx0 - Sg::OXS, xv = (gx0 - Sg::OXV) * NR;
    tma_load_2d(sbase + Sg::OFF_D, &M.d, xs, gy0, bar);
    tma_load_2d(sbase + Sg::OFF_WL, &M.wl, xs, gy0, bar);
    tma_load_2d(sbase + Sg::OFF_WB, &M.wb, xs, gy0, bar);
    tma_load_2d(sbase + Sg::OFF_B, &M.b, xv, gy0, bar);
    if (POST) {
        tma_load_2d(sbase + Sg::OFF_XIN, &M.xin, xv, gy0, bar);
        tma_load_2d(sbase + Sg::OFF_XC, &M.xc, ((gx0 >> 1) - Sg::OXC) * NR, gy0 >> 1, bar);
    }
}

// barrier set-up (thread 0), visible to the block after the barrier
template <typename T, int NR, int H, bool POST>
__device__ inline void stage_init(unsigned char* sbase) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(sbase + Stage<T, NR, H, POST>::OFF_BAR);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
}

// The tiles of a TMA-staged tile kernel, persistent: block b takes tiles b, b + G, ... (G blocks).
// The next tile's boxes are requested as soon as the current tile has been read out of them
// (into registers and the region), so the copies overlap the current tile's sweeps.  work(t,
// after_load) runs tile t and calls after_load() once the boxes have been read and the block has
// passed a barrier.  A copy that does not land within the bound sets st->fault bit 0 and ends
// the loop (the decision is the same in every thread) after one more bounded wait for that
// copy, the only one in flight.
template <typename T, int NR, int H, bool POST, class Work>
__device__ inline void staged_tiles(unsigned char* sbase, const TileMaps& M, int tx, int nt, SolveState* st,
                                    Work&& work) {
    using Sg = Stage<T, NR, H, POST>;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sbase + Sg::OFF_BAR);
    stage_init<T, NR, H, POST>(sbase);
    // tile t = by tx + bx, advanced by gridDim.x = gq tx + gr without a division per tile
    int t = blockIdx.x, bx = t % tx, by = t / tx;
    const int gq = (int)gridDim.x / tx, gr = (int)gridDim.x % tx;
    if (threadIdx.x == 0 && t < nt) stage_issue<T, NR, H, POST>(sbase, M, bx * TX - H, by * TY - H);
    for (uint32_t i = 0; t < nt; ++i) {
        bool landed = mbar_wait_bounded(bar, i & 1u);
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(&st->fault, 1);
            mbar_wait_bounded(bar, i & 1u);
            __syncthreads();
            break;
        }
        int tn = t + gridDim.x, bxn = bx + gr, byn = by + gq;
        if (bxn >= tx) { bxn -= tx; ++byn; }
        work(t, bx, by, [&]() {
            if (threadIdx.x == 0 && tn < nt) {
                fence_proxy_async();
                stage_issue<T, NR, H, POST>(sbase, M, bxn * TX - H, byn * TY - H);
            }
        });
        __syncthreads();   // the region is rewritten by the next tile
        t = tn;
        bx = bxn;
        by = byn;
    }
}


// the thread's four cells: [r][c] = row ry0 + r (ry0 even), colour c; its column is 2k + (c ^ r)
template <typename T, int NR>
struct Cells {
    T b[2][2][NR], id[2][2], wl[2][2], wr[2][2], wb[2][2], wt[2][2], d[2][2];
    // the cells' current x (the copy in shared memory is for the neighbour threads): two of a
    // cell's four neighbours are the thread's own cells of the other colour
    T x[2][2][NR];
};

// load the thread's cells (coefficients to registers, x to shared memory: for pre-smoothing
// the result of the first colour-0 half-sweep from x = 0, for post-smoothing xin + the
// prolongated coarse x); cells outside the domain get D = 1, zero weights, b = x = 0, so
// sweeps leave them 0
template <typename T, int NR, int H, bool POST, bool CHECK>
__device__ inline void tile_load_cells(Region<T, NR, H>& R, Cells<T, NR>& C, int k, int ry0, const Lev<T>& L,
                                       const T* __restrict__ b, const T* __restrict__ xin, const T* __restrict__ xc,
                                       int cnx, int gx0, int gy0, const unsigned char* stage) {
    constexpr int HX = Region<T, NR, H>::HX;
    using Sg = Stage<T, NR, H, POST>;
    static_assert(H % 2 == 0 && TX % 2 == 0 && TY % 2 == 0, "regions must start at an even cell");
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int ry = ry0 + r;
        int gj = gy0 + ry;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            int rx = 2 * k + e;
            int gi = gx0 + rx;
            bool in = !CHECK || (gj >= 0 && gj < L.ny && gi >= 0 && gi < L.nx);
            Vec<T, NR> bv, xv;
            T dv, wlv, wbv, wrv, wtv;
            if (stage) {
                // from the TMA boxes (zeros outside the grid)
                const T* sd = reinterpret_cast<const T*>(stage + Sg::OFF_D);
                const T* swl = reinterpret_cast<const T*>(stage + Sg::OFF_WL);
                const T* swb = reinterpret_cast<const T*>(stage + Sg::OFF_WB);
                const T* sb = reinterpret_cast<const T*>(stage + Sg::OFF_B);
                int qs = ry * Sg::BWS + rx + Sg::OXS, qv = (ry * Sg::BWV + rx + Sg::OXV) * NR;
                dv = sd[qs];
                wlv = swl[qs];
                wbv = swb[qs];
                wrv = swl[qs + 1];
                wtv = swb[qs + Sg::BWS];
#pragma unroll
                for (int k2 = 0; k2 < NR; ++k2) bv.v[k2] = sb[qv + k2];
                if (POST) {
                    const T* sx = reinterpret_cast<const T*>(stage + Sg::OFF_XIN);
                    const T* sc = reinterpret_cast<const T*>(stage + Sg::OFF_XC);
                    int cx = (gi >> 1) - ((gx0 >> 1) - Sg::OXC), cy = (gj >> 1) - (gy0 >> 1);
                    int qc = (cy * Sg::BWC + cx) * NR;
#pragma unroll
                    for (int k2 = 0; k2 < NR; ++k2) xv.v[k2] = sx[qv + k2] + sc[qc + k2];
                } else {
#pragma unroll
                    for (int k2 = 0; k2 < NR; ++k2) xv.v[k2] = T(0);
                }
            } else {
                // unconditional loads (clamped, then masked): all of them can be in flight at once
                int gic = CHECK ? min(max(gi, 0), L.nx - 1) : gi, gjc = CHECK ? min(max(gj, 0), L.ny - 1) : gj;
                int g = gjc * L.nx + gic;
                bv = reinterpret_cast<const Vec<T, NR>*>(b)[g];
                dv = L.diag[g];
                wlv = L.wl[g];
                wbv = L.wb[g];
                wrv = L.wl[!CHECK || gic + 1 < L.nx ? g + 1 : g];
                wtv = L.wb[!CHECK || gjc + 1 < L.ny ? g + L.nx : g];
                if (CHECK && gi + 1 >= L.nx) wrv = T(0);
                if (CHECK && gj + 1 >= L.ny) wtv = T(0);
                if (POST) {
                    xv = reinterpret_cast<const Vec<T, NR>*>(xin)[g];
                    Vec<T, NR> cv = reinterpret_cast<const Vec<T, NR>*>(xc)[(gjc >> 1) * cnx + (gic >> 1)];
#pragma unroll
                    for (int k2 = 0; k2 < NR; ++k2) xv.v[k2] += cv.v[k2];
                } else {
#pragma unroll
                    for (int k2 = 0; k2 < NR; ++k2) xv.v[k2] = T(0);
                }
            }
            if (CHECK && !in) {
#pragma unroll
                for (int k2 = 0; k2 < NR; ++k2) { bv.v[k2] = T(0); xv.v[k2] = T(0); }
                dv = T(1);
                wlv = wbv = wrv = wtv = T(0);
            }
            // this cell's colour is e ^ r (both known at compile time)
            bool mine0 = (e ^ r) == 0;
            T idv = rcp_diag(dv + wlv + wrv + wbv + wtv);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                bool m = (c == 0) == mine0;
                if (m) {
#pragma unroll
                    for (int k2 = 0; k2 < NR; ++k2) C.b[r][c][k2] = bv.v[k2];
                    C.id[r][c] = idv;
                    C.wl[r][c] = wlv;
                    C.wr[r][c] = wrv;
                    C.wb[r][c] = wbv;
                    C.wt[r][c] = wtv;
                    C.d[r][c] = dv;
                }
            }
            int cc = e ^ r;
            if (!POST && cc == 0) {
                // pre-smoothing starts from x = 0: its first (colour-0) half-sweep reads only
                // zeros and reduces to x = b / (full diagonal), done here
#pragma unroll
                for (int k2 = 0; k2 < NR; ++k2) xv.v[k2] = bv.v[k2] * idv;
            }
            T* xd = R.x(cc) + (ry * HX + k) * NR;
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                xd[k2] = xv.v[k2];
                C.x[r][cc][k2] = xv.v[k2];
            }
        }
    }
}

// A region wholly inside the grid, with the right and upper faces of its last cells too (all
// but the tiles along the grid's edges), needs no range tests or masks
template <typename T, int NR, int H, bool POST>
__device__ inline void tile_load(Region<T, NR, H>& R, Cells<T, NR>& C, int k, int ry0, const Lev<T>& L,
                                 const T* __restrict__ b, const T* __restrict__ xin, const T* __restrict__ xc,
                                 int cnx, int gx0, int gy0, const unsigned char* stage) {
    constexpr int SX = Region<T, NR, H>::SX, SY = Region<T, NR, H>::SY;
    if (gx0 >= 0 && gy0 >= 0 && gx0 + SX < L.nx && gy0 + SY < L.ny)
        tile_load_cells<T, NR, H, POST, false>(R, C, k, ry0, L, b, xin, xc, cnx, gx0, gy0, stage);
    else
        tile_load_cells<T, NR, H, POST, true>(R, C, k, ry0, L, b, xin, xc, cnx, gx0, gy0, stage);
}

// A thread's place in a tile region, the same for every tile of a launch (computed once per
// launch, one register): bit 2 (S - 1) + r is set if half-sweep S updates the thread's cell
// (r, COLOR ^ r) (distance >= S from the region's edge; COLOR, the sweep's colour, is S & 1),
// bit 8 + 2 r + c if cell (r, c) lies in the tile's core, bit 12 if the thread owns cells.  The
// column pair k and the row pair ry0 follow from threadIdx (a division by a constant).
struct TileThread {
    unsigned m;
    __device__ bool act() const { return (m >> 12) & 1u; }
    __device__ bool sweeps(int S, int r) const { return (m >> (2 * (S - 1) + r)) & 1u; }
    __device__ bool core(int r, int c) const { return (m >> (8 + 2 * r + c)) & 1u; }
};
template <int H>
__device__ inline TileThread tile_thread() {
    constexpr int SX = TX + 2 * H, SY = TY + 2 * H, HX = SX / 2, THREADS = HX * (SY / 2);
    const int k = threadIdx.x % HX, ry0 = 2 * (threadIdx.x / HX);
    unsigned m = threadIdx.x < THREADS ? 1u << 12 : 0u;
#pragma unroll
    for (int S = 1; S <= 4; ++S)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int ry = ry0 + r, rx = 2 * k + ((S & 1) ^ r);
            if (ry >= S && ry < SY - S && rx >= S && rx < SX - S) m |= 1u << (2 * (S - 1) + r);
        }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            int ry = ry0 + r, rx = 2 * k + (c ^ r);
            if (rx >= H && rx < H + TX && ry >= H && ry < H + TY) m |= 1u << (8 + 2 * r + c);
        }
    return TileThread{m};
}

// one Gauss-Seidel half-sweep of colour COLOR over the region cells at distance >= S from its
// edge; both rows' operands are loaded before either result is stored.  Cell (r, e) of the
// thread (colour COLOR, e = COLOR ^ r) has its horizontal neighbour 2k + 1 - e and its vertical
// neighbour in row 1 - r among the thread's own cells (registers); the other two come from the
// neighbour threads through shared memory.
template <typename T, int NR, int H, int S, int COLOR>
__device__ inline void tile_sweep(Region<T, NR, H>& R, Cells<T, NR>& C, const TileThread& tt) {
    static_assert(COLOR == (S & 1), "half-sweep S has colour S & 1");
    using Rg = Region<T, NR, H>;
    constexpr int HX = Rg::HX;
    const int k = threadIdx.x % HX, ry0 = 2 * (threadIdx.x / HX);
    if (tt.act()) {
        const T* xo = R.x(1 - COLOR);
        T acc[2][NR];
        bool ok[2];
        int qs[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int ry = ry0 + r;
            const int e = COLOR ^ r;
            ok[r] = tt.sweeps(S, r);
            int q = ok[r] ? ry * HX + k : HX + 1;   // a harmless in-range slot otherwise
            qs[r] = q;
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                const T own_h = C.x[r][1 - COLOR][k2], own_v = C.x[1 - r][1 - COLOR][k2];
                T xl = e == 1 ? own_h : xo[(q - 1) * NR + k2];
                T xrt = e == 0 ? own_h : xo[(q + 1) * NR + k2];
                T xd = r == 1 ? own_v : xo[(q - HX) * NR + k2];
                T xu = r == 0 ? own_v : xo[(q + HX) * NR + k2];
                acc[r][k2] = (C.b[r][COLOR][k2] + C.wl[r][COLOR] * xl + C.wr[r][COLOR] * xrt +
                              C.wb[r][COLOR] * xd + C.wt[r][COLOR] * xu) *
                             C.id[r][COLOR];
            }
        }
        T* xs = R.x(COLOR);
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (ok[r])
#pragma unroll
                for (int k2 = 0; k2 < NR; ++k2) {
                    xs[qs[r] * NR + k2] = acc[r][k2];
                    C.x[r][COLOR][k2] = acc[r][k2];
                }
    }
    __syncthreads();
}

// the thread's core cells (inside the TX x TY tile and the domain): f(r, c, rx, ry, q, gi, gj)
template <typename T, int NR, int H, class Fn>
__device__ inline void tile_core_cells(const Cells<T, NR>& C, const TileThread& tt, int gx0, int gy0,
                                       const Lev<T>& L, Fn&& f) {
    constexpr int HX = Region<T, NR, H>::HX;
    const int k = threadIdx.x % HX, ry0 = 2 * (threadIdx.x / HX);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int ry = ry0 + r;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            int rx = 2 * k + (c ^ r);
            int gi = gx0 + rx, gj = gy0 + ry;
            if (tt.core(r, c) && gi < L.nx && gj < L.ny) f(r, c, rx, ry, ry * HX + k, gi, gj);
        }
    }
}

struct NoOp {
    __device__ void operator()() const {}
};

// pre-smoothing of tile (bx, by): x = S^nu(0; b) on the tile (red-black order), coarse
// b = R (b - A x); smem holds the region (stage: its TMA boxes, already landed, or null);
// after_load() runs in every thread once the boxes have been read
template <typename T, int NR, class AfterLoad = NoOp>
__device__ inline void pre_tile(const Lev<T>& L, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ bc,
                                int bx, int by, unsigned char* smem, const unsigned char* stage,
                                const TileThread& tt, AfterLoad after_load = AfterLoad()) {
    constexpr int H = HPRE;
    static_assert(NU == 2, "the sweep sequence below is written out for two pairs");
    using Rg = Region<T, NR, H>;
    constexpr int HX = Rg::HX;
    Rg R(smem);
    int gx0 = bx * TX - H, gy0 = by * TY - H;
    const bool act = tt.act();
    const int k = threadIdx.x % HX, ry0 = 2 * (threadIdx.x / HX);
    Cells<T, NR> C;
    if (act) tile_load<T, NR, H, false>(R, C, k, ry0, L, b, nullptr, nullptr, 0, gx0, gy0, stage);
    __syncthreads();
    after_load();
    // the first colour-0 half-sweep (from x = 0) was done by tile_load
    tile_sweep<T, NR, H, 1, 1>(R, C, tt);
    tile_sweep<T, NR, H, 2, 0>(R, C, tt);
    tile_sweep<T, NR, H, 3, 1>(R, C, tt);
    // x of the core cells to global memory; their residuals stay in registers ([r][e]: row
    // ry0 + r, column 2k + e), or go to shared memory (FP64)
    T res[2][2][NR];
    T* sres = R.res();
    if (act)
        tile_core_cells<T, NR, H>(C, tt, gx0, gy0, L, [&](int r, int c, int rx, int ry, int q, int gi, int gj) {
            const T* xo = R.x(1 - c);
            const int e = c ^ r;   // rx = 2k + e
            Vec<T, NR> xv;
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                T x0v = C.x[r][c][k2];
                xv.v[k2] = x0v;
                const T own_h = C.x[r][1 - c][k2], own_v = C.x[1 - r][1 - c][k2];
                T xl = e == 1 ? own_h : xo[(q - 1) * NR + k2];
                T xrt = e == 0 ? own_h : xo[(q + 1) * NR + k2];
                T xd = r == 1 ? own_v : xo[(q - HX) * NR + k2];
                T xu = r == 0 ? own_v : xo[(q + HX) * NR + k2];
                T ax = C.d[r][c] * x0v + C.wl[r][c] * (x0v - xl) + C.wr[r][c] * (x0v - xrt) +
                       C.wb[r][c] * (x0v - xd) + C.wt[r][c] * (x0v - xu);
                if constexpr (Rg::RES_SMEM) sres[((ry - H) * TX + (rx - H)) * NR + k2] = C.b[r][c][k2] - ax;
                else res[r][e][k2] = C.b[r][c][k2] - ax;
            }
            reinterpret_cast<Vec<T, NR>*>(x)[gj * L.nx + gi] = xv;
        });
    int cnx = L.nx / 2, cny = L.ny / 2;
    if constexpr (Rg::RES_SMEM) {
        __syncthreads();
        // restriction: sum of the four children (the core starts at an even global index, so
        // children (2ti + a, 2tj + b) are core cells)
        for (int t = threadIdx.x; t < (TX / 2) * (TY / 2); t += blockDim.x) {
            int ti = t % (TX / 2), tj = t / (TX / 2);
            int ci = bx * (TX / 2) + ti, cj = by * (TY / 2) + tj;
            if (ci >= cnx || cj >= cny) continue;
            Vec<T, NR> acc;
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2)
                acc.v[k2] = sres[((2 * tj) * TX + 2 * ti) * NR + k2] + sres[((2 * tj) * TX + 2 * ti + 1) * NR + k2] +
                            sres[((2 * tj + 1) * TX + 2 * ti) * NR + k2] +
                            sres[((2 * tj + 1) * TX + 2 * ti + 1) * NR + k2];
            reinterpret_cast<Vec<T, NR>*>(bc)[cj * cnx + ci] = acc;
        }
        return;
    }
    // restriction: sum of the four children.  The region starts H (even) cells before the tile,
    // so a thread's 2 x 2 block is the four children of coarse cell (k - H/2, ry0/2 - H/2) of the
    // tile; a coarse cell of the grid has all four children inside the grid, hence computed above
    int ti = k - H / 2, tj = ry0 / 2 - H / 2;
    if (act && ti >= 0 && ti < TX / 2 && tj >= 0 && tj < TY / 2) {
        int ci = bx * (TX / 2) + ti, cj = by * (TY / 2) + tj;
        if (ci < cnx && cj < cny) {
            Vec<T, NR> acc;
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) acc.v[k2] = res[0][0][k2] + res[0][1][k2] + res[1][0][k2] + res[1][1][k2];
            reinterpret_cast<Vec<T, NR>*>(bc)[cj * cnx + ci] = acc;
        }
    }
}

// k_pre: one tile per block
template <typename T, int NR>
__global__ void __launch_bounds__(tile_block<HPRE>(), tile_min_blocks<T, NR>())
k_pre(Lev<T> L, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ bc, SolveState* st, KTimer* tm,
      const __grid_constant__ TileMaps maps, int use_tma, unsigned* coop_bar) {
    // the cooperative coarse-cycle launch that follows this (level-0) launch counts its
    // barrier arrivals from 0; the previous one has completed (stream order)
    if (coop_bar && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) *coop_bar = 0u;
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    b = zsh(b, zo);
    x = zsh(x, zo);
    bc = zsh(bc, zo);
    st = zsh(st, zo);
    constexpr double bytes_cell = sizeof(T) * (3.0 + NR * 2.25);
    if (skip(st)) {
        timer_arrive(tm, 0.0, false);
        return;
    }
    constexpr int H = HPRE;
    using Rg = Region<T, NR, H>;
    extern __shared__ __align__(128) unsigned char smem[];
    timer_begin(tm);
    if (use_tma) {
        // persistent blocks over the tiles (1-D grid), TMA boxes 128-byte aligned after the
        // region (the launch reserves 128 bytes of slack)
        unsigned char* stage =
            reinterpret_cast<unsigned char*>(align128(reinterpret_cast<uintptr_t>(smem) + Rg::BYTES));
        int tx = (L.nx + TX - 1) / TX, nt = tx * ((L.ny + TY - 1) / TY);
        const TileThread tt = tile_thread<H>();
        staged_tiles<T, NR, H, false>(stage, maps, tx, nt, st, [&](int, int bx, int by, auto after_load) {
            pre_tile<T, NR>(L, b, x, bc, bx, by, smem, stage, tt, after_load);
        });
    } else {
        pre_tile<T, NR>(L, b, x, bc, blockIdx.x, blockIdx.y, smem, nullptr, tile_thread<H>());
    }
    // algorithmic bytes: b, diag, wl, wb read; x and the quarter-size coarse b written
    timer_end(tm, (double)L.nx * L.ny * bytes_cell);
}

// post-smoothing of tile (bx, by): x = xin + P xc, then black-red sweeps; returns the tile's
// part of r.z (each right-hand side) when DOT; after_load() as for pre_tile
template <typename T, int NR, bool DOT, class AfterLoad = NoOp>
__device__ inline Vec<T, 2> post_tile(const Lev<T>& L, const T* __restrict__ b, const T* __restrict__ xin,
                                    T* __restrict__ x, const T* __restrict__ xc, int bx, int by, unsigned char* smem,
                                    const unsigned char* stage, const TileThread& tt,
                                    AfterLoad after_load = AfterLoad()) {
    constexpr int H = HPOST;
    using Rg = Region<T, NR, H>;
    Rg R(smem);
    int gx0 = bx * TX - H, gy0 = by * TY - H;
    constexpr int HX = Rg::HX;
    const bool act = tt.act();
    Cells<T, NR> C;
    if (act)
        tile_load<T, NR, H, true>(R, C, threadIdx.x % HX, 2 * (threadIdx.x / HX), L, b, xin, xc, L.nx / 2, gx0, gy0,
                                  stage);
    __syncthreads();
    after_load();
    tile_sweep<T, NR, H, 1, 1>(R, C, tt);
    tile_sweep<T, NR, H, 2, 0>(R, C, tt);
    tile_sweep<T, NR, H, 3, 1>(R, C, tt);
    tile_sweep<T, NR, H, 4, 0>(R, C, tt);
    // r.z of the thread's (at most four) core cells, summed in T
    Vec<T, 2> dot;
    dot.v[0] = dot.v[1] = T(0);
    if (act)
        tile_core_cells<T, NR, H>(C, tt, gx0, gy0, L, [&](int r, int c, int rx, int ry, int q, int gi, int gj) {
            Vec<T, NR> xv;
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                xv.v[k2] = C.x[r][c][k2];
                if (DOT) dot.v[k2] += xv.v[k2] * C.b[r][c][k2];
            }
            reinterpret_cast<Vec<T, NR>*>(x)[gj * L.nx + gi] = xv;
        });
    return dot;
}

// k_post: one tile per block; at the finest level also r.z -> beta
template <typename T, int NR, bool DOT>
__global__ void __launch_bounds__(tile_block<HPOST>(), tile_min_blocks<T, NR>())
k_post(Lev<T> L, const T* __restrict__ b, const T* __restrict__ xin, T* __restrict__ x, const T* __restrict__ xc,
       SolveState* st, double* partial, unsigned* ticket, KTimer* tm, const __grid_constant__ TileMaps maps,
       int use_tma) {
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    b = zsh(b, zo);
    xin = zsh(xin, zo);
    x = zsh(x, zo);
    xc = zsh(xc, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    constexpr double bytes_cell = sizeof(T) * (3.0 + NR * 3.25);
    if (skip(st)) {
        timer_arrive(tm, 0.0, false);
        return;
    }
    constexpr int H = HPOST;
    using Rg = Region<T, NR, H>;
    extern __shared__ __align__(128) unsigned char smem[];
    timer_begin(tm);
    int nslot = gridDim.x * gridDim.y;
    if (use_tma) {
        // persistent blocks over the tiles (1-D grid); r.z summed over the block's tiles
        unsigned char* stage =
            reinterpret_cast<unsigned char*>(align128(reinterpret_cast<uintptr_t>(smem) + Rg::BYTES));
        int tx = (L.nx + TX - 1) / TX, nt = tx * ((L.ny + TY - 1) / TY);
        // r.z: one slot per tile, summed in tile order as with one block per tile
        const TileThread tt = tile_thread<H>();
        staged_tiles<T, NR, H, true>(stage, maps, tx, nt, st, [&](int t, int bx, int by, auto after_load) {
            Vec<T, 2> d = post_tile<T, NR, DOT>(L, b, xin, x, xc, bx, by, smem, stage, tt, after_load);
            if (DOT) block_partial_t<T, NR>(d.v, partial, nt, t);
        });
        nslot = nt;
    } else {
        Vec<T, 2> d = post_tile<T, NR, DOT>(L, b, xin, x, xc, blockIdx.x, blockIdx.y, smem, nullptr,
                                            tile_thread<H>());
        if (DOT) block_partial_t<T, NR>(d.v, partial, nslot, blockIdx.y * gridDim.x + blockIdx.x);
    }
    if (DOT) {
        double tot[NR];
        if (last_block_total<NR>(partial, nslot, ticket, tot)) {
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                double old = st->rz[k2];
                st->beta[k2] = old != 0.0 ? tot[k2] / old : 0.0;
                st->rz[k2] = tot[k2];
            }
        }
    }
    // algorithmic bytes: b, x, the quarter-size coarse x, diag, wl, wb read; x written
    timer_end(tm, (double)L.nx * L.ny * bytes_cell);
}

// ---- small levels: the rest of the V-cycle in one block ---------------------------------
struct SmallPlan {
    int n;             // number of small levels
    int nx[Solver::MAXLEV], ny[Solver::MAXLEV];
    int soff[Solver::MAXLEV];   // cell offset of each small level inside the shared-memory arrays
    size_t goff[Solver::MAXLEV]; // cell offset in the packed global level arrays
    int total;         // cells of all small levels
    long long zs;      // byte stride between the instances of a batched launch
};

// shared-memory layout: x[NR*total], b[NR*total], diag[total], wl[total], wb[total]
template <typename T, int NR>
struct SmallMem {
    T *x, *b, *d, *wl, *wb, *id;   // id: reciprocal of the full diagonal D + the four face weights
    __device__ SmallMem(unsigned char* base, int total) {
        x = (T*)base;
        b = x + (size_t)NR * total;
        d = b + (size_t)NR * total;
        wl = d + total;
        wb = wl + total;
        id = wb + total;
    }
    static size_t bytes(int total) { return (size_t)total * (2 * NR + 4) * sizeof(T); }
};

// The small levels run in one block.  Their half-sweeps are short, so a block-wide barrier
// between them costs more than the work; the levels with at most SMALL_WARP_CELLS cells (and
// every level below them) therefore run on warp 0 alone, with warp barriers.  Team<WARP> is
// the group of threads of one part: the whole block, or warp 0.
constexpr int SMALL_WARP_CELLS = 64;
template <bool WARP>
struct Team {
    __device__ static int size() { return WARP ? 32 : (int)blockDim.x; }
    __device__ static void sync() {
        if (WARP) __syncwarp();
        else __syncthreads();
    }
};

// lane layout of a row sweep over rows of width w: 2^ls lanes (the smallest power of two >= w,
// at most 32) take a row, so a warp covers 32 >> ls rows at once and no lane idles on the
// narrow levels; row j0 + m * jstep, column i0 + m * istep
template <bool WARP>
struct RowLanes {
    int jr, ic, jstep, istep;
    __device__ RowLanes(int w) {
        int ls = w <= 1 ? 0 : 32 - __clz(w - 1);
        ls = ls < 5 ? ls : 5;
        int rpw = 32 >> ls, lane = threadIdx.x & 31;
        jr = (WARP ? 0 : (int)(threadIdx.x >> 5)) * rpw + (lane >> ls);
        ic = lane & ((1 << ls) - 1);
        jstep = (Team<WARP>::size() >> 5) * rpw;
        istep = 1 << ls;
    }
};

// a small level's sizes, offset and half-sweep lane layout, set up once for all its sweeps
template <bool WARP>
struct SmallLevel {
    int nx, ny, o, hx;
    RowLanes<WARP> G;
    __device__ SmallLevel(const SmallPlan& P, int l)
        : nx(P.nx[l]), ny(P.ny[l]), o(P.soff[l]), hx((P.nx[l] + 1) >> 1), G((P.nx[l] + 1) >> 1) {}
};

// one red-black half-sweep of colour `color` on a level (a row holds ceil(nx / 2) cells of a
// colour)
template <typename T, int NR, bool WARP>
__device__ inline void small_sweep(const SmallLevel<WARP>& V, SmallMem<T, NR>& M, int color) {
    const int nx = V.nx, ny = V.ny, o = V.o, hx = V.hx;
    const RowLanes<WARP>& G = V.G;
    for (int j = G.jr; j < ny; j += G.jstep)
        for (int i2 = G.ic; i2 < hx; i2 += G.istep) {
            int i = 2 * i2 + ((color + j) & 1);
            if (i >= nx) continue;
            int q = o + j * nx + i;
            T w0 = M.wl[q], w1 = i < nx - 1 ? M.wl[q + 1] : T(0), w2 = M.wb[q], w3 = j < ny - 1 ? M.wb[q + nx] : T(0);
            T id = M.id[q];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                T a = M.b[q * NR + k];
                if (i > 0) a += w0 * M.x[(q - 1) * NR + k];
                if (i < nx - 1) a += w1 * M.x[(q + 1) * NR + k];
                if (j > 0) a += w2 * M.x[(q - nx) * NR + k];
                if (j < ny - 1) a += w3 * M.x[(q + nx) * NR + k];
                M.x[q * NR + k] = a * id;
            }
        }
    Team<WARP>::sync();
}

// down-leg smoothing of level l from x = 0 (its first colour-0 half-sweep reads only zeros and
// reduces to x = b / (full diagonal), written together with zeros on colour 1), then the
// residual restricted to level l + 1
template <typename T, int NR, bool WARP>
__device__ inline void small_down(const SmallPlan& P, int l, SmallMem<T, NR>& M) {
    SmallLevel<WARP> V(P, l);
    const int nx = V.nx, ny = V.ny, o = V.o;
    {
        RowLanes<WARP> G(nx);
        for (int j = G.jr; j < ny; j += G.jstep)
            for (int i = G.ic; i < nx; i += G.istep) {
                int q = o + j * nx + i;
                bool c0 = ((i + j) & 1) == 0;
                T id = M.id[q];
#pragma unroll
                for (int k = 0; k < NR; ++k) M.x[q * NR + k] = c0 ? M.b[q * NR + k] * id : T(0);
            }
        Team<WARP>::sync();
    }
    small_sweep<T, NR, WARP>(V, M, 1);
    for (int k = 1; k < NU_SMALL; ++k) {
        small_sweep<T, NR, WARP>(V, M, 0);
        small_sweep<T, NR, WARP>(V, M, 1);
    }
    int cnx = P.nx[l + 1], cny = P.ny[l + 1], co = P.soff[l + 1];
    RowLanes<WARP> G(cnx);
    for (int J = G.jr; J < cny; J += G.jstep)
        for (int I = G.ic; I < cnx; I += G.istep) {
            T acc[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = T(0);
            for (int d2 = 0; d2 < 4; ++d2) {
                int i = 2 * I + (d2 & 1), j = 2 * J + (d2 >> 1);
                int q = o + j * nx + i;
                T w0 = M.wl[q], w1 = i < nx - 1 ? M.wl[q + 1] : T(0), w2 = M.wb[q],
                  w3 = j < ny - 1 ? M.wb[q + nx] : T(0);
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    T xq = M.x[q * NR + k];
                    T ax = M.d[q] * xq;
                    if (i > 0) ax += w0 * (xq - M.x[(q - 1) * NR + k]);
                    if (i < nx - 1) ax += w1 * (xq - M.x[(q + 1) * NR + k]);
                    if (j > 0) ax += w2 * (xq - M.x[(q - nx) * NR + k]);
                    if (j < ny - 1) ax += w3 * (xq - M.x[(q + nx) * NR + k]);
                    acc[k] += M.b[q * NR + k] - ax;
                }
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) M.b[(co + J * cnx + I) * NR + k] = acc[k];
        }
    Team<WARP>::sync();
}

// coarsest level: exact solve with the precomputed inverse (up to 32 cells), else a symmetric
// red-black sweep sequence from zero
template <typename T, int NR, bool WARP>
__device__ inline void small_coarsest(const SmallPlan& P, SmallMem<T, NR>& M, const T* __restrict__ inv) {
    int l = P.n - 1, o = P.soff[l], n = P.nx[l] * P.ny[l];
    if (n <= 32 && inv[n * n] == T(1)) {
        if (threadIdx.x < 32) {
            int r = threadIdx.x;
            T acc[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = T(0);
            if (r < n)
                for (int c = 0; c < n; ++c) {
                    T a = inv[r * n + c];
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += a * M.b[(o + c) * NR + k];
                }
            __syncwarp();
            if (r < n)
#pragma unroll
                for (int k = 0; k < NR; ++k) M.x[(o + r) * NR + k] = acc[k];
        }
        Team<WARP>::sync();
    } else {
        int t = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
        for (int c = t; c < n * NR; c += Team<WARP>::size()) M.x[o * NR + c] = T(0);
        Team<WARP>::sync();
        SmallLevel<WARP> V(P, l);
        for (int k = 0; k < COARSE_PAIRS; ++k) {
            small_sweep<T, NR, WARP>(V, M, 0);
            small_sweep<T, NR, WARP>(V, M, 1);
        }
        for (int k = 0; k < COARSE_PAIRS; ++k) {
            small_sweep<T, NR, WARP>(V, M, 1);
            small_sweep<T, NR, WARP>(V, M, 0);
        }
    }
}

// up-leg of level l: x += P x_{l+1}, then the post-smoothing half-sweeps
template <typename T, int NR, bool WARP>
__device__ inline void small_up(const SmallPlan& P, int l, SmallMem<T, NR>& M) {
    SmallLevel<WARP> V(P, l);
    const int nx = V.nx, ny = V.ny, o = V.o, cnx = P.nx[l + 1], co = P.soff[l + 1];
    RowLanes<WARP> G(nx);
    for (int j = G.jr; j < ny; j += G.jstep)
        for (int i = G.ic; i < nx; i += G.istep) {
#pragma unroll
            for (int k = 0; k < NR; ++k)
                M.x[(o + j * nx + i) * NR + k] += M.x[(co + (j >> 1) * cnx + (i >> 1)) * NR + k];
        }
    Team<WARP>::sync();
    for (int k = 0; k < NU_SMALL; ++k) {
        small_sweep<T, NR, WARP>(V, M, 1);
        small_sweep<T, NR, WARP>(V, M, 0);
    }
}

// the V-cycle on the small levels in one block, from the level-(first small) rhs b_in to its
// correction x_out; with DOT (the cycle starts at the finest level) also r.z -> beta
template <typename T, int NR, bool DOT>
__device__ void small_cycle(const SmallPlan& P, const T* __restrict__ diag, const T* __restrict__ wl,
                            const T* __restrict__ wb, const T* __restrict__ inv, const T* __restrict__ b_in,
                            T* __restrict__ x_out, SolveState* st, unsigned char* smem) {
    SmallMem<T, NR> M(smem, P.total);
    // the small levels are contiguous in the packed level arrays and in shared memory: one flat
    // copy per array, four independent loads in flight per thread and array
    {
        const T* gd = diag + P.goff[0];
        const T* gl = wl + P.goff[0];
        const T* gb = wb + P.goff[0];
        int tot = P.total;
#pragma unroll 4
        for (int c = threadIdx.x; c < tot; c += blockDim.x) {
            T a = gd[c], b2 = gl[c], c2 = gb[c];
            M.d[c] = a;
            M.wl[c] = b2;
            M.wb[c] = c2;
        }
    }
    int n0 = P.nx[0] * P.ny[0];
#pragma unroll 4
    for (int c = threadIdx.x; c < n0 * NR; c += blockDim.x) M.b[c] = b_in[c];
    __syncthreads();
    for (int l = 0; l < P.n; ++l) {
        int nx = P.nx[l], ny = P.ny[l], o = P.soff[l];
        RowLanes<false> G(nx);
        for (int j = G.jr; j < ny; j += G.jstep)
            for (int i = G.ic; i < nx; i += G.istep) {
                int q = o + j * nx + i;
                T dg = M.d[q] + M.wl[q] + (i < nx - 1 ? M.wl[q + 1] : T(0)) + M.wb[q] +
                       (j < ny - 1 ? M.wb[q + nx] : T(0));
                M.id[q] = rcp_diag(dg);
            }
    }
    __syncthreads();
    // down to the first level of at most SMALL_WARP_CELLS cells (lw) on the whole block, the
    // levels from lw on (coarsest included) on warp 0, then up on the whole block
    int lw = P.n;
    for (int l = 0; l < P.n; ++l)
        if (P.nx[l] * P.ny[l] <= SMALL_WARP_CELLS) {
            lw = l;
            break;
        }
    int lb = lw < P.n - 1 ? lw : P.n - 1;   // levels [0, lb) have block-wide down and up legs
    for (int l = 0; l < lb; ++l) small_down<T, NR, false>(P, l, M);
    if (lw < P.n) {
        if (threadIdx.x < 32) {
            for (int l = lw; l < P.n - 1; ++l) small_down<T, NR, true>(P, l, M);
            small_coarsest<T, NR, true>(P, M, inv);
            for (int l = P.n - 2; l >= lw; --l) small_up<T, NR, true>(P, l, M);
        }
        __syncthreads();
    } else {
        small_coarsest<T, NR, false>(P, M, inv);
    }
    for (int l = lb - 1; l >= 0; --l) small_up<T, NR, false>(P, l, M);
    for (int c = threadIdx.x; c < n0 * NR; c += blockDim.x) x_out[c] = M.x[c];
    if (DOT) {
        // the cycle started at the finest level: r.z -> beta (one block, fixed order)
        __shared__ double sh[32];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double a = 0.0;
            for (int c = threadIdx.x; c < n0; c += blockDim.x) a += (double)M.x[c * NR + k] * (double)M.b[c * NR + k];
            a = bsum(a, sh);
            if (threadIdx.x == 0) {
                double old = st->rz[k];
                st->beta[k] = old != 0.0 ? a / old : 0.0;
                st->rz[k] = a;
            }
        }
    }
}

template <typename T, int NR, bool DOT>
__global__ void __launch_bounds__(SMALL_THREADS) k_small(SmallPlan P, const T* __restrict__ diag,
                                                         const T* __restrict__ wl, const T* __restrict__ wb,
                                                         const T* __restrict__ inv, const T* __restrict__ b_in,
                                                         T* __restrict__ x_out, SolveState* st) {
    const long long zo = zoff(P.zs);
    diag = zsh(diag, zo);
    wl = zsh(wl, zo);
    wb = zsh(wb, zo);
    inv = zsh(inv, zo);
    b_in = zsh(b_in, zo);
    x_out = zsh(x_out, zo);
    st = zsh(st, zo);
    if (skip(st)) return;
    extern __shared__ __align__(128) unsigned char smem[];
    small_cycle<T, NR, DOT>(P, diag, wl, wb, inv, b_in, x_out, st, smem);
}


// ---- the coarse part of the V-cycle in one cooperative launch -----------------------------
// Tiled levels with few tiles are latency-bound: each launch costs more than its work.  The
// tiled levels [l0, nb) and the single-block levels run in one cooperative launch whose blocks
// take the tiles of a level in turn and meet at a grid barrier between the phases:
// pre-smoothing down the levels, the single-block cycle (block 0), post-smoothing up.
template <typename T>
struct CoarsePlan {
    int l0, nb;                      // levels handled: tiled [l0, nb), then the single-block ones
    int spin;                        // polls of a grid barrier before it gives up (fault bit 1)
    Lev<T> L[Solver::MAXLEV];
    const T* b[Solver::MAXLEV];      // rhs of level l
    T* x2[Solver::MAXLEV];           // pre-smoothed x of level l
    T* bc[Solver::MAXLEV];           // rhs of level l + 1 (written by the pre phase of level l)
    T* xo[Solver::MAXLEV];           // final x of level l
    const T* xc[Solver::MAXLEV];     // x of level l + 1 (read by the post phase of level l)
};
constexpr int CC_THREADS = 512;

// grid-wide barrier of a cooperative launch (all blocks resident).  bar[0] counts arrivals and
// only grows during a launch (the level-0 pre-smoothing kernel, which precedes every launch,
// zeroes it): barrier k of the launch is passed once it reaches k x (number of blocks).  One
// release reduction per block (it publishes the writes the block's threads made before the
// block barrier) and acquire loads while waiting (the writes of the other blocks are visible to
// this block's threads after the closing block barrier); the wait is bounded and a timeout is
// recorded in st->fault.
__device__ inline unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void red_release_gpu_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline void grid_sync(unsigned* bar, unsigned& target, SolveState* st, int spin) {
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_gpu_add(&bar[0], 1u);
        for (int it = 0; (int)(ld_acquire_gpu(&bar[0]) - target) < 0; ++it)
            if (it > spin) {
                atomicOr(&st->fault, 2);
                break;
            }
    }
    __syncthreads();
}

template <typename T, int NR>
__global__ void __launch_bounds__(CC_THREADS) k_coarse_cycle(CoarsePlan<T> C, SmallPlan P, const T* __restrict__ diag,
                                                             const T* __restrict__ wl, const T* __restrict__ wb,
                                                             const T* __restrict__ inv, SolveState* st,
                                                             unsigned* bar) {
    if (skip(st)) return;   // written by an earlier launch: the same for every block
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned gen = 0;   // arrivals that pass the next barrier (bar[0] starts the launch at 0)
    const TileThread tpre = tile_thread<HPRE>(), tpost = tile_thread<HPOST>();
    for (int l = C.l0; l < C.nb; ++l) {
        const Lev<T>& L = C.L[l];
        int tx = (L.nx + TX - 1) / TX, nt = tx * ((L.ny + TY - 1) / TY);
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            pre_tile<T, NR>(L, C.b[l], C.x2[l], C.bc[l], t % tx, t / tx, smem, nullptr, tpre);
            __syncthreads();
        }
        grid_sync(bar, gen, st, C.spin);
    }
    if (blockIdx.x == 0) small_cycle<T, NR, false>(P, diag, wl, wb, inv, C.bc[C.nb - 1], C.xo[C.nb], st, smem);
    grid_sync(bar, gen, st, C.spin);
    for (int l = C.nb - 1; l >= C.l0; --l) {
        const Lev<T>& L = C.L[l];
        int tx = (L.nx + TX - 1) / TX, nt = tx * ((L.ny + TY - 1) / TY);
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            post_tile<T, NR, false>(L, C.b[l], C.x2[l], C.xo[l], C.xc[l], t % tx, t / tx, smem, nullptr, tpost);
            __syncthreads();
        }
        if (l > C.l0) grid_sync(bar, gen, st, C.spin);
    }
}

// dense inverse of the coarsest operator (at most 32 cells), Gauss-Jordan in one warp in
// precision T: lane l owns columns l and l + 32 of [A | I]; one reciprocal per pivot.
// inv[n * n] = 1 marks a usable inverse; a non-positive or non-finite pivot (a singular
// coarsest operator, e.g. a pure-Neumann pressure problem) leaves 0 there and the cycle
// falls back to sweeps.
template <typename T>
__device__ inline void coarse_inverse_warp(int nx, int ny, const T* __restrict__ diag, const T* __restrict__ wl,
                                           const T* __restrict__ wb, T* __restrict__ inv) {
    __shared__ T A[32][65];
    __shared__ T col[32];
    int n = nx * ny;
    int lane = threadIdx.x & 31;
    for (int r = 0; r < n; ++r) {
        A[r][lane] = T(0);
        A[r][lane + 32] = T(0);
    }
    __syncwarp();
    if (lane < n) {
        int r = lane, i = r % nx, j = r / nx;
        T w0 = wl[r], w1 = i < nx - 1 ? wl[r + 1] : T(0), w2 = wb[r], w3 = j < ny - 1 ? wb[r + nx] : T(0);
        A[r][r] = diag[r] + w0 + w1 + w2 + w3;
        if (i > 0) A[r][r - 1] = -w0;
        if (i < nx - 1) A[r][r + 1] = -w1;
        if (j > 0) A[r][r - nx] = -w2;
        if (j < ny - 1) A[r][r + nx] = -w3;
        A[r][n + r] = T(1);
    }
    __syncwarp();
    bool ok = true;
    for (int p = 0; p < n; ++p) {
        T piv = A[p][p];
        ok = ok && piv > T(0) && piv < T(INFINITY);
        T rp = T(1) / piv;
        if (lane < n) col[lane] = A[lane][p];
        __syncwarp();
        T a0 = A[p][lane] * rp, a1 = A[p][lane + 32] * rp;
        for (int r = 0; r < n; ++r) {
            if (r == p) continue;
            T f = col[r];
            A[r][lane] -= f * a0;
            A[r][lane + 32] -= f * a1;
        }
        A[p][lane] = a0;
        A[p][lane + 32] = a1;
        __syncwarp();
    }
    for (int r = 0; r < n; ++r)
        for (int c = lane; c < n; c += 32) inv[r * n + c] = A[r][n + c];
    if (lane == 0) inv[n * n] = ok ? T(1) : T(0);
}


// an FP64 operator value in the solver precision (FP32: rounded on the integer pipes)
template <typename T>
__device__ __forceinline__ T to_prec(double v);
template <>
__device__ __forceinline__ double to_prec<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_prec<float>(double v) { return d2f_rn(v); }

// Levels of the hierarchy as the setup kernel sees them.
struct SetupPlan {
    int nlev, nx[Solver::MAXLEV], ny[Solver::MAXLEV];
    size_t off[Solver::MAXLEV];
    long long zs;      // byte stride between the instances of a batched launch
};

// The whole multigrid hierarchy in precision T in one launch.  Block (bx, by) converts its
// SB x SB cells of level 0 (D = cd + dd, face weights, cd, dd; with d64 != null also D in FP64
// for the refinement residual) and coarsens its own footprint level by level while a level-l
// cell still lies inside it (2^l <= SB); the last block to finish builds the remaining levels
// from the others' results and, when the coarsest level has at most 32 cells, its dense inverse.
// Footprints are SB x SB: 64 x 64 on large grids leave the last block a quarter of the work of
// 32 x 32 ones (its levels run serially after every other block has finished: 140 against
// 155 us on a 2048 x 4096 grid), 32 x 32 on small grids keep more blocks busy.
template <typename T, int SB>
__global__ void __launch_bounds__(256) k_setup_tree(SetupPlan P, const double* __restrict__ cd,
                                                    const double* __restrict__ dd, const double* __restrict__ wl,
                                                    const double* __restrict__ wb, T* diag, T* owl, T* owb, T* ocd,
                                                    T* odd, double* __restrict__ d64, T* inv, unsigned* ticket) {
    const long long zo = zoff(P.zs);
    cd = zsh(cd, zo);
    dd = zsh(dd, zo);
    wl = zsh(wl, zo);
    wb = zsh(wb, zo);
    diag = zsh(diag, zo);
    owl = zsh(owl, zo);
    owb = zsh(owb, zo);
    ocd = zsh(ocd, zo);
    odd = zsh(odd, zo);
    d64 = zsh(d64, zo);
    inv = zsh(inv, zo);
    ticket = zsh(ticket, zo);
    int nx = P.nx[0], ny = P.ny[0];
    for (int k = threadIdx.x; k < SB * SB; k += blockDim.x) {
        int i = blockIdx.x * SB + k % SB, j = blockIdx.y * SB + k / SB;
        if (i >= nx || j >= ny) continue;
        int c = j * nx + i;
        double ddv = dd ? dd[c] : 0.0;
        double dg = cd[c] + ddv;
        diag[c] = to_prec<T>(dg);
        owl[c] = to_prec<T>(wl[c]);
        owb[c] = to_prec<T>(wb[c]);
        ocd[c] = to_prec<T>(cd[c]);
        odd[c] = to_prec<T>(ddv);
        if (d64) d64[c] = dg;
    }
    __syncthreads();   // this block's level-l cells are read back by its own threads below
    int l = 1;
    for (; l < P.nlev && (1 << l) <= SB; ++l) {
        int w = SB >> l;
        int i0 = blockIdx.x * w, j0 = blockIdx.y * w;
        size_t fo = P.off[l - 1], co = P.off[l];
        for (int k = threadIdx.x; k < w * w; k += blockDim.x) {
            int I = i0 + k % w, J = j0 + k / w;
            if (I >= P.nx[l] || J >= P.ny[l]) continue;
            coarsen_cell(P.nx[l - 1], ocd + fo, odd + fo, owl + fo, owb + fo, P.nx[l], P.ny[l], I, J, ocd + co,
                         odd + co, owl + co, owb + co, diag + co);
        }
        __syncthreads();
    }
    // the last block: the levels above every block's footprint, then the coarsest inverse
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (; l < P.nlev; ++l) {
        size_t fo = P.off[l - 1], co = P.off[l];
        int n = P.nx[l] * P.ny[l];
        for (int k = threadIdx.x; k < n; k += blockDim.x)
            coarsen_cell(P.nx[l - 1], ocd + fo, odd + fo, owl + fo, owb + fo, P.nx[l], P.ny[l], k % P.nx[l],
                         k / P.nx[l], ocd + co, odd + co, owl + co, owb + co, diag + co);
        __syncthreads();
    }
    int lc = P.nlev - 1;
    if (P.nx[lc] * P.ny[lc] <= 32 && threadIdx.x < 32)
        coarse_inverse_warp(P.nx[lc], P.ny[lc], diag + P.off[lc], owl + P.off[lc], owb + P.off[lc], inv);
    if (threadIdx.x == 0) *ticket = 0u;
}


// ---- CG kernels ---------------------------------------------------------------------------
// p_new = z + beta p_old; q = A p_new; p.q -> alpha = r.z / p.q
// Dot-product accumulation of a thread: FP64 for FP64 data; for FP32 data an FP32-pair running
// sum (48-bit, FP32 instructions only), written to the FP64 total by flush().  An earlier form
// summed FP32 chunks of eight cells into FP64 with a counter tested in the per-cell body, which
// the compiler issued as a predicated FP64 add for every cell (the FP64 pipe 40-60 % busy in
// these memory-bound kernels).  The loops of k_update and k_ir_residual walk their cells in
// chunks of DOT_CHUNK (more loads in flight per thread).  The inner FP32 solves of the
// refinement work on a residual scaled to values of order one (k_ir_residual), so FP32 products
// neither underflow nor overflow there.
constexpr int DOT_CHUNK = 8;
template <typename T, int NR>
struct DotAcc {
    double tot[NR];
    __device__ DotAcc() {
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = 0.0;
    }
    __device__ void add(int k, T a, T b) { tot[k] += (double)a * (double)b; }
    __device__ void flush() {}
};
// FP32 data: each product added to an FP32-pair running sum (TwoSum, FP32 instructions only);
// flush() writes the sum so far to tot in FP64 (one FP64 add), so it may be called once at the
// end or after every chunk
template <int NR>
struct DotAcc<float, NR> {
    double tot[NR];
    f32x2 sum[NR];
    __device__ DotAcc() {
#pragma unroll
        for (int k = 0; k < NR; ++k) { tot[k] = 0.0; sum[k] = {0.0f, 0.0f}; }
    }
    __device__ void add(int k, float a, float b) {
        f32x2 t = two_sum(sum[k].hi, a * b);
        sum[k] = quick_two_sum(t.hi, t.lo + sum[k].lo);
    }
    __device__ void flush() {
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = x2_to(sum[k]);
    }
};

template <typename T, int NR>
__global__ void __launch_bounds__(256) k_apply(Lev<T> L, const T* __restrict__ z, T* __restrict__ p0,
                                                T* __restrict__ p1, T* __restrict__ q, SolveState* st,
                                                double* partial, unsigned* ticket, int vb) {
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    z = zsh(z, zo);
    p0 = zsh(p0, zo);
    p1 = zsh(p1, zo);
    q = zsh(q, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    if (skip(st)) return;
    const Vec<T, NR>* __restrict__ Z = reinterpret_cast<const Vec<T, NR>*>(z);
    const Vec<T, NR>* __restrict__ Po = reinterpret_cast<const Vec<T, NR>*>((st->iters & 1) ? p1 : p0);
    Vec<T, NR>* __restrict__ Pn = reinterpret_cast<Vec<T, NR>*>((st->iters & 1) ? p0 : p1);
    Vec<T, NR>* __restrict__ Q = reinterpret_cast<Vec<T, NR>*>(q);
    T beta[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) beta[k] = (T)st->beta[k];
    int N = L.nx * L.ny;
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        DotAcc<T, NR> acc;
#pragma unroll 2
        for (CellWalk cw(L.nx, v, vb); cw.c < N; cw.next()) {
            int c = cw.c, i = cw.i, j = cw.j;
            auto pn = [&](int cc) {
                Vec<T, NR> a = Z[cc], b = Po[cc];
#pragma unroll
                for (int k = 0; k < NR; ++k)
                    if (beta[k] != T(0)) a.v[k] += beta[k] * b.v[k];   // beta = 0: p = z (old p unused)
                return a;
            };
            Vec<T, NR> pc = pn(c), qv;
            T d = L.diag[c];
#pragma unroll
            for (int k = 0; k < NR; ++k) qv.v[k] = d * pc.v[k];
            if (i > 0) {
                T w = L.wl[c];
                Vec<T, NR> a = pn(c - 1);
                for (int k = 0; k < NR; ++k)
                    qv.v[k] += w * (pc.v[k] - a.v[k]);
            }
            if (i < L.nx - 1) {
                T w = L.wl[c + 1];
                Vec<T, NR> a = pn(c + 1);
                for (int k = 0; k < NR; ++k)
                    qv.v[k] += w * (pc.v[k] - a.v[k]);
            }
            if (j > 0) {
                T w = L.wb[c];
                Vec<T, NR> a = pn(c - L.nx);
                for (int k = 0; k < NR; ++k)
                    qv.v[k] += w * (pc.v[k] - a.v[k]);
            }
            if (j < L.ny - 1) {
                T w = L.wb[c + L.nx];
                Vec<T, NR> a = pn(c + L.nx);
                for (int k = 0; k < NR; ++k)
                    qv.v[k] += w * (pc.v[k] - a.v[k]);
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) acc.add(k, pc.v[k], qv.v[k]);
            Pn[c] = pc;
            Q[c] = qv;
        }
        acc.flush();
        block_partial<NR>(acc.tot, partial, vb, v);
    }
    double tot[NR];
    if (last_block_total<NR>(partial, vb, ticket, tot)) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            st->pq[k] = tot[k];
            st->alpha[k] = tot[k] != 0.0 ? st->rz[k] / tot[k] : 0.0;
        }
    }
}

// x += alpha p_new; r -= alpha q; r.r; convergence test; loop condition
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_update(int N, long long zs, T* __restrict__ x, T* __restrict__ r,
                                                 const T* __restrict__ p0,
                                                 const T* __restrict__ p1, const T* __restrict__ q, SolveState* st,
                                                 double* partial, unsigned* ticket, cudaGraphConditionalHandle h,
                                                 int use_h, int vb) {
    const long long zo = zoff(zs);
    x = zsh(x, zo);
    r = zsh(r, zo);
    p0 = zsh(p0, zo);
    p1 = zsh(p1, zo);
    q = zsh(q, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    if (skip(st)) return;
    const Vec<T, NR>* __restrict__ Pn = reinterpret_cast<const Vec<T, NR>*>((st->iters & 1) ? p0 : p1);
    const Vec<T, NR>* __restrict__ Q = reinterpret_cast<const Vec<T, NR>*>(q);
    Vec<T, NR>* __restrict__ X = reinterpret_cast<Vec<T, NR>*>(x);
    Vec<T, NR>* __restrict__ Rr = reinterpret_cast<Vec<T, NR>*>(r);
    T alpha[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) alpha[k] = (T)st->alpha[k];
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        DotAcc<T, NR> acc;
        const int stride = vb * blockDim.x;
        for (int c0 = v * blockDim.x + threadIdx.x; c0 < N; c0 += DOT_CHUNK * stride) {
#pragma unroll
            for (int u = 0; u < DOT_CHUNK; ++u) {
                int c = c0 + u * stride;
                if (c < N) {   // a guard, not an exit: the chunk's loads can all be in flight at once
                    Vec<T, NR> xv = X[c], rv = Rr[c], pv = Pn[c], qv = Q[c];
#pragma unroll
                    for (int k = 0; k < NR; ++k) {
                        xv.v[k] += alpha[k] * pv.v[k];
                        rv.v[k] -= alpha[k] * qv.v[k];
                        acc.add(k, rv.v[k], rv.v[k]);
                    }
                    X[c] = xv;
                    Rr[c] = rv;
                }
            }
            acc.flush();
        }
        block_partial<NR>(acc.tot, partial, vb, v);
    }
    double tot[NR];
    if (last_block_total<NR>(partial, vb, ticket, tot)) {
        bool done = true, bad = false;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            st->rr[k] = tot[k];
            if (!(tot[k] <= st->tol2[k])) done = false;
            bad = bad || !isfinite(tot[k]);
        }
        st->iters += 1;
        if (bad) {   // a NaN or infinity: no further iteration can recover
            st->nonfinite = 1;
            done = true;
        }
        if (done) st->done = 1;
        set_cond(h, use_h, (!done && st->iters < st->max_iters) ? 1u : 0u);
    }
}

// ---- the same two kernels for FP32 and one right-hand side, four cells per thread ---------------
// On rows whose length is a multiple of four (and 16-byte aligned arrays) a thread takes four
// consecutive cells of a row: 16-byte loads and stores, a quarter of the index work and four
// times the bytes in flight per load.  Each cell's arithmetic is k_apply's / k_update's (the
// same flux form, terms in the same order); the dot products add a thread's four cells in order
// to its FP32-pair sum.  Virtual blocks over the quads as in the per-cell kernels, so a batched
// instance still sums exactly as the instance launched alone.

// walk over the groups of a thread (row j, group m of the row: cells G m .. G m + G - 1, G = 4
// or 2) of virtual block v of vb, without a division per step
struct QuadWalk {
    int t, m, j, stride, dm, dj, nq;
    __device__ QuadWalk(int nq_, int v, int nv) : nq(nq_) {
        t = v * blockDim.x + threadIdx.x;
        stride = nv * blockDim.x;
        m = t % nq;
        j = t / nq;
        dm = stride % nq;
        dj = stride / nq;
    }
    __device__ void next() {
        t += stride;
        m += dm;
        j += dj;
        if (m >= nq) { m -= nq; ++j; }
    }
};

__device__ __forceinline__ float f4(const float4& a, int k) { return k == 0 ? a.x : k == 1 ? a.y : k == 2 ? a.z : a.w; }

__global__ void __launch_bounds__(256) k_apply4(Lev<float> L, const float* __restrict__ z, float* __restrict__ p0,
                                                float* __restrict__ p1, float* __restrict__ q, SolveState* st,
                                                double* partial, unsigned* ticket, int vb) {
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    z = zsh(z, zo);
    p0 = zsh(p0, zo);
    p1 = zsh(p1, zo);
    q = zsh(q, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    if (skip(st)) return;
    const float* __restrict__ Po = (st->iters & 1) ? p1 : p0;
    float* __restrict__ Pn = (st->iters & 1) ? p0 : p1;
    const float beta = (float)st->beta[0];
    const int nx = L.nx, ny = L.ny, nq = nx / 4, NQ = nq * ny;
    // p = z + beta p_old of one cell / of four (beta = 0: p = z, the old p unused)
    auto pn1 = [&](int cc) { return beta != 0.0f ? z[cc] + beta * Po[cc] : z[cc]; };
    auto pn4 = [&](int cc) {
        float4 a = *reinterpret_cast<const float4*>(z + cc);
        if (beta != 0.0f) {
            float4 o = *reinterpret_cast<const float4*>(Po + cc);
            a.x += beta * o.x;
            a.y += beta * o.y;
            a.z += beta * o.z;
            a.w += beta * o.w;
        }
        return a;
    };
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        DotAcc<float, 1> acc;
#pragma unroll 2
        for (QuadWalk w(nq, v, vb); w.t < NQ; w.next()) {
            const int i0 = 4 * w.m, j = w.j, c = j * nx + i0;
            float4 pc = pn4(c);
            float4 dg = *reinterpret_cast<const float4*>(L.diag + c);
            float4 wl = *reinterpret_cast<const float4*>(L.wl + c);
            float4 wb = *reinterpret_cast<const float4*>(L.wb + c);
            float pl = i0 > 0 ? pn1(c - 1) : 0.0f;
            float pr = i0 + 4 < nx ? pn1(c + 4) : 0.0f;
            float wr3 = i0 + 4 < nx ? L.wl[c + 4] : 0.0f;
            float4 pd = j > 0 ? pn4(c - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 pu = j < ny - 1 ? pn4(c + nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 wt = j < ny - 1 ? *reinterpret_cast<const float4*>(L.wb + c + nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float qv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float p = f4(pc, a);
                float s = f4(dg, a) * p;
                const int i = i0 + a;
                if (i > 0) s += f4(wl, a) * (p - (a == 0 ? pl : f4(pc, a - 1)));
                if (i < nx - 1) s += (a == 3 ? wr3 : f4(wl, a + 1)) * (p - (a == 3 ? pr : f4(pc, a + 1)));
                if (j > 0) s += f4(wb, a) * (p - f4(pd, a));
                if (j < ny - 1) s += f4(wt, a) * (p - f4(pu, a));
                qv[a] = s;
                acc.add(0, p, s);
            }
            *reinterpret_cast<float4*>(Pn + c) = pc;
            *reinterpret_cast<float4*>(q + c) = make_float4(qv[0], qv[1], qv[2], qv[3]);
        }
        acc.flush();
        block_partial<1>(acc.tot, partial, vb, v);
    }
    double tot[1];
    if (last_block_total<1>(partial, vb, ticket, tot)) {
        st->pq[0] = tot[0];
        st->alpha[0] = tot[0] != 0.0 ? st->rz[0] / tot[0] : 0.0;
    }
}

// two right-hand sides (liquid and vapour values of a cell interleaved): a thread takes two
// consecutive cells of a row, one float4 of each vector, a float2 of each coefficient array
__global__ void __launch_bounds__(256) k_apply2(Lev<float> L, const float* __restrict__ z, float* __restrict__ p0,
                                                float* __restrict__ p1, float* __restrict__ q, SolveState* st,
                                                double* partial, unsigned* ticket, int vb) {
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    z = zsh(z, zo);
    p0 = zsh(p0, zo);
    p1 = zsh(p1, zo);
    q = zsh(q, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    if (skip(st)) return;
    const float* __restrict__ Po = (st->iters & 1) ? p1 : p0;
    float* __restrict__ Pn = (st->iters & 1) ? p0 : p1;
    const float b0 = (float)st->beta[0], b1 = (float)st->beta[1];
    const int nx = L.nx, ny = L.ny, np = nx / 2, NP = np * ny;
    // p = z + beta p_old of one cell (float2) / of two (float4), per right-hand side
    auto pn2 = [&](int cc) {
        float2 a = *reinterpret_cast<const float2*>(z + 2 * cc);
        float2 o = *reinterpret_cast<const float2*>(Po + 2 * cc);
        if (b0 != 0.0f) a.x += b0 * o.x;
        if (b1 != 0.0f) a.y += b1 * o.y;
        return a;
    };
    auto pn4 = [&](int cc) {
        float4 a = *reinterpret_cast<const float4*>(z + 2 * cc);
        float4 o = *reinterpret_cast<const float4*>(Po + 2 * cc);
        if (b0 != 0.0f) { a.x += b0 * o.x; a.z += b0 * o.z; }
        if (b1 != 0.0f) { a.y += b1 * o.y; a.w += b1 * o.w; }
        return a;
    };
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        DotAcc<float, 2> acc;
#pragma unroll 2
        for (QuadWalk w(np, v, vb); w.t < NP; w.next()) {
            const int i0 = 2 * w.m, j = w.j, c = j * nx + i0;
            float4 pc = pn4(c);
            float2 dg = *reinterpret_cast<const float2*>(L.diag + c);
            float2 wl = *reinterpret_cast<const float2*>(L.wl + c);
            float2 wb = *reinterpret_cast<const float2*>(L.wb + c);
            float2 pl = i0 > 0 ? pn2(c - 1) : make_float2(0.f, 0.f);
            float2 pr = i0 + 2 < nx ? pn2(c + 2) : make_float2(0.f, 0.f);
            float wr1 = i0 + 2 < nx ? L.wl[c + 2] : 0.0f;
            float4 pd = j > 0 ? pn4(c - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 pu = j < ny - 1 ? pn4(c + nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            float2 wt = j < ny - 1 ? *reinterpret_cast<const float2*>(L.wb + c + nx) : make_float2(0.f, 0.f);
            float qv[4];
#pragma unroll
            for (int a = 0; a < 2; ++a) {          // cell i0 + a
                const int i = i0 + a;
                const float d = a == 0 ? dg.x : dg.y, wlf = a == 0 ? wl.x : wl.y, wbf = a == 0 ? wb.x : wb.y;
                const float wrf = a == 0 ? wl.y : wr1, wtf = a == 0 ? wt.x : wt.y;
#pragma unroll
                for (int k = 0; k < 2; ++k) {      // right-hand side k
                    const float p = f4(pc, 2 * a + k);
                    float s = d * p;
                    const float left = a == 0 ? (k == 0 ? pl.x : pl.y) : f4(pc, k);
                    const float right = a == 1 ? (k == 0 ? pr.x : pr.y) : f4(pc, 2 + k);
                    if (i > 0) s += wlf * (p - left);
                    if (i < nx - 1) s += wrf * (p - right);
                    if (j > 0) s += wbf * (p - f4(pd, 2 * a + k));
                    if (j < ny - 1) s += wtf * (p - f4(pu, 2 * a + k));
                    qv[2 * a + k] = s;
                    acc.add(k, p, s);
                }
            }
            *reinterpret_cast<float4*>(Pn + 2 * c) = pc;
            *reinterpret_cast<float4*>(q + 2 * c) = make_float4(qv[0], qv[1], qv[2], qv[3]);
        }
        acc.flush();
        block_partial<2>(acc.tot, partial, vb, v);
    }
    double tot[2];
    if (last_block_total<2>(partial, vb, ticket, tot)) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            st->pq[k] = tot[k];
            st->alpha[k] = tot[k] != 0.0 ? st->rz[k] / tot[k] : 0.0;
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(256) k_update4(int N, long long zs, float* __restrict__ x, float* __restrict__ r,
                                                 const float* __restrict__ p0, const float* __restrict__ p1,
                                                 const float* __restrict__ q, SolveState* st, double* partial,
                                                 unsigned* ticket, cudaGraphConditionalHandle h, int use_h, int vb) {
    const long long zo = zoff(zs);
    x = zsh(x, zo);
    r = zsh(r, zo);
    p0 = zsh(p0, zo);
    p1 = zsh(p1, zo);
    q = zsh(q, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    if (skip(st)) return;
    const float4* __restrict__ Pn = reinterpret_cast<const float4*>((st->iters & 1) ? p0 : p1);
    const float4* __restrict__ Q = reinterpret_cast<const float4*>(q);
    float4* __restrict__ X = reinterpret_cast<float4*>(x);
    float4* __restrict__ R = reinterpret_cast<float4*>(r);
    // element e of a float4 belongs to right-hand side e % NR (NR = 2: liquid, vapour interleaved)
    const float a0 = (float)st->alpha[0], a1 = NR > 1 ? (float)st->alpha[1] : a0;
    const int NQ = N * NR / 4;
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        DotAcc<float, NR> acc;
#pragma unroll 2
        for (int t = v * blockDim.x + threadIdx.x; t < NQ; t += vb * blockDim.x) {
            float4 xv = X[t], rv = R[t], pv = Pn[t], qv = Q[t];
            xv.x += a0 * pv.x;
            xv.y += a1 * pv.y;
            xv.z += a0 * pv.z;
            xv.w += a1 * pv.w;
            rv.x -= a0 * qv.x;
            rv.y -= a1 * qv.y;
            rv.z -= a0 * qv.z;
            rv.w -= a1 * qv.w;
            acc.add(0, rv.x, rv.x);
            acc.add(NR - 1, rv.y, rv.y);
            acc.add(0, rv.z, rv.z);
            acc.add(NR - 1, rv.w, rv.w);
            X[t] = xv;
            R[t] = rv;
        }
        acc.flush();
        block_partial<NR>(acc.tot, partial, vb, v);
    }
    double tot[NR];
    if (last_block_total<NR>(partial, vb, ticket, tot)) {
        bool done = true, bad = false;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            st->rr[k] = tot[k];
            if (!(tot[k] <= st->tol2[k])) done = false;
            bad = bad || !isfinite(tot[k]);
        }
        st->iters += 1;
        if (bad) {   // a NaN or infinity: no further iteration can recover
            st->nonfinite = 1;
            done = true;
        }
        if (done) st->done = 1;
        set_cond(h, use_h, (!done && st->iters < st->max_iters) ? 1u : 0u);
    }
}

// ---- a whole inner solve in one cooperative launch (small grids) ---------------------------
// On small grids a CG iteration is a handful of short kernels (the V-cycle legs, p/q, x/r), each
// a graph node whose launch costs as much as its work.  k_cg_persist runs the whole inner FP32
// MG-PCG solve of one refinement pass in one cooperative launch: the V-cycle as in the
// cooperative coarse cycle but from the finest level, then p = z + beta p with q = A p, then x
// and r, with a bounded grid barrier between the phases.  The dot products of a phase are
// written as per-tile (r.z) or per-block (p.q, r.r) slots; after the barrier every block sums
// the slots in the same order with the same code, so all blocks hold the same alpha, beta and
// convergence decision without another barrier; block 0 alone writes the solve state.  The
// arithmetic of each cell is that of the separate kernels; only the grouping of the dot
// products differs (per block instead of per launch block).

// grid barrier that gives up: false if this block's wait ran out or a fault is already recorded
// (every block then leaves at its next barrier, so a fault ends the launch after a bounded time)
__device__ inline bool grid_sync_ok(unsigned* bar, unsigned& target, SolveState* st, int spin) {
    __shared__ int bad;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = *((volatile int*)&st->fault);
        if (!b) {
            red_release_gpu_add(&bar[0], 1u);
            for (int it = 0; (int)(ld_acquire_gpu(&bar[0]) - target) < 0; ++it)
                if (it > spin) {
                    atomicOr(&st->fault, 2);
                    b = 1;
                    break;
                }
        }
        bad = b;
    }
    __syncthreads();
    return bad == 0;
}

// sum of nslot slots per right-hand side (partial[k * nslot + s]) in a fixed order, in every
// block (the result is in every thread)
template <int NR>
__device__ inline void sum_slots(const double* partial, int nslot, double* tot) {
    __shared__ double sh[32];
    __shared__ double res[2];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nslot; b += blockDim.x) a += ((const volatile double*)partial)[k * nslot + b];
        a = bsum(a, sh);
        if (threadIdx.x == 0) res[k] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NR; ++k) tot[k] = res[k];
    __syncthreads();
}

template <typename T, int NR>
__global__ void __launch_bounds__(CC_THREADS)
k_cg_persist(CoarsePlan<T> C, SmallPlan P, const T* __restrict__ diag, const T* __restrict__ wl,
             const T* __restrict__ wb, const T* __restrict__ inv, T* __restrict__ x, T* __restrict__ r,
             T* __restrict__ p0, T* __restrict__ p1, T* __restrict__ q, SolveState* st, double* partial,
             unsigned* bar) {
    if (skip(st)) return;   // the refinement has converged: the same in every block
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned gen = 0;
    const TileThread tpre = tile_thread<HPRE>(), tpost = tile_thread<HPOST>();
    const int G = gridDim.x;
    const Lev<T>& L0 = C.L[0];
    const int N = L0.nx * L0.ny;
    const int tx0 = (L0.nx + TX - 1) / TX, nt0 = tx0 * ((L0.ny + TY - 1) / TY);
    double* prz = partial;                // r.z per finest tile
    double* ppq = partial + 2 * nt0;      // p.q per block
    double* prr = ppq + 2 * G;            // r.r per block
    double rz[2], tol2[2], alpha[2] = {0.0, 0.0}, beta[2] = {0.0, 0.0}, pq[2] = {0.0, 0.0}, rr[2] = {0.0, 0.0};
    int iters = st->iters;
    const int maxit = st->max_iters;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        rz[k] = st->rz[k];
        tol2[k] = st->tol2[k];
    }
    bool done = false, bad = false, ok = true;
    while (!done) {
        // ---- z = M r: the V-cycle from the finest level
        for (int l = 0; l < C.nb && ok; ++l) {
            const Lev<T>& L = C.L[l];
            int tx = (L.nx + TX - 1) / TX, nt = tx * ((L.ny + TY - 1) / TY);
            for (int t = blockIdx.x; t < nt; t += G) {
                pre_tile<T, NR>(L, C.b[l], C.x2[l], C.bc[l], t % tx, t / tx, smem, nullptr, tpre);
                __syncthreads();
            }
            ok = grid_sync_ok(bar, gen, st, C.spin);
        }
        if (!ok) break;
        if (blockIdx.x == 0) small_cycle<T, NR, false>(P, diag, wl, wb, inv, C.bc[C.nb - 1], C.xo[C.nb], st, smem);
        if (!grid_sync_ok(bar, gen, st, C.spin)) break;
        for (int l = C.nb - 1; l >= 1 && ok; --l) {
            const Lev<T>& L = C.L[l];
            int tx = (L.nx + TX - 1) / TX, nt = tx * ((L.ny + TY - 1) / TY);
            for (int t = blockIdx.x; t < nt; t += G) {
                post_tile<T, NR, false>(L, C.b[l], C.x2[l], C.xo[l], C.xc[l], t % tx, t / tx, smem, nullptr, tpost);
                __syncthreads();
            }
            ok = grid_sync_ok(bar, gen, st, C.spin);
        }
        if (!ok) break;
        for (int t = blockIdx.x; t < nt0; t += G) {
            Vec<T, 2> d =
                post_tile<T, NR, true>(L0, C.b[0], C.x2[0], C.xo[0], C.xc[0], t % tx0, t / tx0, smem, nullptr, tpost);
            block_partial_t<T, NR>(d.v, prz, nt0, t);
            __syncthreads();
        }
        if (!grid_sync_ok(bar, gen, st, C.spin)) break;
        double rzn[2] = {0.0, 0.0};
        sum_slots<NR>(prz, nt0, rzn);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            beta[k] = rz[k] != 0.0 ? rzn[k] / rz[k] : 0.0;
            rz[k] = rzn[k];
        }
        // ---- p = z + beta p; q = A p; p.q (the new p of the neighbours recomputed, as k_apply)
        const Vec<T, NR>* __restrict__ Z = reinterpret_cast<const Vec<T, NR>*>(C.xo[0]);
        const Vec<T, NR>* __restrict__ Po = reinterpret_cast<const Vec<T, NR>*>((iters & 1) ? p1 : p0);
        Vec<T, NR>* __restrict__ Pn = reinterpret_cast<Vec<T, NR>*>((iters & 1) ? p0 : p1);
        Vec<T, NR>* __restrict__ Q = reinterpret_cast<Vec<T, NR>*>(q);
        {
            T bt[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) bt[k] = (T)beta[k];
            DotAcc<T, NR> acc;
            for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += G * blockDim.x) {
                int i = c % L0.nx, j = c / L0.nx;
                auto pn = [&](int cc) {
                    Vec<T, NR> a = Z[cc], b = Po[cc];
#pragma unroll
                    for (int k = 0; k < NR; ++k)
                        if (bt[k] != T(0)) a.v[k] += bt[k] * b.v[k];
                    return a;
                };
                Vec<T, NR> pc = pn(c), qv;
                T dg = L0.diag[c];
#pragma unroll
                for (int k = 0; k < NR; ++k) qv.v[k] = dg * pc.v[k];
                if (i > 0) {
                    T w = L0.wl[c];
                    Vec<T, NR> a = pn(c - 1);
                    for (int k = 0; k < NR; ++k) qv.v[k] += w * (pc.v[k] - a.v[k]);
                }
                if (i < L0.nx - 1) {
                    T w = L0.wl[c + 1];
                    Vec<T, NR> a = pn(c + 1);
                    for (int k = 0; k < NR; ++k) qv.v[k] += w * (pc.v[k] - a.v[k]);
                }
                if (j > 0) {
                    T w = L0.wb[c];
                    Vec<T, NR> a = pn(c - L0.nx);
                    for (int k = 0; k < NR; ++k) qv.v[k] += w * (pc.v[k] - a.v[k]);
                }
                if (j < L0.ny - 1) {
                    T w = L0.wb[c + L0.nx];
                    Vec<T, NR> a = pn(c + L0.nx);
                    for (int k = 0; k < NR; ++k) qv.v[k] += w * (pc.v[k] - a.v[k]);
                }
#pragma unroll
                for (int k = 0; k < NR; ++k) acc.add(k, pc.v[k], qv.v[k]);
                Pn[c] = pc;
                Q[c] = qv;
            }
            acc.flush();
            block_partial<NR>(acc.tot, ppq, G, blockIdx.x);
        }
        if (!grid_sync_ok(bar, gen, st, C.spin)) break;
        sum_slots<NR>(ppq, G, pq);
#pragma unroll
        for (int k = 0; k < NR; ++k) alpha[k] = pq[k] != 0.0 ? rz[k] / pq[k] : 0.0;
        // ---- x += alpha p; r -= alpha q; r.r
        {
            T al[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) al[k] = (T)alpha[k];
            Vec<T, NR>* __restrict__ X = reinterpret_cast<Vec<T, NR>*>(x);
            Vec<T, NR>* __restrict__ Rr = reinterpret_cast<Vec<T, NR>*>(r);
            DotAcc<T, NR> acc;
            const int stride = G * blockDim.x;
            for (int c0 = blockIdx.x * blockDim.x + threadIdx.x; c0 < N; c0 += DOT_CHUNK * stride) {
#pragma unroll
                for (int u = 0; u < DOT_CHUNK; ++u) {
                    int c = c0 + u * stride;
                    if (c < N) {
                        Vec<T, NR> xv = X[c], rv = Rr[c], pv = Pn[c], qv = Q[c];
#pragma unroll
                        for (int k = 0; k < NR; ++k) {
                            xv.v[k] += al[k] * pv.v[k];
                            rv.v[k] -= al[k] * qv.v[k];
                            acc.add(k, rv.v[k], rv.v[k]);
                        }
                        X[c] = xv;
                        Rr[c] = rv;
                    }
                }
                acc.flush();
            }
            block_partial<NR>(acc.tot, prr, G, blockIdx.x);
        }
        if (!grid_sync_ok(bar, gen, st, C.spin)) break;
        sum_slots<NR>(prr, G, rr);
        iters += 1;
        done = true;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            if (!(rr[k] <= tol2[k])) done = false;
            bad = bad || !isfinite(rr[k]);
        }
        if (bad || iters >= maxit) done = true;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            st->rz[k] = rz[k];
            st->beta[k] = beta[k];
            st->pq[k] = pq[k];
            st->alpha[k] = alpha[k];
            st->rr[k] = rr[k];
        }
        st->iters = iters;
        if (bad) st->nonfinite = 1;
        st->done = 1;
    }
}

// FP64 CG start: r = b - A x, r.r, b.b, tolerance, state reset
template <int NR>
__global__ void __launch_bounds__(256)
k_init64(Lev<double> L, const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
         SolveState* st, double* partial, unsigned* ticket, double rtol2, int max_iters,
         cudaGraphConditionalHandle h, int use_h, int vb) {
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    b = zsh(b, zo);
    x = zsh(x, zo);
    r = zsh(r, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    int N = L.nx * L.ny;
    const Vec<double, NR>* X = reinterpret_cast<const Vec<double, NR>*>(x);
    const Vec<double, NR>* B = reinterpret_cast<const Vec<double, NR>*>(b);
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        double acc[2 * NR];
#pragma unroll
        for (int k = 0; k < 2 * NR; ++k) acc[k] = 0.0;
        for (CellWalk cw(L.nx, v, vb); cw.c < N; cw.next()) {
            int c = cw.c, i = cw.i, j = cw.j;
            Vec<double, NR> xv = X[c], bv = B[c], s;   // s = (A x)_i in flux form
            double dg = L.diag[c];
#pragma unroll
            for (int k = 0; k < NR; ++k) s.v[k] = dg * xv.v[k];
            if (i > 0) { double w = L.wl[c]; for (int k = 0; k < NR; ++k) s.v[k] += w * (xv.v[k] - X[c - 1].v[k]); }
            if (i < L.nx - 1) {
                double w = L.wl[c + 1];
                for (int k = 0; k < NR; ++k)
                    s.v[k] += w * (xv.v[k] - X[c + 1].v[k]);
            }
            if (j > 0) { double w = L.wb[c]; for (int k = 0; k < NR; ++k) s.v[k] += w * (xv.v[k] - X[c - L.nx].v[k]); }
            if (j < L.ny - 1) {
                double w = L.wb[c + L.nx];
                for (int k = 0; k < NR; ++k)
                    s.v[k] += w * (xv.v[k] - X[c + L.nx].v[k]);
            }
            Vec<double, NR> rv;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                rv.v[k] = bv.v[k] - s.v[k];
                acc[k] += rv.v[k] * rv.v[k];
                acc[NR + k] += bv.v[k] * bv.v[k];
            }
            reinterpret_cast<Vec<double, NR>*>(r)[c] = rv;
        }
        block_partial<2 * NR>(acc, partial, vb, v);
    }
    double tot[2 * NR];
    if (last_block_total<2 * NR>(partial, vb, ticket, tot)) {
        bool done = true, bad = false;
        for (int k = 0; k < 2; ++k) {
            double rr = k < NR ? tot[k] : 0.0, bb = k < NR ? tot[NR + k] : 0.0;
            st->rr[k] = rr;
            st->bb[k] = bb;
            st->tol2[k] = rtol2 * (bb > 1e-300 ? bb : 1e-300);
            st->rz[k] = 0.0;
            st->beta[k] = 0.0;
            if (!(rr <= st->tol2[k])) done = false;
            if (!isfinite(rr) || !isfinite(bb)) bad = true;
        }
        st->nonfinite = bad ? 1 : 0;
        if (bad) done = true;   // no iteration: the system holds a NaN or an infinity
        st->iters = 0;
        st->itot = 0;
        st->max_iters = max_iters;
        st->done = done ? 1 : 0;
        st->odone = 0;
        st->oiters = 0;
        st->nr = NR;
        set_cond(h, use_h, done ? 0u : 1u);
    }
}

// power of two s that brings cell values whose sum of squares over n cells is rr to order one
__device__ inline double unit_scale(double rr, int n) {
    double m = sqrt(rr / (double)n);
    int e = (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
    e = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
    return ldexp(1.0, -e);
}

// refinement start: b.b and the outer tolerance
template <int NR>
__global__ void __launch_bounds__(256) k_ir_init(int N, long long zs, const double* __restrict__ b, SolveState* st,
                                                  double* partial,
                                                  unsigned* ticket, double rtol2, double inner_rtol, int max_iters,
                                                  int max_outer, int vb) {
    const long long zo = zoff(zs);
    b = zsh(b, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        double acc[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = 0.0;
        for (int c = v * blockDim.x + threadIdx.x; c < N; c += vb * blockDim.x) {
            Vec<double, NR> bv = reinterpret_cast<const Vec<double, NR>*>(b)[c];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] += bv.v[k] * bv.v[k];
        }
        block_partial<NR>(acc, partial, vb, v);
    }
    double tot[NR];
    if (last_block_total<NR>(partial, vb, ticket, tot)) {
        for (int k = 0; k < 2; ++k) {
            double bb = k < NR ? tot[k] : 0.0;
            st->obb[k] = bb;
            st->otol2[k] = rtol2 * (bb > 1e-300 ? bb : 1e-300);
            st->scale_next[k] = unit_scale(bb, N);
        }
        st->odone = 0;
        st->oiters = 0;
        st->done = 0;
        st->iters = 0;
        st->itot = 0;
        st->max_iters = max_iters;
        st->max_outer = max_outer;
        st->inner_rtol = inner_rtol;
        st->nr = NR;
        st->nonfinite = 0;
    }
}

// refinement sweep: r64 = b - A64 x, outer test, r32 = r64, e = 0, inner state reset
template <int NR>
__global__ void __launch_bounds__(256) k_ir_residual(Lev<double> L, const double* __restrict__ b,
                                                      const double* __restrict__ x, float* __restrict__ r32,
                                                      float* __restrict__ e32, SolveState* st, double* partial,
                                                      unsigned* ticket, cudaGraphConditionalHandle ho,
                                                      cudaGraphConditionalHandle hi, int use_h, int set_hi,
                                                      unsigned* coop_bar, int vb) {
    // the whole-solve cooperative launch that follows counts its barrier arrivals from 0 (its
    // previous launch has completed: stream order)
    if (coop_bar && blockIdx.x == 0 && blockIdx.z == 0 && threadIdx.x == 0) *coop_bar = 0u;
    const long long zo = zoff(L.zs);
    L.diag = zsh(L.diag, zo);
    L.wl = zsh(L.wl, zo);
    L.wb = zsh(L.wb, zo);
    b = zsh(b, zo);
    x = zsh(x, zo);
    r32 = zsh(r32, zo);
    e32 = zsh(e32, zo);
    st = zsh(st, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    if (st->odone) return;
    int N = L.nx * L.ny;
    // the inner FP32 system is solved for s r, s = 2^k a power of two that brings the residual's
    // cell values to order one, set from the previous residual norm (of b on the first pass) by
    // the launch that computed it: the same in every block.  The FP32 copy is rounded from
    // r 2^k on the integer pipes and the norm is summed from that copy (FP32 chunks added in
    // FP64; relative accuracy about 1e-7, ample for the convergence test), so the FP64 pipe
    // carries the residual alone.
    double sc[NR];
    int ksc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        sc[k] = st->scale_next[k];
        ksc[k] = (int)((__double_as_longlong(sc[k]) >> 52) & 0x7ff) - 1023;
    }
    const Vec<double, NR>* X = reinterpret_cast<const Vec<double, NR>*>(x);
    const Vec<double, NR>* B = reinterpret_cast<const Vec<double, NR>*>(b);
    for (int v = blockIdx.x; v < vb; v += gridDim.x) {
        DotAcc<float, NR> acc;
        for (CellWalk cw(L.nx, v, vb); cw.c < N; acc.flush())
#pragma unroll
        for (int u = 0; u < DOT_CHUNK; ++u, cw.next()) {
            if (cw.c >= N) continue;
            int c = cw.c, i = cw.i, j = cw.j;
            Vec<double, NR> xv = X[c], bv = B[c], s;   // s = (A x)_i in flux form
            double dg = L.diag[c];
#pragma unroll
            for (int k = 0; k < NR; ++k) s.v[k] = dg * xv.v[k];
            if (i > 0) { double w = L.wl[c]; for (int k = 0; k < NR; ++k) s.v[k] += w * (xv.v[k] - X[c - 1].v[k]); }
            if (i < L.nx - 1) {
                double w = L.wl[c + 1];
                for (int k = 0; k < NR; ++k)
                    s.v[k] += w * (xv.v[k] - X[c + 1].v[k]);
            }
            if (j > 0) { double w = L.wb[c]; for (int k = 0; k < NR; ++k) s.v[k] += w * (xv.v[k] - X[c - L.nx].v[k]); }
            if (j < L.ny - 1) {
                double w = L.wb[c + L.nx];
                for (int k = 0; k < NR; ++k)
                    s.v[k] += w * (xv.v[k] - X[c + L.nx].v[k]);
            }
            Vec<float, NR> rf, ez;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float f = d2f_rn2(bv.v[k] - s.v[k], ksc[k]);
                rf.v[k] = f;
                acc.add(k, f, f);
                ez.v[k] = 0.0f;
            }
            reinterpret_cast<Vec<float, NR>*>(r32)[c] = rf;
            reinterpret_cast<Vec<float, NR>*>(e32)[c] = ez;
        }
        block_partial<NR>(acc.tot, partial, vb, v);
    }
    double tot[NR];
    if (last_block_total<NR>(partial, vb, ticket, tot)) {
        bool done = true;
        for (int k = 0; k < 2; ++k) {
            double s2 = k < NR ? sc[k] * sc[k] : 1.0;   // a power of two: the divisions are exact
            double rr = k < NR ? tot[k] / s2 : 0.0;
            st->orr[k] = rr;
            if (!(rr <= st->otol2[k])) done = false;
            if (!isfinite(rr) || !isfinite(st->obb[k])) st->nonfinite = 1;
            st->scale[k] = k < NR ? sc[k] : 1.0;
            st->scale_next[k] = unit_scale(rr, N);
            st->rr[k] = k < NR ? tot[k] : 0.0;
            // the inner solve reduces the residual by inner_rtol, but never below half the
            // outer target: no solve past what the refinement needs (in the scaled units)
            st->tol2[k] = fmax(st->inner_rtol * st->inner_rtol * rr, 0.25 * st->otol2[k]) * s2;
            st->rz[k] = 0.0;
            st->beta[k] = 0.0;
        }
        st->oiters += 1;
        st->itot += st->iters;
        if (st->oiters > st->max_outer || st->nonfinite) done = true;
        st->odone = done ? 1 : 0;
        st->iters = 0;
        st->done = done ? 1 : 0;
        set_cond(ho, use_h, done ? 0u : 1u);
        if (set_hi) set_cond(hi, use_h, done ? 0u : 1u);
    }
}

template <int NR>
__global__ void k_ir_update(int N, long long zs, double* __restrict__ x, const float* __restrict__ e,
                            const SolveState* st) {
    const long long zo = zoff(zs);
    x = zsh(x, zo);
    e = zsh(e, zo);
    st = zsh(st, zo);
    if (st->odone) return;
    // powers of two: exact; an even element belongs to the first right-hand side
    const double inv0 = 1.0 / st->scale[0], inv1 = NR > 1 ? 1.0 / st->scale[1] : inv0;
    const long long n = (long long)N * NR;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, T = gridDim.x * blockDim.x;
    // four elements per step (one 16-byte load of e, two of x) where both arrays allow it
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(e)) & 15u) == 0;
    const long long n4 = vec ? n / 4 : 0;
#pragma unroll 2
    for (long long q = t; q < n4; q += T) {
        float4 ev = reinterpret_cast<const float4*>(e)[q];
        double2* xp = reinterpret_cast<double2*>(x) + 2 * q;
        double2 a = xp[0], b = xp[1];
        a.x += f2d(ev.x) * inv0;
        a.y += f2d(ev.y) * inv1;
        b.x += f2d(ev.z) * inv0;
        b.y += f2d(ev.w) * inv1;
        xp[0] = a;
        xp[1] = b;
    }
    for (long long c = 4 * n4 + t; c < n; c += T) x[c] += f2d(e[c]) * ((c & 1) ? inv1 : inv0);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static inline int nblocks(long long n) {
    long long b = (n + RB - 1) / RB;
    return (int)(b < NRED ? (b < 1 ? 1 : b) : NRED);
}
// Blocks per instance of a launch over nz instances.  The reduction kernels are written for
// nblocks(n) blocks per instance (their virtual blocks, a function of the grid alone) and run
// them on this many real blocks, each taking the virtual blocks b, b + launch, ...: the same cells
// in the same order into the same slots, so that an instance's sums do not depend on how many
// instances share the launch.  One instance keeps one real block per virtual block; a batch
// gets about two blocks per SM slot in total (NRED = 4 per SM), instead of thousands of blocks
// that each reduce a few hundred cells.
static inline int lblocks(long long n, int nz) {
    int v = nblocks(n);
    int per = (2 * NRED) / (nz > 0 ? nz : 1);
    return nz <= 1 ? v : (v < per ? v : (per < 1 ? 1 : per));
}

void Solver::plan(int nx_, int ny_) {
    nx = nx_;
    ny = ny_;
    nlev = 0;
    int x = nx, y = ny;
    size_t off = 0;
    while (true) {
        lnx[nlev] = x;
        lny[nlev] = y;
        loff[nlev] = off;
        off += (size_t)x * y;
        ++nlev;
        if (nlev == MAXLEV) break;
        if ((x & 1) || (y & 1) || (long long)x * y <= 16 || x < 2 || y < 2) break;
        x /= 2;
        y /= 2;
    }
    ncells_all = off;
    if (small_max_f <= 0) small_max_f = SMALL_MAX_F;
    nbig_f = 0;
    while (nbig_f < nlev - 1 && (long long)lnx[nbig_f] * lny[nbig_f] > small_max_f) ++nbig_f;
    nbig_d = 0;
    while (nbig_d < nlev - 1 && (long long)lnx[nbig_d] * lny[nbig_d] > SMALL_MAX_D) ++nbig_d;
    nbig = nbig_f;
}

static size_t tiles(int nx, int ny) { return (size_t)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

size_t Solver::bytes(int nx, int ny) {
    Solver s;
    s.plan(nx, ny);
    size_t total = 0;
    auto add = [&](size_t b) { total += (b + 255) & ~size_t(255); };
    size_t A = s.ncells_all, N = (size_t)nx * ny;
    for (int k = 0; k < 5; ++k) add(A * 4);
    for (int k = 0; k < 5; ++k) add(A * 8);
    add(A * 2 * 4); add(A * 2 * 4); add(A * 2 * 4);
    add(A * 2 * 8); add(A * 2 * 8); add(A * 2 * 8);
    add(N * 2 * 4); add(N * 4 * 4); add(N * 2 * 4); add(N * 2 * 4);
    add(N * 2 * 8); add(N * 4 * 8); add(N * 2 * 8);
    add(1040 * 4); add(1040 * 8);
    size_t mb = tiles(nx, ny) > (size_t)NRED ? tiles(nx, ny) : (size_t)NRED;
    add(mb * 4 * 8);
    add(256);
    add(NSLOT * sizeof(SolveState));
    add(4 * sizeof(KTimer));
    return total;
}

template <typename K>
static void allow_smem(K kern, int bytes, cudaError_t* first) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess && *first == cudaSuccess) *first = e;
}

cudaError_t Solver::bind(void* base, int nx_, int ny_, bool make_streams, cudaStream_t init_stream) {
    plan(nx_, ny_);
    tma_ready = false;   // descriptors hold addresses: re-encode after every binding
    char* p = (char*)base;
    auto take = [&](size_t b) { void* r = p; p += (b + 255) & ~size_t(255); return r; };
    size_t A = ncells_all, N = (size_t)nx * ny;
    f_diag = (float*)take(A * 4); f_wl = (float*)take(A * 4); f_wb = (float*)take(A * 4);
    f_cd = (float*)take(A * 4); f_dd = (float*)take(A * 4);
    d_diag = (double*)take(A * 8); d_wl = (double*)take(A * 8); d_wb = (double*)take(A * 8);
    d_cd = (double*)take(A * 8); d_dd = (double*)take(A * 8);
    f_x = (float*)take(A * 2 * 4); f_b = (float*)take(A * 2 * 4); f_x2 = (float*)take(A * 2 * 4);
    d_x = (double*)take(A * 2 * 8); d_b = (double*)take(A * 2 * 8); d_x2 = (double*)take(A * 2 * 8);
    f_r = (float*)take(N * 2 * 4); f_p = (float*)take(N * 4 * 4); f_q = (float*)take(N * 2 * 4);
    f_e = (float*)take(N * 2 * 4);
    d_r = (double*)take(N * 2 * 8); d_p = (double*)take(N * 4 * 8); d_q = (double*)take(N * 2 * 8);
    f_inv = (float*)take(1040 * 4); d_inv = (double*)take(1040 * 8);
    size_t mb = tiles(nx, ny) > (size_t)NRED ? tiles(nx, ny) : (size_t)NRED;
    partial = (double*)take(mb * 4 * 8);
    tickets = (unsigned*)take(256);
    st_base = (SolveState*)take(NSLOT * sizeof(SolveState));
    st = st_base;
    timer = (KTimer*)take(4 * sizeof(KTimer));
    if (make_streams)
        for (int k = 0; k < 3; ++k) cudaStreamCreateWithFlags(&aux[k], cudaStreamNonBlocking);
    // shared-memory limits of the tile kernels
    // shared-memory opt-in of the tile and small-level kernels (dynamic + static may pass 48 KB)
    const int SM = 200 * 1024;
    cudaError_t err = cudaSuccess;
    allow_smem(k_pre<float, 1>, SM, &err);
    allow_smem(k_pre<float, 2>, SM, &err);
    allow_smem(k_pre<double, 1>, SM, &err);
    allow_smem(k_pre<double, 2>, SM, &err);
    allow_smem(k_post<float, 1, true>, SM, &err);
    allow_smem(k_post<float, 1, false>, SM, &err);
    allow_smem(k_post<float, 2, true>, SM, &err);
    allow_smem(k_post<float, 2, false>, SM, &err);
    allow_smem(k_post<double, 1, true>, SM, &err);
    allow_smem(k_post<double, 1, false>, SM, &err);
    allow_smem(k_post<double, 2, true>, SM, &err);
    allow_smem(k_post<double, 2, false>, SM, &err);
    allow_smem(k_coarse_cycle<float, 1>, SM, &err);
    allow_smem(k_coarse_cycle<float, 2>, SM, &err);
    allow_smem(k_coarse_cycle<double, 1>, SM, &err);
    allow_smem(k_coarse_cycle<double, 2>, SM, &err);
    allow_smem(k_cg_persist<float, 1>, SM, &err);
    allow_smem(k_cg_persist<float, 2>, SM, &err);
    allow_smem(k_small<float, 1, true>, SM, &err);
    allow_smem(k_small<float, 1, false>, SM, &err);
    allow_smem(k_small<float, 2, true>, SM, &err);
    allow_smem(k_small<float, 2, false>, SM, &err);
    allow_smem(k_small<double, 1, true>, SM, &err);
    allow_smem(k_small<double, 1, false>, SM, &err);
    allow_smem(k_small<double, 2, true>, SM, &err);
    allow_smem(k_small<double, 2, false>, SM, &err);
    // device state that must start at zero (tickets, solve states, timers; timer starts at ~0)
    cudaError_t e[4];
    e[0] = cudaMemsetAsync(timer, 0, 4 * sizeof(KTimer), init_stream);
    e[1] = cudaSuccess;
    for (int k = 0; k < 4; ++k) {
        cudaError_t ek = cudaMemsetAsync(&timer[k].start, 0xff, sizeof(unsigned long long), init_stream);
        if (ek != cudaSuccess) e[1] = ek;
    }
    e[2] = cudaMemsetAsync(tickets, 0, 256, init_stream);
    e[3] = cudaMemsetAsync(st_base, 0, NSLOT * sizeof(SolveState), init_stream);
    for (int k = 0; k < 4 && err == cudaSuccess; ++k) err = e[k];
    timing = 1;
    return err;
}

// accessors for precision T
template <typename T> struct PT;
template <> struct PT<float> {
    static float* diag(Solver& s) { return s.f_diag; }
    static float* wl(Solver& s) { return s.f_wl; }
    static float* wb(Solver& s) { return s.f_wb; }
    static float* cd(Solver& s) { return s.f_cd; }
    static float* dd(Solver& s) { return s.f_dd; }
    static float* x(Solver& s) { return s.f_x; }
    static float* x2(Solver& s) { return s.f_x2; }
    static float* inv(Solver& s) { return s.f_inv; }
    static float* b(Solver& s) { return s.f_b; }
    static float* r(Solver& s) { return s.f_r; }
    static constexpr int prec = 1;
};
template <> struct PT<double> {
    static double* diag(Solver& s) { return s.d_diag; }
    static double* wl(Solver& s) { return s.d_wl; }
    static double* wb(Solver& s) { return s.d_wb; }
    static double* cd(Solver& s) { return s.d_cd; }
    static double* dd(Solver& s) { return s.d_dd; }
    static double* x(Solver& s) { return s.d_x; }
    static double* x2(Solver& s) { return s.d_x2; }
    static double* inv(Solver& s) { return s.d_inv; }
    static double* b(Solver& s) { return s.d_b; }
    static double* r(Solver& s) { return s.d_r; }
    static constexpr int prec = 0;
};

// ---- TMA descriptors (host) ----------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        else
            cudaGetLastError();
    }
    return fn;
}

// a 2-D row-major array of w x h elements of T, copied in boxes of bw x bh; false when the base
// or the row pitch is not 16-byte aligned or the encoder refuses
template <typename T>
static bool encode_2d(CUtensorMap* m, const void* base, int w, int h, int bw, int bh) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn || (uintptr_t)base % 16 != 0 || ((size_t)w * sizeof(T)) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t pitch[1] = {(cuuint64_t)w * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t es[2] = {1, 1};
    CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return fn(m, dt, 2, const_cast<void*>(base), dims, pitch, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

static size_t tmap_index(int prec, int nr, int l, int post) {
    return ((size_t)(prec * 2 + (nr - 1)) * Solver::MAXLEV + l) * 2 + post;
}

template <typename T, int NR, bool POST>
static bool encode_tile_maps(Solver& s, int l, TileMaps& M) {
    constexpr int H = POST ? HPOST : HPRE;
    using Sg = Stage<T, NR, H, POST>;
    int nx = s.lnx[l], ny = s.lny[l];
    size_t o = s.loff[l];
    const T* b = l == 0 ? PT<T>::r(s) : PT<T>::b(s) + 2 * o;
    bool ok = encode_2d<T>(&M.d, PT<T>::diag(s) + o, nx, ny, Sg::BWS, Sg::BHS) &&
              encode_2d<T>(&M.wl, PT<T>::wl(s) + o, nx, ny, Sg::BWS, Sg::BHS) &&
              encode_2d<T>(&M.wb, PT<T>::wb(s) + o, nx, ny, Sg::BWS, Sg::BHS) &&
              encode_2d<T>(&M.b, b, nx * NR, ny, Sg::BWV * NR, Sg::BHV);
    if (POST)
        ok = ok && encode_2d<T>(&M.xin, PT<T>::x2(s) + 2 * o, nx * NR, ny, Sg::BWV * NR, Sg::BHV) &&
             encode_2d<T>(&M.xc, PT<T>::x(s) + 2 * s.loff[l + 1], s.lnx[l + 1] * NR, s.lny[l + 1], Sg::BWC * NR,
                          Sg::BHC);
    return ok;
}

template <typename T>
static void encode_precision(Solver& s, int nbig) {
    for (int l = 0; l < nbig; ++l) {
        int p = PT<T>::prec;
        s.tma_ok[tmap_index(p, 1, l, 0)] = encode_tile_maps<T, 1, false>(s, l, s.tmaps[tmap_index(p, 1, l, 0)]);
        s.tma_ok[tmap_index(p, 1, l, 1)] = encode_tile_maps<T, 1, true>(s, l, s.tmaps[tmap_index(p, 1, l, 1)]);
        s.tma_ok[tmap_index(p, 2, l, 0)] = encode_tile_maps<T, 2, false>(s, l, s.tmaps[tmap_index(p, 2, l, 0)]);
        s.tma_ok[tmap_index(p, 2, l, 1)] = encode_tile_maps<T, 2, true>(s, l, s.tmaps[tmap_index(p, 2, l, 1)]);
    }
}

// descriptors of every tiled level, both precisions and right-hand-side counts (host work only)
static void ensure_tile_maps(Solver& s) {
    if (s.tma_ready) return;
    size_t n = tmap_index(1, 2, Solver::MAXLEV - 1, 1) + 1;
    s.tmaps.assign(n, TileMaps{});
    s.tma_ok.assign(n, 0);
    encode_precision<float>(s, s.nbig_f);
    encode_precision<double>(s, s.nbig_d);
    s.tma_ready = true;
}

template <typename T>
static Lev<T> lev(Solver& s, int l) {
    size_t o = s.loff[l];
    return {s.lnx[l], s.lny[l], PT<T>::diag(s) + o, PT<T>::wl(s) + o, PT<T>::wb(s) + o, s.zs};
}

template <typename T>
static void setup_levels(Solver& s, const double* cd, const double* dd, const double* wl, const double* wb,
                         double* d64, cudaStream_t stm) {
    SetupPlan P;
    P.zs = s.zs;
    P.nlev = s.nlev;
    for (int l = 0; l < s.nlev; ++l) { P.nx[l] = s.lnx[l]; P.ny[l] = s.lny[l]; P.off[l] = s.loff[l]; }
    if ((long long)s.nx * s.ny > (1LL << 21)) {
        constexpr int SB = 64;
        dim3 grid((s.nx + SB - 1) / SB, (s.ny + SB - 1) / SB, s.nz);
        k_setup_tree<T, SB><<<grid, 256, 0, stm>>>(P, cd, dd, wl, wb, PT<T>::diag(s), PT<T>::wl(s), PT<T>::wb(s),
                                                   PT<T>::cd(s), PT<T>::dd(s), d64, PT<T>::inv(s), s.tickets + 6);
    } else {
        constexpr int SB = 32;
        dim3 grid((s.nx + SB - 1) / SB, (s.ny + SB - 1) / SB, s.nz);
        k_setup_tree<T, SB><<<grid, 256, 0, stm>>>(P, cd, dd, wl, wb, PT<T>::diag(s), PT<T>::wl(s), PT<T>::wb(s),
                                                   PT<T>::cd(s), PT<T>::dd(s), d64, PT<T>::inv(s), s.tickets + 6);
    }
    ++s.launches;
}

// z = M r: r is the level-0 rhs, z the level-0 output (both NR-interleaved)
template <typename T> static int nbig_of(const Solver& s);
template <> int nbig_of<float>(const Solver& s) { return s.nbig_f; }
template <> int nbig_of<double>(const Solver& s) { return s.nbig_d; }

template <typename T>
static SmallPlan small_plan(const Solver& s) {
    SmallPlan P;
    P.zs = s.zs;
    int nb = nbig_of<T>(s);
    P.n = s.nlev - nb;
    int so = 0;
    for (int k = 0; k < P.n; ++k) {
        int l = nb + k;
        P.nx[k] = s.lnx[l];
        P.ny[k] = s.lny[l];
        P.soff[k] = so;
        P.goff[k] = s.loff[l];
        so += s.lnx[l] * s.lny[l];
    }
    P.total = so;
    return P;
}

// shared memory of the cooperative coarse cycle: the larger of the tile regions and the
// single-block levels
template <typename T, int NR>
static size_t coarse_smem(const SmallPlan& P) {
    size_t a = Region<T, NR, HPRE>::bytes(), b = Region<T, NR, HPOST>::bytes();
    size_t c = SmallMem<T, NR>::bytes(P.total);
    size_t m = a > b ? a : b;
    return m > c ? m : c;
}

// first tiled level of the cooperative coarse cycle (nb: none).  A level joins when its tiles
// fit one per co-resident block; the finest level stays separate (its post-smoothing carries
// the r.z of CG).  Single instances only.
template <typename T, int NR>
static int coarse_start(Solver& s) {
    int nb = nbig_of<T>(s);
    if (!s.use_coop || s.nz != 1 || nb < 2) return nb;
    static int resident[2][2] = {{-1, -1}, {-1, -1}};
    int& res = resident[PT<T>::prec][NR - 1];
    if (res < 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        size_t smem = Region<T, NR, HPRE>::bytes() > Region<T, NR, HPOST>::bytes()
                          ? Region<T, NR, HPRE>::bytes()
                          : Region<T, NR, HPOST>::bytes();
        smem = smem > SmallMem<T, NR>::bytes(5461) ? smem : SmallMem<T, NR>::bytes(5461);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_cycle<T, NR>, CC_THREADS, smem);
        res = per * sms;
        cudaGetLastError();
    }
    for (int l = 1; l < nb; ++l)
        if ((long long)((s.lnx[l] + TX - 1) / TX) * ((s.lny[l] + TY - 1) / TY) <= res) return l;
    return nb;
}

// blocks of a persistent (TMA-staged) tile launch: one per tile, at most as many as are resident
// on the device at once (cached per kernel and shared-memory size)
static int persistent_blocks(const void* kern, int threads, size_t smem, int tiles) {
    struct Entry {
        const void* k;
        size_t smem;
        int dev, blocks;
    };
    thread_local std::vector<Entry> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    int resident = 0;
    for (const Entry& e : cache)
        if (e.k == kern && e.smem == smem && e.dev == dev) resident = e.blocks;
    if (resident == 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
        resident = per > 0 && sms > 0 ? per * sms : 1;
        cudaGetLastError();
        cache.push_back({kern, smem, dev, resident});
    }
    return tiles < resident ? tiles : resident;
}

// z = M r: r is the level-0 rhs, z the level-0 output (both NR-interleaved).
// k_pre of level l writes the pre-smoothed x into X2_l; k_post of level l reads X2_l and the
// coarse correction X_{l+1} (halo included) and writes the final x into X_l (z at level 0):
// no kernel writes an array that another of its blocks still reads.
template <typename T, int NR>
static void vcycle(Solver& s, const T* r, T* z, SolveState* st, cudaStream_t stm) {
    T* X = PT<T>::x(s);
    T* X2 = PT<T>::x2(s);
    T* B = PT<T>::b(s);
    const T* b = r;
    int nb = nbig_of<T>(s);
    ensure_tile_maps(s);
    const int pr = PT<T>::prec;
    int l0 = coarse_start<T, NR>(s);   // tiled levels [l0, nb) go into the cooperative launch
    for (int l = 0; l < l0; ++l) {
        Lev<T> L = lev<T>(s, l);
        dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, s.nz);
        T* bc = B + 2 * s.loff[l + 1];
        size_t ix = tmap_index(pr, NR, l, 0);
        int tma = s.use_tma && s.nz == 1 && s.tma_ok[ix] && (l > 0 || r == PT<T>::r(s));
        using Rg = Region<T, NR, HPRE>;
        size_t smem = tma ? Rg::bytes() + 128 + Stage<T, NR, HPRE, false>::BYTES : Rg::bytes();
        if (tma)
            grid = dim3(persistent_blocks((const void*)k_pre<T, NR>, tile_block<HPRE>(), smem, grid.x * grid.y));
        k_pre<T, NR><<<grid, tile_block<HPRE>(), smem, stm>>>(L, b, X2 + 2 * s.loff[l], bc, st,
                                                              s.timing && l == 0 ? s.timer : nullptr,
                                                              s.tmaps[ix], tma,
                                                              l == 0 && l0 < nb ? s.tickets + 8 : nullptr);
        if (!s.use_graph) ++s.launches;
        b = bc;
    }
    SmallPlan P = small_plan<T>(s);
    if (l0 < nb) {
        CoarsePlan<T> C;
        C.l0 = l0;
        C.nb = nb;
        C.spin = s.barrier_spin > 0 ? s.barrier_spin : (1 << 22);
        for (int l = l0; l < nb; ++l) {
            C.L[l] = lev<T>(s, l);
            C.b[l] = l == 0 ? r : B + 2 * s.loff[l];
            C.x2[l] = X2 + 2 * s.loff[l];
            C.bc[l] = B + 2 * s.loff[l + 1];
            C.xo[l] = l == 0 ? z : X + 2 * s.loff[l];
            C.xc[l] = X + 2 * s.loff[l + 1];
        }
        C.xo[nb] = X + 2 * s.loff[nb];
        size_t smem = coarse_smem<T, NR>(P);
        int tiles = ((s.lnx[l0] + TX - 1) / TX) * ((s.lny[l0] + TY - 1) / TY);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(tiles);
        cfg.blockDim = dim3(CC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stm;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_coarse_cycle<T, NR>, C, P, (const T*)PT<T>::diag(s), (const T*)PT<T>::wl(s),
                           (const T*)PT<T>::wb(s), (const T*)PT<T>::inv(s), st, s.tickets + 8);
        if (!s.use_graph) ++s.launches;
    } else {
        size_t smem = SmallMem<T, NR>::bytes(P.total);
        T* x = nb == 0 ? z : X + 2 * s.loff[nb];
        const T* inv = PT<T>::inv(s);
        if (nb == 0)
            k_small<T, NR, true><<<dim3(1, 1, s.nz), SMALL_THREADS, smem, stm>>>(P, PT<T>::diag(s), PT<T>::wl(s),
                                                                               PT<T>::wb(s), inv, b, x, st);
        else
            k_small<T, NR, false><<<dim3(1, 1, s.nz), SMALL_THREADS, smem, stm>>>(P, PT<T>::diag(s), PT<T>::wl(s),
                                                                                PT<T>::wb(s), inv, b, x, st);
        if (!s.use_graph) ++s.launches;
    }
    for (int l = l0 - 1; l >= 0; --l) {
        Lev<T> L = lev<T>(s, l);
        dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, s.nz);
        const T* bl = l == 0 ? r : B + 2 * s.loff[l];
        const T* xin = X2 + 2 * s.loff[l];
        T* xout = l == 0 ? z : X + 2 * s.loff[l];
        const T* xc = X + 2 * s.loff[l + 1];
        size_t ix = tmap_index(pr, NR, l, 1);
        int tma = s.use_tma && s.nz == 1 && s.tma_ok[ix] && (l > 0 || r == PT<T>::r(s));
        using Rg = Region<T, NR, HPOST>;
        size_t smem = tma ? Rg::bytes() + 128 + Stage<T, NR, HPOST, true>::BYTES : Rg::bytes();
        KTimer* tm = s.timing && l == 0 ? s.timer + 1 : nullptr;
        if (tma) {
            const void* kern = l == 0 ? (const void*)k_post<T, NR, true> : (const void*)k_post<T, NR, false>;
            grid = dim3(persistent_blocks(kern, tile_block<HPOST>(), smem, grid.x * grid.y));
        }
        if (l == 0)
            k_post<T, NR, true><<<grid, tile_block<HPOST>(), smem, stm>>>(L, bl, xin, xout, xc, st, s.partial,
                                                                          s.tickets + 4, tm, s.tmaps[ix], tma);
        else
            k_post<T, NR, false><<<grid, tile_block<HPOST>(), smem, stm>>>(L, bl, xin, xout, xc, st, s.partial,
                                                                           s.tickets + 4, tm, s.tmaps[ix], tma);
        if (!s.use_graph) ++s.launches;
    }
}

// one CG iteration body: z = M r (+beta), p/q/alpha, x/r/test
template <typename T, int NR>
static void cg_body(Solver& s, T* x, T* r, T* z, T* p, T* q, SolveState* st, cudaGraphConditionalHandle h, int use_h,
                    cudaStream_t stm) {
    if (use_h == 2) k_cond_reset<<<1, 32, 0, stm>>>(h, h, 0);
    vcycle<T, NR>(s, r, z, st, stm);
    int N = s.nx * s.ny;
    Lev<T> L0 = lev<T>(s, 0);
    T* p1 = p + (size_t)N * NR;
    if constexpr (sizeof(T) == 4) {
        // four values per thread (four cells, or two cells of two right-hand sides) where the
        // rows and the arrays allow 16-byte accesses
        auto a16 = [](const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; };
        constexpr int G = 4 / NR;   // cells per thread
        if (s.nx % G == 0 && s.zs % 16 == 0 && a16(x) && a16(r) && a16(z) && a16(p) && a16(q) && a16(L0.diag) &&
            a16(L0.wl) && a16(L0.wb)) {
            const int NQ = N / G;
            if constexpr (NR == 1)
                k_apply4<<<dim3(lblocks(NQ, s.nz), 1, s.nz), RB, 0, stm>>>(L0, z, p, p1, q, st, s.partial,
                                                                           s.tickets + 1, nblocks(NQ));
            else
                k_apply2<<<dim3(lblocks(NQ, s.nz), 1, s.nz), RB, 0, stm>>>(L0, z, p, p1, q, st, s.partial,
                                                                           s.tickets + 1, nblocks(NQ));
            k_update4<NR><<<dim3(lblocks(NQ, s.nz), 1, s.nz), RB, 0, stm>>>(N, s.zs, x, r, p, p1, q, st, s.partial,
                                                                            s.tickets + 2, h, use_h, nblocks(NQ));
            if (!s.use_graph) s.launches += 2;
            return;
        }
    }
    k_apply<T, NR><<<dim3(lblocks(N, s.nz), 1, s.nz), RB, 0, stm>>>(L0, z, p, p1, q, st, s.partial, s.tickets + 1,
                                                                   nblocks(N));
    k_update<T, NR><<<dim3(lblocks(N, s.nz), 1, s.nz), RB, 0, stm>>>(N, s.zs, x, r, p, p1, q, st, s.partial,
                                                                    s.tickets + 2, h, use_h, nblocks(N));
    if (!s.use_graph) s.launches += 2;
}

// capture helpers (graph mode): open a WHILE node at the current capture position
struct WhileScope {
    cudaStream_t outer, inner;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t node;
    bool ok = false;
};

static cudaGraphConditionalHandle make_handle(cudaStream_t stm, cudaGraph_t* g_out) {
    cudaStreamCaptureStatus cs;
    unsigned long long id;
    cudaGraph_t g;
    const cudaGraphNode_t* deps;
    const cudaGraphEdgeData* ed;
    size_t nd;
    cudaStreamGetCaptureInfo(stm, &cs, &id, &g, &deps, &ed, &nd);
    cudaGraphConditionalHandle h;
    cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    *g_out = g;
    return h;
}

static cudaStream_t begin_while(cudaStream_t stm, cudaStream_t bs, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cs;
    unsigned long long id;
    cudaGraph_t g;
    const cudaGraphNode_t* deps;
    const cudaGraphEdgeData* ed;
    size_t nd;
    cudaStreamGetCaptureInfo(stm, &cs, &id, &g, &deps, &ed, &nd);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    cudaGraphAddNode(&node, g, deps, ed, nd, &cp);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStreamUpdateCaptureDependencies(stm, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    return bs;
}

static void end_while(cudaStream_t bs) {
    cudaGraph_t g;
    cudaStreamEndCapture(bs, &g);
}

static void poll(Solver& s, cudaStream_t stm) {
    cudaMemcpyAsync(s.st_host + s.slot, s.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stm);
    cudaStreamSynchronize(stm);
}

template <int NR>
static void solve_fp64(Solver& s, const double* b, double* x, double rtol, int max_iter, cudaStream_t stm) {
    int N = s.nx * s.ny;
    Lev<double> L0 = lev<double>(s, 0);
    double* z = s.d_x;   // level-0 slot of the per-level x is z
    if (s.use_graph) {
        cudaGraph_t g;
        cudaGraphConditionalHandle h = make_handle(stm, &g);
        int mode = s.nz > 1 ? 2 : 1;
        k_init64<NR><<<dim3(lblocks(N, s.nz), 1, s.nz), RB, 0, stm>>>(L0, b, x, s.d_r, s.st, s.partial, s.tickets,
                                                                      rtol * rtol, max_iter, h, mode, nblocks(N));
        ++s.launches;
        cudaStream_t bs = begin_while(stm, s.aux[0], h);
        cg_body<double, NR>(s, x, s.d_r, z, s.d_p, s.d_q, s.st, h, mode, bs);
        end_while(bs);
        return;
    }
    k_init64<NR><<<dim3(lblocks(N, s.nz), 1, s.nz), RB, 0, stm>>>(L0, b, x, s.d_r, s.st, s.partial, s.tickets,
                                                                  rtol * rtol, max_iter, 0, 0, nblocks(N));
    ++s.launches;
    poll(s, stm);
    for (int it = 0; it < max_iter && !s.st_host[s.slot].done; ++it) {
        cg_body<double, NR>(s, x, s.d_r, z, s.d_p, s.d_q, s.st, 0, 0, stm);
        poll(s, stm);
    }
}

// The whole inner FP32 solve as one cooperative launch (use_coop == 2): single instances with
// at least one tiled level whose finest tiles and block slots fit the reduction buffer; the
// grid is min(finest tiles, co-resident blocks).  False: the solve runs as separate kernels.
template <int NR>
static bool persist_plan(Solver& s, CoarsePlan<float>& C, SmallPlan& P, int& G, size_t& smem) {
    if (s.use_coop != 2 || s.nz != 1) return false;
    int nb = nbig_of<float>(s);
    if (nb < 1) return false;
    P = small_plan<float>(s);
    smem = coarse_smem<float, NR>(P);
    struct Entry { size_t smem; int dev, res; };
    thread_local std::vector<Entry> cache[2];
    int dev = 0;
    cudaGetDevice(&dev);
    int res = -1;
    for (const Entry& e : cache[NR - 1])
        if (e.smem == smem && e.dev == dev) res = e.res;
    if (res < 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg_persist<float, NR>, CC_THREADS, smem);
        res = per * sms;
        cudaGetLastError();
        cache[NR - 1].push_back({smem, dev, res});
    }
    long long nt0 = (long long)tiles(s.nx, s.ny);
    G = (int)(nt0 < res ? nt0 : res);
    long long mb = nt0 > NRED ? nt0 : NRED;
    if (G < 1 || 2 * nt0 + 4LL * G > 4 * mb) return false;
    float* X = s.f_x;
    float* X2 = s.f_x2;
    float* B = s.f_b;
    C.l0 = 0;
    C.nb = nb;
    C.spin = s.barrier_spin > 0 ? s.barrier_spin : (1 << 22);
    for (int l = 0; l < nb; ++l) {
        C.L[l] = lev<float>(s, l);
        C.b[l] = l == 0 ? s.f_r : B + 2 * s.loff[l];
        C.x2[l] = X2 + 2 * s.loff[l];
        C.bc[l] = B + 2 * s.loff[l + 1];
        C.xo[l] = X + 2 * s.loff[l];
        C.xc[l] = X + 2 * s.loff[l + 1];
    }
    C.xo[nb] = X + 2 * s.loff[nb];
    return true;
}

template <int NR>
static void launch_persist(Solver& s, const CoarsePlan<float>& C, const SmallPlan& P, int G, size_t smem,
                           cudaStream_t stm) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(CC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stm;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_cg_persist<float, NR>, C, P, (const float*)s.f_diag, (const float*)s.f_wl,
                       (const float*)s.f_wb, (const float*)s.f_inv, s.f_e, s.f_r, s.f_p,
                       s.f_p + (size_t)s.nx * s.ny * NR, s.f_q, s.st, s.partial, s.tickets + 8);
    if (!s.use_graph) ++s.launches;
}

template <int NR>
static void solve_mixed(Solver& s, Lev<double> L64, const double* b, double* x, double rtol, int max_iter,
                        cudaStream_t stm) {
    int N = s.nx * s.ny;
    const int max_outer = 8;
    const double inner_rtol = s.inner_rtol;
    float* z = s.f_x;
    const int vb = nblocks(N), lb = lblocks(N, s.nz), lbu = lblocks((long long)N * NR, s.nz);
    k_ir_init<NR><<<dim3(lb, 1, s.nz), RB, 0, stm>>>(N, s.zs, b, s.st, s.partial, s.tickets + 3, rtol * rtol,
                                                     inner_rtol, max_iter, max_outer, vb);
    ++s.launches;
    CoarsePlan<float> PC;
    SmallPlan PS;
    int PG = 0;
    size_t psmem = 0;
    bool persist = persist_plan<NR>(s, PC, PS, PG, psmem);
    unsigned* pbar = persist ? s.tickets + 8 : nullptr;
    if (s.use_graph) {
        cudaGraph_t g;
        cudaGraphConditionalHandle ho = make_handle(stm, &g);
        cudaStream_t obs = begin_while(stm, s.aux[0], ho);
        int mode = s.nz > 1 ? 2 : 1;
        if (persist) {
            k_ir_residual<NR><<<dim3(lb, 1, s.nz), RB, 0, obs>>>(L64, b, x, s.f_r, s.f_e, s.st, s.partial,
                                                                 s.tickets + 5, ho, ho, mode, 0, pbar, vb);
            launch_persist<NR>(s, PC, PS, PG, psmem, obs);
        } else {
            cudaGraph_t og;
            cudaGraphConditionalHandle hi = make_handle(obs, &og);
            if (mode == 2) k_cond_reset<<<1, 32, 0, obs>>>(ho, hi, 1);
            k_ir_residual<NR><<<dim3(lb, 1, s.nz), RB, 0, obs>>>(L64, b, x, s.f_r, s.f_e, s.st, s.partial,
                                                                 s.tickets + 5, ho, hi, mode, 1, nullptr, vb);
            cudaStream_t ibs = begin_while(obs, s.aux[1], hi);
            cg_body<float, NR>(s, s.f_e, s.f_r, z, s.f_p, s.f_q, s.st, hi, mode, ibs);
            end_while(ibs);
        }
        k_ir_update<NR><<<dim3(lbu, 1, s.nz), RB, 0, obs>>>(N, s.zs, x, s.f_e, s.st);
        end_while(obs);
        return;
    }
    for (int o = 0; o <= max_outer; ++o) {
        k_ir_residual<NR><<<dim3(lb, 1, s.nz), RB, 0, stm>>>(L64, b, x, s.f_r, s.f_e, s.st, s.partial,
                                                             s.tickets + 5, 0, 0, 0, 0, pbar, vb);
        ++s.launches;
        poll(s, stm);
        if (s.st_host[s.slot].odone) break;
        if (persist) {
            launch_persist<NR>(s, PC, PS, PG, psmem, stm);
        } else {
            for (int it = 0; it < max_iter && !s.st_host[s.slot].done; ++it) {
                cg_body<float, NR>(s, s.f_e, s.f_r, z, s.f_p, s.f_q, s.st, 0, 0, stm);
                poll(s, stm);
            }
        }
        k_ir_update<NR><<<dim3(lbu, 1, s.nz), RB, 0, stm>>>(N, s.zs, x, s.f_e, s.st);
        ++s.launches;
    }
}

void Solver::solve(const double* cd, const double* dd, const double* wl, const double* wb, const double* b, double* x,
                   int nr, int precision, double rtol, int max_iter, cudaStream_t stm) {
    st = st_base + slot;
    // the FP64 level-0 operator is needed in both modes (outer residual of the refinement)
    if (precision == 0) {
        setup_levels<double>(*this, cd, dd, wl, wb, nullptr, stm);
        if (nr == 1) solve_fp64<1>(*this, b, x, rtol, max_iter, stm);
        else solve_fp64<2>(*this, b, x, rtol, max_iter, stm);
    } else {
        // the FP32 hierarchy, plus D in FP64 for the refinement residual (whose face weights are
        // the caller's FP64 arrays)
        setup_levels<float>(*this, cd, dd, wl, wb, d_diag, stm);
        Lev<double> L64{nx, ny, d_diag, wl, wb, zs};
        if (nr == 1) solve_mixed<1>(*this, L64, b, x, rtol, max_iter, stm);
        else solve_mixed<2>(*this, L64, b, x, rtol, max_iter, stm);
    }
}

bool Solver::set_schedule(int small_max, double inner) {
    if (small_max < 16 || small_max > SMALL_MAX_F_LIMIT || !(inner > 0 && inner < 1)) return false;
    small_max_f = small_max;
    inner_rtol = inner;
    int nb = 0;
    while (nb < nlev - 1 && (long long)lnx[nb] * lny[nb] > small_max_f) ++nb;
    nbig_f = nb;
    nbig = nbig_f;
    tma_ready = false;
    return true;
}

int Solver::body_size(int precision) const { return 2 * (precision == 0 ? nbig_d : nbig_f) + 1 + 2; }

bool Solver::supported(int nx, int ny) {
    Solver s;
    s.plan(nx, ny);
    return (long long)s.lnx[s.nlev - 1] * s.lny[s.nlev - 1] <= SMALL_MAX_D;
}

void Solver::fetch_states(cudaStream_t stm) {
    cudaMemcpyAsync(st_host, st_base, NSLOT * sizeof(SolveState), cudaMemcpyDeviceToHost, stm);
}

SolveResult Solver::read_result(int sl, int precision, cudaStream_t stm, cudaError_t* err) {
    cudaError_t e = cudaMemcpyAsync(st_host + sl, st_base + sl, sizeof(SolveState), cudaMemcpyDeviceToHost, stm);
    cudaError_t es = cudaStreamSynchronize(stm);
    if (e == cudaSuccess) e = es;
    if (err) *err = e;
    SolveResult r{};
    if (e != cudaSuccess) {   // the state was not read back: no valid result
        r.fault = true;
        return r;
    }
    return result_from_host(sl, precision);
}

SolveResult Solver::result_from_host(int sl, int precision) const {
    const SolveState& h = st_host[sl];
    SolveResult r{};
    double worst = 0.0;
    for (int k = 0; k < (h.nr > 0 ? h.nr : 1); ++k) {
        double num = precision == 0 ? h.rr[k] : h.orr[k];
        double den = precision == 0 ? h.bb[k] : h.obb[k];
        double q = sqrt(num / (den > 1e-300 ? den : 1e-300));
        if (q > worst) worst = q;
    }
    r.rel_res = worst;
    r.fault = h.fault != 0;
    r.nonfinite = h.nonfinite != 0;
    if (precision == 0) {
        r.iters = h.iters;
        r.converged = h.done != 0;
    } else {
        r.iters = h.itot;
        r.outer = h.oiters;
        bool ok = true;
        for (int k = 0; k < (h.nr > 0 ? h.nr : 1); ++k) ok = ok && h.orr[k] <= h.otol2[k];
        r.converged = ok;
    }
    return r;
}

}  // namespace ebit

// ---------------------------------------------------------------------------------------
// Allocation-free solve.  Some callers cannot allocate device memory when they call the
// solver: a host framework that owns the whole device memory through its own pool and
// forbids other allocations, or a long-running service loop that must not allocate per call
// (latency, fragmentation).  ebit_solve_system_noalloc takes the caller's device arrays for
// the operator, the right-hand side and the solution, and keeps every scratch array of the
// multigrid-preconditioned CG in the fixed array below.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds its
// 6 MiB until the process exits.  Its device address is looked up once per device, with that
// device current, by the first call on that device.  All calls share the array and it keeps
// the last call's contents; the per-call device state that must start at zero (reduction
// tickets, solver state, timers) is cleared at the start of each call.  Two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the array.
// ---------------------------------------------------------------------------------------
#include <atomic>

#include "../../include/ebit.h"
#include "status.h"

namespace ebit {
constexpr size_t NOALLOC_BYTES = (size_t)6 << 20;
constexpr int NOALLOC_MAX_CELLS = 128 * 128;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
// device address of g_noalloc_scratch per device (host side); every writer stores the same
// address for a device, and the atomics make concurrent first calls well defined
static std::atomic<void*> g_noalloc_addr[64];
}  // namespace ebit

extern "C" ebit_status ebit_solve_system_noalloc(int nx, int ny, const double* D, const double* wl, const double* wb,
                                                 const double* b, double* x, int nr, int precision, double rtol,
                                                 int max_iter, void* stream, int* iters, double* rel_res) {
    using namespace ebit;
    if (nx < 2 || ny < 2 || !D || !wl || !wb || !b || !x || (nr != 1 && nr != 2) ||
        (precision != EBIT_FP64 && precision != EBIT_MIXED) || !(rtol > 0) || max_iter < 1)
        return EBIT_EINVAL;
    if ((long long)nx * ny > NOALLOC_MAX_CELLS || Solver::bytes(nx, ny) > NOALLOC_BYTES || !Solver::supported(nx, ny))
        return EBIT_EINVAL;   // larger than the fixed scratch array (at most 128 x 128 cells)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EBIT_ECUDA;
    void* base = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!base) {
        if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) return EBIT_ECUDA;
        g_noalloc_addr[dev].store(base, std::memory_order_release);
    }
    // an error already pending from an earlier, unrelated runtime call is not this call's: it
    // is left in place, and only an error that appears during this call is taken (and cleared)
    const bool clean = cudaPeekAtLastError() == cudaSuccess;
    cudaStream_t st = (cudaStream_t)stream;
    Solver s;
    if (s.bind(base, nx, ny, false, st) != cudaSuccess) {
        if (clean) cudaGetLastError();
        return EBIT_ECUDA;
    }
    SolveState host[Solver::NSLOT];   // read_result synchronises before returning: the stack copy is safe
    s.st_host = host;
    s.slot = 0;
    s.use_graph = 0;
    s.solve(D, nullptr, wl, wb, b, x, nr, precision, rtol, max_iter, st);
    cudaError_t e = cudaSuccess;
    SolveResult r = s.read_result(0, precision, st, &e);
    if (e == cudaSuccess && clean) e = cudaGetLastError();   // launch errors of the solve
    if (e == cudaSuccess) {
        if (iters) *iters = r.iters;
        if (rel_res) *rel_res = r.rel_res;
    }
    return solve_status(e == cudaSuccess, r.fault, r.nonfinite, r.converged);
}
