// Cell/face field kernels of the EBIT phase-change step (FP64):
//   S1   WENO3 energy advection (energy-advection equation, Sec. 2.4)
//   S6   narrow-band extension (extrapolation equation, Sec. 2.4) over a compacted band list
//   S10  ghost velocities (ghost-velocity equation, Sec. 2.3)
//   S11  momentum predictor pieces (discretization equations 1-3, Sec. 2.3)
//   S12  ghost-fluid Poisson operator/RHS and the projection update (ghost-fluid Poisson
//        equation, discretization equations 4-5)
//   S13  diagnostics (mass-in-domain and mass-with-outflow equations, vapour volume)
// Cell-band compaction uses one warp ballot + popcount prefix per warp and one atomic per
// warp; the resulting list order is irrelevant to every consumer (Jacobi updates).
#include "common.cuh"
#include "kernels.h"

namespace ebit {

// ---------------------------------------------------------------------------------
// boundary-reflected scalar access (two ghost layers)
// ---------------------------------------------------------------------------------
struct Refl {
    int odd[4];      // per side: odd reflection about val[s], else even
    double val[4];
};

__device__ inline double refl_x(const double* F, const Grid& g, const Refl& r, int i, int j) {
    if (i < 0) {
        double v = F[cidx(g, -1 - i, j)];
        return r.odd[0] ? 2.0 * r.val[0] - v : v;
    }
    if (i >= g.nx) {
        double v = F[cidx(g, 2 * g.nx - 1 - i, j)];
        return r.odd[1] ? 2.0 * r.val[1] - v : v;
    }
    return F[cidx(g, i, j)];
}
__device__ inline double refl_y(const double* F, const Grid& g, const Refl& r, int i, int j) {
    if (j < 0) {
        double v = F[cidx(g, i, -1 - j)];
        return r.odd[2] ? 2.0 * r.val[2] - v : v;
    }
    if (j >= g.ny) {
        double v = F[cidx(g, i, 2 * g.ny - 1 - j)];
        return r.odd[3] ? 2.0 * r.val[3] - v : v;
    }
    return F[cidx(g, i, j)];
}

// components of a double2 field viewed as a strided scalar: comp 0/1
struct Comp {
    const double2* F;
    int comp;
    __device__ double operator[](int c) const { return comp == 0 ? F[c].x : F[c].y; }
};
__device__ inline double refl_x(const Comp& F, const Grid& g, const Refl& r, int i, int j) {
    if (i < 0) { double v = F[cidx(g, -1 - i, j)]; return r.odd[0] ? 2.0 * r.val[0] - v : v; }
    if (i >= g.nx) { double v = F[cidx(g, 2 * g.nx - 1 - i, j)]; return r.odd[1] ? 2.0 * r.val[1] - v : v; }
    return F[cidx(g, i, j)];
}
__device__ inline double refl_y(const Comp& F, const Grid& g, const Refl& r, int i, int j) {
    if (j < 0) { double v = F[cidx(g, i, -1 - j)]; return r.odd[2] ? 2.0 * r.val[2] - v : v; }
    if (j >= g.ny) { double v = F[cidx(g, i, 2 * g.ny - 1 - j)]; return r.odd[3] ? 2.0 * r.val[3] - v : v; }
    return F[cidx(g, i, j)];
}

// WENO3 upwind derivative (undivided) from five values along a line (Jiang-Shu, linear weights
// 1/3 and 2/3, smoothness indicators b0 = (v2 - v1)^2, b1 = (v3 - v2)^2, eps = 1e-6).  With the
// undivided upwind differences v1, v2, v3 the two candidates are phi0 = (3 v2 - v1)/2 and
// phi1 = (v2 + v3)/2, and the normalised weight of phi0 is
//   w0 = (1/3)/(eps + b0)^2 / ((1/3)/(eps + b0)^2 + (2/3)/(eps + b1)^2)
//      = (eps + b1)^2 / ((eps + b1)^2 + 2 (eps + b0)^2),
// so the derivative is phi1 + w0 (phi0 - phi1) with phi0 - phi1 = ((v2 - v1) - (v3 - v2))/2:
// the second differences serve both the indicators and the candidates' difference.  The
// differences and the final combination are FP64; the weight w0 is formed from the second
// differences in FP32-pair arithmetic (48-bit, relative error a few times 2^-44: the derivative
// then differs from its FP64 evaluation by a few times 1e-14 of the second difference).
// Second differences of 2^28 or more take the FP64 formula (a call, not an inlined branch, so
// that its FP64 instructions are not issued for every stencil).
__device__ __noinline__ double weno_weight_fp64(double a1, double a2) {
    const double eps = 1e-6;
    double s0 = fma(a1, a1, eps), s1 = fma(a2, a2, eps);
    double q0 = s1 * s1;
    return q0 / fma(s0 + s0, s0, q0);
}
__device__ inline double weno_weight(double a1, double a2) {
    unsigned e1 = (unsigned)(__double_as_longlong(a1) >> 52) & 0x7ffu;
    unsigned e2 = (unsigned)(__double_as_longlong(a2) >> 52) & 0x7ffu;
    if ((e1 > e2 ? e1 : e2) >= 1023u + 28u) return weno_weight_fp64(a1, a2);
    constexpr double EPS = 1e-6;
    constexpr float EPS_HI = (float)EPS;
    constexpr float EPS_LO = (float)(EPS - (double)EPS_HI);
    const f32x2 eps = {EPS_HI, EPS_LO};
    f32x2 A1 = x2_from(a1), A2 = x2_from(a2);
    f32x2 s0 = x2_add(x2_mul(A1, A1), eps), s1 = x2_add(x2_mul(A2, A2), eps);
    f32x2 q0 = x2_mul(s1, s1), t = x2_mul(s0, s0);
    f32x2 d = x2_add({t.hi + t.hi, t.lo + t.lo}, q0);
    return x2_to(x2_div(q0, d));
}
//
// weno3_up takes the stencil ordered from the upwind side, up2 and up1 the two upwind values,
// dn the downwind one, and returns twice the derivative along the flow direction.  For u >= 0
// that is the ordering (T_{i-2}, T_{i-1}, T_i, T_{i+1}) and the derivative along +x; for u < 0
// the mirror image (T_{i+2}, T_{i+1}, T_i, T_{i-1}), whose differences are the negated ones of
// the upwind-from-the-right stencil, so the x-derivative is the negative of the result (every
// difference changes sign, the indicators do not).  u dT/dx is therefore |u| times the result
// / 2: the selection costs no FP64 instruction and the factor 1/2 is folded into dt/h.
__device__ inline double weno3_up(double up2, double up1, double T0, double dn) {
    double v1 = up1 - up2, v2 = T0 - up1, v3 = dn - T0;
    double a1 = v2 - v1, a2 = v3 - v2;
    return fma(weno_weight(a1, a2), a1 - a2, v2 + v3);
}
// u >= 0 from the sign bit (no FP64 comparison); -0.0 takes the mirrored stencil, which only
// multiplies a zero velocity
__device__ inline bool upwind_left(double u) { return __double2hiint(u) >= 0; }

// ---- tiled form: the values a 32 x 8 tile of cells reads (two halo layers, boundary
// reflections applied) are staged once in shared memory, in FP64, and each thread evaluates
// the WENO3 stencils of its cell from there (weno3_up on the staged values, without the
// five-fold re-reading of the field through the cache)
constexpr int WX = 32, WY = 8, WH = 2, WSX = WX + 2 * WH, WSY = WY + 2 * WH;

struct Scal {
    const double* F;
    __device__ double operator[](int c) const { return F[c]; }
};
__device__ inline double refl_x(const Scal& F, const Grid& g, const Refl& r, int i, int j) {
    return refl_x(F.F, g, r, i, j);
}
__device__ inline double refl_y(const Scal& F, const Grid& g, const Refl& r, int i, int j) {
    return refl_y(F.F, g, r, i, j);
}

template <class F>
__device__ inline double tile_value(const F& T, const Grid& g, const Refl& r, int i, int j) {
    // a ragged tile reaches past the two reflected layers (up to WX + 1 cells beyond a grid
    // narrower than the tile): no stencil of a grid cell reads there, and the reflection would
    // index outside the field
    if (i > g.nx + 1 || j > g.ny + 1) return 0.0;
    bool iin = i >= 0 && i < g.nx, jin = j >= 0 && j < g.ny;
    if (iin && jin) return T[cidx(g, i, j)];
    if (jin) return refl_x(T, g, r, i, j);
    if (iin) return refl_y(T, g, r, i, j);
    return 0.0;   // a tile corner: no stencil reads it
}

// stage NF fields of the tile (field f: accessor T[f], reflection rule R[f])
template <int NF, class F>
__device__ inline void tile_stage(const F* T, const Refl* R, const Grid& g, int i0, int j0,
                                  double (*sh)[WSY][WSX]) {
    for (int k = threadIdx.x; k < WSX * WSY; k += blockDim.x) {
        int rx = k % WSX, ry = k / WSX;
        int i = i0 - WH + rx, j = j0 - WH + ry;
#pragma unroll
        for (int f = 0; f < NF; ++f) sh[f][ry][rx] = tile_value(T[f], g, R[f], i, j);
    }
    __syncthreads();
}

// T - dt/h (u . D T) at tile position (rx, ry) of the staged field v; hdth = dt / (2 h)
__device__ inline double tile_advect(const double (*v)[WSX], int rx, int ry, double2 u, double hdth) {
    const double* row = v[ry];
    bool lx = upwind_left(u.x), ly = upwind_left(u.y);
    double T0 = row[rx];
    double ex = weno3_up(row[lx ? rx - 2 : rx + 2], row[lx ? rx - 1 : rx + 1], T0, row[lx ? rx + 1 : rx - 1]);
    double ey = weno3_up(v[ly ? ry - 2 : ry + 2][rx], v[ly ? ry - 1 : ry + 1][rx], T0, v[ly ? ry + 1 : ry - 1][rx]);
    return T0 - hdth * (fabs(u.x) * ex + fabs(u.y) * ey);
}


// ---- the same with the second differences of the tile shared: D_i = T_{i+1} - 2 T_i + T_{i-1}
// along x at tile columns -1 .. WX (rows 0 .. WY-1) and along y at tile rows -1 .. WY (columns
// 0 .. WX-1), formed once per cell and field.  In the upwind-ordered stencil the two second
// differences are a1 = D_{i-1}, a2 = D_i for u >= 0 and a1 = D_{i+1}, a2 = D_i for u < 0, and
// v2 + v3 = +-(T_{i+1} - T_{i-1}), so a stencil costs four FP64 operations instead of nine
// (the mathematical value is that of weno3_up; the rounding differs by a few ulps of T).
constexpr int D2X_N = (WX + 2) * WY, D2Y_N = WX * (WY + 2);
template <int NF>
__device__ inline void tile_d2(const double (*sh)[WSY][WSX], double (*d2x)[WY][WX + 2],
                               double (*d2y)[WY + 2][WX]) {
    for (int k = threadIdx.x; k < D2X_N + D2Y_N; k += blockDim.x) {
        if (k < D2X_N) {
            int cx = k % (WX + 2), cy = k / (WX + 2);   // tile column cx - 1, row cy
            int rx = cx - 1 + WH, ry = cy + WH;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                d2x[f][cy][cx] = fma(-2.0, sh[f][ry][rx], sh[f][ry][rx - 1] + sh[f][ry][rx + 1]);
        } else {
            int q = k - D2X_N;
            int cx = q % WX, cy = q / WX;   // tile column cx, row cy - 1
            int rx = cx + WH, ry = cy - 1 + WH;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                d2y[f][cy][cx] = fma(-2.0, sh[f][ry][rx], sh[f][ry - 1][rx] + sh[f][ry + 1][rx]);
        }
    }
    __syncthreads();
}
// T - dt/h (u . D T) at tile cell (tx, ty) of the staged field v with its second differences
__device__ inline double tile_advect_d2(const double (*v)[WSX], const double (*dx)[WX + 2], const double (*dy)[WX],
                                        int tx, int ty, double2 u, double hdth) {
    const int rx = tx + WH, ry = ty + WH;
    bool lx = upwind_left(u.x), ly = upwind_left(u.y);
    double T0 = v[ry][rx];
    // the central difference oriented along the flow (operands selected, no FP64 negation)
    double cx = v[ry][lx ? rx + 1 : rx - 1] - v[ry][lx ? rx - 1 : rx + 1];
    double cy = v[ly ? ry + 1 : ry - 1][rx] - v[ly ? ry - 1 : ry + 1][rx];
    double ax2 = dx[ty][tx + 1], ax1 = dx[ty][lx ? tx : tx + 2];
    double ay2 = dy[ty + 1][tx], ay1 = dy[ly ? ty : ty + 2][tx];
    double ex = fma(weno_weight(ax1, ax2), ax1 - ax2, cx);
    double ey = fma(weno_weight(ay1, ay2), ay1 - ay2, cy);
    return T0 - hdth * (fabs(u.x) * ex + fabs(u.y) * ey);
}

__host__ inline Refl temperature_refl(const Grid& g) {
    Refl r;
    for (int s = 0; s < 4; ++s) { r.odd[s] = g.Tfix[s]; r.val[s] = g.Tw[s]; }
    return r;
}
__host__ inline Refl velocity_refl(const Grid& g, int comp) {
    Refl r;
    for (int s = 0; s < 4; ++s) { r.odd[s] = vel_odd(g.bc[s], comp, s < 2 ? 0 : 1); r.val[s] = 0.0; }
    return r;
}

// S1: T*_k = T_k - dt u_k . grad T_k on the cells of phase k (centre colours of the interface
// before it moves); elsewhere T*_k = T_k (the other phase's band cells are refilled by the
// extension, cells beyond the band are not read).  Block WX x WY threads, one cell each.
__global__ void __launch_bounds__(WX * WY) k_advect_T(Grid g, Refl r, double dth, const uint8_t* __restrict__ flags,
                                                     const double* __restrict__ T_l,
                                                     const double* __restrict__ T_v,
                                                     const double2* __restrict__ u_l,
                                                     const double2* __restrict__ u_v, double* __restrict__ Ts_l,
                                                     double* __restrict__ Ts_v) {
    if (g.pz) dth = g.pz[blockIdx.z].dt / g.h;
    const double hdth = 0.5 * dth;
    const long long zo = zoff(g.zs);
    flags = zsh(flags, zo);
    T_l = zsh(T_l, zo);
    T_v = zsh(T_v, zo);
    u_l = zsh(u_l, zo);
    u_v = zsh(u_v, zo);
    Ts_l = zsh(Ts_l, zo);
    Ts_v = zsh(Ts_v, zo);
    __shared__ double sh[2][WSY][WSX];
    int i0 = blockIdx.x * WX, j0 = blockIdx.y * WY;
    Scal F[2] = {{T_l}, {T_v}};
    Refl R[2] = {r, r};
    tile_stage<2>(F, R, g, i0, j0, sh);
    int tx = threadIdx.x % WX, ty = threadIdx.x / WX;
    int i = i0 + tx, j = j0 + ty;
    if (i >= g.nx || j >= g.ny) return;
    int c = cidx(g, i, j);
    int sx = tx + WH, sy = ty + WH;
    bool liq = flags[c] & F_CCOL;
    double adv = tile_advect(sh[liq ? 0 : 1], sx, sy, (liq ? u_l : u_v)[c], hdth);
    Ts_l[c] = liq ? adv : sh[0][sy][sx];
    Ts_v[c] = liq ? sh[1][sy][sx] : adv;
}

// ---------------------------------------------------------------------------------
// compaction (warp ballot + popcount prefix, one atomic per warp)
// ---------------------------------------------------------------------------------
__global__ void k_compact(const uint8_t* __restrict__ flags, int N, uint8_t mask, int* __restrict__ list,
                          int* __restrict__ count, int* __restrict__ idxmap, long long zs) {
    const long long zo = zoff(zs);
    flags = zsh(flags, zo);
    list = zsh(list, zo);
    count = zsh(count, zo);
    idxmap = zsh(idxmap, zo);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    bool pred = c < N && (flags[c] & mask);
    unsigned bal = __ballot_sync(0xffffffffu, pred);
    int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(count, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pred) {
        int k = base + __popc(bal & ((1u << lane) - 1u));
        list[k] = c;
        if (idxmap) idxmap[c] = k;
    }
}

// ---------------------------------------------------------------------------------
// S6: one Jacobi sweep of the upwind steady balance of the extrapolation equation
//   mode 0: T_l into vapour band cells, along +n
//   mode 1: T_v into liquid band cells, along -n
//   mode 2: mdot from cut cells into the rest of the band (+n in vapour, -n in liquid)
// Values of band cells being extended live in vcur/vnxt between sweeps; the last sweep
// writes the field itself (its band cells are then read from vcur only).
// ---------------------------------------------------------------------------------
__device__ inline bool ext_update(uint8_t fl, int mode) {
    if (!(fl & F_BAND)) return false;
    if (mode == 0) return !(fl & F_CCOL);
    if (mode == 1) return (fl & F_CCOL) != 0;
    return !(fl & F_CUT);
}

// one Jacobi update of band entry k; mode 3 runs modes 0 and 1 in the same sweep (they update
// disjoint cells of different fields): (f0, vcur0, vnxt0) belong to mode 0 and (f1, vcur1,
// vnxt1) to mode 1
__device__ inline void extend_entry(const Grid& g, int mode, int it, int last, int k, const int* __restrict__ list,
                                    const uint8_t* __restrict__ flags, const int* __restrict__ idxmap,
                                    const double2* __restrict__ nb, double* f0, const double* vcur0, double* vnxt0,
                                    double* f1, const double* vcur1, double* vnxt1) {
    int c = list[k];
    uint8_t fl = flags[c];
    int m = mode == 3 ? ((fl & F_CCOL) ? 1 : 0) : mode;
    if (!ext_update(fl, m)) return;
    double* f = m == 1 && mode == 3 ? f1 : f0;
    const double* vcur = m == 1 && mode == 3 ? vcur1 : vcur0;
    double* vnxt = m == 1 && mode == 3 ? vnxt1 : vnxt0;
    int i = c % g.nx, j = c / g.nx;
    double sgn = m == 0 ? 1.0 : (m == 1 ? -1.0 : ((fl & F_CCOL) ? -1.0 : 1.0));
    double2 nn = nb[c];
    double ax = nn.x * sgn, ay = nn.y * sgn;
    double acc = 0.0, w = 0.0;
    auto val = [&](int cc) -> double {
        if (it > 0 && ext_update(flags[cc], m)) return vcur[idxmap[cc]];
        return f[cc];
    };
    if (ax > 0.0 && i - 1 >= 0) { acc += ax * val(c - 1); w += ax; }
    else if (ax < 0.0 && i + 1 < g.nx) { acc += -ax * val(c + 1); w += -ax; }
    if (ay > 0.0 && j - 1 >= 0) { acc += ay * val(c - g.nx); w += ay; }
    else if (ay < 0.0 && j + 1 < g.ny) { acc += -ay * val(c + g.nx); w += -ay; }
    double nv = w > 0.0 ? acc / w : (it > 0 ? vcur[k] : f[c]);
    if (last) f[c] = nv;
    else vnxt[k] = nv;
}

// one sweep over the band, grid-stride
__global__ void k_extend(Grid g, int mode, int it, int last, const int* __restrict__ list,
                         const int* __restrict__ count, const uint8_t* __restrict__ flags,
                         const int* __restrict__ idxmap, const double2* __restrict__ nb, double* f0,
                         const double* __restrict__ vcur0, double* __restrict__ vnxt0, double* f1,
                         const double* __restrict__ vcur1, double* __restrict__ vnxt1) {
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    flags = zsh(flags, zo);
    idxmap = zsh(idxmap, zo);
    nb = zsh(nb, zo);
    f0 = zsh(f0, zo);
    vcur0 = zsh(vcur0, zo);
    vnxt0 = zsh(vnxt0, zo);
    f1 = zsh(f1, zo);
    vcur1 = zsh(vcur1, zo);
    vnxt1 = zsh(vnxt1, zo);
    int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        extend_entry(g, mode, it, last, k, list, flags, idxmap, nb, f0, vcur0, vnxt0, f1, vcur1, vnxt1);
}

// energy solution (one value per cell) back to the phase fields: T_k = T where f_C = k, T*_k elsewhere
__global__ void k_split_T(int N, const uint8_t* __restrict__ flags, const double* __restrict__ x,
                          const double* __restrict__ Ts_l, const double* __restrict__ Ts_v, double* __restrict__ T_l,
                          double* __restrict__ T_v, long long zs) {
    const long long zo = zoff(zs);
    flags = zsh(flags, zo);
    x = zsh(x, zo);
    Ts_l = zsh(Ts_l, zo);
    Ts_v = zsh(Ts_v, zo);
    T_l = zsh(T_l, zo);
    T_v = zsh(T_v, zo);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    bool liq = flags[c] & F_CCOL;
    T_l[c] = liq ? x[c] : Ts_l[c];
    T_v[c] = liq ? Ts_v[c] : x[c];
}

// ---------------------------------------------------------------------------------
// S10: ghost velocities (cells and faces)
// ---------------------------------------------------------------------------------
// ghost value of a band cell: the other phase's velocity from the velocity-jump equation,
// u_v = u_l - [1/rho] mdot n (liquid centre) or u_l = u_v + [1/rho] mdot n (vapour centre)
__device__ inline void ghost_cell(const Grid& g, double J, int c, const uint8_t* flags, const double* mdot,
                                  const double2* nb, double2* u_l, double2* u_v) {
    uint8_t fl = flags[c];
    double m = mdot[c];
    double2 n = nb[c];
    double mx = m * n.x, my = m * n.y;
    if (fl & F_CCOL) {
        double2 ul = u_l[c];
        u_v[c] = make_double2(ul.x - J * mx, ul.y - J * my);
    } else {
        double2 uv = u_v[c];
        u_l[c] = make_double2(uv.x + J * mx, uv.y + J * my);
    }
}

// ghost value of the interior x-face t (between cells i - 1 and i of row j) or, with y, of the
// interior y-face t (between rows j - 1 and j of column i), if one of its cells is in the band:
// the phase of the face is the colour of its nearer end (the marker position on it decides),
// the face mass flux the mean of its two cells' mdot n
__device__ inline void ghost_face(const Grid& g, double J, bool y, int i, int j, const uint8_t* flags,
                                  const double* mdot, const double2* nb, const uint8_t* vcol, const double* hpos,
                                  const double* vpos, double* uf_l, double* uf_v) {
    if (!y) {
        if (i <= 0 || i >= g.nx) return;
        int a = cidx(g, i - 1, j), b = cidx(g, i, j);
        if (!((flags[a] | flags[b]) & F_BAND)) return;
        long long t = veidx(g, i, j);
        double mf = 0.5 * (mdot[a] * nb[a].x + mdot[b] * nb[b].x);
        uint8_t v0 = vcol[vidx(g, i, j)], v1 = vcol[vidx(g, i, j + 1)];
        int colour = (v0 != v1 && vpos[t] < 0.5) ? v1 : v0;
        if (colour) uf_v[t] = uf_l[t] - J * mf;
        else uf_l[t] = uf_v[t] + J * mf;
    } else {
        if (j <= 0 || j >= g.ny) return;
        int a = cidx(g, i, j - 1), b = cidx(g, i, j);
        if (!((flags[a] | flags[b]) & F_BAND)) return;
        long long t = hidx(g, i, j);
        double mf = 0.5 * (mdot[a] * nb[a].y + mdot[b] * nb[b].y);
        uint8_t v0 = vcol[vidx(g, i, j)], v1 = vcol[vidx(g, i + 1, j)];
        int colour = (v0 != v1 && hpos[t] < 0.5) ? v1 : v0;
        if (colour) uf_v[t] = uf_l[t] - J * mf;
        else uf_l[t] = uf_v[t] + J * mf;
    }
}

// S10 over the band list (O(sqrt N)): five items per band cell, the cell and its four faces.
// A face of two band cells is written twice with the same value from the same inputs (each
// write reads the other phase's face velocity, which neither writes).
__global__ void k_ghost_list(Grid g, double J, const int* __restrict__ list, const int* __restrict__ count,
                             const uint8_t* __restrict__ flags, const double* __restrict__ mdot,
                             const double2* __restrict__ nb, const uint8_t* __restrict__ vcol,
                             const double* __restrict__ hpos, const double* __restrict__ vpos, double2* u_l,
                             double2* u_v, double* ufx_l, double* ufx_v, double* ufy_l, double* ufy_v) {
    if (g.pz) J = 1.0 / g.pz[blockIdx.z].rho_l - 1.0 / g.pz[blockIdx.z].rho_v;
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    flags = zsh(flags, zo);
    mdot = zsh(mdot, zo);
    nb = zsh(nb, zo);
    vcol = zsh(vcol, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    u_l = zsh(u_l, zo);
    u_v = zsh(u_v, zo);
    ufx_l = zsh(ufx_l, zo);
    ufx_v = zsh(ufx_v, zo);
    ufy_l = zsh(ufy_l, zo);
    ufy_v = zsh(ufy_v, zo);
    long long n = 5LL * *count;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int c = list[t / 5], q = (int)(t % 5);
        int i = c % g.nx, j = c / g.nx;
        switch (q) {
            case 0: ghost_cell(g, J, c, flags, mdot, nb, u_l, u_v); break;
            case 1: ghost_face(g, J, false, i, j, flags, mdot, nb, vcol, hpos, vpos, ufx_l, ufx_v); break;
            case 2: ghost_face(g, J, false, i + 1, j, flags, mdot, nb, vcol, hpos, vpos, ufx_l, ufx_v); break;
            case 3: ghost_face(g, J, true, i, j, flags, mdot, nb, vcol, hpos, vpos, ufy_l, ufy_v); break;
            default: ghost_face(g, J, true, i, j + 1, flags, mdot, nb, vcol, hpos, vpos, ufy_l, ufy_v); break;
        }
    }
}

// ---------------------------------------------------------------------------------
// S11: momentum predictor
// ---------------------------------------------------------------------------------
// volume-fraction mixtures rho_l f + rho_v (1 - f), written as rho_v + (rho_l - rho_v) f
__device__ inline double rho_mix(const Phys& p, double vf) { return fma(p.drho, vf, p.rho_v); }
__device__ inline double mu_mix(const Phys& p, double vf) { return fma(p.dmu, vf, p.mu_v); }

// volume fraction of a face: the mean of its two cells (a boundary face takes its cell)
__device__ inline double face_vf_x(const Grid& g, const double* vf, int i, int j) {
    if (i == 0) return vf[cidx(g, 0, j)];
    if (i == g.nx) return vf[cidx(g, g.nx - 1, j)];
    return 0.5 * (vf[cidx(g, i - 1, j)] + vf[cidx(g, i, j)]);
}
__device__ inline double face_vf_y(const Grid& g, const double* vf, int i, int j) {
    if (j == 0) return vf[cidx(g, i, 0)];
    if (j == g.ny) return vf[cidx(g, i, g.ny - 1)];
    return 0.5 * (vf[cidx(g, i, j - 1)] + vf[cidx(g, i, j)]);
}

// surface-tension acceleration sigma kappa_f (H_b - H_a) / (h rho_f) on the interior face
// between cells a and b (CSF force in the well-balanced face form; H the liquid volume
// fraction): kappa_f the mean of the two cells' curvatures where both are defined, else the one
// that is, else 0; zero without surface tension
__device__ inline double st_face(const Phys& p, const Grid& g, const double* kap, const double* vf, int a, int b,
                                 double fvf) {
    if (p.sigma == 0.0 || !kap) return 0.0;
    double ka = kap[a], kb = kap[b];
    bool da = !isnan(ka), db = !isnan(kb);
    double kf = da && db ? 0.5 * (ka + kb) : (da ? ka : (db ? kb : 0.0));
    return p.sigma * kf * (vf[b] - vf[a]) / (g.h * rho_mix(p, fvf));
}

// surface tension on (sigma > 0; sigma >= 0 is validated): the bit pattern of a positive double is
// a positive integer, so the test takes no FP64 comparison
__device__ __forceinline__ bool has_sigma(const Phys& p) { return __double_as_longlong(p.sigma) > 0; }

// viscous Helmholtz operators of both velocity components in one pass (integrated form):
//   cd = h^2 rho_c / dt, dd = 2 mu_c on boundary faces where the component is Dirichlet (odd),
//   wl/wb = mean of the two cells' mu_c on the cell's left/bottom face (0 on domain faces);
// axisymmetric: each term times the radius of its cell or face, and the radial component's hoop
// term mu u_r / r^2 of the vector Laplacian (mu_c / r in cells, integrated over the ring cell).
// cd, wl and wb are the same for both components and are computed once, written to both sets.
template <bool AXI>
__global__ void k_visc_operator(Grid g, Phys p, const double* __restrict__ vf, double* __restrict__ cd0,
                                double* __restrict__ dd0, double* __restrict__ wl0, double* __restrict__ wb0,
                                double* __restrict__ cd1, double* __restrict__ dd1, double* __restrict__ wl1,
                                double* __restrict__ wb1) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    vf = zsh(vf, zo);
    cd0 = zsh(cd0, zo);
    dd0 = zsh(dd0, zo);
    wl0 = zsh(wl0, zo);
    wb0 = zsh(wb0, zo);
    cd1 = zsh(cd1, zo);
    dd1 = zsh(dd1, zo);
    wl1 = zsh(wl1, zo);
    wb1 = zsh(wb1, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    int c = cidx(g, i, j);
    double v = vf[c];
    double mu = mu_mix(p, v);
    const double mc = rad_c<AXI>(g, i);
    double cdv = g.h * g.h * rho_mix(p, v) * p.inv_dt * mc;
    double wlv = i > 0 ? 0.5 * (mu_mix(p, vf[c - 1]) + mu) * rad_fx<AXI>(g, i) : 0.0;
    double wbv = j > 0 ? 0.5 * (mu_mix(p, vf[c - g.nx]) + mu) * mc : 0.0;
    double d[2];
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        double dc = 0.0;
        if (i == 0 && vel_odd(g.bc[0], comp, 0)) dc += 2.0 * mu * rad_fx<AXI>(g, 0);
        if (i == g.nx - 1 && vel_odd(g.bc[1], comp, 0)) dc += 2.0 * mu * rad_fx<AXI>(g, g.nx);
        if (j == 0 && vel_odd(g.bc[2], comp, 1)) dc += 2.0 * mu * mc;
        if (j == g.ny - 1 && vel_odd(g.bc[3], comp, 1)) dc += 2.0 * mu * mc;
        if (AXI && comp == 0) dc += mu / mc;
        d[comp] = dc;
    }
    cd0[c] = cdv;
    wl0[c] = wlv;
    wb0[c] = wbv;
    dd0[c] = d[0];
    cd1[c] = cdv;
    wl1[c] = wlv;
    wb1[c] = wbv;
    dd1[c] = d[1];
}

// RHS of the viscous solves: cd * (WENO3-advected u_c + dt gc_c) for both phase fields (cd as
// in the viscous operator, with the cell's radius on axisymmetric grids),
// one two-RHS system per component (liquid, vapour interleaved); initial guesses = current u
// (block WX x WY threads, one cell each; the four velocity components staged per tile)
template <bool AXI>
__global__ void __launch_bounds__(WX * WY) k_mom_rhs(Grid g, Phys p, Refl rx, Refl ry, double dth,
                                                    const double* __restrict__ vf, const double2* __restrict__ u_l,
                                                    const double2* __restrict__ u_v, const double2* __restrict__ gc,
                                                    double2* __restrict__ bx, double2* __restrict__ by,
                                                    double2* __restrict__ xx, double2* __restrict__ xy) {
    zphys(g, p);
    if (g.pz) dth = g.pz[blockIdx.z].dt / g.h;
    const long long zo = zoff(g.zs);
    vf = zsh(vf, zo);
    u_l = zsh(u_l, zo);
    u_v = zsh(u_v, zo);
    gc = zsh(gc, zo);
    bx = zsh(bx, zo);
    by = zsh(by, zo);
    xx = zsh(xx, zo);
    xy = zsh(xy, zo);
    __shared__ double sh[4][WSY][WSX];
    __shared__ double d2x[4][WY][WX + 2];
    __shared__ double d2y[4][WY + 2][WX];
    int i0 = blockIdx.x * WX, j0 = blockIdx.y * WY;
    Comp F[4] = {{u_l, 0}, {u_l, 1}, {u_v, 0}, {u_v, 1}};
    Refl R[4] = {rx, ry, rx, ry};
    tile_stage<4>(F, R, g, i0, j0, sh);
    tile_d2<4>(sh, d2x, d2y);
    int tx = threadIdx.x % WX, ty = threadIdx.x / WX;
    int i = i0 + tx, j = j0 + ty;
    if (i >= g.nx || j >= g.ny) return;
    int c = cidx(g, i, j);
    double coef = g.h * g.h * rho_mix(p, vf[c]) * p.inv_dt * rad_c<AXI>(g, i);
    double2 a = gc[c];
    double2 ul = u_l[c], uv = u_v[c];
    const double hdth = 0.5 * dth;
    bx[c] = make_double2(coef * (tile_advect_d2(sh[0], d2x[0], d2y[0], tx, ty, ul, hdth) + p.dt * a.x),
                         coef * (tile_advect_d2(sh[2], d2x[2], d2y[2], tx, ty, uv, hdth) + p.dt * a.x));
    by[c] = make_double2(coef * (tile_advect_d2(sh[1], d2x[1], d2y[1], tx, ty, ul, hdth) + p.dt * a.y),
                         coef * (tile_advect_d2(sh[3], d2x[3], d2y[3], tx, ty, uv, hdth) + p.dt * a.y));
    xx[c] = make_double2(ul.x, uv.x);
    xy[c] = make_double2(ul.y, uv.y);
}

// u** = u* - dt gc (cells); u_f* = c->f mean of u** + dt g (faces; outflow faces take the
// boundary cell, wall/symmetry faces are 0)
__global__ void k_ustar(Grid g, Phys p, const double2* __restrict__ sx, const double2* __restrict__ sy,
                        const double2* __restrict__ gc, double2* __restrict__ us_l, double2* __restrict__ us_v) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    sx = zsh(sx, zo);
    sy = zsh(sy, zo);
    gc = zsh(gc, zo);
    us_l = zsh(us_l, zo);
    us_v = zsh(us_v, zo);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nx * g.ny) return;
    double2 a = gc[c], x = sx[c], y = sy[c];
    us_l[c] = make_double2(x.x - p.dt * a.x, y.x - p.dt * a.y);
    us_v[c] = make_double2(x.y - p.dt * a.x, y.y - p.dt * a.y);
}

__global__ void k_face_star(Grid g, Phys p, const double2* __restrict__ us_l, const double2* __restrict__ us_v,
                            const double* __restrict__ kap, const double* __restrict__ vf,
                            double* __restrict__ fx_l, double* __restrict__ fx_v, double* __restrict__ fy_l,
                            double* __restrict__ fy_v) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    kap = zsh(kap, zo);
    vf = zsh(vf, zo);
    us_l = zsh(us_l, zo);
    us_v = zsh(us_v, zo);
    fx_l = zsh(fx_l, zo);
    fx_v = zsh(fx_v, zo);
    fy_l = zsh(fy_l, zo);
    fy_v = zsh(fy_v, zo);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nfx = (long long)g.ny * (g.nx + 1);
    long long nfy = (long long)(g.ny + 1) * g.nx;
    if (t < nfx) {
        // faces < 2^31 (nx ny <= 2^29): 32-bit division
        int j = (int)((unsigned)t / (unsigned)(g.nx + 1)), i = (int)t - j * (g.nx + 1);
        double vl, vv;
        if (i > 0 && i < g.nx) {
            int a = cidx(g, i - 1, j), b = a + 1;
            double acc = has_sigma(p) ? p.gx + st_face(p, g, kap, vf, a, b, face_vf_x(g, vf, i, j)) : p.gx;
            vl = 0.5 * (us_l[a].x + us_l[b].x) + p.dt * acc;
            vv = 0.5 * (us_v[a].x + us_v[b].x) + p.dt * acc;
        } else {
            int s = i == 0 ? 0 : 1;
            if (g.bc[s] == BC_OUTFLOW) {
                int a = cidx(g, i == 0 ? 0 : g.nx - 1, j);
                vl = us_l[a].x + p.dt * p.gx;
                vv = us_v[a].x + p.dt * p.gx;
            } else {
                vl = vv = 0.0;
            }
        }
        fx_l[t] = vl;
        fx_v[t] = vv;
    } else if (t < nfx + nfy) {
        long long e = t - nfx;
        int j = (int)((unsigned)e / (unsigned)g.nx), i = (int)e - j * g.nx;
        double vl, vv;
        if (j > 0 && j < g.ny) {
            int a = cidx(g, i, j - 1), b = cidx(g, i, j);
            double acc = has_sigma(p) ? p.gy + st_face(p, g, kap, vf, a, b, face_vf_y(g, vf, i, j)) : p.gy;
            vl = 0.5 * (us_l[a].y + us_l[b].y) + p.dt * acc;
            vv = 0.5 * (us_v[a].y + us_v[b].y) + p.dt * acc;
        } else {
            int s = j == 0 ? 2 : 3;
            if (g.bc[s] == BC_OUTFLOW) {
                int a = cidx(g, i, j == 0 ? 0 : g.ny - 1);
                vl = us_l[a].y + p.dt * p.gy;
                vv = us_v[a].y + p.dt * p.gy;
            } else {
                vl = vv = 0.0;
            }
        }
        fy_l[e] = vl;
        fy_v[e] = vv;
    }
}

// ---------------------------------------------------------------------------------
// S12: projection
// ---------------------------------------------------------------------------------

// Poisson operator: wl/wb = dt / rho_f (interior faces), dd = 2 dt / rho_f on outflow faces,
// b = -h * (undivided divergence of the face field of the cell's phase); x0 = p
// length (grid units) of the segments of a cut cell, from its segment table and the markers;
// on axisymmetric grids each segment's length times the radius (cells) of its midpoint
template <bool AXI>
__device__ inline double segments_length(const Grid& g, const uint16_t* cseg, const double* hpos,
                                         const double* vpos, int i, int j) {
    uint16_t code = cseg[cidx(g, i, j)];
    int ns = code & 3;
    double L = 0.0;
    for (int q = 0; q < ns; ++q) {
        int k[2] = {(code >> (2 + 4 * q)) & 3, (code >> (4 + 4 * q)) & 3};
        double2 m[2];
        for (int e = 0; e < 2; ++e) {
            switch (k[e]) {
                case 0: m[e] = make_double2(hpos[hidx(g, i, j)], 0.0); break;
                case 1: m[e] = make_double2(1.0, vpos[veidx(g, i + 1, j)]); break;
                case 2: m[e] = make_double2(hpos[hidx(g, i, j + 1)], 1.0); break;
                default: m[e] = make_double2(0.0, vpos[veidx(g, i, j)]); break;
            }
        }
        double dx = m[1].x - m[0].x, dy = m[1].y - m[0].y;
        double l = sqrt(dx * dx + dy * dy);
        L += AXI ? l * (g.r0 + (double)i + 0.5 * (m[0].x + m[1].x)) : l;
    }
    return L;
}

// ghost-fluid Poisson operator (face weights dt / rho_f, outflow faces Dirichlet p = 0) and its
// right-hand side -h div u_f* of each cell's phase; in the one-fluid variant the single field's
// divergence plus h^2 S_pc = mdot S_Gamma (1/rho_v - 1/rho_l) in the cut cells; axisymmetric:
// face weights and face fluxes times the face's radius, S_Gamma times the segment's radius
template <bool AXI>
__global__ void k_poisson_operator(Grid g, Phys p, const double* __restrict__ vf, const uint8_t* __restrict__ flags,
                                   const uint16_t* __restrict__ cseg, const double* __restrict__ hpos,
                                   const double* __restrict__ vpos, const double* __restrict__ mdot,
                                   const double* __restrict__ fx_l, const double* __restrict__ fx_v,
                                   const double* __restrict__ fy_l, const double* __restrict__ fy_v,
                                   double* __restrict__ cd, double* __restrict__ dd, double* __restrict__ wl,
                                   double* __restrict__ wb, double* __restrict__ b) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    vf = zsh(vf, zo);
    flags = zsh(flags, zo);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    mdot = zsh(mdot, zo);
    fx_l = zsh(fx_l, zo);
    fx_v = zsh(fx_v, zo);
    fy_l = zsh(fy_l, zo);
    fy_v = zsh(fy_v, zo);
    cd = zsh(cd, zo);
    dd = zsh(dd, zo);
    wl = zsh(wl, zo);
    wb = zsh(wb, zo);
    b = zsh(b, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    int c = cidx(g, i, j);
    cd[c] = 0.0;
    const double mc = rad_c<AXI>(g, i), ml = rad_fx<AXI>(g, i), mr = rad_fx<AXI>(g, i + 1);
    double d = 0.0;
    // dt / rho_f through recip64 (within an ulp of the division, a third of its FP64 work)
    if (i == 0 && g.bc[0] == BC_OUTFLOW) d += 2.0 * p.dt * recip64(rho_mix(p, face_vf_x(g, vf, 0, j))) * ml;
    if (i == g.nx - 1 && g.bc[1] == BC_OUTFLOW)
        d += 2.0 * p.dt * recip64(rho_mix(p, face_vf_x(g, vf, g.nx, j))) * mr;
    if (j == 0 && g.bc[2] == BC_OUTFLOW) d += 2.0 * p.dt * recip64(rho_mix(p, face_vf_y(g, vf, i, 0))) * mc;
    if (j == g.ny - 1 && g.bc[3] == BC_OUTFLOW)
        d += 2.0 * p.dt * recip64(rho_mix(p, face_vf_y(g, vf, i, g.ny))) * mc;
    dd[c] = d;
    wl[c] = i > 0 ? p.dt * recip64(rho_mix(p, face_vf_x(g, vf, i, j))) * ml : 0.0;
    wb[c] = j > 0 ? p.dt * recip64(rho_mix(p, face_vf_y(g, vf, i, j))) * mc : 0.0;
    const double* fx = (flags[c] & F_CCOL) ? fx_l : fx_v;
    const double* fy = (flags[c] & F_CCOL) ? fy_l : fy_v;
    double div = (mr * fx[veidx(g, i + 1, j)] - ml * fx[veidx(g, i, j)]) +
                 mc * (fy[hidx(g, i, j + 1)] - fy[hidx(g, i, j)]);
    double rhs = -g.h * div;
    if (p.one_fluid && (flags[c] & F_CUT))
        rhs += mdot[c] * segments_length<AXI>(g, cseg, hpos, vpos, i, j) * g.h * (1.0 / p.rho_v - 1.0 / p.rho_l);
    b[c] = rhs;
}


// the pressure part -grad_f p / rho_f of the face acceleration on a face the projection acts on
// (interior, or an outflow boundary face with p = 0 on it): on interior faces with the Poisson
// face weight w = dt / rho_f given (wl != null) as -dp w / (h dt), else through recip64
__device__ inline double pgrad_x(const Grid& g, const Phys& p, const double* P, const double* vf, const double* wl,
                                 int i, int j) {
    if (i > 0 && i < g.nx) {
        double dP = P[cidx(g, i, j)] - P[cidx(g, i - 1, j)];
        if (wl) return -(dP * wl[cidx(g, i, j)] * (g.inv_h * p.inv_dt));
        return -(dP * recip64(g.h * rho_mix(p, face_vf_x(g, vf, i, j))));
    }
    double r = rho_mix(p, face_vf_x(g, vf, i, j));
    if (i == 0) return -((2.0 * P[cidx(g, 0, j)]) / (g.h * r));
    return -((-2.0 * P[cidx(g, g.nx - 1, j)]) / (g.h * r));
}
__device__ inline double pgrad_y(const Grid& g, const Phys& p, const double* P, const double* vf, const double* wb,
                                 int i, int j) {
    if (j > 0 && j < g.ny) {
        double dP = P[cidx(g, i, j)] - P[cidx(g, i, j - 1)];
        if (wb) return -(dP * wb[cidx(g, i, j)] * (g.inv_h * p.inv_dt));
        return -(dP * recip64(g.h * rho_mix(p, face_vf_y(g, vf, i, j))));
    }
    double r = rho_mix(p, face_vf_y(g, vf, i, j));
    if (j == 0) return -((2.0 * P[cidx(g, i, 0)]) / (g.h * r));
    return -((-2.0 * P[cidx(g, i, g.ny - 1)]) / (g.h * r));
}

// face accelerations a_f = g - grad_f p / rho_f (+ the surface-tension term), stored in ax/ay
// (0 on walls and symmetry planes); with fx_l != null also the face update of discretization
// equation 4 for both phase fields, u_f^{n+1} = u_f* + dt (a_f - g - surface tension) =
// u_f* - dt grad_f p / rho_f (u_f* carries dt (g + surface tension) already)
__global__ void k_face_accel(Grid g, Phys p, const double* __restrict__ P, const double* __restrict__ vf,
                             const double* __restrict__ kap, const double* __restrict__ wl_p,
                             const double* __restrict__ wb_p, double* __restrict__ ax, double* __restrict__ ay,
                             double* fx_l, double* fx_v, double* fy_l, double* fy_v) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    P = zsh(P, zo);
    kap = zsh(kap, zo);
    vf = zsh(vf, zo);
    wl_p = zsh(wl_p, zo);
    wb_p = zsh(wb_p, zo);
    ax = zsh(ax, zo);
    ay = zsh(ay, zo);
    fx_l = zsh(fx_l, zo);
    fx_v = zsh(fx_v, zo);
    fy_l = zsh(fy_l, zo);
    fy_v = zsh(fy_v, zo);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nfx = (long long)g.ny * (g.nx + 1);
    long long nfy = (long long)(g.ny + 1) * g.nx;
    if (t < nfx) {
        // faces < 2^31 (nx ny <= 2^29): 32-bit division
        int j = (int)((unsigned)t / (unsigned)(g.nx + 1)), i = (int)t - j * (g.nx + 1);
        bool bnd = i == 0 || i == g.nx;
        if (bnd && g.bc[i == 0 ? 0 : 1] != BC_OUTFLOW) {
            ax[t] = 0.0;
            if (fx_l) { fx_l[t] = 0.0; fx_v[t] = 0.0; }
            return;
        }
        double G = pgrad_x(g, p, P, vf, wl_p, i, j);
        double a = p.gx + G;
        if (!bnd && has_sigma(p))
            a += st_face(p, g, kap, vf, cidx(g, i - 1, j), cidx(g, i, j), face_vf_x(g, vf, i, j));
        ax[t] = a;
        if (!fx_l) return;
        double corr = p.dt * G;
        fx_l[t] += corr;
        fx_v[t] += corr;
    } else if (t < nfx + nfy) {
        long long e = t - nfx;
        int j = (int)((unsigned)e / (unsigned)g.nx), i = (int)e - j * g.nx;
        bool bnd = j == 0 || j == g.ny;
        if (bnd && g.bc[j == 0 ? 2 : 3] != BC_OUTFLOW) {
            ay[e] = 0.0;
            if (fx_l) { fy_l[e] = 0.0; fy_v[e] = 0.0; }
            return;
        }
        double G = pgrad_y(g, p, P, vf, wb_p, i, j);
        double a = p.gy + G;
        if (!bnd && has_sigma(p))
            a += st_face(p, g, kap, vf, cidx(g, i, j - 1), cidx(g, i, j), face_vf_y(g, vf, i, j));
        ay[e] = a;
        if (!fx_l) return;
        double corr = p.dt * G;
        fy_l[e] += corr;
        fy_v[e] += corr;
    }
}

// gc = f->c mean of the face accelerations; optionally u^{n+1} = u** + dt gc (Eq. 15)
__global__ void k_project_cells(Grid g, Phys p, const double* __restrict__ axf, const double* __restrict__ ayf,
                                double2* __restrict__ gc, const double2* __restrict__ us_l,
                                const double2* __restrict__ us_v, double2* __restrict__ u_l,
                                double2* __restrict__ u_v) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    axf = zsh(axf, zo);
    ayf = zsh(ayf, zo);
    gc = zsh(gc, zo);
    us_l = zsh(us_l, zo);
    us_v = zsh(us_v, zo);
    u_l = zsh(u_l, zo);
    u_v = zsh(u_v, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    int c = cidx(g, i, j);
    int fx = j * (g.nx + 1) + i;
    double ax = 0.5 * (axf[fx] + axf[fx + 1]);
    double ay = 0.5 * (ayf[c] + ayf[c + g.nx]);
    gc[c] = make_double2(ax, ay);
    if (us_l) {
        double2 a = us_l[c], b = us_v[c];
        u_l[c] = make_double2(a.x + p.dt * ax, a.y + p.dt * ay);
        u_v[c] = make_double2(b.x + p.dt * ax, b.y + p.dt * ay);
    }
}

// ---------------------------------------------------------------------------------
// S13: diagnostics (block partial sums, last block finalises in a fixed order)
// ---------------------------------------------------------------------------------
__device__ inline double block_sum(double v, double* sh) {
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
    return r;   // valid in thread 0
}

constexpr int NDIAG_SUMS = 8;

// S13 and the film-boiling quantities of Sec. 3.7, one reduction over the cells:
//   s0 vapour area, s1 sum mdot S_Gamma, s2 sum rho_c, s3 outlet mass flux (mass-with-outflow
//   equation), s4 cut cells, s5 vapour volume flux through the outflow faces ((1 - H) u_f . n
//   with the face velocity of the boundary cell's phase), s6 wall heat flux 2 (T_w - T_i) / h
//   summed over the faces of fixed-temperature walls, s7 the number of those faces.
// Axisymmetric grids weight every cell, face and segment by its radius and report the ring's
// volumes, masses and fluxes (the wall Nusselt number stays the plain mean over the faces).
// out: t, vapour volume, dV expected from mdot, M_d, outlet mass, cut cells, vapour volume out,
// wall Nusselt number (l / (T_w - T_sat)) * mean wall flux, l = sqrt(sigma / (|drho| |g|)) when
// sigma and g are nonzero, else 1.
template <bool AXI>
__global__ void k_diagnostics(Grid g, Phys p, const double* __restrict__ vf, const uint16_t* __restrict__ cseg,
                              const double* __restrict__ hpos, const double* __restrict__ vpos,
                              const double* __restrict__ mdot, const uint8_t* __restrict__ flags,
                              const double* __restrict__ fx_l, const double* __restrict__ fx_v,
                              const double* __restrict__ fy_l, const double* __restrict__ fy_v,
                              const double* __restrict__ T_l, const double* __restrict__ T_v,
                              double* __restrict__ partial, unsigned* __restrict__ ticket, double* __restrict__ clock,
                              double* __restrict__ out, int vb) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    vf = zsh(vf, zo);
    T_l = zsh(T_l, zo);
    T_v = zsh(T_v, zo);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    mdot = zsh(mdot, zo);
    flags = zsh(flags, zo);
    fx_l = zsh(fx_l, zo);
    fx_v = zsh(fx_v, zo);
    fy_l = zsh(fy_l, zo);
    fy_v = zsh(fy_v, zo);
    partial = zsh(partial, zo);
    ticket = zsh(ticket, zo);
    clock = zsh(clock, zo);
    out = zsh(out, zo);
    __shared__ double sh[32];
    __shared__ bool lastblk;
    // virtual blocks: the reduction is that of a vb-block launch whatever the launch's size
    // (blocks take the virtual blocks b, b + gridDim.x, ...), as in the solver's reductions
    int N = g.nx * g.ny;
    double tot[NDIAG_SUMS];
    for (int vblk = blockIdx.x; vblk < vb; vblk += gridDim.x) {
        double s[NDIAG_SUMS] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (CellWalk cw(g.nx, vblk, vb); cw.c < N; cw.next()) {
            int c = cw.c, i = cw.i, j = cw.j;
            double v = vf[c];
            double rc = rho_mix(p, v);
            const double mc = rad_c<AXI>(g, i);
            s[0] += (1.0 - v) * mc;
            s[2] += rc * mc;
            uint16_t code = cseg[c];
            int ns = code & 3;
            if (ns) {
                s[4] += 1.0;
                for (int q = 0; q < ns; ++q) {
                    int kP = (code >> (2 + 4 * q)) & 3, kQ = (code >> (4 + 4 * q)) & 3;
                    auto ml = [&](int k) -> double2 {
                        switch (k) {
                            case 0: return make_double2(hpos[hidx(g, i, j)], 0.0);
                            case 1: return make_double2(1.0, vpos[veidx(g, i + 1, j)]);
                            case 2: return make_double2(hpos[hidx(g, i, j + 1)], 1.0);
                            default: return make_double2(0.0, vpos[veidx(g, i, j)]);
                        }
                    };
                    double2 P = ml(kP), Q = ml(kQ);
                    double dx = Q.x - P.x, dy = Q.y - P.y;
                    double ms = AXI ? g.r0 + (double)i + 0.5 * (P.x + Q.x) : 1.0;   // the segment's radius
                    s[1] += mdot[c] * sqrt(dx * dx + dy * dy) * g.h * ms;
                }
            }
            bool liq = flags[c] & F_CCOL;
            if (i == 0 || i == g.nx - 1 || j == 0 || j == g.ny - 1) {
                // boundary faces of this cell: outflow (mass and vapour volume) and fixed-T walls
                for (int sd = 0; sd < 4; ++sd) {
                    bool on = sd == 0 ? i == 0 : sd == 1 ? i == g.nx - 1 : sd == 2 ? j == 0 : j == g.ny - 1;
                    if (!on) continue;
                    if (g.bc[sd] == BC_OUTFLOW) {
                        double u = sd < 2 ? (liq ? fx_l : fx_v)[veidx(g, sd == 0 ? 0 : g.nx, j)]
                                          : (liq ? fy_l : fy_v)[hidx(g, i, sd == 2 ? 0 : g.ny)];
                        double un = ((sd == 0 || sd == 2) ? -u : u) *
                                    (sd == 0 ? rad_fx<AXI>(g, 0) : (sd == 1 ? rad_fx<AXI>(g, g.nx) : mc));
                        s[3] += rc * un;
                        s[5] += (1.0 - v) * un;
                    }
                    if (g.bc[sd] == BC_WALL && g.Tfix[sd]) {
                        s[6] += 2.0 * (g.Tw[sd] - (liq ? T_l : T_v)[c]) * g.inv_h;
                        s[7] += 1.0;
                    }
                }
            }
        }
        for (int q = 0; q < NDIAG_SUMS; ++q) {
            double r = block_sum(s[q], sh);
            if (threadIdx.x == 0) partial[q * vb + vblk] = r;
        }
    }
    __threadfence();
    if (threadIdx.x == 0) lastblk = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!lastblk) return;
    __threadfence();
    for (int q = 0; q < NDIAG_SUMS; ++q) {
        double v = 0.0;
        for (int b = threadIdx.x; b < vb; b += blockDim.x) v += partial[q * vb + b];
        double r = block_sum(v, sh);
        if (threadIdx.x == 0) tot[q] = r;
    }
    if (threadIdx.x == 0) {
        double h2 = g.h * g.h;
        const double ring = AXI ? 6.283185307179586 * g.h : 1.0;   // 2 pi r = 2 pi h times the radius in cells
        clock[0] += p.dt;
        clock[1] += 1.0;
        out[0] = clock[0];
        out[1] = tot[0] * h2 * ring;
        out[2] = tot[1] * p.dt / p.rho_v * ring;
        out[3] = tot[2] * h2 * ring;
        out[4] = tot[3] * g.h * p.dt * ring;
        out[5] = tot[4];
        out[6] = tot[5] * g.h * p.dt * ring;
        double nu = 0.0;
        if (tot[7] > 0.0) {
            double Tw = 0.0;
            for (int sd = 3; sd >= 0; --sd)
                if (g.bc[sd] == BC_WALL && g.Tfix[sd]) Tw = g.Tw[sd];   // the first fixed-T wall
            double gm = sqrt(p.gx * p.gx + p.gy * p.gy), dr = fabs(p.rho_l - p.rho_v);
            double ell = (has_sigma(p) && gm > 0.0 && dr > 0.0) ? sqrt(p.sigma / (dr * gm)) : 1.0;
            if (Tw != p.T_sat) nu = ell / (Tw - p.T_sat) * tot[6] / tot[7];
        }
        out[7] = nu;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------

void launch_advect_T(const Grid& g, const Phys& p, const uint8_t* flags, const double* T_l, const double* T_v,
                     const double2* u_l, const double2* u_v, double* Ts_l, double* Ts_v, cudaStream_t st) {
    k_advect_T<<<dim3(div_up(g.nx, WX), div_up(g.ny, WY), g.nz), WX * WY, 0, st>>>(
        g, temperature_refl(g), p.dt / g.h, flags, T_l, T_v, u_l, u_v, Ts_l, Ts_v);
}

void launch_compact(const Grid& g, const uint8_t* flags, int N, uint8_t mask, int* list, int* count, int* idxmap,
                    cudaStream_t st) {
    if (g.nz > 1)   // the count word of every instance of the batch (one stride apart)
        cudaMemset2DAsync(count, (size_t)g.zs, 0, sizeof(int), g.nz, st);
    else
        cudaMemsetAsync(count, 0, sizeof(int), st);
    k_compact<<<grid1(N, 256, g.nz), 256, 0, st>>>(flags, N, mask, list, count, idxmap, g.zs);
}

// blocks of a band sweep: the band holds at most every cell; four per SM at most
static int extend_grid_blocks(const Grid& g) {
    int n = div_up((long long)g.nx * g.ny, 256);
    return n < 4 * 152 ? n : 4 * 152;
}

void launch_split_T(const Grid& g, const uint8_t* flags, const double* x, const double* Ts_l, const double* Ts_v,
                    double* T_l, double* T_v, cudaStream_t st) {
    int N = g.nx * g.ny;
    k_split_T<<<grid1(N, 256, g.nz), 256, 0, st>>>(N, flags, x, Ts_l, Ts_v, T_l, T_v, g.zs);
}

// every sweep of one extension in one CTA per instance (grid z): a band of a few thousand cells
// takes a few microseconds per sweep, less than a launch; __syncthreads() orders the sweeps
// (each reads the previous one's values, written to global memory by other threads of the CTA)
constexpr int EXT_BLOCK_THREADS = 1024;
__global__ void __launch_bounds__(EXT_BLOCK_THREADS)
k_extend_block(Grid g, int mode, int iters, const int* __restrict__ list, const int* __restrict__ count,
               const uint8_t* __restrict__ flags, const int* __restrict__ idxmap, const double2* __restrict__ nb,
               double* f0, double* va0, double* vb0, double* f1, double* va1, double* vb1) {
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    flags = zsh(flags, zo);
    idxmap = zsh(idxmap, zo);
    nb = zsh(nb, zo);
    f0 = zsh(f0, zo);
    va0 = zsh(va0, zo);
    vb0 = zsh(vb0, zo);
    f1 = zsh(f1, zo);
    va1 = zsh(va1, zo);
    vb1 = zsh(vb1, zo);
    int n = *count;
    for (int it = 0; it < iters; ++it) {
        bool odd = it & 1;
        for (int k = threadIdx.x; k < n; k += blockDim.x)
            extend_entry(g, mode, it, it == iters - 1, k, list, flags, idxmap, nb, f0, odd ? vb0 : va0,
                         odd ? va0 : vb0, f1, odd ? vb1 : va1, odd ? va1 : vb1);
        __syncthreads();
    }
}

void launch_extend(const Grid& g, int mode, int iters, const int* list, const int* count, const uint8_t* flags,
                   const int* idxmap, const double2* nb, double* f, double* va, double* vb, cudaStream_t st) {
    if (g.ext_block) {
        k_extend_block<<<dim3(1, 1, g.nz), EXT_BLOCK_THREADS, 0, st>>>(g, mode, iters, list, count, flags, idxmap, nb,
                                                                      f, va, vb, nullptr, nullptr, nullptr);
        return;
    }
    int nb_ = extend_grid_blocks(g);
    for (int it = 0; it < iters; ++it) {
        const double* cur = (it & 1) ? vb : va;
        double* nxt = (it & 1) ? va : vb;
        k_extend<<<dim3(nb_, 1, g.nz), 256, 0, st>>>(g, mode, it, it == iters - 1, list, count, flags, idxmap, nb,
                                                     f, cur, nxt, nullptr, nullptr, nullptr);
    }
}

void launch_extend_T(const Grid& g, int iters, const int* list, const int* count, const uint8_t* flags,
                     const int* idxmap, const double2* nb, double* T_l, double* T_v, double* const ext[4],
                     cudaStream_t st) {
    if (g.ext_block) {
        k_extend_block<<<dim3(1, 1, g.nz), EXT_BLOCK_THREADS, 0, st>>>(g, 3, iters, list, count, flags, idxmap, nb,
                                                                      T_l, ext[0], ext[1], T_v, ext[2], ext[3]);
        return;
    }
    int nb_ = extend_grid_blocks(g);
    for (int it = 0; it < iters; ++it) {
        int a = it & 1;
        k_extend<<<dim3(nb_, 1, g.nz), 256, 0, st>>>(g, 3, it, it == iters - 1, list, count, flags, idxmap, nb,
                                                     T_l, ext[a], ext[1 - a], T_v, ext[2 + a], ext[3 - a]);
    }
}

void launch_ghost_velocity(const Grid& g, const Phys& p, const int* band_list, const int* band_count,
                           const uint8_t* flags, const double* mdot, const double2* nb, const uint8_t* vcol,
                           const double* hpos, const double* vpos, double2* u_l, double2* u_v, double* ufx_l,
                           double* ufx_v, double* ufy_l, double* ufy_v, cudaStream_t st) {
    double J = 1.0 / p.rho_l - 1.0 / p.rho_v;
    // five items per band cell; the band is O(sqrt N): blocks as for the other list kernels
    long long nbk = div_up(5LL * 8 * (g.nx + g.ny), 256);
    nbk = nbk < 4 ? 4 : (nbk > 4 * 152 ? 4 * 152 : nbk);
    if (g.nz > 1) {   // a batch: about two blocks per SM slot shared among its instances
        long long per = (2LL * 4 * 152) / g.nz;
        nbk = nbk < per ? nbk : (per < 1 ? 1 : per);
    }
    int blocks = (int)nbk;
    k_ghost_list<<<dim3(blocks, 1, g.nz), 256, 0, st>>>(g, J, band_list, band_count, flags, mdot, nb, vcol, hpos,
                                                        vpos, u_l, u_v, ufx_l, ufx_v, ufy_l, ufy_v);
}

void launch_visc_operator(const Grid& g, const Phys& p, const double* vf, double* cd0, double* dd0, double* wl0,
                          double* wb0, double* cd1, double* dd1, double* wl1, double* wb1, cudaStream_t st) {
    auto k = g.axi ? k_visc_operator<true> : k_visc_operator<false>;
    k<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, p, vf, cd0, dd0, wl0, wb0, cd1, dd1, wl1, wb1);
}

void launch_mom_rhs(const Grid& g, const Phys& p, const double* vf, const double2* u_l, const double2* u_v,
                    const double2* gc, double2* bx, double2* by, double2* xx, double2* xy, cudaStream_t st) {
    auto k = g.axi ? k_mom_rhs<true> : k_mom_rhs<false>;
    k<<<dim3(div_up(g.nx, WX), div_up(g.ny, WY), g.nz), WX * WY, 0, st>>>(
        g, p, velocity_refl(g, 0), velocity_refl(g, 1), p.dt / g.h, vf, u_l, u_v, gc, bx, by, xx, xy);
}

void launch_ustar(const Grid& g, const Phys& p, const double2* sx, const double2* sy, const double2* gc,
                  const double* kap, const double* vf, double2* us_l, double2* us_v, double* fx_l, double* fx_v,
                  double* fy_l, double* fy_v, cudaStream_t st) {
    int N = g.nx * g.ny;
    k_ustar<<<grid1(N, 256, g.nz), 256, 0, st>>>(g, p, sx, sy, gc, us_l, us_v);
    long long nf = (long long)g.ny * (g.nx + 1) + (long long)(g.ny + 1) * g.nx;
    k_face_star<<<grid1(nf, 256, g.nz), 256, 0, st>>>(g, p, us_l, us_v, kap, vf, fx_l, fx_v, fy_l, fy_v);
}

void launch_poisson_operator(const Grid& g, const Phys& p, const double* vf, const uint8_t* flags,
                             const uint16_t* cseg, const double* hpos, const double* vpos, const double* mdot,
                             const double* fx_l, const double* fx_v, const double* fy_l, const double* fy_v,
                             double* cd, double* dd, double* wl, double* wb, double* b, cudaStream_t st) {
    auto k = g.axi ? k_poisson_operator<true> : k_poisson_operator<false>;
    k<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, p, vf, flags, cseg, hpos, vpos, mdot, fx_l, fx_v, fy_l,
                                                          fy_v, cd, dd, wl, wb, b);
}

void launch_project(const Grid& g, const Phys& p, const double* P, const double* vf, const double* kap,
                    const double* wl_p, const double* wb_p, double* ax, double* ay, double* fx_l, double* fx_v,
                    double* fy_l, double* fy_v, double2* gc, const double2* us_l, const double2* us_v, double2* u_l,
                    double2* u_v, cudaStream_t st) {
    long long nf = (long long)g.ny * (g.nx + 1) + (long long)(g.ny + 1) * g.nx;
    if (g.axi) wl_p = wb_p = nullptr;   // those weights carry the faces' radii: use dt / rho_f itself
    k_face_accel<<<grid1(nf, 256, g.nz), 256, 0, st>>>(g, p, P, vf, kap, wl_p, wb_p, ax, ay, fx_l, fx_v, fy_l, fy_v);
    k_project_cells<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, p, ax, ay, gc, us_l, us_v, u_l, u_v);
}

// blocks of the diagnostics reduction: four per SM at most (the partial sums hold 5 x 1638),
// fewer for small grids
int diag_blocks(const Grid& g) {
    int n = div_up((long long)g.nx * g.ny, 1024);
    return n < 4 * 152 ? n : 4 * 152;
}

void launch_diagnostics(const Grid& g, const Phys& p, const double* vf, const uint16_t* cseg, const double* hpos,
                        const double* vpos, const double* mdot, const uint8_t* flags, const double* fx_l,
                        const double* fx_v, const double* fy_l, const double* fy_v, const double* T_l,
                        const double* T_v, double* partial, unsigned* ticket, double* clock, double* out,
                        cudaStream_t st) {
    auto k = g.axi ? k_diagnostics<true> : k_diagnostics<false>;
    // a batch: about two blocks per SM slot in total, each taking several virtual blocks
    int vb = diag_blocks(g), per = (2 * 4 * 152) / g.nz;
    int lb = g.nz <= 1 ? vb : (vb < per ? vb : (per < 1 ? 1 : per));
    k<<<dim3(lb, 1, g.nz), 256, 0, st>>>(g, p, vf, cseg, hpos, vpos, mdot, flags, fx_l, fx_v, fy_l, fy_v, T_l, T_v,
                                         partial, ticket, clock, out, vb);
}

}  // namespace ebit
