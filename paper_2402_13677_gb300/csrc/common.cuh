// Shared definitions of the EBIT phase-change step on sm_103a.
//
// Layout (row-major, x fastest):
//   cells    c = j*nx + i                       (ny x nx)
//   vertices v = j*(nx+1) + i                   ((ny+1) x (nx+1))
//   h-edges  (horizontal, on line y=j, between vertices i and i+1): j*nx + i
//   v-edges  (vertical,   on line x=i, between vertices j and j+1): j*(nx+1) + i
//   x-faces  = v-edges, y-faces = h-edges (a face is the edge it lies on)
// Grid units: vertex (i, j) sits at (i, j); cell centres at (i + 0.5, j + 0.5).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ebit {

constexpr double FMIN = 1e-9;   // marker fractions live in [FMIN, 1 - FMIN]
constexpr int BC_WALL = 0, BC_OUTFLOW = 1, BC_SYMMETRY = 2;

// per-cell flag byte
constexpr uint8_t F_CCOL = 1;   // centre colour f_C (1 liquid)
constexpr uint8_t F_BAND = 2;   // narrow band
constexpr uint8_t F_CUT = 4;    // cell holds interface segments

struct Phys {
    double rho_l, rho_v, mu_l, mu_v, lam_l, lam_v, cp_l, cp_v;
    double T_sat, h_lg, gx, gy;
    double sigma;     // surface tension coefficient
    double dt, theta_min;
    int extend_iters, energy;
    double mdot_fixed;
    int one_fluid;    // one velocity field and the phase-change source (no ghost velocities)
    // derived on the host (phys_derive) whenever the above change: 1 / dt and the liquid-minus-
    // vapour differences of density and viscosity (mixtures as one fused multiply-add)
    double inv_dt, drho, dmu;
};

__host__ inline void phys_derive(Phys& p) {
    p.inv_dt = p.dt > 0.0 ? 1.0 / p.dt : 0.0;
    p.drho = p.rho_l - p.rho_v;
    p.dmu = p.mu_l - p.mu_v;
}

// Grid of one instance, or of a batch of instances that share it: a batched launch runs
// instance z = blockIdx.z (of nz) on the arrays at byte offset z * zs from instance 0's, with
// the properties pz[z] (null pz: the Phys passed by value)
struct Grid {
    int nx, ny;
    double h, x0, y0;
    double inv_h;     // 1 / h
    int bc[4];        // left, right, bottom, top
    int Tfix[4];
    double Tw[4];
    int ext_block;    // narrow-band extension: every Jacobi sweep in one CTA per instance (else
                      // one launch per sweep)
    int axi;          // axisymmetric (r, z): x is the radius
    double r0;        // x0 / h, the radius of the left domain side in cells
    int nz;                  // instances in the launch (1 unless batched)
    long long zs;            // byte stride between consecutive instances' arenas
    const Phys* pz;          // device array of the instances' properties, or null
};

// radius in cells of the centre of cell column i (and of its y-faces) and of the x-face on its
// left: every integrated balance of an axisymmetric grid carries the radius of the cell, face or
// segment it lives on (2 pi r times the planar measure, 2 pi h factored out); 1 on planar grids.
// The kernels that use them are instantiated for AXI = g.axi, so that a planar grid spends no
// FP64 instruction on the metric (the FP64 rate bounds those kernels).
template <bool AXI>
__host__ __device__ inline double rad_c(const Grid& g, int i) { return AXI ? g.r0 + (double)i + 0.5 : 1.0; }
template <bool AXI>
__host__ __device__ inline double rad_fx(const Grid& g, int i) { return AXI ? g.r0 + (double)i : 1.0; }

// byte offset of this block's instance, and a pointer moved to it
__device__ __forceinline__ long long zoff(long long zs) { return (long long)blockIdx.z * zs; }
template <class P>
__device__ __forceinline__ P* zsh(P* p, long long off) {
    return p ? reinterpret_cast<P*>(reinterpret_cast<uintptr_t>(p) + off) : p;
}
__device__ __forceinline__ void zphys(const Grid& g, Phys& p) {
    if (g.pz) p = g.pz[blockIdx.z];
}

// grid-stride walk over the cells of an nx-wide grid that keeps (i, j) without a division per
// step
struct CellWalk {
    int c, i, j, stride, di, dj, nx;
    __device__ CellWalk(int nx_) : CellWalk(nx_, blockIdx.x, gridDim.x) {}
    // the walk of block v of an nv-block grid (a virtual block of a reduction kernel)
    __device__ CellWalk(int nx_, int v, int nv) : nx(nx_) {
        c = v * blockDim.x + threadIdx.x;
        stride = nv * blockDim.x;
        i = c % nx;
        j = c / nx;
        di = stride % nx;
        dj = stride / nx;
    }
    __device__ void next() {
        c += stride;
        i += di;
        j += dj;
        if (i >= nx) { i -= nx; ++j; }
    }
};

__host__ __device__ inline int cidx(const Grid& g, int i, int j) { return j * g.nx + i; }
__host__ __device__ inline int vidx(const Grid& g, int i, int j) { return j * (g.nx + 1) + i; }
__host__ __device__ inline int hidx(const Grid& g, int i, int j) { return j * g.nx + i; }
__host__ __device__ inline int veidx(const Grid& g, int i, int j) { return j * (g.nx + 1) + i; }

// Reflection sign of velocity component comp across the boundary on `side`
// (normal component odd at walls and symmetry planes, tangential odd at no-slip walls,
// everything even at outflow).
__host__ __device__ inline bool vel_odd(int kind, int comp, int axis) {
    if (comp == axis) return kind != BC_OUTFLOW;
    return kind == BC_WALL;
}

// cell value of a double2 field with one layer of reflected ghost cells
__device__ inline double cell_vel(const double2* F, const Grid& g, int comp, int i, int j) {
    bool neg = false;
    if (i < 0) { i = 0; neg ^= vel_odd(g.bc[0], comp, 0); }
    else if (i >= g.nx) { i = g.nx - 1; neg ^= vel_odd(g.bc[1], comp, 0); }
    if (j < 0) { j = 0; neg ^= vel_odd(g.bc[2], comp, 1); }
    else if (j >= g.ny) { j = g.ny - 1; neg ^= vel_odd(g.bc[3], comp, 1); }
    double2 v = F[cidx(g, i, j)];
    double s = comp == 0 ? v.x : v.y;
    return neg ? -s : s;
}

// Conversions between FP64 and FP32 on the integer pipes.  The FP64 pipe of this GPU issues at
// a small fraction of the FP32 rate and also performs the hardware conversions, so kernels that
// convert every element (building the FP32 multigrid operators, scaling the refinement residual
// to FP32, applying the FP32 correction to the FP64 solution) were bound by it.  Both follow
// IEEE 754: binary64 -> binary32 rounds to nearest, ties to even (subnormal results, overflow
// to infinity, signed zeros, NaNs kept quiet), binary32 -> binary64 is exact.  Every case is
// integer arithmetic: a fallback to the hardware conversion would be compiled to a predicated
// FP64 instruction issued for every element.
// d2f_rn2(v, k) rounds v 2^k (exact scaling by a power of two, no intermediate binary64) to
// binary32; v a binary64 subnormal gives zero.
__device__ __forceinline__ float d2f_rn2(double v, int k) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    unsigned sign = (unsigned)(b >> 63) << 31;
    unsigned e0 = (unsigned)(b >> 52) & 0x7ffu;           // biased binary64 exponent
    unsigned long long m = b & 0x000fffffffffffffull;
    // exponent of v 2^k (held in range: inputs that are zero, subnormal, infinite or NaN keep
    // their class below)
    int es = (int)e0 + k;
    unsigned e = (e0 == 0u || e0 == 0x7ffu) ? e0 : (unsigned)(es < 1 ? 1 : (es > 2046 ? 2046 : es));
    unsigned f;
    if (e0 != 0u && e0 != 0x7ffu && es != (int)e) {        // scaled beyond the binary64 range
        f = es > 0 ? 0x7f800000u : 0u;
    } else if (e - 897u <= 253u) {                        // normal binary32 result (before rounding)
        unsigned keep = (unsigned)(m >> 29), rest = (unsigned)(m & 0x1fffffffu);
        f = ((e - 896u) << 23) | keep;                    // a rounding carry moves into the exponent
        f += (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    } else if (e == 0x7ffu) {                             // infinity, NaN (made quiet)
        f = 0x7f800000u | (m ? 0x400000u | (unsigned)(m >> 29) : 0u);
    } else if (e > 1150u) {                               // beyond the binary32 range
        f = 0x7f800000u;
    } else {                                              // binary32 subnormal or zero
        unsigned shift = 926u - e;                        // value / 2^-149 = (2^52 + m) >> shift
        if (e == 0u || shift > 53u) {
            f = 0u;
        } else {
            unsigned long long M = m | 0x0010000000000000ull;
            unsigned long long rest = M & ((1ull << shift) - 1ull), half = 1ull << (shift - 1u);
            f = (unsigned)(M >> shift);
            f += (rest > half || (rest == half && (f & 1u))) ? 1u : 0u;
        }
    }
    return __uint_as_float(sign | f);
}
__device__ __forceinline__ float d2f_rn(double v) { return d2f_rn2(v, 0); }
__device__ __forceinline__ double f2d(float v) {
    unsigned u = __float_as_uint(v);
    unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long b;
    if (e - 1u <= 253u) {                                 // normal
        b = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (e == 0xffu) {                              // infinity, NaN (made quiet)
        b = 0x7ff0000000000000ull | (m ? 0x0008000000000000ull | ((unsigned long long)m << 29) : 0ull);
    } else if (m == 0u) {                                 // signed zero
        b = 0ull;
    } else {                                              // binary32 subnormal: m 2^-149, normal here
        unsigned p = 31u - (unsigned)__clz((int)m);       // leading bit, 0..22
        b = ((unsigned long long)(874u + p) << 52) | (((unsigned long long)m << (52u - p)) & 0x000fffffffffffffull);
    }
    return __longlong_as_double((long long)(sign | b));
}

// ---- FP32-pair ("double-single") arithmetic --------------------------------------------
// A value is an unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2 (48-bit
// significand).  Sums use Knuth's TwoSum and the fast renormalisation of Dekker (1971); products
// use the exact product error of a fused multiply-add.  Every operation is FP32 arithmetic, so
// it costs no FP64 instruction (the FP64 pipe of this GPU issues at a small fraction of the
// FP32 rate).  Each operation is accurate to a few units of 2^-44 relative.  Used for the WENO3
// weights and for the FP64-accurate sums of FP32 dot products.
struct f32x2 {
    float hi, lo;
};
__device__ __forceinline__ f32x2 quick_two_sum(float a, float b) {   // |a| >= |b|
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f32x2 two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);                 // the exact error of the product
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}
__device__ __forceinline__ f32x2 x2_div(f32x2 a, f32x2 b) {     // b > 0
    float q1 = __fdiv_rn(a.hi, b.hi);
    f32x2 p = x2_mul(b, {q1, 0.0f});
    f32x2 r = x2_add(a, {-p.hi, -p.lo});             // a - q1 b
    float q2 = __fdiv_rn(r.hi, b.hi);
    return quick_two_sum(q1, q2);
}
// a binary64 value as a pair on the integer pipes: the top 24 significand bits (truncated) and
// the remaining 29 rounded to 24; |a| in [2^-60, 2^28) (smaller values are 0 here)
__device__ __forceinline__ f32x2 x2_from(double a) {
    unsigned long long b = (unsigned long long)__double_as_longlong(a);
    unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    if (e < 963u) return {0.0f, 0.0f};
    unsigned sign = (unsigned)(b >> 63) << 31;
    float hi = __uint_as_float(sign | ((e - 896u) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    float scale = __uint_as_float((e - 948u) << 23);        // 2^(e - 1075), a normal float
    float lo = __uint2float_rn((unsigned)(b & 0x1fffffffu)) * scale;
    return {hi, sign ? -lo : lo};
}
// the pair as a binary64 value: the two widened exactly, one FP64 add
__device__ __forceinline__ double x2_to(f32x2 a) { return f2d(a.hi) + f2d(a.lo); }

// 1 / x for x > 0 without the FP64 division sequence: an FP32 seed (x truncated to FP32 on the
// integer pipes, its IEEE reciprocal, widened exactly) and two Newton-Raphson steps r <- r + r
// (1 - x r), each squaring the relative error (2^-22.4 -> 2^-44.8 -> rounding): within about
// one unit in the last place.  Outside [2^-126, 2^126) the division, in a call (so that its
// instructions are not issued for every element).
static __device__ __noinline__ double recip64_div(double x) { return 1.0 / x; }
__device__ __forceinline__ double recip64(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    if (e - 897u > 251u || (b >> 63)) return recip64_div(x);
    float xf = __uint_as_float(((e - 896u) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    unsigned u = __float_as_uint(__frcp_rn(xf));
    double r = __longlong_as_double((long long)(((unsigned long long)(((u >> 23) & 0xffu) + 896u) << 52) |
                                                ((unsigned long long)(u & 0x7fffffu) << 29)));
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

inline int div_up(long long a, int b) { return (int)((a + b - 1) / b); }
// launch grids that cover every instance of a (possibly batched) launch
inline dim3 grid1(long long n, int bs, int nz) { return dim3(div_up(n, bs), 1, nz); }
inline dim3 rows_grid(int n, int rows, int bs, int nz) { return dim3(div_up(n, bs), rows, nz); }

}  // namespace ebit
