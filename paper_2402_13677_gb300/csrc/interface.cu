// EBIT interface kernels: Color-Vertex reconstruction (S0/S5), narrow band, interfacial
// velocity (S2), dimension-split marker sweeps (S3/S4), ghost-fluid link fractions (S7)
// and the interface mass flux (S9).
//
// Paper (arXiv 2402.13677): Sec. 2.1 (one marker per edge, marker-motion equations,
// aligned/unaligned markers and the circle fit of Fig. 1, Color-Vertex reconnection),
// Sec. 2.2 (property average), Sec. 2.3 (interfacial-velocity equation, bilinear
// interpolation, Fig. 2), Sec. 2.4 (ghost-temperature equation, mass-flux and
// normal-gradient equations, Fig. 3).
//
// This translation unit is compiled with -fmad=false: every double operation is a
// separately rounded IEEE add/mul/div/sqrt in the order written, so cut flags, topology
// and marker positions are reproducible bit for bit by any implementation that uses the
// same operation order.  All geometry is FP64.
//
// Every kernel is one thread per item of a full-grid index space (cells, vertices or
// edges) and gathers what it needs from its neighbours: no atomics, no ordering effects.
#include "common.cuh"
#include "kernels.h"

namespace ebit {

// ---------------------------------------------------------------------------------
// cell-local marker coordinates (cell edge k: 0 bottom, 1 right, 2 top, 3 left; edge k
// runs from corner k to corner k+1, corners 0 BL, 1 BR, 2 TR, 3 TL)
// ---------------------------------------------------------------------------------
__device__ inline double2 marker_local(const Grid& g, const double* hpos, const double* vpos,
                                       int k, int i, int j) {
    switch (k) {
        case 0: return make_double2(hpos[hidx(g, i, j)], 0.0);
        case 1: return make_double2(1.0, vpos[veidx(g, i + 1, j)]);
        case 2: return make_double2(hpos[hidx(g, i, j + 1)], 1.0);
        default: return make_double2(0.0, vpos[veidx(g, i, j)]);
    }
}

__device__ inline double2 corner_local(int k) {
    return make_double2((k == 1 || k == 2) ? 1.0 : 0.0, (k >= 2) ? 1.0 : 0.0);
}

__device__ inline double shoelace3(double2 a, double2 b, double2 c) {
    double s = 0.0;
    s = s + (a.x * b.y - b.x * a.y);
    s = s + (b.x * c.y - c.x * b.y);
    s = s + (c.x * a.y - a.x * c.y);
    return 0.5 * s;
}

__device__ inline double cross_centre(double2 P, double2 Q) {
    return (Q.x - P.x) * (0.5 - P.y) - (Q.y - P.y) * (0.5 - P.x);
}

__device__ inline double dist2d(double2 A, double2 B) {
    double dx = B.x - A.x;
    double dy = B.y - A.y;
    return sqrt(dx * dx + dy * dy);
}

__device__ inline int seg_count(uint16_t code) { return code & 3; }
__device__ inline int seg_P(uint16_t code, int s) { return (code >> (2 + 4 * s)) & 3; }
__device__ inline int seg_Q(uint16_t code, int s) { return (code >> (4 + 4 * s)) & 3; }

// ---------------------------------------------------------------------------------
// S0: Color-Vertex reconstruction of every cell
// ---------------------------------------------------------------------------------
__device__ inline void reconstruct_cell(const Grid& g, const uint8_t* __restrict__ vcol,
                                        const double* __restrict__ hpos, const double* __restrict__ vpos,
                                        uint16_t* __restrict__ cseg, uint8_t* __restrict__ flags,
                                        double* __restrict__ vf, int i, int j) {
    int c[4];
    c[0] = vcol[vidx(g, i, j)];
    c[1] = vcol[vidx(g, i + 1, j)];
    c[2] = vcol[vidx(g, i + 1, j + 1)];
    c[3] = vcol[vidx(g, i, j + 1)];
    int cell = cidx(g, i, j);
    if (c[0] == c[1] && c[0] == c[2] && c[0] == c[3]) {
        cseg[cell] = 0;
        flags[cell] = (uint8_t)(c[0] ? F_CCOL : 0);
        if (vf) vf[cell] = (double)c[0];
        return;
    }
    double2 M[4];
    for (int k = 0; k < 4; ++k) M[k] = marker_local(g, hpos, vpos, k, i, j);
    int ex[2], en[2], nex = 0, nen = 0;
    for (int k = 0; k < 4; ++k) {
        int a = c[k], b = c[(k + 1) & 3];
        if (a == 1 && b == 0) ex[nex++] = k;
        if (a == 0 && b == 1) en[nen++] = k;
    }
    double area;
    int ccol;
    uint16_t code;
    if (nex == 1) {
        int kx = ex[0], kn = en[0];
        // liquid polygon: Q (enter), corners kn+1 .. kx, P (exit)
        double2 pts[6];
        int np = 0;
        pts[np++] = M[kn];
        int k = (kn + 1) & 3;
        while (true) {
            pts[np++] = corner_local(k);
            if (k == kx) break;
            k = (k + 1) & 3;
        }
        pts[np++] = M[kx];
        double s = 0.0;
        for (int a = 0; a < np; ++a) {
            double2 A = pts[a], B = pts[(a + 1) % np];
            s = s + (A.x * B.y - B.x * A.y);
        }
        area = 0.5 * s;
        ccol = cross_centre(M[kx], M[kn]) >= 0.0 ? 1 : 0;
        code = (uint16_t)(1 | (kx << 2) | (kn << 4));
    } else {
        int k1 = ex[0], k2 = ex[1];
        double LA = dist2d(M[k1], M[(k1 + 1) & 3]) + dist2d(M[k2], M[(k2 + 1) & 3]);
        double LB = dist2d(M[k1], M[(k1 + 3) & 3]) + dist2d(M[k2], M[(k2 + 3) & 3]);
        if (LA <= LB) {
            int n1 = (k1 + 1) & 3, n2 = (k2 + 1) & 3;
            double a = 0.0;
            a = a + shoelace3(M[k1], corner_local(n1), M[n1]);
            a = a + shoelace3(M[k2], corner_local(n2), M[n2]);
            area = 1.0 - a;
            ccol = 1;
            if (cross_centre(M[k1], M[n1]) < 0.0) ccol = 0;
            if (cross_centre(M[k2], M[n2]) < 0.0) ccol = 0;
            code = (uint16_t)(2 | (k1 << 2) | (n1 << 4) | (k2 << 6) | (n2 << 8));
        } else {
            int n1 = (k1 + 3) & 3, n2 = (k2 + 3) & 3;
            double a = 0.0;
            a = a + shoelace3(M[n1], corner_local(k1), M[k1]);
            a = a + shoelace3(M[n2], corner_local(k2), M[k2]);
            area = a;
            ccol = 0;
            if (cross_centre(M[k1], M[n1]) >= 0.0) ccol = 1;
            if (cross_centre(M[k2], M[n2]) >= 0.0) ccol = 1;
            code = (uint16_t)(2 | (k1 << 2) | (n1 << 4) | (k2 << 6) | (n2 << 8));
        }
    }
    cseg[cell] = code;
    flags[cell] = (uint8_t)((ccol ? F_CCOL : 0) | F_CUT);
    if (vf) vf[cell] = area;
}

__global__ void k_reconstruct(Grid g, const uint8_t* __restrict__ vcol, const double* __restrict__ hpos,
                              const double* __restrict__ vpos, uint16_t* __restrict__ cseg,
                              uint8_t* __restrict__ flags, double* __restrict__ vf) {
    const long long zo = zoff(g.zs);
    vcol = zsh(vcol, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    cseg = zsh(cseg, zo);
    flags = zsh(flags, zo);
    vf = zsh(vf, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    reconstruct_cell(g, vcol, hpos, vpos, cseg, flags, vf, i, j);
}

// the same over the cells within two of the start-of-step interface (the near list): with every
// marker moving less than a cell per sweep (the sweeps report EBIT_ECFL otherwise) the vertices
// and edges the sweeps change, and every cell they can cut, lie in those cells; the other cells
// keep their geometry
__global__ void k_reconstruct_list(Grid g, const int* __restrict__ list, const int* __restrict__ count,
                                   const uint8_t* __restrict__ vcol, const double* __restrict__ hpos,
                                   const double* __restrict__ vpos, uint16_t* __restrict__ cseg,
                                   uint8_t* __restrict__ flags, double* __restrict__ vf) {
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    vcol = zsh(vcol, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    cseg = zsh(cseg, zo);
    flags = zsh(flags, zo);
    vf = zsh(vf, zo);
    int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int c = list[k];
        reconstruct_cell(g, vcol, hpos, vpos, cseg, flags, vf, c % g.nx, c / g.nx);
    }
}

// narrow band (a cut cell in the 3x3 block) and band normal: normalised sum of (dy, -dx)
// over the segments of the block, visited row by row
__device__ inline void band_cell(const Grid& g, const uint16_t* __restrict__ cseg, const double* __restrict__ hpos,
                                 const double* __restrict__ vpos, uint8_t* __restrict__ flags,
                                 double2* __restrict__ nb, int i, int j) {
    double ax = 0.0, ay = 0.0;
    bool inband = false;
    for (int jj = j - 1; jj <= j + 1; ++jj) {
        if (jj < 0 || jj >= g.ny) continue;
        for (int ii = i - 1; ii <= i + 1; ++ii) {
            if (ii < 0 || ii >= g.nx) continue;
            uint16_t code = cseg[cidx(g, ii, jj)];
            int ns = seg_count(code);
            if (ns == 0) continue;
            inband = true;
            for (int s = 0; s < ns; ++s) {
                double2 P = marker_local(g, hpos, vpos, seg_P(code, s), ii, jj);
                double2 Q = marker_local(g, hpos, vpos, seg_Q(code, s), ii, jj);
                double dx = Q.x - P.x;
                double dy = Q.y - P.y;
                ax = ax + dy;
                ay = ay - dx;
            }
        }
    }
    int cell = cidx(g, i, j);
    double2 n = make_double2(0.0, 0.0);
    uint8_t f = flags[cell] & (uint8_t)(F_CCOL | F_CUT);
    if (inband) {
        f |= F_BAND;
        double nrm = sqrt(ax * ax + ay * ay);
        if (nrm > 0.0) n = make_double2(ax / nrm, ay / nrm);
    }
    flags[cell] = f;
    nb[cell] = n;
}

__global__ void k_band(Grid g, const uint16_t* __restrict__ cseg, const double* __restrict__ hpos,
                       const double* __restrict__ vpos, uint8_t* __restrict__ flags,
                       double2* __restrict__ nb) {
    const long long zo = zoff(g.zs);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    flags = zsh(flags, zo);
    nb = zsh(nb, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    band_cell(g, cseg, hpos, vpos, flags, nb, i, j);
}

// the same over the near list and its neighbours (nine items per listed cell: the new band lies
// within one cell of the new cut cells, which lie in the near list, and the old band lies in the
// near list); a cell reached from several listed cells is written several times with the same
// value (each write masks the band bit it reads)
__global__ void k_band_list(Grid g, const int* __restrict__ list, const int* __restrict__ count,
                            const uint16_t* __restrict__ cseg, const double* __restrict__ hpos,
                            const double* __restrict__ vpos, uint8_t* __restrict__ flags,
                            double2* __restrict__ nb) {
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    flags = zsh(flags, zo);
    nb = zsh(nb, zo);
    long long n = 9LL * *count;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int c = list[t / 9], q = (int)(t % 9);
        int i = c % g.nx + q % 3 - 1, j = c / g.nx + q / 3 - 1;
        if (i < 0 || i >= g.nx || j < 0 || j >= g.ny) continue;
        band_cell(g, cseg, hpos, vpos, flags, nb, i, j);
    }
}

// u_Gamma at cell centres from the jump condition (interfacial-velocity equation)
// bilinear interpolation from the four nearest cell centres (Fig. 2)
__device__ inline double interp_bilinear(const double2* uG, const Grid& g, int comp, double x, double y) {
    double fx = x - 0.5;
    double fy = y - 0.5;
    int ix = (int)floor(fx);
    int iy = (int)floor(fy);
    double xb = fx - (double)ix;
    double yb = fy - (double)iy;
    double u2 = cell_vel(uG, g, comp, ix, iy);
    double u1 = cell_vel(uG, g, comp, ix, iy + 1);
    double u3 = cell_vel(uG, g, comp, ix + 1, iy);
    double u4 = cell_vel(uG, g, comp, ix + 1, iy + 1);
    double wx0 = 1.0 - xb;
    double wy0 = 1.0 - yb;
    return wx0 * wy0 * u2 + wx0 * yb * u1 + xb * wy0 * u3 + xb * yb * u4;
}

// ---------------------------------------------------------------------------------
// S2-S4: one sweep along `axis`
// ---------------------------------------------------------------------------------
__device__ inline bool hcut(const Grid& g, const uint8_t* vcol, int i, int j) {
    return vcol[vidx(g, i, j)] != vcol[vidx(g, i + 1, j)];
}
__device__ inline bool vcut(const Grid& g, const uint8_t* vcol, int i, int j) {
    return vcol[vidx(g, i, j)] != vcol[vidx(g, i, j + 1)];
}

// displaced along-coordinate of the marker on a cut edge (marker-motion equation, explicit
// Euler): horizontal edge (i, j) if hz, else vertical edge (i, j)
__device__ inline void displace_edge(const Grid& g, int axis, double dth, const uint8_t* vcol, const double* hpos,
                                     const double* vpos, const double2* uG, double* hdisp, double* vdisp,
                                     int* status, bool hz, int i, int j) {
    double x, y;
    bool aligned;
    double* out;
    if (hz) {
        if (!hcut(g, vcol, i, j)) return;
        long long t = hidx(g, i, j);
        x = (double)i + hpos[t];
        y = (double)j;
        aligned = axis == 0;
        out = hdisp + t;
    } else {
        if (!vcut(g, vcol, i, j)) return;
        long long e = veidx(g, i, j);
        x = (double)i;
        y = (double)j + vpos[e];
        aligned = axis == 1;
        out = vdisp + e;
    }
    double u = interp_bilinear(uG, g, axis, x, y);
    double d = u * dth;
    double al = axis == 0 ? x : y;
    double nal = (double)(axis == 0 ? g.nx : g.ny);
    if (!aligned && (al == 0.0 || al == nal)) d = 0.0;
    if (!(fabs(d) < 1.0)) atomicOr(status, 1);   // CFL >= 1 (or NaN)
    al = al + d;
    if (aligned) al = fmin(fmax(al, 0.0), nal - FMIN);
    else al = fmin(fmax(al, 0.0), nal);
    *out = al;
}

// Helpers mapping the sweep's (line, index) coordinates to h/v edges.
// axis 0: aligned lines are horizontal (h-edges on line j, index i); unaligned are
//         vertical lines x = m (v-edges on line m, index = row).
// axis 1: aligned lines are vertical (v-edges on line i, index j); unaligned are
//         horizontal lines y = m (h-edges on line m, index = column).
struct SweepView {
    Grid g;
    int axis;
    const uint8_t* vcol;
    const double* hpos;
    const double* vpos;
    const double* hdisp;
    const double* vdisp;

    __device__ int n_al() const { return axis == 0 ? g.nx : g.ny; }
    __device__ int n_ac() const { return axis == 0 ? g.ny : g.nx; }
    // aligned edge e on aligned line l
    __device__ bool a_cut(int l, int e) const {
        return axis == 0 ? hcut(g, vcol, e, l) : vcut(g, vcol, l, e);
    }
    __device__ double a_orig(int l, int e) const {
        return axis == 0 ? (double)e + hpos[hidx(g, e, l)] : (double)e + vpos[veidx(g, l, e)];
    }
    __device__ double a_disp(int l, int e) const {
        return axis == 0 ? hdisp[hidx(g, e, l)] : vdisp[veidx(g, l, e)];
    }
    // unaligned edge e on unaligned line m
    __device__ bool u_cut(int m, int e) const {
        return axis == 0 ? vcut(g, vcol, m, e) : hcut(g, vcol, e, m);
    }
    __device__ double u_disp(int m, int e) const {
        return axis == 0 ? vdisp[veidx(g, m, e)] : hdisp[hidx(g, e, m)];
    }
    __device__ double u_orig_ac(int m, int e) const {
        return axis == 0 ? (double)e + vpos[veidx(g, m, e)] : (double)e + hpos[hidx(g, e, m)];
    }
    // displaced absolute position of the marker on cell-edge k of cell (i, j)
    __device__ double2 disp_pos(int k, int i, int j) const {
        double x, y;
        if (k == 0 || k == 2) {
            int jj = j + (k == 2);
            long long e = hidx(g, i, jj);
            x = (double)i + hpos[e];
            y = (double)jj;
            if (axis == 0) x = hdisp[e]; else y = hdisp[e];
        } else {
            int ii = i + (k == 1);
            long long e = veidx(g, ii, j);
            x = (double)ii;
            y = (double)j + vpos[e];
            if (axis == 0) x = vdisp[e]; else y = vdisp[e];
        }
        return make_double2(x, y);
    }
};

__device__ inline double clampf(double f) { return fmin(fmax(f, FMIN), 1.0 - FMIN); }

__device__ inline double pick_median(double* c, int n) {
    if (n == 0) return 0.5;
    for (int a = 1; a < n; ++a) {
        double v = c[a];
        int b = a - 1;
        while (b >= 0 && c[b] > v) { c[b + 1] = c[b]; --b; }
        c[b + 1] = v;
    }
    return c[(n - 1) / 2];
}

// vertex colours: flip once per aligned marker crossing the vertex
__device__ inline void sweep_vertex(const SweepView& sv, uint8_t* vcol_n, int iv, int jv) {
    const Grid& g = sv.g;
    int l = sv.axis == 0 ? jv : iv;   // aligned line through the vertex
    int m = sv.axis == 0 ? iv : jv;   // position of the vertex along it
    int nal = sv.n_al();
    int flips = 0;
    for (int e = m - 2; e <= m + 1; ++e) {
        if (e < 0 || e >= nal) continue;
        if (!sv.a_cut(l, e)) continue;
        double a0 = sv.a_orig(l, e);
        double a1 = sv.a_disp(l, e);
        if ((a0 < (double)m) != (a1 < (double)m)) flips ^= 1;
    }
    vcol_n[vidx(g, iv, jv)] = (uint8_t)(sv.vcol[vidx(g, iv, jv)] ^ flips);
}

// aligned edges: the markers that slid onto the edge, one kept (lower median)
// (aligned line l, index e along it; 0 <= e < n_al)
__device__ inline void sweep_aligned(const SweepView& sv, const uint8_t* vcol_n, double* out, int l, int e) {
    const Grid& g = sv.g;
    int nal = sv.n_al();
    bool cut;
    long long o;
    if (sv.axis == 0) {
        cut = vcol_n[vidx(g, e, l)] != vcol_n[vidx(g, e + 1, l)];
        o = hidx(g, e, l);
    } else {
        cut = vcol_n[vidx(g, l, e)] != vcol_n[vidx(g, l, e + 1)];
        o = veidx(g, l, e);
    }
    if (!cut) { out[o] = 0.0; return; }
    double cand[8];   // at most five candidates; the first stays in a register
    double first = 0.0;
    int n = 0;
    for (int ee = e - 2; ee <= e + 2; ++ee) {
        if (ee < 0 || ee >= nal || !sv.a_cut(l, ee)) continue;
        double al = sv.a_disp(l, ee);
        double fl = floor(al);
        if ((int)fl != e) continue;
        double v = clampf(al - fl);
        if (n == 0) {
            first = v;
        } else {
            if (n == 1) cand[0] = first;
            cand[n] = v;
        }
        ++n;
    }
    out[o] = n == 1 ? first : pick_median(cand, n);
}

// circle (through E, O, R) or chord (through E, O) crossing of the unaligned line at m
__device__ inline double crossing(double2 E, double2 O, bool hasR, double2 R, int m, int axis) {
    double ea = axis == 0 ? E.x : E.y;
    double ec = axis == 0 ? E.y : E.x;
    double bal = (axis == 0 ? O.x : O.y) - ea;
    double bac = (axis == 0 ? O.y : O.x) - ec;
    double alpha = (double)m - ea;
    double lin = alpha * bac / bal;
    double best = 0.0;
    bool have = false;
    if (hasR) {
        double cal = (axis == 0 ? R.x : R.y) - ea;
        double cac = (axis == 0 ? R.y : R.x) - ec;
        double det = bal * cac - bac * cal;
        double bb = bal * bal + bac * bac;
        double cc = cal * cal + cac * cac;
        double Dp = cc * bac - bb * cac;
        double Ep = bb * cal - cc * bal;
        double qa = det;
        double qb = Ep;
        double qc = det * alpha * alpha + Dp * alpha;
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            double t = qb >= 0.0 ? -0.5 * (qb + sq) : -0.5 * (qb - sq);
            if (t != 0.0) { best = qc / t; have = true; }
            if (qa != 0.0) {
                double r2 = t / qa;
                if (!have || fabs(r2 - lin) < fabs(best - lin)) { best = r2; have = true; }
            }
            if (have && fabs(best - lin) > fabs(bal) + fabs(bac)) have = false;
        }
    }
    if (!have) best = lin;
    return ec + best;
}

// chain neighbour: displaced marker linked, through the cell adjacent across cell-edge kE,
// to the marker on kE of cell (i, j)
__device__ inline bool chain_neighbour(const SweepView& sv, const uint16_t* cseg, int i, int j, int kE,
                                       double2* R) {
    const Grid& g = sv.g;
    int di = (kE == 1) - (kE == 3);
    int dj = (kE == 2) - (kE == 0);
    int in = i + di, jn = j + dj;
    if (in < 0 || in >= g.nx || jn < 0 || jn >= g.ny) return false;
    int kk = (kE + 2) & 3;
    uint16_t code = cseg[cidx(g, in, jn)];
    int ns = seg_count(code);
    for (int s = 0; s < ns; ++s) {
        int kP = seg_P(code, s), kQ = seg_Q(code, s);
        if (kP == kk) { *R = sv.disp_pos(kQ, in, jn); return true; }
        if (kQ == kk) { *R = sv.disp_pos(kP, in, jn); return true; }
    }
    return false;
}

// unaligned edges: crossings of the displaced segments with the edge's grid line, plus
// displaced markers lying exactly on it; one kept (lower median)
// (unaligned line m, index e across; 0 <= e < n_ac)
__device__ inline void sweep_unaligned(const SweepView& sv, const uint16_t* cseg, const uint8_t* vcol_n, double* out,
                                       int* status, int m, int e) {
    const Grid& g = sv.g;
    int nac = sv.n_ac();
    int nal = sv.n_al();
    bool cut;
    long long o;
    if (sv.axis == 0) {
        cut = vcol_n[vidx(g, m, e)] != vcol_n[vidx(g, m, e + 1)];
        o = veidx(g, m, e);
    } else {
        cut = vcol_n[vidx(g, e, m)] != vcol_n[vidx(g, e + 1, m)];
        o = hidx(g, e, m);
    }
    if (!cut) { out[o] = 0.0; return; }
    // candidate positions: the first in a register (most edges have one), the array (local
    // memory) only once a second arrives
    double cand[32];
    double first = 0.0;
    int n = 0;
    auto push = [&](double v) {
        if (n >= 32) {
            atomicOr(status, 2);
            return;
        }
        if (n == 0) {
            first = v;
        } else {
            if (n == 1) cand[0] = first;
            cand[n] = v;
        }
        ++n;
    };
    const double dm = (double)m;
    // (i) displaced segments of the cells of this row/column straddling the line
    for (int c = m - 2; c <= m + 1; ++c) {
        if (c < 0 || c >= nal) continue;
        int ci = sv.axis == 0 ? c : e;
        int cj = sv.axis == 0 ? e : c;
        uint16_t code = cseg[cidx(g, ci, cj)];
        int ns = seg_count(code);
        for (int s = 0; s < ns; ++s) {
            int kP = seg_P(code, s), kQ = seg_Q(code, s);
            double2 Pn = sv.disp_pos(kP, ci, cj);
            double2 Qn = sv.disp_pos(kQ, ci, cj);
            double pa = sv.axis == 0 ? Pn.x : Pn.y;
            double qa = sv.axis == 0 ? Qn.x : Qn.y;
            double lo = fmin(pa, qa), hi = fmax(pa, qa);
            if (!(lo < dm && dm < hi)) continue;
            double2 E, O;
            int kE;
            if (fabs(pa - dm) <= fabs(qa - dm)) { E = Pn; O = Qn; kE = kP; }
            else { E = Qn; O = Pn; kE = kQ; }
            double2 R;
            bool hasR = chain_neighbour(sv, cseg, ci, cj, kE, &R);
            double ac = crossing(E, O, hasR, R, m, sv.axis);
            push(clampf(ac - (double)e));
        }
    }
    // (ii) displaced markers exactly on the line: unaligned markers of nearby lines
    for (int mm = m - 2; mm <= m + 2; ++mm) {
        if (mm < 0 || mm > nal) continue;
        if (!sv.u_cut(mm, e)) continue;
        if (sv.u_disp(mm, e) == dm) {
            double ac = sv.u_orig_ac(mm, e);
            double fl = floor(ac);
            int ee = min(max((int)fl, 0), nac - 1);
            if (ee == e) push(clampf(ac - (double)ee));
        }
    }
    //      and aligned markers whose line maps to this edge index
    for (int l = e; l <= e + 1; ++l) {
        if (l == e + 1 && l != nac) continue;   // line nac clamps to index nac - 1
        for (int ea = m - 3; ea <= m + 2; ++ea) {
            if (ea < 0 || ea >= nal || !sv.a_cut(l, ea)) continue;
            if (sv.a_disp(l, ea) == dm) {
                double ac = (double)l;
                int ee = min(max(l, 0), nac - 1);
                if (ee == e) push(clampf(ac - (double)ee));
            }
        }
    }
    out[o] = n == 1 ? first : pick_median(cand, n);
}

// ---------------------------------------------------------------------------------
// the sweeps over the cells near the interface (O(sqrt N) work)
// ---------------------------------------------------------------------------------
// The cells within two of a cut cell of the geometry at the start of the step: the narrow band
// (cells within one of a cut cell) dilated by one more cell, with an int mark per cell (all
// zero between steps) so that each cell enters the list once.  A marker moves less than a cell
// per sweep, so every edge that is cut before, between or after the two sweeps is an edge of a
// listed cell, and every vertex that can flip colour is a corner of one.
__global__ void k_band_dilate(Grid g, const int* __restrict__ band, const int* __restrict__ nband,
                              int* __restrict__ mark, int* __restrict__ list, int* __restrict__ count) {
    const long long zo = zoff(g.zs);
    band = zsh(band, zo);
    nband = zsh(nband, zo);
    mark = zsh(mark, zo);
    list = zsh(list, zo);
    count = zsh(count, zo);
    int n = *nband;
    int lane = threadIdx.x & 31;
    // whole warps iterate together, so that the appends can be counted with one atomic per warp
    int stride = gridDim.x * blockDim.x;
    int n_up = (n + 31) & ~31;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k - lane < n_up; k += stride) {
        bool valid = k < n;
        int i = 0, j = 0;
        if (valid) {
            int c = band[k];
            j = (int)((unsigned)c / (unsigned)g.nx);
            i = c - j * g.nx;
        }
        for (int q = 0; q < 9; ++q) {
            int ii = i + q % 3 - 1, jj = j + q / 3 - 1;
            bool in = valid && ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny;
            int d = in ? cidx(g, ii, jj) : 0;
            bool add = in && atomicExch(&mark[d], 1) == 0;
            unsigned bal = __ballot_sync(0xffffffffu, add);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(count, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (add) list[base + __popc(bal & ((1u << lane) - 1u))] = d;
        }
    }
}

// the marks of the listed cells back to zero (after the step's sweeps)
__global__ void k_band_unmark(Grid g, const int* __restrict__ list, const int* __restrict__ count,
                              int* __restrict__ mark) {
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    mark = zsh(mark, zo);
    int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) mark[list[k]] = 0;
}

// u_Gamma (k_ug's formula) on the listed cells: the cells the markers' bilinear stencils read in
// both sweeps of the step (a marker moves less than a cell per sweep)
__global__ void k_ug_list(Grid g, Phys p, const int* __restrict__ list, const int* __restrict__ count,
                          const uint8_t* __restrict__ flags, const double2* __restrict__ u_l,
                          const double2* __restrict__ u_v, const double* __restrict__ mdot,
                          const double2* __restrict__ nb, double2* __restrict__ uG) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    flags = zsh(flags, zo);
    u_l = zsh(u_l, zo);
    u_v = zsh(u_v, zo);
    mdot = zsh(mdot, zo);
    nb = zsh(nb, zo);
    uG = zsh(uG, zo);
    int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int c = list[k];
        double m = mdot[c];
        double2 nv = nb[c];
        if (flags[c] & F_CCOL) {
            double cl = m / p.rho_l;
            double2 u = u_l[c];
            uG[c] = make_double2(u.x - cl * nv.x, u.y - cl * nv.y);
        } else {
            double cv = m / p.rho_v;
            double2 u = u_v[c];
            uG[c] = make_double2(u.x - cv * nv.x, u.y - cv * nv.y);
        }
    }
}

// displacement of the cut edges among the four edges of each listed cell (an edge shared by two
// listed cells is computed by both, with the same value)
__global__ void k_displace_list(Grid g, int axis, double dth, const int* __restrict__ list,
                                const int* __restrict__ count, const uint8_t* __restrict__ vcol,
                                const double* __restrict__ hpos, const double* __restrict__ vpos,
                                const double2* __restrict__ uG, double* __restrict__ hdisp,
                                double* __restrict__ vdisp, int* __restrict__ status) {
    if (g.pz) dth = g.pz[blockIdx.z].dt / g.h;
    const long long zo = zoff(g.zs);
    list = zsh(list, zo);
    count = zsh(count, zo);
    vcol = zsh(vcol, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    uG = zsh(uG, zo);
    hdisp = zsh(hdisp, zo);
    vdisp = zsh(vdisp, zo);
    status = zsh(status, zo);
    int n = 4 * *count;   // one thread per (cell, edge): the work is latency-bound
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int c = list[t >> 2], q = t & 3;
        int j = (int)((unsigned)c / (unsigned)g.nx), i = c - j * g.nx;
        displace_edge(g, axis, dth, vcol, hpos, vpos, uG, hdisp, vdisp, status, q < 2, i + (q == 3),
                      j + (q == 1));
    }
}

// the four corners of each listed cell (vcol_n holds a copy of vcol elsewhere)
__global__ void k_sweep_vertices_list(SweepView sv, const int* __restrict__ list, const int* __restrict__ count,
                                      uint8_t* __restrict__ vcol_n) {
    const long long zo = zoff(sv.g.zs);
    sv.vcol = zsh(sv.vcol, zo);
    sv.hpos = zsh(sv.hpos, zo);
    sv.vpos = zsh(sv.vpos, zo);
    sv.hdisp = zsh(sv.hdisp, zo);
    sv.vdisp = zsh(sv.vdisp, zo);
    list = zsh(list, zo);
    count = zsh(count, zo);
    vcol_n = zsh(vcol_n, zo);
    const Grid& g = sv.g;
    int n = 4 * *count;   // one thread per (cell, corner)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int c = list[t >> 2], q = t & 3;
        int j = (int)((unsigned)c / (unsigned)g.nx), i = c - j * g.nx;
        sweep_vertex(sv, vcol_n, i + (q & 1), j + (q >> 1));
    }
}

// the four edges of each listed cell, aligned or unaligned for this sweep (the new marker
// arrays are zero elsewhere); out_al / out_un are the new h- / v-edge arrays as the axis says
__global__ void k_sweep_edges_list(SweepView sv, const int* __restrict__ list, const int* __restrict__ count,
                                   const uint16_t* __restrict__ cseg, const uint8_t* __restrict__ vcol_n,
                                   double* __restrict__ out_al, double* __restrict__ out_un, int* __restrict__ status) {
    const long long zo = zoff(sv.g.zs);
    sv.vcol = zsh(sv.vcol, zo);
    sv.hpos = zsh(sv.hpos, zo);
    sv.vpos = zsh(sv.vpos, zo);
    sv.hdisp = zsh(sv.hdisp, zo);
    sv.vdisp = zsh(sv.vdisp, zo);
    list = zsh(list, zo);
    count = zsh(count, zo);
    cseg = zsh(cseg, zo);
    vcol_n = zsh(vcol_n, zo);
    out_al = zsh(out_al, zo);
    out_un = zsh(out_un, zo);
    status = zsh(status, zo);
    int n = 4 * *count;   // one thread per (cell, edge)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int c = list[t >> 2], q = t & 3;
        int j = (int)((unsigned)c / (unsigned)sv.g.nx), i = c - j * sv.g.nx;
        // axis 0: aligned = horizontal edges (line j, index i), unaligned = vertical (line i, index j)
        // axis 1: aligned = vertical edges (line i, index j), unaligned = horizontal (line j, index i)
        int la = sv.axis == 0 ? j : i, ea = sv.axis == 0 ? i : j;
        if (q < 2) sweep_aligned(sv, vcol_n, out_al, la + q, ea);
        else sweep_unaligned(sv, cseg, vcol_n, out_un, status, ea + (q - 2), la);
    }
}

// ---------------------------------------------------------------------------------
// S7: ghost-fluid link fractions -> per-cell Dirichlet coefficient sum and RHS
// ---------------------------------------------------------------------------------
// crossings of the segments of cell (i, j) with its centre line (dir 0: y = 0.5, giving
// local x; dir 1: x = 0.5, giving local y), restricted to [lo, hi]; returns the minimum
// of (sign * v + off) over them, or +inf
__device__ inline double min_crossing(const Grid& g, const uint16_t* cseg, const double* hpos,
                                      const double* vpos, int i, int j, int dir, double lo, double hi,
                                      double sign, double off) {
    double best = INFINITY;
    uint16_t code = cseg[cidx(g, i, j)];
    int ns = seg_count(code);
    for (int s = 0; s < ns; ++s) {
        double2 P = marker_local(g, hpos, vpos, seg_P(code, s), i, j);
        double2 Q = marker_local(g, hpos, vpos, seg_Q(code, s), i, j);
        double v;
        if (dir == 0) {
            if ((P.y < 0.5) == (Q.y < 0.5)) continue;
            v = P.x + (0.5 - P.y) * (Q.x - P.x) / (Q.y - P.y);
        } else {
            if ((P.x < 0.5) == (Q.x < 0.5)) continue;
            v = P.y + (0.5 - P.x) * (Q.y - P.y) / (Q.x - P.x);
        }
        if (lo <= v && v <= hi) best = fmin(best, sign * v + off);
    }
    return best;
}

__device__ double link_theta(const Grid& g, const uint16_t* cseg, const double* hpos, const double* vpos,
                             int i, int j, int side, double theta_min) {
    double t;
    switch (side) {
        case 0:  // +x: crossings in [0.5, 1] of this cell, [0, 0.5] of the right neighbour
            t = fmin(min_crossing(g, cseg, hpos, vpos, i, j, 0, 0.5, 1.0, 1.0, -0.5),
                     min_crossing(g, cseg, hpos, vpos, i + 1, j, 0, 0.0, 0.5, 1.0, 0.5));
            break;
        case 1:  // -x
            t = fmin(min_crossing(g, cseg, hpos, vpos, i - 1, j, 0, 0.5, 1.0, -1.0, 1.5),
                     min_crossing(g, cseg, hpos, vpos, i, j, 0, 0.0, 0.5, -1.0, 0.5));
            break;
        case 2:  // +y
            t = fmin(min_crossing(g, cseg, hpos, vpos, i, j, 1, 0.5, 1.0, 1.0, -0.5),
                     min_crossing(g, cseg, hpos, vpos, i, j + 1, 1, 0.0, 0.5, 1.0, 0.5));
            break;
        default:  // -y
            t = fmin(min_crossing(g, cseg, hpos, vpos, i, j - 1, 1, 0.5, 1.0, -1.0, 1.5),
                     min_crossing(g, cseg, hpos, vpos, i, j, 1, 0.0, 0.5, -1.0, 0.5));
            break;
    }
    if (t == INFINITY) t = 0.5;
    return fmin(fmax(t, theta_min), 1.0);
}

// Energy operator of the combined (block-diagonal) two-phase system, integrated form:
//   cd = h^2 (rho cp)_k / dt,   dd = sum_cut lambda_k / theta + sum_Tfixed 2 lambda_k,
//   wl/wb (left/bottom face) = lambda_k between two cells of the same phase, 0 across the interface,
//   b = cd T*_k + sum_cut lambda_k T_sat / theta + sum 2 lambda_k T_w,  x0 = T*_k;
// axisymmetric: cd times the cell's radius, every face term times the radius of its face.
template <bool AXI>
__global__ void k_energy_operator(Grid g, Phys p, const uint8_t* __restrict__ flags,
                                  const uint16_t* __restrict__ cseg, const double* __restrict__ hpos,
                                  const double* __restrict__ vpos, const double* __restrict__ Ts_l,
                                  const double* __restrict__ Ts_v, double* __restrict__ cd,
                                  double* __restrict__ dd, double* __restrict__ wl, double* __restrict__ wb,
                                  double* __restrict__ b, double* __restrict__ x0) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    flags = zsh(flags, zo);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    Ts_l = zsh(Ts_l, zo);
    Ts_v = zsh(Ts_v, zo);
    cd = zsh(cd, zo);
    dd = zsh(dd, zo);
    wl = zsh(wl, zo);
    wb = zsh(wb, zo);
    b = zsh(b, zo);
    x0 = zsh(x0, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    int c = cidx(g, i, j);
    int k = flags[c] & F_CCOL;
    double lam = k ? p.lam_l : p.lam_v;
    double rc = k ? p.rho_l * p.cp_l : p.rho_v * p.cp_v;
    const double mc = rad_c<AXI>(g, i);
    double coef = g.h * g.h * rc * p.inv_dt * mc;
    double ts = k ? Ts_l[c] : Ts_v[c];
    double dsum = 0.0, rhs = coef * ts;
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    const int bside[4] = {1, 0, 3, 2};
    for (int s = 0; s < 4; ++s) {
        int ii = i + di[s], jj = j + dj[s];
        // conductance of the face this link crosses
        double lf = AXI ? lam * (s == 0 ? rad_fx<AXI>(g, i + 1) : (s == 1 ? rad_fx<AXI>(g, i) : mc)) : lam;
        if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.ny) {
            int bs = bside[s];
            if (g.Tfix[bs]) {
                dsum += 2.0 * lf;
                rhs += 2.0 * lf * g.Tw[bs];
            }
            continue;
        }
        int kn = flags[cidx(g, ii, jj)] & F_CCOL;
        if (kn != k) {
            double th = link_theta(g, cseg, hpos, vpos, i, j, s, p.theta_min);
            dsum += lf / th;
            rhs += lf * p.T_sat / th;
        }
    }
    cd[c] = coef;
    dd[c] = dsum;
    b[c] = rhs;
    x0[c] = ts;
    // left and bottom face weights of the cell (domain faces carry none)
    wl[c] = (i > 0 && (flags[cidx(g, i - 1, j)] & F_CCOL) == k) ? lam * rad_fx<AXI>(g, i) : 0.0;
    wb[c] = (j > 0 && (flags[cidx(g, i, j - 1)] & F_CCOL) == k) ? lam * mc : 0.0;
}

// ---------------------------------------------------------------------------------
// S9: mass flux on cut cells (mass-flux and normal-gradient equations)
// ---------------------------------------------------------------------------------
__device__ inline double interp_biquadratic(const double* F, const Grid& g, double px, double py) {
    int ic = min(max((int)floor(px), 1), g.nx - 2);
    int jc = min(max((int)floor(py), 1), g.ny - 2);
    double sx = px - ((double)ic + 0.5);
    double sy = py - ((double)jc + 0.5);
    double wx[3] = {0.5 * sx * (sx - 1.0), 1.0 - sx * sx, 0.5 * sx * (sx + 1.0)};
    double wy[3] = {0.5 * sy * (sy - 1.0), 1.0 - sy * sy, 0.5 * sy * (sy + 1.0)};
    double v = 0.0;
    for (int b = 0; b < 3; ++b) {
        double r = 0.0;
        for (int a = 0; a < 3; ++a) r += wx[a] * F[cidx(g, ic - 1 + a, jc - 1 + b)];
        v += wy[b] * r;
    }
    return v;
}

__global__ void k_mass_flux(Grid g, Phys p, const uint16_t* __restrict__ cseg, const double* __restrict__ hpos,
                            const double* __restrict__ vpos, const double* __restrict__ T_l,
                            const double* __restrict__ T_v, double* __restrict__ mdot) {
    zphys(g, p);
    const long long zo = zoff(g.zs);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    T_l = zsh(T_l, zo);
    T_v = zsh(T_v, zo);
    mdot = zsh(mdot, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    int c = cidx(g, i, j);
    uint16_t code = cseg[c];
    int ns = seg_count(code);
    if (ns == 0) { mdot[c] = 0.0; return; }
    if (!p.energy) { mdot[c] = p.mdot_fixed; return; }
    const double D1 = 1.5, D2 = 2.5;
    double num = 0.0, den = 0.0;
    for (int s = 0; s < ns; ++s) {
        double2 P = marker_local(g, hpos, vpos, seg_P(code, s), i, j);
        double2 Q = marker_local(g, hpos, vpos, seg_Q(code, s), i, j);
        double dx = Q.x - P.x, dy = Q.y - P.y;
        double L = sqrt(dx * dx + dy * dy);
        double mx = (double)i + 0.5 * (P.x + Q.x);
        double my = (double)j + 0.5 * (P.y + Q.y);
        double nx = L > 0.0 ? dy / L : 0.0;
        double ny = L > 0.0 ? -dx / L : 0.0;
        double Tv1 = interp_biquadratic(T_v, g, mx + D1 * nx, my + D1 * ny);
        double Tv2 = interp_biquadratic(T_v, g, mx + D2 * nx, my + D2 * ny);
        double Tl1 = interp_biquadratic(T_l, g, mx - D1 * nx, my - D1 * ny);
        double Tl2 = interp_biquadratic(T_l, g, mx - D2 * nx, my - D2 * ny);
        double a_v = ((Tv1 - p.T_sat) * D2 / D1 - (Tv2 - p.T_sat) * D1 / D2) / ((D2 - D1) * g.h);
        double a_l = ((Tl1 - p.T_sat) * D2 / D1 - (Tl2 - p.T_sat) * D1 / D2) / ((D2 - D1) * g.h);
        double ms = (p.lam_l * a_l + p.lam_v * a_v) / p.h_lg;
        num += L * ms;
        den += L;
    }
    mdot[c] = den > 0.0 ? num / den : 0.0;
}

// check of an uploaded interface (one instance): vertex colours 0 or 1 (err bit 0), every cut
// edge's marker fraction inside [FMIN, 1 - FMIN] (err bit 1); fractions of uncut edges are set
// to 0.  One thread per vertex / h-edge / v-edge index.
__global__ void k_check_interface(Grid g, const uint8_t* __restrict__ vcol, double* __restrict__ hpos,
                                  double* __restrict__ vpos, int* __restrict__ err) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nv = (long long)(g.nx + 1) * (g.ny + 1), nh = (long long)(g.ny + 1) * g.nx,
              nve = (long long)g.ny * (g.nx + 1);
    int bad = 0;
    if (t < nv && vcol[t] > 1) bad |= 1;
    if (t < nh) {
        int j = (int)((unsigned)t / (unsigned)g.nx), i = (int)t - j * g.nx;
        double f = hpos[t];
        if (!hcut(g, vcol, i, j)) hpos[t] = 0.0;
        else if (!(f >= FMIN && f <= 1.0 - FMIN)) bad |= 2;
    }
    if (t < nve) {
        int j = (int)((unsigned)t / (unsigned)(g.nx + 1)), i = (int)t - j * (g.nx + 1);
        double f = vpos[t];
        if (!vcut(g, vcol, i, j)) vpos[t] = 0.0;
        else if (!(f >= FMIN && f <= 1.0 - FMIN)) bad |= 2;
    }
    if (bad) atomicOr(err, bad);
}

// ---------------------------------------------------------------------------------
// interface curvature for the surface-tension force (CSF term of the momentum equation)
// ---------------------------------------------------------------------------------
// signed curvature of the circle through A, B, C: positive when A -> B -> C turns left
__device__ inline double menger(double2 A, double2 B, double2 C) {
    double abx = B.x - A.x, aby = B.y - A.y, bcx = C.x - B.x, bcy = C.y - B.y;
    double cross = abx * bcy - aby * bcx;
    double den = sqrt(abx * abx + aby * aby) * sqrt(bcx * bcx + bcy * bcy) *
                 sqrt((C.x - A.x) * (C.x - A.x) + (C.y - A.y) * (C.y - A.y));
    return den > 0.0 ? 2.0 * cross / den : 0.0;
}

// grid position of the marker linked, through the cell across cell-edge k of (i, j), to the
// marker on that edge; false at a domain boundary or if that cell has no such segment
__device__ inline bool across(const Grid& g, const uint16_t* cseg, const double* hpos, const double* vpos, int i,
                              int j, int k, double2* R) {
    int in = i + (k == 1) - (k == 3), jn = j + (k == 2) - (k == 0);
    if (in < 0 || in >= g.nx || jn < 0 || jn >= g.ny) return false;
    int kk = (k + 2) & 3;
    uint16_t code = cseg[cidx(g, in, jn)];
    for (int s = 0; s < seg_count(code); ++s) {
        int kP = seg_P(code, s), kQ = seg_Q(code, s);
        int ko = kP == kk ? kQ : (kQ == kk ? kP : -1);
        if (ko < 0) continue;
        double2 m = marker_local(g, hpos, vpos, ko, in, jn);
        *R = make_double2(in + m.x, jn + m.y);
        return true;
    }
    return false;
}

// Curvature kappa = div n (n from liquid into vapour) of every cut cell, from the markers: for
// its segment P -> Q (liquid on the left) and the chain neighbours R_P before P and R_Q after Q,
// the mean of the curvatures of the circles through (R_P, P, Q) and (P, Q, R_Q) (one circle
// where a neighbour is missing), plus n_r / r on axisymmetric grids; two segments: the
// length-weighted mean; NaN where undefined or not cut.  Grid units in, physical curvature out.
__global__ void k_curvature(Grid g, const uint8_t* __restrict__ flags, const uint16_t* __restrict__ cseg,
                            const double* __restrict__ hpos, const double* __restrict__ vpos,
                            double* __restrict__ kap) {
    const long long zo = zoff(g.zs);
    flags = zsh(flags, zo);
    cseg = zsh(cseg, zo);
    hpos = zsh(hpos, zo);
    vpos = zsh(vpos, zo);
    kap = zsh(kap, zo);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    int c = cidx(g, i, j);
    double out = nan("");
    if (flags[c] & F_CUT) {
        uint16_t code = cseg[c];
        double num = 0.0, den = 0.0;
        for (int s = 0; s < seg_count(code); ++s) {
            int kP = seg_P(code, s), kQ = seg_Q(code, s);
            double2 P = marker_local(g, hpos, vpos, kP, i, j), Q = marker_local(g, hpos, vpos, kQ, i, j);
            P = make_double2(i + P.x, j + P.y);
            Q = make_double2(i + Q.x, j + Q.y);
            double2 R;
            double sum = 0.0;
            int nk = 0;
            if (across(g, cseg, hpos, vpos, i, j, kP, &R)) { sum += menger(R, P, Q); ++nk; }
            if (across(g, cseg, hpos, vpos, i, j, kQ, &R)) { sum += menger(P, Q, R); ++nk; }
            if (!nk) continue;
            double L = sqrt((Q.x - P.x) * (Q.x - P.x) + (Q.y - P.y) * (Q.y - P.y));
            double k2 = sum / nk;
            // axisymmetric: the azimuthal curvature n_r / r at the segment's midpoint (grid units)
            if (g.axi) k2 += ((Q.y - P.y) / L) / (g.r0 + 0.5 * (P.x + Q.x));
            num += L * k2;
            den += L;
        }
        if (den > 0.0) out = num / den * g.inv_h;
    }
    kap[c] = out;
}

// ---------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------

void launch_curvature(const Grid& g, const uint8_t* flags, const uint16_t* cseg, const double* hpos,
                      const double* vpos, double* kap, cudaStream_t st) {
    k_curvature<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, flags, cseg, hpos, vpos, kap);
}

void launch_check_interface(const Grid& g, const uint8_t* vcol, double* hpos, double* vpos, int* err,
                            cudaStream_t st) {
    long long n = (long long)(g.nx + 1) * (g.ny + 1);
    k_check_interface<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, vcol, hpos, vpos, err);
}

void launch_reconstruct(const Grid& g, const uint8_t* vcol, const double* hpos, const double* vpos,
                        uint16_t* cseg, uint8_t* flags, double* vf, cudaStream_t st) {
    k_reconstruct<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, vcol, hpos, vpos, cseg, flags, vf);
}

void launch_band(const Grid& g, const uint16_t* cseg, const double* hpos, const double* vpos, uint8_t* flags,
                 double2* nb, cudaStream_t st) {
    k_band<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, cseg, hpos, vpos, flags, nb);
}

// blocks of a kernel over the cells near the interface (four threads per cell): about 20 cells
// per unit of interface length across the grid (nx + ny), four blocks per SM at most; the
// kernels stride over the list, so a longer interface only takes more iterations.  A batch
// shares about two blocks per SM slot among its instances (at least one each), instead of
// launching each instance's count of mostly idle blocks.
static int list_blocks(const Grid& g) {
    long long n = div_up(80LL * (g.nx + g.ny), 256);
    n = n < 4 ? 4 : (n > 4 * 152 ? 4 * 152 : n);
    if (g.nz > 1) {
        long long per = (2LL * 4 * 152) / g.nz;
        n = n < per ? n : (per < 1 ? 1 : per);
    }
    return (int)n;
}

void launch_reconstruct_list(const Grid& g, const int* list, const int* count, const uint8_t* vcol,
                             const double* hpos, const double* vpos, uint16_t* cseg, uint8_t* flags, double* vf,
                             cudaStream_t st) {
    k_reconstruct_list<<<dim3(list_blocks(g), 1, g.nz), 256, 0, st>>>(g, list, count, vcol, hpos, vpos, cseg,
                                                                      flags, vf);
}

void launch_band_list(const Grid& g, const int* list, const int* count, const uint16_t* cseg, const double* hpos,
                      const double* vpos, uint8_t* flags, double2* nb, cudaStream_t st) {
    k_band_list<<<dim3(list_blocks(g), 1, g.nz), 256, 0, st>>>(g, list, count, cseg, hpos, vpos, flags, nb);
}

// the same byte range of every instance of the launch (instances lie g.zs bytes apart)
static void copy_all(void* dst, const void* src, size_t bytes, const Grid& g, cudaStream_t st) {
    if (g.nz > 1) cudaMemcpy2DAsync(dst, (size_t)g.zs, src, (size_t)g.zs, bytes, g.nz, cudaMemcpyDeviceToDevice, st);
    else cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
}
static void zero_all(void* dst, size_t bytes, const Grid& g, cudaStream_t st) {
    if (g.nz > 1) cudaMemset2DAsync(dst, (size_t)g.zs, 0, bytes, g.nz, st);
    else cudaMemsetAsync(dst, 0, bytes, st);
}

void launch_band_dilate(const Grid& g, const int* band, const int* nband, int* mark, int* list, int* count,
                        cudaStream_t st) {
    zero_all(count, sizeof(int), g, st);
    k_band_dilate<<<dim3(list_blocks(g), 1, g.nz), 256, 0, st>>>(g, band, nband, mark, list, count);
}

void launch_band_unmark(const Grid& g, const int* list, const int* count, int* mark, cudaStream_t st) {
    k_band_unmark<<<dim3(list_blocks(g), 1, g.nz), 256, 0, st>>>(g, list, count, mark);
}

void launch_ug_list(const Grid& g, const Phys& p, const int* list, const int* count, const uint8_t* flags,
                    const double2* u_l, const double2* u_v, const double* mdot, const double2* nb, double2* uG,
                    cudaStream_t st) {
    k_ug_list<<<dim3(list_blocks(g), 1, g.nz), 256, 0, st>>>(g, p, list, count, flags, u_l, u_v, mdot, nb, uG);
}

void launch_sweep(const Grid& g, int axis, double dth, const int* list, const int* count, const uint8_t* vcol,
                  const double* hpos, const double* vpos, const uint16_t* cseg, const double2* uG, double* hdisp,
                  double* vdisp, uint8_t* vcol_n, double* hpos_n, double* vpos_n, int* status, cudaStream_t st) {
    int nb_ = list_blocks(g);
    k_displace_list<<<dim3(nb_, 1, g.nz), 256, 0, st>>>(g, axis, dth, list, count, vcol, hpos, vpos, uG, hdisp,
                                                         vdisp, status);
    size_t nv = (size_t)(g.nx + 1) * (g.ny + 1), nh = (size_t)(g.ny + 1) * g.nx, nve = (size_t)g.ny * (g.nx + 1);
    copy_all(vcol_n, vcol, nv, g, st);
    SweepView sv{g, axis, vcol, hpos, vpos, hdisp, vdisp};
    k_sweep_vertices_list<<<dim3(nb_, 1, g.nz), 256, 0, st>>>(sv, list, count, vcol_n);
    zero_all(hpos_n, nh * sizeof(double), g, st);
    zero_all(vpos_n, nve * sizeof(double), g, st);
    k_sweep_edges_list<<<dim3(nb_, 1, g.nz), 256, 0, st>>>(sv, list, count, cseg, vcol_n,
                                                           axis == 0 ? hpos_n : vpos_n,
                                                           axis == 0 ? vpos_n : hpos_n, status);
}

void launch_energy_operator(const Grid& g, const Phys& p, const uint8_t* flags, const uint16_t* cseg,
                            const double* hpos, const double* vpos, const double* Ts_l, const double* Ts_v,
                            double* cd, double* dd, double* wl, double* wb, double* b, double* x0,
                            cudaStream_t st) {
    auto k = g.axi ? k_energy_operator<true> : k_energy_operator<false>;
    k<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, p, flags, cseg, hpos, vpos, Ts_l, Ts_v, cd, dd, wl, wb, b,
                                                          x0);
}

void launch_mass_flux(const Grid& g, const Phys& p, const uint16_t* cseg, const double* hpos,
                      const double* vpos, const double* T_l, const double* T_v, double* mdot, cudaStream_t st) {
    k_mass_flux<<<rows_grid(g.nx, g.ny, 128, g.nz), 128, 0, st>>>(g, p, cseg, hpos, vpos, T_l, T_v, mdot);
}

}  // namespace ebit
