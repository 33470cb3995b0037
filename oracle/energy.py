"""Per-phase energy equation: advection, extension, sharp-interface diffusion, mass flux.

Paper Sec. 2.4:
  * energy-advection equation: T* = T - dt u_k . grad T_k, third-order WENO
    (Jiang & Shu) upwind derivatives;
  * extrapolation equation: pseudo-time upwind transport along +n (liquid into
    vapour) or -n (vapour into liquid), restricted to the narrow band;
  * energy-diffusion equation with T_Gamma = T_sat imposed through the ghost
    value of the ghost-temperature equation, which turns the arm of a cut link
    into lambda (T_sat - T_i) / (theta h^2) (Txx-ghost equation);
  * mass-flux equation mdot = [q] / h_lg with one-sided normal gradients from two
    points on the normal (normal-gradient equation, Fig. 3b).

Readings:
  * WENO3: two candidate stencils, linear weights 1/3 and 2/3, smoothness
    indicators from undivided differences, epsilon 1e-6, upwinding by the sign of
    the cell velocity of the phase;
  * the extension is iterated with the local pseudo-time step that makes each
    Jacobi update the steady upwind balance
    f_i = (|n_x| f_upx + |n_y| f_upy) / (|n_x| + |n_y|), a fixed number of sweeps;
    T*_k is extended from the phase-k cells of the pre-advection interface (this
    fills the cells the interface sweeps over), and T_k again after the diffusion
    solve (ghost values for the flux and the next advection); mdot is extended
    from the cut cells, along +n into vapour and -n into liquid;
  * the two per-phase diffusion systems share no unknown (a cut link is a
    Dirichlet condition for both sides), so they are assembled as one
    block-diagonal system over all cells; a wall with fixed temperature is a
    Dirichlet face (ghost value 2 T_w - T_i);
  * normal-gradient points at d1 = 1.5 h and d2 = 2.5 h from the segment
    midpoint along the segment normal into each phase, values by biquadratic
    (3x3 Lagrange) interpolation of that phase's field, ghost band included;
    a = [(T1 - T_sat) d2/d1 - (T2 - T_sat) d1/d2] / (d2 - d1) is dT/ds at the
    interface with s the distance into the phase, and
    mdot = (lambda_l a_l + lambda_v a_v) / h_lg (positive for evaporation; with
    n pointing from liquid into vapour this is the mass-flux equation with the
    sign that the jump conditions of Sec. 2.2 need);
    a cell with two segments takes the length-weighted mean.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .geometry import link_thetas, segment_data

WENO_EPS = 1e-6
D1, D2 = 1.5, 2.5


# --------------------------------------------------------------------------
# axisymmetric metric (Sec. 3.4-3.7 run axisymmetric)
# --------------------------------------------------------------------------
def metric(pb):
    """Radius in cells of the cell centres [ny, nx], x-faces [ny, nx+1] and y-faces [ny+1, nx]
    (x is the radius r; a ring of radius r has 2 pi r times the planar area or length); all ones
    for a planar problem.  Every integrated balance -- a row of the energy, viscous and Poisson
    systems, a volume, a face flux -- is multiplied by the radius of the cell or face it lives
    on; the axis faces (r = 0) carry no flux."""
    ny, nx = pb.ny, pb.nx
    if not pb.axi:
        return np.ones((ny, nx)), np.ones((ny, nx + 1)), np.ones((ny + 1, nx))
    r0 = pb.x0 / pb.h
    mc = np.tile(r0 + np.arange(nx) + 0.5, (ny, 1))
    mfx = np.tile(r0 + np.arange(nx + 1, dtype=float), (ny, 1))
    mfy = np.tile(r0 + np.arange(nx) + 0.5, (ny + 1, 1))
    return mc, mfx, mfy


# --------------------------------------------------------------------------
# boundary ghost layers
# --------------------------------------------------------------------------
def pad_scalar(F, sides, layers=2):
    """Pad F [ny, nx] with ghost cells; sides[s] = ('even', _) or ('odd', value) per left/right/bottom/top."""
    ny, nx = F.shape
    P = np.zeros((ny + 2 * layers, nx + 2 * layers))
    P[layers:-layers, layers:-layers] = F
    for L in range(layers):
        # x
        for s, (dst, src) in ((0, (layers - 1 - L, layers + L)), (1, (layers + nx + L, layers + nx - 1 - L))):
            mode, val = sides[s]
            col = P[layers:-layers, src]
            P[layers:-layers, dst] = col if mode == "even" else 2.0 * val - col
    for L in range(layers):
        for s, (dst, src) in ((2, (layers - 1 - L, layers + L)), (3, (layers + ny + L, layers + ny - 1 - L))):
            mode, val = sides[s]
            row = P[src, :]
            P[dst, :] = row if mode == "even" else 2.0 * val - row
    return P


def temperature_sides(T_bc):
    return [("even", 0.0) if v is None else ("odd", float(v)) for v in T_bc]


def velocity_sides(bc, comp):
    """Reflection modes of velocity component comp: normal component odd at walls and
    symmetry planes, tangential odd at no-slip walls, everything even at outflow."""
    out = []
    for s, kind in enumerate(bc):
        axis = 0 if s < 2 else 1
        if kind == 1:       # outflow
            out.append(("even", 0.0))
        elif kind == 0:     # wall
            out.append(("odd", 0.0))
        else:               # symmetry
            out.append(("odd", 0.0) if comp == axis else ("even", 0.0))
    return out


# --------------------------------------------------------------------------
# S1: WENO3 advection (energy-advection equation)
# --------------------------------------------------------------------------
def weno3_derivative(P, upos, axis, layers=2):
    """Undivided upwind WENO3 derivative of the padded field P along axis; upos: u >= 0."""
    ny, nx = P.shape[0] - 2 * layers, P.shape[1] - 2 * layers

    def sh(k):
        if axis == 0:
            return P[layers:layers + ny, layers + k:layers + k + nx]
        return P[layers + k:layers + k + ny, layers:layers + nx]

    Tm2, Tm1, T0, Tp1, Tp2 = sh(-2), sh(-1), sh(0), sh(1), sh(2)
    v1 = np.where(upos, Tm1 - Tm2, Tp2 - Tp1)
    v2 = np.where(upos, T0 - Tm1, Tp1 - T0)
    v3 = np.where(upos, Tp1 - T0, T0 - Tm1)
    phi0 = 0.5 * (3.0 * v2 - v1)
    phi1 = 0.5 * (v2 + v3)
    b0 = (v2 - v1) ** 2
    b1 = (v3 - v2) ** 2
    a0 = (1.0 / 3.0) / (WENO_EPS + b0) ** 2
    a1 = (2.0 / 3.0) / (WENO_EPS + b1) ** 2
    return (a0 * phi0 + a1 * phi1) / (a0 + a1)


def advect(F, u, sides, dt, h):
    """F* = F - dt (u . grad F), WENO3 upwind (energy-advection equation)."""
    P = pad_scalar(F, sides)
    dx = weno3_derivative(P, u[..., 0] >= 0.0, 0)
    dy = weno3_derivative(P, u[..., 1] >= 0.0, 1)
    return F - (dt / h) * (u[..., 0] * dx + u[..., 1] * dy)


def advect_phases(T_l, T_v, u_l, u_v, ccol, T_bc, dt, h):
    """Energy advection of each phase on the cells of that phase (the energy-advection equation
    is written per phase, T*_k = T_k - dt u_k . grad T_k in phase k; centre colours of the
    interface before it moves).  Elsewhere T*_k keeps T_k: the band cells of the other phase
    are refilled by the extension from the phase-k cells, and cells beyond the band are not
    read by any phase-k update."""
    sides = temperature_sides(T_bc)
    Ts_l = np.where(ccol == 1, advect(T_l, u_l, sides, dt, h), T_l)
    Ts_v = np.where(ccol == 0, advect(T_v, u_v, sides, dt, h), T_v)
    return Ts_l, Ts_v


# --------------------------------------------------------------------------
# S6: narrow-band extension (extrapolation equation)
# --------------------------------------------------------------------------
def extend(f, update, nb, sgn, iters):
    """Jacobi sweeps of the upwind steady balance of the extrapolation equation.

    update: cells whose value is extended; sgn: +1 (transport along +n) or -1 (along -n) per cell.
    """
    ny, nx = f.shape
    f = f.copy()
    dx = nb[..., 0] * sgn
    dy = nb[..., 1] * sgn
    js, is_ = np.nonzero(update)
    for _ in range(iters):
        old = f.copy()
        for j, i in zip(js, is_):
            ax = dx[j, i]
            ay = dy[j, i]
            acc = 0.0
            w = 0.0
            if ax > 0.0 and i - 1 >= 0:
                acc += ax * old[j, i - 1]
                w += ax
            elif ax < 0.0 and i + 1 < nx:
                acc += -ax * old[j, i + 1]
                w += -ax
            if ay > 0.0 and j - 1 >= 0:
                acc += ay * old[j - 1, i]
                w += ay
            elif ay < 0.0 and j + 1 < ny:
                acc += -ay * old[j + 1, i]
                w += -ay
            if w > 0.0:
                f[j, i] = acc / w
    return f


def extend_temperatures(T_l, T_v, geom, iters):
    """Fill the ghost band of each phase's temperature from that phase (liquid along +n, vapour along -n)."""
    ones = np.ones(T_l.shape)
    T_l = extend(T_l, geom.band & (geom.ccol == 0), geom.nb, ones, iters)
    T_v = extend(T_v, geom.band & (geom.ccol == 1), geom.nb, -ones, iters)
    return T_l, T_v


def extend_mdot(mdot_cut, geom, iters):
    """Extend mdot from the cut cells over the narrow band."""
    sgn = np.where(geom.ccol == 0, 1.0, -1.0)
    m = np.where(geom.nseg > 0, mdot_cut, 0.0)
    return extend(m, geom.band & (geom.nseg == 0), geom.nb, sgn, iters)


# --------------------------------------------------------------------------
# S7 + S8: ghost-fluid coefficients and the implicit diffusion solve
# --------------------------------------------------------------------------
def assemble_energy(geom, Tstar_l, Tstar_v, pb):
    """Sparse matrix and RHS of the energy-diffusion equation for both phases (one block-diagonal system).

    Row of cell i in phase k, multiplied by the cell area:
      [h^2 (rho cp)_k / dt + sum_regular lambda_k + sum_cut lambda_k / theta + sum_Tfixed-walls 2 lambda_k] T_i
      - sum_regular lambda_k T_j = h^2 (rho cp)_k / dt T*_i + sum_cut lambda_k T_sat / theta + sum 2 lambda_k T_w
    """
    nx, ny, h = pb.nx, pb.ny, pb.h
    mc, mfx, mfy = metric(pb)
    th = link_thetas(geom, pb.theta_min)
    liq = geom.ccol == 1
    lam = np.where(liq, pb.lam_l, pb.lam_v)
    rc = np.where(liq, pb.rho_l * pb.cp_l, pb.rho_v * pb.cp_v)
    coef = h * h * rc / pb.dt * mc
    diag = coef.copy()
    b = coef * np.where(liq, Tstar_l, Tstar_v)
    idx = np.arange(nx * ny).reshape(ny, nx)
    rows, cols, vals = [], [], []
    # regular links between two cells of the same phase
    sx = geom.ccol[:, :-1] == geom.ccol[:, 1:]
    wx = np.where(sx, lam[:, :-1], 0.0) * mfx[:, 1:-1]
    sy = geom.ccol[:-1, :] == geom.ccol[1:, :]
    wy = np.where(sy, lam[:-1, :], 0.0) * mfy[1:-1, :]
    diag[:, :-1] += wx
    diag[:, 1:] += wx
    diag[:-1, :] += wy
    diag[1:, :] += wy
    for w, a, c in ((wx, idx[:, :-1], idx[:, 1:]), (wy, idx[:-1, :], idx[1:, :])):
        m = w != 0.0
        rows += [a[m], c[m]]
        cols += [c[m], a[m]]
        vals += [-w[m], -w[m]]
    # cut links: Dirichlet T_sat at distance theta h
    for (j, i, side), t in th.items():
        mf = (mfx[j, i + 1], mfx[j, i], mfy[j + 1, i], mfy[j, i])[side]   # the face the link crosses
        lk = lam[j, i] * mf
        diag[j, i] += lk / t
        b[j, i] += lk * pb.T_sat / t
    # domain walls with fixed temperature
    for side, Tb in enumerate(pb.T_bc):
        if Tb is None:
            continue
        sl = {0: (slice(None), 0), 1: (slice(None), nx - 1), 2: (0, slice(None)), 3: (ny - 1, slice(None))}[side]
        mf = (mfx[:, 0], mfx[:, -1], mfy[0, :], mfy[-1, :])[side]
        diag[sl] += 2.0 * lam[sl] * mf
        b[sl] += 2.0 * lam[sl] * mf * Tb
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx * ny, nx * ny))
    return A, b.ravel()


def solve_energy(geom, Tstar_l, Tstar_v, pb):
    A, b = assemble_energy(geom, Tstar_l, Tstar_v, pb)
    T = spla.spsolve(A.tocsc(), b).reshape(pb.ny, pb.nx)
    liq = geom.ccol == 1
    T_l = np.where(liq, T, Tstar_l)
    T_v = np.where(liq, Tstar_v, T)
    return T_l, T_v


# --------------------------------------------------------------------------
# S9: interface heat and mass flux
# --------------------------------------------------------------------------
def interp_biquadratic(F, px, py):
    """3x3 Lagrange interpolation of the cell field F at (px, py) in grid units."""
    ny, nx = F.shape
    ic = min(max(int(math.floor(px)), 1), nx - 2)
    jc = min(max(int(math.floor(py)), 1), ny - 2)
    sx = px - (ic + 0.5)
    sy = py - (jc + 0.5)
    wx = (0.5 * sx * (sx - 1.0), 1.0 - sx * sx, 0.5 * sx * (sx + 1.0))
    wy = (0.5 * sy * (sy - 1.0), 1.0 - sy * sy, 0.5 * sy * (sy + 1.0))
    v = 0.0
    for b in range(3):
        r = 0.0
        for a in range(3):
            r += wx[a] * F[jc - 1 + b, ic - 1 + a]
        v += wy[b] * r
    return v


def normal_slope(T1, T2, T_sat, h):
    """dT/ds at the interface of the quadratic through (0, T_sat), (d1, T1), (d2, T2) (normal-gradient equation)."""
    return ((T1 - T_sat) * D2 / D1 - (T2 - T_sat) * D1 / D2) / ((D2 - D1) * h)


def mass_flux(geom, T_l, T_v, pb):
    """mdot per cut cell (mass-flux equation), zero elsewhere."""
    m = np.zeros((pb.ny, pb.nx))
    acc = {}
    for (j, i), (mx, my), n, L in segment_data(geom):
        Tv1 = interp_biquadratic(T_v, mx + D1 * n[0], my + D1 * n[1])
        Tv2 = interp_biquadratic(T_v, mx + D2 * n[0], my + D2 * n[1])
        Tl1 = interp_biquadratic(T_l, mx - D1 * n[0], my - D1 * n[1])
        Tl2 = interp_biquadratic(T_l, mx - D2 * n[0], my - D2 * n[1])
        a_v = normal_slope(Tv1, Tv2, pb.T_sat, pb.h)
        a_l = normal_slope(Tl1, Tl2, pb.T_sat, pb.h)
        ms = (pb.lam_l * a_l + pb.lam_v * a_v) / pb.h_lg
        s = acc.setdefault((j, i), [0.0, 0.0])
        s[0] += L * ms
        s[1] += L
    for (j, i), (num, den) in acc.items():
        m[j, i] = num / den if den > 0 else 0.0
    return m
