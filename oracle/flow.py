"""Mass and momentum: ghost velocities, momentum predictor, ghost-fluid projection.

Paper Sec. 2.3:
  * ghost-velocity equation: in the narrow band, u_vap = u_liq - mdot [1/rho] n where
    f_C = 1 and u_liq = u_vap + mdot [1/rho] n where f_C = 0, [1/rho] = 1/rho_l - 1/rho_v,
    for cell and face velocities;
  * discretization equations 1-3 solved separately for the liquid and the vapour
    velocity fields (time-staggered approximate projection on a collocated grid);
  * ghost-fluid Poisson equation: div(dt/rho_f grad p) = div u*_{f,liq} where
    f_C = 1, div u*_{f,vap} where f_C = 0; face update (discretization equation 4)
    for both fields and the cell update (discretization equation 5).

Readings (the paper gives Eqs. 11-15 only):
  * rho_c, mu_c are the property average of the cell volume fraction; face values
    use the mean of the two cells' volume fractions (rho_f) or of their mu_c (mu_f);
  * advection u . grad u with the WENO3 upwind derivative of the energy equation
    (in place of the BCG scheme, whose equations the paper does not print);
  * viscous term div(mu_f grad u*) implicit (backward Euler, the form of Eq. 11);
    the transpose part of the stress is not included;
  * the pressure-gradient / body-force term of Eqs. 11-15 is the face acceleration
    a_f = g - grad_f p / rho_f averaged to cells (f->c: mean of the two faces; c->f:
    mean of the two cells), with a_f = 0 on walls and symmetry planes;
  * boundaries: no-slip wall (u = 0), symmetry (normal u = 0, tangential free),
    outflow (zero normal gradient of u, p = 0 on the boundary face);
  * a face's phase (for the face ghost velocity) is the colour of its midpoint on
    the EBIT edge; mdot n at a face is the mean of its two cells;
  * the surface-tension, 2[mu du/dn] and -mdot^2 [1/rho] terms of the pressure
    jump are not imposed (the paper's projection changes only the RHS).

Surface tension (the CSF force f = sigma kappa delta_s n of the momentum equation and of
discretization equations 1-5, in the well-balanced form the paper cites): on every interior
face the acceleration sigma kappa_f (H_j - H_i) / (h rho_f) joins g - grad_f p / rho_f, with H
the liquid volume fraction; kappa_f is the mean of the two cells' curvatures where both are
defined, else the one that is, else 0.  It enters the face velocity of the predictor
(discretization eq. 3, at the interface of the new time level), the face accelerations whose
cell average gives the cell update (eq. 5) and, one step later, the predictor's old-time term
(eqs. 1-2).  Readings: kappa = div n with n from liquid into vapour (-1/R for a vapour
bubble), and the force's sign is the one that gives the pressure jump p_liq - p_vap =
sigma kappa of the pressure-jump equation, i.e. higher pressure inside a bubble or a drop.
Curvature: the paper takes height functions of the reconstructed volume fractions (Sec. 3.6);
on EBIT's polygonal volume fractions that curvature does not converge (the chord sagitta
differs from column to column and the second difference of the heights amplifies it: 12 % in
the worst cells of a 25-cell circle, at any resolution), so it is read from the markers
themselves, through the circles the EBIT sweep uses (Sec. 2.1, Fig. 1): for a cut cell's
segment P -> Q (liquid on its left) and the chain neighbours R_P before P and R_Q after Q, the
mean of the signed curvatures of the circles through (R_P, P, Q) and (P, Q, R_Q), the sign
positive when the chain turns left (a drop) -- which is div n; one circle where a neighbour is
missing (a domain boundary), none without both; a saddle cell takes the length-weighted mean of
its two segments.

One-fluid variant (Sec. 2.3, compared with the ghost-fluid method in Sec. 3): one velocity
field (kept in both the liquid and the vapour arrays, which then stay equal), no ghost
velocities, and the phase-change source of the pc-source equation added to the mass equation
of the projection, div u_f^{n+1} = S_pc, nonzero in the cut cells only:
  S_pc V = mdot S_Gamma (1/rho_v - 1/rho_l),
with S_Gamma the length of the cell's segments (times the unit depth) and V = h^2.  Reading of
the sign: the printed source is mdot S_Gamma [1/rho] / V with [.] = liquid - vapour; read with
the normal from liquid into vapour (the orientation under which the jump conditions of Sec. 2.2
hold with mdot > 0 for evaporation) the divergence of the velocity jump is (u_v - u_l) . n
delta = mdot (1/rho_v - 1/rho_l) delta, i.e. evaporation creates volume.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .energy import advect, metric, velocity_sides
from .geometry import segment_data

WALL, OUTFLOW, SYMMETRY = 0, 1, 2


def face_colours(vcol, hx_pos, vy_pos):
    """Colour at the midpoint of every x-face (vertical edge) and y-face (horizontal edge)."""
    vcut = vcol[:-1, :] != vcol[1:, :]
    cx = np.where(vcut & (vy_pos < 0.5), vcol[1:, :], vcol[:-1, :])
    hcut = vcol[:, :-1] != vcol[:, 1:]
    cy = np.where(hcut & (hx_pos < 0.5), vcol[:, 1:], vcol[:, :-1])
    return cx, cy


# --------------------------------------------------------------------------
# S10: ghost velocities
# --------------------------------------------------------------------------
def ghost_velocities(st):
    pb, g = st.pb, st.geom
    if pb.one_fluid:       # one velocity field: no ghost values
        return
    J = 1.0 / pb.rho_l - 1.0 / pb.rho_v
    mn = st.mdot[..., None] * g.nb                # mdot n per cell
    liq = (g.ccol == 1) & g.band
    vap = (g.ccol == 0) & g.band
    for c in range(2):
        st.u_v[..., c] = np.where(liq, st.u_l[..., c] - J * mn[..., c], st.u_v[..., c])
        st.u_l[..., c] = np.where(vap, st.u_v[..., c] + J * mn[..., c], st.u_l[..., c])
    cx, cy = face_colours(st.vcol, st.hx_pos, st.vy_pos)
    # x-faces 1..nx-1
    bx = g.band[:, :-1] | g.band[:, 1:]
    mfx = 0.5 * (mn[:, :-1, 0] + mn[:, 1:, 0])
    fl = bx & (cx[:, 1:-1] == 1)
    fv = bx & (cx[:, 1:-1] == 0)
    ul, uv = st.ufx_l[:, 1:-1], st.ufx_v[:, 1:-1]
    st.ufx_v[:, 1:-1] = np.where(fl, ul - J * mfx, uv)
    st.ufx_l[:, 1:-1] = np.where(fv, uv + J * mfx, ul)
    by = g.band[:-1, :] | g.band[1:, :]
    mfy = 0.5 * (mn[:-1, :, 1] + mn[1:, :, 1])
    fl = by & (cy[1:-1, :] == 1)
    fv = by & (cy[1:-1, :] == 0)
    ul, uv = st.ufy_l[1:-1, :], st.ufy_v[1:-1, :]
    st.ufy_v[1:-1, :] = np.where(fl, ul - J * mfy, uv)
    st.ufy_l[1:-1, :] = np.where(fv, uv + J * mfy, ul)


# --------------------------------------------------------------------------
# properties
# --------------------------------------------------------------------------
def mixture(pb, vf):
    rho_c = pb.rho_l * vf + pb.rho_v * (1.0 - vf)
    mu_c = pb.mu_l * vf + pb.mu_v * (1.0 - vf)
    return rho_c, mu_c


def face_rho(pb, vf):
    """rho on x-faces [ny, nx+1] and y-faces [ny+1, nx]; boundary faces take the boundary cell."""
    ny, nx = vf.shape
    vx = np.empty((ny, nx + 1))
    vx[:, 1:-1] = 0.5 * (vf[:, :-1] + vf[:, 1:])
    vx[:, 0], vx[:, -1] = vf[:, 0], vf[:, -1]
    vy = np.empty((ny + 1, nx))
    vy[1:-1, :] = 0.5 * (vf[:-1, :] + vf[1:, :])
    vy[0, :], vy[-1, :] = vf[0, :], vf[-1, :]
    return pb.rho_l * vx + pb.rho_v * (1.0 - vx), pb.rho_l * vy + pb.rho_v * (1.0 - vy)


_ACROSS = {0: (-1, 0), 1: (0, 1), 2: (1, 0), 3: (0, -1)}   # cell-edge k -> (dj, di) of the cell across it


def _menger(A, B, C):
    """Signed curvature of the circle through A, B, C (positive when A -> B -> C turns left)."""
    abx, aby = B[0] - A[0], B[1] - A[1]
    bcx, bcy = C[0] - B[0], C[1] - B[1]
    cross = abx * bcy - aby * bcx
    den = math.hypot(abx, aby) * math.hypot(bcx, bcy) * math.hypot(C[0] - A[0], C[1] - A[1])
    return 2.0 * cross / den if den > 0.0 else 0.0


def _across(geom, i, j, k):
    """Global position of the marker linked, through the cell across cell-edge k of (i, j), to
    the marker on that edge (None at a domain boundary or if that cell has no such segment)."""
    dj, di = _ACROSS[k]
    jn, in_ = j + dj, i + di
    if not (0 <= jn < geom.ny and 0 <= in_ < geom.nx):
        return None
    kk = (k + 2) % 4
    for s_, (P, Q) in enumerate(geom.seg.get((jn, in_), [])):
        if int(geom.segP[jn, in_, s_]) == kk:
            return (in_ + Q[0], jn + Q[1])
        if int(geom.segQ[jn, in_, s_]) == kk:
            return (in_ + P[0], jn + P[1])
    return None


def curvature(pb, geom):
    """Curvature (div n, n from liquid to vapour) of every cut cell from the circles through its
    segment's markers and their chain neighbours; NaN where undefined or not cut."""
    kap = np.full((geom.ny, geom.nx), np.nan)
    for (j, i), segs in geom.seg.items():
        num, den = 0.0, 0.0
        for s_, (P, Q) in enumerate(segs):
            Pg, Qg = (i + P[0], j + P[1]), (i + Q[0], j + Q[1])
            RP = _across(geom, i, j, int(geom.segP[j, i, s_]))
            RQ = _across(geom, i, j, int(geom.segQ[j, i, s_]))
            ks = [_menger(RP, Pg, Qg)] if RP is not None else []
            if RQ is not None:
                ks.append(_menger(Pg, Qg, RQ))
            if not ks:
                continue
            L = math.hypot(Qg[0] - Pg[0], Qg[1] - Pg[1])
            k2 = sum(ks) / len(ks)
            if pb.axi:   # the azimuthal curvature n_r / r at the segment's midpoint (grid units)
                k2 += ((Qg[1] - Pg[1]) / L) / (pb.x0 / pb.h + 0.5 * (Pg[0] + Qg[0]))
            num += L * k2
            den += L
        if den > 0.0:
            kap[j, i] = num / den / pb.h
    return kap


def surface_tension_faces(pb, geom, rfx, rfy):
    """sigma kappa_f (H_j - H_i) / (h rho_f) on interior faces (zero on boundary faces)."""
    ny, nx = geom.vf.shape
    sx = np.zeros((ny, nx + 1))
    sy = np.zeros((ny + 1, nx))
    if pb.sigma == 0.0:
        return sx, sy
    kap = curvature(pb, geom)
    vf = geom.vf

    def face_kappa(a, b):
        ka, kb = np.nan_to_num(a), np.nan_to_num(b)
        both = ~np.isnan(a) & ~np.isnan(b)
        return np.where(both, 0.5 * (ka + kb), ka + kb)

    kx = face_kappa(kap[:, :-1], kap[:, 1:])
    ky = face_kappa(kap[:-1, :], kap[1:, :])
    sx[:, 1:-1] = pb.sigma * kx * (vf[:, 1:] - vf[:, :-1]) / (pb.h * rfx[:, 1:-1])
    sy[1:-1, :] = pb.sigma * ky * (vf[1:, :] - vf[:-1, :]) / (pb.h * rfy[1:-1, :])
    return sx, sy


def face_acceleration(pb, p, rfx, rfy, st_faces=None):
    """a_f = g - grad_f p / rho_f (+ the surface-tension acceleration) on every face (zero on
    walls/symmetry planes)."""
    ny, nx = p.shape
    h = pb.h
    ax = np.zeros((ny, nx + 1))
    ay = np.zeros((ny + 1, nx))
    ax[:, 1:-1] = pb.gx - (p[:, 1:] - p[:, :-1]) / (h * rfx[:, 1:-1])
    ay[1:-1, :] = pb.gy - (p[1:, :] - p[:-1, :]) / (h * rfy[1:-1, :])
    if st_faces is not None:
        ax += st_faces[0]
        ay += st_faces[1]
    if pb.bc[0] == OUTFLOW:
        ax[:, 0] = pb.gx - (2.0 * p[:, 0]) / (h * rfx[:, 0])
    if pb.bc[1] == OUTFLOW:
        ax[:, -1] = pb.gx - (-2.0 * p[:, -1]) / (h * rfx[:, -1])
    if pb.bc[2] == OUTFLOW:
        ay[0, :] = pb.gy - (2.0 * p[0, :]) / (h * rfy[0, :])
    if pb.bc[3] == OUTFLOW:
        ay[-1, :] = pb.gy - (-2.0 * p[-1, :]) / (h * rfy[-1, :])
    return ax, ay


def faces_to_cells(ax, ay):
    g = np.empty(ax.shape[:1] + (ax.shape[1] - 1, 2))
    g[..., 0] = 0.5 * (ax[:, :-1] + ax[:, 1:])
    g[..., 1] = 0.5 * (ay[:-1, :] + ay[1:, :])
    return g


# --------------------------------------------------------------------------
# S11: momentum predictor
# --------------------------------------------------------------------------
def _five_point(nx, ny, wx, wy, diag_extra):
    """Sparse SPD matrix: diag_extra + sum_faces w (u_i - u_j); wx [ny, nx-1], wy [ny-1, nx]."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    diag = diag_extra.copy()
    diag[:, :-1] += wx
    diag[:, 1:] += wx
    diag[:-1, :] += wy
    diag[1:, :] += wy
    rows = [idx[:, :-1].ravel(), idx[:, 1:].ravel(), idx[:-1, :].ravel(), idx[1:, :].ravel(), idx.ravel()]
    cols = [idx[:, 1:].ravel(), idx[:, :-1].ravel(), idx[1:, :].ravel(), idx[:-1, :].ravel(), idx.ravel()]
    vals = [-wx.ravel(), -wx.ravel(), -wy.ravel(), -wy.ravel(), diag.ravel()]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nx * ny, nx * ny))


def _side_slices(nx, ny):
    return {0: (slice(None), 0), 1: (slice(None), nx - 1), 2: (0, slice(None)), 3: (ny - 1, slice(None))}


def viscous_matrix(pb, rho_c, mu_c, comp):
    """(h^2 rho_c / dt) u + sum_f mu_f (u_i - u_j) + Dirichlet boundary faces 2 mu u_i; axisymmetric:
    every term times the radius (in cells) of its cell or face, and the radial component's hoop
    term mu u_r / r^2 of the vector Laplacian (mu_c / m_c per cell in these units)."""
    ny, nx = rho_c.shape
    h = pb.h
    mc, mfx, mfy = metric(pb)
    wx = 0.5 * (mu_c[:, :-1] + mu_c[:, 1:]) * mfx[:, 1:-1]
    wy = 0.5 * (mu_c[:-1, :] + mu_c[1:, :]) * mfy[1:-1, :]
    extra = h * h * rho_c / pb.dt * mc
    sl = _side_slices(nx, ny)
    mb = (mfx[:, 0], mfx[:, -1], mfy[0, :], mfy[-1, :])
    for s, (mode, _) in enumerate(velocity_sides(pb.bc, comp)):
        if mode == "odd":
            extra[sl[s]] += 2.0 * mu_c[sl[s]] * mb[s]
    if pb.axi and comp == 0:
        extra += mu_c / mc
    return _five_point(nx, ny, wx, wy, extra)


def viscous_system(pb, g, u_l, u_v, gc, c):
    """Implicit viscous system of velocity component c (Eqs. 11-12): the Helmholtz matrix (CSC)
    and one right-hand side per phase field (columns liquid, vapour), h^2 rho_c / dt times the
    WENO3-advected component plus dt gc_c."""
    h, dt = pb.h, pb.dt
    rho_c, mu_c = mixture(pb, g.vf)
    coef = h * h * rho_c / dt * metric(pb)[0]
    A = viscous_matrix(pb, rho_c, mu_c, c).tocsc()
    sides = velocity_sides(pb.bc, c)
    rhs = []
    for u in (u_l, u_v):
        ua = advect(u[..., c], u, sides, dt, h)
        rhs.append((coef * (ua + dt * gc[..., c])).ravel())
    return A, np.stack(rhs, axis=1)


def predictor(st, gc):
    """Eqs. 11-13 for the liquid and the vapour velocity fields.  Returns u** and face u_f*."""
    pb, g = st.pb, st.geom
    ny, nx = pb.ny, pb.nx
    dt = pb.dt
    ustar = {}
    for name, u in (("l", st.u_l), ("v", st.u_v)):
        ustar[name] = np.empty_like(u)
    for c in range(2):
        A, rhs = viscous_system(pb, g, st.u_l, st.u_v, gc, c)
        sol = spla.spsolve(A, rhs)
        for k, name in enumerate(("l", "v")):
            ustar[name][..., c] = sol[:, k].reshape(ny, nx) - dt * gc[..., c]
    return ustar, predicted_faces(pb, g, ustar)


def predicted_faces(pb, g, ustar):
    """Face velocities u_f* of both phase fields from the cell values u** (Eq. 13): the mean of
    the two cells plus dt times gravity and the surface-tension acceleration on interior faces,
    the boundary cell's value plus dt g on outflow faces, zero elsewhere."""
    ny, nx = pb.ny, pb.nx
    dt = pb.dt
    faces = {}
    rfx, rfy = face_rho(pb, g.vf)
    stx, sty = surface_tension_faces(pb, g, rfx, rfy)       # new interface (eq. 3)
    for name in ("l", "v"):
        u2 = ustar[name]
        fx = np.zeros((ny, nx + 1))
        fy = np.zeros((ny + 1, nx))
        fx[:, 1:-1] = 0.5 * (u2[:, :-1, 0] + u2[:, 1:, 0]) + dt * (pb.gx + stx[:, 1:-1])
        fy[1:-1, :] = 0.5 * (u2[:-1, :, 1] + u2[1:, :, 1]) + dt * (pb.gy + sty[1:-1, :])
        if pb.bc[0] == OUTFLOW:
            fx[:, 0] = u2[:, 0, 0] + dt * pb.gx
        if pb.bc[1] == OUTFLOW:
            fx[:, -1] = u2[:, -1, 0] + dt * pb.gx
        if pb.bc[2] == OUTFLOW:
            fy[0, :] = u2[0, :, 1] + dt * pb.gy
        if pb.bc[3] == OUTFLOW:
            fy[-1, :] = u2[-1, :, 1] + dt * pb.gy
        faces[name] = (fx, fy)
    return faces


# --------------------------------------------------------------------------
# S12: projection
# --------------------------------------------------------------------------
def poisson_matrix(pb, rfx, rfy):
    ny, nx = rfx.shape[0], rfy.shape[1]
    mc, mfx, mfy = metric(pb)
    wx = pb.dt / rfx[:, 1:-1] * mfx[:, 1:-1]
    wy = pb.dt / rfy[1:-1, :] * mfy[1:-1, :]
    extra = np.zeros((ny, nx))
    if pb.bc[0] == OUTFLOW:
        extra[:, 0] += 2.0 * pb.dt / rfx[:, 0] * mfx[:, 0]
    if pb.bc[1] == OUTFLOW:
        extra[:, -1] += 2.0 * pb.dt / rfx[:, -1] * mfx[:, -1]
    if pb.bc[2] == OUTFLOW:
        extra[0, :] += 2.0 * pb.dt / rfy[0, :] * mfy[0, :]
    if pb.bc[3] == OUTFLOW:
        extra[-1, :] += 2.0 * pb.dt / rfy[-1, :] * mfy[-1, :]
    return _five_point(nx, ny, wx, wy, extra)


def poisson_rhs(pb, ccol, faces):
    """-h times the undivided divergence of the face field of each cell's phase (ghost-fluid Poisson
    equation); axisymmetric: the face fluxes weighted by their radius."""
    mc, mfx, mfy = metric(pb)
    div = {}
    for name, (fx, fy) in faces.items():
        div[name] = (mfx[:, 1:] * fx[:, 1:] - mfx[:, :-1] * fx[:, :-1]) + mc * (fy[1:, :] - fy[:-1, :])
    return -pb.h * np.where(ccol == 1, div["l"], div["v"])


def phase_change_source(pb, geom, mdot):
    """h^2 S_pc per cell (one-fluid variant, pc-source equation): mdot S_Gamma (1/rho_v - 1/rho_l)
    in the cut cells, S_Gamma = (length of the cell's segments in grid units) h."""
    src = np.zeros((pb.ny, pb.nx))
    jump = 1.0 / pb.rho_v - 1.0 / pb.rho_l
    for (j, i), (mx, my), _, L in segment_data(geom):
        m = (pb.x0 / pb.h + mx) if pb.axi else 1.0     # the segment's radius (axisymmetric)
        src[j, i] += mdot[j, i] * L * pb.h * jump * m
    return src


def project(st, ustar, faces):
    """Solve the ghost-fluid Poisson equation, update faces (Eq. 14), accelerations and cells (Eq. 15)."""
    pb, g = st.pb, st.geom
    ny, nx = pb.ny, pb.nx
    rfx, rfy = face_rho(pb, g.vf)
    A = poisson_matrix(pb, rfx, rfy).tocsc()
    b = poisson_rhs(pb, g.ccol, faces)
    if pb.one_fluid:       # div u_f^{n+1} = S_pc in the cut cells
        b = b + phase_change_source(pb, g, st.mdot)
    b = b.ravel()
    p = spla.spsolve(A, b).reshape(ny, nx)
    stf = surface_tension_faces(pb, g, rfx, rfy)
    ax, ay = face_acceleration(pb, p, rfx, rfy, stf)
    # face update: u_f^{n+1} = u_f* - dt grad_f p / rho_f on faces the projection acts on (u_f*
    # already carries dt g and dt times the surface-tension acceleration)
    gcorr_x = ax - pb.gx - stf[0]
    gcorr_y = ay - pb.gy - stf[1]
    out = {}
    for name, (fx, fy) in faces.items():
        nfx = fx + pb.dt * gcorr_x
        nfy = fy + pb.dt * gcorr_y
        for s, kind in enumerate(pb.bc):
            if kind != OUTFLOW:
                if s == 0:
                    nfx[:, 0] = 0.0
                elif s == 1:
                    nfx[:, -1] = 0.0
                elif s == 2:
                    nfy[0, :] = 0.0
                else:
                    nfy[-1, :] = 0.0
        out[name] = (nfx, nfy)
    gc = faces_to_cells(ax, ay)
    st.p = p
    st.gc = gc
    st.u_l = ustar["l"] + pb.dt * gc
    st.u_v = ustar["v"] + pb.dt * gc
    st.ufx_l, st.ufy_l = out["l"]
    st.ufx_v, st.ufy_v = out["v"]
