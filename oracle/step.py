"""State, preparation and the time iteration of Sec. 2.5; diagnostics of Sec. 3.

One time step, in the paper's order (Sec. 2.5):
  1. energy advection (S1) and extension of T* into the cells the interface will
     sweep (S6);
  2. interface advection by EBIT (S2 interfacial velocity, S3/S4 sweeps, S5
     reconnection);
  3. energy diffusion with the sharp T = T_sat condition (S7 ghost-fluid
     coefficients, S8 solve), then the ghost band of T is refilled;
  4. mass flux (S9) extended over the band, ghost velocities (S10);
  5. mass and momentum: predictor (S11) and ghost-fluid projection (S12).
Diagnostics (S13): vapour volume, the volume the mass flux should have added,
M_d (mass-in-domain equation) and the outlet mass of M_c (mass-with-outflow
equation); for film boiling (Sec. 3.7) the vapour volume that left through the
outflow boundaries (the V_bc of the dimensionless vapour volume) and the
space-averaged Nusselt number of the heated wall.  Axisymmetric problems report
volumes, masses and fluxes of the full ring (2 pi r times the planar measure).

Readings of the two film-boiling quantities (the paper gives the integrals only):
  * V_bc per step: over the outflow boundary faces, (1 - H) u_f . n h dt with H
    the boundary cell's liquid volume fraction and u_f the face velocity of the
    cell's phase (the same faces and velocities as the outlet mass of M_c);
  * Nu = (l / (T_w - T_sat)) times the mean over the faces of the walls with a
    fixed temperature of -dT/dn at the wall, dT/dn from the cell and its ghost
    value 2 T_w - T_i, i.e. 2 (T_w - T_i) / h, T_i of the cell's phase; the
    length l is the paper's sqrt(sigma / ((rho_l - rho_v) |g|)) when sigma and g
    are nonzero, else 1 (the mean wall gradient over the wall superheat).
"""
from __future__ import annotations

import math

import numpy as np

from . import energy, flow, sweep
from .geometry import reconstruct, segment_data


class State:
    """Full oracle state; pb is the Problem (grid, properties, boundary conditions)."""

    def __init__(self, pb):
        self.pb = pb
        self.vcol = pb.vcol.copy()
        self.hx_pos = np.where(pb.vcol[:, :-1] != pb.vcol[:, 1:], pb.hx_pos, 0.0)
        self.vy_pos = np.where(pb.vcol[:-1, :] != pb.vcol[1:, :], pb.vy_pos, 0.0)
        self.T_l = pb.T_l.copy()
        self.T_v = pb.T_v.copy()
        self.u_l = pb.u_l.copy()
        self.u_v = pb.u_v.copy()
        self.ufx_l = pb.ufx_l.copy()
        self.ufx_v = pb.ufx_v.copy()
        self.ufy_l = pb.ufy_l.copy()
        self.ufy_v = pb.ufy_v.copy()
        self.p = pb.p.copy()
        self.gc = np.zeros(pb.u_l.shape)
        self.mdot = np.zeros((pb.ny, pb.nx))
        self.geom = None
        self.t = pb.t0
        self.nstep = 0
        self.diag = []

    def copy(self):
        import copy
        return copy.deepcopy(self)


def interface_mdot(st):
    """mdot on the cut cells (mass-flux equation, or the imposed value), extended over the band."""
    pb, g = st.pb, st.geom
    if pb.energy:
        m = energy.mass_flux(g, st.T_l, st.T_v, pb)
    else:
        m = np.where(g.nseg > 0, pb.mdot_fixed, 0.0)
    return energy.extend_mdot(m, g, pb.extend_iters)


def prepare(pb):
    """Initial state: reconstruction, ghost band of T, mdot, ghost velocities, initial accelerations."""
    st = State(pb)
    if pb.one_fluid:       # one velocity field, held in both phase arrays
        st.u_v, st.ufx_v, st.ufy_v = st.u_l.copy(), st.ufx_l.copy(), st.ufy_l.copy()
    st.geom = reconstruct(st.vcol, st.hx_pos, st.vy_pos)
    if pb.energy:
        st.T_l, st.T_v = energy.extend_temperatures(st.T_l, st.T_v, st.geom, pb.extend_iters)
    st.mdot = interface_mdot(st)
    flow.ghost_velocities(st)
    rfx, rfy = flow.face_rho(pb, st.geom.vf)
    ax, ay = flow.face_acceleration(pb, st.p, rfx, rfy, flow.surface_tension_faces(pb, st.geom, rfx, rfy))
    st.gc = flow.faces_to_cells(ax, ay)
    return st


def advance_interface(st):
    """S2-S5: dimension-split EBIT advection with u_Gamma from the start-of-step state."""
    pb = st.pb
    g0 = st.geom
    uG = sweep.interface_velocity_cells(st.u_l, st.u_v, g0.ccol, st.mdot, g0.nb, pb.rho_l, pb.rho_v)
    dth = pb.dt / pb.h
    order = (0, 1) if (pb.sweep_order == 0 or st.nstep % 2 == 0) else (1, 0)
    g = g0
    for axis in order:
        st.vcol, st.hx_pos, st.vy_pos = sweep.sweep(st.vcol, st.hx_pos, st.vy_pos, g, uG, dth, axis, pb.bc)
        g = reconstruct(st.vcol, st.hx_pos, st.vy_pos)
    st.geom = g


def step(st):
    """Advance st by one time step in place; returns the diagnostics row."""
    pb = st.pb
    g_old = st.geom
    # 1. energy advection + extension of T* (old interface)
    if pb.energy:
        Ts_l, Ts_v = energy.advect_phases(st.T_l, st.T_v, st.u_l, st.u_v, g_old.ccol, pb.T_bc, pb.dt, pb.h)
        Ts_l, Ts_v = energy.extend_temperatures(Ts_l, Ts_v, g_old, pb.extend_iters)
    # 2. interface advection
    advance_interface(st)
    g = st.geom
    # 3. energy diffusion (new interface) and ghost band
    if pb.energy:
        st.T_l, st.T_v = energy.solve_energy(g, Ts_l, Ts_v, pb)
        st.T_l, st.T_v = energy.extend_temperatures(st.T_l, st.T_v, g, pb.extend_iters)
    # 4. mass flux and ghost velocities
    st.mdot = interface_mdot(st)
    flow.ghost_velocities(st)
    # 5. momentum predictor and projection
    ustar, faces = flow.predictor(st, st.gc)
    flow.project(st, ustar, faces)
    st.t += pb.dt
    st.nstep += 1
    row = diagnostics(st)
    st.diag.append(row)
    return row


def nusselt_length(pb):
    g = math.hypot(pb.gx, pb.gy)
    if pb.sigma > 0.0 and g > 0.0 and pb.rho_l != pb.rho_v:
        return math.sqrt(pb.sigma / (abs(pb.rho_l - pb.rho_v) * g))
    return 1.0


def diagnostics(st):
    """[t, vapour volume, dV expected from mdot this step, M_d, outlet mass this step, cut cells,
    vapour volume out of the outflow boundaries this step, wall Nusselt number]."""
    pb, g = st.pb, st.geom
    h2 = pb.h * pb.h
    # volumes and face areas: per unit depth (planar) or of the ring, 2 pi r times (axisymmetric)
    mc, mfx, mfy = energy.metric(pb)
    ring = 2.0 * math.pi * pb.h if pb.axi else 1.0
    Vv = float(np.sum((1.0 - g.vf) * mc)) * h2 * ring
    mS = 0.0
    for (j, i), (mx, my), _, L in segment_data(g):
        mS += st.mdot[j, i] * L * pb.h * ((pb.x0 / pb.h + mx) * ring if pb.axi else 1.0)
    dV = mS * pb.dt / pb.rho_v
    rho_c, _ = flow.mixture(pb, g.vf)
    Md = float(np.sum(rho_c * mc)) * h2 * ring
    out = 0.0
    ccol = g.ccol
    for s, kind in enumerate(pb.bc):
        if kind != flow.OUTFLOW:
            continue
        if s == 0:
            u = np.where(ccol[:, 0] == 1, st.ufx_l[:, 0], st.ufx_v[:, 0])
            out += float(np.sum(-rho_c[:, 0] * u * mfx[:, 0]))
        elif s == 1:
            u = np.where(ccol[:, -1] == 1, st.ufx_l[:, -1], st.ufx_v[:, -1])
            out += float(np.sum(rho_c[:, -1] * u * mfx[:, -1]))
        elif s == 2:
            u = np.where(ccol[0, :] == 1, st.ufy_l[0, :], st.ufy_v[0, :])
            out += float(np.sum(-rho_c[0, :] * u * mfy[0, :]))
        else:
            u = np.where(ccol[-1, :] == 1, st.ufy_l[-1, :], st.ufy_v[-1, :])
            out += float(np.sum(rho_c[-1, :] * u * mfy[-1, :]))
    out *= pb.h * pb.dt * ring
    # vapour volume through the outflow faces, and the heat flux of the fixed-temperature walls
    vout, flux, nf = 0.0, 0.0, 0
    for s, kind in enumerate(pb.bc):
        cells = {0: (slice(None), 0), 1: (slice(None), -1), 2: (0, slice(None)), 3: (-1, slice(None))}[s]
        liq = ccol[cells] == 1
        if kind == flow.OUTFLOW:
            if s < 2:
                u = np.where(liq, st.ufx_l[:, 0 if s == 0 else -1], st.ufx_v[:, 0 if s == 0 else -1])
                mf = mfx[:, 0 if s == 0 else -1]
            else:
                u = np.where(liq, st.ufy_l[0 if s == 2 else -1, :], st.ufy_v[0 if s == 2 else -1, :])
                mf = mfy[0 if s == 2 else -1, :]
            sign = -1.0 if s in (0, 2) else 1.0
            vout += float(np.sum((1.0 - g.vf[cells]) * sign * u * mf))
        if pb.T_bc[s] is not None and kind == flow.WALL:
            Tw = float(pb.T_bc[s])
            Ti = np.where(liq, st.T_l[cells], st.T_v[cells])
            flux += float(np.sum(2.0 * (Tw - Ti) / pb.h))
            nf += Ti.size
    vout *= pb.h * pb.dt * ring
    nu = 0.0
    if nf:
        Tw = next(float(v) for s, v in enumerate(pb.T_bc) if v is not None and pb.bc[s] == flow.WALL)
        nu = nusselt_length(pb) / (Tw - pb.T_sat) * flux / nf if Tw != pb.T_sat else 0.0
    return np.array([st.t, Vv, dV, Md, out, float(np.count_nonzero(g.nseg)), vout, nu])


def run(pb, steps=None):
    st = prepare(pb)
    for _ in range(pb.steps if steps is None else steps):
        step(st)
    return st
