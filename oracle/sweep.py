"""EBIT interface advection: interfacial velocity at markers and 1D sweeps.

Paper: Sec. 2.1 (marker-motion equation and its explicit-Euler discretisation,
dimension splitting, Fig. 1) and Sec. 2.3 (interfacial-velocity jump equation,
bilinear interpolation from the four nearest cell centres, Fig. 2).

All positions are in grid units (vertex (i, j) at (i, j)).  The arithmetic is
plain IEEE double with one operation per Python operator, so that a CUDA kernel
written with the same operation order (no fused multiply-add) reproduces it
bit for bit.

Readings (the sweep details are in refs [chirco2023edge, pan2023edge], which the
paper only cites):
  * one sweep along axis a moves every marker by u_Gamma,a dt (u_Gamma
    interpolated at the marker's pre-sweep position); markers on lines parallel
    to a ("aligned") slide along their line; markers on the other lines
    ("unaligned") leave it and are discarded, except that unaligned markers on a
    domain boundary line are held on it;
  * a vertex flips colour once for every aligned marker that crosses it (a
    marker exactly on a vertex counts as lying after it);
  * new unaligned markers: where a displaced pre-sweep segment P'Q' strictly
    crosses an unaligned grid line, the crossing of the circle through P', Q' and
    R' is taken (R = chain neighbour, through the adjacent cell, of the endpoint
    nearer the line): the root nearest the straight-line (chord) crossing, if it
    lies within |P'Q'|_1 of it, else the chord crossing (also when R is missing);
    the marker is kept inside the cell row of the segment; a displaced marker
    lying exactly on an unaligned line is itself a crossing;
  * one marker per edge: an edge is cut iff its new vertex colours differ; its
    marker is the median (lower median) of the crossings that landed on it, or the
    edge midpoint if none did;
  * x then y on even steps, y then x on odd steps (sweep_order 1), the second
    sweep re-interpolating u_Gamma at the post-first-sweep positions.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import edge_key

FMIN = 1e-9
WALL, OUTFLOW, SYMMETRY = 0, 1, 2


def _parity(kind, comp, axis):
    """Reflection sign of velocity component comp across a boundary normal to axis."""
    if comp == axis:
        return 1.0 if kind == OUTFLOW else -1.0
    return -1.0 if kind == WALL else 1.0


def cell_value(F, comp, i, j, bc):
    """F[j, i, comp] with one layer of boundary ghost cells (velocity reflection rules)."""
    ny, nx = F.shape[0], F.shape[1]
    neg = False
    if i < 0:
        i = 0
        neg ^= _parity(bc[0], comp, 0) < 0
    elif i >= nx:
        i = nx - 1
        neg ^= _parity(bc[1], comp, 0) < 0
    if j < 0:
        j = 0
        neg ^= _parity(bc[2], comp, 1) < 0
    elif j >= ny:
        j = ny - 1
        neg ^= _parity(bc[3], comp, 1) < 0
    v = float(F[j, i, comp])
    return -v if neg else v


def interp_bilinear(F, comp, x, y, bc):
    """Bilinear interpolation from the four nearest cell centres (Sec. 2.3, Fig. 2)."""
    fx = x - 0.5
    fy = y - 0.5
    ix = math.floor(fx)
    iy = math.floor(fy)
    xb = fx - ix
    yb = fy - iy
    u2 = cell_value(F, comp, ix, iy, bc)
    u1 = cell_value(F, comp, ix, iy + 1, bc)
    u3 = cell_value(F, comp, ix + 1, iy, bc)
    u4 = cell_value(F, comp, ix + 1, iy + 1, bc)
    wx0 = 1.0 - xb
    wy0 = 1.0 - yb
    return wx0 * wy0 * u2 + wx0 * yb * u1 + xb * wy0 * u3 + xb * yb * u4


def interface_velocity_cells(u_l, u_v, ccol, mdot, nb, rho_l, rho_v):
    """u_Gamma at every cell centre from the jump condition (interfacial-velocity equation)."""
    uG = np.empty_like(u_l)
    liq = ccol == 1
    cl = mdot / rho_l
    cv = mdot / rho_v
    for c in range(2):
        uG[..., c] = np.where(liq, u_l[..., c] - cl * nb[..., c], u_v[..., c] - cv * nb[..., c])
    return uG


def _clampf(f):
    return min(max(f, FMIN), 1.0 - FMIN)


def _crossing(E, O, R, m, axis):
    """Across-coordinate where the curve through E, O (and R) crosses the unaligned line at m."""
    ea = E[axis]
    ec = E[1 - axis]
    bal = O[axis] - ea
    bac = O[1 - axis] - ec
    alpha = m - ea
    lin = alpha * bac / bal
    best = None
    if R is not None:
        cal = R[axis] - ea
        cac = R[1 - axis] - ec
        det = bal * cac - bac * cal
        bb = bal * bal + bac * bac
        cc = cal * cal + cac * cac
        Dp = cc * bac - bb * cac
        Ep = bb * cal - cc * bal
        qa = det
        qb = Ep
        qc = det * alpha * alpha + Dp * alpha
        disc = qb * qb - 4.0 * qa * qc
        if disc >= 0.0:
            sq = math.sqrt(disc)
            if qb >= 0.0:
                t = -0.5 * (qb + sq)
            else:
                t = -0.5 * (qb - sq)
            if t != 0.0:
                best = qc / t
            if qa != 0.0:
                r2 = t / qa
                if best is None or abs(r2 - lin) < abs(best - lin):
                    best = r2
            if best is not None and abs(best - lin) > abs(bal) + abs(bac):
                best = None
    if best is None:
        best = lin
    return ec + best


_NEIGH = {0: (-1, 0), 1: (0, 1), 2: (1, 0), 3: (0, -1)}   # cell-edge k -> (dj, di)


def sweep(vcol, hx_pos, vy_pos, geom, uG, dth, axis, bc):
    """One 1D EBIT advection along axis (0: x, 1: y).  Returns new (vcol, hx_pos, vy_pos)."""
    ny, nx = vcol.shape[0] - 1, vcol.shape[1] - 1
    n_al = nx if axis == 0 else ny
    n_ac = ny if axis == 0 else nx
    hcut = vcol[:, :-1] != vcol[:, 1:]
    vcut = vcol[:-1, :] != vcol[1:, :]
    aligned_kind = "h" if axis == 0 else "v"

    # 1. displace every marker (marker-motion equation, explicit Euler)
    pos = {}
    new = {}
    for j, i in zip(*np.nonzero(hcut)):
        pos[("h", int(j), int(i))] = (i + float(hx_pos[j, i]), float(j))
    for j, i in zip(*np.nonzero(vcut)):
        pos[("v", int(j), int(i))] = (float(i), j + float(vy_pos[j, i]))
    for key, (x, y) in pos.items():
        u = interp_bilinear(uG, axis, x, y, bc)
        d = u * dth
        p = [x, y]
        al = p[axis]
        if key[0] != aligned_kind and (al == 0.0 or al == float(n_al)):
            d = 0.0
        al = al + d
        if key[0] == aligned_kind:
            al = min(max(al, 0.0), float(n_al) - FMIN)
        else:
            al = min(max(al, 0.0), float(n_al))
        p[axis] = al
        new[key] = (p[0], p[1])

    # 2. vertex colours flip once per aligned marker crossing them
    vnew = vcol.copy()
    for key, P in new.items():
        if key[0] != aligned_kind:
            continue
        a0 = pos[key][axis]
        a1 = P[axis]
        line = key[1] if axis == 0 else key[2]
        for m in range(int(math.floor(min(a0, a1))), int(math.floor(max(a0, a1))) + 2):
            if 0 <= m <= n_al and ((a0 < m) != (a1 < m)):
                if axis == 0:
                    vnew[line, m] ^= 1
                else:
                    vnew[m, line] ^= 1

    # 3. aligned edges: markers re-binned on their line
    abucket = {}
    for key, P in new.items():
        if key[0] != aligned_kind:
            continue
        line = key[1] if axis == 0 else key[2]
        al = P[axis]
        e = int(math.floor(al))
        f = _clampf(al - e)
        abucket.setdefault((line, e), []).append(f)

    # 4. unaligned lines: crossings of the displaced segments, and displaced markers lying on them
    ubucket = {}
    for (j, i), segs in geom.seg.items():
        for s in range(len(segs)):
            kP = int(geom.segP[j, i, s])
            kQ = int(geom.segQ[j, i, s])
            keyP = edge_key(kP, i, j)
            keyQ = edge_key(kQ, i, j)
            Pn = new[keyP]
            Qn = new[keyQ]
            pa, qa = Pn[axis], Qn[axis]
            lo, hi = min(pa, qa), max(pa, qa)
            c_ac = j if axis == 0 else i
            for m in range(int(math.floor(lo)), int(math.floor(hi)) + 2):
                if not (lo < m < hi) or m < 0 or m > n_al:
                    continue
                if abs(pa - m) <= abs(qa - m):
                    E, O, kE = Pn, Qn, kP
                else:
                    E, O, kE = Qn, Pn, kQ
                R = _chain_neighbour(geom, new, i, j, kE, nx, ny)
                ac = _crossing(E, O, R, m, axis)
                ubucket.setdefault((m, c_ac), []).append(_clampf(ac - c_ac))
    for key, P in new.items():
        al = P[axis]
        if al == math.floor(al):
            m = int(al)
            if 0 <= m <= n_al:
                ac = P[1 - axis]
                e = min(max(int(math.floor(ac)), 0), n_ac - 1)
                ubucket.setdefault((m, e), []).append(_clampf(ac - e))

    # 5. one marker per edge
    hx_new = np.zeros_like(hx_pos)
    vy_new = np.zeros_like(vy_pos)
    hcut_n = vnew[:, :-1] != vnew[:, 1:]
    vcut_n = vnew[:-1, :] != vnew[1:, :]

    def pick(cands):
        if not cands:
            return 0.5
        c = sorted(cands)
        return c[(len(c) - 1) // 2]

    if axis == 0:
        for j, i in zip(*np.nonzero(hcut_n)):
            hx_new[j, i] = pick(abucket.get((int(j), int(i))))
        for j, i in zip(*np.nonzero(vcut_n)):
            vy_new[j, i] = pick(ubucket.get((int(i), int(j))))
    else:
        for j, i in zip(*np.nonzero(vcut_n)):
            vy_new[j, i] = pick(abucket.get((int(i), int(j))))
        for j, i in zip(*np.nonzero(hcut_n)):
            hx_new[j, i] = pick(ubucket.get((int(j), int(i))))
    return vnew, hx_new, vy_new


def _chain_neighbour(geom, new, i, j, kE, nx, ny):
    """Displaced position of the marker linked to the marker on cell-edge kE through the adjacent cell."""
    dj, di = _NEIGH[kE]
    jn, in_ = j + dj, i + di
    if not (0 <= jn < ny and 0 <= in_ < nx):
        return None
    kk = (kE + 2) % 4
    for s in range(int(geom.nseg[jn, in_])):
        kP = int(geom.segP[jn, in_, s])
        kQ = int(geom.segQ[jn, in_, s])
        if kP == kk:
            return new[edge_key(kQ, in_, jn)]
        if kQ == kk:
            return new[edge_key(kP, in_, jn)]
    return None
