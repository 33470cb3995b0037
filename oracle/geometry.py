"""Color-Vertex reconstruction, volume fraction, narrow band, ghost-fluid theta.

Grid units: cell (i, j) is the square [i, i+1] x [j, j+1]; its centre is
(i + 0.5, j + 0.5).  Inside a cell the four edges are numbered counter-
clockwise from the bottom (0 bottom, 1 right, 2 top, 3 left) and edge k runs
from corner k to corner k+1 (corners 0 BL, 1 BR, 2 TR, 3 TL).

Readings (the paper defers EBIT details to its refs [chirco2023edge, pan2023edge]):
  * an edge is cut iff its two vertex colours differ (one marker per edge, Sec. 2.1);
  * a segment runs from the marker where the counter-clockwise walk leaves the
    liquid (P, "exit") to the marker where it re-enters (Q, "enter"), so the
    liquid lies on its left and n = (dy, -dx)/|d| points from liquid into vapour;
  * saddle cells (four cut edges) are resolved by the fifth, centre colour vertex
    (Sec. 2.1): the pairing with the smaller total segment length is taken and the
    centre gets the colour of the corners that pairing connects;
  * f_C is the phase of the cell centre with respect to the reconstructed
    segments (centre on a segment counts as liquid);
  * the liquid volume fraction is the area of the liquid polygon (shoelace),
    which is what the property average of Sec. 2.2 needs;
  * narrow band (Sec. 2.4): a cell whose 3x3 block holds a cut cell; the band
    normal is the normalised sum of (dy, -dx) over the segments of that block;
  * ghost-fluid link fraction (ghost-temperature equation): theta is the distance
    from the cell centre to the nearest crossing of the centre-to-centre link with
    a segment of the two cells, 0.5 if none, clamped to [theta_min, 1].
"""
from __future__ import annotations

import math

import numpy as np

_CORNER_LOCAL = ((0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0))


def corner_colours(vcol, i, j):
    return (int(vcol[j, i]), int(vcol[j, i + 1]), int(vcol[j + 1, i + 1]), int(vcol[j + 1, i]))


def marker_local(k, i, j, hx_pos, vy_pos):
    """Marker on cell edge k, in cell-local coordinates."""
    if k == 0:
        return (float(hx_pos[j, i]), 0.0)
    if k == 1:
        return (1.0, float(vy_pos[j, i + 1]))
    if k == 2:
        return (float(hx_pos[j + 1, i]), 1.0)
    return (0.0, float(vy_pos[j, i]))


def edge_key(k, i, j):
    """Global key of cell edge k: ('h', line j, index i) or ('v', row j, line i)."""
    if k == 0:
        return ("h", j, i)
    if k == 1:
        return ("v", j, i + 1)
    if k == 2:
        return ("h", j + 1, i)
    return ("v", j, i)


def _shoelace(pts):
    s = 0.0
    n = len(pts)
    for a in range(n):
        xa, ya = pts[a]
        xb, yb = pts[(a + 1) % n]
        s = s + (xa * yb - xb * ya)
    return 0.5 * s


def _cross_centre(P, Q):
    """(Q - P) x (C - P) for the cell centre C = (0.5, 0.5): > 0 means C left of P->Q."""
    return (Q[0] - P[0]) * (0.5 - P[1]) - (Q[1] - P[1]) * (0.5 - P[0])


def _dist(A, B):
    dx = B[0] - A[0]
    dy = B[1] - A[1]
    return math.sqrt(dx * dx + dy * dy)


class Geometry:
    """Per-cell reconstruction: segments (local coordinates), f_C, vf, band, normals."""

    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny
        self.nseg = np.zeros((ny, nx), np.int8)
        self.segP = -np.ones((ny, nx, 2), np.int8)   # cell-edge index of P (exit)
        self.segQ = -np.ones((ny, nx, 2), np.int8)   # cell-edge index of Q (enter)
        self.seg = {}                                  # (j, i) -> [(P_local, Q_local), ...]
        self.ccol = np.zeros((ny, nx), np.uint8)
        self.vf = np.zeros((ny, nx))
        self.band = np.zeros((ny, nx), bool)
        self.nb = np.zeros((ny, nx, 2))

    def cut_cells(self):
        return list(zip(*np.nonzero(self.nseg)))


def reconstruct(vcol, hx_pos, vy_pos):
    """Color-Vertex reconstruction of every cell (Sec. 2.1, property-average equation)."""
    ny, nx = vcol.shape[0] - 1, vcol.shape[1] - 1
    g = Geometry(nx, ny)
    c0 = vcol[:-1, :-1]
    g.ccol[:] = c0
    g.vf[:] = c0.astype(float)
    mixed = (vcol[:-1, :-1] != vcol[:-1, 1:]) | (vcol[:-1, :-1] != vcol[1:, 1:]) | (vcol[:-1, :-1] != vcol[1:, :-1])
    for j, i in zip(*np.nonzero(mixed)):
        c = corner_colours(vcol, i, j)
        M = [marker_local(k, i, j, hx_pos, vy_pos) for k in range(4)]
        exits = [k for k in range(4) if c[k] == 1 and c[(k + 1) % 4] == 0]
        enters = [k for k in range(4) if c[k] == 0 and c[(k + 1) % 4] == 1]
        if len(exits) == 1:
            kx, kn = exits[0], enters[0]
            pairs = [(kx, kn)]
            poly = [M[kn]]
            k = (kn + 1) % 4
            while True:
                poly.append(_CORNER_LOCAL[k])
                if k == kx:
                    break
                k = (k + 1) % 4
            poly.append(M[kx])
            vf = _shoelace(poly)
            ccol = 1 if _cross_centre(M[kx], M[kn]) >= 0.0 else 0
        else:
            k1, k2 = exits  # ascending edge index
            LA = _dist(M[k1], M[(k1 + 1) % 4]) + _dist(M[k2], M[(k2 + 1) % 4])
            LB = _dist(M[k1], M[(k1 + 3) % 4]) + _dist(M[k2], M[(k2 + 3) % 4])
            if LA <= LB:
                # liquid corners connected through the centre: vapour corners cut off
                pairs = [(k1, (k1 + 1) % 4), (k2, (k2 + 1) % 4)]
                area = 0.0
                for kx, kn in pairs:
                    area = area + _shoelace([M[kx], _CORNER_LOCAL[kn], M[kn]])
                vf = 1.0 - area
                ccol = 1
                for kx, kn in pairs:
                    if _cross_centre(M[kx], M[kn]) < 0.0:
                        ccol = 0
            else:
                # vapour corners connected: liquid corners cut off
                pairs = [(k1, (k1 + 3) % 4), (k2, (k2 + 3) % 4)]
                area = 0.0
                for kx, kn in pairs:
                    area = area + _shoelace([M[kn], _CORNER_LOCAL[kx], M[kx]])
                vf = area
                ccol = 0
                for kx, kn in pairs:
                    if _cross_centre(M[kx], M[kn]) >= 0.0:
                        ccol = 1
        g.nseg[j, i] = len(pairs)
        g.seg[(j, i)] = [(M[kx], M[kn]) for kx, kn in pairs]
        for s, (kx, kn) in enumerate(pairs):
            g.segP[j, i, s] = kx
            g.segQ[j, i, s] = kn
        g.vf[j, i] = vf
        g.ccol[j, i] = ccol
    _band(g)
    return g


def _band(g):
    """Narrow band and band normal (Sec. 2.4)."""
    nx, ny = g.nx, g.ny
    cut = g.nseg > 0
    pad = np.zeros((ny + 2, nx + 2), bool)
    pad[1:-1, 1:-1] = cut
    band = np.zeros((ny, nx), bool)
    for dj in range(3):
        for di in range(3):
            band |= pad[dj:dj + ny, di:di + nx]
    g.band[:] = band
    for j, i in zip(*np.nonzero(band)):
        ax = 0.0
        ay = 0.0
        for jj in range(j - 1, j + 2):
            for ii in range(i - 1, i + 2):
                if 0 <= ii < nx and 0 <= jj < ny and cut[jj, ii]:
                    for P, Q in g.seg[(jj, ii)]:
                        dx = Q[0] - P[0]
                        dy = Q[1] - P[1]
                        ax = ax + dy
                        ay = ay - dx
        nrm = math.sqrt(ax * ax + ay * ay)
        if nrm > 0.0:
            g.nb[j, i, 0] = ax / nrm
            g.nb[j, i, 1] = ay / nrm


def segment_data(g):
    """Per segment: cell, midpoint (grid units), unit normal (liquid->vapour), length (grid units)."""
    out = []
    for (j, i), segs in sorted(g.seg.items()):
        for P, Q in segs:
            dx = Q[0] - P[0]
            dy = Q[1] - P[1]
            L = math.sqrt(dx * dx + dy * dy)
            mx = i + 0.5 * (P[0] + Q[0])
            my = j + 0.5 * (P[1] + Q[1])
            n = (dy / L, -dx / L) if L > 0 else (0.0, 0.0)
            out.append(((j, i), (mx, my), n, L))
    return out


def link_thetas(g, theta_min):
    """Ghost-fluid fractions (ghost-temperature equation) for every link whose two centres differ in colour.

    Returns dict: (j, i, side) -> theta, side in 0 (+x), 1 (-x), 2 (+y), 3 (-y), for the
    cell (j, i) whose link towards that side crosses the interface.
    """
    nx, ny = g.nx, g.ny
    th = {}

    def crossings_x(jc, ic, lo, hi):
        """x (cell-local) where segments of cell (jc, ic) cross y = 0.5, restricted to [lo, hi]."""
        xs = []
        for P, Q in g.seg.get((jc, ic), []):
            if (P[1] < 0.5) != (Q[1] < 0.5):
                x = P[0] + (0.5 - P[1]) * (Q[0] - P[0]) / (Q[1] - P[1])
                if lo <= x <= hi:
                    xs.append(x)
        return xs

    def crossings_y(jc, ic, lo, hi):
        ys = []
        for P, Q in g.seg.get((jc, ic), []):
            if (P[0] < 0.5) != (Q[0] < 0.5):
                y = P[1] + (0.5 - P[0]) * (Q[1] - P[1]) / (Q[0] - P[0])
                if lo <= y <= hi:
                    ys.append(y)
        return ys

    def clamp(t):
        return min(max(t, theta_min), 1.0)

    for j, i in zip(*np.nonzero(g.ccol[:, :-1] != g.ccol[:, 1:])):
        a = crossings_x(j, i, 0.5, 1.0)          # in the left cell
        b = crossings_x(j, i + 1, 0.0, 0.5)      # in the right cell
        dl = [x - 0.5 for x in a] + [0.5 + x for x in b]
        dr = [1.5 - x for x in a] + [0.5 - x for x in b]
        th[(j, i, 0)] = clamp(min(dl)) if dl else clamp(0.5)
        th[(j, i + 1, 1)] = clamp(min(dr)) if dr else clamp(0.5)
    for j, i in zip(*np.nonzero(g.ccol[:-1, :] != g.ccol[1:, :])):
        a = crossings_y(j, i, 0.5, 1.0)
        b = crossings_y(j + 1, i, 0.0, 0.5)
        dl = [y - 0.5 for y in a] + [0.5 + y for y in b]
        dr = [1.5 - y for y in a] + [0.5 - y for y in b]
        th[(j, i, 2)] = clamp(min(dl)) if dl else clamp(0.5)
        th[(j + 1, i, 3)] = clamp(min(dr)) if dr else clamp(0.5)
    return th
