"""Seeded, synthetic initial states for the EBIT phase-change workloads.

This module only *describes problems*: grid, boundary conditions, material
properties, the initial interface (vertex colours + one marker fraction per cut
edge, found by root-finding an analytic level set) and the initial fields
(closed-form similarity solutions where the problem has one).  It holds none of
the method's arithmetic (no reconstruction, advection, ghost-fluid or solver
step), so both the CUDA path and the CPU oracle can start from the same state.

Closed forms:
  * 1D Stefan problem (Sec. 3.1, interface-position and temperature equations):
    X(t) = 2 beta sqrt(alpha_v t),  beta exp(beta^2) erf(beta) = cp_v dT / (sqrt(pi) h_lg).
  * Scriven problem (Sec. 3.4), the paper's spherical case on an axisymmetric grid
    (scriven, scriven_beta, scriven_temperature), and its planar (cylindrical) analogue
    for planar grids (bubble), derived in the same way (liquid velocity eps R R'/r,
    eps = 1 - rho_v/rho_l):
    R = 2 beta sqrt(alpha_l t),  T(eta) = T_inf - dT I(eta)/I(beta),
    I(eta) = int_eta^inf s^(2 eps beta^2 - 1) exp(-s^2) ds,
    Ja = rho_l cp_l dT / (rho_v h_lg) = 2 beta^2 exp(beta^2) beta^(-2 eps beta^2) I(beta).
  * Bubble with a constant mass flux (Sec. 3.3): R(t) = R0 + mdot t / rho_v.

Arrays are row-major with x fastest: cell fields are [ny, nx], vertex colours
[ny+1, nx+1], horizontal edges [ny+1, nx], vertical edges [ny, nx+1].
Colour 1 = liquid, 0 = vapour.  Marker fractions are measured from the
lower/left vertex of their edge, in [FMIN, 1 - FMIN].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import optimize, special

FMIN = 1e-9  # markers never sit exactly on a vertex

# boundary kinds, order of sides: left, right, bottom, top
WALL, OUTFLOW, SYMMETRY = 0, 1, 2
BC_NAMES = {"wall": WALL, "outflow": OUTFLOW, "symmetry": SYMMETRY}


@dataclass
class Problem:
    """Everything that defines one instance: grid, physics, initial state."""
    name: str
    nx: int
    ny: int
    h: float
    x0: float = 0.0
    y0: float = 0.0
    dt: float = 1e-4
    steps: int = 1
    # properties: liquid, vapour
    rho_l: float = 1.0
    rho_v: float = 1.0
    mu_l: float = 0.01
    mu_v: float = 0.01
    lam_l: float = 1.0
    lam_v: float = 1.0
    cp_l: float = 1.0
    cp_v: float = 1.0
    T_sat: float = 0.0
    h_lg: float = 1.0
    sigma: float = 0.0            # surface tension coefficient
    gx: float = 0.0
    gy: float = 0.0
    bc: tuple = (WALL, OUTFLOW, SYMMETRY, SYMMETRY)
    # Dirichlet temperature per side (None = zero normal gradient)
    T_bc: tuple = (None, None, None, None)
    theta_min: float = 1e-3
    extend_iters: int = 5
    sweep_order: int = 1          # 0: always x then y; 1: alternate
    energy: bool = True           # False: mdot imposed (constant-mass-flux bubble)
    mdot_fixed: float = 0.0
    axi: bool = False             # True: axisymmetric, x is the radius (the axis at x = 0 is the
                                  # left side, a symmetry side), y the axial coordinate
    one_fluid: bool = False       # True: one velocity field and the phase-change source S_pc
                                  # (Sec. 2.2-2.3) instead of ghost velocities; the vapour
                                  # velocity arrays then repeat the liquid ones
    # initial state (filled by the generators)
    vcol: np.ndarray = None
    hx_cut: np.ndarray = None
    hx_pos: np.ndarray = None
    vy_cut: np.ndarray = None
    vy_pos: np.ndarray = None
    T_l: np.ndarray = None
    T_v: np.ndarray = None
    u_l: np.ndarray = None        # [ny, nx, 2]
    u_v: np.ndarray = None
    ufx_l: np.ndarray = None      # [ny, nx+1]
    ufx_v: np.ndarray = None
    ufy_l: np.ndarray = None      # [ny+1, nx]
    ufy_v: np.ndarray = None
    p: np.ndarray = None
    t0: float = 0.0
    meta: dict = field(default_factory=dict)

    def copy(self) -> "Problem":
        import copy
        return copy.deepcopy(self)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
def stefan_beta(St: float) -> float:
    """Root of beta exp(beta^2) erf(beta) = St / sqrt(pi), St = cp_v dT / h_lg."""
    f = lambda b: b * math.exp(b * b) * math.erf(b) - St / math.sqrt(math.pi)
    return optimize.brentq(f, 1e-12, 10.0, xtol=1e-15, rtol=1e-15, maxiter=500)


def stefan_position(t, beta, alpha_v):
    return 2.0 * beta * np.sqrt(alpha_v * t)


def stefan_temperature(x, t, beta, alpha_v, T_w, T_sat):
    return T_w + (T_sat - T_w) / math.erf(beta) * special.erf(x / (2.0 * np.sqrt(alpha_v * t)))


def _scriven_integrand(xi, beta, eps):
    return math.exp(-beta * beta * ((1.0 - xi) ** -2 - 2.0 * eps * xi - 1.0))


def scriven_beta(rho_l, rho_v, cp_l, cp_v, dT, h_lg) -> float:
    """Growth constant of a spherical bubble in superheated liquid (Scriven; Sec. 3.4): the root of
    rho_l cp_l dT / (rho_v (h_lg + (cp_l - cp_v) dT)) = 2 beta^2 int_0^1 exp(-beta^2 ((1 - xi)^-2
    - 2 eps xi - 1)) d xi with eps = 1 - rho_v / rho_l (the exponent of the temperature equation;
    the growth-constant equation prints 1 - rho_l / rho_v, for which no root exists)."""
    from scipy import integrate
    lhs = rho_l * cp_l * dT / (rho_v * (h_lg + (cp_l - cp_v) * dT))
    eps = 1.0 - rho_v / rho_l

    def f(b):
        val, _ = integrate.quad(_scriven_integrand, 0.0, 1.0, args=(b, eps), epsabs=0.0, epsrel=1e-13, limit=400)
        return 2.0 * b * b * val - lhs
    return optimize.brentq(f, 1e-6, 100.0, xtol=1e-14, rtol=1e-14, maxiter=500)


def scriven_temperature(r, t, beta, rho_l, rho_v, cp_l, cp_v, dT, h_lg, alpha_l, T_inf):
    """Liquid temperature of the Scriven problem (Sec. 3.4, temperature equation) at radius r >= R."""
    from scipy import integrate
    R = 2.0 * beta * math.sqrt(alpha_l * t)
    eps = 1.0 - rho_v / rho_l
    pref = 2.0 * beta * beta * rho_v * (h_lg + (cp_l - cp_v) * dT) / (rho_l * cp_l)
    out = np.empty_like(np.asarray(r, dtype=float))
    flat = out.reshape(-1)
    for k, rv in enumerate(np.asarray(r, dtype=float).reshape(-1)):
        if rv <= R:
            flat[k] = T_inf - dT
            continue
        val, _ = integrate.quad(_scriven_integrand, 1.0 - R / rv, 1.0, args=(beta, eps), epsabs=0.0,
                                epsrel=1e-12, limit=400)
        flat[k] = T_inf - pref * val
    return out


def sucking_beta(rho_l, rho_v, lam_l, lam_v, cp_l, cp_v, dT, h_lg) -> float:
    """Growth constant of the 1D sucking problem (Sec. 3.2, its beta equation): the root of
    beta = dT cp_v lam_l sqrt(alpha_v) exp(-b^2) / (h_lg lam_v sqrt(pi alpha_l) erfc(b)),
    b = beta rho_v sqrt(alpha_v) / (rho_l sqrt(alpha_l)) (the bracket of the printed equation;
    its factor exp(beta^2) erf(beta) has no root)."""
    al, av = lam_l / (rho_l * cp_l), lam_v / (rho_v * cp_v)
    k = rho_v * math.sqrt(av) / (rho_l * math.sqrt(al))

    def f(b):   # exp(-z^2) / erfc(z) = 1 / erfcx(z), evaluated without underflow
        return b - dT * cp_v * lam_l * math.sqrt(av) / (
            h_lg * lam_v * math.sqrt(math.pi * al) * special.erfcx(b * k))
    return optimize.brentq(f, 1e-12, 100.0, xtol=1e-15, rtol=1e-15, maxiter=500)


def sucking_position(t, beta, alpha_v):
    """Interface position 2 beta sqrt(alpha_v t): the diffusivity that the paper's beta equation
    and temperature profile are written with (its position equation prints alpha_l)."""
    return 2.0 * beta * np.sqrt(alpha_v * t)


def sucking_temperature(x, t, beta, rho_l, rho_v, alpha_l, alpha_v, T_inf, T_sat):
    """Liquid temperature of the sucking problem (Sec. 3.2): T_inf - (T_inf - T_sat)
    erfc(x / (2 sqrt(alpha_l t)) + beta (rho_v - rho_l) sqrt(alpha_v) / (rho_l sqrt(alpha_l)))
    / erfc(beta rho_v sqrt(alpha_v) / (rho_l sqrt(alpha_l)))."""
    k = math.sqrt(alpha_v) / (rho_l * math.sqrt(alpha_l))
    return T_inf - (T_inf - T_sat) * special.erfc(x / (2.0 * np.sqrt(alpha_l * t)) + beta * (rho_v - rho_l) * k) / \
        special.erfc(beta * rho_v * k)


def _bubble2d_logI(eta, a):
    """log of I(eta) = int_eta^inf s^(2a-1) exp(-s^2) ds = Gamma(a) Q(a, eta^2) / 2."""
    q = special.gammaincc(a, eta * eta)
    with np.errstate(divide="ignore"):   # Q underflows to 0 far outside the layer: log -> -inf, I -> 0
        return special.gammaln(a) + np.log(q) - math.log(2.0)


def bubble2d_beta(Ja: float, eps: float) -> float:
    """Growth constant of the planar bubble: Ja = 2 b^2 e^{b^2} b^{-2 eps b^2} I(b)."""
    def g(b):
        a = eps * b * b
        logrhs = math.log(2.0) + 2 * math.log(b) + b * b - 2 * a * math.log(b) + _bubble2d_logI(b, a)
        return logrhs - math.log(Ja)
    return optimize.brentq(g, 1e-3, 60.0, xtol=1e-14, rtol=1e-15, maxiter=500)


def bubble2d_temperature(r, t, beta, eps, alpha_l, T_inf, T_sat):
    a = eps * beta * beta
    eta = np.asarray(r) / (2.0 * np.sqrt(alpha_l * t))
    ratio = np.exp(_bubble2d_logI(np.maximum(eta, 1e-300), a) - _bubble2d_logI(beta, a))
    return T_inf - (T_inf - T_sat) * ratio


# --------------------------------------------------------------------------
# interface from a level set (phi > 0: liquid)
# --------------------------------------------------------------------------
def interface_from_levelset(phi, nx, ny, h, x0=0.0, y0=0.0):
    """Vertex colours and one marker per cut edge, the marker at the root of phi."""
    xs = x0 + h * np.arange(nx + 1)
    ys = y0 + h * np.arange(ny + 1)
    X, Y = np.meshgrid(xs, ys)
    pv = phi(X, Y)
    vcol = (pv > 0).astype(np.uint8)
    hx_cut = (vcol[:, :-1] != vcol[:, 1:]).astype(np.uint8)
    vy_cut = (vcol[:-1, :] != vcol[1:, :]).astype(np.uint8)
    hx_pos = np.zeros((ny + 1, nx))
    vy_pos = np.zeros((ny, nx + 1))

    def root(fn):
        a, b = fn(0.0), fn(1.0)
        if a == 0.0:
            return FMIN
        if b == 0.0:
            return 1.0 - FMIN
        s = optimize.brentq(fn, 0.0, 1.0, xtol=1e-15, rtol=1e-15, maxiter=200)
        return min(max(s, FMIN), 1.0 - FMIN)

    for j, i in zip(*np.nonzero(hx_cut)):
        yv = y0 + h * j
        hx_pos[j, i] = root(lambda s: float(phi(x0 + h * (i + s), yv)))
    for j, i in zip(*np.nonzero(vy_cut)):
        xv = x0 + h * i
        vy_pos[j, i] = root(lambda s: float(phi(xv, y0 + h * (j + s))))
    return vcol, hx_cut, hx_pos, vy_cut, vy_pos


def _grids(nx, ny, h, x0, y0):
    xc = x0 + h * (np.arange(nx) + 0.5)
    yc = y0 + h * (np.arange(ny) + 0.5)
    Xc, Yc = np.meshgrid(xc, yc)
    xf = x0 + h * np.arange(nx + 1)
    Xfx, Yfx = np.meshgrid(xf, yc)           # x-faces
    yf = y0 + h * np.arange(ny + 1)
    Xfy, Yfy = np.meshgrid(xc, yf)           # y-faces
    return (Xc, Yc), (Xfx, Yfx), (Xfy, Yfy)


def _zero_flow(pb):
    nx, ny = pb.nx, pb.ny
    pb.u_l = np.zeros((ny, nx, 2))
    pb.u_v = np.zeros((ny, nx, 2))
    pb.ufx_l = np.zeros((ny, nx + 1))
    pb.ufx_v = np.zeros((ny, nx + 1))
    pb.ufy_l = np.zeros((ny + 1, nx))
    pb.ufy_v = np.zeros((ny + 1, nx))
    pb.p = np.zeros((ny, nx))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def stefan(nx=64, ny=64, X0=0.1, Lx=1.0, rho_l=10.0, rho_v=1.0, St=0.1, dT=1.0,
           mu=0.01, dt=1e-4, steps=100, **kw) -> Problem:
    """1D Stefan problem embedded in 2D: vapour x < X0 on a wall at T_sat + dT.

    Left: no-slip wall at T_w; right: outflow; bottom/top: symmetry.
    Nondimensional: k = cp = 1 in both phases, h_lg = cp dT / St, T_sat = 0.
    """
    h = Lx / nx
    h_lg = 1.0 * dT / St
    pb = Problem("stefan", nx, ny, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v,
                 mu_l=mu, mu_v=mu, lam_l=1.0, lam_v=1.0, cp_l=1.0, cp_v=1.0,
                 T_sat=0.0, h_lg=h_lg, bc=(WALL, OUTFLOW, SYMMETRY, SYMMETRY),
                 T_bc=(dT, None, None, None), **kw)
    beta = stefan_beta(St)
    alpha_v = pb.lam_v / (pb.rho_v * pb.cp_v)
    t0 = (X0 / (2 * beta)) ** 2 / alpha_v
    pb.t0 = t0
    pb.meta.update(beta=beta, alpha_v=alpha_v, T_w=dT, X0=X0)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: x - X0, nx, ny, h)
    (Xc, Yc), (Xfx, Yfx), (Xfy, Yfy) = _grids(nx, ny, h, 0.0, 0.0)
    pb.T_v = stefan_temperature(Xc, t0, beta, alpha_v, dT, 0.0)
    pb.T_l = np.zeros((ny, nx))
    _zero_flow(pb)
    Xdot = beta * math.sqrt(alpha_v / t0)
    mdot = rho_v * Xdot
    U = mdot * (1.0 / rho_v - 1.0 / rho_l)
    pb.meta.update(mdot0=mdot, U=U)
    pb.u_l[..., 0] = U
    pb.ufx_l[:, 1:] = U          # the wall face stays 0
    return pb


def axi_const_mdot_bubble(n=48, L=1.0, R0=0.3, mdot=0.1, rho_l=10.0, rho_v=1.0, mu=0.01, dt=None, cfl=0.3,
                          steps=4, **kw) -> Problem:
    """A spherical bubble centred on the axis with an imposed constant mass flux, energy off
    (Sec. 3.3 in the axisymmetric configuration of Sec. 3.4): a quarter of it on [0, L]^2, the
    axis on the left and a symmetry plane at the bottom, outflow top and right.  Its radius
    grows as R0 + mdot t / rho_v."""
    h = L / n
    if dt is None:
        dt = cfl * h * rho_v / abs(mdot)
    pb = Problem("axi_const_mdot_bubble", n, n, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v, mu_l=mu, mu_v=mu,
                 T_sat=0.0, h_lg=1.0, bc=(SYMMETRY, OUTFLOW, SYMMETRY, OUTFLOW), T_bc=(None,) * 4, energy=False,
                 mdot_fixed=mdot, axi=True, **kw)
    pb.meta.update(R0=R0, mdot=mdot)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: np.hypot(x, y) - R0, n, n, h)
    pb.T_l = np.zeros((n, n))
    pb.T_v = np.zeros((n, n))
    _zero_flow(pb)
    return pb


def scriven(n=64, L=1.0, R0=0.3, rho_ratio=20.0, k_ratio=5.0, St=0.25, dT=1.0, mu=0.01, dt=None, steps=4,
            **kw) -> Problem:
    """Scriven problem (Sec. 3.4): a spherical vapour bubble at T_sat growing in superheated liquid,
    axisymmetric quarter on [0, L]^2 (axis left, symmetry bottom, outflow top and right), initial
    state from the similarity solution at the time the radius is R0: liquid temperature of the
    temperature equation, radial liquid velocity eps R R' R^2 / r^2 (eps = 1 - rho_v / rho_l),
    vapour at rest at T_sat.  Nondimensional, cp = 1 both phases, lambda_v = 1."""
    h = L / n
    rho_v, rho_l = 1.0, rho_ratio
    lam_v, lam_l = 1.0, k_ratio
    h_lg = 1.0 * dT / St
    beta = scriven_beta(rho_l, rho_v, 1.0, 1.0, dT, h_lg)
    alpha_l = lam_l / rho_l
    t0 = (R0 / (2.0 * beta)) ** 2 / alpha_l
    Rdot = beta * math.sqrt(alpha_l / t0)
    if dt is None:
        dt = 0.2 * h / Rdot
    pb = Problem("scriven", n, n, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v, mu_l=mu, mu_v=mu, lam_l=lam_l,
                 lam_v=lam_v, cp_l=1.0, cp_v=1.0, T_sat=0.0, h_lg=h_lg, bc=(SYMMETRY, OUTFLOW, SYMMETRY, OUTFLOW),
                 T_bc=(None,) * 4, axi=True, **kw)
    eps = 1.0 - rho_v / rho_l
    pb.t0 = t0
    pb.meta.update(beta=beta, alpha_l=alpha_l, R0=R0, Rdot0=Rdot, eps=eps)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: np.hypot(x, y) - R0, n, n, h)
    (Xc, Yc), (Xfx, Yfx), (Xfy, Yfy) = _grids(n, n, h, 0.0, 0.0)
    r = np.hypot(Xc, Yc)
    pb.T_l = scriven_temperature(r, t0, beta, rho_l, rho_v, 1.0, 1.0, dT, h_lg, alpha_l, dT)
    pb.T_v = np.zeros((n, n))
    _zero_flow(pb)

    def radial(X, Y):
        rr = np.hypot(X, Y)
        mag = np.where(rr >= R0, eps * Rdot * R0 * R0 / np.maximum(rr, 1e-300) ** 2, eps * Rdot * rr / R0)
        with np.errstate(invalid="ignore", divide="ignore"):
            ex = np.where(rr > 0, X / np.maximum(rr, 1e-300), 0.0)
            ey = np.where(rr > 0, Y / np.maximum(rr, 1e-300), 0.0)
        return mag * ex, mag * ey

    pb.u_l[..., 0], pb.u_l[..., 1] = radial(Xc, Yc)
    pb.ufx_l[:] = radial(Xfx, Yfx)[0]
    pb.ufy_l[:] = radial(Xfy, Yfy)[1]
    return pb


def sucking(nx=64, ny=4, X0=0.2, Lx=1.0, rho_l=10.0, rho_v=1.0, lam_l=1.0, lam_v=1.0, St=0.2, dT=1.0,
            mu=0.01, dt=2e-3, steps=100, **kw) -> Problem:
    """1D sucking problem embedded in 2D (Sec. 3.2): vapour x < X0 at T_sat between a wall at
    T_sat (left) and superheated liquid (T_sat + dT far away) leaving through an outflow (right);
    bottom/top symmetry.  Nondimensional, cp = 1, h_lg = cp dT / St (Ja = rho_l cp dT / (rho_v
    h_lg)); initial state from the similarity solution at the time the front is at X0: vapour at
    rest at T_sat, liquid at the closed-form profile moving at mdot (1/rho_v - 1/rho_l)."""
    h = Lx / nx
    h_lg = 1.0 * dT / St
    pb = Problem("sucking", nx, ny, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v, mu_l=mu, mu_v=mu,
                 lam_l=lam_l, lam_v=lam_v, cp_l=1.0, cp_v=1.0, T_sat=0.0, h_lg=h_lg,
                 bc=(WALL, OUTFLOW, SYMMETRY, SYMMETRY), T_bc=(0.0, None, None, None), **kw)
    beta = sucking_beta(rho_l, rho_v, lam_l, lam_v, 1.0, 1.0, dT, h_lg)
    al, av = lam_l / rho_l, lam_v / rho_v
    t0 = (X0 / (2.0 * beta)) ** 2 / av
    mdot = rho_v * beta * math.sqrt(av / t0)
    pb.t0 = t0
    pb.meta.update(beta=beta, alpha_l=al, alpha_v=av, dT=dT, X0=X0, mdot0=mdot)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: x - X0, nx, ny, h)
    (Xc, Yc), (Xfx, Yfx), _ = _grids(nx, ny, h, 0.0, 0.0)
    pb.T_l = sucking_temperature(Xc, t0, beta, rho_l, rho_v, al, av, dT, 0.0)
    pb.T_v = np.zeros((ny, nx))
    _zero_flow(pb)
    ul = mdot * (1.0 / rho_v - 1.0 / rho_l)
    pb.u_l[..., 0] = ul
    pb.ufx_l[:] = ul
    pb.ufx_l[:, 0] = 0.0          # the wall face
    return pb


def bubble(n=512, R0=0.05, rho_ratio=20.0, k_ratio=5.0, St=0.2, dT=1.0, mu=0.01,
           dt=1.96e-6, steps=2000, seed=0, noise=1e-3, **kw) -> Problem:
    """Circular vapour bubble growing in superheated liquid (planar), outflow on all sides."""
    h = 1.0 / n
    rho_v, rho_l = 1.0, rho_ratio
    lam_v, lam_l = 1.0, k_ratio
    h_lg = 1.0 * dT / St
    pb = Problem("bubble", n, n, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v,
                 mu_l=mu, mu_v=mu, lam_l=lam_l, lam_v=lam_v, cp_l=1.0, cp_v=1.0,
                 T_sat=0.0, h_lg=h_lg, bc=(OUTFLOW,) * 4, T_bc=(None,) * 4, **kw)
    Ja = rho_l * 1.0 * dT / (rho_v * h_lg)
    eps = 1.0 - rho_v / rho_l
    beta = bubble2d_beta(Ja, eps)
    alpha_l = lam_l / (rho_l * 1.0)
    t0 = (R0 / (2 * beta)) ** 2 / alpha_l
    Rdot = beta * math.sqrt(alpha_l / t0)
    pb.t0 = t0
    pb.meta.update(beta=beta, eps=eps, alpha_l=alpha_l, Ja=Ja, R0=R0, Rdot0=Rdot, xc=0.5, yc=0.5)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: np.hypot(x - 0.5, y - 0.5) - R0, n, n, h)
    (Xc, Yc), (Xfx, Yfx), (Xfy, Yfy) = _grids(n, n, h, 0.0, 0.0)
    r = np.hypot(Xc - 0.5, Yc - 0.5)
    pb.T_l = bubble2d_temperature(r, t0, beta, eps, alpha_l, dT, 0.0)
    if seed:
        rng = np.random.default_rng(seed)
        pb.T_l = pb.T_l + rng.uniform(-noise, noise, size=pb.T_l.shape)
    pb.T_v = np.zeros((n, n))
    _zero_flow(pb)

    def radial(X, Y):
        rr = np.hypot(X - 0.5, Y - 0.5)
        mag = np.where(rr >= R0, eps * R0 * Rdot / np.maximum(rr, 1e-300), eps * Rdot * rr / R0)
        with np.errstate(invalid="ignore", divide="ignore"):
            ex = np.where(rr > 0, (X - 0.5) / np.maximum(rr, 1e-300), 0.0)
            ey = np.where(rr > 0, (Y - 0.5) / np.maximum(rr, 1e-300), 0.0)
        return mag * ex, mag * ey

    ux, uy = radial(Xc, Yc)
    pb.u_l[..., 0], pb.u_l[..., 1] = ux, uy
    pb.ufx_l[:] = radial(Xfx, Yfx)[0]
    pb.ufy_l[:] = radial(Xfy, Yfy)[1]
    return pb


def bubble_layer(n=64, R0=0.15, rho_ratio=20.0, St=0.2, dT=1.0, delta=None, mu=0.01, dt=1e-4, steps=100,
                 **kw) -> Problem:
    """Circular vapour bubble in liquid superheated by dT, with a linear thermal layer of
    thickness delta outside the interface and fluid at rest (a synthetic start where the
    planar similarity solution does not exist); outflow on all sides, lambda = cp = 1."""
    h = 1.0 / n
    if delta is None:
        delta = 2.0 * h
    pb = Problem("bubble_layer", n, n, h, dt=dt, steps=steps, rho_l=rho_ratio, rho_v=1.0, mu_l=mu, mu_v=mu,
                 lam_l=1.0, lam_v=1.0, cp_l=1.0, cp_v=1.0, T_sat=0.0, h_lg=1.0 * dT / St,
                 bc=(OUTFLOW,) * 4, T_bc=(None,) * 4, **kw)
    pb.meta.update(R0=R0, xc=0.5, yc=0.5, delta=delta)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: np.hypot(x - 0.5, y - 0.5) - R0, n, n, h)
    (Xc, Yc), _, _ = _grids(n, n, h, 0.0, 0.0)
    r = np.hypot(Xc - 0.5, Yc - 0.5)
    pb.T_l = dT * np.clip((r - R0) / delta, 0.0, 1.0)
    pb.T_v = np.zeros((n, n))
    _zero_flow(pb)
    return pb


def const_mdot_bubble(n=64, L=8.0, R0=2.0, mdot=0.1, rho_l=1000.0, rho_v=1.0,
                      mu_l=1e-3, mu_v=1.26e-5, dt=None, steps=100, **kw) -> Problem:
    """Bubble with an imposed constant mass flux, energy equation off (Sec. 3.3).

    Lengths in mm-like units on [-L/2, L/2]^2 centred on the bubble; outflow on all sides.
    """
    h = L / n
    if dt is None:
        dt = 0.1 * h * rho_v / abs(mdot)
    pb = Problem("const_mdot_bubble", n, n, h, x0=-L / 2, y0=-L / 2, dt=dt, steps=steps,
                 rho_l=rho_l, rho_v=rho_v, mu_l=mu_l, mu_v=mu_v, T_sat=0.0, h_lg=1.0,
                 bc=(OUTFLOW,) * 4, T_bc=(None,) * 4, energy=False, mdot_fixed=mdot, **kw)
    pb.meta.update(R0=R0, mdot=mdot, xc=0.0, yc=0.0)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: np.hypot(x, y) - R0, n, n, h, -L / 2, -L / 2)
    pb.T_l = np.zeros((n, n))
    pb.T_v = np.zeros((n, n))
    _zero_flow(pb)
    return pb


def const_mdot_levelset(phi, n=48, L=1.0, mdot=1.0, rho_l=10.0, rho_v=1.0, mu=0.01, dt=None, cfl=0.35,
                        name="levelset", steps=4, **kw) -> Problem:
    """An arbitrary initial interface (liquid where phi > 0) with an imposed constant mass flux
    and the energy equation off (Sec. 3.3), at rest, outflow on all sides, on [0, L]^2.  Used
    for the topology cases: growing discs that merge, a condensing film that annihilates,
    saddle-shaped level sets, and a bubble that crosses the domain boundary.  dt defaults to
    moving the interface cfl cells per step relative to the vapour (mdot dt / (rho_v h))."""
    h = L / n
    if dt is None:
        dt = cfl * h * rho_v / abs(mdot)
    pb = Problem(name, n, n, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v, mu_l=mu, mu_v=mu,
                 T_sat=0.0, h_lg=1.0, bc=(OUTFLOW,) * 4, T_bc=(None,) * 4, energy=False, mdot_fixed=mdot, **kw)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(phi, n, n, h)
    pb.T_l = np.zeros((n, n))
    pb.T_v = np.zeros((n, n))
    _zero_flow(pb)
    return pb


def film(nx=1024, ny=2048, Lx=1.0, mean=0.05, amp=0.005, modes=None, seed=0,
         rho_l=5.0, rho_v=1.0, mu_l=5e-3, mu_v=1e-3, lam_l=1e-2, lam_v=1e-3,
         St=0.064, dT=1.0, g=-1.0, dt=None, steps=5000, **kw) -> Problem:
    """Film boiling over a heated wall: vapour film y < eta(x), eta = mean + sum_k a_k cos(2 pi k x / Lx).

    Bottom: no-slip wall at T_sat + dT; top: outflow; sides: symmetry.  The seed picks the
    number of modes (1-4 unless given) and a random sign per mode (the side walls are
    symmetry planes, so each mode is a cosine).
    """
    h = Lx / nx
    rng = np.random.default_rng(seed)
    if modes is None:
        modes = int(rng.integers(1, 5))
    signs = rng.choice([-1.0, 1.0], size=modes)
    a = amp / modes
    h_lg = 1.0 * dT / St
    if dt is None:
        dt = 0.25 * h
    pb = Problem("film", nx, ny, h, dt=dt, steps=steps, rho_l=rho_l, rho_v=rho_v,
                 mu_l=mu_l, mu_v=mu_v, lam_l=lam_l, lam_v=lam_v, cp_l=1.0, cp_v=1.0,
                 T_sat=0.0, h_lg=h_lg, gx=0.0, gy=g, bc=(SYMMETRY, SYMMETRY, WALL, OUTFLOW),
                 T_bc=(None, None, dT, None), **kw)
    ks = np.arange(1, modes + 1)

    def eta(x):
        x = np.asarray(x, dtype=float)
        return mean + a * np.sum(signs[:, None] * np.cos(2 * np.pi * ks[:, None] * x.ravel()[None, :] / Lx),
                                 axis=0).reshape(x.shape)

    pb.meta.update(modes=modes, signs=signs.tolist(), amp=a, mean=mean)
    pb.vcol, pb.hx_cut, pb.hx_pos, pb.vy_cut, pb.vy_pos = interface_from_levelset(
        lambda x, y: y - eta(x), nx, ny, h)
    (Xc, Yc), _, _ = _grids(nx, ny, h, 0.0, 0.0)
    e = eta(Xc[0])[None, :]
    pb.T_v = dT * (1.0 - Yc / e)
    pb.T_l = np.zeros((ny, nx))
    _zero_flow(pb)
    return pb


def one_fluid(pb: Problem) -> Problem:
    """The same problem for the one-fluid variant (Sec. 2.3): one velocity field, composed from
    the generator's two phase fields -- the liquid field in cells whose corners are mostly
    liquid, the vapour field elsewhere; faces take the liquid field when both end vertices are
    liquid.  Only the initial single field is composed here; the method's arithmetic is not."""
    q = pb.copy()
    q.one_fluid = True
    q.name = pb.name + "_one_fluid"
    vc = q.vcol.astype(float)
    cc = (vc[:-1, :-1] + vc[:-1, 1:] + vc[1:, :-1] + vc[1:, 1:]) > 2.0
    q.u_l = np.where(cc[..., None], pb.u_l, pb.u_v)
    fx = (vc[:-1, :] + vc[1:, :]) > 1.5          # x-faces: both end vertices liquid
    fy = (vc[:, :-1] + vc[:, 1:]) > 1.5
    q.ufx_l = np.where(fx, pb.ufx_l, pb.ufx_v)
    q.ufy_l = np.where(fy, pb.ufy_l, pb.ufy_v)
    q.u_v, q.ufx_v, q.ufy_v = q.u_l.copy(), q.ufx_l.copy(), q.ufy_l.copy()
    return q


def c1_stefan(**kw):
    return stefan(64, 64, X0=0.1, dt=1e-4, steps=100, **kw)


def c2_bubble(**kw):
    return bubble(512, **kw)


def c3_film(**kw):
    return film(1024, 2048, Lx=1.0, **kw)


def c5_film(**kw):
    return film(4096, 4096, Lx=8.0, modes=32, rho_l=50.0, rho_v=1.0, mu_l=1e-2, mu_v=1e-3,
                lam_l=1e-2, lam_v=1e-3, St=0.1, **kw)


def c5_film_half(**kw):
    """The 4096x4096 film's cell size and properties on the strip [0,4]x[0,8] (2048x4096, 16 modes)."""
    return film(2048, 4096, Lx=4.0, modes=16, rho_l=50.0, rho_v=1.0, mu_l=1e-2, mu_v=1e-3,
                lam_l=1e-2, lam_v=1e-3, St=0.1, **kw)


C4_SIDES = (32, 48, 64, 96, 128, 192, 256)


def c4_instance(k, seed=0):
    """Instance k of the batched workload: side from C4_SIDES, Stefan or bubble with p = 1/2,
    St ~ U[0.05, 0.5], rho_l / rho_v ~ U[2, 100], lambda = cp = 1 in both phases, dt from a CFL
    number of 0.2 on the closed-form interface (or liquid) speed at the start.  Bubbles start at
    R0 = 0.15 (at least 4.8 cells on the 32^2 grids), Stefan fronts at X0 = 0.1."""
    rng = np.random.default_rng([seed, k])
    n = int(rng.choice(C4_SIDES))
    kind = "stefan" if rng.random() < 0.5 else "bubble"
    St = float(rng.uniform(0.05, 0.5))
    ratio = float(rng.uniform(2.0, 100.0))
    h = 1.0 / n
    if kind == "stefan":
        beta = stefan_beta(St)
        t0 = (0.1 / (2 * beta)) ** 2      # alpha_v = 1
        speed = beta * math.sqrt(1.0 / t0)
        dt = 0.2 * h / speed
        pb = stefan(n, n, X0=0.1, rho_l=ratio, rho_v=1.0, St=St, dt=dt, steps=200)
    else:
        eps = 1.0 - 1.0 / ratio
        R0 = 0.15
        try:
            with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
                beta = bubble2d_beta(ratio * St, eps)
        except ValueError:
            beta = None   # Ja = ratio St beyond the planar similarity solution's range
        if beta is not None:
            alpha_l = 1.0 / ratio
            t0 = (R0 / (2 * beta)) ** 2 / alpha_l
            speed = beta * math.sqrt(alpha_l / t0)
            dt = 0.2 * h / speed
            pb = bubble(n, R0=R0, rho_ratio=ratio, k_ratio=1.0, St=St, dt=dt, steps=200, seed=0)
        else:
            delta = 2.0 * h
            speed = St / delta      # interface speed of a linear layer: lambda dT / (delta h_lg rho_v)
            pb = bubble_layer(n, R0=R0, rho_ratio=ratio, St=St, delta=delta, dt=0.2 * h / speed, steps=200)
    pb.meta.update(c4_index=k, c4_kind=kind, c4_St=St, c4_ratio=ratio)
    return pb


def c4_batch(count=4096, seed=0):
    """The batched workload: `count` independent instances (see c4_instance)."""
    return [c4_instance(k, seed) for k in range(count)]


WORKLOADS = {"c1_stefan": c1_stefan, "c2_bubble": c2_bubble, "c3_film": c3_film, "c5_film": c5_film,
             "c5_film_half": c5_film_half}
