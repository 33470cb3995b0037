"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded inputs.

Bar (stated by the method's GPU design): cut-edge flags, topology and reconnection
bit-exact; temperature, pressure, velocities and marker positions within 1e-10 relative
(to the field group's magnitude) in the FP64 path; the mixed path (FP32 inside the FP64
refinement of the solves, everything else FP64) within 1e-7.
The FP64 solves run to a 1e-15 relative residual here: the error of a solve is bounded by
its relative residual times the condition number (1e3-1e5 for these Poisson operators), so
1e-10 on the solution needs a residual below ~1e-14.

Each stage test starts GPU and oracle from the *same* state (the oracle's state uploaded
through ebit_set_*), runs one stage on both and compares.  Interface stages are compared
bit for bit: both sides perform the same IEEE operations in the same order.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_13677_gb300 import ebit as E
from paper_2402_13677_gb300 import workloads as w
from oracle import energy as OE
from oracle import flow as OF
from oracle import step as S

FIELDS = ("T_l", "T_v", "u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v", "p", "gc", "mdot")
TOL64 = 1e-10


class Dev:
    def __init__(self):
        self.alloc = E.TorchAllocator()
        self.stream = torch.cuda.Stream()   # non-default stream: ebit_step runs as a CUDA graph


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return Dev()


def gpu_ctx(dev, st, precision=E.EBIT_FP64, rtol=1e-15, max_iter=600, graph=True):
    pb = st.pb
    ctx = E.ebit_init([E.config_from_problem(pb, precision, rtol, max_iter)], dev.stream.cuda_stream, dev.alloc)
    E.ebit_set_option(ctx, E.EBIT_OPT_GRAPH, 1 if graph else 0)
    E.upload_state(ctx, 0, pb, st.vcol, st.hx_pos, st.vy_pos, {k: getattr(st, k) for k in FIELDS}, st.t)
    E.ebit_run_stage(ctx, E.STAGE_RECONSTRUCT)
    return ctx


def relerr(a, b, scale=None):
    """max |a - b| relative to `scale` (default: max |b|, at least 1e-300)."""
    if scale is None:
        scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / max(scale, 1e-300))


GROUPS = {"T": ("T_l", "T_v"), "U": ("u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v"), "p": ("p",),
          "gc": ("gc",), "mdot": ("mdot",)}


def group_scale(st, k):
    """Magnitude a field is judged against: its group's max over the oracle state (velocities
    together, temperatures together); fields that are identically zero in a case (vapour at
    T_sat, the y-velocity of the 1D Stefan problem) are thereby compared absolutely."""
    umax = max(np.max(np.abs(getattr(st, n))) for n in GROUPS["U"])
    if k == "p":   # pressure: at least the dynamic pressure rho_l |u|^2 of the state
        return max(np.max(np.abs(st.p)), st.pb.rho_l * umax * umax, 1e-300)
    if k == "gc":  # acceleration: at least |g| and u^2 over the domain size (a flow at rest or in
        # uniform motion has gc at round-off, which is not a scale)
        L = min(st.pb.nx, st.pb.ny) * st.pb.h
        return max(np.max(np.abs(st.gc)), abs(st.pb.gx), abs(st.pb.gy), umax * umax / L, 1e-300)
    for names in GROUPS.values():
        if k in names:
            return max(max(np.max(np.abs(getattr(st, n))) for n in names), 1e-300)
    return max(np.max(np.abs(getattr(st, k))), 1e-300)


def _translating_film(n=48):
    """A liquid film 0.6 cells thick around a row of vertices, carried up half a cell per step
    by a uniform flow (no phase change): its lower marker crosses the vertex row, which flips,
    and the film's edges become uncut (EBIT annihilation of a sub-cell film)."""
    h = 1.0 / n
    pb = w.const_mdot_levelset(lambda x, y: np.abs(y - 25.05 * h) - 0.3 * h, n=n, mdot=0.0, dt=0.5 * h,
                               name="annihilate")
    for k in ("u_l", "u_v"):
        getattr(pb, k)[..., 1] = 1.0
    pb.ufy_l[:] = 1.0
    pb.ufy_v[:] = 1.0
    return pb


def _merging_discs(n=48, gap=0.3):
    """Two vapour discs 0.3 cells apart growing at an imposed mass flux: they merge, split and
    merge again at their contact within four steps."""
    h, R = 1.0 / n, 0.15
    d = R + gap * h / 2
    return w.const_mdot_levelset(lambda x, y: np.minimum(np.hypot(x - 0.4969 + d, y - 0.5013) - R,
                                                         np.hypot(x - 0.4969 - d, y - 0.5013) - R),
                                 n=n, mdot=1.0, name="merge")


def _with_sigma(pb, sigma):
    pb.sigma = sigma
    pb.name += "_sigma"
    return pb


def cases():
    return {
        "stefan": lambda: w.stefan(48, 8, X0=0.23, Lx=1.0, dt=2e-4, steps=0),
        "bubble": lambda: w.bubble(n=48, R0=0.17, rho_ratio=5.0, k_ratio=3.0, St=0.3, mu=0.01, dt=1e-4, steps=0),
        "film": lambda: w.film(40, 56, Lx=1.0, mean=0.31, amp=0.04, modes=2, seed=3, steps=0, dt=2e-3),
        "mdot_bubble": lambda: w.const_mdot_bubble(n=40, L=8.0, R0=2.1, mdot=0.1, dt=0.1, steps=0),
        # above 4096 cells: the tiled multigrid kernels run (32x32 tiles, ragged in x and y here)
        "bubble_mid": lambda: w.bubble(n=96, R0=0.21, rho_ratio=5.0, k_ratio=3.0, St=0.3, mu=0.01, dt=5e-5, steps=0),
        "film_mid": lambda: w.film(80, 88, Lx=1.0, mean=0.27, amp=0.03, modes=3, seed=5, steps=0, dt=1e-3),
        # topology: merging and splitting discs, an annihilated film, 36 saddle cells whose
        # liquid components pinch off, a bubble cut by the outflow boundary (markers held on it)
        "merge": _merging_discs,
        "annihilate": _translating_film,
        "saddle": lambda: w.const_mdot_levelset(
            lambda x, y: np.cos(6 * np.pi * (x + 0.0104)) * np.cos(6 * np.pi * (y + 0.009)) + 0.01, n=48,
            mdot=0.5, cfl=0.1, name="saddle"),
        "outflow": lambda: w.const_mdot_levelset(lambda x, y: np.hypot(x - 0.9, y - 0.47) - 0.17, n=48, mdot=1.0,
                                                 cfl=0.2, name="outflow"),
        # the sucking problem (Sec. 3.2): vapour at rest at T_sat, thin thermal layer in the liquid
        "sucking": lambda: w.sucking(48, 8, dt=2.5e-3, steps=0),
        # surface tension (CSF with marker-circle curvature): a static bubble, a film under
        # gravity whose Taylor wavelength is the domain width, a growing bubble
        "static_sigma": lambda: _with_sigma(w.const_mdot_levelset(
            lambda x, y: np.hypot(x - 0.5013, y - 0.4987) - 0.2, n=48, mdot=0.0, dt=2e-4, rho_l=10.0, rho_v=1.0,
            mu=0.05, name="static_sigma"), 1.0),
        "film_sigma": lambda: _with_sigma(w.film(40, 56, Lx=1.0, mean=0.31, amp=0.04, modes=2, seed=3, steps=0,
                                                 dt=1e-3), 4.0 / (12 * np.pi ** 2)),
        "bubble_sigma": lambda: _with_sigma(w.bubble(n=64, R0=0.17, rho_ratio=5.0, k_ratio=3.0, St=0.3, mu=0.01,
                                                     dt=1e-4, steps=0), 0.05),
        # the one-fluid variant (single velocity field, phase-change source in the projection)
        "stefan_1f": lambda: w.one_fluid(w.stefan(48, 8, X0=0.23, Lx=1.0, dt=2e-4, steps=0)),
        "bubble_1f": lambda: w.one_fluid(w.bubble(n=64, R0=0.17, rho_ratio=5.0, k_ratio=3.0, St=0.3, mu=0.01,
                                                  dt=1e-4, steps=0)),
        # axisymmetric (r, z), axis on the left: a sphere with an imposed mass flux, the Scriven
        # problem (Sec. 3.4) and a static sphere held by surface tension (curvature 2 / R)
        "axi_sphere": lambda: w.axi_const_mdot_bubble(n=48, R0=0.3, steps=0),
        "scriven": lambda: w.scriven(n=48, R0=0.3, steps=0),
        "axi_sigma": lambda: _with_sigma(w.axi_const_mdot_bubble(n=48, R0=0.3, mdot=0.0, dt=2e-4, mu=0.05,
                                                                 steps=0), 1.0),
    }


TOPOLOGY = ["merge", "annihilate", "saddle", "outflow"]


CASES = list(cases().keys())


def prepared(name, nsteps=0):
    pb = cases()[name]()
    st = S.prepare(pb)
    for _ in range(nsteps):
        S.step(st)
    return st


# ----------------------------------------------------------------------------- geometry
@pytest.mark.parametrize("name", CASES)
def test_reconstruction_bit_exact(dev, name):
    st = prepared(name)
    ctx = gpu_ctx(dev, st)
    try:
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny, ["vf", "ccol", "band", "nb", "cseg"])
        o = st.geom
        assert np.array_equal(g["ccol"], o.ccol)
        assert np.array_equal(g["band"].astype(bool), o.band)
        code = g["cseg"].astype(np.int64)
        nseg = (code & 3).astype(np.int8)
        assert np.array_equal(nseg, o.nseg)
        for s in range(2):
            P = np.where(nseg > s, (code >> (2 + 4 * s)) & 3, -1)
            Q = np.where(nseg > s, (code >> (4 + 4 * s)) & 3, -1)
            assert np.array_equal(P, o.segP[..., s]) and np.array_equal(Q, o.segQ[..., s])
        assert np.array_equal(g["vf"], o.vf)          # same operations, same order
        assert np.array_equal(g["nb"], o.nb)
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("name", CASES)
def test_prepare_matches_oracle(dev, name):
    pb = cases()[name]()
    st = S.State(pb)
    ctx = E.ebit_init([E.config_from_problem(pb, E.EBIT_FP64, 1e-15, 600)], dev.stream.cuda_stream, dev.alloc)
    try:
        E.upload_state(ctx, 0, pb, st.vcol, st.hx_pos, st.vy_pos, {k: getattr(st, k) for k in FIELDS}, st.t)
        E.ebit_run_stage(ctx, E.STAGE_PREPARE)
        so = S.prepare(pb)
        g = E.download(ctx, 0, pb.nx, pb.ny, list(FIELDS))
        for k in FIELDS:
            assert relerr(g[k], getattr(so, k), group_scale(so, k)) < 1e-12, k
    finally:
        E.ebit_destroy(ctx)


# ----------------------------------------------------------------------------- stages
@pytest.mark.parametrize("name", ["stefan", "bubble", "film", "sucking", "scriven"])
def test_energy_advection_and_extension(dev, name):
    st = prepared(name, 1)
    ctx = gpu_ctx(dev, st)
    try:
        E.ebit_run_stage(ctx, E.STAGE_ADVECT_T)
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny, ["Ts_l", "Ts_v"])
        pb = st.pb
        Tl, Tv = OE.advect_phases(st.T_l, st.T_v, st.u_l, st.u_v, st.geom.ccol, pb.T_bc, pb.dt, pb.h)
        assert relerr(g["Ts_l"], Tl) < 1e-13 or np.max(np.abs(Tl)) == 0
        assert relerr(g["Ts_v"], Tv) < 1e-13
        E.ebit_run_stage(ctx, E.STAGE_EXTEND_TSTAR)
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny, ["Ts_l", "Ts_v"])
        Tl, Tv = OE.extend_temperatures(Tl, Tv, st.geom, pb.extend_iters)
        assert np.max(np.abs(g["Ts_l"] - Tl)) <= 1e-13 * max(1.0, np.max(np.abs(Tl)))
        assert np.max(np.abs(g["Ts_v"] - Tv)) <= 1e-13 * max(1.0, np.max(np.abs(Tv)))
    finally:
        E.ebit_destroy(ctx)


def set_counter(ctx, st, n):
    """Step counter of the GPU instance (it picks the sweep order) and of the oracle state."""
    E.ebit_set_time(ctx, 0, st.t)
    for _ in range(n):
        E.ebit_run_stage(ctx, E.STAGE_DIAGNOSTICS)   # advances the counter (and the clock)
    st.nstep = n


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("order", [0, 1])
def test_interface_advance_bit_exact(dev, name, order):
    st = prepared(name, 1)
    ctx = gpu_ctx(dev, st)
    try:
        so = st.copy()
        set_counter(ctx, so, order)          # 0: x then y, 1: y then x
        E.ebit_run_stage(ctx, E.STAGE_ADVANCE_INTERFACE)
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny, ["vcol", "hx_pos", "vy_pos", "cseg", "vf", "ccol", "nb"])
        S.advance_interface(so)
        assert np.array_equal(g["vcol"], so.vcol)
        assert np.array_equal(g["hx_pos"], so.hx_pos)
        assert np.array_equal(g["vy_pos"], so.vy_pos)
        assert np.array_equal(g["ccol"], so.geom.ccol)
        assert np.array_equal(g["vf"], so.geom.vf)
        assert np.array_equal(g["nb"], so.geom.nb)
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("name", ["stefan", "bubble", "film", "sucking", "scriven"])
def test_energy_solve_flux_and_ghost_velocity(dev, name):
    st = prepared(name, 1)
    pb = st.pb
    # oracle: run the step up to the energy solve (step counter 0 on both sides)
    so = st.copy()
    Ts_l, Ts_v = OE.advect_phases(so.T_l, so.T_v, so.u_l, so.u_v, so.geom.ccol, pb.T_bc, pb.dt, pb.h)
    Ts_l, Ts_v = OE.extend_temperatures(Ts_l, Ts_v, so.geom, pb.extend_iters)
    so.nstep = 0
    S.advance_interface(so)
    ctx = gpu_ctx(dev, st)
    try:
        for s in (E.STAGE_ADVECT_T, E.STAGE_EXTEND_TSTAR, E.STAGE_ADVANCE_INTERFACE, E.STAGE_SOLVE_ENERGY):
            E.ebit_run_stage(ctx, s)
        so.T_l, so.T_v = OE.solve_energy(so.geom, Ts_l, Ts_v, pb)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["T_l", "T_v"])
        assert relerr(g["T_l"], so.T_l, group_scale(so, "T_l")) < TOL64
        assert relerr(g["T_v"], so.T_v, group_scale(so, "T_v")) < TOL64
        E.ebit_run_stage(ctx, E.STAGE_EXTEND_T)
        so.T_l, so.T_v = OE.extend_temperatures(so.T_l, so.T_v, so.geom, pb.extend_iters)
        E.ebit_run_stage(ctx, E.STAGE_MASS_FLUX)
        so.mdot = S.interface_mdot(so)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["T_l", "T_v", "mdot"])
        assert relerr(g["T_l"], so.T_l, group_scale(so, "T_l")) < TOL64
        assert relerr(g["T_v"], so.T_v, group_scale(so, "T_v")) < TOL64
        assert relerr(g["mdot"], so.mdot) < TOL64
        E.ebit_run_stage(ctx, E.STAGE_GHOST_VELOCITY)
        OF.ghost_velocities(so)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v"])
        for k in ("u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v"):
            assert relerr(g[k], getattr(so, k), group_scale(so, k)) < TOL64, k
    finally:
        E.ebit_destroy(ctx)


# ----------------------------------------------------------------------------- whole step
@pytest.mark.parametrize("name", CASES)
def test_full_step_fp64(dev, name):
    st = prepared(name, 1)
    ctx = gpu_ctx(dev, st)
    try:
        so = st.copy()
        so.nstep = 0                                 # ebit_set_time reset the GPU counter to 0
        E.ebit_step(ctx, 1)
        row = S.step(so)
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny)
        assert np.array_equal(g["vcol"], so.vcol)
        assert np.array_equal(g["hx_pos"], so.hx_pos)
        assert np.array_equal(g["vy_pos"], so.vy_pos)
        for k in FIELDS:
            e = relerr(g[k], getattr(so, k), group_scale(so, k))
            assert e < TOL64, (k, e)
        d = E.ebit_get_diagnostics(ctx, 0)
        assert abs(d[0] - row[0]) < 1e-12
        pb = st.pb
        umax = max(np.max(np.abs(getattr(so, n))) for n in GROUPS["U"])
        umax = max(umax, np.sqrt(np.max(np.abs(so.p)) / pb.rho_l))   # a fluid held at rest by its pressure
        L = min(pb.nx, pb.ny) * pb.h
        # scales: vapour volume and its expected change ~ the domain area; mass ~ rho_l area;
        # outlet mass per step ~ rho_l u L dt (sums whose terms cancel end at round-off of it)
        scale = {1: L * L, 2: L * L, 3: pb.rho_l * L * L, 4: pb.rho_l * umax * L * pb.dt}
        for q in (1, 2, 3, 4):
            assert abs(d[q] - row[q]) <= 1e-9 * max(abs(row[q]), 1e-6 * scale[q]), q
        assert d[5] == row[5]
        assert abs(d[12] - row[6]) <= 1e-9 * max(abs(row[6]), 1e-6 * scale[4] / pb.rho_l)   # vapour out
        assert abs(d[13] - row[7]) <= 1e-9 * max(abs(row[7]), 1e-12), (d[13], row[7])      # wall Nusselt
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("name", ["stefan", "bubble", "sucking", "stefan_1f", "bubble_1f", "static_sigma",
                                  "film_sigma", "axi_sphere", "scriven", "axi_sigma"])
def test_several_steps_track_the_oracle(dev, name):
    st = prepared(name, 0)
    ctx = gpu_ctx(dev, st)
    try:
        so = st.copy()
        so.nstep = 0
        for _ in range(4):
            E.ebit_step(ctx, 1)
            S.step(so)
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny)
        assert np.array_equal(g["vcol"], so.vcol)
        assert np.max(np.abs(g["hx_pos"] - so.hx_pos)) < 1e-10
        assert np.max(np.abs(g["vy_pos"] - so.vy_pos)) < 1e-10
        for k in FIELDS:
            assert relerr(g[k], getattr(so, k), group_scale(so, k)) < TOL64, k
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("name", TOPOLOGY)
def test_topology_changes_track_the_oracle(dev, name):
    """Four whole steps through merging, splitting, annihilation, saddle cells and a boundary-
    cut bubble: the first step's markers bit for bit, vertex colours (the topology) identical
    after every step, markers and fields within 1e-10."""
    from scipy import ndimage
    st = prepared(name, 0)
    ctx = gpu_ctx(dev, st)
    try:
        so = st.copy()
        so.nstep = 0
        seen = {(ndimage.label(so.vcol == 0)[1], ndimage.label(so.vcol == 1)[1])}
        for k in range(4):
            E.ebit_step(ctx, 1)
            S.step(so)
            g = E.download(ctx, 0, st.pb.nx, st.pb.ny)
            assert np.array_equal(g["vcol"], so.vcol), k
            if k == 0:
                assert np.array_equal(g["hx_pos"], so.hx_pos) and np.array_equal(g["vy_pos"], so.vy_pos)
            assert np.max(np.abs(g["hx_pos"] - so.hx_pos)) < TOL64
            assert np.max(np.abs(g["vy_pos"] - so.vy_pos)) < TOL64
            for f in FIELDS:
                e = relerr(g[f], getattr(so, f), group_scale(so, f))
                assert e < TOL64, (k, f, e)
            seen.add((ndimage.label(so.vcol == 0)[1], ndimage.label(so.vcol == 1)[1]))
        assert len(seen) > 1 or name == "outflow"   # the topology did change
    finally:
        E.ebit_destroy(ctx)


# Mixed mode: the solves are FP32 MG-PCG inside FP64 refinement; every explicit stencil (WENO3
# advection, operators, fluxes) is FP64.  The error of a solve is bounded by its residual times
# the condition number of the operator (up to ~1e5 for the projection with a density ratio of 20
# on 512^2), so the refinement runs to a 1e-12 relative residual here: what remains is the
# precision of the path, not the tolerance of the solve.
TOL_MIXED = 1e-7
RTOL_MIXED = 1e-12


@pytest.mark.parametrize("name", ["stefan", "bubble", "film", "bubble_mid"])
def test_mixed_precision_error_against_oracle(dev, name):
    """FP32 MG-PCG inside FP64 refinement to 1e-12, FP64 explicit stencils: error vs the FP64
    oracle stated and bounded."""
    st = prepared(name, 1)
    ctx = gpu_ctx(dev, st, precision=E.EBIT_MIXED, rtol=RTOL_MIXED)
    try:
        so = st.copy()
        so.nstep = 0
        E.ebit_step(ctx, 1)
        S.step(so)
        g = E.download(ctx, 0, st.pb.nx, st.pb.ny)
        assert np.array_equal(g["vcol"], so.vcol)
        for k in ("T_l", "T_v", "p", "u_l", "u_v"):
            e = relerr(g[k], getattr(so, k), group_scale(so, k))
            print(f"mixed {name} {k}: {e:.2e}")
            assert e < TOL_MIXED, (k, e)
    finally:
        E.ebit_destroy(ctx)


def test_c2_bubble_full_size_every_cell(dev):
    """512^2 planar bubble (the benchmark workload), one FP64 step and one mixed step, against the
    oracle's step from the same state: markers and vertex colours bit for bit, every cell and
    face of every field (temperatures, velocities, pressure, accelerations, mass flux) within
    1e-10 (FP64, solves to a 1e-15 relative residual) and 1e-7 (mixed, refinement to 1e-12)."""
    pb = w.c2_bubble(steps=0)
    st = S.prepare(pb)
    so = st.copy()
    S.step(so)
    for prec, tol, rtol in ((E.EBIT_FP64, TOL64, 1e-15), (E.EBIT_MIXED, TOL_MIXED, RTOL_MIXED)):
        ctx = gpu_ctx(dev, st, precision=prec, rtol=rtol, max_iter=2000)
        try:
            E.ebit_step(ctx, 1)
            g = E.download(ctx, 0, pb.nx, pb.ny)
            assert np.array_equal(g["vcol"], so.vcol)
            assert np.array_equal(g["hx_pos"], so.hx_pos)
            assert np.array_equal(g["vy_pos"], so.vy_pos)
            for k in FIELDS:
                e = relerr(g[k], getattr(so, k), group_scale(so, k))
                print(f"c2 512^2 {'fp64' if prec == E.EBIT_FP64 else 'mixed'} {k}: {e:.2e}")
                assert e <= tol, (prec, k, e)
        finally:
            E.ebit_destroy(ctx)


def test_edge_cases_empty_interface_and_invalid_input(dev):
    """No interface at all (single-phase liquid at rest), and an interface whose marker sits on a vertex."""
    pb = w.stefan(16, 8, X0=0.1, steps=0)
    pb.vcol[:] = 1
    pb.hx_pos[:] = 0
    pb.vy_pos[:] = 0
    pb.T_bc = (None, None, None, None)
    st = S.prepare(pb)
    ctx = gpu_ctx(dev, st)
    try:
        E.ebit_step(ctx, 2)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["vcol", "band", "mdot"])
        assert np.all(g["vcol"] == 1) and not g["band"].any() and not g["mdot"].any()
        bad = pb.hx_pos.copy()
        vcol = pb.vcol.copy()
        vcol[0, 0] = 0                    # cut edge (0,0) but fraction 0 -> rejected
        with pytest.raises(E.EbitError) as ei:
            E.ebit_set_interface(ctx, 0, vcol, bad, pb.vy_pos)
        assert ei.value.status == E.EBIT_ETOPO
        # a rejected upload (checked on the device) leaves the instance's interface unchanged
        assert np.all(E.download(ctx, 0, pb.nx, pb.ny, ["vcol"])["vcol"] == 1)
        vcol2 = pb.vcol.copy()
        vcol2[1, 1] = 2                   # not a colour
        with pytest.raises(E.EbitError) as ei:
            E.ebit_set_interface(ctx, 0, vcol2, pb.hx_pos, pb.vy_pos)
        assert ei.value.status == E.EBIT_EINVAL
        assert np.all(E.download(ctx, 0, pb.nx, pb.ny, ["vcol"])["vcol"] == 1)
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("prec", [E.EBIT_FP64, E.EBIT_MIXED])
def test_graph_replay_equals_host_driven_step(dev, prec):
    """The CUDA-graph step (solver loops as conditional nodes) and the host-driven step run the
    same kernels on the same data: the results are identical bit for bit."""
    st = prepared("bubble", 1)
    out = []
    for graph in (True, False):
        ctx = gpu_ctx(dev, st, precision=prec, rtol=1e-10, graph=graph)
        try:
            E.ebit_step(ctx, 3)
            out.append((E.download(ctx, 0, st.pb.nx, st.pb.ny), E.ebit_get_diagnostics(ctx, 0)))
        finally:
            E.ebit_destroy(ctx)
    (a, da), (b, db) = out
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(da[6:9], db[6:9])      # iteration counts


def test_solver_statistics_reported(dev):
    st = prepared("bubble", 0)
    ctx = gpu_ctx(dev, st, precision=E.EBIT_MIXED, rtol=1e-8)
    try:
        n0 = E.ebit_launch_count(ctx)
        E.ebit_step(ctx, 2)
        d = E.ebit_get_diagnostics(ctx, 0)
        assert d[6] > 0 and d[7] > 0 and d[8] > 0          # energy, viscous, Poisson iterations
        assert max(d[9], d[10], d[11]) <= 1e-8              # final relative residuals
        assert E.ebit_launch_count(ctx) - n0 > 50
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("name", ["bubble_mid", "film_mid"])
@pytest.mark.parametrize("precision", [E.EBIT_FP64, E.EBIT_MIXED])
def test_tma_staging_equals_plain_loads(dev, name, precision):
    """The tile kernels read the same values whether their regions are staged by TMA copies or
    loaded with ordinary loads: two steps agree bit for bit (80x88 also has a tiled level
    narrower than a TMA box, which falls back to ordinary loads)."""
    st = prepared(name, 0)
    rtol = 1e-13 if precision == E.EBIT_FP64 else 1e-10
    out = []
    for tma in (1, 0):
        ctx = gpu_ctx(dev, st, precision=precision, rtol=rtol)
        try:
            E.ebit_set_option(ctx, E.EBIT_OPT_TMA, tma)
            E.ebit_step(ctx, 2)
            out.append(E.download(ctx, 0, st.pb.nx, st.pb.ny))
        finally:
            E.ebit_destroy(ctx)
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("name", ["bubble_mid", "film_mid"])
@pytest.mark.parametrize("precision", [E.EBIT_FP64, E.EBIT_MIXED])
def test_cooperative_coarse_cycle_equals_separate_launches(dev, name, precision):
    """The coarse tiled levels and the single-block levels give the same values in one
    cooperative launch (grid barriers between the phases) as in one launch per level."""
    st = prepared(name, 0)
    rtol = 1e-13 if precision == E.EBIT_FP64 else 1e-10
    out = []
    for coop in (1, 0):
        ctx = gpu_ctx(dev, st, precision=precision, rtol=rtol)
        try:
            E.ebit_set_option(ctx, E.EBIT_OPT_COOP, coop)
            E.ebit_step(ctx, 2)
            out.append(E.download(ctx, 0, st.pb.nx, st.pb.ny))
        finally:
            E.ebit_destroy(ctx)
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("name", ["bubble_mid", "saddle", "stefan"])
@pytest.mark.parametrize("graph", [True, False])
def test_single_block_extension_equals_launch_per_sweep(dev, name, graph):
    """The narrow-band extensions give the same values with every Jacobi sweep in one thread
    block as with one launch per sweep over the whole device: two steps agree bit for bit."""
    st = prepared(name, 0)
    out = []
    for ext in (1, 0):
        ctx = gpu_ctx(dev, st, precision=E.EBIT_MIXED, rtol=1e-10)
        try:
            E.ebit_set_option(ctx, E.EBIT_OPT_GRAPH, 1 if graph else 0)
            E.ebit_set_option(ctx, E.EBIT_OPT_EXT_BLOCK, ext)
            E.ebit_step(ctx, 2)
            out.append(E.download(ctx, 0, st.pb.nx, st.pb.ny))
        finally:
            E.ebit_destroy(ctx)
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("name", ["bubble_mid", "film_mid", "saddle", "sucking", "axi_sphere"])
@pytest.mark.parametrize("graph", [True, False])
def test_persistent_inner_solve_matches_separate_kernels(dev, name, graph):
    """Mixed precision with each whole inner FP32 solve in one cooperative launch
    (EBIT_OPT_COOP = 2) against one kernel per V-cycle leg and CG update: the dot products are
    grouped differently, so the iterates differ by rounding; both refine to a relative residual
    of 1e-12, two steps agree to 1e-9 of each field group's scale, the vertex colours exactly
    and the markers to 1e-10 of a cell."""
    st = prepared(name, 0)
    out = []
    for coop in (2, 0):
        ctx = gpu_ctx(dev, st, precision=E.EBIT_MIXED, rtol=1e-12, graph=graph)
        try:
            E.ebit_set_option(ctx, E.EBIT_OPT_COOP, coop)
            E.ebit_step(ctx, 2)
            out.append(E.download(ctx, 0, st.pb.nx, st.pb.ny))
        finally:
            E.ebit_destroy(ctx)
    so = st.copy()
    assert np.array_equal(out[0]["vcol"], out[1]["vcol"])
    for k in ("hx_pos", "vy_pos"):
        assert np.max(np.abs(out[0][k] - out[1][k])) < 1e-10, k
    for k in FIELDS:
        ref = out[1][k]
        setattr(so, k, ref)
    for k in FIELDS:
        assert relerr(out[0][k], out[1][k], group_scale(so, k)) < 1e-9, k


def test_batched_field_copies_equal_single_field_copies(dev):
    """ebit_set_fields / ebit_get_fields (one synchronisation per call) move the same bytes as
    one ebit_set_field / ebit_get_field per field, from and to page-locked host buffers and
    device buffers; bad entries are rejected before any copy."""
    st = prepared("bubble_mid", 0)
    nx, ny = st.pb.nx, st.pb.ny
    ctx = gpu_ctx(dev, st)
    try:
        E.ebit_step(ctx, 1)
        ids = [E.F_T_L, E.F_T_V, E.F_U_L, E.F_UFX_V, E.F_UFY_L, E.F_P, E.F_GC, E.F_MDOT, E.F_VCOL, E.F_HX_POS]
        ref = {f: E.ebit_get_field(ctx, 0, f) for f in ids}
        host = {f: torch.empty(ref[f].nbytes, dtype=torch.uint8, pin_memory=True) for f in ids}
        E.ebit_get_fields(ctx, 0, ids, [host[f].data_ptr() for f in ids], 0)
        for f in ids:
            assert np.array_equal(host[f].numpy().view(ref[f].dtype), ref[f]), f
        # device round trip: out to CUDA buffers, perturb the instance, back in
        devb = {f: torch.empty(ref[f].nbytes, dtype=torch.uint8, device="cuda") for f in ids}
        E.ebit_get_fields(ctx, 0, ids, [devb[f].data_ptr() for f in ids], 1)
        torch.cuda.synchronize()
        writable = [f for f in ids if f not in (E.F_VCOL, E.F_HX_POS)]
        for f in writable:
            E.ebit_set_field(ctx, 0, f, np.zeros_like(ref[f]))
        E.ebit_set_fields(ctx, 0, writable, [devb[f].data_ptr() for f in writable], 1)
        for f in writable:
            assert np.array_equal(E.ebit_get_field(ctx, 0, f), ref[f]), f
        # host upload of perturbed values, checked field by field
        for f in writable:
            host[f].numpy().view(ref[f].dtype)[:] = ref[f] + 1
        E.ebit_set_fields(ctx, 0, writable, [host[f].data_ptr() for f in writable], 0)
        for f in writable:
            assert np.array_equal(E.ebit_get_field(ctx, 0, f), ref[f] + 1), f
        with pytest.raises(E.EbitError) as ei:   # read-only field
            E.ebit_set_fields(ctx, 0, [E.F_T_L, E.F_VF], [host[E.F_T_L].data_ptr(), host[E.F_P].data_ptr()], 0)
        assert ei.value.status == E.EBIT_EINVAL
        assert np.array_equal(E.ebit_get_field(ctx, 0, E.F_T_L), ref[E.F_T_L] + 1)   # nothing copied
    finally:
        E.ebit_destroy(ctx)
