"""Parity at the benchmark's full sizes: the 1024x2048 film (C3) and the 4096^2 multi-mode film
(C5), mixed precision at the benchmark's 1e-8 relative residual, the step in the launch
configuration the benchmark times (CUDA graph, TMA-staged persistent tiles, cooperative coarse
cycle).

At these sizes the oracle's sparse direct solves take minutes (one energy solve of C3: about two
minutes) to hours, so each solve is checked by a property that holds at any size: the GPU
solution's relative residual under the oracle's own FP64 assembly of the system, built from
the oracle's state, must meet the requested tolerance (an error in the GPU's ghost-fluid
coefficients, face weights or right-hand side shows there as a residual of the coefficient's
size).  The projected face field must be divergence-free to the same tolerance.  Everything
without a solve (preparation, T advection and extension, the EBIT sweeps and reconnection) is
compared with the oracle element by element from the same oracle-prepared state, the interface
bit for bit.  The graph-replayed step of the benchmark is compared bit for bit with the same
step run stage by stage, host-driven, with plain loads and separate coarse-level launches.
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
RTOL = 1e-8                 # the benchmark's relative residual
# a recomputed relative residual may exceed the solver's own by the rounding of two FP64
# evaluations of b - A x (a few ulps of |A||x| against |b|); the bar leaves room for that only
RES_BAR = 1.05 * RTOL
WORKLOADS = {"c3_film": w.c3_film, "c5_film": w.c5_film}


class Dev:
    def __init__(self):
        self.alloc = E.TorchAllocator()
        self.stream = torch.cuda.Stream()


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return Dev()


@pytest.fixture(scope="module", params=list(WORKLOADS))
def prep(request):
    """(name, the oracle's prepared initial state): module scope, so that pytest runs every test
    of one workload before the next and holds one full-size state at a time."""
    return request.param, S.prepare(WORKLOADS[request.param](steps=0))


def new_ctx(dev, pb, graph=True, tma=None, coop=None):
    ctx = E.ebit_init([E.config_from_problem(pb, E.EBIT_MIXED, RTOL, 400)], dev.stream.cuda_stream, dev.alloc)
    E.ebit_set_option(ctx, E.EBIT_OPT_GRAPH, 1 if graph else 0)
    if tma is not None:
        E.ebit_set_option(ctx, E.EBIT_OPT_TMA, tma)
    if coop is not None:
        E.ebit_set_option(ctx, E.EBIT_OPT_COOP, coop)
    return ctx


def upload(ctx, st):
    """The oracle state st into instance 0 (interface, fields, time) and its reconstruction."""
    E.upload_state(ctx, 0, st.pb, st.vcol, st.hx_pos, st.vy_pos, {k: getattr(st, k) for k in FIELDS}, st.t)
    E.ebit_run_stage(ctx, E.STAGE_RECONSTRUCT)


def relerr(a, b, scale=None):
    if scale is None:
        scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / max(scale, 1e-300))


def rel_residual(A, x, b):
    """||b - A x|| / ||b|| in FP64 (2-norms over the whole system, one per column)."""
    r = b - A @ x
    return np.linalg.norm(r, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)


def test_full_size_prepare_matches_oracle(dev, prep):
    """Preparation (reconstruction, T extension, mdot over the band, ghost velocities, initial
    accelerations) from the raw initial state, every cell and face."""
    name, so = prep
    pb = so.pb
    st = S.State(pb)
    ctx = new_ctx(dev, pb)
    try:
        E.upload_state(ctx, 0, pb, st.vcol, st.hx_pos, st.vy_pos, {k: getattr(st, k) for k in FIELDS}, st.t)
        E.ebit_run_stage(ctx, E.STAGE_PREPARE)
        g = E.download(ctx, 0, pb.nx, pb.ny, list(FIELDS) + ["vf", "ccol", "nb"])
        assert np.array_equal(g["ccol"], so.geom.ccol)
        assert np.array_equal(g["vf"], so.geom.vf)
        assert np.array_equal(g["nb"], so.geom.nb)
        for k in FIELDS:
            ref = getattr(so, k)
            scale = np.max(np.abs(ref))
            assert relerr(g[k], ref, scale if scale > 0 else 1.0) < 1e-12, k
    finally:
        E.ebit_destroy(ctx)


def test_full_size_energy_and_interface_stages(dev, prep):
    """S1 (WENO3 advection of T and the extension of T*) every cell, S2-S5 (u_Gamma, both sweeps,
    reconnection) bit for bit, then the energy solve on the new interface: the GPU's T under the
    oracle's ghost-fluid system (assembled from the oracle's T* and geometry) has a relative
    residual within the requested 1e-8, and the cells of the other phase keep T*."""
    name, st = prep
    pb = st.pb
    so = st.copy()
    ctx = new_ctx(dev, pb)
    try:
        upload(ctx, st)
        E.ebit_run_stage(ctx, E.STAGE_ADVECT_T)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["Ts_l", "Ts_v"])
        Ts_l, Ts_v = OE.advect_phases(so.T_l, so.T_v, so.u_l, so.u_v, so.geom.ccol, pb.T_bc, pb.dt, pb.h)
        assert relerr(g["Ts_l"], Ts_l) < 1e-13
        assert relerr(g["Ts_v"], Ts_v) < 1e-13
        E.ebit_run_stage(ctx, E.STAGE_EXTEND_TSTAR)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["Ts_l", "Ts_v"])
        Ts_l, Ts_v = OE.extend_temperatures(Ts_l, Ts_v, so.geom, pb.extend_iters)
        assert relerr(g["Ts_l"], Ts_l) < 1e-13
        assert relerr(g["Ts_v"], Ts_v) < 1e-13
        E.ebit_run_stage(ctx, E.STAGE_ADVANCE_INTERFACE)
        so.nstep = 0                      # the GPU context starts at step 0: x sweep first
        S.advance_interface(so)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["vcol", "hx_pos", "vy_pos", "ccol", "vf", "nb", "band"])
        assert np.array_equal(g["vcol"], so.vcol)
        assert np.array_equal(g["hx_pos"], so.hx_pos)
        assert np.array_equal(g["vy_pos"], so.vy_pos)
        assert np.array_equal(g["ccol"], so.geom.ccol)
        assert np.array_equal(g["vf"], so.geom.vf)
        assert np.array_equal(g["nb"], so.geom.nb)
        assert np.array_equal(g["band"].astype(bool), so.geom.band)
        E.ebit_run_stage(ctx, E.STAGE_SOLVE_ENERGY)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["T_l", "T_v"])
        A, b = OE.assemble_energy(so.geom, Ts_l, Ts_v, pb)
        liq = so.geom.ccol == 1
        x = np.where(liq, g["T_l"], g["T_v"]).ravel()
        res = rel_residual(A, x[:, None], b[:, None])[0]
        print(f"{name} energy: relative residual under the oracle's system {res:.2e}")
        assert res <= RES_BAR
        assert relerr(np.where(liq, g["T_v"], Ts_v), Ts_v) < 1e-13    # vapour T* kept in liquid cells
        assert relerr(np.where(liq, Ts_l, g["T_l"]), Ts_l) < 1e-13    # and the other way round
    finally:
        E.ebit_destroy(ctx)


def test_full_size_momentum_residuals(dev, prep):
    """S11 + S12 from the prepared state: the viscous solutions recovered from the stage's
    outputs (sol = u^{n+1} - dt gc^{n+1} + dt gc^n, Eqs. 11-15) meet the requested relative
    residual under the oracle's Helmholtz systems, for both components and both phase fields;
    the pressure meets it under the oracle's ghost-fluid Poisson system with the right-hand side
    of the recovered u_f*; and the projected face field of each cell's phase is divergence-free
    to the same tolerance."""
    name, st = prep
    pb = st.pb
    ctx = new_ctx(dev, pb)
    try:
        upload(ctx, st)
        E.ebit_run_stage(ctx, E.STAGE_MOMENTUM)
        g = E.download(ctx, 0, pb.nx, pb.ny, ["u_l", "u_v", "gc", "p", "ufx_l", "ufx_v", "ufy_l", "ufy_v"])
    finally:
        E.ebit_destroy(ctx)
    geom, dt = st.geom, pb.dt
    ustar = {"l": g["u_l"] - dt * g["gc"], "v": g["u_v"] - dt * g["gc"]}   # u** of Eq. 15
    for c in range(2):
        A, rhs = OF.viscous_system(pb, geom, st.u_l, st.u_v, st.gc, c)
        sol = np.stack([(ustar[k][..., c] + dt * st.gc[..., c]).ravel() for k in ("l", "v")], axis=1)
        res = rel_residual(A, sol, rhs)
        print(f"{name} viscous component {c}: relative residuals {res[0]:.2e} (liquid) {res[1]:.2e} (vapour)")
        assert np.all(res <= RES_BAR), (c, res)
    faces = OF.predicted_faces(pb, geom, ustar)
    rfx, rfy = OF.face_rho(pb, geom.vf)
    Ap = OF.poisson_matrix(pb, rfx, rfy)
    bp = OF.poisson_rhs(pb, geom.ccol, faces).ravel()
    res = rel_residual(Ap, g["p"].ravel()[:, None], bp[:, None])[0]
    print(f"{name} Poisson: relative residual under the oracle's system {res:.2e}")
    assert res <= RES_BAR
    # -h div u_f^{n+1} of each cell's phase is the Poisson residual of the final faces
    div = OF.poisson_rhs(pb, geom.ccol, {"l": (g["ufx_l"], g["ufy_l"]), "v": (g["ufx_v"], g["ufy_v"])})
    rd = np.linalg.norm(div) / np.linalg.norm(bp)
    print(f"{name} projected faces: ||h div u_f|| / ||h div u_f*|| {rd:.2e}")
    assert rd <= RES_BAR


def test_full_size_graph_step_equals_stages(dev, prep):
    """One whole step as the benchmark runs it (CUDA graph, TMA-staged persistent tile kernels,
    cooperative coarse cycle) and the same step run stage by stage from the host (plain loads,
    one launch per coarse level): identical bit for bit, every field and the interface."""
    name, st = prep
    pb = st.pb
    out = []
    for graph, tma, coop in ((True, 1, 1), (False, 0, 0)):
        ctx = new_ctx(dev, pb, graph=graph, tma=tma, coop=coop)
        try:
            upload(ctx, st)
            if graph:
                E.ebit_step(ctx, 1)
            else:
                for s in range(E.STAGE_ADVECT_T, E.STAGE_DIAGNOSTICS + 1):
                    E.ebit_run_stage(ctx, s)
            names = list(FIELDS) + ["vcol", "hx_pos", "vy_pos", "vf"]
            out.append((E.download(ctx, 0, pb.nx, pb.ny, names), E.ebit_get_diagnostics(ctx, 0)))
        finally:
            E.ebit_destroy(ctx)
    (a, da), (b, db) = out
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(da, db)


def _scale(st, k):
    """Magnitude a field is judged against: its group's max over the oracle state (temperatures
    together, velocities together; pressure at least rho_l |u|^2, mdot its own max)."""
    groups = (("T_l", "T_v"), ("u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v"))
    umax = max(np.max(np.abs(getattr(st, n))) for n in groups[1])
    if k == "p":
        return max(np.max(np.abs(st.p)), st.pb.rho_l * umax * umax, 1e-300)
    for names in groups:
        if k in names:
            return max(max(np.max(np.abs(getattr(st, n))) for n in names), 1e-300)
    return max(np.max(np.abs(getattr(st, k))), 1e-300)


def test_full_batch_sampled_instances_match_oracle(dev):
    """The whole batched workload (4096 Stefan / bubble instances of sides 32..256) as the
    benchmark runs it (mixed precision, CUDA graphs on the worker streams, schedules chosen by
    the autotuner), one step; one instance of each grid side and kind is compared with the
    oracle's step of that instance, every cell and face: interface bit for bit, fields within
    1e-7 of their group's magnitude with the refinement run to a 1e-12 relative residual."""
    pbs = w.c4_batch(4096)
    ctx = E.ebit_init([E.config_from_problem(pb, E.EBIT_MIXED, 1e-12, 600) for pb in pbs], dev.stream.cuda_stream,
                      dev.alloc)
    picks = {}
    for b, pb in enumerate(pbs):
        picks.setdefault((pb.nx, pb.meta["c4_kind"]), b)
    names = ("T_l", "T_v", "u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v", "p", "mdot", "vcol", "hx_pos",
             "vy_pos")
    try:
        for b, pb in enumerate(pbs):
            E.upload_state(ctx, b, pb, pb.vcol, np.where(pb.hx_cut > 0, pb.hx_pos, 0.0),
                           np.where(pb.vy_cut > 0, pb.vy_pos, 0.0),
                           {"T_l": pb.T_l, "T_v": pb.T_v, "u_l": pb.u_l, "u_v": pb.u_v, "ufx_l": pb.ufx_l,
                            "ufx_v": pb.ufx_v, "ufy_l": pb.ufy_l, "ufy_v": pb.ufy_v, "p": pb.p}, pb.t0)
        E.ebit_run_stage(ctx, E.STAGE_PREPARE)
        E.ebit_autotune(ctx, 2)
        E.ebit_step(ctx, 1, allow_noconv=True)   # judged below, cell by cell
        got = {b: E.download(ctx, b, pbs[b].nx, pbs[b].ny, names) for b in picks.values()}
    finally:
        E.ebit_destroy(ctx)
    assert len(picks) >= 10            # most (side, kind) pairs occur among 4096 draws
    for (n, kind), b in sorted(picks.items()):
        st = S.prepare(pbs[b])
        S.step(st)
        g = got[b]
        assert np.array_equal(g["vcol"], st.vcol), (n, kind)
        assert np.array_equal(g["hx_pos"], st.hx_pos) and np.array_equal(g["vy_pos"], st.vy_pos), (n, kind)
        worst = max(relerr(g[k], getattr(st, k), _scale(st, k)) for k in names[:10])
        print(f"instance {b} ({kind}, {n}^2): largest field error {worst:.2e}")
        assert worst <= 1e-7, (n, kind, worst)
