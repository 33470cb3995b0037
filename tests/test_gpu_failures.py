"""Failure paths of the step and of the solve entry points, on the GPU, through the C ABI.

Every failure here is made on the host or by a bounded device wait that is given a tiny bound;
none faults, traps or hangs the GPU:
  * a solve that reaches max_iter returns EBIT_ENOCONV with the step completed;
  * a time step that moves a marker a whole cell returns EBIT_ECFL (the sweep clamps every
    displaced position into the domain, so the step itself stays in bounds);
  * a NaN in a field the caller set reaches a linear solve within the step, which stops at
    the first non-finite residual norm: EBIT_ENONFINITE;
  * the grid barrier of the cooperative multigrid launch, given a bound of one poll, gives up
    before the other blocks arrive and records a fault: ebit_step and ebit_solve_system return
    EBIT_ECUDA; that launch reads only plain loads (no copies in flight), and a fresh context
    on the same device then steps normally.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_13677_gb300 import ebit as E
from paper_2402_13677_gb300 import workloads as w
from oracle import step as S

FIELDS = ("T_l", "T_v", "u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v", "p", "gc", "mdot")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return E.TorchAllocator(), torch.cuda.Stream()


def bubble(n=48):
    return w.bubble(n=n, R0=0.17 if n < 64 else 0.21, rho_ratio=5.0, k_ratio=3.0, St=0.3, mu=0.01,
                    dt=1e-4 if n < 64 else 5e-5, steps=0)


def make(dev, pb, precision=E.EBIT_FP64, rtol=1e-10, max_iter=600, graph=True, fields=None):
    st = S.prepare(pb)
    ctx = E.ebit_init([E.config_from_problem(pb, precision, rtol, max_iter)], dev[1].cuda_stream, dev[0])
    E.ebit_set_option(ctx, E.EBIT_OPT_GRAPH, 1 if graph else 0)
    vals = {k: getattr(st, k) for k in FIELDS}
    vals.update(fields or {})
    E.upload_state(ctx, 0, pb, st.vcol, st.hx_pos, st.vy_pos, vals, st.t)
    E.ebit_run_stage(ctx, E.STAGE_RECONSTRUCT)
    return ctx, st


@pytest.mark.parametrize("precision", [E.EBIT_FP64, E.EBIT_MIXED])
@pytest.mark.parametrize("graph", [True, False])
def test_max_iter_returns_enoconv_with_the_step_completed(dev, precision, graph):
    pb = bubble()
    ctx, st = make(dev, pb, precision, rtol=1e-14, max_iter=1, graph=graph)
    try:
        with pytest.raises(E.EbitError) as ei:
            E.ebit_step(ctx, 1)
        assert ei.value.status == E.EBIT_ENOCONV
        d = E.ebit_get_diagnostics(ctx, 0)
        assert abs(d[0] - (st.t + pb.dt)) < 1e-15     # the step was completed
        assert max(d[9], d[10], d[11]) > 1e-14         # some final residual above its target
        g = E.download(ctx, 0, pb.nx, pb.ny, ["T_l", "p", "u_l"])
        assert all(np.isfinite(v).all() for v in g.values())   # the last iterates are kept
        # the binding can be told to accept it
        E.ebit_step(ctx, 1, allow_noconv=True)
    finally:
        E.ebit_destroy(ctx)


def test_cfl_violation_returns_ecfl(dev):
    pb = bubble()
    st = S.prepare(pb)
    umax = max(np.abs(st.u_l).max(), np.abs(st.u_v).max())
    pb.dt = 3.0 * pb.h / umax              # markers near the fastest flow move about three cells
    ctx, _ = make(dev, pb)
    try:
        with pytest.raises(E.EbitError) as ei:
            E.ebit_step(ctx, 1)
        assert ei.value.status == E.EBIT_ECFL
        assert "reduce dt" in str(ei.value)
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("precision", [E.EBIT_FP64, E.EBIT_MIXED])
@pytest.mark.parametrize("field", ["T_l", "p"])
def test_nonfinite_field_is_reported(dev, precision, field):
    """A NaN set into the liquid temperature (reaches the energy solve) or the pressure (reaches
    the viscous solves through the face accelerations) is reported as EBIT_ENONFINITE."""
    pb = bubble()
    st = S.prepare(pb)
    bad = getattr(st, field).copy()
    bad[3, 5] = np.nan                      # a liquid cell far from the bubble
    ctx, _ = make(dev, pb, precision, fields={field: bad})
    try:
        with pytest.raises(E.EbitError) as ei:
            E.ebit_step(ctx, 1)
        assert ei.value.status == E.EBIT_ENONFINITE, ei.value
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("coop", [1, 2])
def test_grid_barrier_timeout_is_reported_as_a_fault(dev, coop):
    # 96^2 in the mixed path: the FP32 48^2 level and the single-block levels run in one
    # cooperative launch (coop 1), or each whole inner solve does (coop 2); in FP64 the
    # single-block kernel's shared memory leaves no room for a co-resident grid, so FP64 solves
    # launch every level separately and have no grid barrier
    precision = E.EBIT_MIXED
    pb = bubble(96)
    ctx, _ = make(dev, pb, precision)
    try:
        E.ebit_set_option(ctx, E.EBIT_OPT_COOP, coop)
        E.ebit_set_option(ctx, E.EBIT_OPT_BARRIER_SPIN, 1)
        with pytest.raises(E.EbitError) as ei:
            E.ebit_step(ctx, 1)
        assert ei.value.status == E.EBIT_ECUDA
        assert "bounded wait" in str(ei.value)
        # the same through the solve entry point (a caller-supplied Poisson-like system)
        rng = np.random.default_rng(3)
        n = pb.nx
        wl = np.zeros((n, n)); wl[:, 1:] = rng.uniform(0.5, 1.5, (n, n - 1))
        wb = np.zeros((n, n)); wb[1:, :] = rng.uniform(0.5, 1.5, (n - 1, n))
        D = np.zeros((n, n)); D[-1, :] = 1.0
        b = rng.normal(size=(n, n))
        with pytest.raises(E.EbitError) as ei:
            E.ebit_solve_system(ctx, 0, D, wl, wb, b, precision=precision, rtol=1e-10, max_iter=200)
        assert ei.value.status == E.EBIT_ECUDA
    finally:
        E.ebit_destroy(ctx)
    # the device and the library stay usable: a new context with the default bound steps cleanly
    ctx, _ = make(dev, pb, precision)
    try:
        E.ebit_step(ctx, 1)
    finally:
        E.ebit_destroy(ctx)
