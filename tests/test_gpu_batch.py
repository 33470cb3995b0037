"""Batched stepping: many independent instances of uneven size in one context.

The instances of a context replay their step graphs on a pool of worker streams, forked from and
joined to the context stream.  Every instance's arithmetic is independent of the others, so each
must equal, bit for bit, the same instance stepped alone; one instance is also checked against
the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_13677_gb300 import ebit as E
from paper_2402_13677_gb300 import workloads as w
from oracle import step as S

TOL64 = 1e-10
NAMES = ("T_l", "T_v", "u_l", "u_v", "ufx_l", "ufx_v", "ufy_l", "ufy_v", "p", "mdot", "vcol", "hx_pos", "vy_pos")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return E.TorchAllocator(), torch.cuda.Stream()


def batch_problems():
    """The first instances of the batched workload with sides up to 96 (both kinds, several
    sides), plus a 32x32 bubble, so that the batch exceeds the worker-stream pool."""
    out, k = [], 0
    while len(out) < 19:
        pb = w.c4_instance(k)
        if pb.nx <= 96:
            out.append(pb)
        k += 1
    out.append(w.bubble(32, R0=0.2, rho_ratio=5.0, k_ratio=1.0, St=0.2, dt=1e-4, steps=0))
    return out


def make_ctx(dev, pbs, precision=E.EBIT_FP64, rtol=None):
    if rtol is None:   # the mixed refinement converges to about 1e-12, FP64 further
        rtol = 1e-13 if precision == E.EBIT_FP64 else 1e-10
    alloc, stream = dev
    ctx = E.ebit_init([E.config_from_problem(pb, precision, rtol, 600) for pb in pbs], stream.cuda_stream, alloc)
    for b, pb in enumerate(pbs):
        E.upload_state(ctx, b, pb, pb.vcol, np.where(pb.hx_cut > 0, pb.hx_pos, 0.0),
                       np.where(pb.vy_cut > 0, pb.vy_pos, 0.0),
                       {"T_l": pb.T_l, "T_v": pb.T_v, "u_l": pb.u_l, "u_v": pb.u_v, "ufx_l": pb.ufx_l,
                        "ufx_v": pb.ufx_v, "ufy_l": pb.ufy_l, "ufy_v": pb.ufy_v, "p": pb.p}, pb.t0)
    E.ebit_run_stage(ctx, E.STAGE_PREPARE)
    return ctx


@pytest.mark.parametrize("precision", [E.EBIT_FP64, E.EBIT_MIXED])
def test_batched_instances_equal_single_instance_runs(dev, precision):
    pbs = batch_problems()
    assert len({pb.nx for pb in pbs}) >= 3 and {pb.name for pb in pbs} >= {"stefan", "bubble"}
    ctx = make_ctx(dev, pbs, precision)
    try:
        E.ebit_step(ctx, 2)
        got = [E.download(ctx, b, pb.nx, pb.ny, NAMES) for b, pb in enumerate(pbs)]
        diags = [E.ebit_get_diagnostics(ctx, b) for b in range(len(pbs))]
    finally:
        E.ebit_destroy(ctx)
    for b, pb in enumerate(pbs):
        one = make_ctx(dev, [pb], precision)
        try:
            E.ebit_step(one, 2)
            ref = E.download(one, 0, pb.nx, pb.ny, NAMES)
            dref = E.ebit_get_diagnostics(one, 0)
        finally:
            E.ebit_destroy(one)
        for k in NAMES:
            assert np.array_equal(got[b][k], ref[k]), (b, pb.name, pb.nx, k)
        # solver statistics (entries 6..11) and the physical diagnostics agree as well
        assert np.array_equal(diags[b][:9], dref[:9]), (b, diags[b], dref)


def test_batched_instance_matches_oracle(dev):
    pbs = batch_problems()
    ctx = make_ctx(dev, pbs, E.EBIT_FP64, rtol=1e-15)
    try:
        E.ebit_step(ctx, 1)
        b = min(range(len(pbs)), key=lambda i: pbs[i].nx)
        pb = pbs[b]
        g = E.download(ctx, b, pb.nx, pb.ny, NAMES)
    finally:
        E.ebit_destroy(ctx)
    st = S.prepare(pb)
    S.step(st)
    assert np.array_equal(g["vcol"], st.vcol)
    assert np.array_equal(g["hx_pos"], st.hx_pos) and np.array_equal(g["vy_pos"], st.vy_pos)
    t_scale = max(np.max(np.abs(st.T_l)), np.max(np.abs(st.T_v)))
    for k in ("T_l", "T_v"):
        assert np.max(np.abs(g[k] - getattr(st, k))) <= TOL64 * t_scale, k


def test_autotune_restores_state_and_picks_a_candidate(dev):
    pbs = batch_problems()[:6]
    ctx = make_ctx(dev, pbs, E.EBIT_MIXED)
    try:
        before = [E.download(ctx, b, pb.nx, pb.ny, NAMES) for b, pb in enumerate(pbs)]
        E.ebit_autotune(ctx, 1)
        after = [E.download(ctx, b, pb.nx, pb.ny, NAMES) for b, pb in enumerate(pbs)]
        for b in range(len(pbs)):
            for k in NAMES:
                assert np.array_equal(before[b][k], after[b][k]), (b, k)
            small, inner, tma, coop = E.ebit_get_schedule(ctx, b)
            assert small in (256, 1024, 4096) and inner in (1e-4, 1e-5) and tma in (0, 1) and coop in (0, 1, 2)
        E.ebit_step(ctx, 1)   # the tuned schedules step normally
        tuned = [E.download(ctx, b, pb.nx, pb.ny, ("T_l", "T_v", "vcol")) for b, pb in enumerate(pbs)]
    finally:
        E.ebit_destroy(ctx)
    ref_ctx = make_ctx(dev, pbs, E.EBIT_MIXED)
    try:
        E.ebit_step(ref_ctx, 1)
        for b, pb in enumerate(pbs):
            ref = E.download(ref_ctx, b, pb.nx, pb.ny, ("T_l", "T_v", "vcol"))
            assert np.array_equal(tuned[b]["vcol"], ref["vcol"])
            scale = max(np.max(np.abs(ref["T_l"])), np.max(np.abs(ref["T_v"])))
            for k in ("T_l", "T_v"):   # both solved to the same relative residual
                assert np.max(np.abs(tuned[b][k] - ref[k])) <= 1e-6 * scale, (b, k)
    finally:
        E.ebit_destroy(ref_ctx)


def test_batched_launch_timer_counts_each_launch_once(dev):
    """The device timer of the finest-level smoother kernels counts a batched launch once, with
    the algorithmic bytes of all its instances: a batch of four identical instances reports as
    many timed launches as one instance stepped alone, and four times its bytes per launch."""
    pb = batch_problems()[0]
    nz = 4
    out = []
    for count in (nz, 1):
        ctx = make_ctx(dev, [pb] * count, E.EBIT_MIXED)
        try:
            E.ebit_step(ctx, 1)
            E.ebit_timing_begin(ctx)
            E.ebit_step(ctx, 1)
            out.append(E.ebit_timing_end(ctx))
        finally:
            E.ebit_destroy(ctx)
    (ms_b, n_b, b_b), (ms_1, n_1, b_1) = out
    assert n_1 > 0 and n_b == n_1
    assert ms_b > 0 and ms_1 > 0
    assert b_b == pytest.approx(nz * b_1, rel=1e-12)


def axi_batch_problems():
    """Axisymmetric instances: three constant-flux spheres of different densities and
    viscosities (one batch: the grid, boundaries and imposed flux are shared) and two Scriven
    bubbles of different density ratios (a second batch, energy on)."""
    out = [w.axi_const_mdot_bubble(n=32, R0=0.3, rho_l=rl, mu=mu, dt=1e-3, steps=0)
           for rl, mu in ((10.0, 0.01), (20.0, 0.02), (5.0, 0.005))]
    out += [w.scriven(n=32, R0=0.3, rho_ratio=rr, dt=2e-5, steps=0) for rr in (20.0, 10.0)]
    return out


@pytest.mark.parametrize("precision", [E.EBIT_FP64, E.EBIT_MIXED])
def test_batched_axisymmetric_instances_equal_single_instance_runs(dev, precision):
    pbs = axi_batch_problems()
    ctx = make_ctx(dev, pbs, precision)
    try:
        E.ebit_step(ctx, 2)
        got = [E.download(ctx, b, pb.nx, pb.ny, NAMES) for b, pb in enumerate(pbs)]
    finally:
        E.ebit_destroy(ctx)
    for b, pb in enumerate(pbs):
        one = make_ctx(dev, [pb], precision)
        try:
            E.ebit_step(one, 2)
            ref = E.download(one, 0, pb.nx, pb.ny, NAMES)
        finally:
            E.ebit_destroy(one)
        for k in NAMES:
            assert np.array_equal(got[b][k], ref[k]), (b, pb.name, k)
