"""Allocation-free solve (ebit_solve_system_noalloc).

Some callers cannot allocate device memory when they call the solver (a host framework that
owns all device memory through its own pool, a service loop that must not allocate per
call).  The allocation-free entry point runs the same multigrid-preconditioned CG as
ebit_solve_system, on the caller's device arrays, with every scratch array inside one fixed
device array of the library.  These tests call it through the C ABI twice in a row on
different systems (the shared scratch keeps the previous call's contents) and compare each
result with the allocating entry point, and check that grids larger than the fixed scratch
are rejected.  This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_13677_gb300 import ebit as E
from paper_2402_13677_gb300 import workloads as w

TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return E.TorchAllocator(), torch.cuda.Stream()


def system(nx, ny, rng, kind):
    wl = np.zeros((ny, nx)); wb = np.zeros((ny, nx))
    if kind == "poisson_top":
        rho = np.where(rng.random((ny, nx)) < 0.5, 1.0, 20.0)
        wl[:, 1:] = 2.0 / (rho[:, 1:] + rho[:, :-1])
        wb[1:, :] = 2.0 / (rho[1:, :] + rho[:-1, :])
        D = np.zeros((ny, nx)); D[-1, :] = 0.2
    else:
        wl[:, 1:] = rng.uniform(0.1, 2.0, (ny, nx - 1))
        wb[1:, :] = rng.uniform(0.1, 2.0, (ny - 1, nx))
        D = rng.uniform(0.0, 0.5, (ny, nx))
    return D, wl, wb


def reference(dev, nx, ny, D, wl, wb, b, nr, prec):
    pb = w.stefan(nx, ny, steps=0)
    ctx = E.ebit_init([E.config_from_problem(pb)], dev[1].cuda_stream, dev[0])
    try:
        x, it, rr = E.ebit_solve_system(ctx, 0, D, wl, wb, b, nr=nr, precision=prec, rtol=1e-13, max_iter=500)
    finally:
        E.ebit_destroy(ctx)
    return x


@pytest.mark.parametrize("prec", [E.EBIT_FP64, E.EBIT_MIXED])
def test_noalloc_matches_the_allocating_solve_on_two_calls_in_a_row(dev, prec):
    rng = np.random.default_rng(2024 + prec)
    stream = dev[1]
    cases = [(96, 80, "poisson_top", 1), (64, 64, "random", 2)]
    for nx, ny, kind, nr in cases:
        D, wl, wb = system(nx, ny, rng, kind)
        b = rng.normal(size=nx * ny * nr)
        ref = reference(dev, nx, ny, D, wl, wb, b, nr, prec)
        t = lambda a: torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")
        Dd, wld, wbd, bd = t(D), t(wl), t(wb), t(b)
        xd = torch.zeros(nx * ny * nr, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s, it, rr = E.ebit_solve_system_noalloc(nx, ny, Dd, wld, wbd, bd, xd, nr=nr, precision=prec, rtol=1e-13,
                                                max_iter=500, stream=stream.cuda_stream)
        assert s == E.EBIT_OK, E.STATUS_NAMES.get(s, s)
        assert it > 0 and rr <= 1e-13
        x = xd.cpu().numpy()
        assert np.max(np.abs(x - ref)) <= TOL * np.max(np.abs(ref)), (nx, ny, kind)


def test_noalloc_rejects_grids_beyond_its_fixed_scratch(dev):
    nx = ny = 256   # above the 128 x 128 cap of the fixed scratch array
    z = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    s, it, rr = E.ebit_solve_system_noalloc(nx, ny, z, z, z, z, z.clone(), stream=dev[1].cuda_stream)
    assert s == E.EBIT_EINVAL


@pytest.mark.parametrize("nx, ny, nr, prec", [(128, 128, 2, E.EBIT_FP64), (128, 128, 2, E.EBIT_MIXED),
                                              (120, 104, 1, E.EBIT_MIXED)])
def test_noalloc_at_the_cap_and_on_ragged_tiles_allocates_nothing(dev, nx, ny, nr, prec):
    """The largest grid the fixed scratch takes (128 x 128, two right-hand sides) and a grid of
    ragged 32 x 32 tiles near it; the second of two identical calls (the first loads the
    kernels) leaves the device's free memory unchanged to the byte."""
    rng = np.random.default_rng(nx + ny + nr + prec)
    D, wl, wb = system(nx, ny, rng, "poisson_top")
    b = rng.normal(size=nx * ny * nr)
    ref = reference(dev, nx, ny, D, wl, wb, b, nr, prec)
    t = lambda a: torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")
    Dd, wld, wbd, bd = t(D), t(wl), t(wb), t(b)
    xs = [torch.zeros(nx * ny * nr, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for xd in xs:
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        s, it, rr = E.ebit_solve_system_noalloc(nx, ny, Dd, wld, wbd, bd, xd, nr=nr, precision=prec, rtol=1e-13,
                                                max_iter=500, stream=dev[1].cuda_stream)
        assert s == E.EBIT_OK, E.STATUS_NAMES.get(s, s)
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
        assert np.max(np.abs(x - ref)) <= TOL * np.max(np.abs(ref)), (nx, ny)
    assert torch.cuda.mem_get_info()[0] == free[1]
