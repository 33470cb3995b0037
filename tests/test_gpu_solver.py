"""The library's multigrid-preconditioned CG on caller-supplied five-point systems (ebit_solve_system).

* brute force: random SPD systems on 8x8 grids against a dense numpy solve;
* sparse direct solves (scipy) on Poisson-type systems with a Dirichlet side only (the hardest
  case for the coarse-grid correction), square, non-square and ragged grids, below and above
  the tiled-kernel threshold, FP64 and FP32-inside-FP64-refinement;
* iteration counts bounded independently of the grid size (multigrid efficiency).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_13677_gb300 import ebit as E
from paper_2402_13677_gb300 import workloads as w


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return E.TorchAllocator(), torch.cuda.Stream()


def ctx_for(dev, nx, ny):
    pb = w.stefan(nx, ny, steps=0)
    return E.ebit_init([E.config_from_problem(pb)], dev[1].cuda_stream, dev[0])


def matrix(D, wl, wb):
    ny, nx = D.shape
    idx = np.arange(nx * ny).reshape(ny, nx)
    wr = np.zeros_like(wl); wr[:, :-1] = wl[:, 1:]
    wt = np.zeros_like(wb); wt[:-1, :] = wb[1:, :]
    diag = D + wl + wr + wb + wt
    rows = [idx.ravel(), idx[:, 1:].ravel(), idx[:, :-1].ravel(), idx[1:, :].ravel(), idx[:-1, :].ravel()]
    cols = [idx.ravel(), idx[:, :-1].ravel(), idx[:, 1:].ravel(), idx[:-1, :].ravel(), idx[1:, :].ravel()]
    vals = [diag.ravel(), -wl[:, 1:].ravel(), -wl[:, 1:].ravel(), -wb[1:, :].ravel(), -wb[1:, :].ravel()]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nx * ny, nx * ny))


def random_system(nx, ny, rng, kind):
    wl = np.zeros((ny, nx)); wb = np.zeros((ny, nx))
    if kind == "poisson_top":      # variable coefficient (density-jump like), Dirichlet top only
        rho = np.where(rng.random((ny, nx)) < 0.5, 1.0, 50.0)
        wl[:, 1:] = 2.0 / (rho[:, 1:] + rho[:, :-1])
        wb[1:, :] = 2.0 / (rho[1:, :] + rho[:-1, :])
        D = np.zeros((ny, nx)); D[-1, :] = 2.0 * wb[-1, :].mean()
    else:                          # random positive weights and diagonal
        wl[:, 1:] = rng.uniform(0.1, 2.0, (ny, nx - 1))
        wb[1:, :] = rng.uniform(0.1, 2.0, (ny - 1, nx))
        D = rng.uniform(0.0, 0.5, (ny, nx))
    return D, wl, wb


@pytest.mark.parametrize("prec", [E.EBIT_FP64, E.EBIT_MIXED])
@pytest.mark.parametrize("kind", ["random", "poisson_top"])
def test_dense_brute_force_8x8(dev, prec, kind):
    rng = np.random.default_rng(11)
    ctx = ctx_for(dev, 8, 8)
    try:
        D, wl, wb = random_system(8, 8, rng, kind)
        b = rng.normal(size=64)
        A = matrix(D, wl, wb).toarray()
        assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > 0
        xd = np.linalg.solve(A, b)
        x, it, rr = E.ebit_solve_system(ctx, 0, D, wl, wb, b, precision=prec, rtol=1e-12)
        assert rr <= 1e-12
        assert np.max(np.abs(x - xd)) <= 1e-9 * np.max(np.abs(xd))
    finally:
        E.ebit_destroy(ctx)


@pytest.mark.parametrize("shape", [(64, 64), (96, 160), (80, 88), (256, 256), (512, 256), (256, 1024)])
@pytest.mark.parametrize("prec", [E.EBIT_FP64, E.EBIT_MIXED])
def test_poisson_dirichlet_top_matches_sparse_direct_with_bounded_iterations(dev, shape, prec):
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny)
    ctx = ctx_for(dev, nx, ny)
    try:
        D, wl, wb = random_system(nx, ny, rng, "poisson_top")
        b = rng.normal(size=nx * ny)
        xr = spla.spsolve(matrix(D, wl, wb).tocsc(), b)
        x, it, rr = E.ebit_solve_system(ctx, 0, D, wl, wb, b, precision=prec, rtol=1e-10, max_iter=400)
        assert rr <= 1e-10
        assert np.max(np.abs(x - xr)) <= 1e-7 * np.max(np.abs(xr))
        assert it <= 60, f"{shape} needed {it} iterations"
    finally:
        E.ebit_destroy(ctx)


def test_two_right_hand_sides_equal_two_single_solves(dev):
    rng = np.random.default_rng(5)
    nx, ny = 160, 96
    ctx = ctx_for(dev, nx, ny)
    try:
        D, wl, wb = random_system(nx, ny, rng, "random")
        b1, b2 = rng.normal(size=nx * ny), rng.normal(size=nx * ny)
        x1, _, _ = E.ebit_solve_system(ctx, 0, D, wl, wb, b1, rtol=1e-12)
        x2, _, _ = E.ebit_solve_system(ctx, 0, D, wl, wb, b2, rtol=1e-12)
        b = np.stack([b1, b2], axis=1).ravel()
        x, _, _ = E.ebit_solve_system(ctx, 0, D, wl, wb, b, nr=2, rtol=1e-12)
        x = x.reshape(-1, 2)
        assert np.max(np.abs(x[:, 0] - x1)) <= 1e-10 * np.max(np.abs(x1))
        assert np.max(np.abs(x[:, 1] - x2)) <= 1e-10 * np.max(np.abs(x2))
    finally:
        E.ebit_destroy(ctx)
