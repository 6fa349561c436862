"""A different element order per axis (hofem_plan_orders): solves, the operator, f^h and
algorithm (b) against the oracle, which takes one order per axis throughout."""
import numpy as np
import pytest

from oracle import assemble, load as oload, solve as osolve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_07758_gb300 import build as b
    b.build()


def H():
    import paper_1609_07758_gb300 as hofem
    return hofem


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


CASES = [([2, 5], [32, 12], [1.0, 0.7], 0.0), ([9, 3], [8, 37], [1.2, 1.0], 1.0),
         ([3, 1, 4], [6, 9, 5], [1.0, 0.8, 1.5], 0.0), ([16, 2], [2, 16], [1.0, 1.0], 0.0)]


@pytest.mark.parametrize("ns,Ks,Xs,alpha", CASES)
@pytest.mark.parametrize("dtype,tol", [(0, 1e-12), (1, 1e-5), (4, 1e-12)])
def test_solve_with_per_axis_orders(ns, Ks, Xs, alpha, dtype, tol):
    if dtype == 4 and max(ns) > 9:
        pytest.skip("refinement is held to n <= 9")
    N = len(Ks)
    plan = H().Plan(N, Ks, ns, Xs, dtype, alpha)
    assert list(plan.info().orders)[:N] == ns
    Ms = [n * k - 1 for n, k in zip(ns, Ks)]
    f = np.random.default_rng(sum(ns)).standard_normal([2] + Ms)
    ref = osolve.solve_tensor(f, ns, Ks, Xs, alpha)
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros_like(fd)
    plan.solve(fd, ud, 2)
    torch.cuda.synchronize()
    assert rel(ud.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("ns,Ks,Xs,alpha", CASES)
def test_operator_load_and_banded_with_per_axis_orders(ns, Ks, Xs, alpha):
    N = len(Ks)
    plan = H().Plan(N, Ks, ns, Xs, 0, alpha)
    Ms = [n * k - 1 for n, k in zip(ns, Ks)]
    v = np.random.default_rng(7).standard_normal([1] + Ms)
    r = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
    plan.apply(torch.from_numpy(v).cuda(), r, 1)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy(), assemble.apply_operator(v, ns, Ks, Xs, alpha)) <= 1e-13
    pts = [plan.quadrature_points(i) for i in range(N)]
    for i, (n, K, X) in enumerate(zip(ns, Ks, Xs)):
        np.testing.assert_allclose(pts[i], oload.quadrature_1d(n, K, X)[0], rtol=0, atol=4e-16 * X)
    f = lambda *x: np.exp(x[0]) * np.cos(2 * x[1]) + sum(x)
    grids = np.meshgrid(*[oload.quadrature_1d(n, K, X)[0] for n, K, X in zip(ns, Ks, Xs)], indexing="ij")
    fh = torch.zeros((1,) + tuple(Ms), dtype=torch.float64, device="cuda")
    plan.load(torch.from_numpy(f(*grids)[None].copy()).cuda(), fh, 1)
    torch.cuda.synchronize()
    # the oracle evaluates the basis by FP64 Horner on its monomial coefficients, which
    # cancels to ~1e-13 at order 16 (the library's table is double-double)
    tol = 1e-14 if max(ns) <= 9 else 1e-12
    assert rel(fh.cpu().numpy()[0], oload.load_vector(f, ns, Ks, Xs)) <= tol
    if ns[0] <= 9:
        ub = torch.zeros_like(fh)
        plan.solve_banded(fh, ub, 1)
        torch.cuda.synchronize()
        ref = osolve.solve_tensor(fh.cpu().numpy(), ns, Ks, Xs, alpha)
        assert rel(ub.cpu().numpy(), ref) <= 1e-12
