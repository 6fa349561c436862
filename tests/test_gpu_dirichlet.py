"""GPU parity of hofem_lift_dirichlet (inhomogeneous Dirichlet data moved into f^h, the
remark after Eq. bvp glob 2) against oracle.dirichlet, and the lifted problem end to end
on the GPU: f^h by hofem_load, the lift, a solve; a polynomial of the element space is
reproduced exactly and a manufactured solution converges at Table 1's rate."""
import numpy as np
import pytest

from oracle import dirichlet as od

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("ns,Ks,Xs,alpha,nrhs", [
    ([2, 2], [3, 5], [1.0, 1.5], 0.7, 2),
    ([9, 9], [8, 4], [1.0, 1.0], 0.0, 1),
    ([4, 7], [6, 3], [0.5, 2.0], -1.0, 1),       # per-axis orders
    ([16, 1], [2, 9], [1.0, 1.0], 0.0, 1),
    ([3, 3, 3], [4, 3, 5], [1.0, 0.8, 1.2], 0.5, 2),
    ([2, 5, 1], [3, 2, 6], [1.0, 1.0, 1.0], 0.0, 1),
])
def test_lift_matches_oracle(ns, Ks, Xs, alpha, nrhs):
    N = len(Ks)
    plan = H().Plan(N, Ks, ns if len(set(ns)) > 1 else ns[0], Xs, H().HOFEM_FP64, alpha)
    Ps = [n * K + 1 for n, K in zip(ns, Ks)]
    rng = np.random.default_rng(sum(Ps))
    vb = rng.standard_normal([nrhs] + Ps)
    f = rng.standard_normal([nrhs] + [p - 2 for p in Ps])
    ref = f - od.lift(vb, ns, Ks, Xs, alpha)
    fd = dev(f)
    plan.lift_dirichlet(dev(vb), fd, nrhs)
    torch.cuda.synchronize()
    got = fd.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _lifted_solve(n, K, u_fun, f_fun, alpha, dtype):
    """GPU: f^h (hofem_load), lift of the boundary values of u, solve; returns (v, u) at the
    interior dofs."""
    plan = H().Plan(2, [K, K], n, [1.0, 1.0], dtype, alpha)
    xq = [np.array(plan.quadrature_points(a)) for a in range(2)]
    Xq = np.meshgrid(*xq, indexing="ij")
    fq = dev(f_fun(*Xq)[None])
    fh = torch.empty((1, n * K - 1, n * K - 1), dtype=torch.float64, device="cuda")
    plan.load(fq, fh, 1)
    g = od.full_grid([n, n], [K, K], [1.0, 1.0])
    G = np.meshgrid(*g, indexing="ij")
    ufull = u_fun(*G)
    plan.lift_dirichlet(dev(ufull[None]), fh, 1)
    v = torch.empty_like(fh)
    plan.solve(fh, v, 1)
    torch.cuda.synchronize()
    return v.cpu().numpy()[0], ufull[1:-1, 1:-1]


@pytest.mark.parametrize("dtype,tol", [(0, 1e-11), (4, 1e-11)])
def test_polynomial_with_boundary_data_is_exact(dtype, tol):
    alpha = 0.8
    u = lambda x, y: 1.0 + 2.0 * x - y + x * y + x * x - 0.5 * y * y
    f = lambda x, y: -1.0 + alpha * u(x, y)
    v, ue = _lifted_solve(2, 16, u, f, alpha, dtype)
    assert np.abs(v - ue).max() <= tol * np.abs(ue).max()


def test_manufactured_boundary_data_converge():
    alpha = 1.0
    u = lambda x, y: np.sin(0.5 * np.pi * x + 0.3) * np.exp(y)
    f = lambda x, y: (0.25 * np.pi ** 2 - 1.0 + alpha) * u(x, y)
    errs = []
    for K in (8, 16, 32):
        v, ue = _lifted_solve(2, K, u, f, alpha, H().HOFEM_FP64)
        errs.append(np.abs(v - ue).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 0.8 * 16) and np.all(ratios < 1.25 * 16), (errs, ratios)
