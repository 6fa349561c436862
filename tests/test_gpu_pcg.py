"""The solver as a preconditioner: the matrix-free variable-coefficient operator against
the oracle's quadrature definition, and preconditioned conjugate gradients against a
sparse direct solve of the oracle's assembled matrix."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble as oasm
from oracle import load as oload
from oracle import varcoef

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


def coefficient(n, Ks, Xs, amp=0.5):
    x = [oload.quadrature_1d(n, K, X)[0] for K, X in zip(Ks, Xs)]
    X1, X2 = np.meshgrid(*x, indexing="ij")
    return 1.0 + amp * np.sin(np.pi * X1 / Xs[0]) * np.cos(3.0 * X2)


@pytest.mark.parametrize("n,Ks,Xs", [(1, [9, 5], [1.0, 1.0]), (3, [12, 7], [1.3, 0.8]), (9, [4, 6], [1.0, 2.0]),
                                     (5, [37, 16], [1.0, 1.0])])
def test_varcoef_operator_matches_the_oracle(n, Ks, Xs):
    p = H().Plan(2, Ks, n, Xs, 0)
    aq = coefficient(n, Ks, Xs)
    Ms = [n * k - 1 for k in Ks]
    u = np.random.default_rng(n).standard_normal(Ms)
    r = torch.zeros(Ms, dtype=torch.float64, device="cuda")
    p.apply_varcoef(torch.from_numpy(aq).cuda(), torch.from_numpy(u).cuda(), r)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy(), varcoef.apply(u, n, Ks, Xs, aq)) <= 1e-13
    # a = 1 is the constant-coefficient operator of Eq. bvp glob 2 (alpha = 0)
    r1 = torch.zeros_like(r)
    p.apply_varcoef(torch.ones(aq.shape, dtype=torch.float64, device="cuda"), torch.from_numpy(u).cuda(), r1)
    torch.cuda.synchronize()
    assert rel(r1.cpu().numpy(), oasm.apply_operator(u[None], [n, n], Ks, Xs, 0.0)[0]) <= 1e-13


@pytest.mark.parametrize("dtype", [0, 4])
def test_pcg_matches_a_sparse_direct_solve(dtype):
    n, Ks, Xs = 3, [24, 20], [1.0, 1.0]
    p = H().Plan(2, Ks, n, Xs, dtype)
    aq = coefficient(n, Ks, Xs)
    Ms = [n * k - 1 for k in Ks]
    f = np.random.default_rng(5).standard_normal(Ms)
    ref = spla.spsolve(varcoef.assemble(n, Ks, Xs, aq).tocsc(), f.ravel()).reshape(Ms)
    u = torch.zeros(Ms, dtype=torch.float64, device="cuda")
    iters, res = p.pcg(torch.from_numpy(aq).cuda(), torch.from_numpy(f).cuda(), u, tol=1e-12, maxit=200)
    torch.cuda.synchronize()
    print(f"dtype {dtype}: {iters} PCG steps, relative residual {res:.1e}")
    assert res <= 1e-12 and iters <= 40
    assert rel(u.cpu().numpy(), ref) <= 1e-10


def test_pcg_steps_do_not_grow_with_the_mesh():
    """A spectrally equivalent preconditioner: the step count depends on the coefficient's
    range, not on K."""
    n, Xs = 4, [1.0, 1.0]
    steps = []
    for K in (16, 64, 256):
        p = H().Plan(2, [K, K], n, Xs, 0)
        aq = coefficient(n, [K, K], Xs)
        M = n * K - 1
        f = torch.from_numpy(np.random.default_rng(K).standard_normal((M, M))).cuda()
        u = torch.zeros_like(f)
        it, _ = p.pcg(torch.from_numpy(aq).cuda(), f, u, tol=1e-10, maxit=200)
        steps.append(it)
    print("PCG steps for K = 16, 64, 256:", steps)
    assert max(steps) - min(steps) <= 3
