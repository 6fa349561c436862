"""Algorithm (b) (hofem_solve_banded): transforms along x_2..x_N and banded solves per mode
along x_1 reach the same discrete solution as the oracle's tensor-product solve.  For n >= 2
the banded solve condenses chunks of 32 elements in parallel; K_1 = 65, 100 and 257 give
several chunks and a ragged last one."""
import numpy as np
import pytest

from oracle import solve as osolve

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


CASES = [
    # N, n, K, X, alpha, nrhs
    (2, 1, [16, 8], [1.0, 2.0], 0.0, 2),
    (2, 2, [64, 37], [1.0, 1.0], 0.0, 1),
    (2, 3, [32, 16], [1.5, 0.5], 1.0, 3),
    (2, 4, [8, 128], [1.0, 1.0], -2.0, 1),
    (2, 9, [16, 16], [1.0, 1.0], 0.0, 2),
    (3, 2, [8, 8, 8], [1.0, 1.0, 1.0], 0.0, 2),
    (3, 3, [6, 5, 9], [1.0, 0.6, 2.0], 0.5, 1),
    # several 32-element condensation chunks along x_1, the last one ragged
    (2, 9, [100, 8], [1.0, 1.0], 0.0, 1),
    (2, 2, [257, 3], [1.2, 1.0], 0.3, 2),
    (3, 4, [65, 3, 2], [1.0, 1.0, 0.5], 0.0, 1),
]


@pytest.mark.parametrize("N,n,K,X,alpha,nrhs", CASES)
def test_banded_solve_matches_oracle(N, n, K, X, alpha, nrhs):
    plan = H().Plan(N, K, n, X, H().HOFEM_FP64, alpha)
    Ms = [n * k - 1 for k in K]
    f = np.random.default_rng(N * 100 + n).standard_normal([nrhs] + Ms)
    ref = osolve.solve_tensor(f, [n] * N, K, X, alpha)
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros_like(fd)
    plan.solve_banded(fd, ud, nrhs)
    torch.cuda.synchronize()
    err = float(np.linalg.norm((ud.cpu().numpy() - ref).ravel()) / np.linalg.norm(ref.ravel()))
    print(f"N {N} n {n} K {K}: rel L2 {err:.2e}")
    assert err <= 1e-12


def test_banded_solve_rejects_orders_above_nine():
    plan = H().Plan(2, [2, 4], 16, [1.0, 1.0], H().HOFEM_FP64)
    f = torch.zeros((1, 31, 63), dtype=torch.float64, device="cuda")
    with pytest.raises(H().HofemError):
        plan.solve_banded(f, torch.zeros_like(f), 1)
