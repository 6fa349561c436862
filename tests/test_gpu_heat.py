"""Mass operator and implicit heat stepping (hofem_mass, hofem_heat_steps): an eigenmode
of the discrete operator decays by exactly (alpha / (alpha + lambda))^m, and a constant
source drives the steps to the Poisson solution."""
import numpy as np
import pytest

from oracle import assemble, spectrum

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


@pytest.mark.parametrize("ns,Ks,Xs", [([3, 3], [8, 6], [1.0, 1.5]), ([2, 2, 2], [4, 3, 5], [1.0, 0.7, 1.2]),
                                      ([9, 9], [4, 16], [1.0, 1.0])])
def test_mass_operator_matches_the_oracle(ns, Ks, Xs):
    N = len(Ks)
    p = H().Plan(N, Ks, ns[0], Xs, 0)
    Ms = [n * K - 1 for n, K in zip(ns, Ks)]
    v = np.random.default_rng(11).standard_normal([2] + Ms)
    ref = v
    for m, (n, K) in enumerate(zip(ns, Ks)):       # (C_1 x .. x C_N) v by sparse mode products
        ref = assemble._mode_product(ref, assemble.global_1d_sparse(n, K)[1], m + 1)
    out = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
    p.mass(torch.from_numpy(v).cuda(), out, 2)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref) <= 1e-13


@pytest.mark.parametrize("dtype", [0, 4])
def test_eigenmode_decays_exactly(dtype):
    n, K, X, tau, steps = 3, [8, 6], [1.0, 1.5], 1e-3, 5
    specs = [spectrum.spectrum(n, k, x) for k, x in zip(K, X)]
    qa, qb = 5, 11                                   # one mode per axis
    sa, sb = specs[0].dense_S()[:, qa], specs[1].dense_S()[:, qb]
    lam = specs[0].lam[qa] + specs[1].lam[qb]
    u0 = np.outer(sa, sb)[None]
    alpha = 1.0 / tau
    p = H().Plan(2, K, n, X, dtype, alpha=alpha)
    u = torch.from_numpy(u0.copy()).cuda()
    p.heat_steps(u, steps, 1)
    torch.cuda.synchronize()
    expect = (alpha / (alpha + lam)) ** steps * u0
    assert rel(u.cpu().numpy(), expect) <= 1e-12


def test_constant_source_steps_to_the_poisson_solution():
    n, K, X, tau, steps = 2, [16, 12], [1.0, 0.8], 1e-2, 250
    Ms = [n * k - 1 for k in K]
    g = np.random.default_rng(3).standard_normal([1] + Ms)
    gd = torch.from_numpy(g).cuda()
    poisson = torch.zeros_like(gd)
    H().Plan(2, K, n, X, 0).solve(gd, poisson, 1)
    p = H().Plan(2, K, n, X, H().HOFEM_FP32_REFINED, alpha=1.0 / tau)
    u = torch.zeros_like(gd)
    p.heat_steps(u, steps, 1, g=gd)
    torch.cuda.synchronize()
    assert float(torch.linalg.vector_norm(u - poisson) / torch.linalg.vector_norm(poisson)) <= 1e-12
