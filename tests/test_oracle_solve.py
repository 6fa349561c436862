"""Pins of oracle.solve / oracle.load / oracle.assemble -- no GPU."""
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden_path
from oracle import assemble, load, solve

PI = np.pi


def _table1():
    rows = {}
    for line in open(golden_path("table1_errors.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            parts = line.split()
            rows[int(parts[0])] = [float(x) for x in parts[1:]]
    return rows


def _f_table1(x, y):
    sx, sy, cx, cy = np.sin(PI * x), np.sin(PI * y), np.cos(PI * x), np.cos(PI * y)
    return (2 * PI ** 2 + 1) * sx * sy * (x + y - 1) - 2 * PI * (cx * sy + sx * cy)


def _u_table1(x, y):
    return np.sin(PI * x) * np.sin(PI * y) * (x + y - 1)


def _table1_error(n, K):
    fh = load.load_vector(_f_table1, [n, n], [K, K], [1.0, 1.0])
    v = solve.solve_tensor(fh[None], [n, n], [K, K], [1.0, 1.0], alpha=1.0)[0]
    x = load.grid_points(n, K, 1.0)
    X, Y = np.meshgrid(x, x, indexing="ij")
    return np.abs(v - _u_table1(X, Y)).max()


@pytest.mark.parametrize("n,kappa", [(1, 3), (2, 3), (3, 3), (4, 3), (5, 3), (6, 3), (1, 4), (2, 4),
                                     (3, 4), (4, 4), (5, 4), (2, 5), (3, 5), (4, 5), (1, 6), (2, 6)])
def test_table1_reproduced(n, kappa):
    """Uniform-norm errors of Table 1 above the round-off floor, to the 2 printed digits."""
    printed = _table1()[kappa][n - 1]
    err = _table1_error(n, 2 ** kappa)
    unit = 10.0 ** np.floor(np.log10(printed))      # printed = d.d x unit
    assert abs(err - printed) <= 0.06 * unit        # within 0.6 of the last printed digit


@pytest.mark.slow
@pytest.mark.parametrize("n,kappa", [(2, 9), (2, 10), (3, 9)])
def test_table1_reproduced_large_k(n, kappa):
    """K = 512, 1024 entries near the round-off floor (pins the oracle's accuracy to ~1e-14)."""
    printed = _table1()[kappa][n - 1]
    err = _table1_error(n, 2 ** kappa)
    assert abs(err - printed) <= 0.1 * printed


def test_table1_convergence_rate_n2():
    """n = 2 column of Table 1 drops ~16x per halving of h."""
    e = [_table1_error(2, K) for K in (8, 16, 32)]
    assert 12 < e[0] / e[1] < 20 and 12 < e[1] / e[2] < 20


@pytest.mark.parametrize("ns,Ks,Xs,alpha", [
    ([2, 2], [3, 3], [1, 1], 0),
    ([3, 3], [2, 3], [Fraction(3, 2), 1], 0),
    ([1, 1], [4, 5], [1, 2], 3),
    ([2, 2, 2], [2, 2, 2], [1, 1, 1], 0),
    ([4, 4], [2, 2], [1, Fraction(1, 2)], Fraction(-1, 2)),
])
def test_tensor_solve_matches_exact_kronecker_solve(ns, Ks, Xs, alpha):
    """Algorithm (a) (dense mode products) vs Gaussian elimination on the exact operator."""
    assert all(n == ns[0] for n in ns)  # oracle.solve_tensor supports per-axis n; kept equal here
    rng = np.random.default_rng(7)
    Ms = [n * K - 1 for n, K in zip(ns, Ks)]
    f = rng.integers(-5, 6, size=Ms)
    exact = np.array([float(x) for x in solve.solve_exact(f, ns, Ks, Xs, alpha)]).reshape(Ms)
    got = solve.solve_tensor(f[None].astype(float), ns, Ks, [float(x) for x in Xs], float(alpha))[0]
    np.testing.assert_allclose(got, exact, rtol=1e-11, atol=1e-12 * np.abs(exact).max())


def test_apply_matches_dense_operator_and_inverts_solve():
    ns, Ks, Xs, alpha = [3, 3], [3, 4], [1.0, 2.0], 0.5
    Ms = [n * K - 1 for n, K in zip(ns, Ks)]
    rng = np.random.default_rng(3)
    v = rng.standard_normal([2] + Ms)
    r = assemble.apply_operator(v, ns, Ks, Xs, alpha)
    Aop = np.array(assemble.operator_exact(ns, Ks, [Fraction(x) for x in Xs], Fraction(alpha)), dtype=float)
    for b in range(2):
        np.testing.assert_allclose(r[b].reshape(-1), Aop @ v[b].reshape(-1), rtol=1e-12, atol=1e-10)
    u = solve.solve_tensor(r, ns, Ks, Xs, alpha)
    np.testing.assert_allclose(u, v, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("n,K", [(1, 4), (2, 5), (5, 3), (9, 2)])
def test_load_vector_of_polynomials_is_exact(n, K):
    """(n+1)-point Gauss is exact for f phi of degree <= 2n+1: f = 1 gives the C row sums."""
    X = 1.3
    x, Q = load.quadrature_1d(n, K, X)
    one = Q @ np.ones_like(x)
    Ag, Cg = assemble.global_1d_sparse(n, K)
    # row sums of the assembled mass including the Dirichlet columns = (2/h) int phi_p
    Cfull = np.zeros(n * K - 1)
    from oracle.element import local_matrices
    _, C = local_matrices(n)
    dofs = assemble.element_dofs(n, K)
    rs = [float(sum(r)) for r in C]
    for j in range(K):
        for i in range(n + 1):
            if dofs[j, i] >= 0:
                Cfull[dofs[j, i]] += rs[i]
    np.testing.assert_allclose(one, Cfull, rtol=1e-13, atol=1e-14)
    # a separable load equals the outer product of 1D loads
    g = lambda t: t ** 2 + 1
    f2 = load.load_vector(lambda a, b: g(a) * np.cos(b), [n, n], [K, K], [X, X])
    sep = load.load_vector_separable([(1.0, [g, np.cos])], [n, n], [K, K], [X, X])
    np.testing.assert_allclose(f2, sep, rtol=1e-13, atol=1e-15)
