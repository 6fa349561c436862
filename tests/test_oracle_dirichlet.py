"""Pins of oracle.dirichlet (no GPU): the full 1D matrices against the pinned interior
assembly and their defining sums; the lift against a dense Kronecker brute force; exact
reproduction of a polynomial in the element space with its boundary values; convergence
of a manufactured solution with nonzero boundary values at the rates of Table 1."""
import numpy as np
import pytest

from oracle import assemble as oasm
from oracle import dirichlet as od
from oracle import load as oload
from oracle import solve as osolve


@pytest.mark.parametrize("n,K", [(1, 4), (2, 3), (5, 2)])
def test_full_matrices_extend_the_interior_ones(n, K):
    Ah, Ch = od.full_1d(n, K)
    A, C = oasm.global_1d_sparse(n, K)
    np.testing.assert_allclose(Ah[1:-1, 1:-1], A.toarray(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(Ch[1:-1, 1:-1], C.toarray(), rtol=0, atol=1e-14)
    assert np.abs(Ah.sum(axis=1)).max() < 1e-12          # constants are in the kernel of A^
    assert abs(Ch.sum() - 2.0 * K) < 1e-12                # sum of C^ = K reference lengths of 2


@pytest.mark.parametrize("ns,Ks,Xs,alpha", [([2, 2], [3, 2], [1.0, 1.5], 0.7), ([3, 1], [2, 3], [0.5, 1.0], 0.0),
                                            ([2, 1, 2], [2, 2, 1], [1.0, 2.0, 0.5], 1.3)])
def test_lift_matches_dense_kronecker(ns, Ks, Xs, alpha):
    N = len(Ks)
    rng = np.random.default_rng(3)
    vb = rng.standard_normal([2] + [n * K + 1 for n, K in zip(ns, Ks)])
    mats = [od.full_1d(n, K) for n, K in zip(ns, Ks)]
    L = 0.0
    for i in range(N + 1):
        T = np.ones((1, 1))
        for m in range(N):
            T = np.kron(T, mats[m][0] if m == i else mats[m][1])
        L = L + (4.0 * (Ks[i] / Xs[i]) ** 2 if i < N else alpha) * T
    vB = od.boundary_only(vb).reshape(2, -1)
    full = (vB @ L.T).reshape(vb.shape)
    inner = (slice(None),) + tuple(slice(1, s - 1) for s in vb.shape[1:])
    np.testing.assert_allclose(od.lift(vb, ns, Ks, Xs, alpha), full[inner], rtol=0, atol=1e-12 * np.abs(full).max())


def _solve_with_boundary(u_fun, f_fun, ns, Ks, Xs, alpha):
    """Interior FEM solution for the data (f, b = u on the boundary) and the exact u there."""
    grids = od.full_grid(ns, Ks, Xs)
    G = np.meshgrid(*grids, indexing="ij")
    vb = u_fun(*G)[None]
    fh = oload.load_vector(f_fun, ns, Ks, Xs)[None]
    v = osolve.solve_tensor(fh - od.lift(vb, ns, Ks, Xs, alpha), ns, Ks, Xs, alpha)
    inner = (slice(None),) + tuple(slice(1, s - 1) for s in vb.shape[1:])
    return v, vb[inner]


@pytest.mark.parametrize("N,alpha", [(2, 0.0), (2, 1.5), (3, 0.4)])
def test_polynomial_in_the_space_is_reproduced_exactly(N, alpha):
    # u has degree <= 2 per variable, so for n = 2 it lies in the element space and the
    # Galerkin solution with its boundary values is u itself (the (n+1)-point rule
    # integrates f phi exactly: degree 4 per variable)
    if N == 2:
        u = lambda x, y: 1.0 + 2.0 * x - y + x * y + x * x - 0.5 * y * y
        f = lambda x, y: -(2.0 - 1.0) + alpha * u(x, y)
        Ks, Xs = [3, 4], [1.0, 1.7]
    else:
        u = lambda x, y, z: 0.5 + x * y * z + x * x - z
        f = lambda x, y, z: -2.0 + alpha * u(x, y, z)
        Ks, Xs = [2, 3, 2], [1.0, 0.8, 1.2]
    v, ue = _solve_with_boundary(u, f, [2] * N, Ks, Xs, alpha)
    assert np.abs(v - ue).max() < 1e-12 * max(1.0, np.abs(ue).max())
    # without the lift the same data give a different (homogeneous-boundary) solution
    fh = oload.load_vector(f, [2] * N, Ks, Xs)[None]
    assert np.abs(osolve.solve_tensor(fh, [2] * N, Ks, Xs, alpha) - ue).max() > 1e-3


# error ratio per halving of h, max over all dofs, as Table 1 prints it: 16 for n = 2
# (superconvergent) and for n = 3
RATE = {2: 16.0, 3: 16.0}


@pytest.mark.parametrize("n", [2, 3])
def test_manufactured_boundary_data_converge_at_table1_rates(n):
    alpha = 1.0
    u = lambda x, y: np.sin(0.5 * np.pi * x + 0.3) * np.exp(y)
    f = lambda x, y: (0.25 * np.pi ** 2 - 1.0 + alpha) * u(x, y)
    errs = []
    for K in (4, 8, 16):
        v, ue = _solve_with_boundary(u, f, [n, n], [K, K], [1.0, 1.0], alpha)
        errs.append(np.abs(v - ue).max())
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 0.8 * RATE[n]) and np.all(ratios < 1.25 * RATE[n]), (errs, ratios)
