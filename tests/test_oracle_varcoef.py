"""Pins of oracle.varcoef (no GPU): a = 1 reduces it to the constant-coefficient operator
of Eq. bvp glob 2 (alpha = 0, itself pinned to Table 1 and the exact Kronecker solve); it
is linear in a, symmetric and positive definite."""
import numpy as np
import pytest

from oracle import assemble as oasm
from oracle import load as oload
from oracle import varcoef


@pytest.mark.parametrize("n,Ks,Xs", [(1, [5, 4], [1.0, 2.0]), (3, [4, 6], [1.5, 0.5]), (6, [3, 2], [1.0, 1.0])])
def test_unit_coefficient_is_the_constant_operator(n, Ks, Xs):
    G = n + 1
    aq = np.ones((Ks[0] * G, Ks[1] * G))
    Ms = [n * k - 1 for k in Ks]
    u = np.random.default_rng(1).standard_normal(Ms)
    got = varcoef.apply(u, n, Ks, Xs, aq)
    ref = oasm.apply_operator(u[None], [n, n], Ks, Xs, 0.0)[0]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_linear_symmetric_positive_definite():
    n, Ks, Xs = 3, [4, 5], [1.0, 0.8]
    G = n + 1
    x = [oload.quadrature_1d(n, K, X)[0] for K, X in zip(Ks, Xs)]
    X1, X2 = np.meshgrid(*x, indexing="ij")
    a1 = 1.0 + 0.5 * np.sin(np.pi * X1) * np.cos(2 * X2)
    a2 = np.exp(X1 - X2)
    A1, A2 = varcoef.assemble(n, Ks, Xs, a1), varcoef.assemble(n, Ks, Xs, a2)
    A12 = varcoef.assemble(n, Ks, Xs, 2.0 * a1 + 3.0 * a2)
    assert abs(A12 - 2.0 * A1 - 3.0 * A2).max() <= 1e-12 * abs(A12).max()
    assert abs(A1 - A1.T).max() <= 1e-13 * abs(A1).max()
    assert np.linalg.eigvalsh(A1.toarray()).min() > 0
    assert a1.shape == (Ks[0] * G, Ks[1] * G)
