"""Pins of oracle.varcoef (no GPU): a = 1 reduces it to the constant-coefficient operator
of Eq. bvp glob 2 (alpha = 0, itself pinned to Table 1 and the exact Kronecker solve); it
is linear in a, symmetric and positive definite; for an affine a with different slopes
along the two axes every element matrix equals its exact rational integral; a manufactured
solution with a non-separable a converges at Table 1's rates; and a transposed placement of
a at the Gauss points fails the last two."""
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


def _exact_affine_element(n, Ks, Xs, c, j1, j2):
    """Exact element matrix of -div(a grad) for a = c0 + c1 x + c2 y on element (j1, j2),
    in the scaling of Eq. bvp glob 2, by rational integration of the exact Lagrange
    polynomials (no quadrature): on the element a = al + be xi + ga eta."""
    from fractions import Fraction as F

    from oracle.element import _deriv, _integrate_ref, _polymul, lagrange_basis

    E = [list(e) for e in lagrange_basis(n)]
    dE = [_deriv(e) for e in E]
    h1, h2 = F(Xs[0]) / Ks[0], F(Xs[1]) / Ks[1]
    x0, y0 = j1 * h1, j2 * h2
    al = c[0] + c[1] * (x0 + h1 / 2) + c[2] * (y0 + h2 / 2)
    be, ga = c[1] * h1 / 2, c[2] * h2 / 2
    s1, s2 = 4 / (h1 * h1), 4 / (h2 * h2)

    def I(p, q, first=False):
        pq = _polymul(p, q)
        return _integrate_ref(_polymul([F(0), F(1)], pq) if first else pq)

    G = n + 1
    out = np.zeros((G * G, G * G))
    for a in range(G):
        for b in range(G):
            for cc in range(G):
                for d in range(G):
                    # x-part: a e_a'(xi) e_c'(xi) e_b(eta) e_d(eta); y-part with the roles swapped
                    tx = s1 * (al * I(dE[a], dE[cc]) * I(E[b], E[d]) + be * I(dE[a], dE[cc], True) * I(E[b], E[d])
                               + ga * I(dE[a], dE[cc]) * I(E[b], E[d], True))
                    ty = s2 * (al * I(E[a], E[cc]) * I(dE[b], dE[d]) + be * I(E[a], E[cc], True) * I(dE[b], dE[d])
                               + ga * I(E[a], E[cc]) * I(dE[b], dE[d], True))
                    out[a * G + b, cc * G + d] = float(tx + ty)
    return out


def _affine_case(n):
    from fractions import Fraction as F

    Ks, Xs = [2, 3], [F(3, 2), F(2, 5)]
    c = (F(1), F(7, 10), F(-13, 10))       # slopes differ in size and sign along the two axes
    G = n + 1
    x = [oload.quadrature_1d(n, K, float(X))[0] for K, X in zip(Ks, Xs)]
    X1, X2 = np.meshgrid(*x, indexing="ij")
    aq = float(c[0]) + float(c[1]) * X1 + float(c[2]) * X2
    assert aq.shape == (Ks[0] * G, Ks[1] * G)
    return Ks, Xs, c, aq


@pytest.mark.parametrize("n", [1, 2, 3])
def test_affine_coefficient_matches_exact_integration(n):
    # the (n+1)-point rule integrates a grad e . grad e exactly for affine a (degree <= 2n+1
    # per direction), so every element matrix must equal the rational one
    Ks, Xs, c, aq = _affine_case(n)
    Em = varcoef.element_matrices(n, Ks, [float(X) for X in Xs], aq)
    for j1 in range(Ks[0]):
        for j2 in range(Ks[1]):
            ref = _exact_affine_element(n, Ks, Xs, c, j1, j2)
            np.testing.assert_allclose(Em[j1, j2], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def _manufactured_errors(n, Ks_list):
    """Max dof error of the variable-coefficient FEM solution for u = sin(pi x) sin(pi y),
    a = 1 + x y^2 on the unit square, f = -div(a grad u)."""
    import scipy.sparse.linalg as spla

    def a_fun(x, y):
        return 1.0 + x * y * y

    def f_fun(x, y):
        u = np.sin(np.pi * x) * np.sin(np.pi * y)
        ux = np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
        uy = np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)
        return 2.0 * np.pi ** 2 * a_fun(x, y) * u - y * y * ux - 2.0 * x * y * uy

    errs = []
    for K in Ks_list:
        Ks, Xs = [K, K], [1.0, 1.0]
        x = oload.quadrature_1d(n, K, 1.0)[0]
        X1, X2 = np.meshgrid(x, x, indexing="ij")
        A = varcoef.assemble(n, Ks, Xs, a_fun(X1, X2))
        fh = oload.load_vector(f_fun, [n, n], Ks, Xs)
        v = spla.spsolve(A.tocsc(), fh.ravel()).reshape(fh.shape)
        M = n * K - 1
        g = np.arange(1, M + 1) / (n * K)
        G1, G2 = np.meshgrid(g, g, indexing="ij")
        errs.append(np.abs(v - np.sin(np.pi * G1) * np.sin(np.pi * G2)).max())
    return np.array(errs)


# error ratio per halving of h in the max over all dofs, as Table 1 prints it for the
# constant coefficient: 16 for n = 2 (superconvergent, 1.9e-5 -> 1.2e-6 -> 7.7e-8) and
# 16 = 2^{n+1} for n = 3 (8.6e-6 -> 5.4e-7 -> 3.4e-8)
RATE = {2: 16.0, 3: 16.0}


def _converges(n, errs):
    ratios = errs[:-1] / errs[1:]
    return bool(np.all(ratios > 0.8 * RATE[n]) and np.all(ratios < 1.25 * RATE[n]) and errs[-1] < 1e-5)


@pytest.mark.parametrize("n", [2, 3])
def test_manufactured_solution_converges_at_the_fem_rate(n):
    errs = _manufactured_errors(n, [4, 8, 16])
    assert _converges(n, errs), errs


def test_pins_detect_a_transposed_coefficient(monkeypatch):
    # a plausible slip -- the two axes' Gauss points swapped inside each element -- must
    # fail both pins above
    def swapped(aq, Ks, G):
        return aq.reshape(Ks[0], G, Ks[1], G).transpose(0, 2, 3, 1)

    monkeypatch.setattr(varcoef, "coefficient_at_points", swapped)
    n = 2
    Ks, Xs, c, aq = _affine_case(n)
    Em = varcoef.element_matrices(n, Ks, [float(X) for X in Xs], aq)
    ref = _exact_affine_element(n, Ks, Xs, c, 1, 2)
    assert np.abs(Em[1, 2] - ref).max() > 1e-6 * np.abs(ref).max()
    assert not _converges(n, _manufactured_errors(n, [4, 8, 16]))
