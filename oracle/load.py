"""FEM average f^h of a right-hand side f (Sect. 2 par. 4, "the FEM average of f").

Reading: f^h_p = prod_i (2 / h_i) * integral_Omega f phi_p dx, i.e. the load
vector in the reference-element scaling of Eq. bvp glob 2.  It is computed, as in
the experiments of Sect. 2 par. 5, with the (n+1)-point Gauss-Legendre rule on
every element along every axis.  On element [x_{j-1}, x_j] the map
x = x_{j-1} + (xi + 1) h / 2 makes the factor (2/h) (h/2) = 1, so per axis
f^h = Q F with Q_{p,(j,g)} = w_g e_i(xi_g) summed over the local points i of
element j that are dof p.

Pinned by reproducing Table 1 of the paper (tests/test_oracle_solve.py).
"""
import numpy as np

from .assemble import element_dofs
from .element import lagrange_basis


def _basis_values(n, xi):
    """B[g, i] = e_i(xi_g) from the exact monomial coefficients (Horner, FP64)."""
    E = lagrange_basis(n)
    B = np.zeros((len(xi), n + 1))
    for i, coeffs in enumerate(E):
        c = [float(x) for x in coeffs]
        v = np.zeros_like(xi)
        for a in reversed(c):
            v = v * xi + a
        B[:, i] = v
    return B


def quadrature_1d(n, K, X):
    """(x_q, Q): the K (n+1) quadrature abscissae on [0, X] and the M x K(n+1) matrix Q."""
    xi, w = np.polynomial.legendre.leggauss(n + 1)
    h = X / K
    x = (np.arange(K)[:, None] * h + (xi[None, :] + 1.0) * h / 2.0).reshape(-1)
    B = _basis_values(n, xi)                   # (n+1 gauss, n+1 basis)
    M = n * K - 1
    Q = np.zeros((M, K * (n + 1)))
    dofs = element_dofs(n, K)
    for j in range(K):
        for i in range(n + 1):
            p = dofs[j, i]
            if p >= 0:
                Q[p, j * (n + 1):(j + 1) * (n + 1)] += w * B[:, i]
    return x, Q


def load_vector(f, ns, Ks, Xs):
    """f^h (M_1, ..., M_N) for a vectorised callable f(x_1, ..., x_N)."""
    N = len(Ks)
    quads = [quadrature_1d(n, K, float(X)) for n, K, X in zip(ns, Ks, Xs)]
    grids = np.meshgrid(*[q[0] for q in quads], indexing="ij")
    F = np.asarray(f(*grids), dtype=float)
    for i in range(N):
        F = np.moveaxis(np.tensordot(quads[i][1], F, axes=([1], [i])), 0, i)
    return F


def load_vector_separable(factors, ns, Ks, Xs):
    """f^h for f = sum_m coef_m prod_i g_{m,i}(x_i); factors = [(coef, [g_1, ..., g_N]), ...]."""
    quads = [quadrature_1d(n, K, float(X)) for n, K, X in zip(ns, Ks, Xs)]
    out = None
    for coef, gs in factors:
        term = None
        for (x, Q), g in zip(quads, gs):
            v = Q @ g(x)
            term = v if term is None else np.multiply.outer(term, v)
        term = coef * term
        out = term if out is None else out + term
    return out


def grid_points(n, K, X):
    """Physical coordinates of the dofs of one axis: x_p = (p + 1) h / n."""
    return (np.arange(n * K - 1) + 1.0) * (X / K) / n
