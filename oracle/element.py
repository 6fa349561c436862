"""Exact local matrices of the n-th order equispaced Lagrange element.

Sect. 2, par. 1 (definition of A_kl = int e'_k e'_l and C_kl = int e_k e_l on the
reference element sigma_0 = [-1, 1], Lagrange basis e_l(-1 + 2k/n) = delta_kl) and
Eq. matrAC (3x3 block form).  Arithmetic is exact (``fractions.Fraction``).

Pinned by: exact spectra S~_2..S~_5 printed in Sect. 2 par. 1; textbook P1/P2
element matrices; R A R = A; zero row sums of A; sum of C entries = |sigma_0| = 2.
"""
from fractions import Fraction
from functools import lru_cache


def _polymul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x == 0:
            continue
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _deriv(p):
    return [i * p[i] for i in range(1, len(p))] or [Fraction(0)]


def _integrate_ref(p):
    """Exact integral over [-1, 1] of the polynomial with ascending coefficients p."""
    return sum(c * Fraction(2, i + 1) for i, c in enumerate(p) if i % 2 == 0)


@lru_cache(maxsize=None)
def lagrange_basis(n):
    """Ascending monomial coefficients of e_0..e_n on [-1, 1], nodes -1 + 2k/n."""
    nodes = [Fraction(-1) + Fraction(2 * k, n) for k in range(n + 1)]
    basis = []
    for l in range(n + 1):
        p = [Fraction(1)]
        for m in range(n + 1):
            if m == l:
                continue
            d = nodes[l] - nodes[m]
            p = _polymul(p, [-nodes[m] / d, Fraction(1) / d])
        basis.append(tuple(p))
    return tuple(basis)


@lru_cache(maxsize=None)
def local_matrices(n):
    """Exact (A, C): (n+1)x(n+1) lists of Fractions, A_kl = int e'_k e'_l, C_kl = int e_k e_l."""
    if n < 1:
        raise ValueError("order n must be >= 1")
    E = lagrange_basis(n)
    dE = [_deriv(list(e)) for e in E]
    A = [[_integrate_ref(_polymul(dE[k], dE[l])) for l in range(n + 1)] for k in range(n + 1)]
    C = [[_integrate_ref(_polymul(list(E[k]), list(E[l]))) for l in range(n + 1)] for k in range(n + 1)]
    return tuple(tuple(r) for r in A), tuple(tuple(r) for r in C)


def block_parts(M):
    """Split a centro-symmetric (n+1)x(n+1) matrix into the parts of Eq. matrAC.

    Returns dict with m0 = M[0][0], mn = M[0][n], the interior column
    m = (M[1..n-1][0]), its reflection mcheck = (M[1..n-1][n]) and the interior
    block Mt = M[1..n-1][1..n-1].
    """
    n = len(M) - 1
    return {
        "m0": M[0][0],
        "mn": M[0][n],
        "m": [M[i][0] for i in range(1, n)],
        "mcheck": [M[i][n] for i in range(1, n)],
        "Mt": [[M[i][j] for j in range(1, n)] for i in range(1, n)],
    }
