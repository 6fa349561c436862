"""The discrete Dirichlet problem (Eq. bvp glob 2) solved two plain ways.

* ``solve_tensor``: algorithm (a) of Sect. 2 par. 4 written as dense mode
  products (Eq. decomp phi 2 / Eq. decomp v 2).  The C-solve of step (1) and the
  y = C phi of the direct transform cancel (Theorem 2 part 2 uses y = C w, and
  C phi = f^h), so the coefficients of phi are (f^h, s_q) / ||s_q||^2 along every
  axis; they are divided by sum_i 4 h_i^-2 lambda_i + alpha and synthesised with
  the eigenvectors.  Eigen-data from ``spectrum`` (60-digit, rounded to FP64);
  the mode products are FP64 matrix products.
* ``solve_exact``: Gaussian elimination on the exact Kronecker operator in
  rational arithmetic, for tiny grids (brute force, the plain definition).

Pins: tests/test_oracle_solve.py (exact solve agreement, Table 1 of the paper).
"""
from fractions import Fraction

import numpy as np

from .assemble import operator_exact
from .spectrum import spectrum


def _mode(T, Mat, axis):
    T = np.moveaxis(T, axis, -1)
    out = T @ Mat
    return np.moveaxis(out, -1, axis)


def solve_tensor(f, ns, Ks, Xs, alpha=0.0, specs=None):
    """v with (sum 4 h_i^-2 A_i (x) C.. + alpha C..) v = f, f shaped (nrhs, M_1, .., M_N)."""
    f = np.asarray(f, dtype=float)
    N = len(Ks)
    if specs is None:
        specs = [spectrum(n, K, float(X)) for n, K, X in zip(ns, Ks, Xs)]
    Ss = [s.dense_S() for s in specs]
    w = f
    for i in range(N):                      # direct F_n along every axis
        w = _mode(w, Ss[i], i + 1) / specs[i].norm.reshape([-1] + [1] * (N - 1 - i))
    denom = np.full([s.M for s in specs], float(alpha))
    for i in range(N):
        shape = [1] * N
        shape[i] = specs[i].M
        denom = denom + specs[i].lam.reshape(shape)
    w = w / denom[None]
    for i in range(N):                      # inverse F_n along every axis
        w = _mode(w, Ss[i].T, i + 1)
    return w


def solve_exact(f, ns, Ks, Xs, alpha=0):
    """Exact rational solve on the dense Kronecker operator; f: (M_1..M_N) Fractions/ints/floats."""
    Aop = operator_exact(ns, Ks, [Fraction(x) for x in Xs], Fraction(alpha))
    b = [Fraction(x) for x in np.asarray(f, dtype=object).reshape(-1)]
    m = len(b)
    a = [row[:] + [b[i]] for i, row in enumerate(Aop)]
    for c in range(m):
        piv = next(r for r in range(c, m) if a[r][c] != 0)
        a[c], a[piv] = a[piv], a[c]
        inv = 1 / a[c][c]
        for r in range(c + 1, m):
            if a[r][c] != 0:
                fac = a[r][c] * inv
                a[r] = [x - fac * y for x, y in zip(a[r], a[c])]
    x = [Fraction(0)] * m
    for r in reversed(range(m)):
        x[r] = (a[r][m] - sum(a[r][k] * x[k] for k in range(r + 1, m))) / a[r][r]
    return x
