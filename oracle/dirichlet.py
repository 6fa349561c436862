"""Inhomogeneous Dirichlet data u = b on the boundary (test oracle).

The paper covers u|_{dOmega} = b by reducing the problem to Eq. bvp glob 2 with a modified
right-hand side that depends on the boundary data (the remark right after Eq. bvp glob 2).
Written out (the standard lifting): extend the 1D spaces by the two boundary nodes x_0 and
x_K, so that the full 1D matrices A^, C^ of order nK + 1 are assembled from the same local
A, C as Eq. eig_glob but keep the boundary rows and columns; the full N-D operator is
    L^ = sum_i 4 h_i^-2 A^_i (x) prod_{m != i} C^_m + alpha C^_1 (x) ... (x) C^_N.
With v_B the boundary values (on the full grid, zero at interior dofs) the interior
unknowns v satisfy Eq. bvp glob 2 with
    f^h  <-  f^h - (L^ v_B)|_interior.
Reading taken for b^h: v_B holds the values of b at the boundary Lagrange points
(interpolation); any other boundary coefficients (e.g. the L2 projection of b onto the
trace space) go through the same lift unchanged.

Full-grid layout: axis i has nK_i + 1 points, index 0 and nK_i the boundary nodes, index
p + 1 the interior dof p of Eq. eig_glob's layout.

Pins (tests/test_oracle_dirichlet.py): the dense Kronecker brute force on tiny grids; exact
reproduction of a polynomial of degree <= n per variable, boundary data included; and the
convergence of a manufactured solution with nonzero boundary values at Table 1's rates.
"""
import numpy as np

from .element import local_matrices


def full_1d(n, K):
    """FP64 full 1D matrices (A^, C^) of order nK + 1, boundary nodes included."""
    A, C = local_matrices(n)
    Af, Cf = np.array(A, dtype=float), np.array(C, dtype=float)
    P = n * K + 1
    Ah, Ch = np.zeros((P, P)), np.zeros((P, P))
    for j in range(K):
        s = slice(j * n, j * n + n + 1)
        Ah[s, s] += Af
        Ch[s, s] += Cf
    return Ah, Ch


def _mode(T, Mtx, axis):
    """Apply the matrix Mtx along `axis` of T (axis 0 is the right-hand-side index)."""
    return np.moveaxis(np.tensordot(Mtx, T, axes=([1], [axis])), 0, axis)


def boundary_only(vb):
    """vb with its interior entries set to zero (axis 0 indexes right-hand sides)."""
    out = np.array(vb, dtype=float, copy=True)
    inner = (slice(None),) + tuple(slice(1, s - 1) for s in out.shape[1:])
    out[inner] = 0.0
    return out


def lift(vb, ns, Ks, Xs, alpha=0.0):
    """(L^ v_B)|_interior for full-grid boundary data vb of shape (nrhs, nK_1 + 1, ...)."""
    N = len(Ks)
    vB = boundary_only(vb)
    mats = [full_1d(n, K) for n, K in zip(ns, Ks)]
    out = np.zeros_like(vB)
    for i in range(N + (1 if alpha != 0.0 else 0)):
        T = vB
        for m in range(N):
            Ah, Ch = mats[m]
            T = _mode(T, Ah if m == i else Ch, m + 1)
        coef = 4.0 * (Ks[i] / Xs[i]) ** 2 if i < N else alpha
        out += coef * T
    inner = (slice(None),) + tuple(slice(1, s - 1) for s in out.shape[1:])
    return out[inner]


def full_grid(ns, Ks, Xs):
    """Coordinates of the full grid (boundary included), one 1D array per axis."""
    return [np.arange(n * K + 1) * (X / (n * K)) for n, K, X in zip(ns, Ks, Xs)]
