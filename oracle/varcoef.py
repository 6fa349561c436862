"""Variable-coefficient operator -div(a grad u) on the 2D tensor-product mesh (test oracle).

The paper names the method's use as a preconditioner for general second-order elliptic
equations (Sect. 1).  The operator it would precondition is written here from its
definition, in the scaling of Eq. bvp glob 2: on element (j1, j2), with the reference map
x_i = x_{i, j_i - 1} + (xi_i + 1) h_i / 2,

    (2/h_1)(2/h_2) int a grad phi_p . grad phi_q dx
      = int_{[-1,1]^2} a (4 h_1^-2 d_xi1 phi_p d_xi1 phi_q + 4 h_2^-2 d_xi2 phi_p d_xi2 phi_q) dxi,

evaluated with the (n+1)-point Gauss-Legendre rule per direction (the load vector's rule,
Sect. 2 par. 5), a given by its values at those points.  For a = 1 it is the operator of
Eq. bvp glob 2 with alpha = 0.  Pins (tests/test_oracle_varcoef.py): that a = 1
reduction; entrywise agreement with the exact rational integration of an affine a (which
the rule integrates exactly) on a non-square grid of elements; and the O(h^{n+1}) dof
convergence of a manufactured solution with a non-separable a.  Plain numpy:
element loops vectorised with einsum, scatter-add through the element dof map.
"""
import numpy as np
import scipy.sparse as sps

from .assemble import element_dofs
from .element import lagrange_basis


def _basis_and_derivative(n, xi):
    """B[g, a] = e_a(xi_g), D[g, a] = e_a'(xi_g) from the exact monomial coefficients."""
    E = lagrange_basis(n)
    B = np.zeros((len(xi), n + 1))
    D = np.zeros((len(xi), n + 1))
    for a, coeffs in enumerate(E):
        c = [float(x) for x in coeffs]
        dc = [k * c[k] for k in range(1, len(c))]
        v = np.zeros_like(xi)
        for t in reversed(c):
            v = v * xi + t
        dv = np.zeros_like(xi)
        for t in reversed(dc):
            dv = dv * xi + t
        B[:, a] = v
        D[:, a] = dv
    return B, D


def coefficient_at_points(aq, Ks, G):
    """a[j1, j2, g, h]: the value of a at Gauss point g (axis 1) and h (axis 2) of element
    (j1, j2), from aq whose row index is the axis-1 point (j1 G + g) and whose column index
    is the axis-2 point (j2 G + h).  Pinned by the exact integration of an affine a with
    different slopes along the two axes (tests/test_oracle_varcoef.py)."""
    return aq.reshape(Ks[0], G, Ks[1], G).transpose(0, 2, 1, 3)


def element_matrices(n, Ks, Xs, aq):
    """(K1, K2, (n+1)^2, (n+1)^2) element matrices; aq: (K1 (n+1), K2 (n+1)) values of a.

    Local index p = a (n+1) + b: basis e_a along axis 1 times e_b along axis 2."""
    xi, w = np.polynomial.legendre.leggauss(n + 1)
    B, D = _basis_and_derivative(n, xi)
    G = n + 1
    s1, s2 = 4.0 * (Ks[0] / Xs[0]) ** 2, 4.0 * (Ks[1] / Xs[1]) ** 2
    a = coefficient_at_points(aq, Ks, G) * np.outer(w, w)[None, None]
    # gradients of the basis at the quadrature points, per reference direction
    Gx = np.einsum("ga,hb->ghab", D, B).reshape(G, G, G * G)
    Gy = np.einsum("ga,hb->ghab", B, D).reshape(G, G, G * G)
    Ex = np.einsum("ijgh,ghp,ghq->ijpq", a, Gx, Gx)
    Ey = np.einsum("ijgh,ghp,ghq->ijpq", a, Gy, Gy)
    return s1 * Ex + s2 * Ey


def assemble(n, Ks, Xs, aq):
    """Sparse (M1 M2) x (M1 M2) matrix of the operator (Dirichlet dofs removed)."""
    Em = element_matrices(n, Ks, Xs, aq)
    d1, d2 = element_dofs(n, Ks[0]), element_dofs(n, Ks[1])
    M2 = n * Ks[1] - 1
    rows, cols, vals = [], [], []
    for j1 in range(Ks[0]):
        for j2 in range(Ks[1]):
            g = (d1[j1][:, None] * M2 + d2[j2][None, :]).ravel()
            ok = ((d1[j1][:, None] >= 0) & (d2[j2][None, :] >= 0)).ravel()
            idx = np.nonzero(ok)[0]
            rr, cc = np.meshgrid(idx, idx, indexing="ij")
            rows.append(g[rr].ravel())
            cols.append(g[cc].ravel())
            vals.append(Em[j1, j2][rr, cc].ravel())
    M = (n * Ks[0] - 1) * M2
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(M, M))


def apply(u, n, Ks, Xs, aq):
    """r = A_a u for u of shape (M1, M2)."""
    A = assemble(n, Ks, Xs, aq)
    return (A @ u.ravel()).reshape(u.shape)
