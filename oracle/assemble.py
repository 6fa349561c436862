"""Global 1D matrices and the N-D operator, dense or sparse (Eq. eig_glob, Eq. bvp glob 2).

The global scaled stiffness/mass operators act in S_K^(n) (Sect. 2 par. 1): they
are assembled from the local A, C over the K elements with the Dirichlet node
values v_0 = v_K = 0 removed.  Dof p = (j-1) n + (i-1) holds element j's local
point i, so element j's local index i maps to p = (j-1) n - 1 + i.

The N-D operator (Eq. bvp glob 2) is
    sum_i 4 h_i^-2 A_i (x) prod_{m != i} C_m  +  alpha C_1 (x) ... (x) C_N,
with axis 1 outermost (C-order arrays of shape (M_1, ..., M_N)).

Pins: tests/test_oracle_solve.py (brute-force exact solves, apply vs dense Kronecker).
"""
from fractions import Fraction

import numpy as np
import scipy.sparse as sps

from .element import local_matrices


def element_dofs(n, K):
    """(K, n+1) array: global dof of local point i in element j (-1 for a Dirichlet node)."""
    M = n * K - 1
    idx = np.arange(K)[:, None] * n - 1 + np.arange(n + 1)[None, :]
    idx[(idx < 0) | (idx >= M)] = -1
    return idx


def global_1d_exact(n, K):
    """Exact global (A, C) as lists of Fractions (M x M), for tiny K."""
    A, C = local_matrices(n)
    M = n * K - 1
    Ag = [[Fraction(0)] * M for _ in range(M)]
    Cg = [[Fraction(0)] * M for _ in range(M)]
    dofs = element_dofs(n, K)
    for j in range(K):
        for a in range(n + 1):
            pa = dofs[j, a]
            if pa < 0:
                continue
            for b in range(n + 1):
                pb = dofs[j, b]
                if pb < 0:
                    continue
                Ag[pa][pb] += A[a][b]
                Cg[pa][pb] += C[a][b]
    return Ag, Cg


def global_1d_sparse(n, K):
    """FP64 global (A, C) as scipy CSR matrices."""
    A, C = local_matrices(n)
    Af = np.array(A, dtype=float)
    Cf = np.array(C, dtype=float)
    M = n * K - 1
    dofs = element_dofs(n, K)
    rows, cols, va, vc = [], [], [], []
    for a in range(n + 1):
        for b in range(n + 1):
            pa, pb = dofs[:, a], dofs[:, b]
            ok = (pa >= 0) & (pb >= 0)
            rows.append(pa[ok])
            cols.append(pb[ok])
            va.append(np.full(ok.sum(), Af[a, b]))
            vc.append(np.full(ok.sum(), Cf[a, b]))
    r, c = np.concatenate(rows), np.concatenate(cols)
    Ag = sps.csr_matrix((np.concatenate(va), (r, c)), shape=(M, M))
    Cg = sps.csr_matrix((np.concatenate(vc), (r, c)), shape=(M, M))
    return Ag, Cg


def _mode_product(T, Mat, axis):
    """T x_axis Mat: contract Mat (dense or sparse, M x M) with T along 'axis' (T's axis 0 = rhs)."""
    T = np.moveaxis(T, axis, -1)
    shp = T.shape
    flat = T.reshape(-1, shp[-1])
    out = (Mat @ flat.T).T if sps.issparse(Mat) else flat @ Mat.T
    return np.moveaxis(np.asarray(out).reshape(shp), -1, axis)


def apply_operator(v, ns, Ks, Xs, alpha=0.0):
    """r = (sum_i 4 h_i^-2 A_i (x) C_others + alpha (x) C) v  (Eq. bvp glob 2), FP64.

    v: array (nrhs, M_1, ..., M_N).  Plain sparse mode products, no fusion.
    """
    N = len(Ks)
    mats = [global_1d_sparse(n, K) for n, K in zip(ns, Ks)]
    r = np.zeros_like(v, dtype=float)
    for i in range(N + 1):
        t = np.array(v, dtype=float)
        for m in range(N):
            A, C = mats[m]
            t = _mode_product(t, A if m == i else C, m + 1)
        if i < N:
            s = 4.0 * (Ks[i] / Xs[i]) ** 2
            r += s * t
        elif alpha != 0.0:
            r += alpha * t
    return r


def operator_exact(ns, Ks, Xs, alpha=0):
    """Exact dense N-D operator (Fractions) for tiny grids: Kronecker products of the 1D matrices."""
    N = len(Ks)
    mats = [global_1d_exact(n, K) for n, K in zip(ns, Ks)]

    def kron(P, Q):
        return [[P[i][j] * Q[k][l] for j in range(len(P)) for l in range(len(Q))]
                for i in range(len(P)) for k in range(len(Q))]

    total = None
    for i in range(N + 1):
        term = None
        for m in range(N):
            A, C = mats[m]
            F = A if m == i else C
            term = F if term is None else kron(term, F)
        if i < N:
            s = 4 * (Fraction(Ks[i]) / Fraction(Xs[i])) ** 2
        else:
            s = Fraction(alpha)
        if s == 0:
            continue
        term = [[s * x for x in row] for row in term]
        total = term if total is None else [[x + y for x, y in zip(r1, r2)] for r1, r2 in zip(total, term)]
    return total
