"""Spectrum and eigenvectors of the 1D scaled FEM pencil A v = lambda C v (Theorem 1).

Follows Sect. 2 of Zlotnik & Zlotnik in the paper's order and notation:

1. Element eigenpairs {lambda_0^(l), e^(l)} of A~ e = lambda C~ e, scaled so that
   C~ e . e = 1 (Eq. eig_elem, Lemma 1, the scaling sentence after it).
2. For k = 1..K-1 and theta_k = cos(pi k / K), the n roots lambda_k^(l) of the
   theta-equation (Eq. theta), written with the expansion coefficients
   a^(l) = a . e^(l), c^(l) = c . e^(l), acheck^(l), ccheck^(l) (Lemma 2 and the
   text after Eq. theta).  Roots are located from an FP64 estimate of the
   equivalent determinant form det[[g_0 + theta g_n, (g + theta gcheck)^T], [g, G~]] = 0
   and polished by Newton's method on Eq. theta in 60-digit decimal arithmetic.
3. p_k^(l) from Lemma 2 (the second formula, no C~^{-1} term needed in the first).
4. Squared C-norms ||s_k^(l)||^2 = K (b_{kl,0} + b_{kl,n} theta_k) (Theorem 2, part 2)
   and ||s_0^(l)||^2 = K (Theorem 2, part 2, the k = 0 case).
5. Eigenvectors s_0^(l) and s_k^(l) (Theorem 1, parts 2 and 3) in the physical
   layout: dof p = (j-1) n + (i-1) holds element j's local point i (i = n is node j).

Spectral order used everywhere: q = (k-1) n + (l-1) for k = 1..K-1, l = 1..n
(ascending lambda within k), then the k = 0 block q = n (K-1) + (l-1), l = 1..n-1.
Sign convention: s_k^(l) has nodal part +sin(pi k j / K) (Theorem 1 part 3 as
printed); e^(l) has its first component of magnitude >= 1e-3 max|e| positive.

Pins: tests/test_oracle_spectrum.py (exact S~_n, n = 1 closed form, dense
high-precision eigenvectors of the assembled pencil, C-orthogonality, norm
formula vs s^T C s, convergence of 4 h^-2 lambda_k^(1) to (pi k / X)^2).
"""
from decimal import Decimal, localcontext
from functools import lru_cache

import numpy as np
import scipy.linalg as sla

from . import hp
from .element import block_parts, local_matrices

D = hp.D


def _dec_matrix(M):
    return [[D(x) for x in row] for row in M]


def _cholesky(Cm):
    m = len(Cm)
    L = [[Decimal(0)] * m for _ in range(m)]
    for i in range(m):
        for j in range(i + 1):
            s = Cm[i][j] - sum(L[i][k] * L[j][k] for k in range(j))
            if i == j:
                if s <= 0:
                    raise ValueError("mass block not positive definite")
                L[i][i] = s.sqrt()
            else:
                L[i][j] = s / L[j][j]
    return L


def _lower_solve(L, B):
    """Solve L X = B (B: list of columns as lists)."""
    m = len(L)
    out = []
    for b in B:
        x = [Decimal(0)] * m
        for i in range(m):
            x[i] = (b[i] - sum(L[i][k] * x[k] for k in range(i))) / L[i][i]
        out.append(x)
    return out


def _upper_t_solve(L, B):
    """Solve L^T X = B."""
    m = len(L)
    out = []
    for b in B:
        x = [Decimal(0)] * m
        for i in reversed(range(m)):
            x[i] = (b[i] - sum(L[k][i] * x[k] for k in range(i + 1, m))) / L[i][i]
        out.append(x)
    return out


def _jacobi_eig(S):
    """Cyclic Jacobi eigenvalue method for a symmetric Decimal matrix.

    Returns (eigenvalues, eigenvectors as columns) -- textbook two-sided rotations.
    """
    m = len(S)
    a = [row[:] for row in S]
    V = [[Decimal(int(i == j)) for j in range(m)] for i in range(m)]
    tol = Decimal(10) ** (-(hp.PREC - 6))
    for _sweep in range(100):
        off = sum(a[i][j] * a[i][j] for i in range(m) for j in range(m) if i != j)
        scale = sum(a[i][i] * a[i][i] for i in range(m)) + off
        if off <= tol * tol * scale:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                if a[p][q] == 0:
                    continue
                theta = (a[q][q] - a[p][p]) / (2 * a[p][q])
                sign = 1 if theta >= 0 else -1
                t = sign / (abs(theta) + (theta * theta + 1).sqrt())
                c = 1 / (t * t + 1).sqrt()
                s = t * c
                for k in range(m):
                    akp, akq = a[k][p], a[k][q]
                    a[k][p] = c * akp - s * akq
                    a[k][q] = s * akp + c * akq
                for k in range(m):
                    apk, aqk = a[p][k], a[q][k]
                    a[p][k] = c * apk - s * aqk
                    a[q][k] = s * apk + c * aqk
                for k in range(m):
                    vkp, vkq = V[k][p], V[k][q]
                    V[k][p] = c * vkp - s * vkq
                    V[k][q] = s * vkp + c * vkq
    else:
        raise RuntimeError("Jacobi did not converge")
    w = [a[i][i] for i in range(m)]
    return w, [[V[i][j] for i in range(m)] for j in range(m)]


def _fix_sign(v):
    mx = max(abs(x) for x in v)
    for x in v:
        if abs(x) >= mx / 1000:
            return v if x > 0 else [-y for y in v]
    return v


@lru_cache(maxsize=None)
def element_eigen(n):
    """Eigenpairs of A~ e = lambda C~ e (second problem of Eq. eig_elem), C~ e . e = 1.

    Returns (lambda_0 list ascending, e list of (n-1)-vectors), Decimal.  Empty for n = 1.
    """
    if n < 2:
        return (), ()
    A, C = local_matrices(n)
    At = _dec_matrix(block_parts(A)["Mt"])
    Ct = _dec_matrix(block_parts(C)["Mt"])
    with localcontext() as ctx:
        ctx.prec = hp.PREC + 10
        L = _cholesky(Ct)
        m = n - 1
        # B = L^{-1} A~ L^{-T}
        cols_At = [[At[i][j] for i in range(m)] for j in range(m)]
        Y = _lower_solve(L, cols_At)           # columns of L^{-1} A~
        Yt = [[Y[j][i] for j in range(m)] for i in range(m)]  # rows -> columns of (L^{-1} A~)^T
        Z = _lower_solve(L, Yt)                # columns of L^{-1} (L^{-1} A~)^T = B^T = B
        B = [[(Z[j][i] + Z[i][j]) / 2 for j in range(m)] for i in range(m)]
        w, Q = _jacobi_eig(B)
        E = _upper_t_solve(L, Q)
        order = sorted(range(m), key=lambda i: w[i])
        lam0 = tuple(+w[i] for i in order)
        evecs = tuple(tuple(+x for x in _fix_sign(E[i])) for i in order)
    return lam0, evecs


class ElementData:
    """The scalar and vector data of Eq. matrAC / Eq. theta for order n, in Decimal."""

    def __init__(self, n):
        A, C = local_matrices(n)
        pa, pc = block_parts(A), block_parts(C)
        self.n = n
        self.a0, self.an = D(pa["m0"]), D(pa["mn"])
        self.c0, self.cn = D(pc["m0"]), D(pc["mn"])
        self.a = [D(x) for x in pa["m"]]
        self.c = [D(x) for x in pc["m"]]
        self.acheck = [D(x) for x in pa["mcheck"]]
        self.ccheck = [D(x) for x in pc["mcheck"]]
        self.Ct = _dec_matrix(pc["Mt"])
        self.lam0, self.e = element_eigen(n)
        dot = lambda u, v: sum(x * y for x, y in zip(u, v))
        self.al = [dot(self.a, e) for e in self.e]          # a^(l)
        self.cl = [dot(self.c, e) for e in self.e]          # c^(l)
        self.alc = [dot(self.acheck, e) for e in self.e]    # acheck^(l)
        self.clc = [dot(self.ccheck, e) for e in self.e]    # ccheck^(l)
        # FP64 copies for the determinant-form root estimate
        self.Af = np.array([[float(x) for x in r] for r in A])
        self.Cf = np.array([[float(x) for x in r] for r in C])


@lru_cache(maxsize=None)
def element_data(n):
    return ElementData(n)


def theta_function(ed, theta, lam):
    """Left minus right side of Eq. theta, and its derivative in lambda (Decimal)."""
    F = (ed.a0 - lam * ed.c0) + theta * (ed.an - lam * ed.cn)
    dF = -ed.c0 - theta * ed.cn
    for l in range(ed.n - 1):
        al = ed.al[l] - lam * ed.cl[l]
        be = ed.alc[l] - lam * ed.clc[l]
        d = lam - ed.lam0[l]
        num = al * (al + theta * be)
        dnum = -ed.cl[l] * (al + theta * be) + al * (-ed.cl[l] - theta * ed.clc[l])
        F += num / d
        dF += (dnum * d - num) / (d * d)
    return F, dF


def _estimate_roots(ed, theta_f):
    """FP64 generalized eigenvalues of the determinant form of Eq. theta."""
    n = ed.n
    A, C = ed.Af, ed.Cf
    Ap = A[:n, :n].copy()
    Cp = C[:n, :n].copy()
    Ap[0, 0] = A[0, 0] + theta_f * A[0, n]
    Cp[0, 0] = C[0, 0] + theta_f * C[0, n]
    for b in range(1, n):
        Ap[0, b] = A[b, 0] + theta_f * A[b, n]
        Cp[0, b] = C[b, 0] + theta_f * C[b, n]
    w = sla.eigvals(Ap, Cp)
    return np.sort(w.real)


def theta_roots(n, K, k):
    """The n roots lambda_k^(l) (ascending, Decimal) of Eq. theta for theta = cos(pi k/K)."""
    ed = element_data(n)
    theta = hp.cos_pi_frac(k, K)
    guesses = _estimate_roots(ed, float(theta))
    roots = []
    with localcontext() as ctx:
        ctx.prec = hp.PREC + 10
        for g in guesses:
            lam = Decimal(float(g))
            for _ in range(60):
                F, dF = theta_function(ed, theta, lam)
                step = F / dF
                lam -= step
                if abs(step) <= abs(lam) * Decimal(10) ** (-(hp.PREC - 2)):
                    break
            else:
                raise RuntimeError(f"Newton on Eq. theta did not converge (n={n}, K={K}, k={k})")
            if abs(lam - Decimal(float(g))) > abs(lam) * Decimal("1e-4") + Decimal("1e-12"):
                raise RuntimeError("Newton left the neighbourhood of the FP64 root estimate")
            roots.append(+lam)
    roots.sort()
    for i in range(1, len(roots)):
        if roots[i] - roots[i - 1] <= abs(roots[i]) * Decimal("1e-20"):
            raise RuntimeError("theta-equation roots not distinct (Theorem 1 part 1)")
    return theta, roots


def p_vector(ed, lam):
    """p = sum_l (a^(l) - lambda c^(l)) / (lambda - lambda_0^(l)) e^(l) (Lemma 2)."""
    m = ed.n - 1
    p = [Decimal(0)] * m
    for l in range(m):
        coef = (ed.al[l] - lam * ed.cl[l]) / (lam - ed.lam0[l])
        for i in range(m):
            p[i] += coef * ed.e[l][i]
    return p


def norm_sq(ed, K, theta, p):
    """||s_k^(l)||_C^2 = K (b_0 + b_n theta) with b_0, b_n of Theorem 2 part 2."""
    m = ed.n - 1
    Ctp = [sum(ed.Ct[i][j] * p[j] for j in range(m)) for i in range(m)]
    w = [Ctp[i] + 2 * ed.c[i] for i in range(m)]
    b0 = ed.c0 + sum(w[i] * p[i] for i in range(m))
    bn = ed.cn + sum(w[i] * p[m - 1 - i] for i in range(m))
    return K * (b0 + bn * theta)


class Spectrum1D:
    """Eigen-decomposition of one axis: K elements of order n on [0, X].

    Attributes (FP64 numpy unless noted):
      lam   (M,)      true eigenvalues 4 h^-2 lambda in spectral order
      lam_ref (M,)    scaled eigenvalues lambda (independent of h)
      norm  (M,)      squared C-norms ||s_q||^2 in the scaled pencil
      P     (K-1, n, n-1)  p_k^(l) vectors (k = 1..K-1)
      E     (n-1, n-1)     e^(l) vectors (rows)
      dec   dict of the Decimal values (lam_ref, P, norm) for exact-precision pins
    """

    def __init__(self, n, K, X=1.0):
        if K < 2:
            raise ValueError("K >= 2 required")
        self.n, self.K, self.X = n, K, float(X)
        self.M = n * K - 1
        ed = element_data(n)
        m = n - 1
        lam_d, norm_d, P_d = [], [], []
        thetas = []
        for k in range(1, K):
            theta, roots = theta_roots(n, K, k)
            thetas.append(theta)
            for lam in roots:
                p = p_vector(ed, lam) if m > 0 else []
                lam_d.append(lam)
                P_d.append(p)
                norm_d.append(norm_sq(ed, K, theta, p))
        for l in range(m):
            lam_d.append(ed.lam0[l])
            norm_d.append(D(K))
        self.dec = {"lam_ref": lam_d, "norm": norm_d, "P": P_d, "theta": thetas}
        scale = D(4) * D(K) * D(K) / (D(self.X) * D(self.X))
        self.lam_ref = np.array([float(x) for x in lam_d])
        self.lam = np.array([float(x * scale) for x in lam_d])
        self.norm = np.array([float(x) for x in norm_d])
        self.P = np.array([[float(x) for x in p] for p in P_d]).reshape(K - 1, n, m)
        self.E = np.array([[float(x) for x in e] for e in ed.e]).reshape(m, m)

    def dense_S(self):
        """M x M matrix whose column q is s_q (Theorem 1 parts 2-3), physical dof layout."""
        n, K, M = self.n, self.K, self.M
        S = np.zeros((M, M))
        k = np.arange(1, K)
        j = np.arange(0, K + 1)
        # sin(pi k j / K) with exact integer argument reduction
        arg = np.mod(np.outer(j, k), 2 * K)
        sn = np.sin(np.pi * arg / K)                     # (K+1, K-1): row j, col k
        ncols = n * (K - 1)
        # nodal rows p = j n - 1, j = 1..K-1: sin(pi k j / K) for every l
        S[np.arange(1, K) * n - 1, :ncols] = np.repeat(sn[1:K, :], n, axis=1)
        for i in range(1, n):
            rows = np.arange(0, K) * n + i - 1          # element j = 1..K, local i
            pi_ = self.P[:, :, i - 1].reshape(-1)        # (K-1)*n, column order (k, l)
            pni = self.P[:, :, n - i - 1].reshape(-1)
            s_prev = np.repeat(sn[0:K, :], n, axis=1)    # sin(pi k (j-1)/K), j = 1..K
            s_cur = np.repeat(sn[1:K + 1, :], n, axis=1)  # sin(pi k j / K)
            S[rows, :ncols] = s_prev * pi_[None, :] + s_cur * pni[None, :]
            # k = 0 block: (-P)^{j-1} e^(l): (-1)^{j-1} e_{sigma_j(i)}
            jj = np.arange(1, K + 1)
            sgn = np.where(jj % 2 == 1, 1.0, -1.0)
            for l in range(n - 1):
                vals = np.where(jj % 2 == 1, self.E[l, i - 1], self.E[l, n - i - 1])
                S[rows, ncols + l] = sgn * vals
        return S

    def forward(self, y, S=None):
        """Direct F_n-transform of the last axis: w_q = (y, s_q) / ||s_q||^2 (Theorem 2 part 2)."""
        S = self.dense_S() if S is None else S
        return (y @ S) / self.norm

    def inverse(self, w, S=None):
        """Inverse F_n-transform of the last axis: v = sum_q w_q s_q (Eq. decomp)."""
        S = self.dense_S() if S is None else S
        return w @ S.T


@lru_cache(maxsize=8)
def spectrum(n, K, X=1.0):
    return Spectrum1D(n, K, X)
