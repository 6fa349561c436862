"""Pins of oracle.spectrum (Theorem 1, Eq. theta, Lemma 2, Theorem 2 norms) -- no GPU."""
from decimal import Decimal

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble, hp, spectrum


def test_hp_constants():
    assert abs(float(hp.pi()) - np.pi) < 1e-16
    assert str(hp.pi())[:52] == "3.14159265358979323846264338327950288419716939937510"
    for k, K in [(1, 7), (3, 8), (5, 9), (0, 4), (4, 4), (2, 1024)]:
        assert abs(float(hp.cos_pi_frac(k, K)) - np.cos(np.pi * k / K)) < 2e-16
        assert abs(float(hp.sin_pi_frac(k, K)) - np.sin(np.pi * k / K)) < 2e-16
    # exact special values to 55 digits
    assert abs(hp.cos_pi_frac(1, 3) - Decimal("0.5")) < Decimal("1e-55")
    assert abs(hp.cos_pi_frac(1, 4) ** 2 - Decimal("0.5")) < Decimal("1e-55")


@pytest.mark.parametrize("K", [2, 5, 16, 64])
def test_linear_element_closed_form(K):
    """n = 1: lambda_h = 6 h^-2 (1 - cos(pi k/K)) / (2 + cos(pi k/K)) (classical P1 result)."""
    X = 1.7
    s = spectrum.Spectrum1D(1, K, X)
    h = X / K
    k = np.arange(1, K)
    c = np.cos(np.pi * k / K)
    exact = 6.0 / h ** 2 * (1 - c) / (2 + c)
    np.testing.assert_allclose(s.lam, exact, rtol=1e-13)


def _decimal_eigvec(s, q):
    """s_q built in Decimal from the oracle's Decimal data (Theorem 1 parts 2-3)."""
    n, K = s.n, s.K
    M = n * K - 1
    v = [Decimal(0)] * M
    if q < n * (K - 1):
        k = q // n + 1
        p = s.dec["P"][q]
        sn = []
        for j in range(K + 1):
            r = (k * j) % (2 * K)
            sn.append(hp.sin_pi_frac(r, K) if r <= K else -hp.sin_pi_frac(r - K, K))
        for j in range(1, K):
            v[j * n - 1] = sn[j]
        for j in range(1, K + 1):
            for i in range(1, n):
                v[(j - 1) * n + i - 1] = p[i - 1] * sn[j - 1] + p[n - i - 1] * sn[j]
    else:
        l = q - n * (K - 1)
        e = spectrum.element_eigen(n)[1][l]
        for j in range(1, K + 1):
            for i in range(1, n):
                val = e[i - 1] if j % 2 == 1 else e[n - i - 1]
                v[(j - 1) * n + i - 1] = val if j % 2 == 1 else -val
    return v


@pytest.mark.parametrize("n,K", [(2, 3), (3, 4), (4, 3), (5, 2), (9, 3)])
def test_eigenpairs_satisfy_pencil_exactly(n, K):
    """(A - lambda C) s = 0 for every mode, in 60-digit arithmetic with the exact matrices."""
    s = spectrum.Spectrum1D(n, K)
    Ag, Cg = assemble.global_1d_exact(n, K)
    Ad = [[hp.D(x) for x in r] for r in Ag]
    Cd = [[hp.D(x) for x in r] for r in Cg]
    M = n * K - 1
    for q in range(M):
        v = _decimal_eigvec(s, q)
        lam = s.dec["lam_ref"][q]
        res = max(abs(sum((Ad[i][j] - lam * Cd[i][j]) * v[j] for j in range(M))) for i in range(M))
        scale = max(abs(x) for x in v) * (1 + abs(lam)) * max(abs(x) for r in Ad for x in r)
        assert res <= scale * Decimal("1e-45"), (q, res)
        # C-norm formula of Theorem 2 part 2 against s^T C s
        nrm = sum(v[i] * sum(Cd[i][j] * v[j] for j in range(M)) for i in range(M))
        assert abs(nrm - s.dec["norm"][q]) <= abs(nrm) * Decimal("1e-45")


@pytest.mark.parametrize("n,K", [(1, 9), (2, 8), (3, 7), (4, 6), (6, 5), (9, 8), (9, 16)])
def test_dense_S_is_C_orthogonal_basis(n, K):
    s = spectrum.Spectrum1D(n, K)
    S = s.dense_S()
    Ag, Cg = assemble.global_1d_sparse(n, K)
    G = S.T @ (Cg @ S)
    np.testing.assert_allclose(np.diag(G), s.norm, rtol=1e-13)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-13 * np.abs(np.diag(G)).max()
    R = Ag @ S - (Cg @ S) * s.lam_ref[None, :]
    assert np.abs(R).max() <= 1e-12 * max(1.0, s.lam_ref.max())
    # the spectrum is complete: same eigenvalues as a dense generalized eigensolver
    lam_dense = sla.eigh(Ag.toarray(), Cg.toarray(), eigvals_only=True)
    np.testing.assert_allclose(np.sort(s.lam_ref), lam_dense, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("n", [2, 3])
def test_first_eigenvalue_converges_at_rate_h_2n(n):
    """4 h^-2 lambda_1^(1) -> (pi/X)^2 with error O(h^{2n}) (textbook FEM eigenvalue estimate)."""
    X = 1.0
    errs = []
    for K in (4, 8, 16):
        s = spectrum.Spectrum1D(n, K, X)
        errs.append(s.lam[0] - (np.pi / X) ** 2)
    assert all(e > 0 for e in errs)            # Galerkin eigenvalues are upper bounds
    rate = 2 ** (2 * n)
    for a, b in zip(errs, errs[1:]):
        assert 0.7 * rate < a / b < 1.3 * rate


def test_large_k_spectrum_is_accurate_and_ordered():
    s = spectrum.Spectrum1D(9, 1024)
    lam = s.lam.reshape(-1)[: 9 * 1023].reshape(1023, 9)
    assert np.all(np.diff(lam, axis=1) > 0)
    # lowest branch is increasing in k and tends to (pi k)^2 for k << K
    assert np.all(np.diff(lam[:, 0]) > 0)
    k = np.arange(1, 6)
    np.testing.assert_allclose(lam[:5, 0], (np.pi * k) ** 2, rtol=1e-12)
