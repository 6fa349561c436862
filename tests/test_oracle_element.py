"""Pins of oracle.element (local matrices, Sect. 2 par. 1) -- no GPU."""
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden_path
from oracle import element, spectrum


def _parse_spectra():
    out = {}
    for line in open(golden_path("element_spectra.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, rest = line.split(":")
        vals = []
        for expr in rest.split(";"):
            vals.append(eval(expr.strip().replace("sqrt", "math.sqrt").replace("/", "/"), {"math": math}))
        out[int(n)] = vals
    return out


def test_exact_interior_spectra_match_paper():
    """S~_2..S~_5 printed in Sect. 2 par. 1."""
    for n, vals in _parse_spectra().items():
        lam0, _ = spectrum.element_eigen(n)
        got = [float(x) for x in lam0]
        assert len(got) == len(vals)
        np.testing.assert_allclose(got, sorted(vals), rtol=1e-14, atol=0)


def test_textbook_p1_p2_matrices():
    """Linear and quadratic elements on [-1, 1] (length 2) have the classical matrices."""
    A1, C1 = element.local_matrices(1)
    assert [list(r) for r in A1] == [[Fraction(1, 2), Fraction(-1, 2)], [Fraction(-1, 2), Fraction(1, 2)]]
    assert [list(r) for r in C1] == [[Fraction(2, 3), Fraction(1, 3)], [Fraction(1, 3), Fraction(2, 3)]]
    A2, C2 = element.local_matrices(2)
    assert [list(r) for r in A2] == [[Fraction(x, 6) for x in r] for r in [[7, -8, 1], [-8, 16, -8], [1, -8, 7]]]
    assert [list(r) for r in C2] == [[Fraction(x, 15) for x in r] for r in [[4, 2, -1], [2, 16, 2], [-1, 2, 4]]]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 12])
def test_structure(n):
    A, C = element.local_matrices(n)
    m = n + 1
    for a in range(m):
        assert sum(A[a]) == 0                                 # constants have zero energy
        for b in range(m):
            assert A[a][b] == A[b][a] and C[a][b] == C[b][a]  # symmetric
            assert A[a][b] == A[n - a][n - b]                 # R A R = A (centro-symmetry)
            assert C[a][b] == C[n - a][n - b]
    assert sum(sum(r) for r in C) == 2                        # integral of 1 over [-1, 1]
    assert np.all(np.linalg.eigvalsh(np.array(C, dtype=float)) > 0)


def test_parity_of_element_eigenvectors_alternates():
    """Text after Eq. theta: e^(l) even for odd l, odd for even l, for 2 <= n <= 9."""
    for n in range(2, 10):
        _, E = spectrum.element_eigen(n)
        for l, e in enumerate(E, start=1):
            e = np.array([float(x) for x in e])
            refl = e[::-1]
            if l % 2 == 1:
                np.testing.assert_allclose(refl, e, atol=1e-13)
            else:
                np.testing.assert_allclose(refl, -e, atol=1e-13)
