"""High-precision helpers on Python's ``decimal`` module (60 significant digits).

The smallest eigenvalues of the 1D pencil are O((k/K)^2) while the matrix
entries are O(1)-O(n^2), so FP64 loses up to ~8 digits there; the paper computed
its eigenvalues in quadruple precision for the same reason (Sect. 2, par. 5).
These helpers are plain textbook series (Machin's formula for pi, Taylor series
for cos) written for this oracle.
"""
from decimal import Decimal, getcontext, localcontext
from fractions import Fraction

PREC = 60
getcontext().prec = PREC


def D(x):
    """Decimal from int / Fraction / float / Decimal (Fractions are divided at PREC)."""
    if isinstance(x, Decimal):
        return x
    if isinstance(x, Fraction):
        return Decimal(x.numerator) / Decimal(x.denominator)
    if isinstance(x, int):
        return Decimal(x)
    return Decimal(float(x))


def _arctan_inv(m):
    """arctan(1/m) for integer m > 1 by its Taylor series."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        x = Decimal(1) / m
        x2 = x * x
        term, total, k = x, x, 1
        eps = Decimal(10) ** (-(PREC + 8))
        while abs(term) > eps:
            term *= -x2
            total += term / (2 * k + 1)
            k += 1
    return +total


_PI = None


def pi():
    global _PI
    if _PI is None:
        with localcontext() as ctx:
            ctx.prec = PREC + 10
            val = 4 * (4 * _arctan_inv(5) - _arctan_inv(239))
        _PI = +val
    return _PI


def _cos_series(x):
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        x2 = x * x
        term, total, k = Decimal(1), Decimal(1), 0
        eps = Decimal(10) ** (-(PREC + 8))
        while abs(term) > eps:
            term *= -x2 / ((2 * k + 1) * (2 * k + 2))
            total += term
            k += 1
    return +total


def cos_pi_frac(k, K):
    """cos(pi k / K) for integers 0 <= k <= K, to ~PREC digits."""
    if not 0 <= k <= K:
        raise ValueError("need 0 <= k <= K")
    if 2 * k > K:
        return -cos_pi_frac(K - k, K)
    return _cos_series(pi() * k / K)


def sin_pi_frac(k, K):
    """sin(pi k / K) = cos(pi |K - 2k| / (2K)) for integers 0 <= k <= K."""
    if not 0 <= k <= K:
        raise ValueError("need 0 <= k <= K")
    return cos_pi_frac(abs(K - 2 * k), 2 * K)


def sqrt(x):
    return D(x).sqrt()
