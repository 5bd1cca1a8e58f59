"""Classical side of Shor's algorithm (Sec. 5.4) and the closed-form
x-register distribution after SHORBOX + quantum Fourier transform.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import math
from fractions import Fraction

import numpy as np


def order(y, G):
    """Multiplicative order r of y mod G: the period of f(x) = y^x mod G."""
    if math.gcd(y, G) != 1:
        raise ValueError("y and G are not coprime")
    r, f = 1, y % G
    while f != 1:
        f = (f * y) % G
        r += 1
    return r


def qubit_budget(G):
    """F = ceil(log2 G) qubits for f(x); X = ceil(log2 G^2) for the x-register,
    so that G^2 <= 2^X < 2 G^2 (Sec. 5.4)."""
    F = (G - 1).bit_length()
    X = (G * G - 1).bit_length()
    return X, F


def factors_from_period(y, r, G):
    """Sec. 5.4: for even r with y^{r/2} != -1 mod G, gcd(y^{r/2} +- 1, G)."""
    if r % 2:
        return None
    h = pow(y, r // 2, G)
    if h == G - 1:
        return None
    p, q = math.gcd(h - 1, G), math.gcd(h + 1, G)
    if p in (1, G) or q in (1, G):
        return None
    return tuple(sorted((p, q)))


def period_from_sample(k, X, G):
    """Continued-fraction expansion of k / 2^X; the smallest denominator
    s < G of a convergent with |k/2^X - j/s| <= 1/2^{X+1} (textbook step
    following the measurement in Shor's algorithm)."""
    if k == 0:
        return None
    fr = Fraction(k, 1 << X).limit_denominator(G - 1)
    return fr.denominator


def closed_form_distribution(X, r):
    """P(k), k = 0..2^X-1, of the x-register after SHORBOX (Appendix A) and a
    quantum Fourier transform of the x-register, for a period r:

        P(k) = 2^{-2X} sum_{x0=0}^{r-1} | sum_{m: x0 + m r < 2^X} e^{2 pi i k (x0 + m r)/2^X} |^2,

    because the f-register value y^{x0} is shared exactly by x = x0 + m r.
    The inner sums are evaluated with an FFT (library primitive).  |.|^2 does
    not depend on the sign of the exponent, so the same distribution holds for
    the inverse transform.
    """
    M = 1 << X
    P = np.zeros(M)
    for x0 in range(r):
        ind = np.zeros(M)
        ind[x0::r] = 1.0
        F = np.fft.fft(ind)
        P += F.real ** 2 + F.imag ** 2
    return P / float(M) ** 2


def qz_from_distribution(P, X):
    """<Qz(n)> = probability that bit n of k is 1, for n = 0..X-1."""
    k = np.arange(P.size)
    return np.array([P[((k >> n) & 1) == 1].sum() for n in range(X)])
