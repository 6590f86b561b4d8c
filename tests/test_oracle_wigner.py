"""Pins of the oracle's Wigner-d / spin-weighted harmonics against mathematics the paper fixes.

Everything here is independent of the oracle's own recurrence: Wigner's explicit finite sum
evaluated in 40-digit arithmetic, textbook closed forms, the appendix's symmetry relations and
Fourier identity, and exact quadrature orthonormality.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle as O


def wigner_explicit(j, m1, m2, beta):
    """Wigner's explicit sum for d^j_{m1,m2}(beta), 40 digits."""
    mp.mp.dps = 40
    b = mp.mpf(beta)
    tot = mp.mpf(0)
    for k in range(0, 2 * j + 1):
        a1, a2, a3 = j + m2 - k, j - k - m1, k - m2 + m1
        if min(a1, a2, a3) < 0:
            continue
        num = mp.sqrt(mp.factorial(j + m2) * mp.factorial(j - m2) * mp.factorial(j + m1) * mp.factorial(j - m1))
        den = mp.factorial(a1) * mp.factorial(k) * mp.factorial(a2) * mp.factorial(a3)
        tot += (-1) ** (k - m2 + m1) * num / den * mp.cos(b / 2) ** (2 * j - 2 * k + m2 - m1) * mp.sin(b / 2) ** (2 * k - m2 + m1)
    return float(tot)


@pytest.mark.parametrize("beta", [0.0, 0.31, 1.7, 2.95, math.pi, 4.1, -0.6])
def test_wigner_d_matches_explicit_sum(beta):
    worst = 0.0
    for j in range(0, 9):
        for m in range(-j, j + 1):
            for s in range(0, j + 1):
                for mp_ in (-s, s):
                    o = O.wigner_d(j, m, mp_, beta)[j]
                    worst = max(worst, abs(o - wigner_explicit(j, m, mp_, beta)))
    assert worst < 5e-15


def test_wigner_column_all_l():
    """Every l of a column, not only the top one, against the explicit sum."""
    for (m, mp_, beta) in [(3, -2, 0.8), (0, 0, 2.2), (1, 2, 0.05), (5, 5, 1.3)]:
        col = O.wigner_d(12, m, mp_, beta)
        for l in range(0, 13):
            ref = wigner_explicit(l, m, mp_, beta) if l >= max(abs(m), abs(mp_)) else 0.0
            assert abs(col[l] - ref) < 5e-15


def test_wigner_large_l_underflow_and_unitarity():
    """Scaled arithmetic: at l = 3000 near the pole the column still satisfies
    sum_m |d^l_{m,m'}|^2 = 1 (unitarity of the rotation matrix)."""
    l = 3000
    for beta in (0.02, 0.7):
        for mp_ in (0, -2):
            tot = sum(O.wigner_d(l, m, mp_, beta)[l] ** 2 for m in range(-l, l + 1))
            assert abs(tot - 1.0) < 1e-11


def test_closed_form_harmonics():
    """Closed forms of eq. Ylm with the standard d convention (Condon-Shortley at s = 0)."""
    th, ph = 0.73, 1.21
    e = lambda m: complex(math.cos(m * ph), math.sin(m * ph))
    cases = [
        (0, 0, 0, 1 / math.sqrt(4 * math.pi)),
        (0, 1, 0, math.sqrt(3 / (4 * math.pi)) * math.cos(th)),
        (0, 1, 1, -math.sqrt(3 / (8 * math.pi)) * math.sin(th) * e(1)),
        (0, 2, 1, -math.sqrt(15 / (8 * math.pi)) * math.sin(th) * math.cos(th) * e(1)),
        (0, 2, 2, 0.25 * math.sqrt(15 / (2 * math.pi)) * math.sin(th) ** 2 * e(2)),
        (2, 2, 0, math.sqrt(15 / (32 * math.pi)) * math.sin(th) ** 2),
        (2, 2, 2, 0.5 * math.sqrt(5 / math.pi) * math.sin(th / 2) ** 4 * e(2)),
        (2, 2, -2, 0.5 * math.sqrt(5 / math.pi) * math.cos(th / 2) ** 4 * e(-2)),
    ]
    for s, l, m, ref in cases:
        assert abs(O.sYlm(s, l, m, th, ph) - ref) < 1e-15


def test_pole_crossing_rule():
    """sY_lm(pi + beta, phi) = (-1)^s sY_lm(pi - beta, phi + pi)  (Sec. I.A eq. sht; appendix)."""
    for s in (0, 1, 2, 3):
        for l in range(s, 7):
            for m in range(-l, l + 1):
                for beta, ph in ((0.3, 0.2), (1.1, 4.0)):
                    lhs = O.sYlm(s, l, m, math.pi + beta, ph)
                    rhs = (-1) ** s * O.sYlm(s, l, m, math.pi - beta, ph + math.pi)
                    assert abs(lhs - rhs) < 1e-14


def test_spin_conjugation():
    """sY*_lm = (-1)^(s+m) _{-s}Y_{l,-m}, which the adjoint's projection relies on."""
    for s in (0, 1, 2):
        for l in range(s, 6):
            for m in range(-l, l + 1):
                th, ph = 1.3, 0.4
                lhs = np.conj(O.sYlm(s, l, m, th, ph))
                rhs = (-1) ** (s + m) * O.sYlm(-s, l, -m, th, ph)
                assert abs(lhs - rhs) < 1e-14


@pytest.mark.parametrize("l,s,sp,th", [(3, 0, 0, 0.7), (4, 2, -2, 1.1), (5, 1, 2, 2.0), (6, 2, 0, 0.4), (4, -1, 3, 2.7)])
def test_d_fourier_identity(l, s, sp, th):
    """d^l_{ss'}(theta) = sum_m i^s d^l_{ms}(pi/2) e^{-i m theta} d^l_{ms'}(pi/2) (-i)^{s'} (appendix)."""
    rhs = sum((1j) ** s * O.wigner_d(l, m, s, math.pi / 2)[l] * np.exp(-1j * m * th)
              * O.wigner_d(l, m, sp, math.pi / 2)[l] * (-1j) ** sp for m in range(-l, l + 1))
    lhs = O.wigner_d(l, s, sp, th)[l] if s >= 0 else wigner_explicit(l, s, sp, th)
    assert abs(rhs - lhs) < 1e-14
    # the Fourier series of d^l has band limit l (the basis of the doubled-sphere band limit)
    n = 4 * l + 8
    samples = np.array([O.wigner_d(l, abs(s), sp, 2 * math.pi * k / n)[l] for k in range(n)])
    spec = np.fft.fft(samples) / n
    freq = np.fft.fftfreq(n, 1.0 / n)
    assert np.abs(spec[np.abs(freq) > l]).max() < 1e-14


@pytest.mark.parametrize("s", [0, 2])
def test_orthonormality_gauss_legendre(s):
    """sum over a Gauss-Legendre(cos theta, n = lmax + 1) x uniform-phi (2 lmax + 2) grid of
    sY_lm sY*_l'm' equals delta delta: exact since the products are polynomials of degree <= 2 lmax."""
    lmax = 10
    x, w = np.polynomial.legendre.leggauss(lmax + 1)
    nph = 2 * lmax + 2
    phis = 2 * math.pi * np.arange(nph) / nph
    idx = [(l, m) for l in range(s, lmax + 1) for m in range(-l, l + 1)]
    Y = np.zeros((len(idx), x.size * nph), dtype=complex)
    for a, (l, m) in enumerate(idx):
        for i, xi in enumerate(x):
            d = O.wigner_d(l, m, -s, math.acos(xi))[l] * math.sqrt((2 * l + 1) / (4 * math.pi))
            Y[a, i * nph:(i + 1) * nph] = d * np.exp(1j * m * phis) * math.sqrt(w[i] * 2 * math.pi / nph)
    gram = Y @ Y.conj().T
    assert np.abs(gram - np.eye(len(idx))).max() < 1e-13


def test_reflection_identity():
    """d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b): the symmetry the CUDA recursion uses to run
    every ring at a distance <= pi/2 from a pole (follows from the appendix's d(pi + b) relation
    and d^l_{m'm}(-b) = d^l_{mm'}(b))."""
    for l in range(0, 10):
        for m in range(0, l + 1):
            for s in range(0, l + 1):
                for b in (0.2, 1.1, 2.3):
                    lhs = wigner_explicit(l, m, -s, math.pi - b)
                    rhs = (-1) ** (l + m) * wigner_explicit(l, m, s, b)
                    assert abs(lhs - rhs) < 1e-14
