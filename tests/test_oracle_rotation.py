"""Pins of the oracle's change of frame (rotation of a_lm, of points, the spin-basis angle and the
smallest enclosing cap), all on the CPU and independent of the oracle's own Wigner recurrence where
it matters:

  * a field synthesised directly (O1) from the rotated coefficients at the rotated point equals the
    original field at the original point times e^{-i s psi}: this fixes the D-matrix convention,
    the sign of psi and the spin phase together, against the plain synthesis definition;
  * D from Wigner's explicit finite sum (40 digits) applied by hand reproduces the oracle's rotation;
  * closed forms: a rotation about z is the phase e^{-i m alpha}; beta = pi maps a_lm to
    (-1)^l e^{-i m (alpha - gamma)} a*_lm (d^l_{m m'}(pi) = (-1)^(l+m) delta_{m,-m'});
  * R^-1 R = 1 and the weighted a_lm norm is preserved (D is unitary);
  * the smallest cap around points spread over a cap of known centre and radius is that cap.
"""
import math

import numpy as np
import pytest

import oracle as O
from test_oracle_wigner import wigner_explicit


def _alm(rng, lmax, s=0):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_rotated_synthesis_is_the_rotated_field(s):
    rng = np.random.default_rng(10 + s)
    lmax = 9
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    for ang in [(0.7, 1.1, -2.4), (2.0, 2.9, 0.3), (-1.0, 0.2, 5.0)]:
        gr, cr = O.rotate_alm(lmax, g, *ang), O.rotate_alm(lmax, c, *ang)
        th = rng.uniform(0.05, math.pi - 0.05, 25)
        ph = rng.uniform(0.0, 2.0 * math.pi, 25)
        th2, ph2, psi = O.rotate_points(*ang, th, ph)
        f = O.direct_synthesis(lmax, s, g, c, th, ph)
        f2 = O.direct_synthesis(lmax, s, gr, cr, th2, ph2)
        assert np.abs(f2 * np.exp(1j * s * psi) - f).max() <= 1e-12 * np.abs(f).max()


def test_rotation_matches_explicit_wigner_sum():
    rng = np.random.default_rng(20)
    lmax = 6
    a = _alm(rng, lmax)
    al, be, ga = 0.4, 2.2, -1.3
    got = O.rotate_alm(lmax, a, al, be, ga)
    for l in range(lmax + 1):
        full = {mp_: (a[O.alm_index(lmax, l, abs(mp_))] if mp_ >= 0
                      else (-1) ** mp_ * np.conj(a[O.alm_index(lmax, l, -mp_)])) for mp_ in range(-l, l + 1)}
        full[0] = full[0].real
        for m in range(l + 1):
            ref = sum(np.exp(-1j * m * al) * wigner_explicit(l, m, mp_, be) * np.exp(-1j * mp_ * ga) * full[mp_]
                      for mp_ in range(-l, l + 1))
            assert abs(got[O.alm_index(lmax, l, m)] - ref) < 1e-13


def test_closed_forms():
    rng = np.random.default_rng(21)
    lmax = 24
    a = _alm(rng, lmax)
    l, m = O.lm_of_index(lmax)
    a0 = a.copy()
    a0[m == 0] = a0[m == 0].real
    z = O.rotate_alm(lmax, a, 0.9, 0.0, 0.0)
    assert np.abs(z - np.exp(-1j * m * 0.9) * a0).max() < 1e-13
    z = O.rotate_alm(lmax, a, 0.0, 0.0, -0.35)
    assert np.abs(z - np.exp(0.35j * m) * a0).max() < 1e-13
    al, ga = 0.6, -1.7
    z = O.rotate_alm(lmax, a, al, math.pi, ga)
    assert np.abs(z - (-1.0) ** l * np.exp(-1j * m * (al - ga)) * np.conj(a0)).max() < 1e-12


def test_inverse_and_unitarity():
    rng = np.random.default_rng(22)
    lmax = 40
    a = _alm(rng, lmax)
    al, be, ga = 1.3, 0.77, -2.1
    b = O.rotate_alm(lmax, a, al, be, ga)
    back = O.rotate_alm(lmax, b, -ga, -be, -al)
    _, m = O.lm_of_index(lmax)
    a0 = a.copy()
    a0[m == 0] = a0[m == 0].real
    assert np.abs(back - a0).max() < 1e-12
    assert O.alm_dot(b, b, lmax) == pytest.approx(O.alm_dot(a0, a0, lmax), rel=1e-13)
    # selected coefficients agree with the full form
    ls, ms = np.array([40, 17, 33, 5]), np.array([0, 17, 12, 3])
    sel = O.rotate_alm_lm(lmax, a, al, be, ga, ls, ms)
    assert np.abs(sel - b[O.alm_index(lmax, ls, ms)]).max() < 1e-14


def test_rotation_matrix_and_points():
    """R_z(alpha) R_y(beta) R_z(gamma) of the pole is (beta, alpha) in spherical angles, and the
    rotation (0, theta_c, pi - phi_c) takes (theta_c, phi_c) to the pole."""
    R = O.rotation_matrix(0.8, 0.5, 2.0)
    v = R @ np.array([0.0, 0.0, 1.0])
    assert abs(math.acos(v[2]) - 0.5) < 1e-15 and abs(math.atan2(v[1], v[0]) - 0.8) < 1e-15
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-15
    tc, pc = 2.3, 4.0
    th2, _, _ = O.rotate_points(0.0, tc, math.pi - pc, np.array([tc]), np.array([pc]))
    assert th2[0] < 1e-15
    # psi vanishes for rotations about z (the local bases coincide)
    _, ph2, psi = O.rotate_points(0.5, 0.0, 0.25, np.array([1.0, 2.0]), np.array([0.1, 6.0]))
    assert np.abs(psi).max() < 1e-15
    assert np.abs(ph2 - np.mod(np.array([0.1, 6.0]) + 0.75, 2 * math.pi)).max() < 1e-14


def test_min_enclosing_cap_of_a_cap():
    rng = np.random.default_rng(23)
    tc, pc, r = 2.1, 1.0, math.radians(17.0)
    # points uniform in the cap around the pole, with a ring of boundary points, then rotated there
    u = rng.uniform(math.cos(r), 1.0, 150)
    th = np.concatenate([np.arccos(u), np.full(12, r)])
    ph = np.concatenate([rng.uniform(0, 2 * math.pi, 150), np.linspace(0, 2 * math.pi, 12, endpoint=False)])
    # R_z(pc) R_y(tc) takes the pole to (tc, pc)
    th2, ph2, _ = O.rotate_points(pc, tc, 0.0, th, ph)
    t, p, rad = O.min_enclosing_cap(th2, ph2)
    assert abs(rad - r) < 1e-7
    c = np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])
    c0 = np.array([math.sin(tc) * math.cos(pc), math.sin(tc) * math.sin(pc), math.cos(tc)])
    assert math.acos(min(1.0, float(c @ c0))) < 1e-6
