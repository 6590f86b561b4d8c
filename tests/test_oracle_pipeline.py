"""Pins of the oracle's partial-sky pipeline (O2) and direct sums (O1) against facts the paper
and the mathematics fix: closed-form single-coefficient maps, the reality condition, the
adjoint identity, exactness of the full-sky Fourier-sphere route, the paper's own predicted
speed-ups (Table 1), window and kernel properties, and the error behaviour it describes."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _alm(rng, lmax, s):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


def _cap(rng, n, radius, pole="N"):
    th = np.arccos(rng.uniform(math.cos(radius), 1.0, n))
    if pole == "S":
        th = math.pi - th
    return th, rng.uniform(-math.pi, 3 * math.pi, n)


def test_single_coefficient_maps_closed_form():
    """eq. syn with one unit coefficient and the reality rule a_{l,-m} = (-1)^m a*_lm:
    g_lm = 1 (m > 0) gives f = -(sY_lm + (-1)^m sY_{l,-m}); c_lm = 1 gives i times that."""
    th = np.array([0.4, 1.2, 2.5])
    ph = np.array([0.3, 2.0, 5.1])
    e = lambda m: np.exp(1j * m * ph)
    # scalar Y_11 = -sqrt(3/8pi) sin(th) e^{i phi}:  f = -2 Re Y_11
    lmax = 3
    g = np.zeros(O.nalm(lmax), complex)
    g[O.alm_index(lmax, 1, 1)] = 1.0
    ref = 2 * math.sqrt(3 / (8 * math.pi)) * np.sin(th) * np.cos(ph)
    assert np.abs(O.direct_synthesis(lmax, 0, g, None, th, ph) - ref).max() < 1e-15
    # scalar m = 0: f = -Y_10
    g[:] = 0
    g[O.alm_index(lmax, 1, 0)] = 1.0 + 7.0j  # the imaginary part at m = 0 is ignored
    ref = -math.sqrt(3 / (4 * math.pi)) * np.cos(th)
    assert np.abs(O.direct_synthesis(lmax, 0, g, None, th, ph) - ref).max() < 1e-15
    # spin 2, g_22 = 1: f = -(2Y22 + 2Y2-2), c_22 = 1: f = -i(2Y22 + 2Y2-2)
    Y22 = 0.5 * math.sqrt(5 / math.pi) * np.sin(th / 2) ** 4 * e(2)
    Y2m2 = 0.5 * math.sqrt(5 / math.pi) * np.cos(th / 2) ** 4 * e(-2)
    g[:] = 0
    g[O.alm_index(lmax, 2, 2)] = 1.0
    assert np.abs(O.direct_synthesis(lmax, 2, g, None, th, ph) + (Y22 + Y2m2)).max() < 1e-15
    assert np.abs(O.direct_synthesis(lmax, 2, np.zeros_like(g), g, th, ph) + 1j * (Y22 + Y2m2)).max() < 1e-15
    # spin 2, g_20 = 1: f = -2Y20 = -sqrt(15/32pi) sin^2
    g[:] = 0
    g[O.alm_index(lmax, 2, 0)] = 1.0
    ref = -math.sqrt(15 / (32 * math.pi)) * np.sin(th) ** 2
    assert np.abs(O.direct_synthesis(lmax, 2, g, None, th, ph) - ref).max() < 1e-15


def test_reality_spin0():
    rng = np.random.default_rng(1)
    lmax = 40
    g = _alm(rng, lmax, 0)
    th, ph = _cap(rng, 500, 0.5, "S")
    f = O.direct_synthesis(lmax, 0, g, None, th, ph)
    assert np.abs(f.imag).max() < 1e-13 * np.abs(f.real).max()
    P = O.plan_params(lmax, 0, 1e-10, th)
    f2 = O.pipeline_synthesis(P, g, None, th, ph)
    assert np.abs(f2.imag).max() < 1e-9 * np.abs(f2.real).max()


def test_direct_adjoint_is_paper_formula():
    """O1's projection form equals the adjoint synthesis general formula written with sY and _{-s}Y."""
    rng = np.random.default_rng(2)
    lmax, s = 4, 2
    th, ph = _cap(rng, 7, 1.0)
    f = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    gt, ct = O.direct_adjoint(lmax, s, th, ph, f)
    for l in range(s, lmax + 1):
        for m in range(0, l + 1):
            A = sum(f[p] * np.conj(O.sYlm(s, l, m, th[p], ph[p])) for p in range(7))
            B = sum((-1) ** s * np.conj(f[p]) * np.conj(O.sYlm(-s, l, m, th[p], ph[p])) for p in range(7))
            k = O.alm_index(lmax, l, m)
            assert abs(gt[k] - (-0.5 * (A + B))) < 1e-14
            assert abs(ct[k] - (-(A - B) / 2j)) < 1e-14


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_direct_adjoint_dot(s):
    rng = np.random.default_rng(10 + s)
    lmax = 30
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    th, ph = _cap(rng, 400, 1.0, "S")
    f = rng.standard_normal(400) + 1j * rng.standard_normal(400)
    Aa = O.direct_synthesis(lmax, s, g, c, th, ph)
    gt, ct = O.direct_adjoint(lmax, s, th, ph, f)
    lhs = O.map_dot(f, Aa)
    rhs = O.alm_dot(gt, g, lmax) + O.alm_dot(ct, c, lmax)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("s,pole", [(0, "N"), (1, "S"), (2, "S"), (3, "N")])
def test_full_sky_route_is_exact(s, pole):
    """Sec. I.A/I.B: the doubled-sphere map is band-limited by lmax, so lmax+1 rings plus the exact
    non-uniform DFT reproduce direct summation to round-off (pole-crossing sign included)."""
    rng = np.random.default_rng(20 + s)
    lmax = 24
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    th, ph = _cap(rng, 300, 2.6, pole)
    P = O.plan_params(lmax, s, 1e-10, th)
    assert P["full"]
    f1 = O.direct_synthesis(lmax, s, g, c, th, ph)
    f3 = O.pipeline_synthesis(P, g, c, th, ph, exact=True)
    assert O.rel_l2(f3, f1) < 1e-12
    f2 = O.pipeline_synthesis(P, g, c, th, ph)
    assert O.rel_l2(f2, f1) < 10 * 1e-10


CASES = [
    # lmax, s, cap radius, pole, eps
    (64, 0, math.radians(10), "S", 1e-10),
    (64, 2, math.radians(10), "S", 1e-10),
    (96, 2, 0.45, "N", 1e-7),
    (96, 1, 0.3, "S", 1e-5),
    (128, 0, 0.2, "N", 1e-5),
    (128, 3, 0.6, "S", 1e-8),
]


@pytest.mark.parametrize("lmax,s,radius,pole,eps", CASES)
def test_partial_sky_synthesis_within_tolerance(lmax, s, radius, pole, eps):
    rng = np.random.default_rng(lmax + s)
    g, c = _alm(rng, lmax, s), (_alm(rng, lmax, s) if s else None)
    th, ph = _cap(rng, 3000, radius, pole)
    P = O.plan_params(lmax, s, eps, th)
    assert not P["full"]
    f1 = O.direct_synthesis(lmax, s, g, c, th, ph)
    f2 = O.pipeline_synthesis(P, g, c, th, ph)
    assert O.rel_l2(f2, f1) <= 10 * eps


@pytest.mark.parametrize("lmax,s,radius,pole,eps", CASES[:4])
def test_partial_sky_adjoint(lmax, s, radius, pole, eps):
    """Dot-product identity of O2 to 1e-12 (every stage is an exact transpose), and O2's adjoint
    of f = A a against O1's within 10 eps."""
    rng = np.random.default_rng(100 + lmax + s)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    th, ph = _cap(rng, 2000, radius, pole)
    P = O.plan_params(lmax, s, eps, th)
    f = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    Aa = O.pipeline_synthesis(P, g, c, th, ph)
    gt, ct = O.pipeline_adjoint(P, f, th, ph)
    lhs = O.map_dot(f, Aa)
    rhs = O.alm_dot(gt, g, lmax) + O.alm_dot(ct, c, lmax)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    gt2, ct2 = O.pipeline_adjoint(P, Aa, th, ph)
    gt1, ct1 = O.direct_adjoint(lmax, s, th, ph, Aa)
    both = np.concatenate([gt2, ct2]), np.concatenate([gt1, ct1])
    _, m = O.lm_of_index(lmax)
    wgt = np.tile(np.where(m == 0, 1.0, 2.0), 2)
    assert O.rel_l2(both[0], both[1], wgt) <= 10 * eps


def test_stage_transposes():
    """Each O2 stage pair is an exact transpose (dot tests on random inputs)."""
    rng = np.random.default_rng(7)
    lmax, s = 48, 2
    th, ph = _cap(rng, 900, 0.4, "S")
    P = O.plan_params(lmax, s, 1e-8, th)
    nr, nm = P["nring"], 2 * P["M"] + 1
    F = rng.standard_normal((nr, nm)) + 1j * rng.standard_normal((nr, nm))
    H = rng.standard_normal((2 * P["L"] - 1, nm)) + 1j * rng.standard_normal((2 * P["L"] - 1, nm))
    a = np.vdot(H, O.theta_coefficients(P, F)).real
    b = np.vdot(O.theta_coefficients_adjoint(P, H), F).real
    assert abs(a - b) < 1e-12 * abs(a)
    G = rng.standard_normal((P["nrows"], P["nphi"])) + 1j * rng.standard_normal((P["nrows"], P["nphi"]))
    a = np.vdot(G, O.fourier_to_grid(P, H)).real
    b = np.vdot(O.grid_to_fourier(P, G), H).real
    assert abs(a - b) < 1e-12 * abs(a)
    _, _, t, u = O.point_coords(P, th, ph)
    f = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    a = np.vdot(f, O.interp(P, t, u, G)).real
    b = np.vdot(O.spread(P, t, u, f), G).real
    assert abs(a - b) < 1e-12 * abs(a)


def test_window_properties_and_bell_cdf():
    """Sec. II.D: w = 1 exactly on |Theta| <= pi - dTheta = pi/(1 + eps_apo), w(pi) = 0, monotone;
    the bell CDF agrees with adaptive quadrature of the bell itself (scipy.integrate.quad)."""
    eps, eps_apo = 1e-10, 0.137
    dT = math.pi * eps_apo / (1 + eps_apo)
    Th = np.linspace(0, math.pi, 2001)
    w = O.window(Th, dT, eps)
    assert np.all(w[Th <= math.pi / (1 + eps_apo)] == 1.0)
    assert abs(w[-1]) < 1e-20
    assert np.all(np.diff(w) <= 1e-15)
    c = abs(math.log(eps))
    bell = lambda u: math.exp(c * (math.sqrt(max(0.0, 1 - (2 * u / dT) ** 2)) - 1))
    tot = integrate.quad(bell, -dT / 2, dT / 2, epsabs=0, epsrel=1e-13, limit=200)[0]
    for x in (-0.4 * dT, -0.1 * dT, 0.0, 0.27 * dT, 0.49 * dT):
        ref = integrate.quad(bell, -dT / 2, x, epsabs=0, epsrel=1e-13, limit=200)[0] / tot
        assert abs(O.bell_cdf(x, dT, eps)[0] - ref) < 1e-13
    # window spectrum: the product of the bell and top-hat transforms falls below eps past the
    # main lobe, n = Delta_l pi/dTheta with Delta_l = 2 alpha (Sec. II.C-D, Fig. 4 caption)
    n = 1 << 14
    Th = 2 * math.pi * np.arange(n) / n
    Th = np.where(Th > math.pi, Th - 2 * math.pi, Th)
    spec = np.abs(np.fft.fft(O.window(Th, dT, eps))) / n
    alpha = c / math.pi
    cut = int(math.ceil(2 * alpha * math.pi / dT))
    assert spec[cut:n // 2].max() < eps


def test_es_kernel_transform():
    W, beta, nf = 11, 2.30 * 11, 200
    a = W * math.pi / nf
    for k in (0, 7, 33, 60):
        ref = integrate.quad(lambda x: math.exp(beta * (math.sqrt(max(0.0, 1 - (x / a) ** 2)) - 1)) * math.cos(k * x),
                             -a, a, epsabs=0, epsrel=1e-13, limit=400)[0]
        assert abs(O.es_ft(k, W, beta, nf)[0] - ref) < 1e-13 * abs(ref) + 1e-17


def test_table1_predicted_speedups():
    """The planner's parameter rules reproduce Table 1's predicted speed-up column within 10 %."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_predicted_speedup.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 10
    for name, tdeg, lmax, spin, pred in rows:
        got = O.predicted_speedup(int(lmax), math.radians(float(tdeg)), 1e-7)
        assert abs(got / float(pred) - 1) < 0.10, (name, lmax, got, pred)


def test_parameter_rules_match_formulas():
    """P1: eps_apo, theta_max and Lmax as printed in Sec. II.C-D; L >= Lmax + 1 is FFT friendly."""
    rng = np.random.default_rng(3)
    th, _ = _cap(rng, 1000, 0.6)
    P = O.plan_params(4096, 2, 1e-10, th)
    ts = th.max()
    ea = math.sqrt(2 * abs(math.log(1e-10)) / (ts * 4096))
    assert P["eps_apo"] == pytest.approx(ea, rel=1e-15)
    assert P["theta_max"] == pytest.approx(ts * (1 + ea), rel=1e-15)
    assert P["Lmax"] == math.ceil(4096 * ts / math.pi * (1 + ea) ** 2)
    assert P["L"] >= P["Lmax"] + 1 and O.fft_friendly(P["L"]) == P["L"]
    assert P["alpha"] == pytest.approx(abs(math.log(1e-10)) / math.pi)


def test_polar_cutoff_is_conservative():
    """Past M_j every |N_l d^l_{m,+-s}(theta_j)|, l <= lmax, is below 1e-3 eps N_lmax (Sec. II.A)."""
    for lmax, s, eps, beta in [(512, 2, 1e-10, 0.2), (512, 0, 1e-5, 0.6), (1024, 2, 1e-10, 0.05), (256, 2, 1e-5, 1.1)]:
        M = int(O.mcut(lmax, s, eps, beta)[0])
        if M >= lmax:
            continue
        Nl = np.sqrt((2 * np.arange(lmax + 1) + 1) / (4 * math.pi))
        worst = max(np.abs(Nl * O.wigner_d(lmax, m, sp, beta)).max() for m in range(M + 1, lmax + 1) for sp in (-s, s))
        assert worst < 1e-3 * eps * Nl[-1]


def test_dirichlet_interpolation_identity():
    """Sec. I.B eq. Dnz: sum_j D_j(theta) f(theta_j) = f(theta) for band limit Lb and 2Lb+1 samples."""
    rng = np.random.default_rng(4)
    Lb = 9
    coef = rng.standard_normal(2 * Lb + 1) + 1j * rng.standard_normal(2 * Lb + 1)
    ks = np.arange(-Lb, Lb + 1)
    f = lambda t: np.exp(1j * np.outer(np.atleast_1d(t), ks)) @ coef
    tj = 2 * math.pi * np.arange(2 * Lb + 1) / (2 * Lb + 1)
    for t in (0.1, 1.7, 4.4):
        D = np.exp(1j * np.outer(t - tj, ks)).sum(axis=1) / (2 * Lb + 1)
        assert abs(D @ f(tj) - f(t)[0]) < 1e-13


def test_error_envelope_and_QU_asymmetry():
    """Sec. II.E: the apodisation error is smallest on ring latitudes and largest half-way between
    them; for a pure E (gradient) spin-2 field the Q error exceeds the U error."""
    rng = np.random.default_rng(5)
    lmax, eps = 128, 1e-6
    g = _alm(rng, lmax, 0)
    th0, _ = _cap(rng, 2000, 0.5)
    P = O.plan_params(lmax, 0, eps, th0)
    js = np.arange(1, int(P["L"] / (1 + P["eps_apo"])) - 1)
    errs = []
    for off in (0.0, 0.5):
        Th = (js + off) * math.pi / P["L"]
        th = np.repeat(Th * P["theta_max"] / math.pi, 24)
        ph = np.tile(np.linspace(0, 2 * math.pi, 24, endpoint=False), js.size)
        f1 = O.direct_synthesis(lmax, 0, g, None, th, ph)
        f3 = O.pipeline_synthesis(P, g, None, th, ph, exact=True)
        errs.append(np.sqrt(np.mean(np.abs(f3 - f1) ** 2)))
    assert errs[0] < 0.5 * errs[1]
    lmax = 192
    g = _alm(rng, lmax, 2)
    th, ph = _cap(rng, 8000, 0.4)
    P = O.plan_params(lmax, 2, 1e-5, th)
    d = O.pipeline_synthesis(P, g, None, th, ph, exact=True) - O.direct_synthesis(lmax, 2, g, None, th, ph)
    assert np.sqrt(np.mean(d.real ** 2)) > 1.1 * np.sqrt(np.mean(d.imag ** 2))


def test_direct_adjoint_selected_coefficients():
    """The restricted direct adjoint equals the full direct adjoint at the selected (l, m)."""
    rng = np.random.default_rng(9)
    lmax, s = 20, 2
    th, ph = _cap(rng, 300, 0.8, "S")
    f = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    gt, ct = O.direct_adjoint(lmax, s, th, ph, f)
    sel = [(2, 0), (2, 2), (5, 1), (20, 20), (13, 7), (1, 0)]
    ls, ms = np.array([a for a, _ in sel]), np.array([b for _, b in sel])
    g2, c2 = O.direct_adjoint_lm(s, th, ph, f, ls, ms)
    idx = O.alm_index(lmax, ls, ms)
    assert np.abs(g2 - gt[idx]).max() < 1e-13 * np.abs(gt).max()
    assert np.abs(c2 - ct[idx]).max() < 1e-13 * np.abs(ct).max()
