"""Plain FP64 CPU oracle for partial-sky synthesis general and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.  It
shares no code with the CUDA path (``paper_2603_17166_gb300``) and never imports it.

Two oracles (Carron & Reinecke 2026, "Fast partial-sky spherical harmonic transforms"):

O1  direct summation of the synthesis general equation (Sec. I, eq. syn) and of its adjoint
    (Sec. I, adjoint synthesis general), with sY_lm from the appendix (eq. Ylm).
O2  the partial-sky method step by step (Sec. II, steps 1-4), written plainly:
      P0 frame:   nearest pole, beta_p = colatitude from it, theta* = max beta_p  (Sec. II step 1)
      P1 params:  alpha = |ln eps|/pi, eps_apo = sqrt(2|ln eps|/(theta* lmax)),
                  theta_max = theta*(1+eps_apo), Lmax = ceil(lmax theta*/pi (1+eps_apo)^2)
                  (Sec. II steps 2, II.C eq. Lmax2, II.D summary)
      P2 rings:   Theta_j = j pi/L, theta_j = Theta_j theta_max/pi, w_j = w(Theta_j) with the
                  window = top-hat (x) ES bell (Sec. II.D, Fig. 4 caption, eq. KB)
      P3 rings:   F_j[m] = -sum_l (g+ic)_lm N_l d^l_{m,-s}(theta_j)             (eq. syn, eq. Ylm)
      P4 Theta:   doubled-circle samples with the pole-crossing sign (-1)^(s+m) (Sec. I.A eq. sht,
                  appendix), DFT of length 2L                                    (Sec. I.B)
      P5 points:  ES-kernel type-2 NUFFT (Barnett et al. 2019), or the exact non-uniform DFT
      P6 adjoint: the exact transpose of P5 -> P3 followed by the adjoint projection (Sec. I).

Where the paper is silent, the numerical choices (ring count rounding, polar-optimisation cutoff,
NUFFT grid sizes) are written out in ``plan_params`` below; the product's planner makes the same
choices in its own code.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_WORKERS = [os.cpu_count()]  # FFT threads; set_num_threads changes it with the C part's

try:
    import scipy.fft as _fft

    def _fftn(a, axis):
        return _fft.fft(a, axis=axis, workers=_WORKERS[0])

    def _ifftn(a, axis):
        return _fft.ifft(a, axis=axis, workers=_WORKERS[0])
except Exception:  # pragma: no cover - scipy is in every image used here
    def _fftn(a, axis):
        return np.fft.fft(a, axis=axis)

    def _ifftn(a, axis):
        return np.fft.ifft(a, axis=axis)

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile psht_oracle.c with gcc + OpenMP into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "psht_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.orc_wigner_d_column.argtypes = [I, I, I, D, D, D, P]
        lib.orc_ring_synthesis.argtypes = [I, I, I, P, P, L, P, P]
        lib.orc_ring_adjoint.argtypes = [I, I, I, L, P, P, P, P]
        lib.orc_direct_synthesis.argtypes = [I, I, P, P, L, P, P, P]
        lib.orc_direct_adjoint.argtypes = [I, I, L, P, P, P, P, P]
        lib.orc_interp.argtypes = [L, P, P, I, D, L, L, L, P, P]
        lib.orc_spread.argtypes = [L, P, P, P, I, D, L, L, L, P, P]
        lib.orc_direct_adjoint_lm.argtypes = [I, L, P, P, P, I, P, P, P, P]
        lib.orc_rotate_alm.argtypes = [I, D, D, D, P, I, P, P, P]
        lib.orc_num_threads.restype = I
        lib.orc_set_num_threads.argtypes = [I]
        _lib_handle = lib
    return _lib_handle


def num_threads() -> int:
    """OpenMP threads the C part uses (all cores in the affinity mask unless OMP_NUM_THREADS)."""
    return int(_lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the C part and of the FFTs from now on."""
    _lib().orc_set_num_threads(int(n))
    _WORKERS[0] = int(n)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c128(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.complex128)


# ----------------------------------------------------------------------------- alm packing
def nalm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l, m):
    """Packed m-major index m(2 lmax + 1 - m)/2 + l."""
    return m * (2 * lmax + 1 - m) // 2 + l


def lm_of_index(lmax: int):
    """(l, m) arrays for every packed index."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def canonical_alm(a, lmax: int, s: int):
    """Zero what the transform ignores: Im at m = 0 and l < s (reading of Sec. I reality rule)."""
    a = np.array(a, dtype=np.complex128, copy=True)
    l, m = lm_of_index(lmax)
    a[m == 0] = a[m == 0].real
    a[l < s] = 0
    return a


def alm_dot(a, b, lmax: int):
    """<a, b> = sum_l sum_{m=-l..l} Re(conj(a) b) for reality-constrained a: m=0 once, m>0 twice."""
    _, m = lm_of_index(lmax)
    wgt = np.where(m == 0, 1.0, 2.0)
    return float(np.sum(wgt * (np.conj(a) * b).real))


def map_dot(f, h):
    """<f, h> = Re sum_p conj(f_p) h_p."""
    return float(np.sum((np.conj(f) * h).real))


def rel_l2(x, ref, weights=None):
    x = np.asarray(x)
    ref = np.asarray(ref)
    if weights is None:
        return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))
    num = np.sqrt(np.sum(weights * np.abs(x - ref) ** 2))
    den = np.sqrt(np.sum(weights * np.abs(ref) ** 2))
    return float(num / max(den, 1e-300))


def alm_rel_l2(x, ref, lmax: int):
    _, m = lm_of_index(lmax)
    return rel_l2(x, ref, np.where(m == 0, 1.0, 2.0))


# ----------------------------------------------------------------------------- Wigner d, sY
def wigner_d(lmax: int, m: int, mp: int, beta: float) -> np.ndarray:
    """d^l_{m,mp}(beta) for l = 0..lmax, any integer m, mp (appendix, Wigner small-d).

    Negative m uses d^l_{m,mp} = d^l_{-mp,-m}, or d^l_{m,mp} = (-1)^(mp-m) d^l_{mp,m}."""
    out = np.zeros(lmax + 1)
    if m < 0:
        if mp <= 0:
            return wigner_d(lmax, -mp, -m, beta)
        return (-1.0) ** ((mp - m) % 2) * wigner_d(lmax, mp, m, beta)
    _lib().orc_wigner_d_column(lmax, m, mp, math.cos(beta), math.cos(0.5 * beta), math.sin(0.5 * beta),
                               out.ctypes.data)
    return out


def sYlm(s: int, l: int, m: int, theta: float, phi: float) -> complex:
    """sY_lm(theta, phi) = sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi}  (appendix, eq. Ylm)."""
    if l < max(abs(m), abs(s)):
        return 0j
    d = wigner_d(l, m, -s, theta)[l]
    return math.sqrt((2 * l + 1) / (4 * math.pi)) * d * complex(math.cos(m * phi), math.sin(m * phi))


# ----------------------------------------------------------------------------- O1
def direct_synthesis(lmax: int, s: int, g, c, theta, phi) -> np.ndarray:
    """O1: f_p = -sum_{l,m} (g_lm + i c_lm) sY_lm(theta_p, phi_p)   (Sec. I, eq. syn)."""
    g = _c128(g)
    c = _c128(c)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    f = np.zeros(theta.size, dtype=np.complex128)
    _lib().orc_direct_synthesis(lmax, s, _ptr(g), _ptr(c), theta.size, _ptr(theta), _ptr(phi), _ptr(f))
    return f


def direct_adjoint(lmax: int, s: int, theta, phi, f):
    """O1: adjoint synthesis general (Sec. I):
    g~ = -1/2 sum_p [f_p sY*_lm + (-1)^s f*_p _{-s}Y*_lm],
    c~ = -1/(2i) sum_p [f_p sY*_lm - (-1)^s f*_p _{-s}Y*_lm]."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    f = _c128(f)
    gt = np.zeros(nalm(lmax), dtype=np.complex128)
    ct = np.zeros(nalm(lmax), dtype=np.complex128)
    _lib().orc_direct_adjoint(lmax, s, theta.size, _ptr(theta), _ptr(phi), _ptr(f), _ptr(gt), _ptr(ct))
    return gt, ct


def direct_adjoint_lm(s: int, theta, phi, f, ls, ms):
    """O1 adjoint restricted to selected (l, m >= 0): (g~, c~) at those coefficients only."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    f = _c128(f)
    ls = np.ascontiguousarray(ls, dtype=np.int32)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    gt = np.zeros(ls.size, dtype=np.complex128)
    ct = np.zeros(ls.size, dtype=np.complex128)
    _lib().orc_direct_adjoint_lm(s, theta.size, _ptr(theta), _ptr(phi), _ptr(f), ls.size, _ptr(ls), _ptr(ms),
                                 _ptr(gt), _ptr(ct))
    return gt, ct


# ----------------------------------------------------------------------------- rotations
# The paper centres the patch at the north pole (Sec. II, step 1) without saying how a caller's
# a_lm get there.  These are the plain definitions of that change of frame: the Wigner-D
# rotation of a coefficient set, the rotation of points, and the angle between the two frames'
# local bases at each point, which a spin-s field picks up as a phase.
def rotation_matrix(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """R = R_z(alpha) R_y(beta) R_z(gamma), active rotations of vectors (zyz Euler angles)."""
    def rz(a):
        return np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])

    def ry(b):
        return np.array([[math.cos(b), 0.0, math.sin(b)], [0.0, 1.0, 0.0], [-math.sin(b), 0.0, math.cos(b)]])

    return rz(alpha) @ ry(beta) @ rz(gamma)


def rotate_alm(lmax: int, a, alpha: float, beta: float, gamma: float) -> np.ndarray:
    """a'_lm = sum_m' e^{-i m alpha} d^l_{m m'}(beta) e^{-i m' gamma} a_lm' for one real field's
    packed set (m >= 0, a_{l,-m} = (-1)^m a*_lm): the field carried along by R(alpha, beta, gamma).
    For a spin-s field synthesised from rotated g and c, f'(R p) = e^{-i s psi_p} f(p), psi_p from
    ``rotate_points``."""
    a = _c128(a)
    out = np.zeros(nalm(lmax), dtype=np.complex128)
    _lib().orc_rotate_alm(lmax, alpha, beta, gamma, _ptr(a), -1, None, None, _ptr(out))
    return out


def rotate_alm_lm(lmax: int, a, alpha: float, beta: float, gamma: float, ls, ms) -> np.ndarray:
    """``rotate_alm`` at selected (l, m >= 0) only (O(l^2) each)."""
    a = _c128(a)
    ls = np.ascontiguousarray(ls, dtype=np.int32)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    out = np.zeros(ls.size, dtype=np.complex128)
    _lib().orc_rotate_alm(lmax, alpha, beta, gamma, _ptr(a), int(ls.size), _ptr(ls), _ptr(ms), _ptr(out))
    return out


def _unit(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=-1)


def rotate_points(alpha: float, beta: float, gamma: float, theta, phi):
    """n_p = R p for points p = (theta, phi): returns (theta', phi' in [0, 2pi), psi), where psi is
    the angle from e_theta(p) towards e_phi(p) of the rotated frame's e_theta at n_p carried back by
    R^-1, so that a spin-s field in the two frames' local bases satisfies f(p) = e^{i s psi} f'(n_p)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    R = rotation_matrix(alpha, beta, gamma)
    n = _unit(theta, phi) @ R.T
    th2 = np.arctan2(np.hypot(n[..., 0], n[..., 1]), n[..., 2])
    ph2 = np.mod(np.arctan2(n[..., 1], n[..., 0]), 2.0 * math.pi)
    et2 = np.stack([np.cos(th2) * np.cos(ph2), np.cos(th2) * np.sin(ph2), -np.sin(th2)], axis=-1)
    back = et2 @ R  # R^-1 e_theta'(n), rows
    et = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], axis=-1)
    ep = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=-1)
    psi = np.arctan2(np.sum(back * ep, axis=-1), np.sum(back * et, axis=-1))
    return th2, ph2, psi


def min_enclosing_cap(theta, phi):
    """Smallest spherical cap holding every point: the centre c maximises min_p <p, c>, and by
    duality c is the direction of the minimum-norm point of the points' convex hull, with
    cos(radius) = its norm (valid while the points lie in an open hemisphere).  Solved here as the
    small quadratic programme min |sum_p lambda_p p|^2, lambda >= 0, sum lambda = 1 (SLSQP), for a
    few hundred points at most.  Returns (theta_c, phi_c, radius)."""
    from scipy.optimize import minimize

    P = _unit(np.asarray(theta, dtype=np.float64), np.asarray(phi, dtype=np.float64))
    n = P.shape[0]
    G = P @ P.T
    x0 = np.full(n, 1.0 / n)
    res = minimize(lambda lam: lam @ G @ lam, x0, jac=lambda lam: 2.0 * G @ lam, method="SLSQP",
                   bounds=[(0.0, None)] * n, constraints=[{"type": "eq", "fun": lambda lam: lam.sum() - 1.0,
                                                          "jac": lambda lam: np.ones_like(lam)}],
                   options={"ftol": 1e-16, "maxiter": 2000})
    x = res.x @ P
    c = x / np.linalg.norm(x)
    radius = math.acos(min(1.0, float(np.min(P @ c))))
    return math.atan2(math.hypot(c[0], c[1]), c[2]), math.atan2(c[1], c[0]) % (2.0 * math.pi), radius


# ----------------------------------------------------------------------------- O2 building blocks
def ring_synthesis(lmax: int, s: int, mmax: int, g, c, theta_rings) -> np.ndarray:
    """F[k, m + mmax] = -sum_l u_lm N_l d^l_{m,-s}(theta_k), |m| <= mmax (P3)."""
    g = _c128(g)
    c = _c128(c)
    th = np.ascontiguousarray(theta_rings, dtype=np.float64)
    F = np.zeros((th.size, 2 * mmax + 1), dtype=np.complex128)
    _lib().orc_ring_synthesis(lmax, s, mmax, _ptr(g), _ptr(c), th.size, _ptr(th), _ptr(F))
    return F


def ring_adjoint(lmax: int, s: int, mmax: int, theta_rings, G):
    """Transpose of ring_synthesis followed by the adjoint projection onto (g~, c~) (P6)."""
    th = np.ascontiguousarray(theta_rings, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    assert G.shape == (th.size, 2 * mmax + 1)
    gt = np.zeros(nalm(lmax), dtype=np.complex128)
    ct = np.zeros(nalm(lmax), dtype=np.complex128)
    _lib().orc_ring_adjoint(lmax, s, mmax, th.size, _ptr(th), _ptr(G), _ptr(gt), _ptr(ct))
    return gt, ct


def fft_friendly(n: int) -> int:
    """Smallest integer >= n whose prime factors are in {2, 3, 5, 7}."""
    n = max(int(n), 1)
    while True:
        k = n
        for p in (2, 3, 5, 7):
            while k % p == 0:
                k //= p
        if k == 1:
            return n
        n += 1


_GL_CACHE: dict = {}


def _gauss_legendre(n: int):
    if n not in _GL_CACHE:
        _GL_CACHE[n] = np.polynomial.legendre.leggauss(n)
    return _GL_CACHE[n]


def _integrate(fun, a: float, b: float, n: int = 256) -> float:
    x, w = _gauss_legendre(n)
    xm, xr = 0.5 * (b + a), 0.5 * (b - a)
    return float(xr * np.sum(w * fun(xm + xr * x)))


def bell(v, eps: float, kind: str = "es"):
    """Unnormalised bells on |v| <= 1 (v = 2u/dTheta), shape parameter alpha pi = |ln eps|:
    'es' the exponential of a semicircle exp[alpha pi (sqrt(1 - v^2) - 1)] (Sec. II.D eq. KB), 'kb'
    the Kaiser-Bessel bell I0(alpha pi sqrt(1 - v^2)) whose Fourier transform Sec. II.D prints."""
    c = abs(math.log(eps))
    r = np.sqrt(np.clip(1.0 - np.asarray(v, dtype=np.float64) ** 2, 0.0, None))
    if kind == "es":
        return np.exp(c * (r - 1.0))
    if kind == "kb":
        return np.i0(c * r)
    raise ValueError(kind)


def bell_cdf(x, dTheta: float, eps: float, kind: str = "es"):
    """CDF of the bell of support dTheta (|u| <= dTheta/2), unit area, alpha = |ln eps|/pi (Sec. II.D
    rescaled to support dTheta, Fig. 4 caption).  Integrated with u = (dTheta/2) sin(tau), which
    makes the integrand smooth."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    dens = lambda tau: bell(np.sin(tau), eps, kind) * np.cos(tau)
    total = _integrate(dens, -0.5 * math.pi, 0.5 * math.pi)
    out = np.empty_like(x)
    for i, xi in enumerate(x):
        z = 2.0 * xi / dTheta
        if z <= -1.0:
            out[i] = 0.0
        elif z >= 1.0:
            out[i] = 1.0
        else:
            out[i] = _integrate(dens, -0.5 * math.pi, math.asin(z)) / total
    return out


def window(Theta, dTheta: float, eps: float, kind: str = "es"):
    """w(Theta) = (top-hat of support 2pi - dTheta) convolved with the unit-area bell of support
    dTheta, i.e. w = B(pi - dTheta/2 - |Theta|) with B the bell CDF (Sec. II.D)."""
    Theta = np.abs(np.asarray(Theta, dtype=np.float64))
    return bell_cdf(math.pi - 0.5 * dTheta - Theta, dTheta, eps, kind)


def es_kernel(z, beta: float):
    """psi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1 (Barnett's ES kernel)."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    inside = np.abs(z) <= 1.0
    out[inside] = np.exp(beta * (np.sqrt(1.0 - z[inside] ** 2) - 1.0))
    return out


def es_ft(k, W: int, beta: float, nfine: int):
    """Continuous Fourier transform at integer frequencies k of the kernel psi(x/a) with
    half-width a = W pi/nfine:  a int_{-1}^{1} psi(z) cos(k a z) dz  (z = sin tau)."""
    a = W * math.pi / nfine
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    x, w = _gauss_legendre(256)
    tau = 0.5 * math.pi * x
    base = np.exp(beta * (np.cos(tau) - 1.0)) * np.cos(tau) * (0.5 * math.pi) * w
    return a * np.array([np.sum(base * np.cos(kk * a * np.sin(tau))) for kk in k])


def es_width(eps: float) -> int:
    """W = ceil(log10(1/eps)) + 1, at most 16 (sigma = 2 ES rule of Barnett et al. 2019)."""
    return int(min(16, math.ceil(-math.log10(eps) - 1e-9) + 1))


def mcut(lmax: int, s: int, eps: float, beta) -> np.ndarray:
    """Polar-optimisation cutoff (Sec. II.A): keep |m| <= M_j on a ring at distance beta from
    the pole.  x = (lmax + 1/2) sin(beta) is the turning point; the Airy-type tail beyond it
    is kept until it falls below delta = 1e-3 eps:  M_j = ceil(x + s + 1.25 z (x/2)^(1/3) + 8),
    z = (1.5 ln(1/delta))^(2/3), capped at lmax."""
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    z = (1.5 * math.log(1.0 / (1e-3 * eps))) ** (2.0 / 3.0)
    out = np.empty(beta.size, dtype=np.int64)
    for i, b in enumerate(beta):
        x = (lmax + 0.5) * abs(math.sin(b))
        out[i] = min(lmax, math.ceil(x + s + 1.25 * z * (x / 2.0) ** (1.0 / 3.0) + 8.0))
    return out


def legendre_cost(lmax: int, s: int, Mj) -> int:
    """(ring, m, l) steps of the recursion: sum over rings j and 0 <= m <= M_j of lmax - max(m, s) + 1."""
    tot = 0
    for M in np.asarray(Mj, dtype=np.int64):
        m = np.arange(int(M) + 1)
        tot += int(np.sum(lmax - np.maximum(m, s) + 1))
    return tot


def cost_optimal_eps_apo(lmax: int, s: int, eps: float, tstar: float, kappa: float = 1.0):
    """The apodisation length that minimises the Legendre cost inclusive of polar optimisation, the
    alternative to eq. Lmax2 the paper mentions beside it (Sec. II.C).  For a relative apodisation
    length e = Delta theta / theta*, the window adds Delta Lmax = Delta l pi / Delta theta modes
    (Delta l = 2 alpha), so Lmax(e) = (lmax + Delta l pi / (e theta*)) theta* (1 + e) / pi; eq. Lmax2
    is its minimum over e.  Candidates e = e0 r, r = (20 + k)/40, k = 0..80 (e0 the paper's value);
    returns (e, Lmax) of the cheapest (the first on ties), or None if every candidate needs the full
    sky."""
    lneps = abs(math.log(eps))
    e0 = math.sqrt(2.0 * lneps / (tstar * lmax))
    best = None
    for k in range(81):
        e = e0 * ((20 + k) / 40.0)
        tmax = tstar * (1.0 + e)
        Lmax = math.ceil(kappa * lmax * tstar / math.pi * (1.0 + e) * (1.0 + e0 * e0 / e))
        if tmax >= math.pi or Lmax >= lmax:
            continue
        L = fft_friendly(Lmax + 1)
        beta_j = np.arange(L) * (math.pi / L) * (tmax / math.pi)
        cost = legendre_cost(lmax, s, mcut(lmax, s, eps, beta_j))
        if best is None or cost < best[0]:
            best = (cost, e, Lmax)
    return None if best is None else (best[1], best[2])


def plan_params(lmax: int, s: int, eps: float, theta, kappa: float = 1.0, window_kind: str = "es",
                eps_apo_choice: str = "paper") -> dict:
    """P0-P2 of the partial-sky method plus the NUFFT grid (see module docstring); kappa scales the
    band limit Lmax (Sec. II.C), window_kind picks the bell (Sec. II.D), eps_apo_choice "cost" takes
    the apodisation length from ``cost_optimal_eps_apo`` instead of eq. Lmax2."""
    theta = np.asarray(theta, dtype=np.float64)
    bN = float(theta.max()) if theta.size else 0.0
    bS = float((math.pi - theta).max()) if theta.size else 0.0
    pole = "N" if bN <= bS else "S"
    beta_p = theta if pole == "N" else math.pi - theta
    tstar = max(float(beta_p.max()) if theta.size else 0.0, 1e-9)
    lneps = abs(math.log(eps))
    full = False
    if lmax < 1:
        full = True
    else:
        eps_apo = math.sqrt(2.0 * lneps / (tstar * lmax))
        tmax = tstar * (1.0 + eps_apo)
        Lmax = math.ceil(kappa * lmax * tstar / math.pi * (1.0 + eps_apo) ** 2)
        if tmax >= math.pi or Lmax >= lmax:
            full = True
        if eps_apo_choice == "cost":
            opt = cost_optimal_eps_apo(lmax, s, eps, tstar, kappa)
            full = opt is None
            if opt is not None:
                eps_apo, Lmax = opt
                tmax = tstar * (1.0 + eps_apo)
    if full:
        eps_apo, tmax, Lmax, dTheta = 0.0, math.pi, lmax, 0.0
    else:
        dTheta = math.pi * eps_apo / (1.0 + eps_apo)
    L = fft_friendly(Lmax + 1)
    nring = L + 1 if full else L
    Theta_j = np.arange(nring) * (math.pi / L)
    beta_j = Theta_j * (tmax / math.pi)
    theta_j = beta_j if pole == "N" else math.pi - beta_j
    w_j = np.ones(nring) if full else window(Theta_j, dTheta, eps, window_kind)
    Mj = mcut(lmax, s, eps, beta_j)
    M = int(Mj.max())
    W = es_width(eps)
    nTheta = 4 * L
    nphi = 2 * fft_friendly(2 * M + 1)
    t_max = tstar * nTheta / (2.0 * tmax)
    r_lo = math.ceil(-0.5 * W)
    r_hi = math.ceil(t_max - 0.5 * W) + W
    return dict(lmax=lmax, s=s, eps=eps, pole=pole, theta_star=tstar, eps_apo=eps_apo, theta_max=tmax,
                Lmax=Lmax, L=L, full=full, nring=nring, dTheta=dTheta, alpha=lneps / math.pi,
                Theta_j=Theta_j, theta_j=theta_j, w_j=w_j, Mj=Mj, M=M, W=W, beta_es=2.30 * W,
                nTheta=nTheta, nphi=nphi, r_lo=r_lo, r_hi=r_hi, nrows=r_hi - r_lo + 1)


def predicted_speedup(lmax: int, theta_star: float, eps: float) -> float:
    """Legendre speed-up 1/[(1 + eps_apo) 2 f_sky^cap(theta_max)], f_sky^cap = (1 - cos)/2 (Sec. II.A)."""
    eps_apo = math.sqrt(2.0 * abs(math.log(eps)) / (theta_star * lmax))
    tmax = theta_star * (1.0 + eps_apo)
    return 1.0 / ((1.0 + eps_apo) * (1.0 - math.cos(tmax)))


def point_coords(P: dict, theta, phi):
    """Theta_p = pi beta_p/theta_max (Sec. II step 3) and fine-grid coordinates t_p, u_p."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    beta = theta if P["pole"] == "N" else math.pi - theta
    Th = beta * (math.pi / P["theta_max"])
    ph = phi - 2.0 * math.pi * np.floor(phi / (2.0 * math.pi))
    t = Th * (P["nTheta"] / (2.0 * math.pi))
    u = ph * (P["nphi"] / (2.0 * math.pi))
    return Th, ph, t, u


def _scales(P: dict):
    L, M = P["L"], P["M"]
    n = np.arange(-(L - 1), L)
    m = np.arange(-M, M + 1)
    hT = 2.0 * math.pi / P["nTheta"]
    hP = 2.0 * math.pi / P["nphi"]
    sT = hT / (2.0 * L * es_ft(n, P["W"], P["beta_es"], P["nTheta"]))
    sP = hP / es_ft(m, P["W"], P["beta_es"], P["nphi"])
    return n, m, sT, sP


def _sigma(P: dict):
    m = np.arange(-P["M"], P["M"] + 1)
    return np.where((P["s"] + m) % 2 == 0, 1.0, -1.0)


def theta_coefficients(P: dict, F) -> np.ndarray:
    """P4: doubled-circle samples h_k (k < 2L) from the ring coefficients, then
    H[n, m] = sum_k h_k e^{-i pi n k/L}, |n| <= L-1 (rows n + L - 1)."""
    L = P["L"]
    sig = _sigma(P)
    h = np.zeros((2 * L, F.shape[1]), dtype=np.complex128)
    wF = P["w_j"][:, None] * F
    h[: P["nring"]] = wF
    for k in range(L + 1, 2 * L):
        h[k] = sig * wF[2 * L - k]
    H = _fftn(h, axis=0)
    n = np.arange(-(L - 1), L)
    return H[n % (2 * L)]


def theta_coefficients_adjoint(P: dict, Ht) -> np.ndarray:
    """Transpose of theta_coefficients: h~_k = sum_n H~[n] e^{+i pi n k/L}, then the fold
    F~_j = w_j (h~_j + sigma_m h~_{2L-j}) for 0 < j < L, F~_0 = w_0 h~_0 (and F~_L = w_L h~_L)."""
    L = P["L"]
    sig = _sigma(P)
    n = np.arange(-(L - 1), L)
    pad = np.zeros((2 * L, Ht.shape[1]), dtype=np.complex128)
    pad[n % (2 * L)] = Ht
    ht = _ifftn(pad, axis=0) * (2 * L)
    Ft = np.zeros((P["nring"], Ht.shape[1]), dtype=np.complex128)
    Ft[0] = ht[0]
    for j in range(1, L):
        Ft[j] = ht[j] + sig * ht[2 * L - j]
    if P["full"]:
        Ft[L] = ht[L]
    return P["w_j"][:, None] * Ft


def fourier_to_grid(P: dict, H) -> np.ndarray:
    """Deconvolve by the kernel transforms, zero-pad and inverse-FFT onto the kept grid rows:
    G[r, q] = sum_{n,m} H[n,m] sT(n) sP(m) e^{i 2pi (n r/nTheta + m q/nphi)}, r in [r_lo, r_hi]."""
    n, m, sT, sP = _scales(P)
    b = H * sT[:, None] * sP[None, :]
    padT = np.zeros((P["nTheta"], b.shape[1]), dtype=np.complex128)
    padT[n % P["nTheta"]] = b
    C = _ifftn(padT, axis=0) * P["nTheta"]
    rows = np.arange(P["r_lo"], P["r_hi"] + 1)
    Cr = C[rows % P["nTheta"]]
    padP = np.zeros((rows.size, P["nphi"]), dtype=np.complex128)
    padP[:, m % P["nphi"]] = Cr
    return _ifftn(padP, axis=1) * P["nphi"]


def grid_to_fourier(P: dict, G) -> np.ndarray:
    """Transpose of fourier_to_grid."""
    n, m, sT, sP = _scales(P)
    Ct = _fftn(G, axis=1)[:, m % P["nphi"]]
    rows = np.arange(P["r_lo"], P["r_hi"] + 1)
    padT = np.zeros((P["nTheta"], Ct.shape[1]), dtype=np.complex128)
    np.add.at(padT, rows % P["nTheta"], Ct)
    bt = _fftn(padT, axis=0)[n % P["nTheta"]]
    return bt * sT[:, None] * sP[None, :]


def interp(P: dict, t, u, G) -> np.ndarray:
    t = np.ascontiguousarray(t, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    f = np.zeros(t.size, dtype=np.complex128)
    _lib().orc_interp(t.size, _ptr(t), _ptr(u), P["W"], P["beta_es"], P["r_lo"], G.shape[0], G.shape[1],
                      _ptr(G), _ptr(f))
    return f


def spread(P: dict, t, u, f) -> np.ndarray:
    t = np.ascontiguousarray(t, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = _c128(f)
    r0 = np.ceil(t - 0.5 * P["W"])
    order = np.ascontiguousarray(np.argsort(r0, kind="stable"), dtype=np.int64)
    G = np.zeros((P["nrows"], P["nphi"]), dtype=np.complex128)
    _lib().orc_spread(t.size, _ptr(t), _ptr(u), _ptr(order), P["W"], P["beta_es"], P["r_lo"], P["nrows"],
                      P["nphi"], _ptr(f), _ptr(G))
    return G


def pipeline_synthesis(P: dict, g, c, theta, phi, exact: bool = False, return_stages: bool = False):
    """O2 synthesis general at the points, step by step (P3 -> P4 -> P5)."""
    lmax, s = P["lmax"], P["s"]
    F = ring_synthesis(lmax, s, P["M"], g, c, P["theta_j"])
    H = theta_coefficients(P, F)
    Th, ph, t, u = point_coords(P, theta, phi)
    if exact:
        L, M = P["L"], P["M"]
        n = np.arange(-(L - 1), L)
        m = np.arange(-M, M + 1)
        Hb = H / (2 * L)
        f = np.einsum("pn,nm,pm->p", np.exp(1j * np.outer(Th, n)), Hb, np.exp(1j * np.outer(ph, m)))
        G = None
    else:
        G = fourier_to_grid(P, H)
        f = interp(P, t, u, G)
    if return_stages:
        return f, dict(F=F, H=H, G=G)
    return f


def pipeline_adjoint(P: dict, f, theta, phi, exact: bool = False, return_stages: bool = False):
    """O2 adjoint synthesis general: exact transpose of pipeline_synthesis (P6)."""
    lmax, s = P["lmax"], P["s"]
    Th, ph, t, u = point_coords(P, theta, phi)
    f = _c128(f)
    if exact:
        L, M = P["L"], P["M"]
        n = np.arange(-(L - 1), L)
        m = np.arange(-M, M + 1)
        Ht = np.einsum("pn,p,pm->nm", np.exp(-1j * np.outer(Th, n)), f, np.exp(-1j * np.outer(ph, m))) / (2 * L)
        G = None
    else:
        G = spread(P, t, u, f)
        Ht = grid_to_fourier(P, G)
    Ft = theta_coefficients_adjoint(P, Ht)
    gt, ct = ring_adjoint(lmax, s, P["M"], P["theta_j"], Ft)
    if return_stages:
        return (gt, ct), dict(G=G, H=Ht, F=Ft)
    return gt, ct


# ----------------------------------------------------------------------------- error predictor
def great_circle_spectrum(lmax: int, s: int, cl) -> np.ndarray:
    """c_m, m = -lmax..lmax: power along a great circle through the pole of an isotropic field with
    spectrum C_l (eq. cm for s = 0, eq. cms with C_l = C^E_l + C^B_l for s > 0):
    c_m = sum_l C_l (2l+1)/2 |d^l_{m,-s}(pi/2)|^2."""
    cl = np.asarray(cl, dtype=np.float64)
    l = np.arange(lmax + 1)
    c = np.zeros(2 * lmax + 1)
    for m in range(-lmax, lmax + 1):
        d = wigner_d(lmax, m, -s, 0.5 * math.pi)
        c[m + lmax] = np.sum(cl * (2 * l + 1) / 2.0 * d * d)
    return c


def wave_error(P: dict, m, beta) -> np.ndarray:
    """sigma_m^2(beta) of eq. s2m on the plan's doubled circle, written out: the wave e^{i m theta}
    sampled at Theta_k = k pi/L, k = 0..2L-1 (Theta_k - 2pi past the pole, theta = Theta theta_max/pi),
    weighted by w, its Fourier coefficients H_n = (2L)^-1 sum_k h_k e^{-i n Theta_k} kept for
    |n| <= L-1, summed back at Theta = beta pi/theta_max and compared with the wave there.
    Returns [len(m), len(beta)]."""
    m = np.atleast_1d(np.asarray(m, dtype=np.float64))
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    L, tmax = P["L"], P["theta_max"]
    k = np.arange(2 * L)
    Th_k = np.where(k > L, k - 2 * L, k) * (math.pi / L)
    ring = np.where(k > L, 2 * L - k, k)
    wr = np.zeros(L + 1)
    wr[: min(P["nring"], L + 1)] = P["w_j"][: L + 1]
    h = wr[ring][None, :] * np.exp(1j * np.outer(m, Th_k * tmax / math.pi))
    n = np.arange(-(L - 1), L)
    H = h @ np.exp(-1j * np.outer(Th_k, n)) / (2 * L)
    rec = H @ np.exp(1j * np.outer(n, beta * math.pi / tmax))
    return np.abs(rec - np.exp(1j * np.outer(m, beta))) ** 2


def predict_error(lmax: int, s: int, eps: float, theta_star: float, cl, beta, kappa: float = 1.0,
                  window_kind: str = "es") -> np.ndarray:
    """Relative rms error of the partial-sky route at angles beta from the pole (Sec. II.E eq. st):
    sqrt(sum_m c_m sigma_m^2(beta) / sum_m c_m), on the ring set of plan_params for a cap theta*."""
    P = plan_params(lmax, s, eps, np.array([0.0, theta_star]), kappa, window_kind)
    c = great_circle_spectrum(lmax, s, cl)
    ms = np.arange(-lmax, lmax + 1)
    sig = wave_error(P, ms, beta)
    return np.sqrt(c @ sig / c.sum())
