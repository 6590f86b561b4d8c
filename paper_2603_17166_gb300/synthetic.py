"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only input generation (random numbers, sky-patch geometry); none of the
transform's arithmetic.  The tests and the benchmark feed the same arrays to the CUDA library
and to the CPU oracle.

Stand-ins (the paper's footprint masks and LCDM spectra are not available here):
  * spectra: Gaussian a_lm, Re and Im i.i.d. with variance C_l, C_l = 1 ("white") or
    C_l = (l+1)^-2 for l >= 2 ("inv_l2"), m = 0 real, l < s zero;
  * the ~4% field: RA -50..+50 deg, dec -70..-42 deg (1550 deg^2), a regular 0.5' grid displaced
    by Gaussian deflections of 2.5' rms (SPT-3G main-field stand-in, Sec. II.F Table 1, Fig. 1);
  * the ~1% deep field: RA -30..+30 deg, dec -63.75..-51.25 deg (402 deg^2), uniform random points;
  * small caps: points uniform in area inside a cap around a pole.
Frames: "S" keeps the coordinates as given (the nearer pole is used by the transform);
"R" rotates the points so that the centre of the smallest enclosing cap is the north pole, the
paper's set-up (Sec. II step 1).  Isotropic a_lm are statistically identical in either frame.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20260317
_KIND = {"alm": 0, "points": 1, "deflections": 2, "stream": 3}


def seed(config: int, kind: str, offset: int = 0) -> int:
    return SEED_BASE + 100 * config + _KIND[kind] + 1000 * offset


def rng(config: int, kind: str, offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed(config, kind, offset)))


def nalm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def gaussian_alm(lmax: int, s: int, gen: np.random.Generator, spectrum: str = "white") -> np.ndarray:
    """Packed m-major complex128 a_lm; Re, Im ~ N(0, C_l) i.i.d. (m = 0 real), zero for l < max(s, lmin)."""
    n = nalm(lmax)
    a = gen.standard_normal(n) + 1j * gen.standard_normal(n)
    ls = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    m0 = np.zeros(n, dtype=bool)
    m0[: lmax + 1] = True
    if spectrum == "white":
        amp = np.ones(n)
    elif spectrum == "inv_l2":
        amp = 1.0 / (ls + 1.0)
        amp[ls < 2] = 0.0
    else:
        raise ValueError(spectrum)
    a *= amp
    a[m0] = a[m0].real
    a[ls < s] = 0.0
    return a


def cap_points(n: int, radius_deg: float, gen: np.random.Generator, pole: str = "S"):
    """Points uniform in area in a cap of the given radius around a pole."""
    cr = math.cos(math.radians(radius_deg))
    z = gen.uniform(cr, 1.0, n)
    phi = gen.uniform(0.0, 2.0 * math.pi, n)
    theta = np.arccos(z)
    if pole == "S":
        theta = math.pi - theta
    return theta, phi


def _radec_to_vec(ra_deg, dec_deg):
    ra = np.radians(ra_deg)
    dec = np.radians(dec_deg)
    cd = np.cos(dec)
    return np.stack([cd * np.cos(ra), cd * np.sin(ra), np.sin(dec)], axis=-1)


def _vec_to_thetaphi(v):
    z = np.clip(v[..., 2], -1.0, 1.0)
    theta = np.arccos(z)
    phi = np.mod(np.arctan2(v[..., 1], v[..., 0]), 2.0 * math.pi)
    return theta, phi


def box_points_random(n: int, ra_range, dec_range, gen: np.random.Generator):
    """Points uniform in area in an RA/dec box: RA uniform, sin(dec) uniform."""
    ra = gen.uniform(ra_range[0], ra_range[1], n)
    s0, s1 = math.sin(math.radians(dec_range[0])), math.sin(math.radians(dec_range[1]))
    dec = np.degrees(np.arcsin(gen.uniform(s0, s1, n)))
    return _radec_to_vec(ra, dec)


def box_points_grid(ra_range, dec_range, step_arcmin: float):
    """Regular grid: dec rows every step; per row round(width cos(dec)/step) equispaced RA values."""
    step = step_arcmin / 60.0
    decs = np.arange(dec_range[0] + 0.5 * step, dec_range[1], step)
    width = ra_range[1] - ra_range[0]
    out = []
    for d in decs:
        k = max(1, int(round(width * math.cos(math.radians(d)) / step)))
        ra = ra_range[0] + (np.arange(k) + 0.5) * (width / k)
        out.append(_radec_to_vec(ra, np.full(k, d)))
    return np.concatenate(out, axis=0)


def deflect(v, rms_arcmin: float, gen: np.random.Generator):
    """Geodesic displacement of unit vectors by a Gaussian 2-D deflection of the given rms
    (rms/sqrt(2) per component along e_theta, e_phi)."""
    sig = math.radians(rms_arcmin / 60.0) / math.sqrt(2.0)
    n = v.shape[0]
    dth = gen.standard_normal(n) * sig
    dph = gen.standard_normal(n) * sig
    theta, phi = _vec_to_thetaphi(v)
    ct, st, cp, sp = np.cos(theta), np.sin(theta), np.cos(phi), np.sin(phi)
    e_th = np.stack([ct * cp, ct * sp, -st], axis=-1)
    e_ph = np.stack([-sp, cp, np.zeros_like(cp)], axis=-1)
    amp = np.hypot(dth, dph)
    safe = np.where(amp > 0, amp, 1.0)
    d = (dth / safe)[:, None] * e_th + (dph / safe)[:, None] * e_ph
    return np.cos(amp)[:, None] * v + np.sin(amp)[:, None] * d


def enclosing_centre(v):
    """Approximate centre of the smallest cap containing unit vectors v: start at the mean
    direction and refine by a few rounds of a local search on the max angular distance."""
    c = v.mean(axis=0)
    c /= np.linalg.norm(c)
    sub = v[:: max(1, v.shape[0] // 200000)]

    def radius(cc):
        return float(np.arccos(np.clip(sub @ cc, -1, 1)).max())

    best = radius(c)
    step = 0.05
    while step > 1e-6:
        improved = False
        a = np.cross(c, [0.0, 0.0, 1.0]) if abs(c[2]) < 0.9 else np.cross(c, [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(c, a)
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)):
            cc = c + step * (dx * a + dy * b)
            cc /= np.linalg.norm(cc)
            r = radius(cc)
            if r < best:
                best, c, improved = r, cc, True
        if not improved:
            step *= 0.5
    return c


def rotate_to_north(v, centre):
    """Rotation taking `centre` to the north pole (Rodrigues), applied to v."""
    z = np.array([0.0, 0.0, 1.0])
    axis = np.cross(centre, z)
    sa = np.linalg.norm(axis)
    ca = float(centre @ z)
    if sa < 1e-15:
        return v if ca > 0 else v * np.array([1.0, -1.0, -1.0])
    k = axis / sa
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + sa * K + (1 - ca) * (K @ K)
    return v @ R.T


FIELD_4PCT = dict(ra=(-50.0, 50.0), dec=(-70.0, -42.0))
FIELD_1PCT = dict(ra=(-30.0, 30.0), dec=(-63.75, -51.25))


def field_points(kind: str, frame: str, gen_points: np.random.Generator, gen_defl=None, n: int | None = None,
                 step_arcmin: float = 0.5, defl_arcmin: float = 2.5):
    """(theta, phi) of a synthetic field: kind 'grid4' (regular grid + deflections on the ~4%
    field), 'random4' or 'random1' (uniform random points on the ~4% / ~1% field)."""
    if kind == "grid4":
        v = box_points_grid(FIELD_4PCT["ra"], FIELD_4PCT["dec"], step_arcmin)
        if defl_arcmin > 0:
            v = deflect(v, defl_arcmin, gen_defl if gen_defl is not None else gen_points)
    elif kind == "random4":
        v = box_points_random(n, FIELD_4PCT["ra"], FIELD_4PCT["dec"], gen_points)
    elif kind == "random1":
        v = box_points_random(n, FIELD_1PCT["ra"], FIELD_1PCT["dec"], gen_points)
    else:
        raise ValueError(kind)
    if frame == "R":
        v = rotate_to_north(v, enclosing_centre(v))
    elif frame != "S":
        raise ValueError(frame)
    return _vec_to_thetaphi(v)


def config1(n: int = 10000):
    """Spin 0, lmax 64, unit-variance a_lm, 10^4 points uniform in a 10 deg south cap."""
    g = gaussian_alm(64, 0, rng(1, "alm"), "white")
    theta, phi = cap_points(n, 10.0, rng(1, "points"), "S")
    return dict(lmax=64, s=0, g=g, c=None, theta=theta, phi=phi)


def config2(frame: str = "R", step_arcmin: float = 0.5, realisation: int = 0):
    """Spin 2 (g = E, c = B), lmax 4096, C_l ~ (l+1)^-2, regular 0.5' grid + 2.5' deflections on the ~4% field."""
    lmax = 4096
    g = gaussian_alm(lmax, 2, rng(2, "alm", 2 * realisation), "inv_l2")
    c = gaussian_alm(lmax, 2, rng(2, "alm", 2 * realisation + 1), "inv_l2")
    theta, phi = field_points("grid4", frame, rng(2, "points"), rng(2, "deflections"), step_arcmin=step_arcmin)
    return dict(lmax=lmax, s=2, g=g, c=c, theta=theta, phi=phi)


def config3(s: int = 2, frame: str = "R", n: int = 50_000_000, realisation: int = 0):
    """Spin 0 or 2, lmax 6000, C_l ~ (l+1)^-2, 5e7 uniform random points on the ~1% field."""
    lmax = 6000
    g = gaussian_alm(lmax, s, rng(3, "alm", 2 * realisation), "inv_l2")
    c = gaussian_alm(lmax, s, rng(3, "alm", 2 * realisation + 1), "inv_l2") if s else None
    theta, phi = field_points("random1", frame, rng(3, "points"), n=n)
    return dict(lmax=lmax, s=s, g=g, c=c, theta=theta, phi=phi)


def config5(frame: str = "R", n: int = 100_000_000, realisation: int = 0):
    """Spin 2 (g = E, c = B), lmax 16384, C_l ~ (l+1)^-2, 1e8 uniform random points on the ~4% field."""
    lmax = 16384
    g = gaussian_alm(lmax, 2, rng(5, "alm", 2 * realisation), "inv_l2")
    c = gaussian_alm(lmax, 2, rng(5, "alm", 2 * realisation + 1), "inv_l2")
    theta, phi = field_points("random4", frame, rng(5, "points"), n=n)
    return dict(lmax=lmax, s=2, g=g, c=c, theta=theta, phi=phi)


def small_cap(radius_deg: float = 7.0, lmax: int = 4000, s: int = 2, area_deg2: float = 57.0,
              res_arcmin: float = 0.86, config: int = 6):
    """A small deep field: area / resolution^2 points uniform in a cap of the given radius around
    the north pole (the EDFS row of the paper's Table 1: theta* = 7 deg, 57 deg^2 at 0.86', lmax
    4000, spin 2; its footprint is not available), C_l ~ (l+1)^-2."""
    n = int(round(area_deg2 * 3600.0 / (res_arcmin * res_arcmin)))
    g = gaussian_alm(lmax, s, rng(config, "alm", 0), "inv_l2")
    c = gaussian_alm(lmax, s, rng(config, "alm", 1), "inv_l2") if s else None
    theta, phi = cap_points(n, radius_deg, rng(config, "points"), "N")
    return dict(lmax=lmax, s=s, g=g, c=c, theta=theta, phi=phi)


def _rotate_from_north(v, centre):
    """Rotation taking the north pole to `centre`, applied to v (inverse of rotate_to_north)."""
    z = np.array([0.0, 0.0, 1.0])
    axis = np.cross(z, centre)
    sa = np.linalg.norm(axis)
    ca = float(centre @ z)
    if sa < 1e-15:
        return v if ca > 0 else v * np.array([1.0, -1.0, -1.0])
    k = axis / sa
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + sa * K + (1 - ca) * (K @ K)
    return v @ R.T


def patch_points(n: int, shape: str, dec_centre: float, fsky: float, gen: np.random.Generator):
    """(theta, phi) of n points uniform in area in a patch of sky fraction fsky centred at
    (RA 0, dec_centre): a cap, or an RA/dec box twice as wide (in RA degrees) as it is high."""
    if shape == "cap":
        r = math.degrees(math.acos(1.0 - 2.0 * fsky))
        th, ph = cap_points(n, r, gen, "N")
        st = np.sin(th)
        v = np.stack([st * np.cos(ph), st * np.sin(ph), np.cos(th)], axis=-1)
        return _vec_to_thetaphi(_rotate_from_north(v, _radec_to_vec(0.0, dec_centre)))
    area = 4.0 * math.pi * fsky  # steradians = width_rad * (sin d1 - sin d0)
    h = 1.0  # half height in degrees, grown until the box holds the area at twice its height in RA
    for _ in range(60):
        d0, d1 = max(-89.9, dec_centre - h), min(89.9, dec_centre + h)
        w = area / (math.sin(math.radians(d1)) - math.sin(math.radians(d0)))
        if math.degrees(w) <= 2.0 * (d1 - d0) or h > 40:
            break
        h *= 1.1
    w = min(math.degrees(w), 360.0)
    v = box_points_random(n, (-0.5 * w, 0.5 * w), (d0, d1), gen)
    return _vec_to_thetaphi(v)


SERVING_LMAX = (1024, 2048, 4096, 8192)
SERVING_EPS = (1e-5, 1e-8, 1e-10)


def serving_workload(n_fields: int = 8, n_requests: int = 200, nmax: int = 30_000_000, lmax_max: int = 8192):
    """Mixed request stream: a pool of fields (patch, points, lmax, spin, eps) and a request
    sequence over it.  Per field: lmax from {1024, 2048, 4096, 8192} (capped at lmax_max; field i
    takes the (i mod 4)-th value, so that a pool of 4 or more fields holds every lmax), spin 0 or
    2, cap (centre dec U[-90, -30]) or RA/dec box 50/50, sky fraction log-uniform on [0.1 %, 4 %],
    N log-uniform on [1e5, nmax], eps from {1e-5 (FP32 form), 1e-8, 1e-10} (field i takes the
    (i mod 3)-th, so that every form is in a pool of 3 or more fields).  Requests: field
    uniform over the pool, synthesis or adjoint 50/50, unit-rate Poisson arrival times (scale them
    by 1/lambda).  a_lm and point data are drawn per field."""
    gq = rng(4, "stream", 1)  # field parameters
    gp = rng(4, "points")
    ga = rng(4, "alm")
    gs = rng(4, "stream")
    fields = []
    lms = [l for l in SERVING_LMAX if l <= lmax_max] or [lmax_max]
    for i in range(n_fields):
        lmax = int(lms[i % len(lms)])
        s = int(gq.choice([0, 2]))
        shape = "cap" if gq.uniform() < 0.5 else "box"
        dec_c = float(gq.uniform(-90.0, -30.0))
        fsky = float(math.exp(gq.uniform(math.log(1e-3), math.log(4e-2))))
        n = int(math.exp(gq.uniform(math.log(1e5), math.log(nmax))))
        eps = float(SERVING_EPS[i % len(SERVING_EPS)])
        th, ph = patch_points(n, shape, dec_c, fsky, gp)
        g = gaussian_alm(lmax, s, ga, "inv_l2")
        c = gaussian_alm(lmax, s, ga, "inv_l2") if s else None
        f = ga.standard_normal(n) + 1j * ga.standard_normal(n)
        fields.append(dict(key=i + 1, lmax=lmax, s=s, shape=shape, dec_centre=dec_c, fsky=fsky, npts=n, eps=eps,
                           theta=th, phi=ph, g=g, c=c, f=f))
    which = gs.integers(0, n_fields, n_requests)
    ops = gs.integers(0, 2, n_requests)
    arrivals = np.cumsum(gs.exponential(1.0, n_requests))
    requests = [dict(field=int(w), op=int(o), t=float(t)) for w, o, t in zip(which, ops, arrivals)]
    return fields, requests
