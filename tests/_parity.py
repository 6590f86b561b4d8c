"""Shared checks of the GPU parity tests: a per-point error bound beside the relative L2 error, and
points placed on the grid-tile borders, on the phi wrap-around, on the cap edge and on the pole.

The CUDA library bins points into tiles of TR x TQ fine-grid cells (32 x 16 in the FP32 form, 16 x 32
in the FP64 form) by the base cell of their ES window, r0 = ceil(t - W/2) and q0 = ceil(u - W/2),
where t = Theta nTheta / 2pi and
u = phi nphi / 2pi are the fine-grid coordinates (Sec. II step 3: Theta = pi beta / theta_max);
the tile row is (r0 - r_lo) div TR and the tile column (q0 + PADQ) div TQ.  A tile-seam, halo or
wrap-around mistake shows at the points whose base cell sits on a tile's first or last row or
column, and at phi next to 0 and 2 pi.  The grid geometry (nTheta, nphi, W, r_lo, theta_max) is
taken from the oracle's plan parameters, which the planner parity tests show equal the library's.
"""
import math

import numpy as np

PADQ = 8  # left halo of the library's grid rows
TILES = {"fp32": (32, 16), "fp64": (16, 32)}  # the library's tile shape (TR, TQ) per form


def assert_pointwise(got, ref, eps, C=30.0, what="point"):
    """max_i |got_i - ref_i| <= C eps rms(ref): no single value may be far off even when the
    relative L2 error over all of them is small.  Returns the observed ratio max / (eps rms)."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    rms = math.sqrt(float(np.mean(np.abs(ref) ** 2)))
    worst = float(np.abs(got - ref).max()) if ref.size else 0.0
    ratio = worst / (eps * rms) if rms > 0 else 0.0
    i = int(np.argmax(np.abs(got - ref))) if ref.size else -1
    assert worst <= C * eps * rms, f"{what} {i}: |error| = {worst:.3e} > {C} eps rms ({C * eps * rms:.3e})"
    return ratio


def _beta_of_t(P, t):
    return (2.0 * math.pi * np.asarray(t, dtype=np.float64) / P["nTheta"]) * (P["theta_max"] / math.pi)


def _theta_of_beta(P, beta):
    return beta if P["pole"] == "N" else math.pi - beta


def border_points(P, rng, prec="fp64", per_row=6):
    """Extra points (theta, phi) inside the plan's cap (beta <= theta*, so theta* and every plan
    parameter stay the same) that sit on tile borders and at the phi wrap-around:
      * t at the first and last base rows of every tile row (and just across them);
      * u at the first and last base columns of the first tiles, of the last tile and of a middle
        one (and just across them), and phi = 0, 2 pi (1 - 2^-52), -1e-14, 2 pi + 1e-14, 6 pi + 0.3;
      * the pole itself (beta = 0) and the cap edge (beta = theta*)."""
    TR, TQ = TILES[prec]
    W, r_lo, nphi = P["W"], P["r_lo"], P["nphi"]
    t_star = P["theta_star"] * P["nTheta"] / (2.0 * P["theta_max"])
    ts = []
    k = 0
    while True:
        first = r_lo + TR * k + 0.5 * W          # ceil(t - W/2) = r_lo + TR k exactly
        if first - 1.0 > t_star:
            break
        ts += [first, first - 0.999999, first + 1e-9, first - 1e-9, first + TR - 1.0]
        k += 1
    ts = [t for t in ts if 0.0 <= t <= t_star] + [0.0, t_star]
    us = []
    for kq in (0, 1, 2, (nphi + PADQ) // (2 * TQ), (nphi + PADQ) // TQ - 1, (nphi + PADQ) // TQ):
        first = TQ * kq - PADQ + 0.5 * W       # ceil(u - W/2) + PADQ = TQ kq exactly
        us += [first, first - 0.999999, first + 1e-9, first + TQ - 1.0]
    us = [u for u in us if 0.0 <= u < nphi]
    phis = [2.0 * math.pi * u / nphi for u in us]
    phis += [0.0, 2.0 * math.pi * (1.0 - 2.0 ** -52), -1e-14, 2.0 * math.pi + 1e-14, 6.0 * math.pi + 0.3]
    th, ph = [], []
    for t in ts:
        for p in rng.choice(phis, size=min(per_row, len(phis)), replace=False):
            th.append(float(_theta_of_beta(P, _beta_of_t(P, t))))
            ph.append(float(p))
    for p in phis:  # every phi on three rows: the pole side, the middle and the cap edge
        for t in (0.25, 0.5 * t_star, t_star):
            th.append(float(_theta_of_beta(P, _beta_of_t(P, t))))
            ph.append(float(p))
    th = np.clip(np.array(th), 0.0, math.pi)
    beta = th if P["pole"] == "N" else math.pi - th
    keep = beta <= P["theta_star"]
    return th[keep], np.array(ph)[keep]


def border_sample(P, theta, phi, k_each=8, prec="fp64"):
    """Indices of existing points next to tile borders and the phi wrap-around, for workloads too
    large to add points to: the k_each points with the smallest and the largest phi mod 2 pi, and
    those whose base row or column lies on a tile's first or last row or column with the window
    start closest to a cell boundary; plus the pole-side and cap-edge extremes."""
    TR, TQ = TILES[prec]
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    beta = theta if P["pole"] == "N" else math.pi - theta
    t = beta * (math.pi / P["theta_max"]) * (P["nTheta"] / (2.0 * math.pi))
    ph = phi - 2.0 * math.pi * np.floor(phi / (2.0 * math.pi))
    u = ph * (P["nphi"] / (2.0 * math.pi))
    W = P["W"]
    r0 = np.ceil(t - 0.5 * W)
    q0 = np.ceil(u - 0.5 * W)
    dr = (r0 - P["r_lo"]) % TR
    dq = (q0 + PADQ) % TQ
    frac_t = r0 - (t - 0.5 * W)   # in [0, 1): 0 when the window starts exactly on a cell
    frac_u = q0 - (u - 0.5 * W)
    sel = [int(np.argmin(beta)), int(np.argmax(beta))]
    k = min(k_each, ph.size - 1)
    if k > 0:
        sel += list(np.argpartition(ph, k)[:k]) + list(np.argpartition(ph, -k)[-k:])
    for mask, frac in ((dr == 0, frac_t), (dr == TR - 1, 1.0 - frac_t), (dq == 0, frac_u), (dq == TQ - 1, 1.0 - frac_u)):
        idx = np.flatnonzero(mask)
        if idx.size > k_each:
            idx = idx[np.argpartition(frac[idx], k_each)[:k_each]]
        sel += list(idx)
    return np.unique(np.array(sel, dtype=np.int64))
