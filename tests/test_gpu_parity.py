"""CUDA path against the FP64 oracle through the C ABI (marked gpu).

Small cases that the oracle finishes in seconds but that span several tiles, several FFT
stages and ragged ring chunks: plan parameters, ring coefficients (stage parity), end-to-end
synthesis and adjoint against direct summation (<= 10 eps), against the oracle pipeline
(same plan, FP64 to 1e-11), the adjoint identity, and the edge cases."""
import math

import numpy as np
import pytest

import _parity as PP
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _alm(rng, lmax, s):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


def _cap(rng, n, radius, pole="N"):
    th = np.arccos(rng.uniform(math.cos(radius), 1.0, n))
    if pole == "S":
        th = math.pi - th
    return th, rng.uniform(-math.pi, 3 * math.pi, n)


def _cap_with_borders(rng, n, radius, pole, lmax, s, eps, prec):
    """Random cap points plus points on the tile borders, the phi wrap-around, the pole and the cap
    edge of the plan those points lead to (the added points leave every plan parameter as it is)."""
    th, ph = _cap(rng, n, radius, pole)
    P = O.plan_params(lmax, s, eps, th)
    tb, pb = PP.border_points(P, rng, prec)
    return np.concatenate([th, tb]), np.concatenate([ph, pb])


def _plan(s, lmax, th, ph, eps, prec):
    from paper_2603_17166_gb300 import Plan

    return Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec)


def _cu(a, plan):
    return None if a is None else torch.from_numpy(np.asarray(a)).cuda().to(plan.cdtype)


CASES = [
    # lmax, s, cap radius, pole, eps, precision
    (64, 0, math.radians(10), "S", 1e-10, "fp64"),
    (64, 2, math.radians(10), "S", 1e-10, "fp64"),
    (96, 2, 0.45, "N", 1e-7, "fp64"),
    (160, 1, 0.3, "S", 1e-8, "fp64"),
    (128, 3, 1.0, "N", 1e-10, "fp64"),
    (64, 0, math.radians(10), "S", 1e-5, "fp32"),
    (200, 2, 0.5, "N", 1e-5, "fp32"),
    (150, 1, 0.35, "S", 1e-6, "fp32"),
]


@pytest.mark.parametrize("lmax,s,radius,pole,eps,prec", CASES)
def test_plan_parameters_match_oracle(lmax, s, radius, pole, eps, prec):
    rng = np.random.default_rng(1)
    th, ph = _cap(rng, 3000, radius, pole)
    plan = _plan(s, lmax, th, ph, eps, prec)
    P = O.plan_params(lmax, s, eps, th)
    i = plan.info
    assert i["pole"] == (1 if P["pole"] == "N" else -1)
    assert i["full_sky"] == int(P["full"])
    for k in ("theta_star", "eps_apo", "theta_max", "dTheta"):
        assert i[k] == pytest.approx(P[k], rel=1e-14, abs=1e-15)
    for k in ("Lmax", "L", "nring", "M", "W", "nTheta", "nphi", "r_lo", "nrows"):
        assert i[k] == P[k], k
    tj, wj, mj = plan.rings()
    assert np.abs(tj - P["theta_j"]).max() < 1e-15
    assert np.abs(wj - P["w_j"]).max() < 1e-13
    assert np.array_equal(mj, P["Mj"])


@pytest.mark.parametrize("lmax,s,radius,pole,eps,prec", CASES)
def test_ring_coefficients_stage_parity(lmax, s, radius, pole, eps, prec):
    """F_j[m] of the recursion kernel against the oracle's ring synthesis at the same rings."""
    rng = np.random.default_rng(2)
    th, ph = _cap(rng, 500, radius, pole)
    g, c = _alm(rng, lmax, s), (_alm(rng, lmax, s) if s else None)
    plan = _plan(s, lmax, th, ph, eps, prec)
    P = O.plan_params(lmax, s, eps, th)
    F = plan.ring_coeffs(_cu(g, plan), _cu(c, plan)).cpu().numpy()
    Fo = O.ring_synthesis(lmax, s, P["M"], g, c, P["theta_j"])
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert O.rel_l2(F, Fo) < tol
    # per ring, where the ring has any power
    for j in range(0, P["nring"], max(1, P["nring"] // 7)):
        if np.linalg.norm(Fo[j]) > 1e-8 * np.linalg.norm(Fo):
            assert O.rel_l2(F[j], Fo[j]) < 50 * tol


@pytest.mark.parametrize("lmax,s,radius,pole,eps,prec", CASES)
def test_synthesis_against_direct_sum(lmax, s, radius, pole, eps, prec):
    rng = np.random.default_rng(3)
    th, ph = _cap_with_borders(rng, 4000, radius, pole, lmax, s, eps, prec)
    g, c = _alm(rng, lmax, s), (_alm(rng, lmax, s) if s else None)
    plan = _plan(s, lmax, th, ph, eps, prec)
    f = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy()
    assert plan.status() == 0
    ref = O.direct_synthesis(lmax, s, g, c, th, ph)
    assert O.rel_l2(f, ref) <= 10 * eps
    PP.assert_pointwise(f, ref, eps)
    PP.assert_pointwise(f[4000:], ref[4000:], eps, what="border point")
    if prec == "fp64":
        P = O.plan_params(lmax, s, eps, th)
        f2 = O.pipeline_synthesis(P, g, c, th, ph)
        assert O.rel_l2(f, f2) < 1e-11


@pytest.mark.parametrize("lmax,s,radius,pole,eps,prec", CASES)
def test_adjoint_against_direct_sum(lmax, s, radius, pole, eps, prec):
    rng = np.random.default_rng(4)
    th, ph = _cap_with_borders(rng, 4000, radius, pole, lmax, s, eps, prec)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, prec)
    f = O.direct_synthesis(lmax, s, g, c, th, ph)      # f = A a: the adjoint's accuracy target
    gt, ct = plan.adjoint(_cu(f, plan))
    assert plan.status() == 0
    gt, ct = gt.cpu().numpy(), ct.cpu().numpy()
    gt1, ct1 = O.direct_adjoint(lmax, s, th, ph, f)
    _, m = O.lm_of_index(lmax)
    wgt = np.tile(np.where(m == 0, 1.0, 2.0), 2)
    assert O.rel_l2(np.concatenate([gt, ct]), np.concatenate([gt1, ct1]), wgt) <= 10 * eps
    PP.assert_pointwise(np.concatenate([gt, ct]), np.concatenate([gt1, ct1]), eps, what="coefficient")
    # written zeros: Im at m = 0 and l < s
    l, m = O.lm_of_index(lmax)
    assert np.all(gt[m == 0].imag == 0) and np.all(ct[m == 0].imag == 0)
    assert np.all(gt[l < s] == 0)
    if prec == "fp64":
        P = O.plan_params(lmax, s, eps, th)
        gt2, ct2 = O.pipeline_adjoint(P, f, th, ph)
        assert O.rel_l2(np.concatenate([gt, ct]), np.concatenate([gt2, ct2]), wgt) < 1e-11


@pytest.mark.parametrize("lmax,s,radius,pole,eps,prec", CASES)
def test_adjoint_identity(lmax, s, radius, pole, eps, prec):
    """<f, A a> = <A^H f, a> for random a, f: every GPU stage is an exact transpose."""
    rng = np.random.default_rng(5)
    th, ph = _cap(rng, 3000, radius, pole)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    f = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    plan = _plan(s, lmax, th, ph, eps, prec)
    Aa = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy().astype(np.complex128)
    gt, ct = plan.adjoint(_cu(f, plan))
    lhs = O.map_dot(f, Aa)
    rhs = O.alm_dot(gt.cpu().numpy().astype(np.complex128), g, lmax) + \
        O.alm_dot(ct.cpu().numpy().astype(np.complex128), c, lmax)
    assert abs(lhs - rhs) <= (1e-12 if prec == "fp64" else 1e-5) * abs(lhs)


def test_full_sky_mode_and_pole_points():
    """A cap beyond the equator switches to full-sky mode; points exactly on the pole and on
    theta = pi are valid."""
    rng = np.random.default_rng(6)
    lmax, s, eps = 40, 2, 1e-10
    th, ph = _cap(rng, 1500, 2.5, "N")
    th[:3] = [0.0, math.pi, 1e-300]
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, "fp64")
    assert plan.info["full_sky"] == 1
    f = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy()
    assert O.rel_l2(f, O.direct_synthesis(lmax, s, g, c, th, ph)) <= 10 * eps


def test_tiny_inputs():
    from paper_2603_17166_gb300 import Plan

    rng = np.random.default_rng(7)
    lmax, s = 8, 0
    g = _alm(rng, lmax, s)
    # one point
    th, ph = np.array([0.3]), np.array([1.0])
    plan = _plan(s, lmax, th, ph, 1e-10, "fp64")
    f = plan.synthesis(_cu(g, plan)).cpu().numpy()
    assert O.rel_l2(f, O.direct_synthesis(lmax, s, g, None, th, ph)) < 1e-9
    # no points: synthesis writes nothing, adjoint writes zeros
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    p0 = Plan(s, lmax, e, e, 1e-10, precision="fp64")
    assert p0.synthesis(_cu(g, p0)).numel() == 0
    gt, ct = p0.adjoint(torch.empty(0, dtype=torch.complex128, device="cuda"))
    assert float(gt.abs().max()) == 0.0
    # lmax = spin = 0
    p1 = _plan(0, 0, th, ph, 1e-10, "fp64")
    g0 = np.array([2.0 + 0j])
    f = p1.synthesis(_cu(g0, p1)).cpu().numpy()
    ref = -2.0 / math.sqrt(4 * math.pi)
    assert abs(f[0] - ref) <= 10 * 1e-10 * abs(ref)


def test_invalid_arguments_are_rejected():
    from paper_2603_17166_gb300 import Plan, PshtError

    th = torch.tensor([0.1, 0.2], dtype=torch.float64, device="cuda")
    ph = torch.tensor([0.0, 1.0], dtype=torch.float64, device="cuda")
    for kw in (dict(spin=-1, lmax=8, eps=1e-8), dict(spin=3, lmax=2, eps=1e-8), dict(spin=0, lmax=8, eps=1e-20),
               dict(spin=0, lmax=8, eps=0.5)):
        with pytest.raises(PshtError):
            Plan(kw["spin"], kw["lmax"], th, ph, kw["eps"])
    bad = torch.tensor([0.1, float("nan")], dtype=torch.float64, device="cuda")
    with pytest.raises(PshtError):
        Plan(0, 8, bad, ph, 1e-8)
    bad = torch.tensor([0.1, 3.5], dtype=torch.float64, device="cuda")
    with pytest.raises(PshtError):
        Plan(0, 8, bad, ph, 1e-8)
    with pytest.raises(PshtError):
        Plan(0, 8, th, ph, 1e-9, precision="fp32")   # FP32 form needs eps >= 1e-6
    with pytest.raises(PshtError):
        Plan(0, 8, th, ph, 9.9e-7, precision="fp32")


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-5), ("fp64", 1e-9)])
def test_full_sky_both_poles_reflection(prec, eps):
    """Full-sky plan with points next to both poles: rings beyond the equator run reflected."""
    rng = np.random.default_rng(8)
    lmax, s = 48, 2
    th = np.concatenate([np.arccos(rng.uniform(0.98, 1.0, 600)), math.pi - np.arccos(rng.uniform(0.98, 1.0, 600)),
                         np.arccos(rng.uniform(-1, 1, 600))])
    ph = rng.uniform(0, 2 * math.pi, th.size)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, prec)
    assert plan.info["full_sky"] == 1
    f = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy().astype(np.complex128)
    ref = O.direct_synthesis(lmax, s, g, c, th, ph)
    assert O.rel_l2(f, ref) <= 10 * eps
    gt, ct = plan.adjoint(_cu(ref, plan))
    gt1, ct1 = O.direct_adjoint(lmax, s, th, ph, ref)
    _, m = O.lm_of_index(lmax)
    wgt = np.tile(np.where(m == 0, 1.0, 2.0), 2)
    got = np.concatenate([gt.cpu().numpy(), ct.cpu().numpy()]).astype(np.complex128)
    assert O.rel_l2(got, np.concatenate([gt1, ct1]), wgt) <= 10 * eps


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_forced_full_sky_matches_partial(prec, eps):
    """PSHT_FULL_SKY runs the full-sky route (theta_max = pi, w = 1, L = lmax rings + 1) on a small
    cap; both routes approximate the same f to within the tolerance."""
    rng = np.random.default_rng(41)
    lmax, s = 96, 2
    th, ph = _cap(rng, 2000, 0.4, "S")
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    from paper_2603_17166_gb300 import Plan

    pp = _plan(s, lmax, th, ph, eps, prec)
    pf = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec, full_sky=True)
    assert pp.info["full_sky"] == 0 and pf.info["full_sky"] == 1
    assert pf.info["nring"] == pf.info["L"] + 1 and pf.info["theta_max"] == pytest.approx(math.pi)
    ref = O.direct_synthesis(lmax, s, g, c, th, ph)
    fp = pp.synthesis(_cu(g, pp), _cu(c, pp)).cpu().numpy().astype(np.complex128)
    ff = pf.synthesis(_cu(g, pf), _cu(c, pf)).cpu().numpy().astype(np.complex128)
    assert O.rel_l2(fp, ref) <= 10 * eps
    assert O.rel_l2(ff, ref) <= 10 * eps
    gt, ct = pf.adjoint(_cu(ref, pf))
    g1, c1 = O.direct_adjoint(lmax, s, th, ph, ref)
    got = np.concatenate([gt.cpu().numpy(), ct.cpu().numpy()]).astype(np.complex128)
    assert O.alm_rel_l2(got[: g1.size], g1, lmax) <= 10 * eps


def test_block_adjoint_ring_chunks():
    """The FP64 adjoint runs one CTA per order over chunks of 1024 rings; a full-sky plan at
    lmax 1500 has 1501 rings (two chunks per ring part, the second adding to the first)."""
    rng = np.random.default_rng(42)
    lmax, s, eps = 1500, 1, 1e-8
    th, ph = _cap(rng, 3000, 2.0, "N")
    from paper_2603_17166_gb300 import Plan

    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision="fp64",
                full_sky=True)
    assert plan.info["nring"] > 1024
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    f = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy()
    gt, ct = plan.adjoint(_cu(f, plan))
    ls = np.array([1, 2, 7, 30, 200, 900, 1400, 1500])
    ms = np.array([0, 1, 5, 30, 3, 450, 1399, 1500])
    g1, c1 = O.direct_adjoint_lm(s, th, ph, f, ls, ms)
    idx = O.alm_index(lmax, ls, ms)
    got = np.concatenate([gt.cpu().numpy()[idx], ct.cpu().numpy()[idx]])
    assert O.rel_l2(got, np.concatenate([g1, c1])) <= 10 * eps
    lhs = O.map_dot(f, f)
    rhs = O.alm_dot(gt.cpu().numpy(), g, lmax) + O.alm_dot(ct.cpu().numpy(), c, lmax)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("prec,eps,s", [("fp32", 1e-5, 2), ("fp64", 1e-10, 2), ("fp32", 1e-5, 0)])
def test_host_buffer_entry_points_match_device_ones(prec, eps, s):
    """psht_plan_synthesis_host / _adjoint_host (host arrays in and out; the FP32 form runs the
    recursions in chunks of orders so that the copies overlap them) give the device entry points'
    results: synthesis bit for bit, the adjoint up to the scatter's atomic summation order."""
    rng = np.random.default_rng(43)
    lmax = 300
    th, ph = _cap(rng, 20000, 0.5, "N")
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, prec)
    cd = plan.np_cdtype
    gh = np.ascontiguousarray(g.astype(cd))
    ch = np.ascontiguousarray(c.astype(cd))
    for rep in range(2):
        fh = np.zeros(th.size, dtype=cd)
        plan.synthesis_host(gh, ch, fh)
        fd = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy()
        assert np.array_equal(fh, fd)
        gt_h = np.zeros(O.nalm(lmax), dtype=cd)
        ct_h = np.zeros(O.nalm(lmax), dtype=cd)
        plan.adjoint_host(fh, gt_h, ct_h)
        gt_d, ct_d = plan.adjoint(torch.from_numpy(fh).cuda())
        tol = 1e-12 if prec == "fp64" else 1e-5
        for a, b in ((gt_h, gt_d), (ct_h, ct_d)):
            b = b.cpu().numpy().astype(np.complex128)
            assert O.alm_rel_l2(a.astype(np.complex128), b, lmax) <= tol


@pytest.mark.parametrize("eps,cd", [(1e-10, np.complex128), (1e-5, np.complex64)])
def test_one_shot_calls_with_the_papers_argument_list(eps, cd):
    """psht_synthesis / psht_adjoint_synthesis take (g, c, spin, lmax, theta, phi, eps) as the
    problem is stated in Sec. I (eq. syn and the adjoint synthesis general); precision follows eps
    (FP32 form at eps >= 1e-5).  Against the direct sums, <= 10 eps."""
    from paper_2603_17166_gb300 import psht

    rng = np.random.default_rng(44)
    lmax, s = 80, 2
    th, ph = _cap_with_borders(rng, 3000, 0.4, "S", lmax, s, eps, "fp32" if eps >= 1e-5 else "fp64")
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    tt, pt = torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda()
    f = psht.synthesis(torch.from_numpy(g).cuda(), torch.from_numpy(c).cuda(), s, lmax, tt, pt, eps)
    assert f.dtype == (torch.complex128 if cd == np.complex128 else torch.complex64)
    ref = O.direct_synthesis(lmax, s, g, c, th, ph)
    got = f.cpu().numpy().astype(np.complex128)
    assert O.rel_l2(got, ref) <= 10 * eps
    PP.assert_pointwise(got, ref, eps)
    gt, ct = psht.adjoint_synthesis(torch.from_numpy(ref).cuda(), s, lmax, tt, pt, eps)
    g1, c1 = O.direct_adjoint(lmax, s, th, ph, ref)
    _, m = O.lm_of_index(lmax)
    wgt = np.tile(np.where(m == 0, 1.0, 2.0), 2)
    got = np.concatenate([gt.cpu().numpy(), ct.cpu().numpy()]).astype(np.complex128)
    assert O.rel_l2(got, np.concatenate([g1, c1]), wgt) <= 10 * eps


@pytest.mark.parametrize("lmax,s,prec,eps,pole", [(40, 1, "fp64", 1e-10, "N"), (48, 2, "fp64", 1e-9, "S"),
                                                   (40, 2, "fp32", 1e-5, "N"), (48, 0, "fp32", 1e-5, "S"),
                                                   (48, 3, "fp64", 1e-10, "N")])
def test_full_sky_mirror_pairs(lmax, s, prec, eps, pole):
    """Full-sky plans evaluate the rings at b and pi - b as pairs sharing their Wigner columns
    (d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b)).  lmax 40 has an equator ring (its own mirror),
    lmax 48 has none; odd spins check the signs.  Ring coefficients against the oracle's ring
    synthesis, synthesis and adjoint against the direct sums, and the adjoint identity."""
    from paper_2603_17166_gb300 import Plan

    rng = np.random.default_rng(lmax + 10 * s)
    th, ph = _cap(rng, 3000, 0.6, pole)
    g, c = _alm(rng, lmax, s), (_alm(rng, lmax, s) if s else None)
    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec,
                full_sky=True)
    i = plan.info
    assert i["full_sky"] == 1 and i["nring"] == i["L"] + 1
    tj, _, _ = plan.rings()
    F = plan.ring_coeffs(_cu(g, plan), _cu(c, plan)).cpu().numpy().astype(np.complex128)
    Fo = O.ring_synthesis(lmax, s, i["M"], g, c, tj)
    assert O.rel_l2(F, Fo) < (1e-12 if prec == "fp64" else 2e-5)
    # rings past the equator, each against the oracle alone
    for j in (i["nring"] - 1, i["nring"] - 2, i["nring"] // 2 + 1):
        assert O.rel_l2(F[j], Fo[j]) < (1e-11 if prec == "fp64" else 1e-4), j
    f = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy().astype(np.complex128)
    ref = O.direct_synthesis(lmax, s, g, c, th, ph)
    assert O.rel_l2(f, ref) <= 10 * eps
    gt, ct = plan.adjoint(_cu(ref, plan))
    g1, c1 = O.direct_adjoint(lmax, s, th, ph, ref)
    _, m = O.lm_of_index(lmax)
    wgt = np.tile(np.where(m == 0, 1.0, 2.0), 2)
    got = np.concatenate([gt.cpu().numpy(), ct.cpu().numpy()]).astype(np.complex128)
    assert O.rel_l2(got, np.concatenate([g1, c1]), wgt) <= 10 * eps
    fr = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    gr, cr = plan.adjoint(_cu(fr, plan))
    gg = _alm(rng, lmax, s)
    cc = _alm(rng, lmax, s)
    Aa = plan.synthesis(_cu(gg, plan), _cu(cc, plan)).cpu().numpy().astype(np.complex128)
    lhs = O.map_dot(fr, Aa)
    rhs = O.alm_dot(gr.cpu().numpy().astype(np.complex128), gg, lmax) + \
        O.alm_dot(cr.cpu().numpy().astype(np.complex128), cc, lmax)
    # rounding scales with the norms (Cauchy-Schwarz), not with |lhs|, which random inputs make
    # small by cancellation
    assert abs(lhs - rhs) <= (1e-14 if prec == "fp64" else 1e-6) * np.linalg.norm(fr) * np.linalg.norm(Aa)
