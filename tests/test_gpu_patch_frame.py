"""Plans in the patch-centred frame (PSHT_PATCH_FRAME) through the C ABI (marked gpu): the caller's
points and a_lm stay in their own frame (a box near the south pole, as given), the plan rotates them
so that the patch is centred on the north pole, and every result is checked in the caller's frame
against the oracle's direct sums: synthesis and adjoint (<= 10 eps), the adjoint identity, the
packed-gradient and host-buffer entry points, and the smaller theta* the frame buys."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _alm(rng, lmax, s):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


def _box(rng, n):
    """Uniform in area on RA -50..50 deg, dec -70..-42 deg (colatitude 132..160 deg)."""
    ra = np.radians(rng.uniform(-50.0, 50.0, n))
    dec = np.arcsin(rng.uniform(math.sin(math.radians(-70.0)), math.sin(math.radians(-42.0)), n))
    return math.pi / 2 - dec, np.mod(ra, 2 * math.pi)


def _plan(s, lmax, th, ph, eps, prec, patch=True):
    from paper_2603_17166_gb300 import Plan

    return Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec,
                patch_frame=patch)


def _cu(a, plan):
    return None if a is None else torch.from_numpy(np.asarray(a)).cuda().to(plan.cdtype)


CASES = [(96, 2, 1e-10, "fp64"), (128, 0, 1e-10, "fp64"), (80, 1, 1e-8, "fp64"), (96, 2, 1e-5, "fp32"),
         (700, 2, 1e-5, "fp32")]


@pytest.mark.parametrize("lmax,s,eps,prec", CASES)
def test_patch_frame_synthesis_and_adjoint(lmax, s, eps, prec):
    rng = np.random.default_rng(30 + s)
    npts = 2000 if lmax < 500 else 600
    th, ph = _box(rng, npts)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, prec)
    info = plan.info
    assert info["patch_frame"] == 1
    # the patch frame's theta* is the smallest enclosing cap, well below the 48 deg about the south pole
    sel = rng.choice(npts, 200, replace=False)
    _, _, rad = O.min_enclosing_cap(th[sel], ph[sel])
    assert rad - 1e-9 <= info["theta_star"] < math.radians(36.0) < math.pi - th.min()
    f = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy().astype(np.complex128)
    assert plan.status() == 0
    ref = O.direct_synthesis(lmax, s, g, c, th, ph)
    assert O.rel_l2(f, ref) <= 10 * eps
    gt, ct = plan.adjoint(_cu(ref, plan))
    gt, ct = gt.cpu().numpy().astype(np.complex128), ct.cpu().numpy().astype(np.complex128)
    if lmax <= 128:
        gt1, ct1 = O.direct_adjoint(lmax, s, th, ph, ref)
        _, m = O.lm_of_index(lmax)
        wgt = np.tile(np.where(m == 0, 1.0, 2.0), 2)
        assert O.rel_l2(np.concatenate([gt, ct]), np.concatenate([gt1, ct1]), wgt) <= 10 * eps
    else:  # selected coefficients of the direct adjoint
        ls = np.array([lmax, lmax, 500, 350, 2 + s, 699])
        ms = np.array([0, 600, 250, 1, 2, 3])
        g1, c1 = O.direct_adjoint_lm(s, th, ph, ref, ls, ms)
        idx = O.alm_index(lmax, ls, ms)
        scale = np.sqrt(O.alm_dot(gt, gt, lmax) / O.nalm(lmax))
        assert np.abs(gt[idx] - g1).max() <= 10 * eps * 10 * scale
        assert np.abs(ct[idx] - c1).max() <= 10 * eps * 10 * scale
    l, m = O.lm_of_index(lmax)
    assert np.all(gt[m == 0].imag == 0) and np.all(ct[m == 0].imag == 0)


@pytest.mark.parametrize("s,prec", [(2, "fp64"), (2, "fp32"), (0, "fp64")])
def test_patch_frame_adjoint_identity(s, prec):
    rng = np.random.default_rng(40)
    lmax = 90
    th, ph = _box(rng, 1500)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    f = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    plan = _plan(s, lmax, th, ph, 1e-10 if prec == "fp64" else 1e-5, prec)
    Aa = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy().astype(np.complex128)
    gt, ct = plan.adjoint(_cu(f, plan))
    lhs = O.map_dot(f, Aa)
    rhs = O.alm_dot(gt.cpu().numpy().astype(np.complex128), g, lmax) + \
        O.alm_dot(ct.cpu().numpy().astype(np.complex128), c, lmax)
    assert abs(lhs - rhs) <= (1e-12 if prec == "fp64" else 1e-5) * abs(lhs)


def test_patch_frame_packed_and_host_entry_points():
    rng = np.random.default_rng(41)
    lmax, s, eps = 100, 2, 1e-10
    th, ph = _box(rng, 1800)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, "fp64")
    _, m = O.lm_of_index(lmax)
    half = np.where(m == 0, 1.0, 0.5)
    f_packed = plan.synthesis(_cu(g, plan), _cu(c, plan), packed_grad=True).cpu().numpy()
    f_half = plan.synthesis(_cu(g * half, plan), _cu(c * half, plan)).cpu().numpy()
    assert O.rel_l2(f_packed, f_half) < 1e-13
    fin = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    gp, cp = plan.adjoint(_cu(fin, plan), packed_grad=True)
    gu, cu = plan.adjoint(_cu(fin, plan))
    dbl = np.where(m == 0, 1.0, 2.0)
    assert O.rel_l2(gp.cpu().numpy(), gu.cpu().numpy() * dbl) < 1e-13
    assert O.rel_l2(cp.cpu().numpy(), cu.cpu().numpy() * dbl) < 1e-13
    # host buffers
    fh = np.zeros(th.size, dtype=np.complex128)
    plan.synthesis_host(g, c, fh)
    assert O.rel_l2(fh, plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy()) < 1e-14
    gh = np.zeros(O.nalm(lmax), dtype=np.complex128)
    ch = np.zeros_like(gh)
    plan.adjoint_host(fin, gh, ch)
    assert O.rel_l2(gh, gu.cpu().numpy()) < 1e-14 and O.rel_l2(ch, cu.cpu().numpy()) < 1e-14


def test_patch_frame_matches_plain_plan():
    """The same points and a_lm through a plan about the nearer pole and a patch-frame plan."""
    rng = np.random.default_rng(42)
    lmax, s, eps = 128, 2, 1e-10
    th, ph = _box(rng, 3000)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    a = _plan(s, lmax, th, ph, eps, "fp64", patch=False)
    b = _plan(s, lmax, th, ph, eps, "fp64", patch=True)
    # theta* 48 -> ~35 deg; at this small band limit the apodisation margin and polar cutoff keep the
    # triple count ratio near 0.8 (0.62 at lmax 4096)
    assert b.info["theta_star"] < math.radians(36.0) < math.radians(47.0) < a.info["theta_star"]
    assert b.info["recursion_triples"] < 0.9 * a.info["recursion_triples"]
    fa = a.synthesis(_cu(g, a), _cu(c, a)).cpu().numpy()
    fb = b.synthesis(_cu(g, b), _cu(c, b)).cpu().numpy()
    assert O.rel_l2(fb, fa) <= 10 * eps


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_in_frame_entry_points(prec, eps):
    """a_lm already in the plan's frame: synthesis_inframe(D a) = synthesis(a) and
    D^-1 adjoint_inframe(f) = adjoint(f); a plan without the frame refuses them."""
    from paper_2603_17166_gb300 import PshtError, Rotator

    rng = np.random.default_rng(43)
    lmax, s = 110, 2
    th, ph = _box(rng, 1600)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    plan = _plan(s, lmax, th, ph, eps, prec)
    al, be, ga = plan.info["euler"]
    rot = Rotator(lmax, precision=prec)
    gr, cr = rot.apply(_cu(g, plan), _cu(c, plan), al, be, ga)
    f1 = plan.synthesis(gr, cr, in_frame=True).cpu().numpy()
    f0 = plan.synthesis(_cu(g, plan), _cu(c, plan)).cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert O.rel_l2(f1, f0) <= tol
    fin = _cu(rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size), plan)
    g1, c1 = plan.adjoint(fin, in_frame=True)
    g1, c1 = rot.apply(g1, c1, -ga, -be, -al)
    g0, c0 = plan.adjoint(fin)
    assert O.alm_rel_l2(g1.cpu().numpy(), g0.cpu().numpy(), lmax) <= tol
    assert O.alm_rel_l2(c1.cpu().numpy(), c0.cpu().numpy(), lmax) <= tol
    plain = _plan(s, lmax, th, ph, eps, prec, patch=False)
    with pytest.raises(PshtError):
        plain.synthesis(_cu(g, plain), in_frame=True)
