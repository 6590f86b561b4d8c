"""Batched execution on one plan (psht_plan_synthesis_batch / psht_plan_adjoint_batch, marked gpu).

Up to four a_lm sets (or maps) share one pass of the Wigner-d recursion.  Each set's result must
equal the single-set call on the same plan (the per-set arithmetic is the same; the adjoint's
spreading and the FP32 adjoint's accumulation use atomics, so those agree to rounding), and the
direct sums of the oracle (<= 10 eps), for batch sizes that exercise groups of 4, 2 and 1 sets,
with c present, absent, or absent for some sets only."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _alm(rng, lmax, s):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


def _plan(s, lmax, n, radius, eps, prec, seed, patch=False):
    from paper_2603_17166_gb300 import Plan

    rng = np.random.default_rng(seed)
    th = math.pi - np.arccos(rng.uniform(math.cos(radius), 1.0, n))
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec,
                patch_frame=patch)
    return rng, plan, th, ph


def _rel(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


CASES = [("fp32", 1e-5, 2, 7), ("fp64", 1e-10, 2, 5), ("fp32", 1e-5, 0, 3), ("fp64", 1e-8, 1, 2)]


@pytest.mark.parametrize("prec,eps,s,nsets", CASES)
def test_batch_synthesis_equals_single_calls(prec, eps, s, nsets):
    rng, plan, th, ph = _plan(s, 160, 6000, 0.45, eps, prec, 71 + nsets)
    gs = [_alm(rng, 160, s) for _ in range(nsets)]
    cs = [(_alm(rng, 160, s) if (s and k % 3 != 1) else None) for k in range(nsets)]
    cu = lambda a: None if a is None else torch.from_numpy(a).cuda().to(plan.cdtype)
    fb = plan.synthesis_batch([cu(g) for g in gs], [cu(c) for c in cs])
    assert plan.status() == 0
    tol = 1e-13 if prec == "fp64" else 1e-6
    for k in range(nsets):
        f1 = plan.synthesis(cu(gs[k]), cu(cs[k]))
        assert _rel(fb[k], f1) <= tol, k
    k = nsets - 1  # one set against the direct sum
    ref = O.direct_synthesis(160, s, gs[k], cs[k], th, ph)
    assert O.rel_l2(fb[k].cpu().numpy().astype(np.complex128), ref) <= 10 * eps


@pytest.mark.parametrize("prec,eps,s,nsets", CASES)
def test_batch_adjoint_equals_single_calls(prec, eps, s, nsets):
    rng, plan, th, ph = _plan(s, 160, 6000, 0.45, eps, prec, 81 + nsets)
    a = [_alm(rng, 160, s) for _ in range(nsets)]
    fs = [O.direct_synthesis(160, s, x, None, th, ph) for x in a]  # f = A a: the 10 eps target
    fb = plan.adjoint_batch([torch.from_numpy(f).cuda() for f in fs], want_c=bool(s))
    assert plan.status() == 0
    tol = 1e-12 if prec == "fp64" else 1e-5
    for k in range(nsets):
        g1, c1 = plan.adjoint(torch.from_numpy(fs[k]).cuda(), want_c=bool(s))
        assert _rel(fb[k][0], g1) <= tol, k
        if s:
            assert _rel(fb[k][1], c1) <= tol, k
    k = 0
    g_ref, c_ref = O.direct_adjoint(160, s, th, ph, fs[k])
    _, m = O.lm_of_index(160)
    w = np.where(m == 0, 1.0, 2.0)
    got = fb[k][0].cpu().numpy().astype(np.complex128)
    assert O.rel_l2(got, g_ref, w) <= 10 * eps
    # a second batch on the same plan: the accumulators were left at zero
    fb2 = plan.adjoint_batch([torch.from_numpy(f).cuda() for f in fs], want_c=bool(s))
    for k in range(nsets):
        assert _rel(fb2[k][0], fb[k][0]) <= tol, k


def test_batch_on_full_size_workload_equals_single_calls():
    """The benchmark's workload (lmax 4096, spin 2, 2.2e7 points, FP32 at eps 1e-5) in batches of
    three: the adjoint's orders spread over several items meet in the per-set accumulators."""
    from paper_2603_17166_gb300 import Plan, synthetic

    wl = synthetic.config2(frame="R")
    plan = Plan(2, 4096, torch.from_numpy(wl["theta"]).cuda(), torch.from_numpy(wl["phi"]).cuda(), 1e-5,
                precision="fp32")
    g = torch.from_numpy(wl["g"]).cuda().to(torch.complex64)
    c = torch.from_numpy(wl["c"]).cuda().to(torch.complex64)
    gs, cs = [g, 0.5 * g, c], [c, None, g]
    fb = plan.synthesis_batch(gs, cs)
    for k in range(3):
        assert _rel(fb[k], plan.synthesis(gs[k], cs[k])) <= 1e-6
    ab = plan.adjoint_batch(fb)
    for k in range(3):
        g1, c1 = plan.adjoint(fb[k])
        assert _rel(ab[k][0], g1) <= 1e-5 and _rel(ab[k][1], c1) <= 1e-5
    assert plan.status() == 0
    plan.close()
    torch.cuda.empty_cache()


def test_batch_patch_frame_and_invalid_arguments():
    from paper_2603_17166_gb300 import PshtError

    rng, plan, th, ph = _plan(2, 64, 2000, 0.3, 1e-10, "fp64", 91, patch=True)
    gs = [torch.from_numpy(_alm(rng, 64, 2)).cuda() for _ in range(3)]
    fb = plan.synthesis_batch(gs)
    for k in range(3):
        assert _rel(fb[k], plan.synthesis(gs[k])) <= 1e-13
    with pytest.raises(PshtError):
        plan.synthesis_batch([])
    with pytest.raises(PshtError):
        plan.synthesis_batch([gs[0]] * 65)
