"""Full-size parity at the benchmark's workload and launch configuration (marked gpu).

Spin-2 synthesis and adjoint at lmax 4096 on the ~4% field (2.2e7 points, regular 0.5' grid +
2.5' deflections, patch-centred frame), in the FP32 form at eps = 1e-5 and the FP64 form at
eps = 1e-10.  The oracle cannot run the whole problem in seconds, so:
  * synthesis: a random sample of points, each summed directly (O1), <= 10 eps;
  * adjoint of f = A a: selected coefficients of low degree or close to the diagonal, each summed
    over all 2.2e7 points by the restricted direct adjoint, <= 10 eps relative to their norm;
  * the adjoint identity <f, A a> = <A^H f, a> for random f (holds at any size);
  * the ring coefficients of a sample of rings against the oracle's ring synthesis (stage parity).
"""
import numpy as np
import pytest

import _parity as PP
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    from paper_2603_17166_gb300 import synthetic

    return synthetic.config2(frame="R")


@pytest.fixture(scope="module", params=[("fp32", 1e-5), ("fp64", 1e-10)], ids=["fp32", "fp64"])
def planned(request, workload):
    from paper_2603_17166_gb300 import Plan

    prec, eps = request.param
    th = torch.from_numpy(workload["theta"]).cuda()
    ph = torch.from_numpy(workload["phi"]).cuda()
    plan = Plan(2, 4096, th, ph, eps, precision=prec)
    yield plan, eps
    plan.close()
    torch.cuda.empty_cache()


def test_workload_shape(workload):
    assert workload["theta"].size > 2.0e7
    assert 34.0 < np.degrees(workload["theta"].max()) < 35.5


def test_synthesis_sampled_points(planned, workload):
    plan, eps = planned
    g = torch.from_numpy(workload["g"]).cuda().to(plan.cdtype)
    c = torch.from_numpy(workload["c"]).cuda().to(plan.cdtype)
    f = plan.synthesis(g, c)
    rng = np.random.default_rng(11)
    sel = rng.choice(workload["theta"].size, size=160, replace=False)
    # add the extreme points (pole side and cap edge), the smallest and largest phi, and points whose
    # ES window starts on a grid tile's first or last row or column
    P = O.plan_params(4096, 2, eps, workload["theta"])
    prec = "fp32" if plan.precision == 32 else "fp64"
    sel = np.unique(np.concatenate([sel, PP.border_sample(P, workload["theta"], workload["phi"], prec=prec)]))
    ref = O.direct_synthesis(4096, 2, workload["g"], workload["c"], workload["theta"][sel], workload["phi"][sel])
    got = f[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.complex128)
    assert O.rel_l2(got, ref) <= 10 * eps
    PP.assert_pointwise(got, ref, eps)
    assert torch.isfinite(torch.view_as_real(f)).all()


def test_adjoint_selected_coefficients(planned, workload):
    plan, eps = planned
    g = torch.from_numpy(workload["g"]).cuda().to(plan.cdtype)
    c = torch.from_numpy(workload["c"]).cuda().to(plan.cdtype)
    f = plan.synthesis(g, c)
    gt, ct = plan.adjoint(f)
    sel = [(2, 0), (2, 2), (3, 1), (6, 5), (12, 0), (20, 17), (40, 40), (64, 60), (300, 297), (1200, 1198),
           (2200, 2199), (2500, 2496)]
    ls = np.array([a for a, _ in sel])
    ms = np.array([b for _, b in sel])
    fh = f.cpu().numpy().astype(np.complex128)
    g1, c1 = O.direct_adjoint_lm(2, workload["theta"], workload["phi"], fh, ls, ms)
    idx = torch.from_numpy(O.alm_index(4096, ls, ms)).cuda()
    g2 = gt[idx].cpu().numpy().astype(np.complex128)
    c2 = ct[idx].cpu().numpy().astype(np.complex128)
    assert O.rel_l2(np.concatenate([g2, c2]), np.concatenate([g1, c1])) <= 10 * eps


def test_adjoint_identity_full_size(planned, workload):
    plan, eps = planned
    rng = np.random.default_rng(12)
    n = workload["theta"].size
    fr = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(plan.np_cdtype)
    g = torch.from_numpy(workload["g"]).cuda().to(plan.cdtype)
    c = torch.from_numpy(workload["c"]).cuda().to(plan.cdtype)
    Aa = plan.synthesis(g, c).cpu().numpy().astype(np.complex128)
    gt, ct = plan.adjoint(torch.from_numpy(fr).cuda())
    lhs = O.map_dot(fr.astype(np.complex128), Aa)
    rhs = O.alm_dot(gt.cpu().numpy().astype(np.complex128), workload["g"], 4096) + \
        O.alm_dot(ct.cpu().numpy().astype(np.complex128), workload["c"], 4096)
    assert abs(lhs - rhs) <= (1e-11 if plan.precision == 64 else 1e-4) * abs(lhs)


def test_ring_coefficients_sampled_rings(planned, workload):
    plan, eps = planned
    g = torch.from_numpy(workload["g"]).cuda().to(plan.cdtype)
    c = torch.from_numpy(workload["c"]).cuda().to(plan.cdtype)
    F = plan.ring_coeffs(g, c).cpu().numpy().astype(np.complex128)
    th_j, _, _ = plan.rings()
    i = plan.info
    js = np.unique(np.linspace(0, i["nring"] - 1, 24).astype(int))
    Fo = O.ring_synthesis(4096, 2, i["M"], workload["g"], workload["c"], th_j[js])
    assert O.rel_l2(F[js], Fo) <= (1e-11 if plan.precision == 64 else 10 * eps)


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_patch_frame_full_size(prec, eps):
    """The same field's points as given (centre near dec -55 deg, theta* 48 deg about the south pole)
    through a patch-frame plan: theta* drops to the smallest cap's 34.7 deg; sampled points against
    the direct sum in the caller's frame, selected adjoint coefficients summed over all points, and
    the adjoint identity."""
    from paper_2603_17166_gb300 import Plan, synthetic

    wl = synthetic.config2(frame="S")
    th = torch.from_numpy(wl["theta"]).cuda()
    ph = torch.from_numpy(wl["phi"]).cuda()
    plan = Plan(2, 4096, th, ph, eps, precision=prec, patch_frame=True)
    assert 34.0 < np.degrees(plan.info["theta_star"]) < 35.0
    g = torch.from_numpy(wl["g"]).cuda().to(plan.cdtype)
    c = torch.from_numpy(wl["c"]).cuda().to(plan.cdtype)
    f = plan.synthesis(g, c)
    assert plan.status() == 0
    sel = np.random.default_rng(13).choice(wl["theta"].size, size=96, replace=False)
    ref = O.direct_synthesis(4096, 2, wl["g"], wl["c"], wl["theta"][sel], wl["phi"][sel])
    got = f[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.complex128)
    assert O.rel_l2(got, ref) <= 10 * eps
    gt, ct = plan.adjoint(f)
    ls = np.array([2, 3, 12, 40, 300, 1200])
    ms = np.array([0, 1, 0, 40, 297, 1198])
    g1, c1 = O.direct_adjoint_lm(2, wl["theta"], wl["phi"], f.cpu().numpy().astype(np.complex128), ls, ms)
    idx = torch.from_numpy(O.alm_index(4096, ls, ms)).cuda()
    got = np.concatenate([gt[idx].cpu().numpy(), ct[idx].cpu().numpy()]).astype(np.complex128)
    assert O.rel_l2(got, np.concatenate([g1, c1])) <= 10 * eps
    rng = np.random.default_rng(14)
    n = wl["theta"].size
    fr = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(plan.np_cdtype)
    Aa = f.cpu().numpy().astype(np.complex128)
    gt, ct = plan.adjoint(torch.from_numpy(fr).cuda())
    lhs = O.map_dot(fr.astype(np.complex128), Aa)
    rhs = O.alm_dot(gt.cpu().numpy().astype(np.complex128), wl["g"], 4096) + \
        O.alm_dot(ct.cpu().numpy().astype(np.complex128), wl["c"], 4096)
    assert abs(lhs - rhs) <= (1e-11 if prec == "fp64" else 1e-4) * abs(lhs)
    plan.close()
    torch.cuda.empty_cache()
