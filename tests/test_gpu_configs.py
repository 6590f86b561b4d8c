"""Parity at the other workloads' full sizes (marked gpu), beyond the benchmark's own:

  * lmax 6000 on the ~1% deep field, 5e7 uniform random points: spin 2 in the patch-centred frame
    (FP32 at eps = 1e-5, FP64 at 1e-10) and spin 0 with the points as given (nearer pole, FP64);
  * lmax 16384 on the ~4% field, 1e8 uniform random points, spin 2, patch-centred frame: the eps
    sweep 1e-4 .. 1e-12, the FP32 form at eps >= 1e-5 and the plain FP64 form at every eps (phi FFT
    of ~40000 points on global buffers).

The oracle sums a sample of points directly (O1), <= 10 eps in relative L2 and <= 30 eps rms at
every sampled point; the sample holds random points, the extreme ones (nearest the pole, on the cap
edge), the points with the smallest and largest phi and points whose ES window starts on a grid
tile's first or last row or column.  At lmax 16384 the oracle's direct sum costs ~40 core-seconds
per point, so that sample is 16 random points plus about 14 such border points.  The adjoint is
checked at selected coefficients, each summed by the oracle over all points, and by the adjoint
identity, which holds at any size."""
import numpy as np
import pytest

import _parity as PP
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sample(theta, phi, k, seed, s, lmax, eps, k_each=8, prec="fp64"):
    rng = np.random.default_rng(seed)
    sel = rng.choice(theta.size, size=k, replace=False)
    P = O.plan_params(lmax, s, eps, theta)
    return np.unique(np.concatenate([sel, PP.border_sample(P, theta, phi, k_each, prec)]))


def _check_synthesis(wl, eps, prec, k, seed):
    from paper_2603_17166_gb300 import Plan

    th = torch.from_numpy(wl["theta"]).cuda()
    ph = torch.from_numpy(wl["phi"]).cuda()
    plan = Plan(wl["s"], wl["lmax"], th, ph, eps, precision=prec)
    g = torch.from_numpy(wl["g"]).cuda().to(plan.cdtype)
    c = None if wl["c"] is None else torch.from_numpy(wl["c"]).cuda().to(plan.cdtype)
    f = plan.synthesis(g, c)
    sel = _sample(wl["theta"], wl["phi"], k, seed, wl["s"], wl["lmax"], eps, prec=prec)
    ref = O.direct_synthesis(wl["lmax"], wl["s"], wl["g"], wl["c"], wl["theta"][sel], wl["phi"][sel])
    got = f[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.complex128)
    err = O.rel_l2(got, ref)
    assert plan.status() == 0
    PP.assert_pointwise(got, ref, eps)
    return plan, f, g, c, err


@pytest.fixture(scope="module")
def deep_field_spin2():
    from paper_2603_17166_gb300 import synthetic

    return synthetic.config3(s=2, frame="R")


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_lmax6000_spin2_deep_field(deep_field_spin2, prec, eps):
    wl = deep_field_spin2
    assert wl["theta"].size == 50_000_000
    plan, f, g, c, err = _check_synthesis(wl, eps, prec, 96, 31)
    assert err <= 10 * eps
    rng = np.random.default_rng(32)
    n = wl["theta"].size
    fr = torch.complex(torch.randn(n, dtype=torch.float64), torch.randn(n, dtype=torch.float64)).to(plan.cdtype)
    gt, ct = plan.adjoint(fr.cuda())
    lhs = O.map_dot(fr.numpy().astype(np.complex128), f.cpu().numpy().astype(np.complex128))
    rhs = O.alm_dot(gt.cpu().numpy().astype(np.complex128), wl["g"], wl["lmax"]) + \
        O.alm_dot(ct.cpu().numpy().astype(np.complex128), wl["c"], wl["lmax"])
    assert abs(lhs - rhs) <= (1e-11 if prec == "fp64" else 1e-4) * abs(lhs)
    plan.close()
    torch.cuda.empty_cache()


def test_lmax6000_spin0_as_given():
    from paper_2603_17166_gb300 import synthetic

    wl = synthetic.config3(s=0, frame="S")
    plan, f, g, c, err = _check_synthesis(wl, 1e-10, "fp64", 64, 33)
    assert plan.info["pole"] == -1  # the field lies in the south
    assert err <= 10 * 1e-10
    plan.close()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def wide_lmax16384():
    from paper_2603_17166_gb300 import synthetic

    wl = synthetic.config5(frame="R")
    sel = np.unique(np.concatenate([_sample(wl["theta"], wl["phi"], 16, 51, 2, 16384, 1e-10, k_each=2),
                                    _sample(wl["theta"], wl["phi"], 0, 52, 2, 16384, 1e-5, k_each=1, prec="fp32")]))
    ref = O.direct_synthesis(wl["lmax"], wl["s"], wl["g"], wl["c"], wl["theta"][sel], wl["phi"][sel])
    return wl, sel, ref


# the eps sweep of the lmax 16384 workload: FP32 form for eps >= 1e-5, plain FP64 for all 9 values
SWEEP = [("fp32", 1e-4), ("fp32", 1e-5)] + [("fp64", 10.0 ** -k) for k in range(4, 13)]

# adjoint coefficients summed directly over all 1e8 points (low degree: the oracle's cost per
# point grows with l - max(m, s))
ADJ_LM = [(2, 0), (2, 2), (3, 1), (12, 0), (40, 40), (64, 60)]


@pytest.fixture(scope="module")
def wide_lmax16384_adjoint_ref(wide_lmax16384):
    """f ~ A a from the FP64 form at eps = 1e-12 (the adjoint's accuracy target is f = A a), and the
    oracle's adjoint of that f at ADJ_LM summed over all points; shared by every eps of the sweep."""
    from paper_2603_17166_gb300 import Plan

    wl, _, _ = wide_lmax16384
    plan = Plan(2, 16384, torch.from_numpy(wl["theta"]).cuda(), torch.from_numpy(wl["phi"]).cuda(), 1e-12,
                precision="fp64")
    f = plan.synthesis(torch.from_numpy(wl["g"]).cuda(), torch.from_numpy(wl["c"]).cuda()).cpu().numpy()
    plan.close()
    torch.cuda.empty_cache()
    ls = np.array([a for a, _ in ADJ_LM])
    ms = np.array([b for _, b in ADJ_LM])
    g1, c1 = O.direct_adjoint_lm(2, wl["theta"], wl["phi"], f, ls, ms)
    return f, ls, ms, np.concatenate([g1, c1])


@pytest.mark.parametrize("prec,eps", SWEEP, ids=[f"{p}-{e:g}" for p, e in SWEEP])
def test_lmax16384_eps_sweep(wide_lmax16384, wide_lmax16384_adjoint_ref, prec, eps):
    from paper_2603_17166_gb300 import Plan

    wl, sel, ref = wide_lmax16384
    fa, ls, ms, adj_ref = wide_lmax16384_adjoint_ref
    assert wl["theta"].size == 100_000_000
    plan = Plan(2, 16384, torch.from_numpy(wl["theta"]).cuda(), torch.from_numpy(wl["phi"]).cuda(), eps,
                precision=prec)
    g = torch.from_numpy(wl["g"]).cuda().to(plan.cdtype)
    c = torch.from_numpy(wl["c"]).cuda().to(plan.cdtype)
    f = plan.synthesis(g, c)
    got = f[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.complex128)
    err = O.rel_l2(got, ref)
    print(f"lmax 16384 {prec} eps {eps:g}: rel L2 error {err:.3e} (W {plan.info['W']}, nphi {plan.info['nphi']})")
    assert plan.status() == 0
    assert err <= 10 * eps
    PP.assert_pointwise(got, ref, eps)
    # adjoint of f ~ A a at the selected coefficients, and the adjoint identity with the same a
    gt, ct = plan.adjoint(torch.from_numpy(fa).cuda().to(plan.cdtype))
    assert plan.status() == 0
    idx = torch.from_numpy(O.alm_index(16384, ls, ms)).cuda()
    got_a = np.concatenate([gt[idx].cpu().numpy(), ct[idx].cpu().numpy()]).astype(np.complex128)
    err_a = O.rel_l2(got_a, adj_ref)
    print(f"lmax 16384 {prec} eps {eps:g}: adjoint rel L2 error {err_a:.3e} at {len(ls)} (l, m)")
    assert err_a <= 10 * eps
    lhs = O.map_dot(fa, f.cpu().numpy().astype(np.complex128))
    rhs = O.alm_dot(gt.cpu().numpy().astype(np.complex128), wl["g"], 16384) + \
        O.alm_dot(ct.cpu().numpy().astype(np.complex128), wl["c"], 16384)
    assert abs(lhs - rhs) <= (1e-11 if prec == "fp64" else 1e-4) * abs(lhs)
    plan.close()
    del f, g, c, gt, ct
    torch.cuda.empty_cache()
