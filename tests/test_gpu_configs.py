"""Parity at the other workloads' full sizes (marked gpu), beyond the benchmark's own:

  * lmax 6000 on the ~1% deep field, 5e7 uniform random points: spin 2 in the patch-centred frame
    (FP32 at eps = 1e-5, FP64 at 1e-10) and spin 0 with the points as given (nearer pole, FP64);
  * lmax 16384 on the ~4% field, 1e8 uniform random points, spin 2, patch-centred frame: the eps
    sweep 1e-4 .. 1e-12, the FP32 form at eps >= 1e-5 and the plain FP64 form at every eps (phi FFT
    of ~40000 points on global buffers).

The oracle sums a random sample of points directly (O1), <= 10 eps; the adjoint identity holds at
any size.  The extreme points (nearest the pole, on the cap edge) are always in the sample."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sample(theta, k, seed):
    rng = np.random.default_rng(seed)
    sel = rng.choice(theta.size, size=k, replace=False)
    sel[:2] = [int(np.argmin(theta)), int(np.argmax(theta))]
    return sel


def _check_synthesis(wl, eps, prec, k, seed):
    from paper_2603_17166_gb300 import Plan

    th = torch.from_numpy(wl["theta"]).cuda()
    ph = torch.from_numpy(wl["phi"]).cuda()
    plan = Plan(wl["s"], wl["lmax"], th, ph, eps, precision=prec)
    g = torch.from_numpy(wl["g"]).cuda().to(plan.cdtype)
    c = None if wl["c"] is None else torch.from_numpy(wl["c"]).cuda().to(plan.cdtype)
    f = plan.synthesis(g, c)
    sel = _sample(wl["theta"], k, seed)
    ref = O.direct_synthesis(wl["lmax"], wl["s"], wl["g"], wl["c"], wl["theta"][sel], wl["phi"][sel])
    got = f[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.complex128)
    err = O.rel_l2(got, ref)
    assert plan.status() == 0
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
    sel = _sample(wl["theta"], 16, 51)
    ref = O.direct_synthesis(wl["lmax"], wl["s"], wl["g"], wl["c"], wl["theta"][sel], wl["phi"][sel])
    return wl, sel, ref


# the eps sweep of the lmax 16384 workload: FP32 form for eps >= 1e-5, plain FP64 for all
SWEEP = [("fp32", 1e-4), ("fp32", 1e-5), ("fp64", 1e-4), ("fp64", 1e-6), ("fp64", 1e-8), ("fp64", 1e-10),
         ("fp64", 1e-12)]


@pytest.mark.parametrize("prec,eps", SWEEP, ids=[f"{p}-{e:g}" for p, e in SWEEP])
def test_lmax16384_eps_sweep(wide_lmax16384, prec, eps):
    from paper_2603_17166_gb300 import Plan

    wl, sel, ref = wide_lmax16384
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
    plan.close()
    del f, g, c
    torch.cuda.empty_cache()
