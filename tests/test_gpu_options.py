"""Plan options (Kaiser-Bessel window, band-limit factor kappa) and the error predictor through the
C ABI (marked gpu): the planner's ring weights against the oracle's, synthesis against direct
summation, the GPU predictor against the oracle's predictor, and the predictor against the error a
lowered band limit actually produces."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cap(rng, n, radius):
    return np.arccos(rng.uniform(math.cos(radius), 1.0, n)), rng.uniform(0.0, 2.0 * math.pi, n)


def _alm(rng, lmax, s):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


@pytest.mark.parametrize("window,kappa,prec,eps", [("kb", 1.0, "fp64", 1e-10), ("kb", 1.0, "fp32", 1e-5),
                                                   ("es", 1.25, "fp64", 1e-10), ("kb", 1.5, "fp64", 1e-8)])
def test_options_plan_parity(window, kappa, prec, eps):
    from paper_2603_17166_gb300 import Plan

    rng = np.random.default_rng(61)
    lmax, s = 128, 2
    th, ph = _cap(rng, 2500, math.radians(25.0))
    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec,
                window=window, kappa=kappa)
    P = O.plan_params(lmax, s, eps, th, kappa=kappa, window_kind=window)
    i = plan.info
    assert (i["Lmax"], i["L"], i["nring"]) == (P["Lmax"], P["L"], P["nring"])
    _, w, _ = plan.rings()
    assert np.allclose(w, P["w_j"], rtol=0, atol=1e-12)
    g, c = _alm(rng, lmax, s), _alm(rng, lmax, s)
    f = plan.synthesis(torch.from_numpy(g).cuda().to(plan.cdtype),
                       torch.from_numpy(c).cuda().to(plan.cdtype)).cpu().numpy().astype(np.complex128)
    assert O.rel_l2(f, O.direct_synthesis(lmax, s, g, c, th, ph)) <= 10 * eps


@pytest.mark.parametrize("s,spectrum,window,kappa", [(0, "white", "es", 1.0), (2, "inv_l2", "kb", 0.9),
                                                     (1, "white", "es", 0.8)])
def test_predictor_matches_oracle(s, spectrum, window, kappa):
    from paper_2603_17166_gb300 import predict_error

    lmax, eps = 200, 1e-8
    ts = math.radians(30.0)
    l = np.arange(lmax + 1)
    cl = np.ones(lmax + 1) if spectrum == "white" else np.where(l >= 2, 1.0 / (l + 1.0) ** 2, 0.0)
    beta = np.linspace(0.1 * ts, ts, 12)
    got = predict_error(s, lmax, ts, eps, cl, beta, window=window, kappa=kappa)
    ref = O.predict_error(lmax, s, eps, ts, cl, beta, kappa=kappa, window_kind=window)
    # sigma_m^2 is the squared difference of two O(1) values, so at predicted errors ~1e-10 FP64
    # cancellation leaves ~1e-5 relative agreement between two summation orders
    assert np.allclose(got, ref, rtol=1e-3, atol=1e-14), (got, ref)


def test_predictor_bounds_lowered_band_limit():
    """kappa = 0.8 shrinks the ring set below what eps asks for: the measured rms error on white
    fields at the cap edge is far above eps and within a factor 2 of the prediction."""
    from paper_2603_17166_gb300 import Plan, predict_error

    rng = np.random.default_rng(62)
    lmax, s, eps, kappa = 160, 0, 1e-8, 0.8
    ts = math.radians(25.0)
    beta = np.array([0.7, 0.85, 1.0]) * ts
    nphi = 64
    th = np.repeat(beta, nphi)
    ph = np.tile(np.linspace(0.0, 2.0 * math.pi, nphi, endpoint=False), beta.size)
    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision="fp64",
                kappa=kappa)
    assert plan.info["theta_star"] == pytest.approx(ts, rel=1e-12)
    err2 = np.zeros(beta.size)
    var = np.zeros(beta.size)
    for _ in range(6):
        g = _alm(rng, lmax, s)
        ref = O.direct_synthesis(lmax, s, g, None, th, ph)
        got = plan.synthesis(torch.from_numpy(g).cuda()).cpu().numpy()
        err2 += (np.abs(got - ref) ** 2).reshape(beta.size, nphi).mean(axis=1)
        var += (np.abs(ref) ** 2).reshape(beta.size, nphi).mean(axis=1)
    measured = np.sqrt(err2 / var)
    pred = predict_error(s, lmax, ts, eps, np.ones(lmax + 1), beta, kappa=kappa)
    assert measured.max() > 100 * eps
    ratio = measured / pred
    assert np.all(ratio > 0.5) and np.all(ratio < 2.0), ratio


@pytest.mark.parametrize("s,deg,prec,eps", [(2, 25.0, "fp64", 1e-10), (0, 7.0, "fp64", 1e-8), (2, 20.0, "fp32", 1e-5)])
def test_cost_optimal_apodisation(s, deg, prec, eps):
    """PSHT_APO_COST: the planner's apodisation length and ring set equal the oracle's search, the
    recursion takes no more steps than with eq. Lmax2, and the result stays within 10 eps."""
    from paper_2603_17166_gb300 import Plan

    rng = np.random.default_rng(63)
    lmax = 256
    th, ph = _cap(rng, 2500, math.radians(deg))
    P = O.plan_params(lmax, s, eps, th, eps_apo_choice="cost")
    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec,
                apodisation="cost")
    ref_plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), eps, precision=prec)
    i = plan.info
    assert (i["Lmax"], i["L"], i["nring"], i["M"]) == (P["Lmax"], P["L"], P["nring"], P["M"])
    assert i["eps_apo"] == pytest.approx(P["eps_apo"], rel=1e-15)
    assert i["recursion_triples"] <= ref_plan.info["recursion_triples"]
    _, w, _ = plan.rings()
    assert np.allclose(w, P["w_j"], rtol=0, atol=1e-12)
    g = _alm(rng, lmax, s)
    f = plan.synthesis(torch.from_numpy(g).cuda().to(plan.cdtype)).cpu().numpy().astype(np.complex128)
    assert O.rel_l2(f, O.direct_synthesis(lmax, s, g, None, th, ph)) <= 10 * eps
